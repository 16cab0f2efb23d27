"""Pins of the oracle's reverse-mode gradient against central finite differences (CPU only).

The misfit of a short ripening run (no flow, periodic) is differentiated with
respect to theta = (D_0, D_1, M_phi) and phi_0. Central differences of the
FP64 oracle with h = 1e-6 fix the answer independently of autograd. The
gradient also vanishes exactly at the parameters that made the target.
"""
import pytest
import torch

from oracle import adjoint
from workloads import configs


def _problem(steps=6):
    p, fields = configs.adjoint_problem(shape=(8, 9, 10), theta=configs.THETA_EVAL)
    phi0, cA0, cB0 = fields()
    target = adjoint.target_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps)
    return p, phi0, cA0, cB0, target, steps


def test_theta_gradient_matches_central_differences():
    p, phi0, cA0, cB0, target, steps = _problem()
    theta = configs.THETA_EVAL
    L, g_theta, _ = adjoint.misfit_gradient(p, theta, phi0, cA0, cB0, steps, target)
    assert L > 0
    h = 1e-6
    for i in range(3):
        tp = list(theta)
        tm = list(theta)
        tp[i] += h
        tm[i] -= h
        fd = (adjoint.forward_misfit(p, tp, phi0, cA0, cB0, steps, target)
              - adjoint.forward_misfit(p, tm, phi0, cA0, cB0, steps, target)) / (2 * h)
        assert abs(float(g_theta[i]) - fd) <= 1e-6 * abs(fd) + 1e-12, (i, float(g_theta[i]), fd)


def test_phi0_gradient_matches_directional_difference():
    p, phi0, cA0, cB0, target, steps = _problem()
    theta = configs.THETA_EVAL
    _, _, g_phi = adjoint.misfit_gradient(p, theta, phi0, cA0, cB0, steps, target)
    v = torch.randn(phi0.shape, generator=torch.Generator().manual_seed(3), dtype=torch.float64)
    v = v * (phi0 > 0.05) * (phi0 < 0.95)                # stay clear of the phi = 1/2 threshold of Eq. 66
    h = 1e-6
    fd = (adjoint.forward_misfit(p, theta, phi0 + h * v, cA0, cB0, steps, target)
          - adjoint.forward_misfit(p, theta, phi0 - h * v, cA0, cB0, steps, target)) / (2 * h)
    got = float((g_phi * v).sum())
    assert abs(got - fd) <= 1e-6 * abs(fd) + 1e-12


def test_gradient_vanishes_at_the_target_parameters():
    p, phi0, cA0, cB0, target, steps = _problem()
    L, g_theta, g_phi = adjoint.misfit_gradient(p, configs.THETA_TARGET, phi0, cA0, cB0, steps, target)
    assert L == 0.0
    assert float(g_theta.abs().max()) == 0.0
    assert float(g_phi.abs().max()) == 0.0
