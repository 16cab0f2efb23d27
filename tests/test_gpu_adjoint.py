"""Hand-written adjoint of the coupled step (no flow) against the FP64 oracle's reverse mode
and against central finite differences of the CUDA forward.

* FP64 storage: gradient w.r.t. theta = (D_0, D_1, M_phi) and phi_0 within 1e-9 of the
  oracle's autograd gradient (ragged checkpoint segments included).
* FP32 storage: within 1e-4 of the oracle (FP32 rounding of a 40-step run).
* The 128^3, 2000-step workload with checkpoints every 100 steps: dL/dtheta against
  central differences of the FP32 forward with h = 1e-3 (bar 2e-2 relative: truncation
  O(h^2) plus FP32 noise of the misfit), and a directional derivative in phi_0.
* At the parameters that generated the target the misfit and its gradient are exactly 0.
"""
import pytest
import torch

from oracle import adjoint as oracle_adjoint
from workloads import configs

pytestmark = pytest.mark.gpu


def _problem(shape, storage, steps):
    p, fields = configs.adjoint_problem(shape=shape, storage=storage)
    phi0, cA0, cB0 = fields()
    return p, phi0, cA0, cB0


def _gpu_grad(p, phi0, cA0, cB0, steps, target, K, theta=configs.THETA_EVAL):
    from paper_2409_03401_gb300.adjoint import misfit_and_gradient
    dev = "cuda"
    tgt = [t.to(dev) for t in target]
    return misfit_and_gradient(p, theta, phi0.to(dev), cA0.to(dev), cB0.to(dev), steps, tgt, K=K)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_adjoint_matches_oracle_reverse_mode(storage, tol):
    steps, K = 20, 7                                   # segments of 7, 7, 6 steps
    p, phi0, cA0, cB0 = _problem((24, 24, 24), storage, steps)
    target = oracle_adjoint.target_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps)
    L_ref, gth_ref, gphi_ref = oracle_adjoint.misfit_gradient(p, configs.THETA_EVAL, phi0, cA0, cB0, steps, target)
    L, gth, gphi = _gpu_grad(p, phi0, cA0, cB0, steps, (target["phi"], target["muA"], target["muB"]), K)
    assert abs(L - L_ref) <= tol * abs(L_ref)
    rel = (gth - gth_ref).abs().max() / gth_ref.abs().max()
    assert float(rel) <= tol, (gth, gth_ref)
    gphi = gphi.double().cpu()
    assert float((gphi - gphi_ref).abs().max() / gphi_ref.abs().max()) <= 10 * tol


def test_adjoint_d3q19_scalar_lattice():
    # the same reverse mode on the paper's D3Q19 lattice for phi, c^A, c^B (FP64 storage)
    steps, K = 12, 5
    p, phi0, cA0, cB0 = _problem((16, 16, 16), "f64", steps)
    p = p.with_(lattice="D3Q19")
    target = oracle_adjoint.target_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps)
    L_ref, gth_ref, gphi_ref = oracle_adjoint.misfit_gradient(p, configs.THETA_EVAL, phi0, cA0, cB0, steps, target)
    L, gth, gphi = _gpu_grad(p, phi0, cA0, cB0, steps, (target["phi"], target["muA"], target["muB"]), K)
    assert abs(L - L_ref) <= 1e-9 * abs(L_ref)
    assert float((gth - gth_ref).abs().max() / gth_ref.abs().max()) <= 1e-9
    gphi = gphi.double().cpu()
    assert float((gphi - gphi_ref).abs().max() / gphi_ref.abs().max()) <= 1e-8


def test_adjoint_d2q9_lattice():
    # the reverse mode on the 2D D2Q9 lattice (FP64 storage, periodic)
    steps, K = 14, 6
    p, fields = configs.ripening_2d(shape=(1, 40, 56), storage="f64", seed=12)
    phi0, cA0, cB0 = fields()
    target = oracle_adjoint.target_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps)
    L_ref, gth_ref, gphi_ref = oracle_adjoint.misfit_gradient(p, configs.THETA_EVAL, phi0, cA0, cB0, steps, target)
    L, gth, gphi = _gpu_grad(p, phi0, cA0, cB0, steps, (target["phi"], target["muA"], target["muB"]), K)
    assert abs(L - L_ref) <= 1e-9 * abs(L_ref)
    assert float((gth - gth_ref).abs().max() / gth_ref.abs().max()) <= 1e-9
    gphi = gphi.double().cpu()
    assert float((gphi - gphi_ref).abs().max() / gphi_ref.abs().max()) <= 1e-8


def test_gradient_vanishes_at_target_parameters():
    from paper_2409_03401_gb300.adjoint import forward_fields
    steps = 30
    p, phi0, cA0, cB0 = _problem((24, 24, 24), "f32", steps)
    target = forward_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps, device="cuda")
    L, gth, gphi = _gpu_grad(p, phi0, cA0, cB0, steps, target, 10, theta=configs.THETA_TARGET)
    assert L == 0.0
    assert float(gth.abs().max()) == 0.0 and float(gphi.abs().max()) == 0.0


@pytest.fixture(scope="module")
def full_adjoint():
    from paper_2409_03401_gb300.adjoint import forward_fields, misfit
    p, fields = configs.adjoint_problem()             # 128^3, FP32
    phi0, cA0, cB0 = [t.cuda() for t in fields(device="cuda")]
    steps = 2000
    target = forward_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps)
    L, gth, gphi = _gpu_grad(p, phi0, cA0, cB0, steps, target, 100)

    def L_at(theta, phi=phi0):
        return float(misfit(forward_fields(p, theta, phi, cA0, cB0, steps), target))
    return L, gth, gphi, L_at, phi0


def test_full_size_theta_gradient_vs_central_differences(full_adjoint):
    L, gth, _, L_at, _ = full_adjoint
    h = 1e-3
    th = list(configs.THETA_EVAL)
    fd = []
    for i in range(3):
        tp, tm = list(th), list(th)
        tp[i] += h
        tm[i] -= h
        fd.append((L_at(tp) - L_at(tm)) / (2 * h))
    fd = torch.tensor(fd, dtype=torch.float64)
    print("128^3 x 2000 adjoint gradient", gth.tolist(), "central differences", fd.tolist(), "L", L)
    assert float(((gth - fd).abs() / fd.abs().max()).max()) <= 2e-2


def test_full_size_phi0_directional_derivative(full_adjoint):
    _, _, gphi, L_at, phi0 = full_adjoint
    g = torch.Generator(device="cuda").manual_seed(11)
    v = torch.randn(phi0.shape, generator=g, device="cuda", dtype=torch.float64)
    v = v * ((phi0 > 0.05) & (phi0 < 0.95))           # perturb the interfaces only
    h = 1e-3
    fd = (L_at(configs.THETA_EVAL, phi0 + h * v) - L_at(configs.THETA_EVAL, phi0 - h * v)) / (2 * h)
    got = float((gphi.double() * v).sum())
    print("phi0 directional derivative: adjoint", got, "central differences", fd)
    assert abs(got - fd) <= 2e-2 * abs(fd)


def test_adjoint_rejects_flow():
    from paper_2409_03401_gb300 import LBMError
    p, phi0, cA0, cB0 = _problem((16, 16, 16), "f32", 4)
    q = p.with_(flow=True)
    with pytest.raises((LBMError, ValueError)):
        _gpu_grad(q, phi0, cA0, cB0, 4, (phi0, phi0, phi0), 2)
