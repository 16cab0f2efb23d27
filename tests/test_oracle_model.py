"""Pins of the oracle's lattice tables, pointwise model and equilibria (CPU only).

Each check compares against something fixed independently of the oracle's own
formulas: lattice isotropy identities, numerical derivatives, the paper's
printed lambda* and relaxation times, and exact moment identities that a
dropped or mis-signed term would break.
"""
import math
import os
import sys

import pytest
import torch

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from values import paper_values  # noqa: E402

from oracle import lattice as L, model as m  # noqa: E402
from oracle.lbm import OracleLBM, _col  # noqa: E402
from workloads.params import LBMParams  # noqa: E402

PV = paper_values()


@pytest.mark.parametrize("lat", [L.D2Q5, L.D3Q7, L.D3Q19, L.D2Q9])
def test_lattice_isotropy(lat):
    e = lat.e_tensor()
    w = lat.w_tensor()
    assert abs(float(w.sum()) - 1.0) < 1e-15
    assert torch.allclose((w[:, None] * e).sum(0), torch.zeros(3, dtype=torch.float64), rtol=0, atol=1e-15)
    dim = 2 if all(v[2] == 0 for v in lat.e) else 3
    second = torch.einsum("k,ki,kj->ij", w, e, e)
    eye = torch.diag(torch.tensor([1.0] * dim + [0.0] * (3 - dim), dtype=torch.float64))
    assert torch.allclose(second, lat.cs2 * eye, rtol=0, atol=1e-15)
    for k in range(lat.Q):
        j = lat.opposite(k)
        assert lat.e[j] == tuple(-v for v in lat.e[k])


@pytest.mark.parametrize("lat", [L.D3Q19, L.D2Q9])
def test_fourth_moment_isotropy(lat):
    # sum w e_i e_j e_k e_l = cs2^2 (d_ij d_kl + d_ik d_jl + d_il d_jk) on the flow lattices
    e = lat.e_tensor()
    w = lat.w_tensor()
    dim = 2 if lat.name == "D2Q9" else 3
    d = torch.eye(3, dtype=torch.float64)
    four = torch.einsum("k,ki,kj,kl,km->ijlm", w, e, e, e, e)
    iso = lat.cs2 ** 2 * (torch.einsum("ij,lm->ijlm", d, d) + torch.einsum("il,jm->ijlm", d, d)
                          + torch.einsum("im,jl->ijlm", d, d))
    assert torch.allclose(four[:dim, :dim, :dim, :dim], iso[:dim, :dim, :dim, :dim], rtol=0, atol=1e-15)


def test_d3q19_matches_paper_table():
    # 6 axis vectors of weight 1/18, 12 face diagonals of weight 1/36 (§3, D3Q19 table)
    for k, (v, w) in enumerate(zip(L.D3Q19.e, L.D3Q19.w)):
        n = sum(abs(c) for c in v)
        assert w == {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[n]
    assert len(set(L.D3Q19.e)) == 19


# the velocity tables of §3 as printed (k = 0..18 and k = 0..8, in the tables' order)
PAPER_D3Q19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
               (1, 1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, -1, -1),
               (1, -1, 0), (-1, 1, 0), (1, 0, -1), (-1, 0, 1), (0, 1, -1), (0, -1, 1)]
PAPER_D2Q9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def test_velocity_tables_in_the_papers_order():
    assert list(L.D3Q19.e) == PAPER_D3Q19
    assert [v[:2] for v in L.D2Q9.e] == PAPER_D2Q9 and all(v[2] == 0 for v in L.D2Q9.e)
    assert list(L.D2Q9.w) == [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    # D3Q19 pairs each direction with its opposite at k +- 1 (k = 1, 3, ..., 17)
    for k in range(1, 19, 2):
        assert tuple(-c for c in PAPER_D3Q19[k]) == PAPER_D3Q19[k + 1]


def test_derivatives_match_finite_differences():
    x = torch.linspace(-0.3, 1.3, 41, dtype=torch.float64)
    h = 1e-6
    assert torch.allclose((m.omega_dw(x + h) - m.omega_dw(x - h)) / (2 * h), m.omega_dw_prime(x), rtol=0, atol=1e-8)
    assert torch.allclose((m.p_interp(x + h) - m.p_interp(x - h)) / (2 * h), m.p_prime(x), rtol=0, atol=1e-8)
    # p(0) = 0, p(1) = 1, p'(0) = p'(1) = 0 and p(1 - phi) = 1 - p(phi) (§2.2)
    assert m.p_interp(0.0) == 0.0 and m.p_interp(1.0) == 1.0
    assert m.p_prime(0.0) == 0.0 and m.p_prime(1.0) == 0.0
    assert torch.allclose(m.p_interp(1 - x), 1 - m.p_interp(x), rtol=0, atol=1e-14)


@pytest.mark.parametrize("axis", ["x", "z"])
def test_stencil_mirror_ghost_at_walls(axis):
    # phi = s^2 along the walled axis s only. On D3Q19 the stencil of Eqs. 42-45 reduces to
    # grad_s = (phi(s+1) - phi(s-1)) / 2 and lap = phi(s+1) - 2 phi(s) + phi(s-1) (the weights
    # with e_s = +1 sum to 1/6); the mirror ghost phi(-1) = phi(0) of a wall (zero normal
    # gradient, §4.2.4) gives grad_s = 1/2 and lap = 1 at s = 0, and grad_s = -(2n - 3)/2,
    # lap = -(2n - 3) at s = n - 1. A periodic wrap or a dropped mirror would differ.
    n = 7
    if axis == "x":
        p = LBMParams(nx=n, ny=3, nz=4, lattice="D3Q7", flow=True, wall_x=True)
        s = torch.arange(n, dtype=torch.float64).reshape(1, 1, -1).expand(p.shape)
        a, pick = 0, (lambda f, i: f[:, :, i])
    else:
        p = LBMParams(nx=3, ny=4, nz=n, lattice="D3Q7", flow=True, wall_z=True)
        s = torch.arange(n, dtype=torch.float64).reshape(-1, 1, 1).expand(p.shape)
        a, pick = 2, (lambda f, i: f[i])
    phi = (s * s).contiguous()
    grad, lap = OracleLBM(p).gradient_laplacian(phi)
    sv = torch.arange(n, dtype=torch.float64)
    up = torch.cat([sv[1:], sv[-1:]]) ** 2            # phi(s + 1), mirrored at the top wall
    dn = torch.cat([sv[:1], sv[:-1]]) ** 2            # phi(s - 1), mirrored at the bottom wall
    for i in range(n):
        assert torch.allclose(pick(grad[a], i), (up[i] - dn[i]) / 2 + 0 * pick(phi, i), rtol=0, atol=1e-13)
        assert torch.allclose(pick(lap, i), up[i] - 2 * sv[i] ** 2 + dn[i] + 0 * pick(phi, i), rtol=0, atol=1e-13)
    assert float(pick(grad[a], 0).max()) == 0.5 and float(pick(lap, 0).max()) == 1.0
    for b in range(3):
        if b != a:
            assert float(grad[b].abs().max()) < 1e-13


def test_tanh_profile_is_the_flat_equilibrium():
    # W^2 phi'' = omega_dw'(phi) for phi_0 of Eq. 13 (the interfacial part of the Allen-Cahn equation)
    W = 3.0
    x = torch.linspace(-8, 8, 3201, dtype=torch.float64)
    dx = float(x[1] - x[0])
    phi = m.tanh_profile(x, W)
    lap = (phi[2:] - 2 * phi[1:-1] + phi[:-2]) / dx ** 2
    assert torch.allclose(W ** 2 * lap, m.omega_dw_prime(phi[1:-1]), rtol=0, atol=1e-5)


def test_delta_omega_two_forms():
    # Eq. 20 (-sum mu (c0 - c1)) equals omega_0 - omega_1 built from Eq. 18
    g = torch.Generator().manual_seed(0)
    mu = torch.randn(2, 50, generator=g, dtype=torch.float64) * 0.1
    ce = ((0.3, 0.25), (0.45, 0.1))
    lhs = m.delta_omega((mu[0], mu[1]), ce)
    rhs = m.grand_potential((mu[0], mu[1]), ce[0]) - m.grand_potential((mu[0], mu[1]), ce[1])
    assert torch.allclose(lhs, rhs, rtol=0, atol=1e-15)


def test_closure_vanishes_at_phase_equilibrium():
    # Eq. 24: mu = 0 for c = c_pi^eq in bulk phase pi, and mu = c - c_1^eq - (phi ... ) is linear in c
    ce = ((0.3, 0.25), (0.45, 0.1))
    for a in range(2):
        assert m.mu_closure(ce[0][a], 0.0, ce[0][a], ce[1][a]) == 0.0
        assert abs(m.mu_closure(ce[1][a], 1.0, ce[0][a], ce[1][a])) < 1e-16
    # the interface-average composition at phi = 1/2 also gives mu = 0
    assert abs(m.mu_closure(0.5 * (ce[0][0] + ce[1][0]), 0.5, ce[0][0], ce[1][0])) < 1e-16


def test_lambda_star_reproduces_paper():
    # §4.1 table: lambda* = 155.94541910 cancels beta (Eq. 27) for M_phi = 1.2, M = (1, 0.8),
    # c_0^eq = (0.3, 0.3), c_1^eq = (0.4, 0.4); W cancels
    want = PV["lambda_star"][0]
    ce = ((0.3, 0.3), (0.4, 0.4))
    got = m.lambda_star(1.2e-3, 1.2, ce, (1.0, 0.8))
    assert abs(got - want) < 5e-9
    assert abs(m.kinetic_coefficient(1.2e-3, got, 1.2, ce, (1.0, 0.8))) < 1e-15


def test_closure_reproduces_the_couple_table_caption():
    # §4.1 caption: the far-field compositions (0.4, 0.175) and (0.225, 0.6) are the chemical
    # potentials (0.1, -0.125) in phase 0 and (-0.175, 0.2) in phase 1 (Eq. 33 with p(0) = 0,
    # p(1) = 1 and the table's c_eq = (0.3, 0.3), (0.4, 0.4))
    ce = ((0.3, 0.3), (0.4, 0.4))
    for side, phi in (("minus", 0.0), ("plus", 1.0)):
        for a, comp in enumerate("AB"):
            c = PV[f"couple_c_{side}_{comp}"][0]
            want = PV[f"couple_mu_{side}_{comp}"][0]
            got = m.mu_closure(c, phi, ce[0][a], ce[1][a])
            assert abs(got - want) < 1e-15, (side, comp, got, want)


def test_relaxation_time_mapping_matches_2d_table():
    # §4.2.3 table: classic tau = 1/rate for M_phi = 1.2, M^A = 1, M^B = 0.8 with the
    # table's dx, dt on D2Q9 (c_s^2 = 1/3): lattice D = M dt / dx^2
    dx, dt = PV["ripening2d_dx"][0], PV["ripening2d_dt"][0]
    for M, key in ((1.2, "ripening2d_tau_g"), (1.0, "ripening2d_tau_hA"), (0.8, "ripening2d_tau_hB")):
        tau = 1.0 / m.relaxation_rate(M * dt / dx ** 2, 1.0 / 3.0)
        assert abs(tau - PV[key][0]) < 2e-4, key


def _random_node_state(seed, flow=True):
    g = torch.Generator().manual_seed(seed)
    shape = (1, 2, 3)
    r = lambda s=1.0: torch.rand(shape, generator=g, dtype=torch.float64) * s  # noqa: E731
    phi = r()
    c = 0.3 + r(0.1)
    mu = r(0.02) - 0.01
    u = [r(0.02) - 0.01 for _ in range(3)]
    F = [r(1e-3) - 5e-4 for _ in range(3)]
    S = r(0.01) - 0.005
    ph = r(1e-3)
    return phi, c, mu, u, F, S, ph


@pytest.mark.parametrize("lattice", ["D3Q7", "D3Q19", "D2Q9"])
def test_equilibrium_moment_identities(lattice):
    p = LBMParams(nx=3, ny=2, nz=1, lattice=lattice, flow=lattice != "D2Q9")
    o = OracleLBM(p)
    phi, c, mu, u, F, S, ph = _random_node_state(1)
    ls = L.BY_NAME[lattice]
    es = ls.e_tensor()
    dims = 2 if lattice == "D2Q9" else 3
    if dims == 2:
        u[2] = torch.zeros_like(u[2])                   # planar motion on a 2D lattice
    # Eq. 51: sum h = c, sum h e = c u, sum h e e = c_s^2 mu I
    h = o._h_eq(c, mu, u)
    assert torch.allclose(h.sum(0), c, rtol=0, atol=1e-15)
    for a in range(dims):
        assert torch.allclose((h * es[:, a].reshape(-1, 1, 1, 1)).sum(0), c * u[a], rtol=0, atol=1e-15)
        for b in range(dims):
            mom = (h * (es[:, a] * es[:, b]).reshape(-1, 1, 1, 1)).sum(0)
            want = ls.cs2 * mu if a == b else torch.zeros_like(mu)
            assert torch.allclose(mom, want, rtol=0, atol=1e-15)
    # Eq. 47: sum g^eq = phi - S/2 and sum g^eq e = phi u (equilibrium as the step builds it)
    w = _col(ls.w)
    cu = torch.stack([sum(ls.e[k][a] * u[a] for a in range(3)) for k in range(ls.Q)])
    geq = w * phi * (1 + cu / ls.cs2) - 0.5 * w * S
    assert torch.allclose(geq.sum(0), phi - S / 2, rtol=0, atol=1e-15)
    for a in range(dims):
        assert torch.allclose((geq * es[:, a].reshape(-1, 1, 1, 1)).sum(0), phi * u[a], rtol=0, atol=1e-15)
    # Eqs. 37-41: sum F_k = 0, sum F_k c_k = c_s^2 F exactly on D3Q19, sum f^eq = p_h,
    # and the velocity moment of f^eq returns u
    lf = L.D3Q19
    ef = lf.e_tensor()
    Fk = o._forcing(u, F)
    assert torch.allclose(Fk.sum(0), torch.zeros_like(phi), rtol=0, atol=1e-18)
    for a in range(3):
        assert torch.allclose((Fk * ef[:, a].reshape(-1, 1, 1, 1)).sum(0), lf.cs2 * F[a], rtol=0, atol=1e-18)
    feq = o._f_eq(ph, u, Fk)
    assert torch.allclose(feq.sum(0), ph, rtol=0, atol=1e-17)
    for a in range(3):
        j = (feq * ef[:, a].reshape(-1, 1, 1, 1)).sum(0)
        assert torch.allclose(j / lf.cs2 + 0.5 * F[a], u[a], rtol=0, atol=1e-16)


def test_source_sign_and_balance():
    # Eq. 35: S vanishes in the bulk phases; Delta omega > 0 (phase 0 has the higher grand
    # potential density) raises phi at the interface, Delta omega < 0 lowers it
    ce = ((0.3, 0.3), (0.4, 0.4))
    W, lam, Mphi = 3.0, 155.95, 0.12
    for phi in (0.0, 1.0):
        assert m.source_phi(phi, (0.01, -0.02), W, lam, Mphi, ce) == 0.0
    up = m.source_phi(0.5, (0.01, 0.01), W, lam, Mphi, ce)      # Delta omega = +0.002
    down = m.source_phi(0.5, (-0.01, -0.01), W, lam, Mphi, ce)
    assert up > 0 > down
    assert abs(up - Mphi / W ** 2 * lam * 1.5 * 0.002) < 1e-15
    # at phi = 1/4 the double well alone pulls phi back towards 0: -(M_phi/W^2) 16 (1/4)(3/4)(1/2)
    assert abs(m.source_phi(0.25, (0.0, 0.0), W, lam, Mphi, ce) + Mphi / W ** 2 * 1.5) < 1e-15
