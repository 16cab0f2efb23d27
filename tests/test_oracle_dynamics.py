"""Dynamic pins of the FP64 oracle against closed forms and exact invariants (CPU only).

* bulk fixed points stay bit-identical (S = 0, mu = 0 at the phase equilibria, §2.2-2.3);
* sum c^A, sum c^B, sum p_h are invariant and sum g changes by exactly sum S (Eqs. 46-52);
* a Fourier mode of c decays with M^alpha, of phi (source off) with M_phi, and a shear
  wave with nu (the tau <-> D relations beside Eqs. 36, 46, 50);
* body-force Poiseuille flow between half-way bounce-back walls (Eqs. 36-41, §4.2.4);
* the flat tanh interface with mu = 0 is stationary (Eqs. 13, 35, 46-49);
* the ternary diffusion couple follows x_I = xi sqrt(t) and the erfc profiles (Eqs. 53-61);
* a static droplet reaches Gibbs-Thomson equilibrium Delta omega = delta kappa (Eqs. 25-26);
* the capillary force gives the Laplace pressure jump sigma kappa (Eq. 34).
"""
import math

import numpy as np
import pytest
import torch

from oracle import analytic, model as m
from oracle.lbm import OracleLBM
from workloads import configs
from workloads.droplets import planar_couple
from workloads.params import LBMParams


def _amp(field, k, n):
    x = torch.arange(n, dtype=torch.float64)
    s = torch.sin(k * x)
    f = field.reshape(-1)
    return float((f * s).sum() / (s * s).sum())


def _mu_uniform_fields(phi, mu, c_eq):
    """Compositions that give a uniform mu through Eq. 24 for a given phi."""
    p = m.p_interp(phi)
    return [mu[a] + (1 - p) * c_eq[0][a] + p * c_eq[1][a] for a in range(2)]


@pytest.mark.parametrize("flow", [False, True])
def test_bulk_fixed_point_is_bit_identical(flow):
    p = LBMParams(nx=6, ny=5, nz=4, lattice="D3Q7", flow=flow, wall_z=flow)
    phi = torch.zeros(p.shape, dtype=torch.float64)
    c = torch.full_like(phi, 0.3)
    o = OracleLBM(p)
    o.init(phi, c, c)
    before = {k: v.clone() for k, v in o.populations().items()}
    o.step(7)
    for k, v in o.populations().items():
        assert torch.equal(v, before[k]), k


def test_bulk_phase_one_fixed_point():
    p = LBMParams(nx=5, ny=4, nz=1, lattice="D2Q5")
    phi = torch.ones(p.shape, dtype=torch.float64)
    c = torch.full_like(phi, 0.4)
    o = OracleLBM(p)
    o.init(phi, c, c)
    before = {k: v.clone() for k, v in o.populations().items()}
    o.step(5)
    # sum_k w_k is 1 only up to rounding (1/3 + 4/6), so S is of order 1e-16 here, not 0
    for k, v in o.populations().items():
        assert float((v - before[k]).abs().max()) < 1e-14, k


@pytest.mark.parametrize("case", ["flow_walls", "periodic", "couple_walls", "flow_walls_d3q19", "periodic_d2q9"])
def test_conservation_and_phi_budget(case):
    if case == "flow_walls":
        p, fields = configs.sedimentation(shape=(16, 16, 18), fraction=0.04, r=(3.0, 4.5))
    elif case == "periodic_d2q9":
        p, fields = configs.ripening(shape=(1, 40, 48))
        p = p.with_(lattice="D2Q9")
    elif case == "flow_walls_d3q19":
        p, fields = configs.sedimentation(shape=(16, 16, 18), fraction=0.04, r=(3.0, 4.5))
        p = p.with_(lattice="D3Q19")
    elif case == "periodic":
        p, fields = configs.ripening(shape=(12, 14, 16))
    else:
        p, fields = configs.diffusion_couple(nx=64, ny=3)
    o = OracleLBM(p)
    o.init(*fields())
    s = o.sums()
    for _ in range(6):
        o.step(1)
        s1 = o.sums()
        for key in ("cA", "cB"):
            assert abs(s1[key] - s[key]) <= 1e-13 * abs(s[key]), key
        assert abs(s1["p"] - s["p"]) <= 1e-15 * p.nodes
        # sum over nodes of sum_k g_k(t+1) = sum g_k(t) + sum S(t)
        assert abs(s1["g"] - (s["g"] + s["S"])) <= 1e-13 * abs(s["g"])
        s = s1


@pytest.mark.parametrize("lattice", ["D3Q7", "D2Q5", "D3Q19", "D2Q9"])
def test_mode_decay_rates(lattice):
    n = 64
    k = 2 * math.pi / n
    p = LBMParams(nx=n, ny=1, nz=1, lattice=lattice, M=((0.1, 0.08), (0.1, 0.08)))
    x = torch.arange(n, dtype=torch.float64).reshape(1, 1, n)
    phi = torch.ones(1, 1, n, dtype=torch.float64)
    cA = 0.4 + 1e-3 * torch.sin(k * x)
    cB = 0.4 + 1e-3 * torch.sin(k * x)
    o = OracleLBM(p)
    o.init(phi, cA, cB)
    a0 = (_amp(o.fields()["cA"], k, n), _amp(o.fields()["cB"], k, n))
    o.step(800)
    for a, M in ((0, 0.1), (1, 0.08)):
        rate = -math.log(_amp(o.fields()["cA" if a == 0 else "cB"], k, n) / a0[a]) / 800
        assert abs(rate / (M * k * k) - 1) < 0.01
    # phase field with the source switched off: pure diffusion with M_phi
    q = p.with_(source_off=True, M_phi=0.12)
    o = OracleLBM(q)
    o.init(0.5 + 0.1 * torch.sin(k * x), cA, cB)
    a0 = _amp(o.fields()["phi"], k, n)
    o.step(800)
    rate = -math.log(_amp(o.fields()["phi"], k, n) / a0) / 800
    assert abs(rate / (0.12 * k * k) - 1) < 0.01


@pytest.mark.parametrize("collision", ["BGK", "TRT", "MRT"])
def test_shear_wave_decay(collision):
    # the shear mode decays at nu k^2 with either collision: omega+ alone sets nu
    n = 32
    k = 2 * math.pi / n
    p = LBMParams(nx=1, ny=n, nz=1, lattice="D3Q7", flow=True, nu=0.1, g=(0.0, 0.0, 0.0), collision=collision)
    y = torch.arange(n, dtype=torch.float64).reshape(1, n, 1)
    phi = torch.zeros(1, n, 1, dtype=torch.float64)
    c = torch.full_like(phi, 0.3)
    o = OracleLBM(p)
    o.init(phi, c, c)
    ux = 1e-3 * torch.sin(k * y)
    z = torch.zeros_like(ux)
    o.f = o._f_eq(z, [ux, z, z], o._forcing([ux, z, z], [z, z, z]))
    a0 = _amp(o.fields()["ux"], k, n)
    o.step(400)
    rate = -math.log(_amp(o.fields()["ux"], k, n) / a0) / 400
    assert abs(rate / (0.1 * k * k) - 1) < 0.01


def test_poiseuille_between_walls():
    H, nu, F = 8, 1.0 / 6.0, 1e-6
    p = LBMParams(nx=1, ny=1, nz=H, lattice="D3Q7", flow=True, wall_z=True, nu=nu, g=(F, 0.0, 0.0))
    phi = torch.ones(H, 1, 1, dtype=torch.float64)   # phi = 1: F_g = g, no capillary force, S = 0
    c = torch.full_like(phi, 0.4)
    o = OracleLBM(p)
    o.init(phi, c, c)
    o.step(int(14 * H * H / (math.pi ** 2 * nu)))
    u = o.fields()["ux"].reshape(-1).numpy()
    ua = analytic.poiseuille(np.arange(H), H, F, nu)
    assert np.abs(u - ua).max() / ua.max() < 0.01
    assert float(o.fields()["uz"].abs().max()) < 1e-12 * ua.max()


@pytest.mark.parametrize("nu", [0.05, 1.0 / 6.0, 0.5])
def test_trt_poiseuille_is_exact_for_any_viscosity(nu):
    # With Lambda = 3/16 the TRT scheme holds the half-way bounce-back wall exactly half-way
    # for every viscosity, so the steady body-force Poiseuille profile equals the analytic
    # parabola at the nodes to round-off (BGK misses it by 0.5-17 % over this range of nu).
    # A dropped or mis-signed even/odd term, or a wrong omega-, breaks the exactness.
    H, F = 8, 1e-6
    p = LBMParams(nx=1, ny=1, nz=H, lattice="D3Q7", flow=True, wall_z=True, nu=nu, g=(F, 0.0, 0.0),
                  collision="TRT", trt_magic=3.0 / 16.0)
    phi = torch.ones(H, 1, 1, dtype=torch.float64)
    c = torch.full_like(phi, 0.4)
    o = OracleLBM(p)
    o.init(phi, c, c)
    o.step(int(40 * H * H / (math.pi ** 2 * nu)))      # transient below exp(-40)
    u = o.fields()["ux"].reshape(-1).numpy()
    ua = analytic.poiseuille(np.arange(H), H, F, nu)
    assert np.abs(u - ua).max() / ua.max() < 1e-12


def test_trt_with_equal_rates_is_bgk():
    # Lambda = (1/omega - 1/2)^2 = (3 nu)^2 makes omega- = omega+: the TRT update is then the
    # BGK update of Eq. 36, up to round-off, on a droplet lattice with walls and forcing
    p, fields = configs.sedimentation(shape=(12, 14, 16), fraction=0.05, r=(2.0, 3.0))
    runs = []
    for coll, lam in (("BGK", 3.0 / 16.0), ("TRT", (3.0 * p.nu) ** 2)):
        o = OracleLBM(p.with_(collision=coll, trt_magic=lam))
        o.init(*fields())
        o.step(10)
        runs.append(o)
    assert float((runs[0].f - runs[1].f).abs().max()) < 1e-15
    # and a different Lambda changes the run (the odd part really relaxes at omega-)
    o = OracleLBM(p.with_(collision="TRT"))
    o.init(*fields())
    o.step(10)
    assert float((runs[0].f - o.f).abs().max()) > 1e-9


def _flow_run(p, fields, steps=10):
    o = OracleLBM(p)
    o.init(*fields())
    o.step(steps)
    return o


def test_mrt_reduces_to_bgk_and_trt():
    # The MRT moments are each even or odd under k -> opp(k). With every rate equal to the
    # BGK rate the MRT update is BGK; with the even moments at omega+ and the odd ones (energy
    # flux, m) at the TRT omega- it is TRT. Both up to round-off on a droplet lattice with walls
    # and forcing; generic rates give a different run.
    p, fields = configs.sedimentation(shape=(12, 14, 16), fraction=0.05, r=(2.0, 3.0))
    om = 1.0 / (3.0 * p.nu + 0.5)
    bgk = _flow_run(p, fields)
    mrt_bgk = _flow_run(p.with_(collision="MRT", mrt_rates=(om,) * 5), fields)
    assert float((bgk.f - mrt_bgk.f).abs().max()) < 1e-15
    lam = 3.0 / 16.0
    om_m = 1.0 / (lam / (1.0 / om - 0.5) + 0.5)
    trt = _flow_run(p.with_(collision="TRT", trt_magic=lam), fields)
    mrt_trt = _flow_run(p.with_(collision="MRT", mrt_rates=(om, om, om_m, om, om_m)), fields)
    assert float((trt.f - mrt_trt.f).abs().max()) < 1e-15
    mrt = _flow_run(p.with_(collision="MRT"), fields)
    assert float((mrt.f - bgk.f).abs().max()) > 1e-9


def test_mrt_moment_basis_is_orthogonal():
    from oracle.lbm import _mrt_matrix
    M = torch.tensor(_mrt_matrix(), dtype=torch.float64)
    G = M @ M.T
    norms = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    assert torch.equal(G, torch.diag(torch.tensor(norms, dtype=torch.float64)))


@pytest.mark.parametrize("lattice", ["D2Q5", "D3Q7", "D3Q19", "D2Q9"])
@pytest.mark.parametrize("W,tol", [(3.0, 1e-2), (6.0, 3e-3)])
def test_flat_interface_is_stationary(lattice, W, tol):
    # a slab of phase 1 with mu = 0 keeps the tanh profile of Eq. 13; the residual gap is the
    # lattice's discrete profile, which shrinks as the interface spans more nodes. The
    # compositions do not relax with phi, so a small mu appears and diffuses away slowly.
    n = 64
    p = LBMParams(nx=n, ny=1, nz=1, lattice=lattice, W=W, M_phi=0.12, lam=10.0,
                  c_eq=((0.1, 0.3), (0.6, 0.1)), M=((0.05, 0.05), (0.1, 0.1)))
    x = torch.arange(n, dtype=torch.float64).reshape(1, 1, n)
    phi0 = m.tanh_profile(x - 15.5, W) * m.tanh_profile(47.5 - x, W)
    cA, cB = _mu_uniform_fields(phi0, (0.0, 0.0), p.c_eq)
    o = OracleLBM(p)
    o.init(phi0, cA, cB)
    o.step(1500)
    f1 = o.fields()["phi"]
    o.step(500)
    f2 = o.fields()["phi"]
    assert float((f2 - f1).abs().max()) < 3e-5
    assert float((f2 - phi0).abs().max()) < tol
    assert float(o.fields()["muA"].abs().max()) < 5e-5


def _interface_position(phi_row):
    cr = np.where(np.diff((phi_row >= 0.5).astype(int)) != 0)[0]
    assert len(cr) == 1, cr
    i = cr[0]
    return i + (phi_row[i] - 0.5) / (phi_row[i] - phi_row[i + 1])


@pytest.mark.slow
def test_diffusion_couple_matches_analytic_solution():
    p, _ = configs.diffusion_couple(nx=512, ny=1)
    ce = p.c_eq
    mu_l, mu_r = (-0.05, 0.05), (0.05, -0.05)
    D1, D0 = p.M[1], p.M[0]
    xi, mu_int = analytic.couple_solution(mu_l, mu_r, D1, D0, ce[1], ce[0], ce)
    assert abs(m.delta_omega(mu_int, ce)) < 1e-14
    o = OracleLBM(p)
    o.init(*planar_couple(p.shape, 255.5, p.W, (0.55, 0.15), (0.15, 0.25)))
    x0 = _interface_position(o.fields()["phi"][0, 0].numpy())
    pos = {}
    for t in (1000, 4000):
        o.step(t - o.t)
        pos[t] = _interface_position(o.fields()["phi"][0, 0].numpy()) - x0
        assert abs(pos[t] - xi * math.sqrt(t)) < 0.5
    # the sqrt(t) law after the start-up transient
    assert abs((pos[4000] - pos[1000]) - xi * (math.sqrt(4000) - math.sqrt(1000))) < 0.05
    f = o.fields()
    muA, muB = analytic.couple_mu_profile(np.arange(512), 4000, xi, mu_int, mu_l, mu_r, D1, D0, x0=255.5)
    assert np.abs(f["muA"][0, 0].numpy() - muA).max() < 2e-3
    assert np.abs(f["muB"][0, 0].numpy() - muB).max() < 2e-3


def test_symmetric_couple_of_the_paper_table():
    # §4.1 table in lattice units: tau_g = 0.6333, tau_h = (0.6111, 0.5888) on c_s^2 = 1/3 give
    # M_phi = 0.0444, M = (0.0370, 0.0296); W = 1.2e-3 / (1/1500) = 1.8 nodes; lambda = 155.95.
    # Phase 0 on the left with mu = (0.1, -0.125), phase 1 on the right with mu = (-0.175, 0.2).
    # Eqs. 53-61 then have the root xi = 0 with mu_int = the mean of the far fields (the
    # printed xi = -0.269824 is not a root of these equations).
    ce = ((0.3, 0.3), (0.4, 0.4))
    M = ((0.6111 - 0.5) / 3, (0.5888 - 0.5) / 3)
    p = LBMParams(nx=256, ny=1, nz=1, lattice="D2Q5", wall_x=True, W=1.8, lam=155.95,
                  M_phi=(0.6333 - 0.5) / 3, c_eq=ce, M=(M, M))
    mu_l, mu_r = (0.1, -0.125), (-0.175, 0.2)
    xi, mu_int = analytic.couple_solution(mu_l, mu_r, M, M, ce[0], ce[1], ce)
    assert abs(xi) < 1e-12
    assert abs(mu_int[0] + 0.0375) < 1e-12 and abs(mu_int[1] - 0.0375) < 1e-12
    c_left = (ce[0][0] + mu_l[0], ce[0][1] + mu_l[1])
    c_right = (ce[1][0] + mu_r[0], ce[1][1] + mu_r[1])
    phi0, cA, cB = planar_couple(p.shape, 127.5, p.W, c_right, c_left)
    phi0 = 1.0 - phi0                                  # phase 0 on the left
    cA = torch.where(phi0 < 0.5, torch.full_like(cA, c_left[0]), torch.full_like(cA, c_right[0]))
    cB = torch.where(phi0 < 0.5, torch.full_like(cB, c_left[1]), torch.full_like(cB, c_right[1]))
    o = OracleLBM(p)
    o.init(phi0, cA, cB)
    o.step(4000)
    f = o.fields()
    muA, muB = analytic.couple_mu_profile(np.arange(256), 4000, 0.0, mu_int, mu_l, mu_r, M, M, x0=127.5)
    assert np.abs(f["muA"][0, 0].numpy() - muA).max() < 5e-3
    assert np.abs(f["muB"][0, 0].numpy() - muB).max() < 5e-3
    row = 1.0 - f["phi"][0, 0].numpy()
    assert abs(_interface_position(row) - 127.5) < 0.25


def _disc(n, R, W):
    x = torch.arange(n, dtype=torch.float64)
    d = torch.sqrt((x.reshape(-1, 1) - (n - 1) / 2) ** 2 + (x.reshape(1, -1) - (n - 1) / 2) ** 2)
    return m.tanh_profile(R - d, W).reshape(1, n, n)


@pytest.mark.slow
def test_gibbs_thomson_static_disc():
    # a disc of phase 1 in a closed periodic box settles where Delta omega = delta kappa,
    # delta = 2W/(3 lambda) (Eq. 26), kappa = 1/R in 2D. It starts at 0.8 of that mu, shrinks,
    # and the released solute raises mu until the relation holds (the box is small enough
    # for this closed-system equilibrium to be stable).
    n, W, lam, R0 = 48, 3.0, 100.0, 12.0
    ce = ((0.3, 0.3), (0.4, 0.4))
    p = LBMParams(nx=n, ny=n, nz=1, lattice="D2Q5", W=W, lam=lam, M_phi=0.12, c_eq=ce,
                  M=((0.3, 0.3), (0.3, 0.3)))
    phi0 = _disc(n, R0, W)
    mu0 = 0.8 * m.capillary_length(W, lam) / R0 / 0.2      # Delta omega = 0.2 mu for these c_eq
    cA, cB = _mu_uniform_fields(phi0, (mu0, mu0), ce)
    o = OracleLBM(p)
    o.init(phi0, cA, cB)
    o.step(4500)
    f = o.fields()
    R = math.sqrt(float(f["phi"].sum()) / math.pi)
    assert R < R0 - 0.3                                       # it shrank towards equilibrium
    mu_far = (float(f["muA"][0, :4, :4].mean()), float(f["muB"][0, :4, :4].mean()))
    dw = m.delta_omega(mu_far, ce)
    assert abs(dw / (m.capillary_length(W, lam) / R) - 1) < 0.04
    assert float(f["muA"].max() - f["muA"].min()) < 3e-5      # mu uniform at rest


@pytest.mark.slow
def test_gibbs_thomson_static_sphere():
    # 3D: a sphere of phase 1 settles where Delta omega = delta kappa with kappa = 2/R (the sum
    # of the principal curvatures). It starts at 1.3 times that mu, grows and depletes the
    # closed periodic box until the relation holds (growing is the stable side in 3D at this
    # size: started below it, the sphere dissolves).
    n, W, lam, R0 = 28, 3.0, 100.0, 9.0
    ce = ((0.3, 0.3), (0.4, 0.4))
    p = LBMParams(nx=n, ny=n, nz=n, lattice="D3Q7", W=W, lam=lam, M_phi=0.12, c_eq=ce,
                  M=((0.3, 0.3), (0.3, 0.3)))
    x = torch.arange(n, dtype=torch.float64)
    c = (n - 1) / 2
    d = torch.sqrt((x.reshape(-1, 1, 1) - c) ** 2 + (x.reshape(1, -1, 1) - c) ** 2 + (x.reshape(1, 1, -1) - c) ** 2)
    phi0 = m.tanh_profile(R0 - d, W)
    delta = m.capillary_length(W, lam)
    mu0 = 1.3 * delta * 2.0 / R0 / 0.2                    # Delta omega = 0.2 mu for these c_eq
    cA, cB = _mu_uniform_fields(phi0, (mu0, mu0), ce)
    o = OracleLBM(p)
    o.init(phi0, cA, cB)
    o.step(2000)
    f = o.fields()
    R = (3.0 * float(f["phi"].sum()) / (4.0 * math.pi)) ** (1.0 / 3.0)
    assert R > R0 + 1.5                                    # it grew towards equilibrium
    mu_far = (float(f["muA"][:3, :3, :3].mean()), float(f["muB"][:3, :3, :3].mean()))
    dw = m.delta_omega(mu_far, ce)
    assert abs(dw / (delta * 2.0 / R) - 1) < 0.02
    assert float(f["muA"].max() - f["muA"].min()) < 3e-5   # mu uniform at rest


@pytest.mark.slow
def test_laplace_pressure_of_a_cylinder():
    # capillary force of Eq. 34 on a cylinder (3D lattice, one node thick in y):
    # p_in - p_out = sigma / R; mu starts at its Gibbs-Thomson value so the cylinder is at rest
    n, W, lam, sigma, R0 = 32, 3.0, 100.0, 1e-2, 9.0
    ce = ((0.3, 0.3), (0.4, 0.4))
    p = LBMParams(nx=n, ny=1, nz=n, lattice="D3Q7", flow=True, W=W, lam=lam, M_phi=0.12, c_eq=ce,
                  M=((0.1, 0.1), (0.1, 0.1)), nu=1.0 / 6.0, sigma=sigma, g=(0.0, 0.0, 0.0))
    phi0 = _disc(n, R0, W).reshape(n, 1, n)
    mu_gt = m.capillary_length(W, lam) / R0 / 0.2
    cA, cB = _mu_uniform_fields(phi0, (mu_gt, mu_gt), ce)
    o = OracleLBM(p)
    o.init(phi0, cA, cB)
    o.step(1500)
    f = o.fields()
    R = math.sqrt(float(f["phi"].sum()) / math.pi)
    pr = f["p"][:, 0, :]
    c = n // 2
    dp = float(pr[c - 2:c + 2, c - 2:c + 2].mean() - pr[:3, :3].mean())
    # at W = 3 the central-difference gradient integrates (3/2) W |grad phi|^2 across the tanh
    # profile to 0.898 instead of 1, so the jump is ~8% low (0.9945 at W = 6, not run here);
    # a wrong prefactor or a dropped laplacian term misses by a third or more
    assert abs(dp / (sigma / R) - 1) < 0.1
    # spurious currents stay small: capillary number u nu / sigma below 1e-2
    assert float(torch.sqrt(f["ux"] ** 2 + f["uz"] ** 2).max()) * (1.0 / 6.0) / sigma < 1e-2


@pytest.mark.slow
def test_laplace_pressure_of_a_sphere():
    # 3D: p_in - p_out = 2 sigma / R (Eq. 34 with the full D3Q19 stencil in all three
    # directions); mu starts at its Gibbs-Thomson value for R0 so the sphere stays put. As for
    # the cylinder, W = 3 leaves the jump ~7 % low; a curvature of 1/R would halve it
    n, W, lam, sigma, R0 = 28, 3.0, 100.0, 1e-2, 8.0
    ce = ((0.3, 0.3), (0.4, 0.4))
    p = LBMParams(nx=n, ny=n, nz=n, lattice="D3Q7", flow=True, W=W, lam=lam, M_phi=0.12, c_eq=ce,
                  M=((0.1, 0.1), (0.1, 0.1)), nu=1.0 / 6.0, sigma=sigma, g=(0.0, 0.0, 0.0))
    x = torch.arange(n, dtype=torch.float64)
    c = (n - 1) / 2
    d = torch.sqrt((x.reshape(-1, 1, 1) - c) ** 2 + (x.reshape(1, -1, 1) - c) ** 2 + (x.reshape(1, 1, -1) - c) ** 2)
    phi0 = m.tanh_profile(R0 - d, W)
    mu_gt = m.capillary_length(W, lam) * 2.0 / R0 / 0.2
    cA, cB = _mu_uniform_fields(phi0, (mu_gt, mu_gt), ce)
    o = OracleLBM(p)
    o.init(phi0, cA, cB)
    o.step(500)
    f = o.fields()
    R = (3.0 * float(f["phi"].sum()) / (4.0 * math.pi)) ** (1.0 / 3.0)
    h = n // 2
    dp = float(f["p"][h - 2:h + 2, h - 2:h + 2, h - 2:h + 2].mean() - f["p"][:3, :3, :3].mean())
    assert abs(dp / (2.0 * sigma / R) - 1) < 0.1
    u = torch.sqrt(f["ux"] ** 2 + f["uy"] ** 2 + f["uz"] ** 2)
    assert float(u.max()) * (1.0 / 6.0) / sigma < 1e-2


def _wave_phase(profile, k, L):
    """(amplitude, shift) of profile ~ amp sin(k (x - shift)) by projection on sin and cos."""
    x = torch.arange(L, dtype=torch.float64)
    a = float((profile * torch.sin(k * x)).sum()) * 2 / L
    b = float((profile * torch.cos(k * x)).sum()) * 2 / L
    return math.hypot(a, b), math.atan2(-b, a) / k


@pytest.mark.parametrize("lattice", ["D3Q7", "D3Q19"])
def test_composition_is_advected_by_the_flow(lattice):
    # phase 1 everywhere (phi = 1: no source, no capillary force) under a uniform buoyancy
    # phi g: the fluid starts at rest and gains g per step (u_T = T g, Eq. 41 with the forcing
    # of Eq. 36), and a sine wave of c^A rides on it through the c u / c_s^2 term of Eq. 51:
    # it moves by sum_{n<T} u_n = g T (T - 1) / 2 and decays as exp(-D k^2 T)
    L, T, gx, D, eps = 64, 400, 2e-5, 0.1, 1e-3
    ce = ((0.3, 0.3), (0.4, 0.4))
    p = LBMParams(nx=L, ny=4, nz=4, lattice=lattice, flow=True, W=3.0, lam=100.0, M_phi=0.12, c_eq=ce,
                  M=((D, D), (D, D)), nu=0.1, sigma=1e-3, g=(gx, 0.0, 0.0))
    k = 2 * math.pi / L
    x = torch.arange(L, dtype=torch.float64)
    phi = torch.ones(p.shape, dtype=torch.float64)
    cA = (0.4 + eps * torch.sin(k * x)).reshape(1, 1, L).expand(p.shape).contiguous()
    cB = torch.full(p.shape, 0.4, dtype=torch.float64)
    o = OracleLBM(p)
    o.init(phi, cA, cB)
    o.step(T)
    f = o.fields()
    assert float((f["phi"] - 1).abs().max()) < 1e-14
    assert abs(float(f["ux"].mean()) - T * gx) < 1e-12 and float(f["ux"].std()) < 1e-14
    amp, shift = _wave_phase(f["cA"][0, 0] - f["cA"][0, 0].mean(), k, L)
    assert abs(shift - gx * T * (T - 1) / 2) < 0.01                 # of 1.596 nodes
    assert abs(amp / eps / math.exp(-D * k * k * T) - 1) < 2e-3


def test_phase_field_is_advected_by_the_flow():
    # the phi equation alone (source off, sigma = 0): a small sine wave of phi around 1/2 under
    # buoyancy phi g moves with the mean velocity 0.5 g n through the phi u / c_s^2 term of
    # Eq. 47 and decays as exp(-M_phi k^2 T); the wave itself makes the force slightly
    # non-uniform, so the shift is held to 0.03 of its 1.596 nodes
    L, T, gx, Mphi, eps = 64, 400, 4e-5, 0.05, 1e-3
    ce = ((0.3, 0.3), (0.4, 0.4))
    p = LBMParams(nx=L, ny=4, nz=4, lattice="D3Q7", flow=True, W=3.0, lam=100.0, M_phi=Mphi, c_eq=ce,
                  M=((0.1, 0.1), (0.1, 0.1)), nu=0.1, sigma=0.0, g=(gx, 0.0, 0.0), source_off=True)
    k = 2 * math.pi / L
    x = torch.arange(L, dtype=torch.float64)
    phi = (0.5 + eps * torch.sin(k * x)).reshape(1, 1, L).expand(p.shape).contiguous()
    c = torch.full(p.shape, 0.35, dtype=torch.float64)
    o = OracleLBM(p)
    o.init(phi, c, c.clone())
    o.step(T)
    f = o.fields()
    amp, shift = _wave_phase(f["phi"][0, 0] - f["phi"][0, 0].mean(), k, L)
    assert abs(shift - 0.5 * gx * T * (T - 1) / 2) < 0.03
    assert abs(amp / eps / math.exp(-Mphi * k * k * T) - 1) < 2e-3
