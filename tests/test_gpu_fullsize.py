"""The 512^3 flow workload in the launch configuration the benchmark times.

The oracle cannot run 512^3, so the check samples: after two steps, every node of
a 6^3 block inside a 20^3 window is compared with an FP64 oracle run of the same
window (a node after s steps depends on the state within 2s + 1 nodes, so the
window's artificial edges do not reach the compared block). Windows sit in the
bulk, on droplet interfaces and against both walls. Global FP64 invariants are
checked over the whole lattice.
"""
import numpy as np
import pytest
import torch

from parity import FLOORS, TOL, rel_linf
from workloads import configs

pytestmark = pytest.mark.gpu

N = 512
WIN, MARGIN, STEPS = 20, 7, 2


@pytest.fixture(scope="module")
def full_run():
    from paper_2409_03401_gb300 import Simulation
    p, fields = configs.sedimentation(n=N)
    phi0, cA0, cB0 = fields(device="cuda")
    sim = Simulation(p, phi0, cA0, cB0)
    s0 = sim.sums()
    sim.step(STEPS)
    out = sim.fields()
    s1 = sim.sums()
    torch.cuda.synchronize()
    yield p, (phi0, cA0, cB0), out, s0, s1, fields.geometry()
    del sim


def _window(t, z0, y0, x0, wall_top):
    zi = torch.arange(z0, z0 + WIN, device=t.device)
    yi = torch.arange(y0, y0 + WIN, device=t.device) % N
    xi = torch.arange(x0, x0 + WIN, device=t.device) % N
    return t[zi][:, yi][:, :, xi].cpu()


def _corners(geometry):
    centres, radii = geometry
    c, r = centres[0], radii[0]
    # (z0, y0, x0): bulk, droplet interface, bottom wall, top wall, interface across the x wrap
    return [(200, 100, 300),
            (int(c[2]) - WIN // 2, int(c[1]) - WIN // 2, int(c[0] + r) - WIN // 2),
            (0, 40, 77),
            (N - WIN, 333, 5),
            (250, 250, N - 10)]


def test_sampled_windows_match_oracle(full_run):
    from oracle.lbm import OracleLBM
    p, init, out, _, _, geometry = full_run
    worst = {}
    for z0, y0, x0 in _corners(geometry):
        z0 = min(max(z0, 0), N - WIN)
        wp = p.with_(nx=WIN, ny=WIN, nz=WIN)          # walls at both window ends along z
        o = OracleLBM(wp)
        o.init(*[_window(t, z0, y0, x0, True) for t in init])
        o.step(STEPS)
        ref = o.fields()
        zlo = 0 if z0 == 0 else MARGIN
        zhi = WIN if z0 == N - WIN else WIN - MARGIN
        sl = (slice(zlo, zhi), slice(MARGIN, WIN - MARGIN), slice(MARGIN, WIN - MARGIN))
        for k in ("phi", "muA", "muB", "cA", "cB", "p", "ux", "uy", "uz"):
            g = _window(out[k], z0, y0, x0, True)[sl]
            err = rel_linf(g, ref[k][sl], k)
            worst[k] = max(worst.get(k, 0.0), err)
    print("512^3 sampled-window errors:", worst)
    assert all(v <= TOL["f32"] for v in worst.values()), worst


def test_full_lattice_invariants(full_run):
    p, init, out, s0, s1, _ = full_run
    for k in ("cA", "cB"):
        assert abs(s1[k] - s0[k]) <= 1e-6 * abs(s0[k])
    assert s1["nonfinite"] == 0
    assert abs(s1["p"] - s0["p"]) <= 1e-6 * N ** 3 * 1e-4
    phi = out["phi"]
    assert float(phi.min()) > -0.05 and float(phi.max()) < 1.05
    # initial sums against the FP64 inputs
    assert abs(s0["cA"] - float(init[1].sum())) <= 1e-6 * float(init[1].sum())


def test_full_lattice_droplet_count(full_run):
    # the Euler count of the reduction on the whole 512^3 lattice: the placed droplets at
    # t = 0 (none overlap or touch a wall), and the oracle's count of the GPU's phi after the steps
    from oracle import measure
    p, _, out, s0, s1, geometry = full_run
    assert s0["euler"] == float(len(geometry[1]))
    phi = out["phi"].cpu().numpy()
    assert s1["euler"] == float(measure.euler_characteristic(phi, (p.wall_x, False, p.wall_z)))


def test_reduction_sums_carry_fp64_accuracy(full_run):
    # the reduction forms each node's value in FP32 and sums it per thread as a float-float
    # pair (about 1,200 nodes per thread at this size, error bound 1,200 * 2^-47 relative):
    # its sum of phi over the whole lattice equals the FP64 sum of the same FP32 values
    # (the fields' phi comes from the same phi pass) far below FP32's own rounding
    _, _, out, _, s1, _ = full_run
    ref = float(out["phi"].double().sum())
    assert abs(s1["phi"] - ref) <= 1e-11 * abs(ref), (s1["phi"], ref)


@pytest.mark.parametrize("inplace", [False, True], ids=["two_buffers", "in_place"])
def test_fp16_storage_sampled_windows_match_oracle(full_run, inplace):
    # the FP16-storage lines of the benchmark (fused two-buffer kernel, and the in-place
    # layout) on the same 512^3 workload: the same sampled windows after the same two steps,
    # held to the 16-bit bar. The scale of each field is its largest magnitude over all
    # windows (a quiet bulk window alone would measure u against its own tiny values).
    from oracle.lbm import OracleLBM
    from paper_2409_03401_gb300 import Simulation
    p, init, _, _, _, geometry = full_run
    sim = Simulation(p.with_(storage="f16", inplace=inplace), *init)
    sim.step(STEPS)
    out = sim.fields()
    torch.cuda.synchronize()
    err, scale = {}, {}
    for z0, y0, x0 in _corners(geometry):
        z0 = min(max(z0, 0), N - WIN)
        o = OracleLBM(p.with_(nx=WIN, ny=WIN, nz=WIN))
        o.init(*[_window(t, z0, y0, x0, True) for t in init])
        o.step(STEPS)
        ref = o.fields()
        zlo = 0 if z0 == 0 else MARGIN
        zhi = WIN if z0 == N - WIN else WIN - MARGIN
        sl = (slice(zlo, zhi), slice(MARGIN, WIN - MARGIN), slice(MARGIN, WIN - MARGIN))
        for k in ("phi", "muA", "muB", "cA", "cB", "p", "ux", "uy", "uz"):
            g = _window(out[k], z0, y0, x0, True)[sl].double()
            r = ref[k][sl].double()
            err[k] = max(err.get(k, 0.0), float((g - r).abs().max()))
            scale[k] = max(scale.get(k, 0.0), float(r.abs().max()))
    del sim, out
    torch.cuda.synchronize()
    rel = {k: err[k] / max(scale[k], FLOORS[k]) for k in err}
    print(f"512^3 FP16 ({'in place' if inplace else 'two buffers'}) sampled-window errors:", rel)
    assert all(v <= TOL["f16"] for v in rel.values()), rel
