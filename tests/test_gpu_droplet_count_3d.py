"""The one-pass 3D droplet count of the reduction (LBM_RED_EULER on D3Q7/D3Q19 lattices)
against the oracle's Euler characteristic (§4.2.2 counts droplets by the Euler
characteristic; the oracle's is written from the definition of the closed-cube complex).

* Sets of known topology written as the initial phi (0 or 1 at every node, so phi after
  the initialisation is exactly the input): a ball, a shell around a cavity (2), a ring
  (0), a rod closed through the periodic x axis (0) and cut by x walls (1), cubes sharing
  one corner (1: 26-connected).
* Droplet fields after some steps, periodic, with z walls and flow, with x walls, FP32 and
  FP16 storage: the count equals the oracle's on the same phi field (the threshold is taken
  on the kernel's own phi on both sides), and equals the union-find count of the regions.
* The same through the allocation-free reduction.
"""
import numpy as np
import pytest
import torch

from oracle import measure
from parity import run_gpu
from workloads import configs
from workloads.droplets import composition_fields

pytestmark = pytest.mark.gpu


def _walls(p):
    return (p.wall_x, False, p.wall_z)


def _binary(p, a):
    phi = torch.from_numpy(a.astype(np.float64))
    cA, cB = composition_fields(phi, p.c_eq, 0.02)
    return phi, cA, cB


def _shapes():
    shape = (10, 11, 12)
    z = lambda: np.zeros(shape)
    out = []
    a = z(); a[4:7, 4:7, 4:7] = 1
    out.append(("ball", a, False, 1))
    a = z(); a[3:8, 3:8, 3:8] = 1; a[4:7, 4:7, 4:7] = 0
    out.append(("shell", a, False, 2))
    a = z(); a[5, 3:8, 3:8] = 1; a[5, 4:7, 4:7] = 0
    out.append(("ring", a, False, 0))
    a = z(); a[5, 5, :] = 1
    out.append(("rod_periodic", a, False, 0))
    out.append(("rod_walled", a, True, 1))
    a = z(); a[2, 2, 2] = a[3, 3, 3] = 1; a[7, 7, 8] = 1
    out.append(("corner", a, False, 2))
    return out


@pytest.mark.parametrize("name,a,wall_x,chi", _shapes(), ids=[s[0] for s in _shapes()])
def test_known_topologies(name, a, wall_x, chi):
    p, _ = configs.ripening(shape=a.shape, storage="f64")
    p = p.with_(wall_x=wall_x)
    sim, g = run_gpu(p, _binary(p, a), 0)
    assert torch.equal(g["phi"].cpu(), torch.from_numpy(a))
    assert measure.euler_characteristic(a, _walls(p)) == chi
    assert sim.sums()["euler"] == float(chi)


def _case(kind, storage):
    if kind == "periodic":
        p, f = configs.ripening(shape=(40, 48, 56), storage=storage)
    elif kind == "walls_flow":
        p, f = configs.sedimentation(shape=(40, 48, 56), storage=storage, fraction=0.1, r=(4.0, 7.0))
    else:
        p, f = configs.ripening(shape=(40, 48, 56), storage=storage)
        p = p.with_(wall_x=True)
    return p, f()


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("kind", ["periodic", "walls_flow", "wall_x"])
def test_droplet_fields(kind, storage):
    p, f = _case(kind, storage)
    for steps in (0, 30):
        sim, g = run_gpu(p, f, steps)
        phi = g["phi"].cpu().numpy()
        chi = measure.euler_characteristic(phi, _walls(p))
        n = measure.count_droplets(phi, _walls(p))
        assert n > 5
        assert sim.sums()["euler"] == float(chi) == float(n)
        assert sim.droplets()["N"] == float(n)


def test_static_reduce_counts_too():
    import ctypes
    from paper_2409_03401_gb300 import _lib as L
    lib = L.load()
    p, f = _case("periodic", "f32")
    sim, g = run_gpu(p, f, 5)
    cp = L.make_params(sim.params)
    out = (ctypes.c_double * L.NRED)()
    st = lib.lbm_reduce_static(ctypes.byref(cp), ctypes.c_void_p(sim.state.data_ptr()), sim.t, out,
                               ctypes.c_void_p(sim.stream.cuda_stream))
    assert st == L.LBM_OK
    chi = measure.euler_characteristic(g["phi"].cpu().numpy(), _walls(p))
    assert out[L.REDUCTIONS.index("euler")] == float(chi) == sim.sums()["euler"]
