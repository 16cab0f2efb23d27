"""A lattice decomposed into z slabs (lbm_slab_*) against the same lattice undivided.

The slabs exchange, after every step, the populations leaving through their faces and
phi of their edge planes (paper §3: domain decomposition with one halo exchange per
step). Each node's arithmetic is that of the undivided lattice, so the fields must agree
bit for bit: walls and periodic ends, flow (the fused kernel, and the D3Q19 phi pass +
pull step) and no flow, FP64, FP32 and 16-bit storage, uneven splits down to one-plane
slabs, slabs longer than one z chunk of the fused kernel, and one periodic slab that is its
own neighbour.
"""
import pytest
import torch

from paper_2409_03401_gb300 import Simulation
from paper_2409_03401_gb300.slabs import SlabGroup
from workloads import configs

pytestmark = pytest.mark.gpu

NAMES = ("phi", "muA", "muB", "cA", "cB", "p", "ux", "uy", "uz")


def _run(p, fields, n, steps):
    f = fields()
    ref = Simulation(p, *f)
    ref.step(steps)
    grp = SlabGroup(p, n, *f)
    grp.step(steps)
    names = NAMES if p.flow else NAMES[:5]
    a, b = ref.fields(names), grp.fields(names)
    torch.cuda.synchronize()
    return a, b, ref, grp


def _equal(a, b):
    bad = {k: float((a[k].double() - b[k].double()).abs().max()) for k in a if not torch.equal(a[k], b[k])}
    assert not bad, f"slab run differs from the undivided lattice: {bad}"


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("walls", [True, False])
@pytest.mark.parametrize("n", [2, 3])
def test_flow_slabs_equal_undivided(storage, walls, n):
    p, fields = configs.sedimentation(shape=(37, 20, 36), fraction=0.06, r=(3.0, 5.0), storage=storage)
    a, b, _, _ = _run(p.with_(wall_z=walls), fields, n, 12)
    _equal(a, b)


def test_flow_slabs_longer_than_a_chunk_and_one_plane_slabs():
    # 75 planes into 2 slabs of 38 and 37 (two z chunks each), and 7 planes into 4 slabs
    p, fields = configs.sedimentation(shape=(75, 16, 34), fraction=0.05, r=(3.0, 4.0))
    a, b, _, _ = _run(p, fields, 2, 8)
    _equal(a, b)
    # (the ripening workload's droplets, placed periodically: no droplet fits between walls
    # seven planes apart)
    p, fields = configs.ripening(shape=(7, 18, 40))
    for walls in (True, False):
        a, b, _, _ = _run(p.with_(flow=True, wall_z=walls), fields, 4, 9)
        _equal(a, b)


def test_single_periodic_slab_is_its_own_neighbour():
    p, fields = configs.ripening(shape=(12, 14, 40))
    for q in (p, p.with_(flow=True)):
        a, b, _, _ = _run(q, fields, 1, 10)
        _equal(a, b)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_ripening_slabs_equal_undivided(storage):
    # no flow: the undivided lattice runs in place (AA pattern), the slabs with two copies
    p, fields = configs.ripening(shape=(30, 18, 50), storage=storage)
    a, b, _, _ = _run(p, fields, 3, 15)
    _equal(a, b)


def test_d3q19_flow_slabs_equal_undivided():
    # the D3Q19 scalar lattice with flow: phi pass + pull step, ghost phi copied into the
    # phi field
    p, fields = configs.sedimentation(shape=(24, 14, 40), fraction=0.05, r=(3.0, 5.0))
    a, b, _, _ = _run(p.with_(lattice="D3Q19"), fields, 3, 8)
    _equal(a, b)


def test_slab_sums_add_up():
    p, fields = configs.sedimentation(shape=(30, 20, 36), fraction=0.06, r=(3.0, 5.0), storage="f64")
    _, _, ref, grp = _run(p, fields, 3, 6)
    s, g = ref.sums(), grp.sums()
    for k in ("phi", "cA", "cB", "p", "S", "g", "interface"):
        assert abs(s[k] - g[k]) <= 1e-12 * max(abs(s[k]), 1.0), (k, s[k], g[k])
    assert s["umax"] == g["umax"]


def test_slab_refuses_multi_step_calls_and_walls():
    from paper_2409_03401_gb300 import _lib
    from paper_2409_03401_gb300.slabs import Slab
    p, fields = configs.ripening(shape=(12, 10, 32))
    p = p.with_(flow=True, wall_z=True)
    s = Slab(p, 0, 6, *fields())
    assert s.has == (False, True)
    assert s.lib.lbm_step(s._ctx, 2) == _lib.LBM_ERR_STATE
    with pytest.raises(_lib.LBMError):
        s.unpack(0, s.pack(1))            # no neighbour below a wall
