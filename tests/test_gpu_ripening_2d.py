"""2D ripening on D2Q9 (the paper's 2D lattice, §4.2.2 table) against the FP64 oracle, and
the one-pass droplet measurements of the reduction kernel against the oracle's own.

* FP64 storage to 1e-12 and FP32 to 1e-5 of the oracle on a ragged 2D lattice, periodic
  and with x walls (the diffusion couple on D2Q9).
* LBM_RED_EULER (Gray's bit quads) equals the number of 8-connected regions of
  phi >= 1/2 that the oracle's union-find counts on the same FP32 phi field (the threshold
  is taken in the kernel's precision on both sides), periodic and with x walls.
* LBM_RED_INTERFACE equals the oracle's sum of (4/W) phi (1 - phi) (Eq. 67) to FP32 accuracy,
  so <R> = interface / (2 pi N) agrees.
"""
import math

import numpy as np
import pytest
import torch

from oracle import measure
from parity import TOL, compare, run_gpu, run_oracle
from workloads import configs
from workloads.droplets import composition_fields, phi_field, place_droplets

pytestmark = pytest.mark.gpu


def _close(errs, tol):
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"tolerance {tol}: {bad} (all: {errs})"


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_d2q9_ripening_parity(storage):
    p, fields = configs.ripening_2d(shape=(1, 90, 130), storage=storage)
    _close(compare(p, fields(), 40), TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_d2q9_couple_parity(storage):
    p, fields = configs.diffusion_couple(nx=96, ny=6, storage=storage)
    _close(compare(p.with_(lattice="D2Q9"), fields(), 300), TOL[storage])


def _walled_droplets(shape, seed):
    p, _ = configs.ripening_2d(shape=shape)
    p = p.with_(wall_x=True)
    centres, radii = place_droplets(p.shape, 0.08, configs.RIPENING_2D_R[0], configs.RIPENING_2D_R[1], p.W,
                                    seed, walls=(True, False, False), sample_volume=True)
    phi = phi_field(p.shape, centres, radii, p.W, walls=(True, False, False))
    cA, cB = composition_fields(phi, p.c_eq, 0.1)
    return p, (phi, cA, cB)


@pytest.mark.parametrize("walls", [False, True])
def test_droplet_count_and_mean_radius(walls):
    if walls:
        p, f = _walled_droplets((1, 256, 320), 8)
    else:
        p, fields = configs.ripening_2d(shape=(1, 256, 320), seed=7)
        f = fields()
    steps = 60
    sim, g = run_gpu(p, f, steps)
    s = sim.sums()
    phi32 = g["phi"].cpu().numpy()
    n_ref = measure.count_droplets(phi32, walls=(walls, False, False))
    assert n_ref > 10
    assert s["euler"] == float(n_ref)
    o, r = run_oracle(p, f, steps)
    a_ref = measure.interface_measure(r["phi"].numpy(), p.W)
    assert abs(s["interface"] - a_ref) <= 1e-5 * a_ref
    R_gpu = s["interface"] / (2 * math.pi * s["euler"])
    R_ref, N_ref = measure.mean_radius(r["phi"].numpy(), p.W, walls=(walls, False, False))
    assert N_ref == n_ref
    assert abs(R_gpu - R_ref) <= 1e-5 * R_ref


def test_full_size_4096_squared_matches_oracle():
    # the 4096^2 D2Q9 run as the bench times it (FP32, in place), against the oracle on the
    # whole lattice after 3 steps, and the droplet count of the initial field
    p, fields = configs.ripening_2d()
    f = fields()
    sim, g = run_gpu(p, [t.cuda() for t in f], 3)
    _, r = run_oracle(p, f, 3)
    from parity import rel_linf
    errs = {k: rel_linf(g[k], r[k], k) for k in ("phi", "muA", "muB", "cA", "cB")}
    _close(errs, TOL["f32"])
    s = sim.sums()
    assert s["euler"] == float(measure.count_droplets(g["phi"].cpu().numpy()))
