"""Pins of the seeded input generators and of the droplet measurements (CPU only)."""
import math

import numpy as np
import pytest
import torch

from oracle import measure, model as m
from workloads import configs
from workloads.droplets import place_droplets, phi_field, composition_fields
from workloads.rng import SplitMix64


def test_splitmix64_reference_vectors():
    # outputs of the published splitmix64 reference for seeds 0 and 1234567
    r = SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973, 9817491932198370423]
    u = SplitMix64(5).uniform()
    assert 0.0 <= u < 1.0 and (u * 2 ** 53) == int(u * 2 ** 53)


@pytest.mark.parametrize("walls", [(False, False, False), (False, False, True)])
def test_droplet_placement_constraints(walls):
    shape = (40, 36, 44)
    W = 3.0
    centres, radii = place_droplets(shape, 0.08, 3.0, 6.0, W, seed=11, walls=walls)
    nz, ny, nx = shape
    ext = np.array([nx, ny, nz], dtype=float)
    vol = (4.0 / 3.0 * math.pi * radii ** 3).sum()
    assert vol >= 0.08 * nx * ny * nz
    assert np.all((radii >= 3.0) & (radii <= 6.0))
    for i in range(len(radii)):
        for j in range(i):
            d = centres[i] - centres[j]
            for ax in range(3):
                if not walls[ax]:
                    d[ax] -= ext[ax] * round(d[ax] / ext[ax])
            assert np.linalg.norm(d) >= radii[i] + radii[j] + W
        if walls[2]:
            assert centres[i, 2] + 0.5 - radii[i] >= W / 2
            assert ext[2] - 0.5 - centres[i, 2] - radii[i] >= W / 2
    again = place_droplets(shape, 0.08, 3.0, 6.0, W, seed=11, walls=walls)
    assert np.array_equal(again[0], centres) and np.array_equal(again[1], radii)


def test_fields_and_measurements_on_known_spheres():
    shape = (48, 48, 48)
    W = 3.0
    centres = np.array([[12.3, 14.1, 13.0], [34.0, 33.2, 30.7], [36.5, 10.0, 38.0]])
    radii = np.array([7.0, 9.0, 6.0])
    phi = phi_field(shape, centres, radii, W)
    assert float(phi.max()) <= 1.0 and float(phi.min()) >= 0.0
    # the tanh of Eq. 13 at the centre of the largest sphere, and (1 + tanh(2r/W))/2 at r from a surface
    c = np.round(centres[1]).astype(int)
    d = float(np.linalg.norm(c - centres[1]))
    assert abs(float(phi[c[2], c[1], c[0]]) - m.tanh_profile(9.0 - d, W)) < 1e-12
    R, n = measure.mean_radius(phi.numpy(), W)
    assert n == 3
    want = math.sqrt((4 * math.pi * (radii ** 2)).sum() / (4 * math.pi * 3))
    assert abs(R / want - 1) < 0.03
    cA, cB = composition_fields(phi, ((0.3, 0.3), (0.4, 0.4)), 0.02)
    inside = phi >= 0.5
    assert torch.all(cA[inside] == 0.4) and torch.allclose(cA[~inside], torch.full_like(cA[~inside], 0.302),
                                                           rtol=0, atol=1e-15)


def test_periodic_droplet_counts_once():
    shape = (32, 32, 32)
    phi = phi_field(shape, np.array([[1.0, 16.0, 16.0]]), np.array([6.0]), 3.0)
    assert measure.count_droplets(phi.numpy()) == 1
    assert measure.count_droplets(phi.numpy(), walls=(True, False, False)) == 2


def test_configs_build():
    p, fields = configs.ripening(shape=(24, 24, 24))
    phi, cA, cB = fields()
    assert phi.shape == p.shape and cA.dtype == torch.float64
    p, fields = configs.diffusion_couple(nx=32, ny=2)
    phi, cA, cB = fields()
    assert phi.shape == (1, 2, 32)
    assert float(cA[0, 0, 0]) == 0.55 and float(cB[0, 0, -1]) == 0.25


def _brute_chi(a, walls):
    """Euler characteristic by listing the cells of every closed unit cube (square) in doubled
    coordinates: node p spans 2p..2p+2 along each axis, a coordinate is odd inside that span
    and even on its boundary; a cell's dimension is its number of odd coordinates. Periodic
    axes wrap modulo 2n. Each distinct cell counts (-1)^dimension."""
    a = np.asarray(a) >= 0.5
    walled = [walls[2], walls[1], walls[0]]
    if a.shape[0] == 1:
        a, walled = a[0], walled[1:]
    cells = set()
    for p in np.argwhere(a):
        for off in np.ndindex(*([3] * a.ndim)):
            c = []
            for ax in range(a.ndim):
                v = 2 * int(p[ax]) + off[ax]
                if not walled[ax]:
                    v %= 2 * a.shape[ax]
                c.append(v)
            cells.add(tuple(c))
    return sum((-1) ** sum(v & 1 for v in c) for c in cells)


def test_euler_closed_forms():
    chi = measure.euler_characteristic
    z = lambda: np.zeros((9, 10, 11))
    a = z(); a[4, 5, 6] = 1
    assert chi(a) == 1                                            # one closed cube: a ball
    a = z(); a[2:5, 3:6, 4:7] = 1; a[3, 4, 5] = 0
    assert chi(a) == 2                                            # a shell enclosing a cavity
    a = z(); a[4, 3:6, 3:6] = 1; a[4, 4, 4] = 0
    assert chi(a) == 0                                            # a ring: a solid torus
    a = z(); a[1, 1, 1] = a[2, 2, 2] = 1
    assert chi(a) == 1                                            # cubes sharing a corner: one region
    a = z(); a[1, 1, 1] = a[3, 3, 3] = 1
    assert chi(a) == 2
    a = z(); a[4, 4, :] = 1
    assert chi(a) == 0                                            # a rod closed on itself through x
    assert chi(a, walls=(True, False, False)) == 1                # the same rod cut by x walls
    assert chi(np.ones((5, 6, 7))) == 0                           # the 3-torus
    assert chi(np.ones((5, 6, 7)), walls=(False, False, True)) == 0   # slab x 2-torus
    assert chi(np.ones((5, 6, 7)), walls=(True, True, True)) == 1     # a box
    a2 = np.zeros((1, 8, 9)); a2[0, 2:5, 2:5] = 1; a2[0, 3, 3] = 0
    assert chi(a2) == 0                                           # 2D annulus
    a2 = np.zeros((1, 8, 9)); a2[0, 2, 2] = a2[0, 3, 3] = 1
    assert chi(a2) == 1                                           # 8-connected diagonal pair
    assert chi(np.ones((1, 4, 5))) == 0 and chi(np.ones((1, 4, 5)), walls=(True, True, False)) == 1


@pytest.mark.parametrize("walls", [(False, False, False), (True, False, False), (False, False, True),
                                   (True, False, True)])
@pytest.mark.parametrize("nz", [1, 5])
def test_euler_matches_cell_enumeration_on_random_sets(walls, nz):
    rng = np.random.default_rng(17 + nz)
    for density in (0.1, 0.35, 0.6):
        a = (rng.random((nz, 6, 7)) < density).astype(float)
        w = walls if nz > 1 else (walls[0], walls[1], False)
        assert measure.euler_characteristic(a, w) == _brute_chi(a, w)


@pytest.mark.parametrize("walls", [(False, False, False), (False, False, True)])
def test_euler_counts_droplets(walls):
    shape = (40, 36, 44)
    centres, radii = place_droplets(shape, 0.12, 3.0, 6.0, 3.0, seed=21, walls=walls)
    phi = phi_field(shape, centres, radii, 3.0, walls=walls).numpy()
    n = measure.count_droplets(phi, walls)
    assert n == len(radii) > 10
    assert measure.euler_characteristic(phi, walls) == n


@pytest.mark.parametrize("dims", [2, 3])
def test_droplet_stats_of_the_binding_match_the_oracle(dims):
    # the package's <R> and N from the reduction's two outputs, fed here with the oracle's
    # Euler characteristic and interface measure of a known droplet field
    from paper_2409_03401_gb300 import droplet_stats
    W = 3.0
    if dims == 3:
        shape = (40, 36, 44)
        centres, radii = place_droplets(shape, 0.1, 4.0, 7.0, W, seed=5)
    else:
        shape = (1, 96, 110)
        centres, radii = place_droplets(shape, 0.1, 4.0, 9.0, W, seed=5)
    phi = phi_field(shape, centres, radii, W).numpy()
    from paper_2409_03401_gb300 import _lib
    from workloads import configs
    params = (configs.ripening_2d if dims == 2 else configs.ripening)(shape=shape)[0]
    sums = dict.fromkeys(_lib.REDUCTIONS, 0.0)
    sums.update(euler=float(measure.euler_characteristic(phi)), interface=measure.interface_measure(phi, W))
    got = droplet_stats(params, sums)
    R, n = measure.mean_radius(phi, W)
    assert got["N"] == n == len(radii)
    assert abs(got["R_mean"] - R) < 1e-12 * R
    sums.update(euler=0.0, interface=1.0)
    assert math.isnan(droplet_stats(params, sums)["R_mean"])
