"""Seeded synthetic droplet fields shaped like the paper's ripening runs (§4.2.1).

Recipe (input generation only, shared by the oracle tests and the CUDA path):

* ``place_droplets`` - random sequential addition driven by SplitMix64: a
  centre uniform in the box and a radius uniform in [r_min, r_max] (or, with
  ``sample_volume``, a disc area / sphere volume uniform between those of
  r_min and r_max, as the paper samples droplet volumes, §4.2.1); a
  candidate is rejected when it comes closer than r_i + r_j + W to a previous
  droplet (minimum-image distance along periodic axes) or, along a walled axis,
  when its surface comes closer than W/2 to the wall plane (walls at -1/2 and
  n - 1/2). Placement stops once the summed sphere volumes (disc areas in 2D)
  reach the target fraction of the box.
* ``phi_field`` - each droplet carries the equilibrium tanh profile of §2.2,
  phi = (1 + tanh(2 (r - d) / W)) / 2 with d the (minimum-image) distance to
  its centre; a node takes the largest value over droplets, i.e. the profile of
  the closest droplet surface. Each droplet is evaluated within r + 5 W of its
  centre (the profile there is below 2.1e-9) and nodes beyond every cut-off
  hold 0.
* ``composition_fields`` - the piecewise initial composition of Eq. 66: the
  droplet equilibrium composition where phi >= 1/2, the matrix composition
  (1 - delta) c_0^eq + delta c_1^eq elsewhere.
"""
import math
import numpy as np
import torch

from .rng import SplitMix64


def place_droplets(shape, fraction, r_min, r_max, W, seed, walls=(False, False, False),
                   max_attempts=1_000_000, sample_volume=False):
    """Return (centres [N, 3] as (x, y, z), radii [N]) as float64 numpy arrays.

    ``shape`` is (nz, ny, nx); ``walls`` flags the (x, y, z) axes bounded by
    walls. For nz == 1 the droplets are discs in the z = 0 plane. Previous
    droplets are looked up in a grid of cells no smaller than the largest
    exclusion distance, which gives the same accept/reject sequence as testing
    every previous droplet.
    """
    nz, ny, nx = shape
    ext = np.array([nx, ny, nz], dtype=np.float64)
    two_d = nz == 1
    dims = 2 if two_d else 3
    box = nx * ny * (1 if two_d else nz)
    rng = SplitMix64(seed)
    reach = 2.0 * r_max + W                                  # largest r_i + r_j + W
    ncell = [max(1, int(ext[ax] // reach)) for ax in range(3)]
    if two_d:
        ncell[2] = 1
    csize = [ext[ax] / ncell[ax] for ax in range(3)]
    cells = {}
    centres, radii = [], []
    covered = 0.0
    attempts = 0
    while covered < fraction * box:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError(
                f"droplet placement gave up after {max_attempts} attempts at fraction "
                f"{covered / box:.4f} < {fraction}")
        c = (rng.uniform() * nx, rng.uniform() * ny, 0.0 if two_d else rng.uniform() * nz)
        if sample_volume:                                    # disc area (2D) or sphere volume
            if two_d:
                r = math.sqrt(rng.uniform_range(r_min * r_min, r_max * r_max))
            else:
                r = rng.uniform_range(r_min ** 3, r_max ** 3) ** (1.0 / 3.0)
        else:
            r = rng.uniform_range(r_min, r_max)
        ok = True
        for ax in range(dims):
            if walls[ax]:
                if (c[ax] + 0.5) - r < W / 2 or (ext[ax] - 0.5 - c[ax]) - r < W / 2:
                    ok = False
        if not ok:
            continue
        home = [min(int(c[ax] / csize[ax]), ncell[ax] - 1) for ax in range(3)]
        rng_ax = []
        for ax in range(3):
            if ncell[ax] == 1:
                rng_ax.append((0,))
            elif walls[ax] or (two_d and ax == 2):
                rng_ax.append(tuple(i for i in (home[ax] - 1, home[ax], home[ax] + 1) if 0 <= i < ncell[ax]))
            else:
                rng_ax.append(tuple(sorted({(home[ax] + d) % ncell[ax] for d in (-1, 0, 1)})))
        for ix in rng_ax[0]:
            for iy in rng_ax[1]:
                for iz in rng_ax[2]:
                    for j in cells.get((ix, iy, iz), ()):
                        d2 = 0.0
                        for ax in range(dims):
                            d = centres[j][ax] - c[ax]
                            if not walls[ax]:
                                d -= ext[ax] * round(d / ext[ax])
                            d2 += d * d
                        if d2 < (radii[j] + r + W) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        cells.setdefault(tuple(home), []).append(len(radii))
        centres.append(c)
        radii.append(r)
        covered += math.pi * r * r if two_d else 4.0 / 3.0 * math.pi * r ** 3
    return np.array(centres, dtype=np.float64).reshape(-1, 3), np.array(radii, dtype=np.float64)


def _axis_points(c, R, n, periodic, device):
    """Node indices within R of coordinate c along one axis, and their signed offsets."""
    if periodic:
        if 2 * R + 1 >= n:
            idx = torch.arange(n, device=device, dtype=torch.int64)
        else:
            idx = torch.arange(math.floor(c - R), math.ceil(c + R) + 1, device=device,
                               dtype=torch.int64) % n
        d = idx.to(torch.float64) - c
        d = d - n * torch.round(d / n)
    else:
        lo = max(0, math.floor(c - R))
        hi = min(n - 1, math.ceil(c + R))
        idx = torch.arange(lo, hi + 1, device=device, dtype=torch.int64)
        d = idx.to(torch.float64) - c
    return idx, d


def phi_field(shape, centres, radii, W, walls=(False, False, False), device="cpu",
              dtype=torch.float64, cutoff_widths=5.0, z_range=None):
    """Droplet phase field of shape (nz, ny, nx) (see the module docstring).

    ``z_range=(z0, z1)`` returns only the planes z0 <= z < z1 of that field.
    """
    nz, ny, nx = shape
    z0, z1 = z_range if z_range is not None else (0, nz)
    phi = torch.zeros((z1 - z0, ny, nx), dtype=torch.float64, device=device)
    for (cx, cy, cz), r in zip(np.asarray(centres), np.asarray(radii)):
        R = float(r) + cutoff_widths * W
        ix, dx = _axis_points(float(cx), R, nx, not walls[0], device)
        iy, dy = _axis_points(float(cy), R, ny, not walls[1], device)
        if nz == 1:
            iz = torch.zeros(1, dtype=torch.int64, device=device)
            dz = torch.zeros(1, dtype=torch.float64, device=device)
        else:
            iz, dz = _axis_points(float(cz), R, nz, not walls[2], device)
        keep = (iz >= z0) & (iz < z1)
        if not bool(keep.any()):
            continue
        iz, dz = iz[keep] - z0, dz[keep]
        dist = torch.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        prof = 0.5 * (1.0 + torch.tanh(2.0 * (float(r) - dist) / W))
        sel = (iz[:, None, None], iy[None, :, None], ix[None, None, :])
        phi[sel] = torch.maximum(phi[sel], prof)
    return phi.to(dtype)


def composition_fields(phi, c_eq, delta):
    """Eq. 66: c^alpha = c_1^eq in droplets (phi >= 1/2), (1-delta) c_0^eq + delta c_1^eq outside."""
    out = []
    for a in range(2):
        c_mat = (1.0 - delta) * c_eq[0][a] + delta * c_eq[1][a]
        out.append(torch.where(phi >= 0.5, torch.full_like(phi, c_eq[1][a]),
                               torch.full_like(phi, c_mat)))
    return out[0], out[1]


def planar_couple(shape, x_interface, W, c_left, c_right, device="cpu", dtype=torch.float64):
    """Diffusion-couple start (§4.1): phase 1 on the left of x_interface, phase 0 on the right.

    phi = (1 - tanh(2 (x - x_interface) / W)) / 2; compositions are step
    functions, c_left where phi >= 1/2 and c_right elsewhere.
    """
    nz, ny, nx = shape
    x = torch.arange(nx, dtype=torch.float64, device=device)
    prof = 0.5 * (1.0 - torch.tanh(2.0 * (x - x_interface) / W))
    phi = prof.expand(nz, ny, nx).clone()
    cA = torch.where(phi >= 0.5, torch.full_like(phi, c_left[0]), torch.full_like(phi, c_right[0]))
    cB = torch.where(phi >= 0.5, torch.full_like(phi, c_left[1]), torch.full_like(phi, c_right[1]))
    return phi.to(dtype), cA.to(dtype), cB.to(dtype)
