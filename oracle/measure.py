"""Droplet count and mean radius (§4.2.2; test infrastructure only).

* ``count_droplets`` - number of connected regions of phi >= 1/2 with
  26-connectivity (8 in 2D), periodic along axes without walls, by union-find.
  For droplets without holes or handles this equals the Euler characteristic
  the paper measures.
* ``euler_characteristic`` - the Euler characteristic the paper uses as its
  droplet count (§4.2.2), from its definition: the alternating count of the
  cells of the cubical complex that the closed unit squares (2D) or cubes (3D)
  centred on the nodes with phi >= 1/2 make up. Closed cells touching at a
  corner share it, so the connectivity is 8 (2D) or 26 (3D), as above.
* ``interface_measure`` - Eq. 67's integrand: sum over nodes of
  (4/W) phi (1 - phi), which approximates the total interface length (2D) or
  area (3D), since the tanh profile integrates to one across the interface.
* ``mean_radius`` - <R> = A / (2 pi N) in 2D (Eq. 67) and the 3D analogue
  sqrt(A / (4 pi N)) (sum of sphere areas 4 pi R^2; exact for equal radii).
"""
import itertools
import math
import numpy as np


def _find(parent, i):
    while parent[i] != i:
        parent[i] = parent[parent[i]]
        i = parent[i]
    return i


def count_droplets(phi, walls=(False, False, False)):
    """Connected components of phi >= 1/2; ``phi`` has shape (nz, ny, nx)."""
    a = np.asarray(phi) >= 0.5
    nz, ny, nx = a.shape
    idx = -np.ones(a.shape, dtype=np.int64)
    pts = np.argwhere(a)
    idx[a] = np.arange(len(pts))
    parent = list(range(len(pts)))
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dz, dy, dx) > (0, 0, 0) and not (nz == 1 and dz != 0)]
    for n, (z, y, x) in enumerate(pts):
        for dz, dy, dx in offs:
            zz, yy, xx = z + dz, y + dy, x + dx
            if walls[2] and not 0 <= zz < nz:
                continue
            if walls[1] and not 0 <= yy < ny:
                continue
            if walls[0] and not 0 <= xx < nx:
                continue
            j = idx[zz % nz, yy % ny, xx % nx]
            if j >= 0:
                ri, rj = _find(parent, n), _find(parent, j)
                if ri != rj:
                    parent[ri] = rj
    return len({_find(parent, i) for i in range(len(pts))})


def euler_characteristic(phi, walls=(False, False, False)):
    """chi = sum over cell dimensions d of (-1)^d (number of d-cells) of the complex made of
    the closed unit cells centred on the nodes with phi >= 1/2; ``phi`` has shape
    (nz, ny, nx), nz == 1 meaning a 2D lattice. ``walls`` per axis (x, y, z): outside a wall
    is empty, other axes wrap around.

    A cell of the complex has a type t (one flag per axis): t_i = 1 when the cell spans a
    node's unit interval along axis i, t_i = 0 when it lies on the boundary plane between
    nodes p_i - 1 and p_i. It belongs to the union when any node it bounds is set, i.e. the
    OR over the two nodes along every axis with t_i = 0; its dimension is the sum of t.
    Along a walled axis the boundary positions run 0..n (one more than the nodes).
    """
    a = np.asarray(phi) >= 0.5
    walled = [walls[2], walls[1], walls[0]]          # array axes are (z, y, x)
    if a.shape[0] == 1:
        a, walled = a[0], walled[1:]
    chi = 0
    for t in itertools.product((0, 1), repeat=a.ndim):
        cells = a
        for ax, ti in enumerate(t):
            if ti == 1:
                continue
            if walled[ax]:
                pad = [(0, 0)] * a.ndim
                pad[ax] = (1, 1)
                c = np.pad(cells, pad)
                lo = [slice(None)] * a.ndim
                hi = [slice(None)] * a.ndim
                lo[ax], hi[ax] = slice(0, -1), slice(1, None)
                cells = c[tuple(lo)] | c[tuple(hi)]
            else:
                cells = cells | np.roll(cells, 1, axis=ax)
        chi += (-1) ** sum(t) * int(np.count_nonzero(cells))
    return chi


def interface_measure(phi, W):
    phi = np.asarray(phi, dtype=np.float64)
    return float((4.0 / W * phi * (1.0 - phi)).sum())


def mean_radius(phi, W, walls=(False, False, False)):
    """(<R>, N) from Eq. 67 (2D) or its 3D analogue."""
    phi = np.asarray(phi, dtype=np.float64)
    n = count_droplets(phi, walls)
    if n == 0:
        return 0.0, 0
    A = interface_measure(phi, W)
    if phi.shape[0] == 1:
        return A / (2.0 * math.pi * n), n
    return math.sqrt(A / (4.0 * math.pi * n)), n
