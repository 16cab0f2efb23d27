"""The six synthetic workloads of the coupled step, in lattice units.

Each builder returns ``(params, fields)`` where ``fields(device)`` yields the
initial (phi, c^A, c^B) as float64 tensors of shape (nz, ny, nx). Sizes can be
shrunk (``shape=``) for tests while keeping the same physics and statistics.

Parameter choices where the paper or the workload description is silent:

* The 3D ripening set (§4.2.4 table): c_0^eq = (0.3, 0.3), c_1^eq = (0.4, 0.4),
  lambda = 155.95, W = 3 nodes. Mobility ratios M^A : M^B : M_phi = 1 : 0.8 :
  1.2 as in that table, scaled to the lattice as M^A = 0.1, M^B = 0.08,
  M_phi = 0.12 (the lambda that cancels the kinetic coefficient, Eq. 27, is
  unchanged by a common scale). Matrix supersaturated by 2% of the gap
  (delta = 0.02 in Eq. 66).
* Flow: nu = 0.1, sigma = 1e-3, buoyancy 1e-5 along -z, walls at the z ends.
* Diffusion couple (§4.1 geometry, composition set of the 2D couple workload):
  phase 1 on the left with c = (0.55, 0.15), phase 0 on the right with
  c = (0.15, 0.25); c_1^eq = (0.6, 0.1), c_0^eq = (0.1, 0.3); D_1 = 1.0,
  D_0 = 0.5 for both components; no-flux walls at the x ends. M_phi = 0.12
  (the lattice value of the 3D sets): the explicit source relaxes phi at the
  bulk values with rate 16 M_phi / W^2 per step, which must stay well below 2,
  and the paper's ratio M_phi = 1.2 D_1 would give 2.13. lambda = 60: a bulk
  phase stays linearly stable only while 6 lambda |Delta omega| < 16 (|Delta
  omega| = 0.035 at the start), which rules out the lambda = 90.7 that would
  cancel the kinetic coefficient of Eq. 27 at this M_phi; at lambda = 60 the
  kinetic coefficient is 0.094 and the interface follows x_I ~ sqrt(t).
"""
import math

from .params import LBMParams
from .droplets import place_droplets, phi_field, composition_fields, planar_couple

LAMBDA_COUPLE = 60.0
M_PHI_COUPLE = 0.12
# matrix composition c_0^eq + delta (c_1^eq - c_0^eq) of the 3D workloads (the 2D workload
# takes the 2D table's delta = 0.1; the paper's 3D table has delta = 0.2)
SUPERSATURATION = 0.02


def diffusion_couple(nx=512, ny=8, storage="f64"):
    p = LBMParams(nx=nx, ny=ny, nz=1, lattice="D2Q5", flow=False, storage=storage,
                  wall_x=True, W=3.0, lam=LAMBDA_COUPLE, M_phi=M_PHI_COUPLE,
                  c_eq=((0.1, 0.3), (0.6, 0.1)), M=((0.5, 0.5), (1.0, 1.0)))
    x_i = nx / 2 - 0.5

    def fields(device="cpu"):
        return planar_couple(p.shape, x_i, p.W, (0.55, 0.15), (0.15, 0.25), device=device)
    return p, fields


def _droplet_workload(p, fraction, r_min, r_max, seed, sample_volume=False, supersaturation=SUPERSATURATION):
    walls = (p.wall_x, False, p.wall_z)
    cache = {}

    def geometry():
        if "g" not in cache:
            cache["g"] = place_droplets(p.shape, fraction, r_min, r_max, p.W, seed, walls=walls,
                                        sample_volume=sample_volume)
        return cache["g"]

    def fields(device="cpu", z_range=None):
        centres, radii = geometry()
        phi = phi_field(p.shape, centres, radii, p.W, walls=walls, device=device, z_range=z_range)
        cA, cB = composition_fields(phi, p.c_eq, supersaturation)
        return phi, cA, cB
    fields.geometry = geometry
    return fields


def ripening(n=256, storage="f32", shape=None, seed=2, supersaturation=SUPERSATURATION):
    """3D Ostwald ripening without flow, periodic, spheres at fraction 0.15, r in [4, 10]."""
    nz, ny, nx = shape or (n, n, n)
    p = LBMParams(nx=nx, ny=ny, nz=nz, lattice="D3Q7", flow=False, storage=storage)
    return p, _droplet_workload(p, 0.15, 4.0, 10.0, seed, supersaturation=supersaturation)


def sedimentation(n=512, storage="f32", shape=None, seed=3, fraction=0.2, r=(6.0, 16.0),
                  supersaturation=SUPERSATURATION):
    """3D coarsening with flow and buoyancy, walls at the z ends."""
    nz, ny, nx = shape or (n, n, n)
    p = LBMParams(nx=nx, ny=ny, nz=nz, lattice="D3Q7", flow=True, storage=storage, wall_z=True)
    return p, _droplet_workload(p, fraction, r[0], r[1], seed, supersaturation=supersaturation)


# 2D ripening without flow (§4.2.2 table, D2Q9): the table's collision times tau_g = 0.8776,
# tau_h^A = 0.8146, tau_h^B = 0.7517 are classic BGK times, so M = (tau - 1/2) c_s^2 with
# c_s^2 = 1/3; the matrix composition c_g = 0.31 is 10 % of the gap above c_0^eq; droplet
# areas uniform in (1.02 +- 0.957) x 10^-4 L^2 at dx = 4.882 x 10^-4 L, i.e. 26.5 to 829.5
# nodes^2 (radii 2.90 to 16.25 nodes), at phase fraction 0.08.
RIPENING_2D_M = ((0.8146 - 0.5) / 3.0, (0.7517 - 0.5) / 3.0)
RIPENING_2D_M_PHI = (0.8776 - 0.5) / 3.0
RIPENING_2D_R = (math.sqrt(26.5 / math.pi), math.sqrt(829.5 / math.pi))


def ripening_2d(n=4096, storage="f32", shape=None, seed=6, r_max=RIPENING_2D_R[1]):
    """2D Ostwald ripening without flow, periodic, on D2Q9 (the paper's 4096^2 run). ``r_max``
    caps the droplet radii (smaller boxes hold more, smaller droplets)."""
    nz, ny, nx = shape or (1, n, n)
    p = LBMParams(nx=nx, ny=ny, nz=nz, lattice="D2Q9", flow=False, storage=storage, W=3.0, lam=155.95,
                  M_phi=RIPENING_2D_M_PHI, c_eq=((0.3, 0.3), (0.4, 0.4)),
                  M=(RIPENING_2D_M, RIPENING_2D_M))
    return p, _droplet_workload(p, 0.08, RIPENING_2D_R[0], r_max, seed, sample_volume=True,
                                supersaturation=0.1)


def drift(n=384, storage="f32", shape=None, seed=4):
    """Same physics as ``sedimentation`` at fraction 0.1, r in [8, 20] (long-run drift study)."""
    return sedimentation(n=n, storage=storage, shape=shape, seed=seed, fraction=0.1, r=(8.0, 20.0))


# adjoint workload: target generated at THETA_TARGET, gradient evaluated at THETA_EVAL,
# theta = (D_0, D_1, M_phi) with D_pi the diffusivity of phase pi for both components
THETA_TARGET = (0.4, 0.8, 0.05)
THETA_EVAL = (0.5, 0.7, 0.06)


def with_theta(p, theta):
    d0, d1, mphi = theta
    return p.with_(M=((d0, d0), (d1, d1)), M_phi=mphi)


def adjoint_problem(n=128, storage="f32", shape=None, seed=5, theta=THETA_EVAL, supersaturation=SUPERSATURATION):
    nz, ny, nx = shape or (n, n, n)
    p = with_theta(LBMParams(nx=nx, ny=ny, nz=nz, lattice="D3Q7", flow=False, storage=storage), theta)
    return p, _droplet_workload(p, 0.15, 4.0, 10.0, seed, supersaturation=supersaturation)


CONFIGS = {
    "couple": diffusion_couple,
    "ripening": ripening,
    "ripening_2d": ripening_2d,
    "sedimentation": sedimentation,
    "drift": drift,
    "adjoint": adjoint_problem,
}

