"""Plain parameter container for one lattice, in lattice units (dx = dt = 1, rho0 = 1).

Values only: no formula of the method lives here. The CUDA binding packs these
fields into the C struct ``lbm_params``; the FP64 oracle reads them directly.

Symbols follow the paper (Tables of §4): W interface width, lam the coupling
constant lambda, M_phi the scaled phase-field mobility, c_eq[pi][alpha] the
equilibrium compositions of phase pi in {0, 1} for component alpha in {A, B},
M[pi][alpha] the scaled species mobility of component alpha in phase pi (the
diffusivity of the bulk phase, §2.3), nu the kinematic viscosity, sigma the
surface tension, g the buoyancy acceleration times the density contrast
(F_g = phi * g, §2.5). collision selects the flow collision operator: the paper's BGK,
or the two- and multiple-relaxation-time operators it names as alternatives (§3).
"""
from dataclasses import dataclass, field, asdict, replace
from typing import Tuple

LATTICES = ("D2Q5", "D3Q7", "D3Q19", "D2Q9")
COLLISIONS = ("BGK", "TRT", "MRT")
STORAGES = ("f64", "f32", "f16", "bf16")


@dataclass(frozen=True)
class LBMParams:
    nx: int
    ny: int
    nz: int
    lattice: str = "D3Q7"          # lattice of the phi, c^A, c^B equations (D3Q19: the paper's choice)
    flow: bool = False             # D3Q19 flow populations with capillary + buoyancy forcing
    storage: str = "f32"           # population storage type on the GPU (oracle is always FP64)
    wall_x: bool = False           # half-way bounce-back planes at x = -1/2 and x = nx - 1/2
    wall_z: bool = False           # half-way bounce-back planes at z = -1/2 and z = nz - 1/2
    source_off: bool = False       # test switch: drop the phase-field source (pure advection-diffusion)
    inplace: bool = False          # flow on the GPU: one in-place AA copy + phi pass instead of two copies
    W: float = 3.0
    lam: float = 155.95
    M_phi: float = 0.12
    c_eq: Tuple[Tuple[float, float], Tuple[float, float]] = ((0.3, 0.3), (0.4, 0.4))
    M: Tuple[Tuple[float, float], Tuple[float, float]] = ((0.1, 0.08), (0.1, 0.08))
    nu: float = 0.1
    sigma: float = 1.0e-3
    g: Tuple[float, float, float] = (0.0, 0.0, -1.0e-5)
    f_scale: float = 1024.0        # reserved field of lbm_params (the 16-bit formats have fixed scales)
    collision: str = "BGK"         # flow collision: "BGK" (one rate), "TRT" (two) or "MRT"
    trt_magic: float = 3.0 / 16.0  # TRT: Lambda = (1/omega+ - 1/2)(1/omega- - 1/2)
    # MRT rates of the energy, energy-square, energy-flux, pi and m moments (d'Humieres 2002)
    mrt_rates: Tuple[float, float, float, float, float] = (1.19, 1.4, 1.2, 1.4, 1.98)

    def __post_init__(self):
        if self.lattice not in LATTICES:
            raise ValueError(f"lattice must be one of {LATTICES}")
        if self.storage not in STORAGES:
            raise ValueError(f"storage must be one of {STORAGES}")
        if min(self.nx, self.ny, self.nz) < 1:
            raise ValueError("lattice extents must be >= 1")
        if self.lattice in ("D2Q5", "D2Q9") and self.nz != 1:
            raise ValueError("the 2D lattices need nz == 1")
        if self.collision not in COLLISIONS:
            raise ValueError(f"collision must be one of {COLLISIONS}")
        if not self.trt_magic > 0:
            raise ValueError("trt_magic must be > 0")
        if len(self.mrt_rates) != 5 or not all(0 < r < 2 for r in self.mrt_rates):
            raise ValueError("mrt_rates: five rates in (0, 2)")
        if self.flow and self.lattice in ("D2Q5", "D2Q9"):
            raise ValueError("flow is implemented on 3D lattices (D3Q19 flow + D3Q7 or D3Q19 scalars)")

    @property
    def shape(self):
        """Array shape of one field, slowest axis first: (nz, ny, nx)."""
        return (self.nz, self.ny, self.nx)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def with_(self, **kw) -> "LBMParams":
        return replace(self, **kw)

    def as_dict(self):
        return asdict(self)
