"""ctypes binding of liblbm_gb300.so: the C-ABI of include/lbm.h, same names.

Argument marshalling only. Loading fails loudly when the library is missing:
there is no CPU fallback anywhere in this package.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_STATE = 0, -1, -2, -3, -4
LBM_D2Q5, LBM_D3Q7, LBM_D3Q19, LBM_D2Q9 = 0, 1, 2, 3
LBM_F64, LBM_F32, LBM_F16, LBM_BF16 = 0, 1, 2, 3
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}
LATTICE = {"D2Q5": LBM_D2Q5, "D3Q7": LBM_D3Q7, "D3Q19": LBM_D3Q19, "D2Q9": LBM_D2Q9}
LBM_BGK, LBM_TRT, LBM_MRT = 0, 1, 2
COLLISION = {"BGK": LBM_BGK, "TRT": LBM_TRT, "MRT": LBM_MRT}
FIELDS = ("phi", "muA", "muB", "cA", "cB", "p", "ux", "uy", "uz", "S")
REDUCTIONS = ("phi", "cA", "cB", "p", "S", "umax", "g", "nonfinite", "interface", "euler")
NFIELDS = len(FIELDS)
NRED = len(REDUCTIONS)


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("lattice", ctypes.c_int32), ("flow", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("wall_x", ctypes.c_int32), ("wall_z", ctypes.c_int32), ("source_off", ctypes.c_int32),
        ("inplace", ctypes.c_int32),
        ("W", ctypes.c_double), ("lambda_", ctypes.c_double), ("M_phi", ctypes.c_double),
        ("c_eq", (ctypes.c_double * 2) * 2), ("M", (ctypes.c_double * 2) * 2),
        ("nu", ctypes.c_double), ("sigma", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("f_scale", ctypes.c_double),
        ("collision", ctypes.c_int32), ("trt_magic", ctypes.c_double), ("mrt_rates", ctypes.c_double * 5),
    ]


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"lbm status {status}: {message}")
        self.status = status


_lib = None


def load():
    """Load liblbm_gb300.so (built by paper_2409_03401_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                          "g.build()\"` (nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(lbm_params)
    vp = ctypes.c_void_p
    ctx_pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "lbm_state_bytes": (ctypes.c_size_t, [P]),
        "lbm_work_bytes": (ctypes.c_size_t, [P]),
        "lbm_init": (ctypes.c_int, [P, vp, vp, vp, vp, vp, vp, ctx_pp]),
        "lbm_attach": (ctypes.c_int, [P, vp, vp, ctypes.c_int64, vp, ctx_pp]),
        "lbm_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_step_graph": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_time": (ctypes.c_int64, [vp]),
        "lbm_fields": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_void_p)]),
        "lbm_reduce": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
        "lbm_destroy": (ctypes.c_int, [vp]),
        "lbm_profile_begin": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_profile_end": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
        "lbm_kernels_per_step": (ctypes.c_int, [vp]),
        "lbm_copy_bytes": (ctypes.c_size_t, [P]),
        "lbm_step_buffers": (ctypes.c_int, [P, vp, vp, ctypes.c_int64, vp, vp]),
        "lbm_adjoint_bytes": (ctypes.c_size_t, [P]),
        "lbm_adjoint_work_bytes": (ctypes.c_size_t, [P]),
        "lbm_adjoint_reset": (ctypes.c_int, [P, vp, vp]),
        "lbm_adjoint_seed": (ctypes.c_int, [P, vp, ctypes.c_int64, vp, vp, vp, vp, vp, vp]),
        "lbm_adjoint_step": (ctypes.c_int, [P, vp, ctypes.c_int64, vp, vp, vp, vp]),
        "lbm_adjoint_segment": (ctypes.c_int, [P, vp, ctypes.c_int64, ctypes.c_int, vp, vp, vp, vp, vp,
                                                ctypes.POINTER(ctypes.c_int)]),
        "lbm_adjoint_init": (ctypes.c_int, [P, vp, vp, vp, vp, vp, vp, vp]),
        "lbm_adjoint_theta": (ctypes.c_int, [P, vp, ctypes.POINTER(ctypes.c_double), vp]),
        "lbm_reduce_static": (ctypes.c_int, [P, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), vp]),
        "lbm_slab_planes": (ctypes.c_int32, [P, ctypes.c_int32, ctypes.c_int32]),
        "lbm_slab_state_bytes": (ctypes.c_size_t, [P, ctypes.c_int32, ctypes.c_int32]),
        "lbm_slab_work_bytes": (ctypes.c_size_t, [P, ctypes.c_int32, ctypes.c_int32]),
        "lbm_slab_init": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, vp, ctx_pp]),
        "lbm_slab_ghosts": (ctypes.c_int32, [vp]),
        "lbm_slab_halo_bytes": (ctypes.c_size_t, [vp]),
        "lbm_slab_phi_bytes": (ctypes.c_size_t, [vp]),
        "lbm_slab_pack": (ctypes.c_int, [vp, ctypes.c_int32, vp]),
        "lbm_slab_unpack": (ctypes.c_int, [vp, ctypes.c_int32, vp]),
        "lbm_slab_phi_pack": (ctypes.c_int, [vp, ctypes.c_int32, vp]),
        "lbm_slab_phi_unpack": (ctypes.c_int, [vp, ctypes.c_int32, vp]),
        "lbm_mean_radius": (ctypes.c_double, [P, ctypes.POINTER(ctypes.c_double)]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_build_info": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C-ABI entry points this binding expects."""
    return ["lbm_state_bytes", "lbm_work_bytes", "lbm_init", "lbm_attach", "lbm_step", "lbm_step_graph", "lbm_time",
            "lbm_fields", "lbm_reduce", "lbm_profile_begin", "lbm_profile_end", "lbm_kernels_per_step",
            "lbm_copy_bytes", "lbm_step_buffers", "lbm_adjoint_bytes", "lbm_adjoint_work_bytes",
            "lbm_adjoint_reset", "lbm_adjoint_seed", "lbm_adjoint_step", "lbm_adjoint_segment", "lbm_adjoint_init",
            "lbm_adjoint_theta", "lbm_reduce_static", "lbm_slab_planes", "lbm_slab_state_bytes",
            "lbm_slab_work_bytes", "lbm_slab_init", "lbm_slab_ghosts", "lbm_slab_halo_bytes", "lbm_slab_phi_bytes",
            "lbm_slab_pack", "lbm_slab_unpack", "lbm_slab_phi_pack", "lbm_slab_phi_unpack", "lbm_mean_radius",
            "lbm_destroy",
            "lbm_last_error", "lbm_build_info"]


def check(status, ctx=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(ctx).decode()
        raise LBMError(status, msg)


def make_params(p):
    """Pack a workloads.LBMParams into the C struct."""
    c = lbm_params()
    c.nx, c.ny, c.nz = p.nx, p.ny, p.nz
    c.lattice = LATTICE[p.lattice]
    c.flow = int(p.flow)
    c.storage = STORAGE[p.storage]
    c.wall_x, c.wall_z = int(p.wall_x), int(p.wall_z)
    c.source_off = int(p.source_off)
    c.inplace = int(getattr(p, "inplace", False))
    c.W, c.lambda_, c.M_phi = p.W, p.lam, p.M_phi
    for i in range(2):
        for a in range(2):
            c.c_eq[i][a] = p.c_eq[i][a]
            c.M[i][a] = p.M[i][a]
    c.nu, c.sigma = p.nu, p.sigma
    for i in range(3):
        c.g[i] = p.g[i]
    c.f_scale = p.f_scale
    c.collision = COLLISION[p.collision]
    c.trt_magic = p.trt_magic
    for i, r in enumerate(p.mrt_rates):
        c.mrt_rates[i] = r
    return c
