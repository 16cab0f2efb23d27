"""lbm_reduce_static, the allocation-free diagnostics, against lbm_reduce.

Some callers cannot allocate device memory when they need the sums (a host application
that owns every allocation and lends this library its state buffer, or a real-time loop
that forbids allocation after start-up). lbm_reduce_static serves them from a static
device array; its results must equal lbm_reduce's on the same state, call after call.
"""
import ctypes

import pytest
import torch

from workloads import configs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _lib():
    from paper_2409_03401_gb300 import _lib as L
    lib = L.load()
    lib.lbm_reduce_static.restype = ctypes.c_int
    lib.lbm_reduce_static.argtypes = [ctypes.POINTER(L.lbm_params), ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    return L, lib


def _static_sums(L, lib, sim):
    cp = L.make_params(sim.params)
    out = (ctypes.c_double * L.NRED)()
    st = lib.lbm_reduce_static(ctypes.byref(cp), ctypes.c_void_p(sim.state.data_ptr()), sim.t, out,
                               ctypes.c_void_p(sim.stream.cuda_stream))
    assert st == L.LBM_OK, lib.lbm_last_error(None).decode()
    return {k: out[i] for i, k in enumerate(L.REDUCTIONS)}


def _close(a, b):
    for k in a:
        assert abs(a[k] - b[k]) <= TOL * max(abs(b[k]), 1e-30), (k, a[k], b[k])


@pytest.mark.parametrize("case", ["ripening", "flow", "flow_inplace", "couple_f64"])
def test_static_reduce_matches_reduce(case):
    from paper_2409_03401_gb300 import Simulation
    L, lib = _lib()
    if case == "ripening":
        p, fields = configs.ripening(shape=(40, 48, 64))
    elif case == "couple_f64":
        p, fields = configs.diffusion_couple()
    else:
        p, fields = configs.sedimentation(shape=(32, 32, 48), fraction=0.06, r=(6.0, 9.0))
        p = p.with_(inplace=(case == "flow_inplace"))
    sim = Simulation(p, *fields())
    for steps in (3, 0, 4):            # two calls in a row at the same time level, then later
        sim.step(steps)
        ref = sim.sums()
        got = _static_sums(L, lib, sim)
        _close(got, ref)


@pytest.mark.parametrize("case", ["flow_128", "ripening_384", "couple_f64_1024"])
def test_static_reduce_rejects_lattices_beyond_the_array(case):
    # the phi field of a flow lattice (FP32), the bit field of a 3D lattice without flow
    # (384^3 > 2^25 nodes) and the FP64 phi field of a 2D lattice over half a million nodes
    L, lib = _lib()
    if case == "flow_128":
        p, _ = configs.sedimentation(n=128)
    elif case == "ripening_384":
        p, _ = configs.ripening(n=384)
    else:
        p, _ = configs.diffusion_couple(nx=1024, ny=1024, storage="f64")
    cp = L.make_params(p)
    state = torch.empty(256, dtype=torch.uint8, device="cuda")
    out = (ctypes.c_double * L.NRED)()
    st = lib.lbm_reduce_static(ctypes.byref(cp), ctypes.c_void_p(state.data_ptr()), 0, out, None)
    assert st == L.LBM_ERR_ARG
    assert b"static array" in lib.lbm_last_error(None)


def test_static_reduce_just_under_the_array_size():
    # a 2D D2Q9 lattice of 1,024,000 nodes: FP32 phi field, partials and results fill the
    # 4 MiB array to within 768 bytes
    from paper_2409_03401_gb300 import Simulation
    L, lib = _lib()
    p, fields = configs.ripening_2d(shape=(1, 1024, 1000))
    assert lib.lbm_work_bytes(ctypes.byref(L.make_params(p))) == 4 * 1024 * 1024 - 768
    sim = Simulation(p, *fields())
    for steps in (2, 0):
        sim.step(steps)
        _close(_static_sums(L, lib, sim), sim.sums())


def test_static_reduce_rejects_host_memory():
    L, lib = _lib()
    p, _ = configs.ripening(shape=(8, 8, 8))
    cp = L.make_params(p)
    host = (ctypes.c_double * 4096)()
    out = (ctypes.c_double * L.NRED)()
    st = lib.lbm_reduce_static(ctypes.byref(cp), ctypes.cast(host, ctypes.c_void_p), 0, out, None)
    assert st == L.LBM_ERR_ARG
