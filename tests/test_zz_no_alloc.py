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


def test_static_reduce_rejects_large_flow_lattice():
    L, lib = _lib()
    p, _ = configs.sedimentation(n=128)
    cp = L.make_params(p)
    state = torch.empty(256, dtype=torch.uint8, device="cuda")
    out = (ctypes.c_double * L.NRED)()
    st = lib.lbm_reduce_static(ctypes.byref(cp), ctypes.c_void_p(state.data_ptr()), 0, out, None)
    assert st == L.LBM_ERR_ARG
    assert b"static array" in lib.lbm_last_error(None)
