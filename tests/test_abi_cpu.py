"""The C-ABI library loads and exports every entry point of include/lbm.h (no GPU needed),
and its host-side validation and sizing work without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_03401_gb300 import build as pkg_build
    pkg_build()
    from paper_2409_03401_gb300 import _lib
    return _lib.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "lbm_init" in names and "lbm_step" in names and "lbm_fields" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    from paper_2409_03401_gb300 import _lib
    assert set(_lib.exported_symbols()) <= names


def test_sizes_and_validation_on_the_host(lib):
    from paper_2409_03401_gb300 import _lib
    from workloads import configs
    p, _ = configs.sedimentation(n=512)
    cp = _lib.make_params(p)
    n = 512 ** 3
    state = lib.lbm_state_bytes(ctypes.byref(cp))
    assert state == 2 * 40 * 4 * n                     # two copies of 19 + 3 x 7 FP32 planes
    inplace = lib.lbm_state_bytes(ctypes.byref(_lib.make_params(p.with_(inplace=True))))
    assert inplace == 40 * 4 * n                       # one in-place AA copy
    p16 = p.with_(storage="f16")
    s16 = lib.lbm_state_bytes(ctypes.byref(_lib.make_params(p16)))
    assert s16 == 2 * (40 * 2 * n + 5 * 4 * n)         # 16-bit planes + 5 FP32 rest planes, two copies
    noflow = lib.lbm_state_bytes(ctypes.byref(_lib.make_params(p.with_(flow=False))))
    assert noflow == 21 * 4 * n                        # scalars only: always one in-place copy
    assert lib.lbm_state_bytes(ctypes.byref(_lib.make_params(p.with_(nx=2048, ny=1024, nz=1024)))) == 0
    bad = _lib.make_params(p.with_(nz=70000))
    assert lib.lbm_state_bytes(ctypes.byref(bad)) == 0
    ctx = ctypes.c_void_p()
    st = lib.lbm_init(ctypes.byref(bad), ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(8),
                      ctypes.c_void_p(8), ctypes.c_void_p(8), None, ctypes.byref(ctx))
    assert st == _lib.LBM_ERR_ARG and not ctx.value
    assert b"65535" in lib.lbm_last_error(None)
    st = lib.lbm_init(ctypes.byref(cp), ctypes.c_void_p(258), ctypes.c_void_p(256), ctypes.c_void_p(8),
                      ctypes.c_void_p(8), ctypes.c_void_p(8), None, ctypes.byref(ctx))
    assert st == _lib.LBM_ERR_ARG and b"aligned" in lib.lbm_last_error(None)
    assert lib.lbm_step(None, 1) == _lib.LBM_ERR_ARG
    assert lib.lbm_time(None) == -1
    # collision operator: TRT keeps the state size; an unknown operator or a negative
    # magic parameter is rejected before any device work
    trt = _lib.make_params(p.with_(collision="TRT"))
    assert lib.lbm_state_bytes(ctypes.byref(trt)) == state
    for field, value in (("collision", 3), ("trt_magic", -1.0), ("mrt_rates", 2.5)):
        badc = _lib.make_params(p.with_(collision="TRT"))
        if field == "mrt_rates":
            badc.mrt_rates[2] = value
        else:
            setattr(badc, field, value)
        assert lib.lbm_state_bytes(ctypes.byref(badc)) == 0
        st = lib.lbm_init(ctypes.byref(badc), ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(8),
                          ctypes.c_void_p(8), ctypes.c_void_p(8), None, ctypes.byref(ctx))
        assert st == _lib.LBM_ERR_ARG
        assert field.encode() in lib.lbm_last_error(None)


def test_header_is_plain_c99(tmp_path):
    # the boundary is a C ABI: the header, and a C caller of it, compile as C99 with warnings
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    cuda_inc = "/usr/local/cuda/include"
    out = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                          "-I", cuda_inc, "-c", os.path.join(ROOT, "tests", "c_abi_example.c"),
                          "-o", str(tmp_path / "c_abi_example.o")], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr


def test_python_binding_checks_buffers_before_any_device_call(lib):
    # wrong-sized inputs would be read out of bounds by the kernels: the binding refuses them
    import torch
    from paper_2409_03401_gb300 import Simulation
    from workloads import configs
    p, fields = configs.ripening(shape=(8, 9, 10))
    phi, cA, cB = fields()
    with pytest.raises(ValueError, match="phi0 has"):
        Simulation(p, phi[:4], cA, cB, device="cuda:0")
    with pytest.raises(ValueError, match="cB0 has"):
        Simulation(p, phi, cA, cB.reshape(-1)[:-1], device="cuda:0")
    with pytest.raises(ValueError, match="CUDA device"):
        Simulation(p, phi, cA, cB, device="cpu")
    from paper_2409_03401_gb300 import _lib
    need = lib.lbm_state_bytes(ctypes.byref(_lib.make_params(p)))
    with pytest.raises(ValueError, match="at least"):
        Simulation.attach(p, torch.empty(need - 1, dtype=torch.uint8), 0)
    with pytest.raises(ValueError, match="at least"):
        Simulation.attach(p, torch.empty(need // 4, dtype=torch.float32), 0)
    with pytest.raises(ValueError, match="CUDA device"):
        Simulation.attach(p, torch.empty(need, dtype=torch.uint8), 0)


def test_adjoint_wrapper_rejects_bad_arguments_up_front(lib):
    # checked before the forward run: K = 0 would never advance the checkpoint loop
    import torch
    from paper_2409_03401_gb300.adjoint import CoupledRun
    from workloads import configs
    p, fields = configs.ripening(shape=(8, 9, 10))
    phi, cA, cB = fields()
    th = torch.tensor([0.1, 0.1, 0.1], dtype=torch.float64)
    with pytest.raises(ValueError, match="K >= 1"):
        CoupledRun.apply(phi, th, p, cA, cB, 10, 0)
    with pytest.raises(ValueError, match="steps >= 0"):
        CoupledRun.apply(phi, th, p, cA, cB, -1, 5)
    with pytest.raises(ValueError, match="f32 or f64"):
        CoupledRun.apply(phi, th, p.with_(storage="f16"), cA, cB, 10, 5)
    with pytest.raises(ValueError, match="without flow"):
        CoupledRun.apply(phi, th, p.with_(flow=True), cA, cB, 10, 5)


def test_mean_radius_is_host_arithmetic(lib):
    # <R> from the reduction sums (Eq. 67 in 2D, the sphere-area analogue in 3D): no device
    import math
    from paper_2409_03401_gb300 import _lib
    from workloads.params import LBMParams
    idx = {k: i for i, k in enumerate(_lib.REDUCTIONS)}
    sums = (ctypes.c_double * _lib.NRED)()
    sums[idx["interface"]] = 2 * math.pi * 5.0 * 7                  # seven discs of radius 5
    sums[idx["euler"]] = 7
    p2 = _lib.make_params(LBMParams(nx=64, ny=64, nz=1, lattice="D2Q9"))
    assert lib.lbm_mean_radius(ctypes.byref(p2), sums) == pytest.approx(5.0)
    sums[idx["interface"]] = 4 * math.pi * 6.0 ** 2 * 3              # three spheres of radius 6
    sums[idx["euler"]] = 3
    p3 = _lib.make_params(LBMParams(nx=32, ny=32, nz=32))
    assert lib.lbm_mean_radius(ctypes.byref(p3), sums) == pytest.approx(6.0)
    sums[idx["euler"]] = 0
    assert math.isnan(lib.lbm_mean_radius(ctypes.byref(p3), sums))
    assert math.isnan(lib.lbm_mean_radius(None, sums))
