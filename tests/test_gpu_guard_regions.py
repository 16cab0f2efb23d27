"""Out-of-bounds writes: every buffer the library is given sits between guard regions of a
known byte pattern inside one larger allocation, and after init, steps of both parities,
fields, reductions and destroy the guards must be untouched (the check a memory sanitizer
would make, here without one). The layouts covered: fused two-copy flow, in-place flow,
16-bit flow, D3Q19 scalars with flow, FP64 in-place scalars, D2Q9, the walled D2Q5 couple.
A stray write lands in this test's own allocation, so it is reported, not a fault.
"""
import ctypes

import pytest
import torch

from workloads import configs

pytestmark = pytest.mark.gpu

GUARD = 1 << 16          # bytes of pattern before and after each buffer (a multiple of 256)
FILL = 0xA5
FIELD_FILL = 12345.0


def _round(n, a=256):
    return (n + a - 1) // a * a


def _cases():
    sed = lambda **kw: configs.sedimentation(shape=(20, 22, 40), fraction=0.06, r=(3.0, 5.0), **kw)  # noqa: E731
    return {
        "flow_two_copies_f32": sed(),
        "flow_inplace_f32": (sed()[0].with_(inplace=True), sed()[1]),
        "flow_f16": sed(storage="f16"),
        "flow_d3q19_scalars": (sed()[0].with_(lattice="D3Q19"), sed()[1]),
        "ripening_f64": configs.ripening(shape=(12, 14, 33), storage="f64"),
        "ripening_d2q9": configs.ripening_2d(shape=(1, 90, 130)),
        "couple_d2q5_walls": configs.diffusion_couple(nx=96, ny=6),
    }


@pytest.mark.parametrize("case", list(_cases()))
def test_no_write_outside_the_given_buffers(case):
    from paper_2409_03401_gb300 import _lib
    lib = _lib.load()
    p, fields = _cases()[case]
    phi, cA, cB = [t.to("cuda", torch.float64).contiguous() for t in fields()]
    cp = _lib.make_params(p)
    sb = lib.lbm_state_bytes(ctypes.byref(cp))
    wb = lib.lbm_work_bytes(ctypes.byref(cp))
    assert sb > 0 and wb > 0
    o_s = GUARD
    o_w = _round(o_s + sb) + GUARD
    total = _round(o_w + wb) + GUARD
    buf = torch.full((total,), FILL, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    assert base % 256 == 0
    guards = [(0, o_s), (o_s + sb, o_w), (o_w + wb, total)]

    n = p.nx * p.ny * p.nz
    rdt = torch.float64 if p.storage == "f64" else torch.float32
    g_el = GUARD // 8
    outs = [torch.full((n + 2 * g_el,), FIELD_FILL, dtype=rdt, device="cuda") for _ in range(_lib.NFIELDS)]
    ptrs = (ctypes.c_void_p * _lib.NFIELDS)()
    for i, t in enumerate(outs):
        ptrs[i] = t.data_ptr() + g_el * t.element_size()

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ctx = ctypes.c_void_p()
    _lib.check(lib.lbm_init(ctypes.byref(cp), ctypes.c_void_p(base + o_s), ctypes.c_void_p(base + o_w),
                            ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(cA.data_ptr()),
                            ctypes.c_void_p(cB.data_ptr()), stream, ctypes.byref(ctx)))
    try:
        red = (ctypes.c_double * _lib.NRED)()
        for steps in (1, 4, 3):                       # odd and even time levels
            _lib.check(lib.lbm_step(ctx, steps), ctx)
            _lib.check(lib.lbm_fields(ctx, ptrs), ctx)
            _lib.check(lib.lbm_reduce(ctx, red), ctx)
        assert red[_lib.REDUCTIONS.index("nonfinite")] == 0
    finally:
        lib.lbm_destroy(ctx)
    torch.cuda.synchronize()

    for a, b in guards:
        bad = int((buf[a:b] != FILL).sum())
        assert bad == 0, f"{case}: {bad} bytes changed in the guard region [{a}, {b}) around state/work"
    for i, t in enumerate(outs):
        name = _lib.FIELDS[i]
        assert bool((t[:g_el] == FIELD_FILL).all()) and bool((t[g_el + n:] == FIELD_FILL).all()), name
        assert not bool((t[g_el:g_el + n] == FIELD_FILL).any()), f"{name} not written"
