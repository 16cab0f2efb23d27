"""Python front end of the C-ABI: PyTorch owns the device memory and the stream.

``Simulation`` allocates the state and scratch buffers as torch tensors on a CUDA
device, binds them with lbm_init, and forwards lbm_step / lbm_fields / lbm_reduce.
Every step of the method runs in the sm_103a kernels of liblbm_gb300.so.
"""
import ctypes

import torch

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def droplet_stats(params, sums):
    """Droplet count N (the Euler characteristic of the reduction) and mean radius <R>
    (lbm_mean_radius: Eq. 67 in 2D, the sphere-area analogue in 3D) from a dict of lbm_reduce
    sums. <R> is NaN when N <= 0."""
    lib = _lib.load()
    cp = _lib.make_params(params)
    arr = (ctypes.c_double * _lib.NRED)(*[float(sums[k]) for k in _lib.REDUCTIONS])
    return {"N": sums["euler"], "R_mean": lib.lbm_mean_radius(ctypes.byref(cp), arr),
            "interface": sums["interface"]}


class Simulation:
    """One lattice bound to caller-owned device memory.

    ``params``: workloads.LBMParams. ``phi0, cA0, cB0``: float64 tensors of shape
    (nz, ny, nx) on the target CUDA device (or on the host: they are copied).
    """

    def __init__(self, params, phi0, cA0, cB0, device=None, stream=None):
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        device = torch.device(device)
        if device.type != "cuda":
            raise ValueError("Simulation needs a CUDA device")
        # the library reads nx*ny*nz values of each initial field: check before any device call
        n = params.nx * params.ny * params.nz
        for name, t in (("phi0", phi0), ("cA0", cA0), ("cB0", cB0)):
            if t.numel() != n:
                raise ValueError(f"{name} has {t.numel()} values; the lattice has nx*ny*nz = {n}")
        self.lib = _lib.load()
        self.params = params
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        self._cp = _lib.make_params(params)
        nbytes = self.lib.lbm_state_bytes(ctypes.byref(self._cp))
        wbytes = self.lib.lbm_work_bytes(ctypes.byref(self._cp))
        if nbytes == 0 or wbytes == 0:
            raise _lib.LBMError(_lib.LBM_ERR_ARG, "invalid parameters")
        # torch's caching allocator returns 512-byte aligned blocks
        self.state = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.work = torch.empty(wbytes, dtype=torch.uint8, device=device)
        self._ctx = ctypes.c_void_p()
        self._init_fields = [t.to(device=device, dtype=torch.float64).contiguous() for t in (phi0, cA0, cB0)]
        with torch.cuda.device(device):
            _lib.check(self.lib.lbm_init(ctypes.byref(self._cp), _ptr(self.state), _ptr(self.work),
                                              *[_ptr(t) for t in self._init_fields],
                                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._ctx)))

    @classmethod
    def attach(cls, params, state, t, device=None, stream=None):
        """Resume from a state tensor saved earlier (checkpoint/resume). ``state``: a
        contiguous uint8 CUDA tensor holding at least lbm_state_bytes(params) bytes, as
        written by the same build of the library for the same parameters."""
        self = cls.__new__(cls)
        self.lib = _lib.load()
        self._cp = _lib.make_params(params)
        need = self.lib.lbm_state_bytes(ctypes.byref(self._cp))
        if need == 0:
            raise _lib.LBMError(_lib.LBM_ERR_ARG, "invalid parameters")
        # the library cannot see the buffer's size: a short one would be read out of bounds
        if state.dtype != torch.uint8 or not state.is_contiguous() or state.numel() < need:
            raise ValueError(f"state must be a contiguous uint8 tensor of at least {need} bytes "
                             f"(got {state.dtype}, {state.numel()} elements)")
        if state.device.type != "cuda":
            raise ValueError("state must live on a CUDA device")
        if device is not None:
            want = torch.device(device)
            if want.type != "cuda" or (want.index is not None and want != state.device):
                raise ValueError(f"state is on {state.device}, not on {want}")
        device = state.device
        self.params = params
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        wbytes = self.lib.lbm_work_bytes(ctypes.byref(self._cp))
        self.state = state
        self.work = torch.empty(wbytes, dtype=torch.uint8, device=device)
        self._ctx = ctypes.c_void_p()
        self._init_fields = []
        _lib.check(self.lib.lbm_attach(ctypes.byref(self._cp), _ptr(self.state), _ptr(self.work), int(t),
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._ctx)))
        return self

    def save(self, path):
        """Checkpoint: the parameters, the time level and the raw state bytes (on the host)."""
        torch.cuda.synchronize(self.device)
        torch.save({"params": self.params.as_dict(), "t": self.t, "state": self.state.cpu()}, path)

    @classmethod
    def load(cls, path, device=None, stream=None):
        """Resume a checkpoint written by ``save`` (same build of the library)."""
        from workloads.params import LBMParams
        ck = torch.load(path, map_location="cpu")
        d = dict(ck["params"])
        for key in ("c_eq", "M"):
            d[key] = tuple(tuple(r) for r in d[key])
        d["g"] = tuple(d["g"])
        params = LBMParams(**d)
        device = torch.device(device or "cuda")
        state = ck["state"].to(device)
        return cls.attach(params, state, ck["t"], device=device, stream=stream)

    @property
    def t(self):
        return int(self.lib.lbm_time(self._ctx))

    @property
    def real_dtype(self):
        return torch.float64 if self.params.storage == "f64" else torch.float32

    def step(self, n=1, graph=False):
        """Advance n steps; ``graph=True`` replays a captured CUDA graph of two steps (needs a
        created stream, e.g. Simulation(..., stream=torch.cuda.Stream()))."""
        fn = self.lib.lbm_step_graph if graph else self.lib.lbm_step
        _lib.check(fn(self._ctx, int(n)), self._ctx)
        return self

    def fields(self, names=_lib.FIELDS):
        """Dict of (nz, ny, nx) tensors of the current time level."""
        unknown = [k for k in names if k not in _lib.FIELDS]
        if unknown:
            raise ValueError(f"unknown fields {unknown}; the library writes {_lib.FIELDS}")
        out = {k: torch.empty(self.params.shape, dtype=self.real_dtype, device=self.device) for k in names}
        ptrs = (ctypes.c_void_p * _lib.NFIELDS)()
        for i, k in enumerate(_lib.FIELDS):
            ptrs[i] = out[k].data_ptr() if k in out else None
        _lib.check(self.lib.lbm_fields(self._ctx, ptrs), self._ctx)
        return out

    def sums(self, raise_unstable=True):
        """FP64 diagnostics (synchronises the stream)."""
        buf = (ctypes.c_double * _lib.NRED)()
        st = self.lib.lbm_reduce(self._ctx, buf)
        if st != _lib.LBM_OK and (raise_unstable or st != _lib.LBM_ERR_UNSTABLE):
            _lib.check(st, self._ctx)
        return {k: buf[i] for i, k in enumerate(_lib.REDUCTIONS)}

    def droplets(self):
        """Droplet count N and mean radius <R> of the current time level (§4.2.2, one
        reduction pass on the device; synchronises the stream)."""
        return droplet_stats(self.params, self.sums())

    def profile_begin(self, max_steps):
        """Record CUDA events around this context's kernels for the next max_steps steps."""
        _lib.check(self.lib.lbm_profile_begin(self._ctx, int(max_steps)), self._ctx)

    def profile_end(self):
        """(ms of phi passes, ms of fused step kernels, steps timed); synchronises."""
        buf = (ctypes.c_double * 3)()
        _lib.check(self.lib.lbm_profile_end(self._ctx, buf), self._ctx)
        return buf[0], buf[1], int(buf[2])

    @property
    def kernels_per_step(self):
        return int(self.lib.lbm_kernels_per_step(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self.lib.lbm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
