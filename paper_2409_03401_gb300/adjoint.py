"""Reverse mode of the coupled step without flow, as a torch.autograd.Function.

``CoupledRun.apply(phi0, theta, params, cA0, cB0, steps, K)`` runs ``steps`` coupled
steps from the initial phase field ``phi0`` with theta = (D_0, D_1, M_phi) (D_pi is the
mobility of both components in phase pi) and returns (phi, mu^A, mu^B) of the final time
level. Forward: the state is checkpointed every K steps. Backward: for each segment in
reverse order, one lbm_adjoint_segment call recomputes the K states out of place from the
checkpoint into a ring, then runs the hand-written adjoint kernels from the segment's last
step down to its first; lbm_adjoint_init maps the adjoint of the initial populations to
dL/dphi0. Every step runs in the library's CUDA kernels.
"""
import ctypes

import torch

from . import _lib
from .lattice import Simulation


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _with_theta(params, theta):
    d0, d1, mphi = (float(v) for v in theta)
    return params.with_(M=((d0, d0), (d1, d1)), M_phi=mphi)


class CoupledRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, theta, params, cA0, cB0, steps, K):
        if params.flow:
            raise ValueError("the adjoint covers the step without flow")
        if params.storage not in ("f32", "f64"):
            raise ValueError("the adjoint needs f32 or f64 storage")
        if int(K) < 1 or int(steps) < 0:
            raise ValueError(f"need K >= 1 and steps >= 0 (got K = {K}, steps = {steps})")
        steps, K = int(steps), int(K)
        p = _with_theta(params, theta.detach().cpu())
        device = phi0.device
        phi0d = phi0.detach().to(device=device, dtype=torch.float64).contiguous()
        cA0d = cA0.to(device=device, dtype=torch.float64).contiguous()
        cB0d = cB0.to(device=device, dtype=torch.float64).contiguous()
        sim = Simulation(p, phi0d, cA0d, cB0d, device=device)
        ckpts = []
        t = 0
        while t < steps:
            ckpts.append((t, sim.state.clone()))
            n = min(K, steps - t)
            sim.step(n)
            t += n
        f = sim.fields(("phi", "muA", "muB"))
        ctx.p, ctx.steps, ctx.K = p, steps, K
        ctx.ckpts = ckpts
        ctx.sim = sim
        ctx.init = (phi0d, cA0d, cB0d)
        ctx.phi0_dtype = phi0.dtype
        return f["phi"], f["muA"], f["muB"]

    @staticmethod
    def backward(ctx, gphi, gmuA, gmuB):
        lib = _lib.load()
        p, steps, K = ctx.p, ctx.steps, ctx.K
        cp = _lib.make_params(p)
        sim = ctx.sim
        device = sim.device
        stream = ctypes.c_void_p(sim.stream.cuda_stream)
        rdt = sim.real_dtype
        lam_bytes = lib.lbm_adjoint_bytes(ctypes.byref(cp))
        lam = torch.empty(lam_bytes, dtype=torch.uint8, device=device)
        lam2 = torch.empty(lam_bytes, dtype=torch.uint8, device=device)
        adj_work = torch.empty(lib.lbm_adjoint_work_bytes(ctypes.byref(cp)), dtype=torch.uint8, device=device)
        g = [None if x is None else x.to(dtype=rdt).contiguous() for x in (gphi, gmuA, gmuB)]
        _lib.check(lib.lbm_adjoint_reset(ctypes.byref(cp), _vp(adj_work), stream))
        _lib.check(lib.lbm_adjoint_seed(ctypes.byref(cp), _vp(sim.state), steps, _vp(g[0]), _vp(g[1]), _vp(g[2]),
                                        _vp(lam), _vp(adj_work), stream))
        copy = lib.lbm_copy_bytes(ctypes.byref(cp))
        ring = torch.empty(min(K, steps) * copy, dtype=torch.uint8, device=device)
        which = ctypes.c_int(0)
        for t0, ck in reversed(ctx.ckpts):
            n = min(K, steps - t0)
            ring[:copy].copy_(ck)
            # recompute the segment's states and sweep it in reverse (one library call)
            _lib.check(lib.lbm_adjoint_segment(ctypes.byref(cp), _vp(ring), t0, n, _vp(lam), _vp(lam2),
                                               _vp(adj_work), _vp(sim.work), stream, ctypes.byref(which)))
            if which.value == 1:
                lam, lam2 = lam2, lam
        phi0d, cA0d, cB0d = ctx.init
        phi0b = torch.empty_like(phi0d)
        _lib.check(lib.lbm_adjoint_init(ctypes.byref(cp), _vp(phi0d), _vp(cA0d), _vp(cB0d), _vp(lam), _vp(phi0b),
                                        _vp(adj_work), stream))
        out = (ctypes.c_double * 5)()
        _lib.check(lib.lbm_adjoint_theta(ctypes.byref(cp), _vp(adj_work), out, stream))
        gtheta = torch.tensor([out[0] + out[1], out[2] + out[3], out[4]], dtype=torch.float64)
        ctx.ckpts = None
        return phi0b.to(ctx.phi0_dtype), gtheta, None, None, None, None, None


def misfit(fields, target):
    """L = 1/2 sum [(phi - phi*)^2 + (mu^A - mu^A*)^2 + (mu^B - mu^B*)^2] in FP64."""
    return 0.5 * sum(((a.double() - b.double()) ** 2).sum() for a, b in zip(fields, target))


def misfit_and_gradient(params, theta, phi0, cA0, cB0, steps, target, K=100):
    """(L, dL/dtheta [3] float64, dL/dphi0) of the L2 misfit to ``target`` = (phi*, mu^A*, mu^B*)."""
    th = torch.as_tensor(theta, dtype=torch.float64).clone().requires_grad_(True)
    p0 = phi0.detach().clone().requires_grad_(True)
    out = CoupledRun.apply(p0, th, params, cA0, cB0, steps, K)
    L = misfit(out, target)
    L.backward()
    return float(L.detach()), th.grad.detach().clone(), p0.grad.detach().clone()


def forward_fields(params, theta, phi0, cA0, cB0, steps, device=None):
    """(phi, mu^A, mu^B) after ``steps`` steps at theta, no gradient."""
    p = _with_theta(params, theta)
    sim = Simulation(p, phi0, cA0, cB0, device=device)
    sim.step(steps)
    f = sim.fields(("phi", "muA", "muB"))
    return f["phi"], f["muA"], f["muB"]
