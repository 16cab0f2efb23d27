"""Domain decomposition along z: slabs with ghost planes and their halo exchange.

The paper runs its largest lattice by domain decomposition over many GPUs (§3, §4.2.4).
Here a lattice splits into z slabs (``split_planes``); each ``Slab`` is one lbm_slab_init
context with a ghost plane on every side that has a neighbour. One step of the whole lattice
is, for every slab (``exchange`` moves the messages):

  1. lbm_step on every slab (it reads the ghost populations and ghost phi of time level t);
  2. populations: every slab packs what leaves through its faces (lbm_slab_pack); the
     neighbours unpack it into their ghost planes (lbm_slab_unpack);
  3. phi (flow only): every slab computes phi of its edge planes (lbm_slab_phi_pack), which
     the neighbours keep as ghost phi (lbm_slab_phi_unpack) for the capillary stencil.

After initialisation only phase 3 is needed. The messages travel by ``LocalTransport``
(slabs of one process: the message tensors are handed over) or ``DistTransport`` (one slab
per rank, torch.distributed point-to-point: NCCL between GPUs, gloo for host tensors).
Every step of the method runs in the library's kernels; this module only routes buffers.
"""
import ctypes

import torch

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def split_planes(nz, n):
    """Split nz planes into n contiguous slabs as evenly as possible: [(z0, nzl), ...]."""
    if not 1 <= n <= nz:
        raise ValueError(f"cannot split {nz} planes into {n} slabs")
    base, extra = divmod(nz, n)
    out, z0 = [], 0
    for i in range(n):
        nzl = base + (1 if i < extra else 0)
        out.append((z0, nzl))
        z0 += nzl
    return out


def neighbours(i, n, wall_z):
    """(lower, upper) slab index of slab i of n; None where a wall ends the lattice. With
    periodic z the first and last slabs are neighbours (a single slab is its own)."""
    lower = i - 1 if i > 0 else (None if wall_z else n - 1)
    upper = i + 1 if i < n - 1 else (None if wall_z else 0)
    return lower, upper


def ghost_range(nz, z0, nzl, wall_z):
    """Global planes (wrapped) of a slab's own lattice: one ghost plane on each side that has
    a neighbour, then the own planes."""
    lo = [] if (wall_z and z0 == 0) else [(z0 - 1) % nz]
    hi = [] if (wall_z and z0 + nzl == nz) else [(z0 + nzl) % nz]
    return lo + list(range(z0, z0 + nzl)) + hi


class Slab:
    """Planes [z0, z0 + nzl) of the lattice ``params`` on one device.

    ``phi0, cA0, cB0``: the global initial fields (nz, ny, nx) or only the slab's planes
    ``ghost_range(...)`` (lbm_slab_planes of them)."""

    def __init__(self, params, z0, nzl, phi0, cA0, cB0, device=None, stream=None):
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.lib = _lib.load()
        self.params, self.z0, self.nzl, self.device = params, z0, nzl, device
        self.stream = stream or torch.cuda.current_stream(device)
        self._cp = _lib.make_params(params)
        cp = ctypes.byref(self._cp)
        self.planes = self.lib.lbm_slab_planes(cp, z0, nzl)
        if self.planes == 0:
            raise _lib.LBMError(_lib.LBM_ERR_ARG, f"invalid slab z0={z0} nzl={nzl} of nz={params.nz}")
        zs = ghost_range(params.nz, z0, nzl, params.wall_z)
        assert len(zs) == self.planes
        self.lo = 1 if zs[0] != z0 else 0        # index of the first own plane
        idx = torch.tensor(zs, dtype=torch.long)
        fields = []
        for name, t in (("phi0", phi0), ("cA0", cA0), ("cB0", cB0)):
            if t.shape[0] == params.nz:
                t = t.index_select(0, idx.to(t.device))
            if tuple(t.shape) != (self.planes, params.ny, params.nx):
                raise ValueError(f"{name}: expected {params.nz} or {self.planes} planes of {params.ny} x {params.nx}")
            fields.append(t.to(device=device, dtype=torch.float64).contiguous())
        self._init_fields = fields
        self.state = torch.empty(self.lib.lbm_slab_state_bytes(cp, z0, nzl), dtype=torch.uint8, device=device)
        self.work = torch.empty(self.lib.lbm_slab_work_bytes(cp, z0, nzl), dtype=torch.uint8, device=device)
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(device):
            _lib.check(self.lib.lbm_slab_init(cp, z0, nzl, _ptr(self.state), _ptr(self.work),
                                              *[_ptr(t) for t in fields], ctypes.c_void_p(self.stream.cuda_stream),
                                              ctypes.byref(self._ctx)))
        g = self.lib.lbm_slab_ghosts(self._ctx)
        self.has = (bool(g & 1), bool(g & 2))
        self.halo_bytes = self.lib.lbm_slab_halo_bytes(self._ctx)
        self.phi_bytes = self.lib.lbm_slab_phi_bytes(self._ctx)

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx is not None and ctx.value:
            self.lib.lbm_destroy(ctx)
            self._ctx = None

    @property
    def t(self):
        return int(self.lib.lbm_time(self._ctx))

    def step(self):
        _lib.check(self.lib.lbm_step(self._ctx, 1), self._ctx)

    def pack(self, side):
        m = torch.empty(self.halo_bytes, dtype=torch.uint8, device=self.device)
        _lib.check(self.lib.lbm_slab_pack(self._ctx, side, _ptr(m)), self._ctx)
        return m

    def unpack(self, side, msg):
        _lib.check(self.lib.lbm_slab_unpack(self._ctx, side, _ptr(msg)), self._ctx)

    def phi_pack(self, side):
        m = torch.empty(self.phi_bytes, dtype=torch.uint8, device=self.device)
        _lib.check(self.lib.lbm_slab_phi_pack(self._ctx, side, _ptr(m)), self._ctx)
        return m

    def phi_unpack(self, side, msg):
        _lib.check(self.lib.lbm_slab_phi_unpack(self._ctx, side, _ptr(msg)), self._ctx)

    def fields(self, names=_lib.FIELDS):
        """Dict of (nzl, ny, nx) tensors of the own planes at the current time level."""
        real = torch.float64 if self.params.storage == "f64" else torch.float32
        shape = (self.planes, self.params.ny, self.params.nx)
        out = {k: torch.zeros(shape, dtype=real, device=self.device) for k in names}
        ptrs = (ctypes.c_void_p * _lib.NFIELDS)()
        for i, k in enumerate(_lib.FIELDS):
            ptrs[i] = out[k].data_ptr() if k in out else None
        _lib.check(self.lib.lbm_fields(self._ctx, ptrs), self._ctx)
        return {k: v[self.lo:self.lo + self.nzl] for k, v in out.items()}

    def sums(self):
        """FP64 sums over the own planes (the droplet count is not formed per slab)."""
        out = (ctypes.c_double * _lib.NRED)()
        _lib.check(self.lib.lbm_reduce(self._ctx, out), self._ctx)
        return {k: out[i] for i, k in enumerate(_lib.REDUCTIONS)}


def exchange_round(slabs, transport, pack, unpack):
    """Send every slab's face messages to its neighbours and unpack what arrives.
    ``slabs``: the slabs this process holds, keyed by slab index."""
    out = {i: {side: pack(s, side) for side in (0, 1) if s.has[side]} for i, s in slabs.items()}
    got = transport.exchange(out)
    for i, s in slabs.items():
        for side, msg in got[i].items():
            unpack(s, side, msg)


def halo_exchange(slabs, transport, flow, populations=True):
    """Phases 2 and 3 of a step (phase 3 alone after initialisation)."""
    if populations:
        exchange_round(slabs, transport, lambda s, d: s.pack(d), lambda s, d, m: s.unpack(d, m))
    if flow:
        exchange_round(slabs, transport, lambda s, d: s.phi_pack(d), lambda s, d, m: s.phi_unpack(d, m))


class LocalTransport:
    """Slabs held by one process: a message sent through a slab's face is handed to the
    neighbour on that side, arriving at its opposite side."""

    def __init__(self, n, wall_z):
        self.n, self.wall_z = n, wall_z

    def exchange(self, out):
        got = {i: {} for i in out}
        for i, msgs in out.items():
            lower, upper = neighbours(i, self.n, self.wall_z)
            if 0 in msgs:
                got[lower][1] = msgs[0]
            if 1 in msgs:
                got[upper][0] = msgs[1]
        return got


class DistTransport:
    """One slab per rank of a torch.distributed group (rank i holds slab i). Two exchanges of
    point-to-point messages, upward then downward, so that every pair of ranks exchanges at
    most one message per direction per exchange (NCCL matches sends and receives by order)."""

    def __init__(self, wall_z, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.n = dist.get_world_size(group)
        self.wall_z = wall_z

    def exchange(self, out):
        (i, msgs), = out.items()
        assert i == self.rank
        lower, upper = neighbours(i, self.n, self.wall_z)
        got = {}
        # first exchange: messages through upper faces (received at the neighbour's side 0);
        # second exchange: through lower faces (received at side 1)
        for send_side, nbr_to, nbr_from in ((1, upper, lower), (0, lower, upper)):
            recv_side = 1 - send_side
            if nbr_to == i:                                    # a single periodic slab
                got[recv_side] = msgs[send_side]
                continue
            ops = []
            if send_side in msgs and nbr_to is not None:
                ops.append(self.dist.P2POp(self.dist.isend, msgs[send_side], nbr_to, self.group))
            if nbr_from is not None:
                # both faces' messages of one phase have the same size
                buf = torch.empty_like(next(iter(msgs.values())))
                ops.append(self.dist.P2POp(self.dist.irecv, buf, nbr_from, self.group))
                got[recv_side] = buf
            if ops:
                for r in self.dist.batch_isend_irecv(ops):
                    r.wait()
        return {i: got}


class SlabGroup:
    """A lattice decomposed into ``n`` z slabs held by this process (one device by default,
    or one device each): the same results as one Simulation of the whole lattice."""

    def __init__(self, params, n, phi0, cA0, cB0, devices=None, stream=None):
        self.params = params
        self.parts = split_planes(params.nz, n)
        devices = devices or [None] * n
        self.slabs = {i: Slab(params, z0, nzl, phi0, cA0, cB0, device=devices[i], stream=stream)
                      for i, (z0, nzl) in enumerate(self.parts)}
        self.transport = LocalTransport(n, params.wall_z)
        halo_exchange(self.slabs, self.transport, params.flow, populations=False)

    def step(self, n=1):
        for _ in range(n):
            for s in self.slabs.values():
                s.step()
            halo_exchange(self.slabs, self.transport, self.params.flow)
        return self

    @property
    def t(self):
        return self.slabs[0].t

    def fields(self, names=_lib.FIELDS):
        parts = [s.fields(names) for s in self.slabs.values()]
        return {k: torch.cat([p[k].to(parts[0][k].device) for p in parts], 0) for k in names}

    def sums(self):
        """Sums over the whole lattice (additive entries summed, max |u| maximised)."""
        tot = None
        for s in self.slabs.values():
            d = s.sums()
            if tot is None:
                tot = dict(d)
            else:
                for k, v in d.items():
                    tot[k] = max(tot[k], v) if k == "umax" else tot[k] + v
        return tot
