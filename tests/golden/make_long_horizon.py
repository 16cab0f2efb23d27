"""Write the FP64 oracle's expected values for the long-horizon GPU parity tests.

The oracle needs minutes to tens of minutes per run at these horizons, too long for a
test, so this script runs it once and stores, per case, sampled fields at a few snapshot
times plus whole-lattice sums and the droplet count. It calls only ``oracle/`` (and the
seeded input generators of ``workloads/``); nothing here comes from the CUDA path.

    python tests/golden/make_long_horizon.py [case ...]      # all cases by default
    python tests/golden/make_long_horizon.py --sensitivity [case ...]   # after the above

Cases (the workloads' physics at reduced size and their full step counts):
  ripening_48  - 3D Ostwald ripening, D3Q7, periodic, 48^3, fraction 0.15, r in [4, 10],
                 2 % supersaturation, 20,000 steps (at this size every droplet is below the
                 critical radius: all have dissolved by step 5000)
  ripening_48_grow - the same at 30 % supersaturation, where the droplets grow and then
                 coarsen over the whole run
  sedimentation_64 - coarsening with flow and buoyancy, walls at the z ends, 64^3,
                 fraction 0.2, r in [6, 16], 10,000 steps
  adjoint_32   - misfit gradient w.r.t. (D_0, D_1, M_phi) and phi_0 on a 32^3 ripening
                 lattice at 30 % supersaturation (at 2 % every droplet of so small a box
                 dissolves and target and run meet: the misfit falls to 1e-20), 2,000 steps,
                 target at (0.4, 0.8, 0.05), evaluated at (0.5, 0.7, 0.06); reverse mode
                 through the oracle with recomputation per 100-step segment

Sampled nodes: every node of two z planes (z = 1 and z = nz // 2 + 1) and 4096 further
nodes drawn with a seeded generator. Values are stored as float32 (relative rounding
6e-8, far below the 1e-5 FP32-storage bar).
"""
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import adjoint as oracle_adjoint          # noqa: E402
from oracle.lbm import OracleLBM                      # noqa: E402
from oracle.measure import euler_characteristic      # noqa: E402
from workloads import configs                         # noqa: E402

CASES = {
    "ripening_48": dict(kind="forward", builder="ripening", shape=(48, 48, 48),
                        snapshots=(1000, 5000, 10000, 20000)),
    "ripening_48_grow": dict(kind="forward", builder="ripening", shape=(48, 48, 48), supersaturation=0.3,
                             snapshots=(1000, 5000, 10000, 20000)),
    "sedimentation_64": dict(kind="forward", builder="sedimentation", shape=(64, 64, 64),
                             snapshots=(1000, 2500, 5000, 10000)),
    "adjoint_32": dict(kind="adjoint", shape=(32, 32, 32), steps=2000, K=100, supersaturation=0.3),
}
FIELDS = ("phi", "muA", "muB", "cA", "cB", "p", "ux", "uy", "uz")


def path(name):
    return os.path.join(HERE, f"long_{name}.npz")


def case_params(name, storage="f64"):
    c = CASES[name]
    kw = {"supersaturation": c["supersaturation"]} if "supersaturation" in c else {}
    if c["kind"] == "adjoint":
        return configs.adjoint_problem(shape=c["shape"], storage=storage, **kw)
    return getattr(configs, c["builder"])(shape=c["shape"], storage=storage, **kw)


def sample_index(shape, n_random=4096, seed=1234):
    """Flat node indices of the sample: two full z planes and seeded random nodes."""
    nz, ny, nx = shape
    plane = ny * nx
    idx = [np.arange(plane) + z * plane for z in (1, nz // 2 + 1)]
    rng = np.random.default_rng(seed)
    idx.append(rng.choice(nz * plane, size=n_random, replace=False))
    return np.unique(np.concatenate(idx))


def forward(name):
    c = CASES[name]
    p, fields = case_params(name)
    o = OracleLBM(p)
    o.init(*fields())
    idx = sample_index(p.shape)
    out = {"index": idx, "snapshots": np.array(c["snapshots"])}
    walls = (p.wall_x, False, p.wall_z)
    t0 = time.time()
    for t in c["snapshots"]:
        o.step(t - o.t)
        f = o.fields()
        names = FIELDS if p.flow else FIELDS[:5]
        for k in names:
            out[f"{k}@{t}"] = f[k].reshape(-1).numpy()[idx].astype(np.float32)
        s = o.sums()
        for k in ("phi", "cA", "cB", "g"):
            out[f"sum_{k}@{t}"] = np.float64(s[k])
        out[f"euler@{t}"] = np.int64(euler_characteristic(f["phi"].numpy(), walls=walls))
        print(f"{name}: t={t} sum phi={s['phi']:.6f} droplets={int(out[f'euler@{t}'])} "
              f"({time.time() - t0:.0f} s)", flush=True)
    np.savez_compressed(path(name), **out)


def sensitivity(name):
    """The dynamics' own response to FP32-level rounding: the oracle (FP64) run again from
    its initial populations rounded once to FP32, compared at every snapshot with the stored
    run by the same measure as the GPU tests (relative L-infinity over the sample). Where this
    exceeds the FP32 bar, no FP32 run can follow the FP64 one pointwise any longer."""
    c = CASES[name]
    p, fields = case_params(name)
    ref = np.load(path(name))
    idx = ref["index"]
    o = OracleLBM(p)
    o.init(*fields())
    # as FP32 storage holds them: the rest populations of h shifted by c_0^eq
    shift = {"hA": p.c_eq[0][0], "hB": p.c_eq[0][1]}
    for key, pops in o.populations().items():
        s = shift.get(key, 0.0)
        pops[0].copy_(((pops[0] - s).to(torch.float32).to(torch.float64)) + s)
        pops[1:].copy_(pops[1:].to(torch.float32).to(torch.float64))
    floors = {"muA": 1e-3, "muB": 1e-3, "p": 1e-6, "ux": 1e-6, "uy": 1e-6, "uz": 1e-6}
    out = {"snapshots": np.array(c["snapshots"])}
    t0 = time.time()
    for t in c["snapshots"]:
        o.step(t - o.t)
        f = o.fields()
        names = FIELDS if p.flow else FIELDS[:5]
        msg = []
        for k in names:
            a = f[k].reshape(-1).numpy()[idx]
            b = ref[f"{k}@{t}"].astype(np.float64)
            e = float(np.abs(a - b).max()) / max(float(np.abs(b).max()), floors.get(k, 1e-12))
            out[f"{k}@{t}"] = np.float64(e)
            msg.append(f"{k} {e:.2e}")
        print(f"{name} (FP32-rounded start): t={t} " + ", ".join(msg) + f" ({time.time() - t0:.0f} s)", flush=True)
    np.savez_compressed(os.path.join(HERE, f"long_{name}_sensitivity.npz"), **out)


def adjoint(name):
    """Gradient through the oracle in segments of K steps: each segment's forward is re-run
    under autograd from its stored start state (the exact discrete adjoint, in FP64)."""
    c = CASES[name]
    p, fields = case_params(name)
    phi0, cA0, cB0 = fields()
    steps, K = c["steps"], c["K"]
    target = oracle_adjoint.target_fields(p, configs.THETA_TARGET, phi0, cA0, cB0, steps)
    t0 = time.time()
    th = torch.tensor(configs.THETA_EVAL, dtype=torch.float64, requires_grad=True)
    p0 = phi0.clone().requires_grad_(True)
    o = OracleLBM(p, theta=(th[0], th[1], th[2]))
    # forward pass without a graph, keeping the segment start states
    starts = []
    with torch.no_grad():
        o.init(phi0, cA0, cB0)
        for s in range(0, steps, K):
            starts.append({k: v.clone() for k, v in o.populations().items()})
            o.step(min(K, steps - s))
    # reverse sweep: last segment first
    adj = None
    gth = torch.zeros(3, dtype=torch.float64)
    L = None
    for i in reversed(range(len(starts))):
        s = i * K
        n = min(K, steps - s)
        seg = OracleLBM(p, theta=(th[0], th[1], th[2]))
        if i == 0:
            seg.init(p0, cA0, cB0)
            leaves = None
        else:
            leaves = {k: v.clone().requires_grad_(True) for k, v in starts[i].items()}
            seg.g, seg.hA, seg.hB = leaves["g"], leaves["hA"], leaves["hB"]
        seg.step(n)
        if adj is None:
            L = oracle_adjoint.misfit(seg.fields(), target)
            out = [L]
            grads_in = [None]
        else:
            pops = seg.populations()
            out = [pops[k] for k in ("g", "hA", "hB")]
            grads_in = [adj[k] for k in ("g", "hA", "hB")]
        inputs = [th] + ([p0] if i == 0 else [leaves[k] for k in ("g", "hA", "hB")])
        grads = torch.autograd.grad(out, inputs, grad_outputs=grads_in, allow_unused=True)
        if grads[0] is not None:
            gth += grads[0]
        if i > 0:
            adj = dict(zip(("g", "hA", "hB"), grads[1:]))
        else:
            gphi = grads[1]
        print(f"{name}: segment {i} done ({time.time() - t0:.0f} s)", flush=True)
    np.savez_compressed(path(name), L=np.float64(L.detach()), grad_theta=gth.numpy(),
                        grad_phi0=gphi.numpy().astype(np.float32), steps=np.int64(steps), K=np.int64(K))
    print(f"{name}: L={float(L.detach()):.6e} dL/dtheta={gth.numpy()}", flush=True)


def main(names):
    torch.set_num_threads(int(os.environ.get("ORACLE_THREADS", torch.get_num_threads())))
    sens = "--sensitivity" in names
    names = [n for n in names if n != "--sensitivity"]
    for name in names or list(CASES):
        if sens:
            if CASES[name]["kind"] == "forward":
                sensitivity(name)
        else:
            (adjoint if CASES[name]["kind"] == "adjoint" else forward)(name)


if __name__ == "__main__":
    main(sys.argv[1:])
