"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64 oracle from
the same seeded inputs and compare field by field.

Relative L-infinity error of a field: |x_gpu - x_ref|_inf / max(|x_ref|_inf, floor),
with floors 1e-3 for mu (it tends to 0 at equilibrium) and 1e-6 for p and u (they
start at 0); phi and c use their own maximum.
"""
import torch

FLOORS = {"phi": 1e-12, "cA": 1e-12, "cB": 1e-12, "muA": 1e-3, "muB": 1e-3,
          "p": 1e-6, "ux": 1e-6, "uy": 1e-6, "uz": 1e-6}
TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-3, "bf16": 1e-2}


def rel_linf(gpu, ref, name):
    ref = ref.to(torch.float64).cpu()
    gpu = gpu.to(torch.float64).cpu()
    scale = max(float(ref.abs().max()), FLOORS[name])
    return float((gpu - ref).abs().max()) / scale


def run_gpu(params, fields, steps, device="cuda"):
    from paper_2409_03401_gb300 import Simulation
    sim = Simulation(params, *fields, device=device)
    sim.step(steps)
    out = sim.fields()
    torch.cuda.synchronize()
    return sim, out


def run_oracle(params, fields, steps):
    from oracle.lbm import OracleLBM
    o = OracleLBM(params)
    o.init(*[f.cpu() for f in fields])
    o.step(steps)
    return o, o.fields()


def compare(params, fields, steps, names=None):
    """Return {field: rel_linf} after ``steps`` steps on both sides."""
    names = names or (["phi", "muA", "muB", "cA", "cB"] + (["p", "ux", "uy", "uz"] if params.flow else []))
    _, g = run_gpu(params, fields, steps)
    _, r = run_oracle(params, fields, steps)
    return {k: rel_linf(g[k], r[k], k) for k in names}
