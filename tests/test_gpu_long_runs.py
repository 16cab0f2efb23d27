"""Bounded versions of the two long-run studies (bench.py --drift, --ripening-law).

* Drift: on the wall-bounded flow workload the invariants sum c^A and sum c^B (FP64
  reductions) stay put to round-off for FP32 and for 16-bit storage (whose rounding
  residuals go into the FP32 rest populations), and sum phi of the 16-bit runs follows
  the FP32 run.
* Ripening law: on a 2D D2Q9 ripening run the droplet count falls and <R>^3 from Eq. 67
  grows linearly in time in the second half of the run (Lifshitz-Slyozov-Wagner).
"""
import math

import pytest
import torch

from workloads import configs

pytestmark = pytest.mark.gpu


def test_drift_of_invariants_fp32_and_16bit():
    from paper_2409_03401_gb300 import Simulation
    p, fields = configs.drift(shape=(96, 96, 96))
    init = fields(device="cuda")
    res = {}
    for storage in ("f32", "f16", "bf16"):
        sim = Simulation(p.with_(storage=storage), *init, device="cuda")
        s0 = sim.sums()
        sim.step(2000)
        s1 = sim.sums()
        res[storage] = (s0, s1)
        del sim
    for storage, (s0, s1) in res.items():
        for key in ("cA", "cB"):
            drift = abs(s1[key] - s0[key]) / abs(s0[key])
            print(f"{storage} relative drift of sum {key} over 2000 steps: {drift:.3e}")
            assert drift < 1e-6, (storage, key, drift)
    phi32 = res["f32"][1]["phi"]
    for storage in ("f16", "bf16"):
        dev = abs(res[storage][1]["phi"] - phi32) / abs(phi32)
        print(f"{storage} sum phi vs FP32 after 2000 steps: {dev:.3e}")
        assert dev < (1e-4 if storage == "f16" else 1e-3)


def test_ripening_law_2d():
    from paper_2409_03401_gb300 import Simulation
    p, fields = configs.ripening_2d(shape=(1, 1024, 1024), seed=9)
    sim = Simulation(p, *fields(device="cuda"), device="cuda")
    ts, R3, N = [], [], []
    for t in range(0, 40001, 4000):
        if t:
            sim.step(4000)
        s = sim.sums()
        ts.append(t)
        N.append(s["euler"])
        R3.append((s["interface"] / (2 * math.pi * s["euler"])) ** 3)
    print("t", ts, "N", N, "R^3", [round(v, 1) for v in R3])
    assert N[-1] < 0.8 * N[0]
    late = [(t, r) for t, r in zip(ts, R3) if t >= 20000]
    x = torch.tensor([a for a, _ in late], dtype=torch.float64)
    y = torch.tensor([b for _, b in late], dtype=torch.float64)
    A = torch.stack([torch.ones_like(x), x], 1)
    coef = torch.linalg.lstsq(A, y.unsqueeze(1)).solution.squeeze(1)
    fit = A @ coef
    r2 = 1 - float(((y - fit) ** 2).sum() / ((y - y.mean()) ** 2).sum())
    print("slope of <R>^3 per step", float(coef[1]), "R^2", r2)
    assert float(coef[1]) > 0 and r2 > 0.95
