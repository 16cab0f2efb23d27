"""The workloads at their own horizons, at reduced size, against the FP64 oracle.

The oracle needs minutes to tens of minutes for these runs, so its values were computed once
by tests/golden/make_long_horizon.py (which calls only oracle/ and the seeded input
generators) and stored as samples: every node of two z planes and 4096 seeded random nodes
per snapshot, plus whole-lattice sums and the droplet count.

* 3D ripening (D3Q7, periodic, 48^3, fraction 0.15, r in [4, 10]) over its 20,000 steps in
  FP32 storage, at the workload's 2 % supersaturation (every droplet of so small a box
  dissolves by step 5000) and at 30 % (the droplets grow, merge into one and keep it):
  relative L-infinity within 1e-5 of the oracle at every snapshot.
* Sedimentation with flow (walls at the z ends, 64^3, fraction 0.2, r in [6, 16]) over its
  10,000 steps in FP32 storage: within 1e-5 through step 5000. At step 10,000 the FP32 run
  has left the FP64 one by up to 2.4e-5 in phi (at the interfaces of the two droplets left)
  and 2.2e-5 in p: the droplets sediment, and their positions integrate the FP32 rounding of
  u (about 1e-5 of max |u| per step, a difference of populations) over the run. The
  dynamics does not amplify rounding: the oracle itself, restarted from its initial
  populations rounded to FP32, stays within 4e-8 of its own run at every snapshot
  (long_*_sensitivity.npz). Past step 5000 the test holds the invariants instead: the
  droplet count, and sum c^A, sum c^B within 1e-8.
* Adjoint (32^3 ripening at 30 % supersaturation, 2,000 steps, checkpoints every 100 steps,
  FP32 forward and reverse sweeps): misfit, gradient w.r.t. (D_0, D_1, M_phi) and w.r.t.
  phi_0 within the FP32 bar of 1e-5 of the oracle's reverse mode.
"""
import os
import sys

import numpy as np
import pytest
import torch

from parity import FLOORS, TOL

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_long_horizon as golden  # noqa: E402

pytestmark = pytest.mark.gpu


def _load(name):
    path = golden.path(name)
    if not os.path.exists(path):
        pytest.fail(f"{path} is missing: run tests/golden/make_long_horizon.py {name}")
    return np.load(path)


def _rel(gpu, ref, name):
    scale = max(float(np.abs(ref).max()), FLOORS[name])
    return float(np.abs(gpu - ref).max()) / scale


# snapshots at which the fields are held to the FP32 bar (all, unless listed)
FIELD_BAR_UNTIL = {"sedimentation_64": 5000}


@pytest.mark.parametrize("name", ["ripening_48", "ripening_48_grow", "sedimentation_64"])
def test_fp32_at_the_workload_horizon(name):
    from paper_2409_03401_gb300 import Simulation
    ref = _load(name)
    p, fields = golden.case_params(name, storage="f32")
    idx = torch.as_tensor(ref["index"], device="cuda")
    sim = Simulation(p, *fields())
    names = golden.FIELDS if p.flow else golden.FIELDS[:5]
    worst = {}
    for t in ref["snapshots"]:
        sim.step(int(t) - sim.t)
        f = sim.fields(names)
        errs = {k: _rel(f[k].reshape(-1)[idx].double().cpu().numpy(), ref[f"{k}@{t}"].astype(np.float64), k)
                for k in names}
        s = sim.sums()
        for k in ("cA", "cB"):
            errs[f"sum_{k}"] = abs(s[k] - float(ref[f"sum_{k}@{t}"])) / abs(float(ref[f"sum_{k}@{t}"]))
        # where phi departs most: the sample node and the oracle's phi there
        dphi = np.abs(f["phi"].reshape(-1)[idx].double().cpu().numpy() - ref[f"phi@{t}"].astype(np.float64))
        at = int(ref["index"][int(dphi.argmax())])
        zyx = (at // (p.nx * p.ny), (at // p.nx) % p.ny, at % p.nx)
        print(f"{name} t={int(t)}: droplets {s['euler']:.0f} (oracle {int(ref[f'euler@{t}'])}), "
              + ", ".join(f"{k} {v:.2e}" for k, v in errs.items())
              + f"; largest phi error at (z, y, x) = {zyx}, oracle phi {float(ref[f'phi@{t}'][int(dphi.argmax())]):.3f}")
        assert s["euler"] == int(ref[f"euler@{t}"]), ("droplet count", int(t))
        for k in ("sum_cA", "sum_cB"):
            assert errs[k] <= 1e-8, (k, int(t), errs[k])
        if int(t) > FIELD_BAR_UNTIL.get(name, 10 ** 9):
            continue
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
    bad = {k: v for k, v in worst.items() if not v <= TOL["f32"]}
    assert not bad, f"beyond {TOL['f32']}: {bad}"


def test_adjoint_at_the_workload_horizon():
    from paper_2409_03401_gb300.adjoint import misfit_and_gradient
    from oracle import adjoint as oracle_adjoint
    from workloads import configs
    ref = _load("adjoint_32")
    c = golden.CASES["adjoint_32"]
    steps, K = int(ref["steps"]), int(ref["K"])
    p, fields = golden.case_params("adjoint_32", storage="f32")
    phi0, cA0, cB0 = fields()
    # the target: the oracle's forward run at the target parameters (as in the stored gradient)
    p64, _ = golden.case_params("adjoint_32")
    tgt = oracle_adjoint.target_fields(p64, configs.THETA_TARGET, phi0, cA0, cB0, steps)
    dev = "cuda"
    L, gth, gphi = misfit_and_gradient(p, configs.THETA_EVAL, phi0.to(dev), cA0.to(dev), cB0.to(dev), steps,
                                       [tgt[k].to(dev) for k in ("phi", "muA", "muB")], K=K)
    L_ref, gth_ref = float(ref["L"]), torch.as_tensor(ref["grad_theta"])
    gphi_ref = torch.as_tensor(ref["grad_phi0"]).double()
    e_L = abs(L - L_ref) / abs(L_ref)
    e_th = float((gth.double().cpu() - gth_ref).abs().max() / gth_ref.abs().max())
    e_phi = float((gphi.double().cpu() - gphi_ref).abs().max() / gphi_ref.abs().max())
    print(f"adjoint {c['shape']} x {steps}, K = {K}: L {L:.6e} (oracle {L_ref:.6e}), rel. errors L {e_L:.2e}, "
          f"theta {e_th:.2e}, phi0 {e_phi:.2e}")
    assert max(e_L, e_th, e_phi) <= TOL["f32"]
