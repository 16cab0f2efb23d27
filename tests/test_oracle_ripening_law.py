"""The FP64 oracle against the Lifshitz-Slyozov-Wagner law of Ostwald ripening (CPU, slow).

In the coarsening regime the mean droplet radius grows as <R>^3 ~ t (§4.2.2, the law the
paper's 2D ripening run follows). The oracle runs the 2D table's parameters (D2Q9, phase
fraction 0.08, matrix 10 % of the gap above c_0^eq, W = 3) on a 224^2 periodic lattice with
droplet radii capped at 6 nodes, so that a box the oracle advances in minutes holds some
sixty droplets. <R> is Eq. 67's estimator: the interface measure over 2 pi N, N the Euler
characteristic of {phi >= 1/2}. Over the second half of 24,000 steps the droplet count keeps
falling and <R>^3 grows linearly (least-squares fit, R^2 > 0.95); a mistake in the
closure, the source or the relaxation rates stops the coarsening or bends the curve.
"""
import math

import numpy as np
import pytest

from oracle.lbm import OracleLBM
from oracle.measure import euler_characteristic, interface_measure
from workloads import configs


@pytest.mark.slow
def test_mean_radius_cubed_grows_linearly_in_time():
    p, fields = configs.ripening_2d(shape=(1, 224, 224), storage="f64", seed=9, r_max=6.0)
    o = OracleLBM(p)
    o.init(*fields())
    ts, N, R3 = [], [], []
    for t in range(0, 24001, 2000):
        if t:
            o.step(2000)
        phi = o.fields()["phi"]
        n = euler_characteristic(phi.numpy(), walls=(False, False, False))
        a = float(interface_measure(phi, p.W))
        ts.append(t)
        N.append(n)
        R3.append((a / (2.0 * math.pi * n)) ** 3)
    print("t", ts, "N", N, "<R>^3", [round(v, 1) for v in R3])
    late = [i for i, t in enumerate(ts) if t >= 12000]
    assert N[-1] < 0.8 * N[late[0]] and N[late[0]] < 0.5 * N[0]      # droplets keep vanishing
    x = np.array([ts[i] for i in late], dtype=np.float64)
    y = np.array([R3[i] for i in late])
    A = np.stack([np.ones_like(x), x], 1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    r2 = 1.0 - float(((y - A @ coef) ** 2).sum() / ((y - y.mean()) ** 2).sum())
    print("slope of <R>^3 per step", float(coef[1]), "R^2", r2)
    assert coef[1] > 0 and r2 > 0.95
