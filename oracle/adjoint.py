"""Gradient of a final-field misfit through the FP64 oracle (test infrastructure only).

The misfit of a run of ``steps`` coupled steps from phi_0 is
    L = 1/2 sum_x [(phi - phi*)^2 + (mu^A - mu^A*)^2 + (mu^B - mu^B*)^2]
with the fields of the final time level (Eqs. 49 and 33). Its gradient with
respect to theta = (D_0, D_1, M_phi) and to phi_0 is taken by reverse-mode
automatic differentiation through every operation of ``oracle.lbm`` in
float64, which is the exact discrete adjoint of the oracle's step. The initial
compositions are the piecewise-constant map of Eq. 66, whose derivative with
respect to phi_0 vanishes almost everywhere, so c_0 enters as a constant.
"""
import torch

from .lbm import OracleLBM


def misfit(fields, target):
    return 0.5 * (((fields["phi"] - target["phi"]) ** 2).sum()
                  + ((fields["muA"] - target["muA"]) ** 2).sum()
                  + ((fields["muB"] - target["muB"]) ** 2).sum())


def forward_misfit(params, theta, phi0, cA0, cB0, steps, target):
    """L at theta = (D_0, D_1, M_phi) (floats); no gradient."""
    with torch.no_grad():
        th = tuple(torch.tensor(v, dtype=torch.float64) for v in theta)
        o = OracleLBM(params, theta=th)
        o.init(phi0, cA0, cB0)
        o.step(steps)
        return float(misfit(o.fields(), target))


def misfit_gradient(params, theta, phi0, cA0, cB0, steps, target):
    """Return (L, dL/dtheta [3], dL/dphi_0 [nz, ny, nx])."""
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    p0 = phi0.detach().to(torch.float64).clone().requires_grad_(True)
    o = OracleLBM(params, theta=(th[0], th[1], th[2]))
    o.init(p0, cA0.detach(), cB0.detach())
    o.step(steps)
    L = misfit(o.fields(), target)
    L.backward()
    return float(L.detach()), th.grad.detach().clone(), p0.grad.detach().clone()


def target_fields(params, theta, phi0, cA0, cB0, steps):
    """phi, mu^A, mu^B after ``steps`` steps at theta (the synthetic target)."""
    with torch.no_grad():
        th = tuple(torch.tensor(v, dtype=torch.float64) for v in theta)
        o = OracleLBM(params, theta=th)
        o.init(phi0, cA0, cB0)
        o.step(steps)
        f = o.fields()
        return {k: f[k].clone() for k in ("phi", "muA", "muB")}
