"""Closed forms that pin the oracle (test infrastructure only).

* ``couple_solution`` - the self-similar ternary diffusion couple of §4.1
  (Eqs. 53-61): each side diffuses mu with its own diffusivity, the interface
  moves as x_I = xi sqrt(t) (Eq. 59), mu takes the erfc profiles of Eq. 60
  with a common interface value mu_int, and (xi, mu_int^A, mu_int^B) solve
  the two interface mass balances (Eq. 55, flux -D d mu/dx on each side, c
  jumping by the equilibrium gap across the interface) together with the
  flat-interface Gibbs-Thomson condition Delta omega(mu_int) = 0 (Eq. 61, i.e.
  Eq. 25 with kappa = beta = 0). Eq. 60 writes one mobility per component; a
  side-dependent diffusivity enters the same way through each side's erfc.
* Linear decay rates of a Fourier mode for diffusion (textbook: the heat
  equation, amplitude exp(-D k^2 t)) and for a shear wave (exp(-nu k^2 t)).
* Plane Poiseuille flow between walls at -1/2 and H - 1/2 driven by a body
  force F: u(z) = F (z + 1/2)(H - 1/2 - z) / (2 nu).
"""
import math
import numpy as np
from scipy.optimize import fsolve
from scipy.special import erfc

from . import model as m


def couple_solution(mu_left, mu_right, D_left, D_right, c_eq_left, c_eq_right, c_eq, guess=None):
    """Solve the diffusion couple of §4.1.

    ``mu_left``/``mu_right`` are (mu^A, mu^B) far left / far right,
    ``D_left``/``D_right`` the per-component diffusivities on each side,
    ``c_eq_left``/``c_eq_right`` the equilibrium compositions of the phase on
    each side (c = mu + c_eq in a bulk phase, Eq. 24), ``c_eq`` = (c_0^eq,
    c_1^eq) for Delta omega. Returns (xi, mu_int) with mu_int = (A, B).
    """
    def residual(v):
        xi, mA, mB = v
        mu_int = (mA, mB)
        res = []
        for a in range(2):
            DL, DR = D_left[a], D_right[a]
            AL = (mu_int[a] - mu_left[a]) / erfc(-xi / (2.0 * math.sqrt(DL)))
            AR = (mu_int[a] - mu_right[a]) / erfc(xi / (2.0 * math.sqrt(DR)))
            # sqrt(t) * (D_R dmu/dx|+ - D_L dmu/dx|-) at x = xi sqrt(t)
            flux_jump = (-AR * math.sqrt(DR / math.pi) * math.exp(-xi ** 2 / (4.0 * DR))
                         - AL * math.sqrt(DL / math.pi) * math.exp(-xi ** 2 / (4.0 * DL)))
            jump_c = c_eq_left[a] - c_eq_right[a]             # c(x_I^-) - c(x_I^+)
            res.append(0.5 * xi * jump_c - flux_jump)         # Eq. 55 times sqrt(t)
        res.append(m.delta_omega(mu_int, c_eq))               # Eq. 61
        return res

    if guess is None:
        guess = (0.0, 0.5 * (mu_left[0] + mu_right[0]), 0.5 * (mu_left[1] + mu_right[1]))
    sol, info, ier, msg = fsolve(residual, guess, full_output=True, xtol=1e-14)
    if ier != 1:
        raise RuntimeError(f"diffusion couple solve failed: {msg}")
    return float(sol[0]), (float(sol[1]), float(sol[2]))


def couple_mu_profile(x, t, xi, mu_int, mu_left, mu_right, D_left, D_right, x0=0.0):
    """Eq. 60: mu^alpha(x, t) for both components; x measured from the initial interface x0."""
    x = np.asarray(x, dtype=np.float64) - x0
    xI = xi * math.sqrt(t)
    out = []
    for a in range(2):
        DL, DR = D_left[a], D_right[a]
        left = mu_left[a] + (mu_int[a] - mu_left[a]) * erfc(-x / (2.0 * math.sqrt(DL * t))) \
            / erfc(-xi / (2.0 * math.sqrt(DL)))
        right = mu_right[a] + (mu_int[a] - mu_right[a]) * erfc(x / (2.0 * math.sqrt(DR * t))) \
            / erfc(xi / (2.0 * math.sqrt(DR)))
        out.append(np.where(x < xI, left, right))
    return out


def diffusion_decay(D, k, t):
    """Amplitude factor of a Fourier mode sin(k x) under d_t c = D lap c."""
    return math.exp(-D * k * k * t)


def poiseuille(z, H, F, nu):
    """Steady body-force-driven channel profile with walls at z = -1/2 and z = H - 1/2."""
    z = np.asarray(z, dtype=np.float64)
    return F * (z + 0.5) * (H - 0.5 - z) / (2.0 * nu)
