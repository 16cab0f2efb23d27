"""Pointwise model functions of §2 (oracle copy; test infrastructure only).

All arguments are float64 tensors or Python floats; nothing is fused or
rearranged beyond what the equations state, so each line can be read against
the paper.
"""
import math


def omega_dw(phi):
    """Double well omega_dw(phi) = 8 phi^2 (1 - phi)^2 (§2.2, after Eq. 12)."""
    return 8.0 * phi ** 2 * (1.0 - phi) ** 2


def omega_dw_prime(phi):
    """d omega_dw / d phi = 16 phi (1 - phi) (1 - 2 phi)."""
    return 16.0 * phi * (1.0 - phi) * (1.0 - 2.0 * phi)


def p_interp(phi):
    """Interpolation function p(phi) = 3 phi^2 - 2 phi^3 (§2.2, after Eq. 16)."""
    return 3.0 * phi ** 2 - 2.0 * phi ** 3


def p_prime(phi):
    """p'(phi) = 6 phi (1 - phi)."""
    return 6.0 * phi * (1.0 - phi)


def mu_closure(c, phi, c0_eq, c1_eq):
    """Eq. 24 / Eq. 33: mu = c - p(1 - phi) c_0^eq - p(phi) c_1^eq (one component)."""
    return c - p_interp(1.0 - phi) * c0_eq - p_interp(phi) * c1_eq


def grand_potential(mu, c_eq_phase):
    """Eq. 18: dimensionless grand potential of one phase,
    omega_pi = -1/2 sum_alpha (mu_alpha^2 + 2 mu_alpha c_pi^{alpha,eq}); ``mu`` = (mu_A, mu_B)."""
    return -0.5 * sum(mu[a] ** 2 + 2.0 * mu[a] * c_eq_phase[a] for a in range(2))


def delta_omega(mu, c_eq):
    """Eq. 20: Delta omega = omega_0 - omega_1 = -sum_alpha mu_alpha (c_0^{alpha,eq} - c_1^{alpha,eq})."""
    return -sum(mu[a] * (c_eq[0][a] - c_eq[1][a]) for a in range(2))


def source_phi(phi, mu, W, lam, M_phi, c_eq):
    """Eq. 35: S_phi = -(1/tau_phi) omega_dw'(phi) + (lambda/tau_phi) p'(phi) Delta omega,
    with 1/tau_phi = M_phi / W^2 (§2.2, M_phi = W^2 / tau_phi)."""
    inv_tau_phi = M_phi / W ** 2
    return -inv_tau_phi * omega_dw_prime(phi) + lam * inv_tau_phi * p_prime(phi) * delta_omega(mu, c_eq)


def mobility(phi, M_phase0, M_phase1):
    """§2.3: M^alpha(phi) = M_0^alpha (1 - phi) + M_1^alpha phi."""
    return M_phase0 * (1.0 - phi) + M_phase1 * phi


def relaxation_rate(D, cs2):
    """BGK rate 1 / (tau + 1/2) with D = tau c_s^2 dt (§3, Eqs. 36, 46, 50 and the
    relations stated beside them), dt = 1."""
    return 1.0 / (D / cs2 + 0.5)


def lambda_star(W, M_phi, c_eq, M):
    """Eq. 27 solved for beta = 0: lambda* = (2/3) W / (M_phi (19/120) sum W (dc)^2 / M^alpha).
    ``M`` = (M^A, M^B)."""
    s = sum(W * (c_eq[0][a] - c_eq[1][a]) ** 2 / M[a] for a in range(2))
    return (2.0 / 3.0) * W / (M_phi * (19.0 / 120.0) * s)


def kinetic_coefficient(W, lam, M_phi, c_eq, M):
    """Eq. 27: beta."""
    s = sum(W * (c_eq[0][a] - c_eq[1][a]) ** 2 / M[a] for a in range(2))
    return (2.0 / 3.0) * W / (lam * M_phi) - (19.0 / 120.0) * s


def capillary_length(W, lam):
    """Eq. 26: delta = (2/3) W / lambda."""
    return (2.0 / 3.0) * W / lam


def tanh_profile(x, W):
    """Eq. 13: phi_0(x) = (1 + tanh(2 x / W)) / 2."""
    if isinstance(x, float):
        return 0.5 * (1.0 + math.tanh(2.0 * x / W))
    return 0.5 * (1.0 + (2.0 * x / W).tanh())
