"""The coupled lattice Boltzmann step in float64 (oracle; test infrastructure only).

One time step follows §3 in the paper's order, on plain [Q, nz, ny, nx]
tensors with TWO buffers and PULL streaming (the CUDA path uses one in-place
buffer; the two schemes share nothing but the equations):

  1. moments of the incoming populations: phi~ = sum g (Eq. 49 without the
     source), c^alpha = sum h^alpha (Eq. 52), p_h = sum f (Eq. 40),
     j = sum f c_k;
  2. mu~ = closure(c, phi~) (Eq. 33) and S = S_phi(phi~, mu~) (Eq. 35);
  3. phi = phi~ + S/2 (Eq. 49), mu = closure(c, phi);
  4. flow only: grad phi and lap phi by the directional differences of
     Eqs. 42-45 on D3Q19 neighbours of phi (all nodes at the same time level),
     F_tot = F_sigma (Eq. 34) + phi g (Boussinesq, §2.5), u = 3 j + F_tot / 2
     (Eq. 41 with rho_0 = 1, c_s^2 = 1/3);
  5. BGK collisions: f with the He-Shan-Doolen forcing and the He-Luo
     equilibrium (Eqs. 36-39), g with its source (Eqs. 46-48), h^alpha with
     the modified equilibrium and phi-dependent rate (Eqs. 50-51);
  6. pull streaming: f_k(x, t+1) = f*_k(x - e_k, t), periodic wrap, or the
     half-way bounce-back f*_{-k}(x, t) when x - e_k lies beyond a wall.

Readings of points the paper leaves open (each stated where it is used):
  * the implicit phi moment of Eq. 49 is evaluated in one explicit pass, the
    source taken at phi~ = sum g;
  * phi, c^A, c^B use D2Q5 (2D), D3Q7 or D3Q19 (3D; D3Q19 is the paper's own
    choice for every equation) with their own c_s^2 (1/3, 1/4, 1/3) wherever
    the equations write c_s^2 for those populations; the flow and the phi
    stencil use D3Q19 (c_s^2 = 1/3, the "3" of Eqs. 43 and 45);
  * the stencil sees phi of step 3 at every neighbour; across a wall it sees
    the mirror value (zero normal gradient, §4.2.4);
  * tau is the paper's, D = tau c_s^2, so the BGK rate is 1/(tau + 1/2);
  * initial populations: g = w phi_0 - w S_0/2, h = h^eq(c_0, mu_0) with
    mu_0 = closure(c_0, phi_0), f = f^eq(p_h = 0, u = 0) shifted by the
    initial forcing, F_0 from the stencil of phi_0.
"""
import torch

from . import model as m
from .lattice import BY_NAME, D3Q19


def _col(vals):
    """Per-direction constants as a [Q, 1, 1, 1] float64 tensor."""
    return torch.tensor(vals, dtype=torch.float64).reshape(-1, 1, 1, 1)


def _mrt_matrix():
    """Rows of d'Humieres' D3Q19 moment basis evaluated on the D3Q19 velocities: density,
    energy, energy square, (momentum, energy flux) per axis, (3 p_xx, pi_xx), (p_ww, pi_ww),
    p_xy, p_yz, p_xz, m_x, m_y, m_z."""
    rows = []
    for k in range(D3Q19.Q):
        cx, cy, cz = D3Q19.e[k]
        c2 = cx * cx + cy * cy + cz * cz
        rows.append([1.0, 19.0 * c2 - 30.0, (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0,
                     cx, (5.0 * c2 - 9.0) * cx, cy, (5.0 * c2 - 9.0) * cy, cz, (5.0 * c2 - 9.0) * cz,
                     3.0 * cx * cx - c2, (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2),
                     cy * cy - cz * cz, (3.0 * c2 - 5.0) * (cy * cy - cz * cz),
                     cx * cy, cy * cz, cx * cz,
                     (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz])
    return [list(r) for r in zip(*rows)]


class OracleLBM:
    """FP64 state of f (D3Q19, flow only), g, h^A, h^B and the step that advances it.

    ``theta`` optionally replaces (D_0, D_1, M_phi) by tensors, so that
    autograd can differentiate through the run: D_pi then serves both
    components of phase pi.
    """

    def __init__(self, params, theta=None):
        self.p = params
        self.ls = BY_NAME[params.lattice]
        self.flow = bool(params.flow)
        self.M_phi = params.M_phi
        self.M = [[params.M[0][0], params.M[0][1]], [params.M[1][0], params.M[1][1]]]
        if theta is not None:
            d0, d1, mphi = theta
            self.M = [[d0, d0], [d1, d1]]
            self.M_phi = mphi
        self.t = 0
        self.f = None
        self.g = self.hA = self.hB = None
        self._masks = {}

    # ---------------------------------------------------------------- geometry
    def _outside(self, e):
        """Boolean field: True where x - e lies beyond a wall (no wrap on walled axes)."""
        key = tuple(e)
        if key not in self._masks:
            nz, ny, nx = self.p.shape
            z = torch.arange(nz).reshape(-1, 1, 1)
            x = torch.arange(nx).reshape(1, 1, -1)
            out = torch.zeros(self.p.shape, dtype=torch.bool)
            if self.p.wall_z and e[2] != 0:
                out = out | ((z - e[2] < 0) | (z - e[2] >= nz)).expand(self.p.shape)
            if self.p.wall_x and e[0] != 0:
                out = out | ((x - e[0] < 0) | (x - e[0] >= nx)).expand(self.p.shape)
            self._masks[key] = out
        return self._masks[key]

    def _stream(self, post, lat):
        """Pull streaming with periodic wrap and half-way bounce-back (step 6)."""
        moved = []
        for k in range(lat.Q):
            ex, ey, ez = lat.e[k]
            pulled = torch.roll(post[k], shifts=(ez, ey, ex), dims=(0, 1, 2))  # post_k(x - e_k)
            if (self.p.wall_z and ez != 0) or (self.p.wall_x and ex != 0):
                pulled = torch.where(self._outside(lat.e[k]), post[lat.opposite(k)], pulled)
            moved.append(pulled)
        return torch.stack(moved)

    def _neighbour(self, phi, e):
        """phi(x + e): periodic on open axes; across a wall (z walls of §4.2.4, x walls of the
        couple geometry) the mirror ghost, i.e. the walled component of e is dropped."""
        ex, ey, ez = e
        nz, ny, nx = self.p.shape
        beyond_z = beyond_x = None
        if self.p.wall_z and ez != 0:
            z = torch.arange(nz).reshape(-1, 1, 1)
            beyond_z = ((z + ez < 0) | (z + ez >= nz)).expand(self.p.shape)
        if self.p.wall_x and ex != 0:
            x = torch.arange(nx).reshape(1, 1, -1)
            beyond_x = ((x + ex < 0) | (x + ex >= nx)).expand(self.p.shape)

        def rolled(dx, dz):
            return torch.roll(phi, shifts=(-dz, -ey, -dx), dims=(0, 1, 2))

        out = rolled(ex, ez)
        if beyond_z is not None:
            out = torch.where(beyond_z, rolled(ex, 0), out)
        if beyond_x is not None:
            out = torch.where(beyond_x, rolled(0, ez), out)
        if beyond_z is not None and beyond_x is not None:
            out = torch.where(beyond_z & beyond_x, rolled(0, 0), out)
        return out

    def gradient_laplacian(self, phi):
        """Eqs. 42-45 on D3Q19: grad = 3 sum_k w_k e_k (phi(x+e_k) - phi(x-e_k)) / 2,
        lap = 3 sum_{k != 0} w_k (phi(x+e_k) - 2 phi(x) + phi(x-e_k))."""
        lat = D3Q19
        grad = [torch.zeros_like(phi) for _ in range(3)]
        lap = torch.zeros_like(phi)
        for k in range(1, lat.Q):
            e = lat.e[k]
            plus = self._neighbour(phi, e)
            minus = self._neighbour(phi, (-e[0], -e[1], -e[2]))
            d1 = (plus - minus) / 2.0                       # Eq. 42
            for a in range(3):
                grad[a] = grad[a] + 3.0 * lat.w[k] * e[a] * d1  # Eq. 43
            lap = lap + 3.0 * lat.w[k] * (plus - 2.0 * phi + minus)  # Eqs. 44-45
        return grad, lap

    def total_force(self, phi):
        """F_tot = F_sigma + F_g: Eq. 34 with grad/lap of Eqs. 43, 45, and F_g = phi * g (§2.5)."""
        p = self.p
        grad, lap = self.gradient_laplacian(phi)
        bracket = m.omega_dw_prime(phi) / p.W ** 2 - lap
        F = [1.5 * p.sigma * p.W * bracket * grad[a] + phi * p.g[a] for a in range(3)]
        return F

    # ---------------------------------------------------------------- moments
    def _source(self, phi, muA, muB):
        if self.p.source_off:
            return torch.zeros_like(phi)
        p = self.p
        return m.source_phi(phi, (muA, muB), p.W, p.lam, self.M_phi, p.c_eq)

    def macroscopic(self):
        """Steps 1-4 on the current (incoming) populations; returns a dict of fields."""
        p = self.p
        ce = p.c_eq
        phi_t = self.g.sum(0)                                        # Eq. 49, sum g
        cA = self.hA.sum(0)                                          # Eq. 52
        cB = self.hB.sum(0)
        muA_t = m.mu_closure(cA, phi_t, ce[0][0], ce[1][0])          # Eq. 33 at phi~
        muB_t = m.mu_closure(cB, phi_t, ce[0][1], ce[1][1])
        S = self._source(phi_t, muA_t, muB_t)                        # Eq. 35
        phi = phi_t + 0.5 * S                                        # Eq. 49
        muA = m.mu_closure(cA, phi, ce[0][0], ce[1][0])              # Eq. 33 at phi
        muB = m.mu_closure(cB, phi, ce[0][1], ce[1][1])
        out = dict(phi_t=phi_t, cA=cA, cB=cB, S=S, phi=phi, muA=muA, muB=muB)
        if self.flow:
            lat = D3Q19
            ph = self.f.sum(0)                                       # Eq. 40
            j = [sum(self.f[k] * lat.e[k][a] for k in range(lat.Q)) for a in range(3)]
            F = self.total_force(phi)
            u = [j[a] / lat.cs2 + 0.5 * F[a] for a in range(3)]     # Eq. 41, rho_0 = 1
            out.update(p=ph, u=u, F=F)
        else:
            z = torch.zeros_like(phi)
            out.update(p=z, u=[z, z, z], F=[z, z, z])
        return out

    # ---------------------------------------------------------------- init
    def init(self, phi0, cA0, cB0):
        """Initial populations at rest (see the module docstring)."""
        p = self.p
        ce = p.c_eq
        ls = self.ls
        w = _col(ls.w)
        phi0 = phi0.to(torch.float64)
        cA0 = cA0.to(torch.float64)
        cB0 = cB0.to(torch.float64)
        muA = m.mu_closure(cA0, phi0, ce[0][0], ce[1][0])
        muB = m.mu_closure(cB0, phi0, ce[0][1], ce[1][1])
        S0 = self._source(phi0, muA, muB)
        self.g = w * phi0 - w * S0 / 2.0                             # Eq. 47 at u = 0
        zero = [torch.zeros_like(phi0)] * 3
        self.hA = self._h_eq(cA0, muA, zero)                         # Eq. 51 at u = 0
        self.hB = self._h_eq(cB0, muB, zero)
        if self.flow:
            F0 = self.total_force(phi0)
            Fk = self._forcing(zero, F0)
            self.f = self._f_eq(torch.zeros_like(phi0), zero, Fk)   # Eq. 39, p_h = 0, u = 0
        self.t = 0

    # ---------------------------------------------------------------- equilibria
    def _h_eq(self, c, mu, u):
        """Eq. 51: h_0 = c - (1 - w_0) mu; h_k = w_k mu + w_k c (c_k . u) / c_s^2."""
        ls = self.ls
        parts = [c - (1.0 - ls.w[0]) * mu]
        for k in range(1, ls.Q):
            cu = sum(ls.e[k][a] * u[a] for a in range(3))
            parts.append(ls.w[k] * mu + ls.w[k] * c * cu / ls.cs2)
        return torch.stack(parts)

    def _forcing(self, u, F):
        """Eqs. 37-38: F_k = Gamma_k (c_k - u) . F, Gamma_k = w_k [1 + cu/cs2 + cu^2/(2 cs2^2) - u^2/(2 cs2)]."""
        lat = D3Q19
        usq = sum(u[a] * u[a] for a in range(3))
        parts = []
        for k in range(lat.Q):
            cu = sum(lat.e[k][a] * u[a] for a in range(3))
            gamma = lat.w[k] * (1.0 + cu / lat.cs2 + cu ** 2 / (2.0 * lat.cs2 ** 2) - usq / (2.0 * lat.cs2))
            cF = sum((lat.e[k][a] - u[a]) * F[a] for a in range(3))
            parts.append(gamma * cF)
        return torch.stack(parts)

    def _f_eq(self, ph, u, Fk):
        """Eq. 39 (rho_0 = 1): w_k [p_h + c_s^2 (cu/cs2 + cu^2/(2 cs2^2) - u^2/(2 cs2))] - F_k / 2."""
        lat = D3Q19
        usq = sum(u[a] * u[a] for a in range(3))
        parts = []
        for k in range(lat.Q):
            cu = sum(lat.e[k][a] * u[a] for a in range(3))
            parts.append(lat.w[k] * (ph + lat.cs2 * (cu / lat.cs2 + cu ** 2 / (2.0 * lat.cs2 ** 2)
                                                     - usq / (2.0 * lat.cs2))) - 0.5 * Fk[k])
        return torch.stack(parts)

    def _trt(self, f, f_eq, Fk, om_plus):
        """Two-relaxation-time collision of the flow populations (the TRT operator that the
        paper names as an alternative to BGK, §3): the parts of f - f^eq that are even and
        odd under k -> opp(k) relax at omega+ and omega-. omega+ is the BGK rate of Eq. 36
        (it sets nu); omega- follows from the magic parameter
        Lambda = (1/omega+ - 1/2)(1/omega- - 1/2). f^eq is Eq. 39 with its -F_k/2, and F_k is
        added as in Eq. 36, so omega- = omega+ gives back the BGK update exactly."""
        lam = self.p.trt_magic
        om_minus = 1.0 / (lam / (1.0 / om_plus - 0.5) + 0.5)
        opp = [D3Q19.opposite(k) for k in range(D3Q19.Q)]
        d = f - f_eq
        d_bar = d[opp]
        even = 0.5 * (d + d_bar)
        odd = 0.5 * (d - d_bar)
        return f - om_plus * even - om_minus * odd + Fk

    def _mrt(self, f, f_eq, Fk, om_nu):
        """Multiple-relaxation-time collision of the flow populations (the MRT operator the
        paper names as an alternative to BGK, §3), on d'Humieres' orthogonal D3Q19 moment
        basis: the moments of f - f^eq relax at their own rates, f* = f - M^-1 S M (f - f^eq)
        + F_k. The shear moments (3p_xx, p_ww, p_xy, p_yz, p_xz) relax at omega_nu of Eq. 36
        (they set nu); energy, energy square, energy flux, the fourth-order pi and the third-
        order m moments at the rates of ``mrt_rates`` = (s_e, s_eps, s_q, s_pi, s_m); the
        conserved density and momentum carry no non-equilibrium part. f^eq keeps the -F_k/2 of
        Eq. 39 and F_k is added as in Eq. 36; M^-1 = M^T diag(1 / |row|^2)."""
        M = torch.tensor(_mrt_matrix(), dtype=torch.float64)
        norms = (M * M).sum(1)
        s_e, s_eps, s_q, s_pi, s_m = self.p.mrt_rates
        rates = torch.tensor([om_nu, s_e, s_eps, om_nu, s_q, om_nu, s_q, om_nu, s_q, om_nu, s_pi, om_nu, s_pi,
                              om_nu, om_nu, om_nu, s_m, s_m, s_m], dtype=torch.float64)
        dm = torch.tensordot(M, f - f_eq, dims=1)
        relax = torch.tensordot(M.T, (rates / norms).reshape(-1, 1, 1, 1) * dm, dims=1)
        return f - relax + Fk

    # ---------------------------------------------------------------- step
    def step(self, n=1):
        for _ in range(n):
            self._one_step()
        return self

    def _one_step(self):
        p = self.p
        ls = self.ls
        mac = self.macroscopic()
        phi, S, u = mac["phi"], mac["S"], mac["u"]
        w = _col(ls.w)

        # Eqs. 46-48: g* = g - (g - g^eq)/(tau_g + 1/2) + G_k, g^eq = w phi (1 + c.u/cs2) - G_k/2, G_k = w S
        om_g = m.relaxation_rate(self.M_phi, ls.cs2)
        cu_s = torch.stack([sum(ls.e[k][a] * u[a] for a in range(3)) for k in range(ls.Q)])
        G = w * S
        g_eq = w * phi * (1.0 + cu_s / ls.cs2) - 0.5 * G
        g_post = self.g - om_g * (self.g - g_eq) + G

        # Eqs. 50-51 with tau_h^alpha(phi) from M^alpha(phi) = tau c_s^2 (§3.3, §2.3)
        h_post = []
        for a, (h, c, mu) in enumerate(((self.hA, mac["cA"], mac["muA"]), (self.hB, mac["cB"], mac["muB"]))):
            om_h = m.relaxation_rate(m.mobility(phi, self.M[0][a], self.M[1][a]), ls.cs2)
            h_eq = self._h_eq(c, mu, u)
            h_post.append(h - om_h * (h - h_eq))

        if self.flow:
            # Eqs. 36-39, tau_f = nu / c_s^2
            Fk = self._forcing(u, mac["F"])
            f_eq = self._f_eq(mac["p"], u, Fk)
            om_f = m.relaxation_rate(p.nu, D3Q19.cs2)
            if p.collision == "TRT":
                f_post = self._trt(self.f, f_eq, Fk, om_f)
            elif p.collision == "MRT":
                f_post = self._mrt(self.f, f_eq, Fk, om_f)
            else:
                f_post = self.f - om_f * (self.f - f_eq) + Fk
            self.f = self._stream(f_post, D3Q19)
        self.g = self._stream(g_post, ls)
        self.hA = self._stream(h_post[0], ls)
        self.hB = self._stream(h_post[1], ls)
        self.t += 1

    # ---------------------------------------------------------------- outputs
    def fields(self):
        """phi, mu^A, mu^B, c^A, c^B, p_h, u_x, u_y, u_z at the current time level."""
        mac = self.macroscopic()
        return dict(phi=mac["phi"], muA=mac["muA"], muB=mac["muB"], cA=mac["cA"], cB=mac["cB"],
                    p=mac["p"], ux=mac["u"][0], uy=mac["u"][1], uz=mac["u"][2], S=mac["S"],
                    phi_t=mac["phi_t"])

    def sums(self):
        """Global FP64 diagnostics: sum phi, sum c^A, sum c^B, sum p_h, sum S, max |u|, sum g."""
        mac = self.macroscopic()
        umag = torch.sqrt(sum(mac["u"][a] ** 2 for a in range(3)))
        return dict(phi=float(mac["phi"].sum()), cA=float(mac["cA"].sum()), cB=float(mac["cB"].sum()),
                    p=float(mac["p"].sum()), S=float(mac["S"].sum()), umax=float(umag.max()),
                    g=float(mac["phi_t"].sum()))

    def populations(self):
        """Incoming populations at the current time level: dict of [Q, nz, ny, nx] tensors."""
        d = dict(g=self.g, hA=self.hA, hB=self.hB)
        if self.flow:
            d["f"] = self.f
        return d


def run(params, phi0, cA0, cB0, steps):
    """Convenience: initialise, advance ``steps`` steps, return the oracle."""
    o = OracleLBM(params)
    o.init(phi0, cA0, cB0)
    o.step(steps)
    return o
