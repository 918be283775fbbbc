"""Discrete adjoint of the implicit MGFLD step (CPU oracle).

TEST INFRASTRUCTURE ONLY (like mgfld_oracle): imported by tests and the benchmark's CPU
baseline, never by the product path.

Objective (reading R11 of mgfld_oracle): J = sum over steps of the energy deposited in matter by
nu_e and nubar_e between 100 and 300 km.  Parameters: the per-(species, group) opacity scales s
(multiplying kappa_abs and kappa_scat) and the initial occupation psi^0.

One implicit step maps p = (psi^n, Ye^n, T^n, s) to x = (psi^{n+1}, Ye^{n+1}) through
G(x; p) = 0 (Eqs. a58, a59, a62a with the coefficients frozen at p), then to T^{n+1}
(Eq. a62b and the EoS) and to the step's heating H.  For upstream gradients x_bar, T_bar,
the implicit-function theorem gives
    J_x^T mu = x_bar + T_bar dT/dx + dH/dx,     p_bar = T_bar dT/dp + dH/dp - mu^T dG/dp,
where J_x = dG/dx is the exact Jacobian of the oracle (mgfld_oracle.jacobian) and the partial
derivatives with respect to p (through every frozen coefficient: NES kernels, emissivity,
mean free path, limiter, neutrinosphere, ghost) are taken by reverse-mode automatic
differentiation of a torch float64 restatement of the same formulas.  Steps are chained in
reverse order from stored states.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import mgfld_oracle as O

T64 = torch.float64


def _t(a):
    return torch.as_tensor(np.array(a, dtype=np.float64), dtype=T64)


# ---------------------------------------------------------------------------- torch restatement

def _mu_nue(rho, T, ye, eos):
    n_e = rho * ye / eos.m_b
    n_n = rho * (1.0 - ye) / eos.m_b
    lam3 = (O.HC * O.HC / (2.0 * np.pi * eos.mb_c2 * T)) ** eos.e_coef
    mu_e = eos.gamma1 * eos.f1 * n_e ** (eos.gamma1 - 1.0) * (eos.m_b / eos.rho_0) ** (eos.gamma1 - 4.0 / 3.0)
    mu_n = eos.gamma2 * eos.f2 * n_n ** (eos.gamma2 - 1.0) + T * torch.log(n_n * lam3 / eos.g_n)
    mu_p = T * torch.log(n_e * lam3 / eos.g_p)
    return mu_e + mu_p - mu_n


def _e_cold(rho, ye, eos):
    n_b = rho / eos.m_b
    n_e = rho * ye / eos.m_b
    n_n = rho * (1.0 - ye) / eos.m_b
    return (eos.f1 * n_e ** eos.gamma1 * (eos.m_b / eos.rho_0) ** (eos.gamma1 - 4.0 / 3.0)
            + eos.f2 * n_n ** eos.gamma2) / n_b


class Step:
    """Differentiable coefficient chain of one step at p = (psi_n, ye_n, T_n, scale)."""

    def __init__(self, prob, psi_n, ye_n, T_n, scale):
        eos = prob.get('eos') or O.EosParams()
        self.eos = eos
        self.prob = prob
        r_edge = _t(prob['r_edge'])
        n_ray, n_r = r_edge.shape[0], r_edge.shape[1] - 1
        lapse = prob.get('lapse')
        a = torch.ones(n_ray, n_r, dtype=T64) if lapse is None else _t(lapse)
        self.a = a
        self.rho = _t(prob['rho'])
        self.dt = float(prob['dt'])
        self.bc = int(prob.get('outer_bc', O.BC_GHOST))
        self.psi_n, self.ye_n, self.T_n, self.scale = psi_n, ye_n, T_n, scale
        self.rc = 0.5 * (r_edge[:, :-1] + r_edge[:, 1:])
        self.area = 4.0 * np.pi * r_edge ** 2
        self.vol = 4.0 * np.pi * (r_edge[:, 1:] ** 3 - r_edge[:, :-1] ** 3) / 3.0
        self.r_edge = r_edge
        E, dE = O.group_centres(prob['e_edge'])
        self.E, self.dE = _t(E), _t(dE)
        inv_a = 1.0 / a
        self.eps = self.E[None, None, :] * inv_a[:, :, None]
        deps = self.dE[None, None, :] * inv_a[:, :, None]
        self.w = self.eps ** 2 * deps
        self.kabs = _t(prob['kappa_abs']) * scale[None, :, None, :]
        self.kscat = _t(prob['kappa_scat']) * scale[None, :, None, :]
        coef = prob.get('nes_coef')
        coef = torch.zeros(n_ray, n_r, dtype=T64) if coef is None else _t(coef)
        d = self.eps[:, :, :, None] - self.eps[:, :, None, :]
        Tb = T_n[:, :, None, None]
        n_e = self.eps.shape[2]
        k = torch.arange(n_e)
        down = (k[None, :] <= k[:, None])[None, None]
        self.phi_out = torch.where(down, coef[:, :, None, None] * torch.exp(-torch.where(down, d, 0.0 * d) / Tb),
                                   coef[:, :, None, None] * torch.exp(2.0 * torch.where(down, 0.0 * d, d) / Tb))
        self.phi_in = torch.swapaxes(self.phi_out, 2, 3)
        mu_q_n = self._species_mu(ye_n)
        j_n = self._emissivity(mu_q_n)
        inv_lam = self.kabs + j_n + self.kscat + self._nes_mfp(psi_n)
        self.lam = 1.0 / inv_lam
        self.r_nu = self._neutrinosphere()
        r_i = self.rc[:, -1][:, None, None]
        r_g = (2.0 * r_edge[:, -1] - self.rc[:, -1])[:, None, None]
        rn = torch.minimum(self.r_nu, r_i)
        self.ghost = (r_i ** 2 - 0.25 * rn ** 2) / (r_g ** 2 - 0.25 * rn ** 2)
        self.alpha = self._edges()
        self.e_n = _e_cold(self.rho, ye_n, eos) + eos.e_coef * T_n

    def _species_mu(self, ye):
        m = _mu_nue(self.rho, self.T_n, ye, self.eos)
        z = torch.zeros_like(m)
        return torch.stack([m, -m, z, z], dim=1)

    def _emissivity(self, mu_q):
        x = (mu_q[:, :, :, None] - self.eps[:, None, :, :]) / self.T_n[:, None, :, None]
        return self.kabs * torch.exp(torch.clamp(x, max=O.EXP_CAP))

    def _nes_mfp(self, psi):
        return O.C_NES * (torch.einsum('rikm,rim,rqim->rqik', self.phi_in, self.w, psi)
                          + torch.einsum('rikm,rim,rqim->rqik', self.phi_out, self.w, 1.0 - psi))

    def _neutrinosphere(self):
        lam = self.lam
        dr = (self.r_edge[:, 1:] - self.r_edge[:, :-1])[:, None, :, None]
        dtau = dr / lam
        tau_out = torch.flip(torch.cumsum(torch.flip(dtau, [2]), 2), [2]) - dtau
        tau_in = tau_out + dtau
        hit = (tau_in >= 2.0 / 3.0).detach().numpy()
        n_ray, n_s, n_r, n_e = lam.shape
        out = []
        for r in range(n_ray):
            row = []
            for q in range(n_s):
                for k in range(n_e):
                    idx = np.nonzero(hit[r, q, :, k])[0]
                    if idx.size == 0:
                        row.append(self.r_edge[r, 0] + 0.0 * lam[r, q, 0, k])
                    else:
                        i = int(idx[-1])
                        row.append(self.r_edge[r, i + 1] - (2.0 / 3.0 - tau_out[r, q, i, k]) * lam[r, q, i, k])
            out.append(torch.stack(row).reshape(n_s, n_e))
        return torch.stack(out)

    def _edges(self):
        psi, lam = self.psi_n, self.lam
        psi_r = torch.cat([psi[:, :, 1:], (self.ghost * psi[:, :, -1])[:, :, None]], dim=2)
        lam_r = torch.cat([lam[:, :, 1:], lam[:, :, -1:]], dim=2)
        rc_r = torch.cat([self.rc[:, 1:], (2.0 * self.r_edge[:, -1] - self.rc[:, -1])[:, None]], dim=1)
        a_r = torch.cat([self.a[:, 1:], self.a[:, -1:]], dim=1)
        lam_e = torch.sqrt(lam * lam_r)
        dpsi = psi_r - psi
        dR = (rc_r - self.rc)[:, None, :, None]
        psi_e = 0.5 * (psi + psi_r)
        x = lam_e * torch.abs(dpsi / dR) / 3.0
        r_e = self.r_edge[:, 1:][:, None, :, None]
        r_nu = self.r_nu[:, :, None, :]
        safe_pe = torch.where(psi_e > 1e-300, psi_e, torch.ones_like(psi_e))
        f_int = safe_pe / (safe_pe + x)
        outside = r_e > r_nu
        mu = torch.sqrt(torch.where(outside, 1.0 - (r_nu / r_e) ** 2, torch.ones_like(r_nu / r_e)))
        h = 0.5 * (1.0 + mu)
        # min(F_intrp, F_geom) taken as the branch it selects (F_geom < F_intrp exactly when
        # h psi_e < (1 - h) x): the same value, and the unselected quotient, whose denominator
        # may be tiny, stays out of the derivative.
        use_geo = (outside & (h * safe_pe < (1.0 - h) * x)).detach()
        safe_x = torch.where(use_geo, x, torch.ones_like(x))
        F = torch.where(use_geo, h * safe_pe / safe_x, f_int)
        F = torch.where(dpsi == 0.0, torch.ones_like(F), F)
        F = torch.where(psi_e <= 1e-300, torch.zeros_like(F), F)
        D = lam_e * F / (3.0 * dR)
        a_e = 0.5 * (self.a + a_r)
        alpha = self.area[:, 1:][:, None, :, None] * D / (a_e ** 2)[:, None, :, None]
        if self.bc == O.BC_REFLECT:
            alpha = torch.cat([alpha[:, :, :-1], torch.zeros_like(alpha[:, :, -1:])], dim=2)
        return alpha

    # ---- residual and outputs at x = (psi, ye)
    def sources(self, psi, ye):
        mu_q = self._species_mu(ye)
        j = self._emissivity(mu_q)
        s_ae = j * (1.0 - psi) - self.kabs * psi
        gain = torch.einsum('rikm,rim,rqim->rqik', self.phi_in, self.w, psi)
        loss = torch.einsum('rikm,rim,rqim->rqik', self.phi_out, self.w, 1.0 - psi)
        s_nes = O.C_NES * ((1.0 - psi) * gain - psi * loss)
        return s_ae + s_nes, s_ae

    def residual(self, psi, ye):
        S, s_ae = self.sources(psi, ye)
        a = self.a[:, None, :, None]
        psi_r = torch.cat([psi[:, :, 1:], (self.ghost * psi[:, :, -1])[:, :, None]], dim=2)
        flux_out = -self.alpha * (psi_r - psi)
        flux_in = torch.cat([torch.zeros_like(flux_out[:, :, :1]), flux_out[:, :, :-1]], dim=2)
        pre = (self.a ** 2 / self.vol)[:, None, :, None]
        G = (psi - self.psi_n) / (a * O.C_LIGHT * self.dt) + pre * (flux_out - flux_in) - S
        sign = torch.as_tensor(O.LEPTON_SIGN, dtype=T64)
        lep = torch.einsum('q,rik,rqik->ri', sign, self.w, s_ae)
        GY = (ye - self.ye_n) / (self.a * O.C_LIGHT * self.dt) + O.FOUR_PI_HC3 * (self.eos.m_b / self.rho) * lep
        return G, GY

    def outputs(self, psi, ye, r_lo=1.0e7, r_hi=3.0e7):
        S, _ = self.sources(psi, ye)
        stat = torch.as_tensor(O.STAT_WEIGHT, dtype=T64)
        de = -(self.a * O.C_LIGHT * self.dt) * O.FOUR_PI_HC3 * (self.eos.m_b / self.rho) * torch.einsum(
            'q,rik,rqik->ri', stat, self.w * self.eps, S)
        e_new = self.e_n + de
        T_new = (e_new - _e_cold(self.rho, ye, self.eos)) / self.eos.e_coef
        mask = ((self.rc >= r_lo) & (self.rc <= r_hi)).to(T64)
        heat = -(self.a * O.C_LIGHT * self.dt) * self.vol * O.FOUR_PI_HC3 * torch.einsum(
            'rik,rqik->ri', self.w * self.eps, S[:, :2])
        return T_new, torch.sum(heat * mask, dim=1)


# ---------------------------------------------------------------------------- adjoint

def step_vjp(prob, psi_n, ye_n, T_n, scale, psi1, ye1, psi1_bar, ye1_bar, T1_bar, heat_weight=1.0):
    """Gradients of L = <psi1_bar, psi1> + <ye1_bar, ye1> + <T1_bar, T1> + heat_weight * sum(H)
    with respect to (psi_n, ye_n, T_n, scale), for one step whose root is (psi1, ye1)."""
    if prob.get('u') is not None or prob.get('pair_coef') is not None:
        raise NotImplementedError('the shock (Eqs. a91-a99) and pair (Eq. d14) terms are not differentiated')
    p = [_t(psi_n).requires_grad_(), _t(ye_n).requires_grad_(), _t(T_n).requires_grad_(),
         _t(scale).requires_grad_()]
    st = Step(prob, *p)
    x_psi = _t(psi1).requires_grad_()
    x_ye = _t(ye1).requires_grad_()
    T1, H = st.outputs(x_psi, x_ye)
    L_out = torch.sum(_t(T1_bar) * T1) + heat_weight * torch.sum(H)
    # Explicit parts: derivative of the outputs with respect to x and p.
    gx = torch.autograd.grad(L_out, [x_psi, x_ye] + p, retain_graph=False, allow_unused=True)
    dx_psi = gx[0].numpy() + np.asarray(psi1_bar, dtype=np.float64)
    dx_ye = gx[1].numpy() + np.asarray(ye1_bar, dtype=np.float64)
    explicit = [g.numpy() if g is not None else np.zeros(tuple(t.shape)) for g, t in zip(gx[2:], p)]
    # Transposed solve with the exact coupled Jacobian at the root (block form of Eq. a62ae).
    f = O.setup_step(dict(prob, scale=np.asarray(scale)), psi_n, ye_n, T_n)
    A, Bm, Bp = O.jacobian(f, np.asarray(psi1), np.asarray(ye1))
    At = np.swapaxes(A, 2, 3)
    Bm_t = np.zeros_like(Bm)
    Bp_t = np.zeros_like(Bp)
    Bm_t[:, 1:] = Bp[:, :-1]           # row i of J^T couples to i-1 through Bp_{i-1}
    Bp_t[:, :-1] = Bm[:, 1:]           # and to i+1 through Bm_{i+1}
    mu = O.block_thomas(At, Bm_t, Bp_t, O.pack(dx_psi, dx_ye))
    mu_psi, mu_ye = O.unpack(mu, f.n_e)
    # -mu^T dG/dp by reverse mode through the coefficient chain.
    p2 = [_t(psi_n).requires_grad_(), _t(ye_n).requires_grad_(), _t(T_n).requires_grad_(),
          _t(scale).requires_grad_()]
    st2 = Step(prob, *p2)
    G, GY = st2.residual(_t(psi1), _t(ye1))
    inner = torch.sum(_t(mu_psi) * G) + torch.sum(_t(mu_ye) * GY)
    gp = torch.autograd.grad(inner, p2, allow_unused=True)
    out = []
    for e, g, t in zip(explicit, gp, p2):
        out.append(e - (g.numpy() if g is not None else np.zeros(tuple(t.shape))))
    return tuple(out)


def objective_and_gradients(prob, psi0, ye0, T0, scale, n_steps, rtol=1e-14):
    """J = total gain-region heating over n_steps (oracle forward), dJ/dpsi0 and dJ/dscale."""
    p = dict(prob, scale=np.asarray(scale, dtype=np.float64))
    states = [(np.asarray(psi0, dtype=np.float64), np.asarray(ye0, dtype=np.float64),
               np.asarray(T0, dtype=np.float64))]
    J = np.zeros(np.asarray(psi0).shape[0])
    for _ in range(n_steps):
        o = O.step(p, *states[-1], rtol=rtol)
        J += o['heating']
        states.append((o['psi'], o['ye'], o['T']))
    psi_bar = np.zeros_like(states[-1][0])
    ye_bar = np.zeros_like(states[-1][1])
    T_bar = np.zeros_like(states[-1][2])
    s_bar = np.zeros_like(np.asarray(scale, dtype=np.float64))
    for n in range(n_steps - 1, -1, -1):
        pn, yn, tn = states[n]
        p1, y1, _ = states[n + 1]
        psi_bar, ye_bar, T_bar, sb = step_vjp(prob, pn, yn, tn, scale, p1, y1, psi_bar, ye_bar, T_bar)
        s_bar += sb
    return J, psi_bar, s_bar
