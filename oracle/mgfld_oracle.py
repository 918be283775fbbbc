"""Plain FP64 CPU oracle for the implicit MGFLD Lagrangian transport step.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  The product path (the
CUDA library and its Python binding) never calls it and shares no code with it.

What it computes (Bruenn et al., CHIMERA, Sec. "Lagrangian Transport Step" and
"Solution of the Transport Equations"): one backward-Euler step of ray-by-ray
multi-group flux-limited diffusion.  The result is *defined* as the root of the
nonlinear system formed by Eq. a58 (zeroth moment, conservative differencing)
with the flux of Eq. a59, for every (zone i, group k, species q), together with
Eq. a62a (electron fraction) for every zone; it is followed by Eq. a62b
(internal energy) and the temperature from the equation of state (Eq. a62d is
the linearised form of that inversion).  The oracle finds the root by Newton's
method on the fully coupled per-zone block of size N_nu*N_k + 1 (Eq. a62ae),
with an exact Jacobian and a plain block-Thomas elimination that calls
numpy's LU solver (LAPACK gesv) on each dense block.

Readings of passages that are silent, garbled or ambiguous (each one is applied
identically here and documented with the project's design notes):
  R1  Eq. a01 is dimensionally wrong; centres satisfy Eq. a01b:
      eps_k = sqrt((e+^2 + e+ e- + e-^2)/3).
  R2  Eq. a59 uses lambda and the limiter at n+1, but Eq. a62ae makes the
      off-diagonal blocks diagonal: lambda^(t) and F (hence the diffusion
      coefficient) are frozen at psi^n, T^n, Ye^n for the step.
  R3  Edge psi in Eq. a20 is the arithmetic mean of the neighbours; the edge
      mean free path (geometric mean, Eq. a59 text) is used in Eq. a20 and
      Eq. a23; beta = 0 and ray bending G = 1 (static, Newtonian) in a24-a26.
      psi_edge <= 1e-300 gives F = 0; a zero gradient gives F = 1.
  R4  The neutrinosphere R_nu(k,q) is where the transport optical depth,
      integrated inward from the outer edge with 1/lambda^(t) at psi^n,
      reaches 2/3 (linear inside the zone); if it never does, R_nu = R_1/2.
  R5  Eq. a62af reads psi_{I+1} = psi_I (R_I^2 - R_nu^2/4)/(R_{I+1}^2 - R_nu^2/4)
      (the printed "R_nu" lacks its square); R_nu is clamped to <= R_I; the
      ghost centre is R_{I+1} = 2 R_{I+1/2} - R_I with lambda_{I+1} = lambda_I
      and a_{I+1} = a_I.  The centre boundary is zero flux (R_1/2 > 0).
  R6  Synthetic neutrino-electron scattering: the down- and iso-scattering
      out-kernel is coef * exp(-(eps_k - eps_k')/T) (k' <= k); up-scattering
      follows from Eq. d7up and the in-kernel from Eq. d7down; Phi_1 = 0.
  R7  Edge lapse a_{i+1/2} = (a_i + a_{i+1})/2.
  R8  The chemical potentials of Eqs. e11-e13 are +dF/dN (the printed leading
      minus sign contradicts the printed right-hand sides); mu_nue =
      mu_e + mu_p - mu_n, mu_nuebar = -mu_nue, mu_numu,tau = 0.
  R9  T^{n+1} solves e_int(rho, T, Ye^{n+1}) = e^{n+1} exactly (the double-gamma
      e_int is linear in T); Eq. a62d is the first Newton iterate of this.
  R10 The absorption/emission source is j(1 - psi) - kappa_a psi (Eq. a55) with
      j = kappa_a exp((mu - eps)/T) (Kirchhoff); the exponent is capped at 700
      so that 1/(1 - f_eq) stays finite.
  R11 Gain-region heating weights each zone by its lapse (proper time a_i dt).
  P1  Optional synthetic pair term (Eq. d14, zeroth moment): Legendre order 0 only (Phi_1 = 0,
      as R6 for NES), no angular correction (chi = 1), annihilation kernel Phi0^a = pair_coef
      (per zone, cm^3/s, energy independent), creation Phi0^p = exp(-(eps + eps')/T) Phi0^a
      (Eq. d12 with the pair energy eps + eps' given to the e-e+ pair); partners nu_e/nubar_e and
      nu_mu,tau/nubar_mu,tau.  It enters the sources (hence Eq. a62b) but not lambda^(t) (a1) and,
      being symmetric in the pair, leaves the lepton number and Eq. a62a unchanged.
  P2  Optional angular correction of the pair annihilation kernel (Eqs. d16-d22, prob['pair_chi']):
      chi = min(chi_1, chi_2) per (zone, eps, eps') formed at the start of the step from the flux
      factors eta1 (the same input as S2; absent, 0) and the neutrinospheres of the step's
      coefficients at psi^n, with the cone edges of Eqs. d17-d18 extended by Eq. d22 at the zone
      centre R_i.  Eq. d14 puts chi on the annihilation kernel only.  Eq. d16 is kept as printed,
      1 - eta etabar / 6, which is the average for distributions psi0 (1 + eta mu); Eq. d15's
      psi0 + 3 mu psi1 would give 1 - 3 eta etabar / 2 (negative for forward-peaked radiation).
  R12 (optional, the paper-literal form of Eq. a59) lambda^(t) and F at n+1: the flux
      coefficients (mean free path with j at the iterate's Ye and the NES rates at its psi,
      neutrinosphere, ghost factor, limiter) are formed again at every outer iterate with
      T = T^n; the Jacobian adds the limiter's derivative on the two zones of each edge and holds
      the rest (the mean free path couples all groups through NES, the neutrinosphere all zones).
      The root then satisfies Eqs. a58/a59 with the coefficients of the root itself.  It is not
      combined with the shock terms: their flux part multiplies the limiter (Eq. a93), whose
      derivative then needs the frame shift of every edge, and without it the iteration took
      ~30 outer iterations.

Transport through a shock (Sec. "Transport through a Shock", Eqs. a90-a99), taken when the
problem carries zone velocities u:
  S1  dpsi0_shock (Eq. a91) and dpsi1_shock (Eq. a97) are formed at the start of the step, from
      psi^n, like lambda and the limiter (R2): Eq. a93 writes every flux coefficient at n+1 and the
      frozen reading treats them alike.  The shock terms are then constants of the step and the
      Jacobian of Eq. a62ae is unchanged.
  S2  psi1 = eta1 psi^n and psi2 = eta2 psi^n at zone centres, with the flux factor eta1 an input
      (clamped to [0, 1]; absent, eta1 = 0) and eta2 from the Minerbo closure (Eqs. a86-a87).
  S3  The psi2 of Eq. a97 at edge i+1/2 is zone i+1's (the frame-(i+1) moment that Eq. a96
      transforms), on zone i's energy grid (the grid is velocity independent).
  S4  The group-edge values of Eqs. a92/a98 at the lowest and highest group edges are zero, so the
      energy-space terms telescope: dpsi1_shock carries no neutrino number (as Eq. a96 carries
      none in the continuum) and dpsi0_shock removes beta sum_k eps^2 d eps psi1.
  S5  beta_{i+1/2} = (u_{i+1} - u_i)/c at the interior edges, u zone-centred; the terms are
      multiplied by a roll-in weight rising linearly from 0 at |beta| = 0.01 to 1 at 0.02; the
      outermost edge (no zone above) and the centre edge carry none.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Physical constants (CGS, MeV).
C_LIGHT = 2.99792458e10          # cm / s
HC = 1.23984198e-10              # MeV cm
FOUR_PI_HC3 = 4.0 * np.pi / HC**3    # converts eps^2 d eps psi to a number density
C_NES = 2.0 * np.pi / (C_LIGHT * HC**3)  # Eq. d8 divided by c (source per unit length)
STAT_WEIGHT = np.array([1.0, 1.0, 2.0, 2.0])  # N_stwt,q of Eq. a62b
LEPTON_SIGN = np.array([1.0, -1.0, 0.0, 0.0])  # nue carries +1, nuebar -1 (Eq. a50)
EXP_CAP = 700.0                  # reading R10
N_SPECIES = 4

BC_GHOST = 0      # Eq. a62af outer boundary
BC_REFLECT = 1    # zero flux at the outer edge (test switch for equilibrium pins)


@dataclasses.dataclass
class EosParams:
    """Double-gamma EoS constants (Sec. "Double-gamma EoS", Eqs. e2-e13)."""
    gamma1: float = 4.0 / 3.0
    gamma2: float = 2.5
    e_coef: float = 1.5
    g_n: float = 2.0
    g_p: float = 2.0
    rho_nuc: float = 2.5e14          # g / cm^3
    rho_0: float = 2.5e14            # reference density of Eq. e2 (enters only if gamma1 != 4/3)
    mb_c2: float = 939.565           # MeV
    m_b: float = 1.674927e-24        # g

    @property
    def f1(self):
        return 0.75 * (3.0 / (8.0 * np.pi)) ** (1.0 / 3.0) * HC        # Eq. e4

    @property
    def f2(self):                                                       # Eq. e7
        g1, g2 = self.gamma1, self.gamma2
        return ((g1 - 1.0) / (g2 - 1.0) * self.f1
                * (0.5 * self.rho_nuc / self.m_b) ** (g1 - g2)
                * (self.m_b / self.rho_0) ** (g1 - 4.0 / 3.0))


# ----------------------------------------------------------------------------
# Grids
# ----------------------------------------------------------------------------

def group_centres(e_edge):
    """Energy-group centres and widths (reading R1 of Eq. a01; Eq. a01b)."""
    e_edge = np.asarray(e_edge, dtype=np.float64)
    lo, hi = e_edge[:-1], e_edge[1:]
    eps = np.sqrt((hi * hi + hi * lo + lo * lo) / 3.0)
    return eps, hi - lo


def local_energies(e_edge, lapse):
    """Local comoving energies eps = E/a of the fixed-at-infinity grid (Eq. a8a).

    Returns eps, d_eps with shape [n_ray, n_r, n_e]."""
    E, dE = group_centres(e_edge)
    inv_a = 1.0 / lapse
    return E[None, None, :] * inv_a[:, :, None], dE[None, None, :] * inv_a[:, :, None]


def radial_geometry(r_edge):
    """Zone centres R_i = (R_- + R_+)/2, edge areas 4 pi R^2, volumes (Eq. a59 text, Gamma = 1)."""
    r_edge = np.asarray(r_edge, dtype=np.float64)
    rc = 0.5 * (r_edge[:, :-1] + r_edge[:, 1:])
    area = 4.0 * np.pi * r_edge**2
    vol = 4.0 * np.pi * (r_edge[:, 1:]**3 - r_edge[:, :-1]**3) / 3.0
    return rc, area, vol


# ----------------------------------------------------------------------------
# Double-gamma equation of state (Eqs. e2-e13)
# ----------------------------------------------------------------------------

def _thermal_volume(T, p: EosParams):
    """(h^2 / (2 pi m_B k T))^{E_coef} in cm^3 (T in MeV)."""
    return (HC * HC / (2.0 * np.pi * p.mb_c2 * T)) ** p.e_coef


def eos_chemical_potentials(rho, T, ye, p: EosParams):
    """mu_e, mu_n, mu_p (MeV) from Eqs. e13, e11, e12 (reading R8)."""
    n_e = rho * ye / p.m_b
    n_n = rho * (1.0 - ye) / p.m_b
    n_p = rho * ye / p.m_b
    lam3 = _thermal_volume(T, p)
    mu_e = p.gamma1 * p.f1 * n_e ** (p.gamma1 - 1.0) * (p.m_b / p.rho_0) ** (p.gamma1 - 4.0 / 3.0)
    mu_n = p.gamma2 * p.f2 * n_n ** (p.gamma2 - 1.0) + T * np.log(n_n * lam3 / p.g_n)
    mu_p = T * np.log(n_p * lam3 / p.g_p)
    return mu_e, mu_n, mu_p


def mu_nue(rho, T, ye, p: EosParams):
    """Electron-neutrino equilibrium chemical potential mu_e + mu_p - mu_n (beta equilibrium)."""
    mu_e, mu_n, mu_p = eos_chemical_potentials(rho, T, ye, p)
    return mu_e + mu_p - mu_n


def dmu_nue_dye(rho, T, ye, p: EosParams):
    """d mu_nue / d Ye at fixed rho, T (analytic derivative of Eqs. e11-e13)."""
    mu_e, mu_n, _ = eos_chemical_potentials(rho, T, ye, p)
    n_n = rho * (1.0 - ye) / p.m_b
    mu_n_nuc = p.gamma2 * p.f2 * n_n ** (p.gamma2 - 1.0)
    return ((p.gamma1 - 1.0) * mu_e / ye + T / ye
            + (p.gamma2 - 1.0) * mu_n_nuc / (1.0 - ye) + T / (1.0 - ye))


def species_mu(rho, T, ye, p: EosParams):
    """Per-species chemical potentials [n_ray, 4, n_r] and their Ye-derivatives."""
    m = mu_nue(rho, T, ye, p)
    dm = dmu_nue_dye(rho, T, ye, p)
    z = np.zeros_like(m)
    return np.stack([m, -m, z, z], axis=1), np.stack([dm, -dm, z, z], axis=1)


def e_int(rho, T, ye, p: EosParams):
    """Internal energy per baryon in MeV (Eq. e10 divided by N_B = rho V / m_B)."""
    n_b = rho / p.m_b
    n_e = rho * ye / p.m_b
    n_n = rho * (1.0 - ye) / p.m_b
    cold = (p.f1 * n_e ** p.gamma1 * (p.m_b / p.rho_0) ** (p.gamma1 - 4.0 / 3.0)
            + p.f2 * n_n ** p.gamma2) / n_b
    return cold + p.e_coef * T


def temperature_from_e(rho, e, ye, p: EosParams):
    """Invert e_int(rho, T, Ye) = e for T (reading R9; e_int is linear in T)."""
    cold = e_int(rho, np.zeros_like(e), ye, p)
    return (e - cold) / p.e_coef


# ----------------------------------------------------------------------------
# Sources (Sec. "Transport Sources")
# ----------------------------------------------------------------------------

def nes_kernels(eps, T, coef):
    """Synthetic NES Legendre-0 kernels Phi_out[k,k'], Phi_in[k,k'] per zone (reading R6).

    eps: [n_ray, n_r, n_e] local energies; T, coef: [n_ray, n_r].
    Down/iso-scattering (eps_k' <= eps_k) is computed directly; up-scattering
    from Eq. d7up; the in-kernel from Eq. d7down (Phi_in[k,k'] = Phi_out[k',k])."""
    d = eps[:, :, :, None] - eps[:, :, None, :]          # eps_k - eps_k'
    Tb = T[:, :, None, None]
    cb = coef[:, :, None, None]
    k = np.arange(eps.shape[2])
    down = (k[None, :] <= k[:, None])[None, None]        # k' <= k
    phi_out = np.where(down, cb * np.exp(-np.where(down, d, 0.0) / Tb),
                       cb * np.exp(2.0 * np.where(down, 0.0, d) / Tb))
    phi_in = np.swapaxes(phi_out, 2, 3)
    return phi_out, phi_in


def emissivity(kappa_abs, eps, mu_q, T):
    """j = kappa_a exp((mu - eps)/T) (reading R10), shape [n_ray, 4, n_r, n_e]."""
    x = (mu_q[:, :, :, None] - eps[:, None, :, :]) / T[:, None, :, None]
    return kappa_abs * np.exp(np.minimum(x, EXP_CAP)), x < EXP_CAP


def nes_source(psi, w, phi_out, phi_in):
    """Zeroth-moment NES source per unit length, Eq. d8 with Phi_1 = 0, divided by c.

    S_k = C [(1 - psi_k) sum_k' w_k' Phi_in[k,k'] psi_k' - psi_k sum_k' w_k' Phi_out[k,k'] (1 - psi_k')]"""
    gain = np.einsum('rikm,rim,rqim->rqik', phi_in, w, psi)
    loss = np.einsum('rikm,rim,rqim->rqik', phi_out, w, 1.0 - psi)
    return C_NES * ((1.0 - psi) * gain - psi * loss)


PAIR_PARTNER = np.array([1, 0, 3, 2])   # nu_e <-> nubar_e, nu_mu,tau <-> nubar_mu,tau


def pair_kernels(eps, T, coef):
    """Synthetic pair kernels (reading P1): annihilation Phi0^a(eps, eps') = coef, creation
    Phi0^p = exp(-(eps + eps')/T) Phi0^a (Eq. d12 with E_e- + E_e+ = eps + eps'), per zone
    [n_ray, n_r, n_e, n_e]; the species' own energies on the rows, the partner's on the columns."""
    e = eps[:, :, :, None] + eps[:, :, None, :]
    cb = np.broadcast_to(coef[:, :, None, None], e.shape)
    return cb, cb * np.exp(-e / T[:, :, None, None])


def chi_isotropic(eta, eta_bar):
    """chi_1 of Eq. d16 as printed, 1 - eta etabar / 6: the annihilation factor (1 - n.nbar)^2
    averaged over the near-isotropic distributions psi0 (1 + eta mu), relative to isotropic ones
    (reading P2: Eq. d15's psi0 + 3 mu psi1 would give 1 - 3 eta etabar / 2); eta = psi1/psi0 of the
    neutrino at eps, eta_bar of the antineutrino at eps'."""
    return 1.0 - eta * eta_bar / 6.0


def pair_mu(r_nu, R):
    """The cone edge of Eqs. d17-d18 extended to any radius by Eq. d22:
    max(sign(1 - (R_nu/R)^2) sqrt(|1 - (R_nu/R)^2|), -1)."""
    x = 1.0 - (np.asarray(r_nu, dtype=np.float64) / R) ** 2
    return np.maximum(np.sign(x) * np.sqrt(np.abs(x)), -1.0)


def chi_beamed(mu, mu_bar):
    """chi_2 of Eq. d19 for radiation emitted isotropically by the neutrinospheres and seen inside
    the cones mu >= mu_i, mu' >= mu_i' (Eqs. d17-d18), relative to isotropic radiation."""
    return (8.0 + (mu * mu_bar - 3.0) * (1.0 + mu) * (1.0 + mu_bar)) / 8.0


def pair_chi(eta, r_nu, rc):
    """chi = min(chi_1, chi_2) (Eq. d21) per (ray, species q, zone, k, k') for species q at eps_k
    against its partner at eps_k': eta [n_ray, 4, n_r, n_e] flux factors, r_nu [n_ray, 4, n_e]
    neutrinosphere radii, rc [n_ray, n_r] zone centres (reading P2)."""
    mu = pair_mu(r_nu[:, :, None, :], rc[:, None, :, None])           # [ray, q, zone, k]
    bar = PAIR_PARTNER
    c1 = chi_isotropic(eta[..., :, None], eta[:, bar][..., None, :])
    c2 = chi_beamed(mu[..., :, None], mu[:, bar][..., None, :])
    return np.minimum(c1, c2)


def pair_source(psi, w, phi_a, phi_p, chi=None):
    """Zeroth-moment pair source per unit length, Eq. d14 with Phi_1 = 0 (reading P1), divided by c
    like the NES source:
    S_k = C [(1 - psi_k) sum_k' w_k' Phi^p[k,k'] (1 - psibar_k') - psi_k sum_k' w_k' chi Phi^a[k,k'] psibar_k'],
    psibar the partner species' occupation; chi [n_ray, 4, n_r, n_e, n_e] the angular correction of
    the annihilation kernel (Eqs. d16-d22), or None for 1."""
    bar = psi[:, PAIR_PARTNER]
    make = np.einsum('rikm,rim,rqim->rqik', phi_p, w, 1.0 - bar)
    if chi is None:
        kill = np.einsum('rikm,rim,rqim->rqik', phi_a, w, bar)
    else:
        kill = np.einsum('rikm,rqikm,rim,rqim->rqik', phi_a, chi, w, bar)
    return C_NES * ((1.0 - psi) * make - psi * kill)


def nes_inverse_mfp(psi, w, phi_out, phi_in):
    """NES contribution to 1/lambda^(t): Eq. a17 applied to the first moment of Eq. d8 (Phi_1 = 0)."""
    return C_NES * (np.einsum('rikm,rim,rqim->rqik', phi_in, w, psi)
                    + np.einsum('rikm,rim,rqim->rqik', phi_out, w, 1.0 - psi))


def absem_source(psi, j, kappa_abs):
    """Absorption/emission source per unit length, j (1 - psi) - kappa_a psi (Eq. a55 bracket)."""
    return j * (1.0 - psi) - kappa_abs * psi


# ----------------------------------------------------------------------------
# Problem set-up and the frozen (psi^n) coefficients
# ----------------------------------------------------------------------------

class Frozen:
    """Everything held fixed during the Newton iteration of one step (reading R2)."""


def setup_step(prob, psi_n, ye_n, T_n):
    """Build the frozen coefficients of one step from the start-of-step state.

    prob: dict with r_edge [n_ray,n_r+1], lapse [n_ray,n_r] or None, e_edge [n_e+1],
    rho [n_ray,n_r], kappa_abs/kappa_scat [n_ray,4,n_r,n_e], nes_coef [n_ray,n_r] or None,
    dt, eos (EosParams), outer_bc (BC_GHOST/BC_REFLECT), scale [4,n_e] or None."""
    f = Frozen()
    eos = prob.get('eos') or EosParams()
    f.eos = eos
    r_edge = np.asarray(prob['r_edge'], dtype=np.float64)
    n_ray, n_r = r_edge.shape[0], r_edge.shape[1] - 1
    lapse = prob.get('lapse')
    lapse = np.ones((n_ray, n_r)) if lapse is None else np.asarray(lapse, dtype=np.float64)
    f.n_ray, f.n_r = n_ray, n_r
    f.n_e = len(prob['e_edge']) - 1
    f.dt = float(prob['dt'])
    f.lapse = lapse
    f.rho = np.asarray(prob['rho'], dtype=np.float64)
    f.T_n = np.asarray(T_n, dtype=np.float64)
    f.ye_n = np.asarray(ye_n, dtype=np.float64)
    f.psi_n = np.asarray(psi_n, dtype=np.float64)
    f.outer_bc = int(prob.get('outer_bc', BC_GHOST))
    f.rc, f.area, f.vol = radial_geometry(r_edge)
    f.r_edge = r_edge
    f.E, f.dE = group_centres(prob['e_edge'])
    f.eps, f.deps = local_energies(prob['e_edge'], lapse)
    f.w = f.eps**2 * f.deps                                   # eps^2 d eps (Eq. a01b)
    scale = prob.get('scale')
    s = np.ones((N_SPECIES, f.n_e)) if scale is None else np.asarray(scale, dtype=np.float64)
    f.kappa_abs = np.asarray(prob['kappa_abs'], dtype=np.float64) * s[None, :, None, :]
    f.kappa_scat = np.asarray(prob['kappa_scat'], dtype=np.float64) * s[None, :, None, :]
    coef = prob.get('nes_coef')
    coef = np.zeros((n_ray, n_r)) if coef is None else np.asarray(coef, dtype=np.float64)
    f.phi_out, f.phi_in = nes_kernels(f.eps, f.T_n, coef)     # at T^n (Sec. LTS: T held fixed)
    pc = prob.get('pair_coef')
    f.pair_a, f.pair_p = (None, None) if pc is None else pair_kernels(f.eps, f.T_n, np.asarray(pc, dtype=np.float64))

    f.e_n = e_int(f.rho, f.T_n, f.ye_n, eos)
    f.e_edge = np.asarray(prob['e_edge'], dtype=np.float64)
    f.u, f.eta1 = prob.get('u'), prob.get('eta1')
    flux_coefficients(f, f.psi_n, f.ye_n)                     # at psi^n, Ye^n: reading R2
    f.chi = None
    if f.pair_a is not None and prob.get('pair_chi'):
        eta = np.zeros_like(f.psi_n) if f.eta1 is None else np.clip(np.asarray(f.eta1, dtype=np.float64), 0.0, 1.0)
        f.chi = pair_chi(eta, f.r_nu, f.rc)                   # reading P2
    return f


def flux_coefficients(f, psi, ye):
    """The transport mean free path (Eq. a17 with a55, d8c, d8), the neutrinosphere and ghost
    factor (R4, R5), the edge coefficients of Eq. a59 with the limiter (a20-a26a) and, with zone
    velocities, the shock terms (Eqs. a91, a97), all at the state (psi, Ye) with T = T^n; set on
    f.  The step forms them at psi^n, Ye^n (R2), or with reading R12 at every outer iterate."""
    mu_q, _ = species_mu(f.rho, f.T_n, ye, f.eos)
    j, _ = emissivity(f.kappa_abs, f.eps, mu_q, f.T_n)
    inv_lam = (f.kappa_abs + j + f.kappa_scat + nes_inverse_mfp(psi, f.w, f.phi_out, f.phi_in))
    f.lam = 1.0 / inv_lam
    f.r_nu = neutrinosphere(f.lam, f.r_edge)
    f.ghost = ghost_factor(f.rc, f.r_edge, f.r_nu)
    f.alpha, f.D, f.F = edge_coefficients(f, psi)
    f.shock = None if f.u is None else shock_corrections(f, f.e_edge, f.u, f.eta1, psi)


def neutrinosphere(lam, r_edge):
    """R_nu per (ray, species, group): tau = 2/3 from the outside (reading R4)."""
    n_ray, n_s, n_r, n_e = lam.shape
    dr = (r_edge[:, 1:] - r_edge[:, :-1])[:, None, :, None]
    dtau = dr / lam
    tau_out = np.flip(np.cumsum(np.flip(dtau, axis=2), axis=2), axis=2) - dtau   # tau at R_{i+1/2}
    tau_in = tau_out + dtau                                                    # tau at R_{i-1/2}
    r_nu = np.empty((n_ray, n_s, n_e))
    for r in range(n_ray):
        for q in range(n_s):
            for k in range(n_e):
                hit = np.nonzero(tau_in[r, q, :, k] >= 2.0 / 3.0)[0]
                if hit.size == 0:
                    r_nu[r, q, k] = r_edge[r, 0]
                else:
                    i = hit[-1]
                    r_nu[r, q, k] = (r_edge[r, i + 1]
                                     - (2.0 / 3.0 - tau_out[r, q, i, k]) * lam[r, q, i, k])
    return r_nu


def ghost_factor(rc, r_edge, r_nu):
    """Outer ghost ratio psi_{I+1}/psi_I of Eq. a62af (reading R5), shape [n_ray, 4, n_e]."""
    r_i = rc[:, -1][:, None, None]
    r_g = (2.0 * r_edge[:, -1] - rc[:, -1])[:, None, None]
    rn = np.minimum(r_nu, r_i)
    return (r_i**2 - 0.25 * rn**2) / (r_g**2 - 0.25 * rn**2)


def edge_coefficients(f, psi=None):
    """Frozen flux coefficients at the outer edge i+1/2 of every zone (Eqs. a59, a20-a26a).

    Returns alpha = A_{i+1/2} D_{i+1/2} / a_{i+1/2}^2, D = lambda F / (3 (R_{i+1} - R_i)) and the
    limiter F itself, all [n_ray, 4, n_r, n_e]; psi^(1)_{i+1/2} = -D (psi_{i+1} - psi_i)."""
    psi = f.psi_n if psi is None else psi
    lam = f.lam
    n_r = f.n_r
    psi_r = np.empty_like(psi)
    psi_r[:, :, :-1] = psi[:, :, 1:]
    psi_r[:, :, -1] = f.ghost * psi[:, :, -1]
    lam_r = np.empty_like(lam)
    lam_r[:, :, :-1] = lam[:, :, 1:]
    lam_r[:, :, -1] = lam[:, :, -1]
    rc_r = np.empty_like(f.rc)
    rc_r[:, :-1] = f.rc[:, 1:]
    rc_r[:, -1] = 2.0 * f.r_edge[:, -1] - f.rc[:, -1]
    a_r = np.empty_like(f.lapse)
    a_r[:, :-1] = f.lapse[:, 1:]
    a_r[:, -1] = f.lapse[:, -1]

    lam_e = np.sqrt(lam * lam_r)
    dpsi = psi_r - psi
    dR = (rc_r - f.rc)[:, None, :, None]
    psi_e = 0.5 * (psi + psi_r)
    x = lam_e * np.abs(dpsi / dR) / 3.0
    r_e = f.r_edge[:, 1:][:, None, :, None]
    r_nu = f.r_nu[:, :, None, :]
    with np.errstate(divide='ignore', invalid='ignore'):
        f_int = 1.0 / (1.0 + x / psi_e)
        mu = np.sqrt(np.maximum(1.0 - (r_nu / r_e) ** 2, 0.0))
        f_geo = np.where(r_e > r_nu, 0.5 * (1.0 + mu) * psi_e / x, np.inf)
        F = np.minimum(f_int, f_geo)
    F = np.where(dpsi == 0.0, 1.0, F)
    F = np.where(psi_e <= 1e-300, 0.0, F)
    D = lam_e * F / (3.0 * dR)
    a_e = 0.5 * (f.lapse + a_r)
    alpha = f.area[:, 1:][:, None, :, None] * D / (a_e**2)[:, None, :, None]
    # Derivatives of the edge flux A psi1/a^2 = -K Phi, Phi = F (psi_r - psi) and K = alpha / F,
    # with respect to psi_i and psi_{i+1} through the limiter (lambda and R_nu held), on the
    # branch the limiter selects (reading R12); with b = lambda_e/(3 dR), s = sign(d psi):
    #   F_intrp: Phi = e d/(e + b|d|),  F_geom: Phi = (h/b) e s,  d psi = 0: Phi = d.
    K = f.area[:, 1:][:, None, :, None] * lam_e / (3.0 * dR) / (a_e**2)[:, None, :, None]
    b = lam_e / (3.0 * dR)
    s = np.sign(dpsi)
    den = psi_e + b * np.abs(dpsi)
    with np.errstate(divide='ignore', invalid='ignore'):
        geo = F == f_geo
        h_b = 0.5 * (1.0 + mu) / b
        phi = psi_e * dpsi / den
        dl = np.where(geo, 0.5 * h_b * s, ((0.5 * dpsi - psi_e) - phi * (0.5 - b * s)) / den)
        dr = np.where(geo, 0.5 * h_b * s, ((0.5 * dpsi + psi_e) - phi * (0.5 + b * s)) / den)
    dl = np.where(dpsi == 0.0, -1.0, dl)
    dr = np.where(dpsi == 0.0, 1.0, dr)
    dl = np.where(psi_e <= 1e-300, 0.0, dl)
    dr = np.where(psi_e <= 1e-300, 0.0, dr)
    f.jl, f.jr = -K * dl, -K * dr
    if f.outer_bc == BC_REFLECT:
        alpha[:, :, -1, :] = 0.0
        f.jl[:, :, -1, :] = 0.0
        f.jr[:, :, -1, :] = 0.0
    return alpha, D, F


# ----------------------------------------------------------------------------
# Transport through a shock (Eqs. a90-a99), readings S1-S5
# ----------------------------------------------------------------------------

SHOCK_ROLL_IN = (0.01, 0.02)        # |u_{i+1} - u_i| / c where the shock terms start / are whole


def shock_beta(u):
    """beta_{i+1/2} (Eq. a90) at the n_r - 1 interior edges and the roll-in weight (S5)."""
    u = np.asarray(u, dtype=np.float64)
    beta = (u[:, 1:] - u[:, :-1]) / C_LIGHT
    lo, hi = SHOCK_ROLL_IN
    return beta, np.clip((np.abs(beta) - lo) / (hi - lo), 0.0, 1.0)


def group_edge_mean(m):
    """m_{k+1/2} = (m_k + m_{k+1})/2 (Eqs. a92, a98) at the N + 1 group edges, zero at the
    lowest and highest edge (S4)."""
    out = np.zeros(m.shape[:-1] + (m.shape[-1] + 1,))
    out[..., 1:-1] = 0.5 * (m[..., :-1] + m[..., 1:])
    return out


def energy_divergence(eps_lo, eps_hi, m):
    """(eps_+^3 m_{k+1/2} - eps_-^3 m_{k-1/2}) / ((eps_+^3 - eps_-^3)/3): the energy-space term
    of Eqs. a91 and a97 (the discrete (1/eps^2) d(eps^3 m)/d eps of Eq. a96)."""
    me = group_edge_mean(m)
    return (eps_hi**3 * me[..., 1:] - eps_lo**3 * me[..., :-1]) / ((eps_hi**3 - eps_lo**3) / 3.0)


def shock_corrections(f, e_edge, u, eta1, psi=None):
    """(dpsi0, dpsi1, A/a^2) for the outer edge i+1/2 of every zone, [n_ray, 4, n_r, n_e]:
    dpsi0 = psi^up_i - psi_i of Eq. a91 (frame change of zone i's psi0 into frame i+1),
    dpsi1 = the frame-(i+1) to frame-i change of the edge flux, Eq. a97, and A_{i+1/2}/a_{i+1/2}^2
    (Eq. a99).  Zero at the outermost edge."""
    from oracle.energy_advection_oracle import minerbo_eta2
    beta, wgt = shock_beta(u)
    bw = (beta * wgt)[:, None, :, None]                          # [n_ray, 1, n_r - 1, 1]
    psi = f.psi_n if psi is None else psi
    x = np.zeros_like(psi) if eta1 is None else np.clip(np.asarray(eta1, dtype=np.float64), 0.0, 1.0)
    psi1 = x * psi                                               # S2
    psi2 = minerbo_eta2(x) * psi
    E = np.asarray(e_edge, dtype=np.float64)
    lo = E[:-1][None, None, :] / f.lapse[:, :, None]             # zone i's comoving group edges
    hi = E[1:][None, None, :] / f.lapse[:, :, None]
    lo, hi = lo[:, None, :-1], hi[:, None, :-1]                  # zones 0 .. n_r - 2
    dpsi0 = np.zeros_like(psi)
    dpsi1 = np.zeros_like(psi)
    p1 = psi1[:, :, :-1]
    dpsi0[:, :, :-1] = bw * (-p1 + energy_divergence(lo, hi, p1))           # Eq. a91
    dpsi1[:, :, :-1] = -bw * energy_divergence(lo, hi, psi2[:, :, 1:])      # Eq. a97 (S3)
    a_e = np.empty_like(f.lapse)
    a_e[:, :-1] = 0.5 * (f.lapse[:, :-1] + f.lapse[:, 1:])                  # R7
    a_e[:, -1] = f.lapse[:, -1]
    aa = (f.area[:, 1:] / a_e**2)[:, None, :, None]
    return dpsi0, dpsi1, aa


# ----------------------------------------------------------------------------
# Residual (Eqs. a58, a59, a62a) and exact Jacobian (Eqs. a62ac-a62ae)
# ----------------------------------------------------------------------------

def sources(f, psi, ye):
    """Total zeroth-moment source S and its absorption/emission part at (psi, Ye), with T = T^n."""
    mu_q, dmu_q = species_mu(f.rho, f.T_n, ye, f.eos)
    j, live = emissivity(f.kappa_abs, f.eps, mu_q, f.T_n)
    s_ae = absem_source(psi, j, f.kappa_abs)
    s_nes = nes_source(psi, f.w, f.phi_out, f.phi_in)
    if f.pair_a is not None:
        s_nes = s_nes + pair_source(psi, f.w, f.pair_a, f.pair_p, f.chi)
    return s_ae + s_nes, s_ae, j, dmu_q, live


def flux_divergence(f, psi):
    """(a_i^2/V_i) [A psi1/a^2 |_{i+1/2} - A psi1/a^2 |_{i-1/2}] of Eq. a58 with Eq. a59, or, with
    a shock, Eq. a99 with Eq. a93.  Also returns A psi1/a^2 at every outer edge (in the frame of
    the zone above it)."""
    psi_r = np.empty_like(psi)
    psi_r[:, :, :-1] = psi[:, :, 1:]
    psi_r[:, :, -1] = f.ghost * psi[:, :, -1]
    pre = (f.lapse**2 / f.vol)[:, None, :, None]
    if f.shock is None:
        flux_out = -f.alpha * (psi_r - psi)        # A psi1 / a^2 at i+1/2
        frame = 0.0
    else:
        dpsi0, dpsi1, aa = f.shock
        flux_out = -f.alpha * (psi_r - psi - dpsi0)            # Eq. a93
        frame = aa * dpsi1                                      # Eq. a99: the flux seen from zone i
    flux_in = np.zeros_like(flux_out)
    flux_in[:, :, 1:] = flux_out[:, :, :-1]        # zero flux at the centre edge
    return pre * (flux_out + frame - flux_in), flux_out


def residual(f, psi, ye):
    """G (Eq. a58) [n_ray,4,n_r,n_e] and G_Y (Eq. a62a) [n_ray,n_r]."""
    S, s_ae, _, _, _ = sources(f, psi, ye)
    a = f.lapse[:, None, :, None]
    div, _ = flux_divergence(f, psi)
    G = (psi - f.psi_n) / (a * C_LIGHT * f.dt) + div - S
    lep = np.einsum('q,rik,rqik->ri', LEPTON_SIGN, f.w, s_ae)
    GY = (ye - f.ye_n) / (f.lapse * C_LIGHT * f.dt) + FOUR_PI_HC3 * (f.eos.m_b / f.rho) * lep
    return G, GY


def jacobian(f, psi, ye):
    """Exact Jacobian of (G, G_Y) in the coupled block form of Eq. a62ae.

    Unknowns per zone: alpha = q*n_e + k for psi, alpha = 4 n_e for Ye.
    Returns A [n_ray,n_r,M,M] (dense diagonal blocks), Bm, Bp [n_ray,n_r,M]
    (the diagonal sub- and super-diagonal blocks; their Ye entries are zero)."""
    n_ray, n_r, n_e = f.n_ray, f.n_r, f.n_e
    M = N_SPECIES * n_e + 1
    _, s_ae, j, dmu_q, live = sources(f, psi, ye)
    a = f.lapse
    pre = (a**2 / f.vol)[:, None, :, None]
    # d(flux at i+1/2)/d psi_i and d/d psi_{i+1}: alpha and -alpha with frozen coefficients (R2);
    # at the iterate (R12) with the limiter's own dependence on psi_i, psi_{i+1}
    if getattr(f, 'coef_iterate', False):
        jl, jr = f.jl, f.jr
    else:
        jl, jr = f.alpha, -f.alpha
    ghost_term = np.zeros_like(jl)
    ghost_term[:, :, -1, :] = f.ghost[:, :, :]
    jr_in = np.zeros_like(jr)
    jr_in[:, :, 1:] = jr[:, :, :-1]
    jl_in = np.zeros_like(jl)
    jl_in[:, :, 1:] = jl[:, :, :-1]

    # d S_nes,k / d psi_k' (full matrix) per (ray, species, zone).
    w = f.w
    dS = C_NES * (np.einsum('rikm,rim,rqik->rqikm', f.phi_in, w, 1.0 - psi)
                  + np.einsum('rikm,rim,rqik->rqikm', f.phi_out, w, psi))
    diag_nes = C_NES * (np.einsum('rikm,rim,rqim->rqik', f.phi_in, w, psi)
                        + np.einsum('rikm,rim,rqim->rqik', f.phi_out, w, 1.0 - psi))
    diag = (1.0 / (a[:, None, :, None] * C_LIGHT * f.dt)
            + pre * (jl + ghost_term * jr - jr_in)
            + j + f.kappa_abs + diag_nes)
    if f.pair_a is not None:
        # d S_pair,k / d psi_k (own species, diagonal) and d S_pair,k / d psibar_k' (partner)
        bar = psi[:, PAIR_PARTNER]
        pa = f.pair_a[:, None] if f.chi is None else f.pair_a[:, None] * f.chi   # [ray, q|1, zone, k, k']
        diag = diag + C_NES * (np.einsum('rikm,rim,rqim->rqik', f.pair_p, w, 1.0 - bar)
                               + np.einsum('rqikm,rim,rqim->rqik', np.broadcast_to(pa, psi.shape + psi.shape[-1:]),
                                           w, bar))
        dP = -C_NES * (np.einsum('rikm,rim,rqik->rqikm', f.pair_p, w, 1.0 - psi)
                       + np.einsum('rqikm,rim,rqik->rqikm', np.broadcast_to(pa, psi.shape + psi.shape[-1:]), w, psi))
    A = np.zeros((n_ray, n_r, M, M))
    for q in range(N_SPECIES):
        sl = slice(q * n_e, (q + 1) * n_e)
        A[:, :, sl, sl] = -dS[:, q]
        if f.pair_a is not None:
            qb = PAIR_PARTNER[q]
            A[:, :, sl, qb * n_e:(qb + 1) * n_e] = -dP[:, q]
        idx = np.arange(q * n_e, (q + 1) * n_e)
        A[:, :, idx, idx] += diag[:, q]
        # d G_q / d Ye = -(1 - psi) dj/dYe, dj/dYe = j dmu/dYe / T (zero where capped).
        dj = np.where(live[:, q], j[:, q] * dmu_q[:, q, :, None] / f.T_n[:, :, None], 0.0)
        A[:, :, sl, M - 1] = -(1.0 - psi[:, q]) * dj
        # d G_Y / d psi_q = c_Y * sign_q * dS_ae/dpsi = -c_Y sign_q w (j + kappa_a).
        cy = FOUR_PI_HC3 * (f.eos.m_b / f.rho)[:, :, None]
        A[:, :, M - 1, sl] = -cy * LEPTON_SIGN[q] * w * (j[:, q] + f.kappa_abs[:, q])
        # d G_Y / d Ye (contribution of species q).
        A[:, :, M - 1, M - 1] += (cy[:, :, 0] * LEPTON_SIGN[q]
                                  * np.sum(w * (1.0 - psi[:, q]) * dj, axis=2))
    A[:, :, M - 1, M - 1] += 1.0 / (a * C_LIGHT * f.dt)
    Bm = np.zeros((n_ray, n_r, M))
    Bp = np.zeros((n_ray, n_r, M))
    Bm[:, :, :M - 1] = (-pre * jl_in).transpose(0, 2, 1, 3).reshape(n_ray, n_r, M - 1)
    up = pre * jr
    up[:, :, -1, :] = 0.0            # the ghost is folded into the diagonal
    Bp[:, :, :M - 1] = up.transpose(0, 2, 1, 3).reshape(n_ray, n_r, M - 1)
    return A, Bm, Bp


def pack(G, GY):
    """[n_ray,4,n_r,n_e] + [n_ray,n_r] -> [n_ray, n_r, M] in the Eq. a62ae ordering."""
    n_ray, _, n_r, n_e = G.shape
    return np.concatenate([G.transpose(0, 2, 1, 3).reshape(n_ray, n_r, -1), GY[:, :, None]], axis=2)


def unpack(u, n_e):
    n_ray, n_r, _ = u.shape
    psi = u[:, :, :-1].reshape(n_ray, n_r, N_SPECIES, n_e).transpose(0, 2, 1, 3)
    return psi, u[:, :, -1]


# ----------------------------------------------------------------------------
# Linear solvers for the block-tridiagonal system
# ----------------------------------------------------------------------------

def block_thomas(A, Bm, Bp, rhs):
    """Solve sum_a' A_i x_i + Bm_i * x_{i-1} + Bp_i * x_{i+1} = rhs_i (Bm, Bp diagonal).

    Plain block forward elimination and back substitution; every block solve is
    numpy's LU with partial pivoting (LAPACK gesv), batched over rays."""
    n_ray, n_r, M = rhs.shape
    Ap = np.empty_like(A)
    cp = np.empty_like(rhs)
    Ap[:, 0] = A[:, 0]
    cp[:, 0] = rhs[:, 0]
    for i in range(1, n_r):
        # A'_i = A_i - diag(Bm_i) A'_{i-1}^{-1} diag(Bp_{i-1});  c'_i = rhs_i - Bm_i * A'_{i-1}^{-1} c'_{i-1}
        X = np.linalg.solve(Ap[:, i - 1], np.concatenate(
            [np.eye(M)[None] * Bp[:, i - 1][:, None, :], cp[:, i - 1][:, :, None]], axis=2))
        Ap[:, i] = A[:, i] - Bm[:, i][:, :, None] * X[:, :, :M]
        cp[:, i] = rhs[:, i] - Bm[:, i] * X[:, :, M]
    x = np.empty_like(rhs)
    x[:, -1] = np.linalg.solve(Ap[:, -1], cp[:, -1][:, :, None])[:, :, 0]
    for i in range(n_r - 2, -1, -1):
        x[:, i] = np.linalg.solve(Ap[:, i], (cp[:, i] - Bp[:, i] * x[:, i + 1])[:, :, None])[:, :, 0]
    return x


def dense_matrix(A, Bm, Bp):
    """The full matrix of one ray (brute force; for tiny systems only)."""
    n_r, M = A.shape[0], A.shape[1]
    J = np.zeros((n_r * M, n_r * M))
    for i in range(n_r):
        J[i * M:(i + 1) * M, i * M:(i + 1) * M] = A[i]
        if i > 0:
            J[i * M:(i + 1) * M, (i - 1) * M:i * M] = np.diag(Bm[i])
        if i < n_r - 1:
            J[i * M:(i + 1) * M, (i + 1) * M:(i + 2) * M] = np.diag(Bp[i])
    return J


# ----------------------------------------------------------------------------
# The implicit step
# ----------------------------------------------------------------------------

def group_rel_change(d_psi, psi):
    """Per (ray, species, group): max_i |d psi| / max_i |psi| (zone-wise max norms)."""
    num = np.max(np.abs(d_psi), axis=2)
    den = np.maximum(np.max(np.abs(psi), axis=2), 1e-300)
    return num / den


def rel_change(d_psi, psi):
    """Per (ray, species): max |d psi| / max |psi| over all zones and groups (normwise)."""
    num = np.max(np.abs(d_psi), axis=(2, 3))
    den = np.maximum(np.max(np.abs(psi), axis=(2, 3)), 1e-300)
    return num / den


def newton_solve(f, max_iter=50, rtol=1e-14, coef_iterate=False):
    """Newton iteration on the coupled system (Eqs. a62aa, a62ae) to the root.

    Stops once the normwise relative correction (per ray and species) is <= rtol, or
    when it has reached the rounding level (below 1e-10 and no longer halving); the
    root is then accurate to rounding because the convergence is quadratic.
    With coef_iterate (reading R12) the flux coefficients are formed again at every iterate
    after the first and the Jacobian adds the limiter's dependence on the two zones of each edge
    (the mean free path's, through the NES rates of all groups, and the neutrinosphere's are held:
    the iteration is then nearly quadratic on the benchmark rays).
    Returns psi, Ye, iterations, last correction."""
    psi = f.psi_n.copy()
    ye = f.ye_n.copy()
    prev = np.inf
    it = 0
    err = np.inf
    if coef_iterate and f.u is not None:
        raise NotImplementedError('reading R12 is not combined with the shock terms')
    f.coef_iterate = coef_iterate
    for it in range(1, max_iter + 1):
        if coef_iterate and it > 1:
            flux_coefficients(f, psi, ye)
        G, GY = residual(f, psi, ye)
        A, Bm, Bp = jacobian(f, psi, ye)
        du = block_thomas(A, Bm, Bp, -pack(G, GY))
        d_psi, d_ye = unpack(du, f.n_e)
        psi = psi + d_psi
        ye = ye + d_ye
        err = max(float(np.max(rel_change(d_psi, psi))),
                  float(np.max(np.abs(d_ye) / np.abs(ye))))
        if err <= rtol or (err < 1e-10 and err >= 0.5 * prev):
            break
        prev = err
    return psi, ye, it, err


def ledger_lepton(f, psi, ye):
    """Matter + neutrino lepton number per ray (Eqs. a49, a50 on the grid)."""
    matter = np.sum(f.rho * f.vol * ye / f.eos.m_b, axis=1)
    nu = np.sum(f.vol * FOUR_PI_HC3 * np.einsum('q,rik,rqik->ri', LEPTON_SIGN, f.w, psi), axis=1)
    return matter + nu


def ledger_energy(f, psi, e):
    """Matter + neutrino energy at infinity per ray, MeV (weights a_i; Eq. a62 with a62b)."""
    matter = np.sum(f.lapse * f.rho * f.vol * e / f.eos.m_b, axis=1)
    nu = np.sum(f.lapse * f.vol * FOUR_PI_HC3
                * np.einsum('q,rik,rqik->ri', STAT_WEIGHT, f.w * f.eps, psi), axis=1)
    return matter + nu


def step(prob, psi_n, ye_n, T_n, max_iter=50, rtol=1e-14, coef_iterate=False):
    """One implicit transport step.  Returns a dict with psi, ye, T, e, iterations,
    the ledgers [n_ray, 8] = (lepton before, after, boundary loss, residual,
    energy before, after, boundary loss, residual) and the gain-region heating.
    coef_iterate: the flux coefficients at the outer iterate (reading R12) instead of at psi^n."""
    f = setup_step(prob, psi_n, ye_n, T_n)
    psi, ye, iters, err = newton_solve(f, max_iter=max_iter, rtol=rtol, coef_iterate=coef_iterate)
    S, _, _, _, _ = sources(f, psi, ye)
    a = f.lapse
    # Eq. a62b: internal energy update with the converged sources.
    de = -(a * C_LIGHT * f.dt) * FOUR_PI_HC3 * (f.eos.m_b / f.rho) * np.einsum(
        'q,rik,rqik->ri', STAT_WEIGHT, f.w * f.eps, S)
    e_new = f.e_n + de
    T_new = temperature_from_e(f.rho, e_new, ye, f.eos)
    # Boundary losses over the step (the outer-edge flux of Eq. a62 at n+1).
    _, flux_out = flux_divergence(f, psi)
    fb = flux_out[:, :, -1, :]                                   # A psi1/a^2 at R_{I+1/2}
    W = f.E**2 * f.dE
    lep_loss = C_LIGHT * f.dt * FOUR_PI_HC3 * np.einsum('q,k,rqk->r', LEPTON_SIGN, W, fb)
    en_loss = C_LIGHT * f.dt * FOUR_PI_HC3 * np.einsum('q,k,rqk->r', STAT_WEIGHT, W * f.E, fb)
    lb, la = ledger_lepton(f, f.psi_n, f.ye_n), ledger_lepton(f, psi, ye)
    eb, ea = ledger_energy(f, f.psi_n, f.e_n), ledger_energy(f, psi, e_new)
    ledger = np.stack([lb, la, lep_loss, la + lep_loss - lb,
                       eb, ea, en_loss, ea + en_loss - eb], axis=1)
    return dict(psi=psi, ye=ye, T=T_new, e=e_new, iters=iters, err=err, ledger=ledger,
                heating=gain_heating(f, S), frozen=f)


def gain_heating(f, S, r_lo=1.0e7, r_hi=3.0e7):
    """Energy (MeV) deposited in matter by nue + nuebar in 100-300 km over the step (reading R11)."""
    mask = (f.rc >= r_lo) & (f.rc <= r_hi)
    per_zone = -(f.lapse * C_LIGHT * f.dt) * f.vol * FOUR_PI_HC3 * np.einsum(
        'rik,rqik->ri', f.w * f.eps, S[:, :2])
    return np.sum(np.where(mask, per_zone, 0.0), axis=1)


def run_steps(prob, psi0, ye0, T0, n_steps, **kw):
    """n_steps consecutive implicit steps; returns the final state and per-step outputs."""
    psi, ye, T = psi0, ye0, T0
    outs = []
    for _ in range(n_steps):
        o = step(prob, psi, ye, T, **kw)
        psi, ye, T = o['psi'], o['ye'], o['T']
        outs.append(o)
    return psi, ye, T, outs
