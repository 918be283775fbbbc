"""Seeded synthetic post-bounce profiles for the MGFLD transport step.

This module only manufactures inputs (numpy arrays); it contains none of the
transport arithmetic.  Both the CUDA path and the CPU oracle consume the arrays
it returns.

Profile family (one radial ray; r in cm, rho in g/cm^3, T = kT in MeV):
  * N_r + 1 radial edges log-spaced from 10 km to 1e4 km;
  * rho = 3e14 (r/10 km)^-3 (1 + d_rho) floored at 1e6,
    T = 30 (r/10 km)^-1 (1 + d_T) floored at 0.1,
    Ye rising from 0.1 to 0.5 linearly in log r; sampled at zone midpoints;
  * d_rho, d_T: per-ray angular perturbations 0.05 * sum_{l=1..8} sum_m c_lm Y_lm
    normalised to a maximum of 0.05, with c_lm ~ N(0,1) (axisymmetric m = 0 for
    2D ray sets on theta_j = (j + 1/2) pi / N_ray; real Y_lm for 3D sets on a
    theta x phi grid of cell centres);
  * N_E + 1 energy edges log-spaced from 2 to 250 MeV (energies at infinity);
  * kappa_abs = kappa_scat = 1e-40 rho e_g^2 /cm with iid lognormal(0, 0.2)
    noise per (ray, zone, group) shared by the four species, where e_g is the
    geometric mean of the group's edges;
  * NES kernel scale 1e-41 rho (cm^3/s), the synthetic neutrino-electron
    scattering strength;
  * initial occupation psi0 = 1/(1 + exp(e_g/T)) (Fermi-Dirac, zero chemical
    potential) for all species.
Seeds are 1809_05608 + 1000 * config + field, so every ray subset of a
configuration sees exactly the values of the full configuration.
"""
from __future__ import annotations

import dataclasses

import numpy as np

KM = 1.0e5
BASE_SEED = 180905608
N_SPECIES = 4

FIELD_RHO, FIELD_T, FIELD_KAPPA = 1, 2, 3
FIELD_HYDRO = 4
FIELD_SHOCK = 5


@dataclasses.dataclass(frozen=True)
class ConfigSpec:
    name: str
    n_ray: int
    n_r: int
    n_e: int
    steps: int
    geometry: str            # '1d', '2d' or '3d'
    precision: str           # 'fp64' or 'mixed'
    tol: float
    n_theta: int = 0         # 3D only
    n_phi: int = 0


CONFIGS = {
    1: ConfigSpec('single-ray 64x12 fp64', 1, 64, 12, 1, '1d', 'fp64', 1e-13),
    2: ConfigSpec('2d 256 rays 512x20 fp64', 256, 512, 20, 10, '2d', 'fp64', 1e-13),
    3: ConfigSpec('2d 1024 rays 512x20 mixed', 1024, 512, 20, 20, '2d', 'mixed', 1e-10),
    4: ConfigSpec('3d 64x64 rays 540x20 mixed', 4096, 540, 20, 10, '3d', 'mixed', 1e-10, 64, 64),
    5: ConfigSpec('adjoint 512 rays 512x20', 512, 512, 20, 20, '2d', 'mixed', 1e-10),
}


def _seed(config: int, field: int) -> int:
    return BASE_SEED + 1000 * config + field


def _legendre_p(l, m, x):
    """Associated Legendre P_l^m(x) by the standard upward recurrence (unnormalised)."""
    pmm = np.ones_like(x)
    if m > 0:
        somx2 = np.sqrt((1.0 - x) * (1.0 + x))
        fact = 1.0
        for _ in range(m):
            pmm = -pmm * fact * somx2
            fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = pmmp1
    for ll in range(m + 2, l + 1):
        pll = (x * (2 * ll - 1) * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def angular_perturbation(spec: ConfigSpec, config: int, field: int) -> np.ndarray:
    """Per-ray relative perturbation in [-0.05, 0.05] (l = 1..8 harmonics)."""
    if spec.geometry == '1d':
        return np.zeros(spec.n_ray)
    rng = np.random.default_rng(_seed(config, field))
    if spec.geometry == '2d':
        theta = (np.arange(spec.n_ray) + 0.5) * np.pi / spec.n_ray
        x = np.cos(theta)
        d = np.zeros(spec.n_ray)
        for l in range(1, 9):
            d += rng.standard_normal() * _legendre_p(l, 0, x)
    else:
        th = (np.arange(spec.n_theta) + 0.5) * np.pi / spec.n_theta
        ph = (np.arange(spec.n_phi) + 0.5) * 2.0 * np.pi / spec.n_phi
        TH, PH = np.meshgrid(th, ph, indexing='ij')
        x = np.cos(TH)
        d = np.zeros_like(TH)
        for l in range(1, 9):
            for m in range(-l, l + 1):
                c = rng.standard_normal()
                p = _legendre_p(l, abs(m), x)
                d += c * p * (np.cos(m * PH) if m >= 0 else np.sin(-m * PH))
        d = d.reshape(-1)
    return 0.05 * d / np.max(np.abs(d))


def make_problem(config: int, rays=None, n_ray=None, n_r=None, n_e=None):
    """Inputs of configuration `config` (1-5), optionally for a ray subset.

    `rays` (index array or slice) selects rays of the full configuration; n_ray,
    n_r, n_e override the sizes (a resized problem is its own workload with the
    same recipe).  Returns dict(problem=..., psi0, ye0, T0, spec)."""
    spec = CONFIGS[config]
    if n_ray is not None or n_r is not None or n_e is not None:
        nr_new = n_ray or spec.n_ray
        geometry = spec.geometry
        if geometry == '3d' and nr_new != spec.n_theta * spec.n_phi:
            geometry = '2d'
        if nr_new == 1:
            geometry = '1d'
        spec = dataclasses.replace(spec, n_ray=nr_new, n_r=n_r or spec.n_r,
                                   n_e=n_e or spec.n_e, geometry=geometry)
    NR, NE, NRAY = spec.n_r, spec.n_e, spec.n_ray
    r_edge1 = np.logspace(np.log10(10 * KM), np.log10(1e4 * KM), NR + 1)
    r_mid = 0.5 * (r_edge1[1:] + r_edge1[:-1])
    x = r_mid / (10 * KM)
    d_rho = angular_perturbation(spec, config, FIELD_RHO)
    d_T = angular_perturbation(spec, config, FIELD_T)
    rho = np.maximum(3e14 * x[None, :] ** -3 * (1.0 + d_rho[:, None]), 1e6)
    T = np.maximum(30.0 * x[None, :] ** -1 * (1.0 + d_T[:, None]), 0.1)
    ye = np.broadcast_to(0.1 + 0.4 * np.log(x) / np.log(1e3), (NRAY, NR)).copy()
    e_edge = np.logspace(np.log10(2.0), np.log10(250.0), NE + 1)
    e_g = np.sqrt(e_edge[1:] * e_edge[:-1])
    rng = np.random.default_rng(_seed(config, FIELD_KAPPA))
    noise = rng.lognormal(0.0, 0.2, size=(NRAY, NR, NE))
    kappa = 1e-40 * rho[:, :, None] * e_g[None, None, :] ** 2 * noise
    kappa4 = np.ascontiguousarray(np.broadcast_to(kappa[:, None], (NRAY, N_SPECIES, NR, NE)))
    xg = np.exp(-e_g[None, None, None, :] / T[:, None, :, None])
    psi0 = xg / (1.0 + xg)
    psi0 = np.ascontiguousarray(np.broadcast_to(psi0, (NRAY, N_SPECIES, NR, NE)))
    r_edge = np.ascontiguousarray(np.broadcast_to(r_edge1, (NRAY, NR + 1)))
    prob = dict(r_edge=r_edge, lapse=None, e_edge=e_edge, rho=rho,
                kappa_abs=kappa4, kappa_scat=kappa4.copy(), nes_coef=1e-41 * rho,
                dt=1e-6, outer_bc=0, scale=None)
    out = dict(problem=prob, psi0=psi0, ye0=ye, T0=T, spec=spec)
    if rays is not None:
        out = subset_rays(out, rays)
    return out


def subset_rays(inp, rays):
    """Restrict every per-ray array of an input dict to the selected rays."""
    prob = dict(inp['problem'])
    for key in ('r_edge', 'lapse', 'rho', 'kappa_abs', 'kappa_scat', 'nes_coef', 'u', 'eta1', 'pair_coef'):
        if prob.get(key) is not None:
            prob[key] = np.ascontiguousarray(prob[key][rays])
    out = dict(inp)
    out['problem'] = prob
    for key in ('psi0', 'ye0', 'T0'):
        out[key] = np.ascontiguousarray(inp[key][rays])
    return out


def flux_factor(rc, e_g):
    """Synthetic flux factor eta1 [n_ray, n_r, n_e]: 0.02 inside to 0.82 outside an
    energy-dependent neutrinosphere radius 30 km (E / 10 MeV)^(1/2), over a 5 km width."""
    r_nu = 30.0 * KM * np.sqrt(e_g / 10.0)
    return 0.02 + 0.4 * (1.0 + np.tanh((rc[:, :, None] - r_nu[None, None, :]) / (5.0 * KM)))


def make_shock_problem(config: int, rays=None, n_ray=None, n_r=None, n_e=None, beta_max=0.2):
    """Configuration `config` with an imposed accretion-shock velocity and a flux factor, for
    the shock-transport terms.  The velocity follows the imposed-shock test profile (Eq. t8):
    zero inside r_s - 15 km, falling linearly to -beta_max c at r_s, and -beta_max c (r_s / r)^2
    outside, with the shock radius r_s = 150 km (1 + d) varying by ray (d the recipe's seeded
    angular perturbation, |d| <= 0.05).  eta1 as in flux_factor, shared by the species."""
    out = make_problem(config, n_ray=n_ray, n_r=n_r, n_e=n_e)
    spec = out['spec']
    prob = dict(out['problem'])
    r_edge, e_edge = prob['r_edge'], prob['e_edge']
    rc = 0.5 * (r_edge[:, 1:] + r_edge[:, :-1])
    r_s = 150.0 * KM * (1.0 + angular_perturbation(spec, config, FIELD_SHOCK))[:, None]
    ramp = -beta_max * (rc - (r_s - 15.0 * KM)) / (15.0 * KM)
    beta = np.where(rc < r_s - 15.0 * KM, 0.0, np.where(rc < r_s, ramp, -beta_max * (r_s / rc) ** 2))
    prob['u'] = np.ascontiguousarray(beta * 2.99792458e10)
    e_g = np.sqrt(e_edge[1:] * e_edge[:-1])
    eta1 = flux_factor(rc, e_g)
    prob['eta1'] = np.ascontiguousarray(np.broadcast_to(eta1[:, None], rc.shape[:1] + (N_SPECIES,) + eta1.shape[1:]))
    out = dict(out, problem=prob)
    if rays is not None:
        out = subset_rays(out, rays)
    return out


def make_pair_problem(config: int, rays=None, n_ray=None, n_r=None, n_e=None, pair=1.0, chi=True):
    """Configuration `config` with the synthetic pair process: the pair kernel scale pair_coef =
    pair x the NES scale (1e-41 rho, cm^3/s) per zone and, with chi, the angular correction on with
    the flux factor of flux_factor (shared by the species)."""
    out = make_problem(config, n_ray=n_ray, n_r=n_r, n_e=n_e)
    prob = dict(out['problem'])
    prob['pair_coef'] = np.ascontiguousarray(1e-41 * pair * prob['rho'])
    if chi:
        r_edge, e_edge = prob['r_edge'], prob['e_edge']
        rc = 0.5 * (r_edge[:, 1:] + r_edge[:, :-1])
        eta1 = flux_factor(rc, np.sqrt(e_edge[1:] * e_edge[:-1]))
        prob['eta1'] = np.ascontiguousarray(np.broadcast_to(eta1[:, None], rc.shape[:1] + (N_SPECIES,) + eta1.shape[1:]))
        prob['pair_chi'] = True
    out = dict(out, problem=prob)
    if rays is not None:
        out = subset_rays(out, rays)
    return out


def stress_inputs(inp):
    """Matter pressure and inner mass for the neutrino stress and the lapse on a transport
    workload: p = 1.2435e15 (Ye rho)^(4/3) + rho kT / m_B (relativistic degenerate electrons plus
    ideal nucleons, erg/cm^3), and the mass inside the innermost edge that a uniform sphere of the
    innermost zone's density would hold (g).  Returns (p [n_ray, n_r], m_inner [n_ray])."""
    prob = inp['problem']
    rho, T, ye = prob['rho'], inp['T0'], inp['ye0']
    p = 1.2435e15 * (ye * rho) ** (4.0 / 3.0) + rho * T * 1.602176634e-6 / 1.674927e-24
    r0 = prob['r_edge'][:, 0]
    m_inner = 4.0 * np.pi / 3.0 * r0 ** 3 * rho[:, 0]
    return np.ascontiguousarray(p), np.ascontiguousarray(m_inner)


def _smooth_coeffs(rng, n_ray, modes=4):
    return rng.standard_normal((n_ray, modes))


def _smooth_eval(c, x, amp):
    """Per-ray smooth profiles amp * sum_m c_m sin(m pi x) / modes at the points x."""
    m = np.arange(1, c.shape[1] + 1)
    return amp * (c[:, :, None] * np.sin(np.pi * m[None, :, None] * x[None, None, :])).sum(axis=1) / c.shape[1]


def make_energy_advection(config: int, rays=None, n_ray=None, n_r=None, n_e=None):
    """Inputs of one energy-advection step on configuration `config`'s profile family.

    The zone state before the step is the transport profile (edges, rho) with the lapse
    a = sqrt(1 - 0.2 R_1 / R) (0.89 at the inner edge to 1); a hydrodynamics step is imitated by
    smooth seeded per-ray relative changes: of the density g (amplitude 1e-2), of the edge radii
    -g/3 (homologous compression or expansion) plus an independent part of amplitude 3e-4, and of
    the lapse (amplitude 1e-4).  psi is the transport profile's Fermi-Dirac occupation, with the electron
    neutrinos degenerate (chemical potential 3 T) where rho > 1e12 g/cm^3.  The flux factor eta1
    rises from 0.02 inside to 0.82 outside an energy-dependent neutrinosphere radius
    30 km (E / 10 MeV)^(1/2), over a 5 km width.  Returns a dict of numpy arrays."""
    base = make_problem(config, n_ray=n_ray, n_r=n_r, n_e=n_e)
    prob = base['problem']
    r_edge, rho, e_edge = prob['r_edge'], prob['rho'], prob['e_edge']
    NRAY, NR = rho.shape
    NE = len(e_edge) - 1
    rc = 0.5 * (r_edge[:, 1:] + r_edge[:, :-1])
    x_edge = np.log(r_edge[0] / r_edge[0, 0]) / np.log(r_edge[0, -1] / r_edge[0, 0])
    x_mid = 0.5 * (x_edge[1:] + x_edge[:-1])
    rng = np.random.default_rng(_seed(config, FIELD_HYDRO))
    c_g, c_r, c_a = (_smooth_coeffs(rng, NRAY) for _ in range(3))
    d_rho = _smooth_eval(c_g, x_mid, 1e-2)
    d_r = -_smooth_eval(c_g, x_edge, 1e-2) / 3.0 + _smooth_eval(c_r, x_edge, 3e-4)
    d_a = _smooth_eval(c_a, x_mid, 1e-4)
    lapse_n = np.sqrt(1.0 - 0.2 * rc[:, :1] / rc)
    e_g = np.sqrt(e_edge[1:] * e_edge[:-1])
    T = base['T0']
    mu = np.where(rho > 1e12, 3.0 * T, 0.0)
    psi = np.array(base['psi0'], copy=True)
    x = (e_g[None, None, :] - mu[:, :, None]) / T[:, :, None]
    z = np.exp(-np.abs(x))
    psi[:, 0] = np.where(x > 0.0, z / (1.0 + z), 1.0 / (1.0 + z))
    r_nu = 30.0 * KM * np.sqrt(e_g / 10.0)
    eta1 = 0.02 + 0.4 * (1.0 + np.tanh((rc[:, :, None] - r_nu[None, None, :]) / (5.0 * KM)))
    eta1 = np.ascontiguousarray(np.broadcast_to(eta1[:, None], (NRAY, N_SPECIES, NR, NE)))
    out = dict(e_edge=e_edge, r_edge_n=r_edge, r_edge_np1=np.ascontiguousarray(r_edge * (1.0 + d_r)),
               rho_n=rho, rho_np1=np.ascontiguousarray(rho * (1.0 + d_rho)),
               lapse_n=np.ascontiguousarray(lapse_n),
               lapse_np1=np.ascontiguousarray(lapse_n * (1.0 + d_a)),
               psi=np.ascontiguousarray(psi), eta1=eta1, spec=base['spec'])
    if rays is not None:
        for key in ('r_edge_n', 'r_edge_np1', 'rho_n', 'rho_np1', 'lapse_n', 'lapse_np1', 'psi', 'eta1'):
            out[key] = np.ascontiguousarray(out[key][rays])
    return out
