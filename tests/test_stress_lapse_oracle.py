"""Pins of the neutrino-stress and lapse oracle (Eqs. a62e-a62l) against the continuum
relations they difference: in the diffusion limit the stress is the radiation-pressure force
-(1/rho) dP_nu/dR (Eq. a62g's limit), converging at second order in the zone width; the lapse
scan integrates d ln a / dR = -(dp/dR - rho f) / (rho c^2) (Eq. a46 with Eq. a62j), which for a
polytrope without neutrinos has the closed form ln a_i - ln a_I = (h_I - h_i)/c^2 with the
enthalpy h = K gamma rho^(gamma-1) / (gamma - 1); the outer value is the Schwarzschild lapse of
the enclosed rest mass."""
import numpy as np
import pytest

from oracle import mgfld_oracle as O
from oracle import stress_lapse_oracle as S

E_EDGE = np.geomspace(2.0, 250.0, 21)


def _fd_problem(n_r, kappa=1e6):
    """One ray on R in [10, 20] km (uniform zones), rho ~ R^-2, T = 10 MeV (10 km / R), psi a
    Fermi-Dirac occupation at zone centres; opacities so large that the limiter is 1."""
    r_edge = np.linspace(1e6, 2e6, n_r + 1)[None, :]
    rc = 0.5 * (r_edge[:, 1:] + r_edge[:, :-1])
    rho = 1e12 * (rc / 1e6) ** -2
    T = 10.0 * 1e6 / rc
    eps, _ = O.local_energies(E_EDGE, np.ones_like(rc))
    psi = np.broadcast_to(1.0 / (np.exp(eps[:, None] / T[:, None, :, None]) + 1.0), (1, 4, n_r, 20)).copy()
    kap = np.full((1, 4, n_r, 20), kappa)
    prob = dict(r_edge=r_edge, lapse=None, e_edge=E_EDGE, rho=rho, kappa_abs=kap, kappa_scat=kap,
                nes_coef=None, dt=1e-6, outer_bc=O.BC_GHOST)
    return prob, psi, np.full_like(rc, 0.3), T, rc


def _continuum_stress(R):
    """-(1/rho) dP_nu/dR at R for the profile of _fd_problem, P_nu = sum_q N_q (4 pi/(hc)^3) / 3
    sum_k eps^3 d eps psi (the same group sums, differentiated exactly in R)."""
    E, dE = O.group_centres(E_EDGE)
    T = 10.0 * 1e6 / R
    dT = -10.0 * 1e6 / R**2
    x = E[None, :] / T[:, None]
    psi = 1.0 / (np.exp(x) + 1.0)
    dpsi = psi * (1.0 - psi) * x / T[:, None] * dT[:, None]
    dP = np.sum(O.STAT_WEIGHT) * O.FOUR_PI_HC3 / 3.0 * np.sum(E**3 * dE * dpsi, axis=1) * S.MEV_ERG
    rho = 1e12 * (R / 1e6) ** -2
    return -dP / rho


def test_diffusion_limit_stress_is_the_radiation_pressure_force():
    errs = []
    for n_r in (16, 32, 64):
        prob, psi, ye, T, rc = _fd_problem(n_r)
        out = S.stress_and_lapse(prob, psi, ye, T, np.zeros_like(rc), 0.0)
        f = O.setup_step(prob, psi, ye, T)
        assert np.all(np.abs(f.F[:, :, :-1] - 1.0) < 1e-10)           # the limiter is 1 here
        Re = prob['r_edge'][0, 1:-1]
        exact = _continuum_stress(Re)
        fe = out['f_edge'][0, :-1]
        assert np.all(fe > 0.0)                  # neutrinos pushing outward where psi falls outward
        errs.append(np.max(np.abs(fe - exact)) / np.max(np.abs(exact)))
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3


@pytest.mark.parametrize('gamma', [4.0 / 3.0, 2.5])
def test_lapse_scan_integrates_the_hydrostatic_relation(gamma):
    errs = []
    for n_r in (32, 64, 128):
        r_edge = np.linspace(1e6, 4e6, n_r + 1)[None, :]
        rc = 0.5 * (r_edge[:, 1:] + r_edge[:, :-1])
        _, _, vol = O.radial_geometry(r_edge)
        rho = 1e13 * (rc / 1e6) ** -2.5
        K = 5e14 if gamma < 2 else 1e-5
        p = K * rho**gamma
        a = S.lapse(r_edge, rho, vol, p, np.zeros_like(rho), 1.4 * 1.989e33)
        h = K * gamma / (gamma - 1.0) * rho ** (gamma - 1.0)
        exact = (h[:, -1:] - h) / O.C_LIGHT**2
        got = np.log(a) - np.log(a[:, -1:])
        assert np.all(got[:, :-1] < 0.0)             # the lapse falls inward
        errs.append(np.max(np.abs(got - exact)) / np.max(np.abs(exact)))
    assert errs[-1] < 2e-4                          # measured 7.9e-5 (4/3), 9.2e-5 (5/2)
    assert errs[0] / errs[1] > 3.7 and errs[1] / errs[2] > 3.7


def test_stress_term_of_the_lapse_scan():
    """p = 0 and a uniform outward stress f: ln a_i - ln a_I = -f (R_I - R_i) / c^2 up to
    second order in the zone width (Delta M / (4 pi R^2 rho) stands for the centre spacing)."""
    errs = []
    for n_r in (32, 64, 128):
        r_edge = np.linspace(1e6, 2e6, n_r + 1)[None, :]
        rc = 0.5 * (r_edge[:, 1:] + r_edge[:, :-1])
        _, _, vol = O.radial_geometry(r_edge)
        rho = np.full_like(rc, 1e11)
        f = 3e8
        a = S.lapse(r_edge, rho, vol, np.zeros_like(rc), np.full_like(rc, f), 0.0)
        exact = -f * (rc[:, -1:] - rc) / O.C_LIGHT**2
        got = np.log(a) - np.log(a[:, -1:])
        errs.append(np.max(np.abs(got - exact)) / np.max(np.abs(exact)))
    assert errs[-1] < 1e-4
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3


def test_outer_lapse_is_schwarzschild_of_the_enclosed_mass():
    r_edge = np.geomspace(1e6, 5e8, 101)[None, :]
    rc = 0.5 * (r_edge[:, 1:] + r_edge[:, :-1])
    _, _, vol = O.radial_geometry(r_edge)
    rho = np.full_like(rc, 2.5e9)
    m_in = 1.2 * 1.989e33
    a = S.lapse(r_edge, rho, vol, np.zeros_like(rc), np.zeros_like(rc), m_in)
    M = m_in + 2.5e9 * 4.0 * np.pi / 3.0 * (5e8**3 - 1e6**3)
    assert abs(a[0, -1] - np.sqrt(1.0 - 2.0 * 6.67430e-8 * M / (O.C_LIGHT**2 * 5e8))) < 1e-15
    assert np.all(a == a[0, -1])                    # no pressure, no stress: a flat lapse


def test_zone_stress_and_boundaries():
    prob, psi, ye, T, rc = _fd_problem(12)
    out = S.stress_and_lapse(prob, psi, ye, T, np.zeros_like(rc), 0.0)
    fe, fz = out['f_edge'], out['f_zone']
    assert fz[0, 0] == 0.5 * fe[0, 0]               # the centre edge carries no stress
    assert np.allclose(fz[0, 1:], 0.5 * (fe[0, 1:] + fe[0, :-1]), rtol=1e-15, atol=0)
    refl = dict(prob, outer_bc=O.BC_REFLECT)
    assert S.stress_and_lapse(refl, psi, ye, T, np.zeros_like(rc), 0.0)['f_edge'][0, -1] == 0.0
