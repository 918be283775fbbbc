"""Pin of the gain-region heating (reading R11), the objective of every adjoint check, against the
matter energy balance of Eq. a62b.

Eq. a62b gives each zone the internal-energy change rho (e^{n+1} - e^n) / m_B per unit volume from
the converged sources of all species (weights 1, 1, 2, 2).  With the heavy-lepton species switched
off (psi = 0 and kappa = 0, so their absorption, emission and NES sources vanish at every state),
the energy deposited in the matter of the zones with 100 km <= R_i <= 300 km by nu_e and nubar_e
must equal sum rho_i V_i (e_int(rho, T^{n+1}, Ye^{n+1}) - e_int(rho, T^n, Ye^n)) / m_B over those
zones: the matter's energy, from the equation of state at the step's own output, not from the
sources the heating sums.  A wrong sign, group weight, lapse weight, volume, radial window or a
missing flavour in the heating fails it; with the electron flavours off instead, the heating must
vanish while the heavy species still heat the matter."""
import numpy as np

from oracle import mgfld_oracle as O
from tests import small_problems as SP

KM = 1.0e5


def _species_off(inp, off):
    """The problem with the species `off` emptied: psi^n = 0 and zero opacities."""
    p = dict(inp['problem'])
    p['kappa_abs'] = p['kappa_abs'].copy()
    p['kappa_scat'] = p['kappa_scat'].copy()
    psi0 = inp['psi0'].copy()
    for q in off:
        p['kappa_abs'][:, q] = 0.0
        p['kappa_scat'][:, q] = 0.0
        psi0[:, q] = 0.0
    return dict(inp, problem=p, psi0=psi0)


def _matter_energy_gain(inp, out, r_lo=100 * KM, r_hi=300 * KM):
    """sum over the zones with r_lo <= R_i <= r_hi (R_i the mean of the zone's edges) of
    rho_i V_i (e^{n+1}_i - e^n_i) / m_B, V_i = 4 pi (R_{i+1/2}^3 - R_{i-1/2}^3) / 3, per ray (MeV)."""
    p = inp['problem']
    eos = O.EosParams()
    re = p['r_edge']
    rc = 0.5 * (re[:, 1:] + re[:, :-1])
    vol = 4.0 * np.pi * (re[:, 1:] ** 3 - re[:, :-1] ** 3) / 3.0
    e0 = O.e_int(p['rho'], inp['T0'], inp['ye0'], eos)
    e1 = O.e_int(p['rho'], out['T'], out['ye'], eos)
    gain = p['rho'] * vol * (e1 - e0) / eos.m_b
    inside = (rc >= r_lo) & (rc <= r_hi)
    return np.sum(np.where(inside, gain, 0.0), axis=1), np.sum(np.where(inside, np.abs(p['rho'] * vol * e1 / eos.m_b), 0.0), axis=1)


def _problem(lapse):
    inp = SP.strong(n_ray=2, n_r=24, n_e=6, kabs=3e16, kscat=1e15, nes=30.0, lapse=lapse)
    re = inp['problem']['r_edge']
    rc = 0.5 * (re[:, 1:] + re[:, :-1])
    assert np.sum((rc >= 100 * KM) & (rc <= 300 * KM)) >= 3          # the window holds zones
    return inp


def test_heating_equals_the_matter_energy_gain_of_the_electron_flavours():
    for lapse in (False, True):
        inp = _species_off(_problem(lapse), off=(2, 3))
        out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
        assert np.all(out['psi'][:, 2:] == 0.0)                           # the heavy species stay empty
        gain, size = _matter_energy_gain(inp, out)
        J = out['heating']
        # rounding: e^{n+1} - e^n is a difference of energies ~size (FP64, a few operations each)
        tol = 1e-14 * size + 1e-12 * np.abs(gain)
        print(f'lapse {lapse}: heating {J}, matter energy gain {gain}, rounding bound {tol}')
        assert np.all(np.abs(gain) > 1e3 * tol)                           # a real energy exchange
        assert np.all(np.abs(J - gain) <= tol)


def test_heating_vanishes_without_the_electron_flavours():
    inp = _species_off(_problem(True), off=(0, 1))
    out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    gain, size = _matter_energy_gain(inp, out)
    assert np.all(np.abs(gain) > 1e-10 * size)                            # the heavy species heat the matter
    assert np.all(out['heating'] == 0.0)


def test_heating_window_is_the_zone_centre_radius():
    """Moving the window's edges across one zone centre changes the heating by that zone's
    share of the matter energy gain exactly (the window selects zone centres)."""
    inp = _species_off(_problem(False), off=(2, 3))
    out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    f = out['frozen']
    S, _, _, _, _ = O.sources(f, out['psi'], out['ye'])
    re = inp['problem']['r_edge']
    rc = 0.5 * (re[0, 1:] + re[0, :-1])
    inside = np.nonzero((rc >= 100 * KM) & (rc <= 300 * KM))[0]
    i = inside[0]
    r_lo = 0.5 * (rc[i] + rc[i + 1])                                     # excludes zone i only
    narrower = O.gain_heating(f, S, r_lo=r_lo, r_hi=300 * KM)
    g_all, size = _matter_energy_gain(inp, out)
    g_less, _ = _matter_energy_gain(inp, out, r_lo=r_lo)
    assert np.all(np.abs((out['heating'] - narrower) - (g_all - g_less)) <= 1e-14 * size + 1e-12 * np.abs(g_all))


def _variant(f, S, kind):
    """The heating with one plausible mistake planted (CPU, from the oracle's sources)."""
    a = f.lapse
    w = f.w * f.eps
    mask = (f.rc >= 100 * KM) & (f.rc <= 300 * KM)
    if kind == 'no lapse weight':
        a = np.ones_like(a)
    if kind == 'eps^2 weight':
        w = f.w
    if kind == 'edge window':
        mask = (f.r_edge[:, 1:] >= 100 * KM) & (f.r_edge[:, 1:] <= 300 * KM)
    qs = [0] if kind == 'nu_e only' else [0, 1]
    sign = 1.0 if kind == 'sign' else -1.0
    per = sign * (a * O.C_LIGHT * f.dt) * f.vol * O.FOUR_PI_HC3 * np.einsum('rik,rqik->ri', w, S[:, qs])
    return np.sum(np.where(mask, per, 0.0), axis=1)


def test_planted_mistakes_in_the_heating_fail_the_pin():
    inp = _species_off(_problem(True), off=(2, 3))
    out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    f = out['frozen']
    S, _, _, _, _ = O.sources(f, out['psi'], out['ye'])
    gain, size = _matter_energy_gain(inp, out)
    tol = 1e-14 * size + 1e-12 * np.abs(gain)
    assert np.all(np.abs(_variant(f, S, 'none') - gain) <= tol)
    for kind in ('no lapse weight', 'eps^2 weight', 'edge window', 'nu_e only', 'sign'):
        bad = _variant(f, S, kind)
        assert np.any(np.abs(bad - gain) > 1e3 * tol), kind
