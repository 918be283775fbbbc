"""Pins of the oracle's shock-transport terms (Sec. "Transport through a Shock").

The discrete frame corrections of Eqs. a91 and a97 are checked against a brute-force Lorentz
transformation of an explicit angular distribution f(eps, mu): the invariance of f under the maps
of Eq. a90 (for dpsi0) and the number count through a surface of Eq. a95 (for dpsi1), each
integrated over mu by Gauss-Legendre quadrature.  The odd part in beta of the exact transform is
the first-order term the paper keeps; a sign, index or frame mistake in the oracle fails it by
O(1).  Also pinned: the roll-in weights, the number moments the terms carry (summation by parts),
exact lepton-number conservation of a full step through a shock, and that a zero velocity
reproduces the shock-free step."""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import mgfld_oracle as O
from oracle.energy_advection_oracle import minerbo_eta2
from tests import small_problems as SP

MU, WMU = np.polynomial.legendre.leggauss(96)
P2 = lambda m: 0.5 * (3.0 * m * m - 1.0)


def _distribution(g, eta):
    """f(eps, mu) = g(eps) [1 + 3 eta(eps) mu + c(eps) P2(mu)] with c chosen so that
    psi2/psi0 equals the Minerbo factor of eta1 = eta (moments M_n = (1/2) int mu^n f dmu:
    M0 = g, M1 = eta g, M2 = (1/3 + 2c/15) g)."""
    def f(eps, mu):
        e = eta(eps)
        c = 7.5 * (minerbo_eta2(e) - 1.0 / 3.0)
        return g(eps) * (1.0 + 3.0 * e * mu + c * P2(mu))
    return f


G_A = lambda e: e * e * np.exp(-e / 9.0) / 81.0           # zone i
G_B = lambda e: 0.7 * e ** 1.5 * np.exp(-e / 12.0) / 40.0   # zone i + 1
ETA_A = lambda e: 0.15 + 0.1 * np.tanh(e / 30.0)
ETA_B = lambda e: 0.35 - 0.1 * np.tanh(e / 40.0)
F_A, F_B = _distribution(G_A, ETA_A), _distribution(G_B, ETA_B)


def _psi0_up_exact(f, eps, beta):
    """Zone i's psi0 seen from frame i+1 (moving at beta relative to frame i) at energy eps:
    f_{i+1}(eps', mu') = f_i(eps, mu) with Eq. a90's maps, inverted for (eps, mu)."""
    g = 1.0 / np.sqrt(1.0 - beta * beta)
    e_i = g * eps[:, None] * (1.0 + beta * MU[None, :])
    m_i = (MU[None, :] + beta) / (1.0 + beta * MU[None, :])
    return 0.5 * np.sum(WMU * f(e_i, m_i), axis=1)


def _psi1_down_exact(f, eps, beta):
    """Zone i+1's first moment transformed to frame i through the number count of Eq. a95:
    gamma^2 (1/2) int dmu f_{i+1}(gamma eps (1 - beta mu), (mu - beta)/(1 - beta mu)) (mu - beta)."""
    g = 1.0 / np.sqrt(1.0 - beta * beta)
    e1 = g * eps[:, None] * (1.0 - beta * MU[None, :])
    m1 = (MU[None, :] - beta) / (1.0 - beta * MU[None, :])
    return g * g * 0.5 * np.sum(WMU * f(e1, m1) * (MU[None, :] - beta), axis=1)


def _frozen(e_edge, beta_c, zones=(F_A, F_B)):
    """A two-zone frozen state whose group values are the distributions' moments at the group
    centres (Eq. a01b), for shock_corrections."""
    E, _ = O.group_centres(e_edge)
    n_e = len(E)
    psi = np.empty((1, 4, len(zones), n_e))
    eta1 = np.empty_like(psi)
    for i, (g, eta) in enumerate(((G_A, ETA_A), (G_B, ETA_B))[:len(zones)]):
        psi[0, :, i] = g(E)
        eta1[0, :, i] = eta(E)
    r_edge = np.array([[1e6, 2e6, 3e6]])[:, :len(zones) + 1]
    rc, area, vol = O.radial_geometry(r_edge)
    f = SimpleNamespace(psi_n=psi, lapse=np.ones((1, len(zones))), area=area)
    u = np.array([[0.0, beta_c * O.C_LIGHT]])
    return f, u, eta1, E


def _first_order(exact, f, eps, beta):
    """The O(beta) term of an exact transformation: its odd part in beta, with the O(beta^3)
    term removed by Richardson extrapolation between beta and 2 beta."""
    odd = lambda b: 0.5 * (exact(f, eps, b) - exact(f, eps, -b))
    return (8.0 * odd(beta) - odd(2.0 * beta)) / 6.0


@pytest.mark.parametrize('n_e', [20, 80])
def test_shock_terms_are_the_first_order_lorentz_transformation(n_e):
    """Second order in the group width (measured 5.1e-2, 2.6e-2 at 20 groups; 4x less per
    halving); a flipped sign gives a relative error of 2."""
    e_edge = np.geomspace(2.0, 250.0, n_e + 1)
    beta = 0.03
    f, u, eta1, E = _frozen(e_edge, beta)
    d0, d1, _ = O.shock_corrections(f, e_edge, u, eta1)
    up = _first_order(_psi0_up_exact, F_A, E, beta)
    down = _first_order(_psi1_down_exact, F_B, E, beta)
    inner = slice(2, -2)           # the end groups see the zero edge values of reading S4
    tol = 0.06 * (20.0 / n_e) ** 2
    for q in range(4):
        assert np.max(np.abs(d0[0, q, 0, inner] - up[inner])) < tol * np.max(np.abs(up[inner]))
        assert np.max(np.abs(d1[0, q, 0, inner] - down[inner])) < tol * np.max(np.abs(down[inner]))
    # the outermost edge has no zone above it
    assert np.all(d0[:, :, -1] == 0.0) and np.all(d1[:, :, -1] == 0.0)


def test_partial_roll_in_scales_the_terms():
    e_edge = np.geomspace(2.0, 250.0, 21)
    f, u, eta1, _ = _frozen(e_edge, 0.03)
    full = O.shock_corrections(f, e_edge, u, eta1)
    half = O.shock_corrections(f, e_edge, u * 0.5, eta1)      # |beta| = 0.015: weight 1/2
    assert np.allclose(half[0], 0.25 * full[0], rtol=1e-12, atol=0)
    assert np.allclose(half[1], 0.25 * full[1], rtol=1e-12, atol=0)


def test_energy_term_converges_at_second_order():
    """The discrete (1/eps^2) d(eps^3 m)/d eps of Eqs. a91/a97 on a geometric grid."""
    errs = []
    for n_e in (40, 80, 160):
        e_edge = np.geomspace(2.0, 250.0, n_e + 1)
        E, _ = O.group_centres(e_edge)
        m = G_A(E)
        exact = 3.0 * m + E * (2.0 * E / 81.0 - E * E / (9.0 * 81.0)) * np.exp(-E / 9.0)
        d = O.energy_divergence(e_edge[:-1], e_edge[1:], m)
        errs.append(np.max(np.abs(d - exact)[2:-2]) / np.max(np.abs(exact)))
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.2 and errs[1] / errs[2] > 3.2


def test_roll_in_weight():
    c = O.C_LIGHT
    u = np.array([[0.0, -0.005 * c, -0.02 * c, -0.035 * c, -0.060 * c, -0.061 * c]])
    beta, w = O.shock_beta(u)
    assert np.allclose(beta, [[-0.005, -0.015, -0.015, -0.025, -0.001]], rtol=1e-12, atol=1e-15)
    assert np.allclose(w, [[0.0, 0.5, 0.5, 1.0, 0.0]], rtol=0, atol=1e-12)


def test_shock_terms_number_moments():
    """Summation by parts with zero end values (reading S4): dpsi1 carries no neutrino number and
    dpsi0 removes beta sum_k w_k psi1_k, for any spectra."""
    rng = np.random.default_rng(11)
    e_edge = np.geomspace(2.0, 250.0, 21)
    n_r = 6
    psi = rng.uniform(0.0, 1.0, (2, 4, n_r, 20))
    eta1 = rng.uniform(0.0, 1.0, psi.shape)
    lapse = rng.uniform(0.8, 1.0, (2, n_r))
    r_edge = np.cumsum(rng.uniform(1e5, 2e5, (2, n_r + 1)), axis=1)
    _, area, _ = O.radial_geometry(r_edge)
    u = rng.uniform(-0.03, 0.03, (2, n_r)) * O.C_LIGHT
    f = SimpleNamespace(psi_n=psi, lapse=lapse, area=area)
    d0, d1, _ = O.shock_corrections(f, e_edge, u, eta1)
    beta, wgt = O.shock_beta(u)
    assert np.any((wgt > 0) & (wgt < 1)) and np.any(wgt == 1.0)
    eps, deps = O.local_energies(e_edge, lapse)
    w = (eps**2 * deps)[:, None]                              # [ray, 1, zone, group]
    n1 = np.sum(w * d1, axis=-1)
    assert np.max(np.abs(n1)) < 1e-13 * np.max(np.sum(w * psi, axis=-1))
    n0 = np.sum(w * d0, axis=-1)
    expect = np.zeros_like(n0)
    expect[:, :, :-1] = -(beta * wgt)[:, None, :] * np.sum((w * eta1 * psi)[:, :, :-1], axis=-1)
    assert np.max(np.abs(n0 - expect)) < 1e-13 * np.max(np.sum(w * psi, axis=-1))


def _shocked(inp, jump=-0.1):
    p = dict(inp['problem'])
    n_ray, n_r = p['rho'].shape
    u = np.zeros((n_ray, n_r))
    u[:, n_r // 2:] = jump * O.C_LIGHT
    u[:, n_r // 2 - 1] = 0.4 * jump * O.C_LIGHT               # a partly rolled-in edge below it
    rc = 0.5 * (p['r_edge'][:, 1:] + p['r_edge'][:, :-1])
    eta1 = np.broadcast_to(np.clip(0.05 + rc / rc[:, -1:], 0.0, 1.0)[:, None, :, None],
                           inp['psi0'].shape).copy()
    p['u'], p['eta1'] = u, eta1
    return p


def test_step_through_a_shock_conserves_lepton_number():
    """The frame terms move neutrinos between groups and frames without creating any (S4), so
    Eqs. a60-a62 still balance to rounding; the energy changes by the frame shift."""
    inp = SP.strong(n_ray=2, n_r=16, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True)
    p = _shocked(inp)
    out = O.step(p, inp['psi0'], inp['ye0'], inp['T0'])
    plain = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    L = out['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-13 * np.abs(L[:, 1]))
    # the shock terms matter here: the solution moves by far more than rounding
    assert np.max(np.abs(out['psi'] - plain['psi'])) > 1e-6 * np.max(np.abs(plain['psi']))


def test_zero_velocity_is_the_shock_free_step():
    inp = SP.strong(n_ray=1, n_r=10, n_e=4, kabs=1e16, kscat=1e15, nes=3.0)
    p = _shocked(inp, jump=0.0)
    out = O.step(p, inp['psi0'], inp['ye0'], inp['T0'])
    plain = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    assert np.array_equal(out['psi'], plain['psi']) and np.array_equal(out['ye'], plain['ye'])
