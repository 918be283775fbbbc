"""Pins of the energy-advection oracle against what the paper and the mathematics fix:
closure limits, exactness of the parabolic reconstruction on polynomials, exact conservation of
neutrino number and energy, the identity step, the diffusion-limit scaling eps ~ rho^(1/3)
(Eq. a77), an exact one-group shift and the occupation limiter's conservation laws."""
import numpy as np
import pytest

from oracle import energy_advection_oracle as E

EDGES = np.geomspace(2.0, 250.0, 21)


def _random_case(seed, shape=(3, 4), n=20, scale=1e-3):
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, n)
    # Fermi-Dirac spectra in energy (T 3-8 MeV, mu 0-20 MeV): the top groups stay nearly empty, as
    # the method assumes; 1 % noise
    eps = E.group_centres(EDGES[:-1], EDGES[1:])
    T = rng.uniform(3.0, 8.0, shape)[..., None]
    mu = rng.uniform(0.0, 20.0, shape)[..., None]
    psi = 1.0 / (np.exp((eps - mu) / T) + 1.0) * (1.0 + 0.01 * rng.uniform(-1, 1, shape + (n,)))
    a_n = rng.uniform(0.8, 1.0, shape)
    r_n = rng.uniform(1e6, 1e8, shape)
    rho_n = rng.uniform(1e8, 1e12, shape)
    a1 = a_n * (1.0 + scale * rng.standard_normal(shape))
    r1 = r_n * (1.0 + scale * rng.standard_normal(shape))
    rho1 = rho_n * (1.0 + 10 * scale * rng.standard_normal(shape))
    # flux factors smooth in energy (forward-peaked at high energy), different per zone
    eta1 = np.clip(rng.uniform(0.0, 0.5, shape)[..., None] + 0.4 * x, 0.0, 1.0)
    return psi, a_n, a1, r_n, r1, rho_n, rho1, eta1


def test_minerbo_closure_limits():
    # Eq. a87 interpolates between the thick (1/3) and thin (1) Eddington factors
    assert E.minerbo_eta2(0.0) == pytest.approx(1.0 / 3.0, abs=1e-16)
    assert E.minerbo_eta2(1.0) == pytest.approx(1.0, abs=1e-15)
    x = np.linspace(0.0, 1.0, 101)
    e = E.minerbo_eta2(x)
    assert np.all(np.diff(e) > 0) and np.all((e >= 1.0 / 3.0) & (e <= 1.0))
    # free-streaming slope: d eta2 / d eta1 -> 0 at eta1 = 0 (even in eta1 near isotropy)
    assert (E.minerbo_eta2(1e-4) - 1.0 / 3.0) < 1e-8


@pytest.mark.parametrize('deg', [1, 2, 3])
def test_parabolic_interfaces_exact_on_polynomials(deg):
    """The interface values of Eq. h12 (read as Colella & Woodward's Eq. 1.6) interpolate the
    cell integrals by a cubic, so they are exact for number densities up to cubic in energy on a
    non-uniform grid (interior interfaces; the ghost groups at the ends are zero-slope copies)."""
    coef = [[3.0, 0.5], [1.0, 0.2, 0.01], [1e3, 0.5, -0.01, 1e-4]][deg - 1]
    f = np.polynomial.Polynomial(coef)
    F = f.integ()
    dx = np.diff(EDGES)
    avg = (F(EDGES[1:]) - F(EDGES[:-1])) / dx
    aL, aR, a6 = E.ppm_profile(avg, dx)
    ref = np.abs(f(EDGES)).max()
    assert np.max(np.abs(aL - f(EDGES[:-1]))[3:-3]) < 1e-14 * ref
    assert np.max(np.abs(aR - f(EDGES[1:]))[3:-3]) < 1e-14 * ref
    if deg <= 2:
        # the parabola of Eq. h22 reproduces a quadratic inside the cell as well
        for y in (0.1, 0.5, 0.9):
            sub = E.parabola_average_right(aL, aR, a6, y)
            lo = EDGES[1:] - y * dx
            exact = (F(EDGES[1:]) - F(lo)) / (y * dx)
            assert np.max(np.abs(sub - exact)[3:-3]) < 1e-13 * ref


def test_identity_when_nothing_changes():
    psi, a_n, _, r_n, _, rho_n, _, eta1 = _random_case(1)
    out = E.step(EDGES, a_n, a_n, r_n, r_n, rho_n, rho_n, psi, eta1)
    assert np.max(np.abs(out['psi'] - psi)) < 1e-15
    assert np.all(out['F'] == 0.0) and np.all(out['xi'] == 1.0)


@pytest.mark.parametrize('seed,scale', [(2, 1e-3), (3, 1e-2)])
def test_number_and_energy_are_conserved(seed, scale):
    psi, a_n, a1, r_n, r1, rho_n, rho1, eta1 = _random_case(seed, scale=scale)
    out = E.step(EDGES, a_n, a1, r_n, r1, rho_n, rho1, psi, eta1, limit=False)
    n0, _ = E.number_energy(psi, EDGES, a_n)
    n1, e1 = E.number_energy(out['psi'], EDGES, a1)
    # number per comoving mass (V = m / rho) is carried unchanged by both steps (Eqs. a74, p5)
    assert np.max(np.abs(n1 / rho1 - n0 / rho_n) / (n0 / rho_n)) < 1e-14
    # the remap keeps the energy the Lagrangian step left (Eqs. p6-p8)
    eps_d = out['eps_d']
    nd = out['psi_d'] * E.cube_moment(eps_d[..., :-1], eps_d[..., 1:])
    e_d = np.sum(nd * E.group_centres(eps_d[..., :-1], eps_d[..., 1:]), axis=-1)
    assert np.max(np.abs(e1 - e_d) / e_d) < 1e-14
    # smooth spectra with empty top groups need only a small energy fix
    assert np.all(np.abs(out['xi'] - 1.0) < 0.05)


def test_diffusion_limit_energy_scales_as_cube_root_of_density():
    """Eq. a77: with eta2 = 1/3 and no lapse change the energies scale as rho^(1/3); Eq. a79 is
    its first-order form, so the displaced edges agree to O(delta^2)."""
    for delta in (1e-3, 1e-4):
        rho_n, rho1 = 1e11, 1e11 * (1.0 + delta)
        r_n = 1e7
        r1 = r_n * (1.0 - delta / 3.0)          # any radius change: it cancels at eta2 = 1/3 to first order
        psi = np.full((1, 20), 0.5)
        eps_d, _, _ = E.lagrangian_shift(EDGES, [1.0], [1.0], [r_n], [r1], [rho_n], [rho1],
                                         np.full((1, 20), 1.0 / 3.0), psi)
        ratio = eps_d[0] / EDGES
        assert np.max(np.abs(ratio - (1.0 + delta) ** (1.0 / 3.0))) < 3 * delta * delta


def test_shift_by_one_group_moves_every_group_up():
    """Displaced grid = target grid shifted by exactly one group (geometric grid): every slice
    is a whole group, so group k's number lands in group k + 1 and, with the top group empty,
    the energy balance needs no correction (xi = 1)."""
    ratio = EDGES[1] / EDGES[0]
    n = 20
    rng = np.random.default_rng(5)
    nd = rng.uniform(0.1, 1.0, (2, n))
    nd[:, -1] = 0.0
    eps_t = np.broadcast_to(EDGES, (2, n + 1))
    eps_d = eps_t * ratio
    dxd = eps_d[..., 1:] - eps_d[..., :-1]
    aL, aR, a6 = E.ppm_profile(nd / dxd, dxd)
    F = E.remap_fluxes(eps_d, eps_t, aL, aR, a6)
    xi, div = E.energy_fix(nd, E.group_centres(eps_d[..., :-1], eps_d[..., 1:]),
                           E.group_centres(eps_t[..., :-1], eps_t[..., 1:]), F)
    new = nd + xi[:, None] * div
    assert np.allclose(xi, 1.0, rtol=0, atol=1e-13)
    assert np.max(np.abs(new[:, 1:] - nd[:, :-1])) < 1e-14
    assert np.max(np.abs(new[:, 0])) < 1e-15


def test_linear_density_is_remapped_exactly():
    """A number density linear in energy is reproduced by the parabolas, so the fluxes of a
    sub-group shift give the exact integrals over the target groups (before the energy fix)."""
    f = np.polynomial.Polynomial([5.0, -0.01])
    F_ = f.integ()
    s = 1.0 + 0.03
    eps_t = EDGES[None, :]
    eps_d = eps_t * s
    dxd = eps_d[..., 1:] - eps_d[..., :-1]
    nd = (F_(eps_d[..., 1:]) - F_(eps_d[..., :-1]))
    aL, aR, a6 = E.ppm_profile(nd / dxd, dxd)
    Fl = E.remap_fluxes(eps_d, eps_t, aL, aR, a6)
    new = nd + (Fl[..., :-1] - Fl[..., 1:])
    exact = F_(eps_t[..., 1:]) - F_(eps_t[..., :-1])
    assert np.max(np.abs(new - exact)[..., 3:-3]) < 1e-13 * np.max(np.abs(exact))


def test_occupation_limiter_conserves_number_and_energy():
    n = 20
    eps = EDGES
    c = E.group_centres(eps[:-1], eps[1:])
    d = np.diff(eps)
    x = np.linspace(0, 1, n)
    psi = 0.8 / (np.exp(6 * x - 2) + 1)
    psi[5] = 1.3
    psi[9] = 1.05
    out = E.limit_occupation(psi[None], c[None], d[None])[0]
    w = c * c * d
    assert abs(np.sum(out * w) - np.sum(psi * w)) < 1e-14 * np.sum(psi * w)
    assert abs(np.sum(out * w * c) - np.sum(psi * w * c)) < 1e-14 * np.sum(psi * w * c)
    assert np.all(out[:n - 2] <= 1.0 + 1e-15) and np.all(out >= 0.0)
    assert np.all(out[:5] == psi[:5])           # groups below the first overfilled one untouched


def test_occupation_limiter_leaves_groups_that_are_not_overfilled():
    """The limiter acts on psi > 1 only: negative occupations above (the remap has no positivity
    limiter) are not touched, and an overfilled group cannot draw a group below zero."""
    c = E.group_centres(EDGES[:-1], EDGES[1:])
    d = np.diff(EDGES)
    psi = np.full(20, 0.3)
    psi[7] = -1e-9
    out = E.limit_occupation(psi[None], c[None], d[None])[0]
    assert np.array_equal(out, psi)
    psi[5] = 1.2                                 # group 7 (= 5 + 2) holds nothing to remove
    out = E.limit_occupation(psi[None], c[None], d[None])[0]
    assert out[5] == psi[5] and out[7] == psi[7]


def test_rollout_at_a_shock():
    """Reading E8: with the displacement fully rolled out the grid does not move, so no slice
    crosses an edge and psi only takes Eq. a78's number factor; keep = 1 is the plain step; the
    zones on either side of a shock edge keep 1 - w of their displacement."""
    psi, a_n, a1, r_n, r1, rho_n, rho1, eta1 = _random_case(4, scale=1e-2)
    out0 = E.step(EDGES, a_n, a1, r_n, r1, rho_n, rho1, psi, eta1, limit=False, keep=np.zeros(a_n.shape))
    factor = (rho1 * a1**3) / (rho_n * a_n**3)
    assert np.max(np.abs(out0['psi'] - psi * factor[..., None]) / np.abs(psi * factor[..., None])) < 1e-15
    assert np.all(out0['F'] == 0.0)
    full = E.step(EDGES, a_n, a1, r_n, r1, rho_n, rho1, psi, eta1, limit=False)
    ones = E.step(EDGES, a_n, a1, r_n, r1, rho_n, rho1, psi, eta1, limit=False, keep=np.ones(a_n.shape))
    assert np.array_equal(full['psi'], ones['psi'])
    c = 2.99792458e10
    u = np.array([[0.0, 0.0, -0.015 * c, -0.05 * c, -0.05 * c, -0.05 * c]])
    keep = E.shock_keep(u)
    assert np.allclose(keep, [[1.0, 0.5, 0.0, 0.0, 1.0, 1.0]], rtol=0, atol=1e-12)
