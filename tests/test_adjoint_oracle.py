"""Pins of the oracle adjoint: central finite differences of the oracle's own forward map.

J = gain-region (100-300 km) heating by nu_e + nubar_e summed over steps (reading R11);
gradients with respect to the per-(species, group) opacity scales and the initial psi."""
import numpy as np
import pytest

from oracle import mgfld_adjoint_oracle as A
from oracle import mgfld_oracle as O
from tests import small_problems as SP

torch = pytest.importorskip('torch')


def _problem():
    inp = SP.strong(n_ray=1, n_r=12, n_e=4, kabs=1e16, kscat=1e15, nes=10.0, lapse=True)
    return inp


def _J(inp, scale, psi0, n_steps):
    p = dict(inp['problem'], scale=scale)
    psi, ye, T = psi0, inp['ye0'], inp['T0']
    J = 0.0
    for _ in range(n_steps):
        o = O.step(p, psi, ye, T, rtol=1e-15)
        J += float(o['heating'].sum())
        psi, ye, T = o['psi'], o['ye'], o['T']
    return J


@pytest.mark.parametrize('n_steps', [1, 3])
def test_oracle_adjoint_matches_central_differences(n_steps):
    inp = _problem()
    n_e = inp['psi0'].shape[3]
    scale = np.ones((4, n_e)) * (1.0 + 0.1 * np.arange(4 * n_e).reshape(4, n_e) / (4 * n_e))
    J, g_psi, g_s = A.objective_and_gradients(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], scale,
                                              n_steps)
    assert np.isclose(J.sum(), _J(inp, scale, inp['psi0'], n_steps), rtol=1e-12)
    gmax = np.max(np.abs(g_s))
    for q in range(4):
        for k in range(n_e):
            h = 1e-5 * scale[q, k]
            sp, sm = scale.copy(), scale.copy()
            sp[q, k] += h
            sm[q, k] -= h
            fd = (_J(inp, sp, inp['psi0'], n_steps) - _J(inp, sm, inp['psi0'], n_steps)) / (2 * h)
            assert abs(fd - g_s[q, k]) <= 1e-6 * gmax + 1e-6 * abs(fd), (q, k, fd, g_s[q, k])
    rng = np.random.default_rng(5)
    psi0 = inp['psi0']
    big = np.argwhere(psi0 > 1e-4)
    gpmax = np.max(np.abs(g_psi))
    for idx in big[rng.choice(len(big), size=8, replace=False)]:
        idx = tuple(idx)
        h = 1e-6 * psi0[idx]
        pp, pm = psi0.copy(), psi0.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (_J(inp, scale, pp, n_steps) - _J(inp, scale, pm, n_steps)) / (2 * h)
        assert abs(fd - g_psi[idx]) <= 1e-6 * gpmax + 1e-6 * abs(fd), (idx, fd, g_psi[idx])
