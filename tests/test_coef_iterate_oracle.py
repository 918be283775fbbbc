"""Pins of the oracle's paper-literal flux coefficients (reading R12: lambda^(t) and the limiter of
Eq. a59 at n+1, formed again at every outer iterate).

* The root satisfies Eqs. a58/a59 with the coefficients formed from scratch at the root itself
  (a fresh setup at (psi, Ye) of the root, the time levels of the start state), while the frozen
  root of R2 does not: the test tells the two readings apart.
* The Jacobian the iteration uses carries the limiter's derivative: it equals central differences
  of the residual whose edge coefficients are re-formed at each perturbed state with the mean
  free path and the neutrinosphere held.
* Lepton number and energy stay conserved to rounding; the iteration converges in as few outer
  iterations as the frozen step."""
import numpy as np
import pytest

from oracle import mgfld_oracle as O
from paper_1809_05608_gb300 import problems
from tests import small_problems as SP


def fresh_residual(prob, psi_n, ye_n, T_n, psi, ye):
    """G of Eq. a58 at (psi, Ye) with every flux coefficient formed by a fresh setup at (psi, Ye),
    scaled by a c dt and normalised per ray and species by max |psi|."""
    f = O.setup_step(prob, psi, ye, T_n)
    f.psi_n = np.asarray(psi_n, dtype=np.float64)
    f.ye_n = np.asarray(ye_n, dtype=np.float64)
    G, GY = O.residual(f, psi, ye)
    G = G * (f.lapse * O.C_LIGHT * f.dt)[:, None, :, None]
    return float(np.max(np.max(np.abs(G), axis=(2, 3)) / np.max(np.abs(psi), axis=(2, 3))))


@pytest.mark.parametrize('case', ['bench ray', 'strong'])
def test_root_satisfies_the_equations_with_its_own_coefficients(case):
    if case == 'bench ray':
        inp = problems.make_problem(2, rays=[101])
    else:
        inp = SP.strong(n_ray=2, n_r=12, n_e=5, kabs=1e13, kscat=1e14, nes=5.0)
    p, psi_n, ye_n, T_n = inp['problem'], inp['psi0'], inp['ye0'], inp['T0']
    lit = O.step(p, psi_n, ye_n, T_n, coef_iterate=True)
    frozen = O.step(p, psi_n, ye_n, T_n)
    r_lit = fresh_residual(p, psi_n, ye_n, T_n, lit['psi'], lit['ye'])
    r_frz = fresh_residual(p, psi_n, ye_n, T_n, frozen['psi'], frozen['ye'])
    print(f'{case}: residual with own coefficients {r_lit:.1e} (frozen root {r_frz:.1e}), '
          f'iterations {lit["iters"]} vs {frozen["iters"]}')
    assert r_lit < 1e-11 and r_frz > 1e3 * r_lit
    assert lit['iters'] <= frozen['iters'] + 2
    L = lit['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-13 * np.abs(L[:, 1]))
    assert np.all(np.abs(L[:, 7]) <= 1e-12 * np.abs(L[:, 5]))


def test_jacobian_carries_the_limiter_derivative():
    """Central differences (step 1e-5 psi) on the entries whose psi is resolvable (>= 1e-6; the
    rows of emptier groups are dominated by the time term at that step); a hot medium (3 T) so
    that several groups are populated.  The flux parts are ~1e-5 of the diagonal here, so a
    wrong limiter derivative moves the diagonal and the couplings far beyond the bounds."""
    inp = SP.strong(n_ray=1, n_r=6, n_e=3, kabs=1e12, kscat=1e13, nes=2.0)
    p = inp['problem']
    f = O.setup_step(p, inp['psi0'], inp['ye0'], 3.0 * inp['T0'])
    rng = np.random.default_rng(7)
    psi = f.psi_n * (1.0 + 0.05 * rng.uniform(-1, 1, f.psi_n.shape))
    ye = f.ye_n.copy()
    f.coef_iterate = True
    O.edge_coefficients(f, psi)                        # the limiter's derivatives at psi
    A, Bm, Bp = O.jacobian(f, psi, ye)

    def G_at(x):
        g = O.Frozen()
        g.__dict__.update(f.__dict__)
        g.alpha, g.D, g.F = O.edge_coefficients(g, x)   # lambda and R_nu held
        return O.residual(g, x, ye)[0]

    n_e = f.n_e
    worst_d = worst_o = 0.0
    checked = 0
    for i in range(f.n_r):
        for q in range(4):
            for k in range(n_e):
                if psi[0, q, i, k] < 1e-6:
                    continue
                h = 1e-5 * psi[0, q, i, k]
                xp, xm = psi.copy(), psi.copy()
                xp[0, q, i, k] += h
                xm[0, q, i, k] -= h
                col = (G_at(xp) - G_at(xm)) / (2 * h)          # d G / d psi_(q, i, k)
                a = q * n_e + k
                worst_d = max(worst_d, abs(col[0, q, i, k] - A[0, i, a, a]) / abs(A[0, i, a, a]))
                # couplings, measured against their row's diagonal (the scale of its rounding)
                if i > 0:   # zone i-1's equation couples to psi_i through its upper block
                    worst_o = max(worst_o, abs(col[0, q, i - 1, k] - Bp[0, i - 1, a]) / abs(A[0, i - 1, a, a]))
                if i < f.n_r - 1:
                    worst_o = max(worst_o, abs(col[0, q, i + 1, k] - Bm[0, i + 1, a]) / abs(A[0, i + 1, a, a]))
                checked += 1
    print(f'{checked} columns: diagonal {worst_d:.1e}, couplings {worst_o:.1e}')
    assert checked >= 20 and worst_d < 1e-6 and worst_o < 1e-7
    # and it differs from the frozen Jacobian, whose couplings hold the limiter
    f.coef_iterate = False
    _, _, Bp0 = O.jacobian(f, psi, ye)
    assert np.max(np.abs(Bp0 - Bp)) > 1e-3 * np.max(np.abs(Bp))


def test_not_combined_with_the_shock_terms():
    """Refused by the argument checks (host only; the fake pointers are never dereferenced)."""
    import ctypes
    from paper_1809_05608_gb300 import mgfld
    fake = ctypes.c_void_p(0x10000)
    prob = mgfld.Problem(*[fake] * 8, mgfld.lib().mgfld_eos_default(), 1e-6, 0, fake, None)
    st = mgfld.State(fake, fake, fake)
    dims = mgfld.Dims(1, 8, 4, 4)
    opts = mgfld.step_opts(coef_iterate=True)
    rc = mgfld.lib().mgfld_step(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st), ctypes.byref(opts),
                                None, ctypes.c_void_p(0x100000), 1 << 30, None)
    assert rc == mgfld.MGFLD_EINVAL
    with pytest.raises(NotImplementedError):
        inp = problems.make_shock_problem(1)
        O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], coef_iterate=True)
