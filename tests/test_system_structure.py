"""Structure of the per-species linear systems that the mixed path factors without row exchanges.

The FP32 factor of the outer iteration eliminates each zone block of the block-tridiagonal
system (Eq. a62ae, psi part) without pivoting.  That is stable when the blocks met along the
elimination (the diagonal blocks and their Schur complements) are nonsingular M-matrices:
non-positive off-diagonal entries and an entrywise non-negative inverse.  The NES terms
conserve neutrino number (Eq. d8 with the detailed balance of Eq. d7), so a diagonal block's
columns weighted by the group weights w_k = eps_k^2 d eps_k sum to 1/(a c dt) + transport +
kappa_a + j > 0; the transport couplings are non-positive diagonal blocks.  These tests check
both facts on the oracle's Jacobian for the benchmark profile and the strong-coupling problem,
at psi^n and at a perturbed iterate, and then walk the two-sided elimination of every system."""
import numpy as np
import pytest

from oracle import mgfld_oracle as O
from paper_1809_05608_gb300 import problems
from tests import small_problems as SP


def _cases():
    bench = problems.make_problem(2, rays=[0, 97, 255], n_r=48)
    strong = SP.strong(n_ray=2, n_r=16, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True)
    return [('benchmark profile', bench), ('strong coupling', strong)]


def _species_blocks(A, Bm, Bp, n_e, q):
    sl = slice(q * n_e, (q + 1) * n_e)
    return A[:, :, sl, sl], Bm[:, :, sl], Bp[:, :, sl]


def _is_m_matrix(S):
    off = S - np.diag(np.diag(S))
    scale = np.max(np.abs(S))
    inv = np.linalg.inv(S)
    return (np.all(off <= 1e-14 * scale) and np.all(np.diag(S) > 0)
            and np.all(inv >= -1e-12 * np.max(np.abs(inv))))


@pytest.mark.parametrize('name,inp', _cases(), ids=['benchmark', 'strong'])
@pytest.mark.parametrize('perturb', [False, True])
def test_zone_blocks_are_weighted_column_dominant_z_matrices(name, inp, perturb):
    f = O.setup_step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    psi = f.psi_n
    if perturb:
        rng = np.random.default_rng(3)
        psi = np.clip(psi * (1 + 0.2 * rng.uniform(-1, 1, psi.shape)), 0.0, 1.0)
    A, Bm, Bp = O.jacobian(f, psi, f.ye_n)
    for q in range(O.N_SPECIES):
        D, L, U = _species_blocks(A, Bm, Bp, f.n_e, q)
        off = D * (1 - np.eye(f.n_e))
        assert np.all(off <= 0), name
        assert np.all(L <= 0) and np.all(U <= 0), name
        colsum = np.einsum('rik,rikm->rim', f.w, D)          # sum_k w_k D[k][k']
        margin = f.w / (f.lapse * O.C_LIGHT * f.dt)[:, :, None]
        # weighted column sums are at least the time-derivative term (up to rounding of the
        # cancelling NES rates)
        rate = np.einsum('rik,rikm->rim', f.w, np.abs(D))
        assert np.all(colsum >= margin - 1e-12 * rate), name


@pytest.mark.parametrize('name,inp', _cases(), ids=['benchmark', 'strong'])
def test_two_sided_elimination_meets_only_m_matrices(name, inp):
    f = O.setup_step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    A, Bm, Bp = O.jacobian(f, f.psi_n, f.ye_n)
    n_r = f.n_r
    m = n_r // 2
    for q in range(O.N_SPECIES):
        D, L, U = _species_blocks(A, Bm, Bp, f.n_e, q)
        for r in range(f.n_ray):
            top = D[r, 0]
            assert _is_m_matrix(top), (name, r, q, 0)
            for i in range(1, m):
                top = D[r, i] - np.diag(L[r, i]) @ np.linalg.inv(top) @ np.diag(U[r, i - 1])
                assert _is_m_matrix(top), (name, r, q, i)
            bot = D[r, n_r - 1]
            assert _is_m_matrix(bot), (name, r, q, n_r - 1)
            for i in range(n_r - 2, m, -1):
                bot = D[r, i] - np.diag(U[r, i]) @ np.linalg.inv(bot) @ np.diag(L[r, i + 1])
                assert _is_m_matrix(bot), (name, r, q, i)
            mid = D[r, m].copy()
            if m > 0:
                mid -= np.diag(L[r, m]) @ np.linalg.inv(top) @ np.diag(U[r, m - 1])
            if m < n_r - 1:
                mid -= np.diag(U[r, m]) @ np.linalg.inv(bot) @ np.diag(L[r, m + 1])
            assert _is_m_matrix(mid), (name, r, q, m)
