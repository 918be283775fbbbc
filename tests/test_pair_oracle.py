"""Pins of the oracle's synthetic pair process (Eq. d14, zeroth moment, reading P1).

* Detailed balance (Eq. d12): at Fermi-Dirac occupations whose chemical potentials cancel in the
  pair (mu_nubar = -mu_nu, as beta equilibrium gives), creation and annihilation balance in every
  group, and a uniform medium in equilibrium with a reflecting edge stays put through a full step
  with pairs, absorption/emission and NES together.
* The process makes and destroys neutrinos in pairs: each flavour's lepton number is untouched
  for any occupations, so a full step conserves lepton number (and energy with matter) exactly.
* The Jacobian, now coupling the partner species, equals central differences of the residual.
* Switching the process on changes the result (it is not inert in the cases below)."""
import numpy as np
import pytest

from oracle import mgfld_oracle as O
from tests import small_problems as SP


def test_detailed_balance_at_opposite_chemical_potentials():
    rng = np.random.default_rng(3)
    e_edge = np.geomspace(2.0, 250.0, 21)
    T = rng.uniform(2.0, 20.0, (2, 6))
    mu = rng.uniform(-15.0, 30.0, (2, 6))
    eps, deps = O.local_energies(e_edge, rng.uniform(0.8, 1.0, (2, 6)))
    w = eps**2 * deps
    mu_q = np.stack([mu, -mu, np.zeros_like(mu), np.zeros_like(mu)], axis=1)
    psi = 1.0 / (1.0 + np.exp((eps[:, None] - mu_q[..., None]) / T[:, None, :, None]))
    coef = rng.uniform(1e-30, 1e-27, (2, 6))
    a, p = O.pair_kernels(eps, T, coef)
    S = O.pair_source(psi, w, a, p)
    scale = O.C_NES * np.einsum('rikm,rim,rqim->rqik', a, w, psi[:, O.PAIR_PARTNER]) * psi
    assert np.max(np.abs(S) / scale) < 1e-13
    # away from it the process is not balanced
    S2 = O.pair_source(np.clip(psi * 1.1, 0.0, 1.0), w, a, p)
    assert np.max(np.abs(S2) / scale) > 1e-2


def test_pairs_carry_no_lepton_number():
    rng = np.random.default_rng(4)
    e_edge = np.geomspace(2.0, 250.0, 13)
    eps, deps = O.local_energies(e_edge, np.ones((3, 5)))
    w = eps**2 * deps
    psi = rng.uniform(0.0, 1.0, (3, 4, 5, 12))
    a, p = O.pair_kernels(eps, rng.uniform(3.0, 10.0, (3, 5)), rng.uniform(1e-30, 1e-28, (3, 5)))
    S = O.pair_source(psi, w, a, p)
    n = np.einsum('rik,rqik->rqi', w, S)
    scale = np.einsum('rik,rqik->rqi', w, np.abs(S)).max()
    assert np.max(np.abs(n[:, 0] - n[:, 1])) < 1e-14 * scale
    assert np.max(np.abs(n[:, 2] - n[:, 3])) < 1e-14 * scale
    assert np.max(np.abs(n[:, 0])) > 1e-3 * scale            # pairs are made (or destroyed)


def test_jacobian_with_pairs_matches_central_differences():
    inp = SP.strong(n_ray=1, n_r=5, n_e=3, kabs=1e17, kscat=1e15, nes=30.0, lapse=True, pair=30.0)
    f = O.setup_step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    rng = np.random.default_rng(1)
    psi = np.clip(f.psi_n * (1 + 0.3 * rng.uniform(-1, 1, f.psi_n.shape)), 0, 1)
    ye = f.ye_n * (1 + 0.01 * rng.uniform(-1, 1, f.ye_n.shape))
    A, Bm, Bp = O.jacobian(f, psi, ye)
    J = O.dense_matrix(A[0], Bm[0], Bp[0])
    u0 = O.pack(psi, ye)
    n = u0.size
    M = u0.shape[-1]
    Jfd = np.zeros((n, n))
    for c in range(n):
        h = 1e-6 * abs(u0.flat[c]) if c % M == M - 1 else 1e-2    # G is quadratic in psi
        up = u0.copy(); up.flat[c] += h
        um = u0.copy(); um.flat[c] -= h
        gp = O.pack(*O.residual(f, *O.unpack(up, f.n_e)))
        gm = O.pack(*O.residual(f, *O.unpack(um, f.n_e)))
        Jfd[:, c] = ((gp - gm) / (2 * h)).reshape(-1)
    scale = np.maximum(np.abs(J), np.abs(Jfd)).max(axis=1, keepdims=True)
    assert np.max(np.abs(J - Jfd) / scale) < 1e-6
    # the partner blocks are there: nu_e rows depend on nubar_e
    assert np.max(np.abs(A[0, :, 0:3, 3:6])) > 1e-3 * np.max(np.abs(A[0, :, 0:3, 0:3]))


@pytest.mark.parametrize('pair', [1.0, 30.0])
def test_step_with_pairs_conserves_lepton_number_and_energy(pair):
    inp = SP.strong(n_ray=2, n_r=12, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True, pair=pair)
    out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    plain = O.step(dict(inp['problem'], pair_coef=None), inp['psi0'], inp['ye0'], inp['T0'])
    L = out['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-13 * np.abs(L[:, 1]))
    assert np.all(np.abs(L[:, 7]) <= 1e-12 * np.abs(L[:, 5]))
    assert np.max(O.rel_change(out['psi'] - plain['psi'], plain['psi'])) > 1e-3
    assert out['iters'] <= 10


def test_equilibrium_with_pairs_is_a_fixed_point():
    inp = SP.strong(n_ray=2, n_r=10, n_e=6, kabs=1e17, kscat=1e15, nes=20.0, bc=O.BC_REFLECT, pair=20.0)
    p = inp['problem']
    p['rho'] = np.full_like(p['rho'], 4e12)
    p['nes_coef'] = 1e-41 * p['rho'] * 20.0
    p['pair_coef'] = 1e-41 * p['rho'] * 20.0
    T = np.full_like(inp['T0'], 6.0)
    ye = np.full_like(inp['ye0'], 0.28)
    mu_q, _ = O.species_mu(p['rho'], T, ye, O.EosParams())
    eps, _ = O.local_energies(p['e_edge'], np.ones_like(T))
    psi = 1.0 / (1.0 + np.exp((eps[:, None] - mu_q[:, :, :, None]) / T[:, None, :, None]))
    out = O.step(p, psi, ye, T)
    assert np.max(O.rel_change(out['psi'] - psi, psi)) < 1e-13
    assert np.max(np.abs(out['T'] / T - 1)) < 1e-13


def test_adjoint_refuses_pairs_before_touching_the_device():
    """mgfld_adjoint does not differentiate the pair process: refused by the argument checks
    (host only; the fake pointers are never dereferenced)."""
    import ctypes
    from paper_1809_05608_gb300 import mgfld as M
    fake = ctypes.c_void_p(0x10000)
    prob = M.Problem(*[fake] * 8, M.lib().mgfld_eos_default(), 1e-6, 0, None, None, fake)
    st = M.State(fake, fake, fake)
    io = M.AdjointIO(None, None, None, 1.0, fake, fake, fake, None, 0, 0.0, 0, 0.0)
    dims = M.Dims(1, 8, 4, 4)
    rc = M.lib().mgfld_adjoint(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st), ctypes.byref(st),
                               ctypes.byref(io), ctypes.c_void_p(0x100000), 1 << 30, None)
    assert rc == M.MGFLD_EINVAL


def test_gpu_step_refuses_the_pair_process():
    """The library's per-species blocks do not hold the partner coupling: mgfld_step and
    mgfld_assemble refuse a problem with pair_coef in their argument checks (host only)."""
    import ctypes
    from paper_1809_05608_gb300 import mgfld as M
    fake = ctypes.c_void_p(0x10000)
    prob = M.Problem(*[fake] * 8, M.lib().mgfld_eos_default(), 1e-6, 0, None, None, fake)
    st = M.State(fake, fake, fake)
    dims = M.Dims(1, 8, 4, 4)
    rc = M.lib().mgfld_step(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st),
                            ctypes.byref(M.step_opts()), None, ctypes.c_void_p(0x100000), 1 << 30, None)
    assert rc == M.MGFLD_EINVAL
    sys_ = M.System(fake, fake, fake, fake)
    rc = M.lib().mgfld_assemble(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st), ctypes.byref(sys_),
                                ctypes.c_void_p(0x100000), 1 << 30, None)
    assert rc == M.MGFLD_EINVAL
