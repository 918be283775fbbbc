"""Pins of the oracle's synthetic pair process (Eq. d14, zeroth moment, reading P1).

* Detailed balance (Eq. d12): at Fermi-Dirac occupations whose chemical potentials cancel in the
  pair (mu_nubar = -mu_nu, as beta equilibrium gives), creation and annihilation balance in every
  group, and a uniform medium in equilibrium with a reflecting edge stays put through a full step
  with pairs, absorption/emission and NES together.
* The process makes and destroys neutrinos in pairs: each flavour's lepton number is untouched
  for any occupations, so a full step conserves lepton number (and energy with matter) exactly.
* The Jacobian, now coupling the partner species, equals central differences of the residual.
* Switching the process on changes the result (it is not inert in the cases below).
The GPU's coupled pair systems are checked against this oracle in tests/test_gpu_pair.py."""
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


def test_gpu_assemble_refuses_the_pair_process():
    """mgfld_assemble writes the per-species system, which has no partner coupling: it refuses a
    problem with pair_coef in its argument checks (host only); mgfld_step takes the process with
    its coupled pair systems (tests/test_gpu_pair.py)."""
    import ctypes
    from paper_1809_05608_gb300 import mgfld as M
    fake = ctypes.c_void_p(0x10000)
    prob = M.Problem(*[fake] * 8, M.lib().mgfld_eos_default(), 1e-6, 0, None, None, fake)
    st = M.State(fake, fake, fake)
    dims = M.Dims(1, 8, 4, 4)
    sys_ = M.System(fake, fake, fake, fake)
    rc = M.lib().mgfld_assemble(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st), ctypes.byref(sys_),
                                ctypes.c_void_p(0x100000), 1 << 30, None)
    assert rc == M.MGFLD_EINVAL


# ------------------------------------------------------------------ angular correction (Eqs. d16-d22)

MU_GL, W_GL = np.polynomial.legendre.leggauss(24)
PHI = np.linspace(0.0, 2.0 * np.pi, 64, endpoint=False)        # exact for trigonometric degree < 64


def _pair_average(f_nu, f_bar, lo=-1.0, lo_bar=-1.0):
    """(4 pi)^-2 int dOmega dOmega' f_nu(mu) f_bar(mu') (1 - n.nbar)^2 by quadrature: Gauss-Legendre
    in mu on [lo, 1] and mu' on [lo_bar, 1], the rectangle rule in the relative azimuth (the
    integrand is a trigonometric polynomial of degree 2 in it)."""
    m = lo + (1.0 - lo) * 0.5 * (MU_GL + 1.0)
    wm = 0.5 * (1.0 - lo) * W_GL
    mb = lo_bar + (1.0 - lo_bar) * 0.5 * (MU_GL + 1.0)
    wb = 0.5 * (1.0 - lo_bar) * W_GL
    M, MB, P = np.meshgrid(m, mb, PHI, indexing='ij')
    dot = M * MB + np.sqrt(1.0 - M * M) * np.sqrt(1.0 - MB * MB) * np.cos(P)
    g = f_nu(M) * f_bar(MB) * (1.0 - dot) ** 2
    # dOmega = dmu dphi and the azimuth of the first direction integrates to 2 pi
    return np.einsum('i,j,ijk->', wm, wb, g) * (2.0 * np.pi) * (2.0 * np.pi / len(PHI)) / (4.0 * np.pi) ** 2


@pytest.mark.parametrize('eta,eta_bar', [(0.1, 0.3), (0.25, 0.25), (0.0, 0.4), (0.33, 0.05)])
def test_chi1_is_the_near_isotropic_angular_average(eta, eta_bar):
    """Eq. d16 as printed is the average for the distributions psi0 (1 + eta mu), relative to
    isotropic radiation of the same number.  Eq. d15 writes psi0 + 3 mu psi1, for which the same
    average is 1 - 3 eta etabar / 2 (shown here too): the paper is at odds with itself, and the
    oracle keeps the printed Eq. d16 (reading P2), which stays positive for any flux factors."""
    den = _pair_average(lambda m: np.ones_like(m), lambda m: np.ones_like(m))
    num = _pair_average(lambda m: 1.0 + m * eta, lambda m: 1.0 + m * eta_bar)
    assert abs(num / den - O.chi_isotropic(eta, eta_bar)) < 1e-13
    num3 = _pair_average(lambda m: 1.0 + 3.0 * m * eta, lambda m: 1.0 + 3.0 * m * eta_bar)
    assert abs(num3 / den - (1.0 - 1.5 * eta * eta_bar)) < 1e-13


@pytest.mark.parametrize('mu,mu_bar', [(0.3, 0.6), (0.8, 0.8), (-0.5, 0.2), (0.95, 0.1)])
def test_chi2_is_the_beamed_angular_average(mu, mu_bar):
    """Eq. d19 against the average over radiation confined to the cones mu >= mu_i with the
    occupation 2/(1 - mu_i) psi0 there (Eqs. d17-d18); Eq. d20 at equal cones."""
    num = _pair_average(lambda m: np.full_like(m, 2.0 / (1.0 - mu)), lambda m: np.full_like(m, 2.0 / (1.0 - mu_bar)),
                        lo=mu, lo_bar=mu_bar)
    den = _pair_average(lambda m: np.ones_like(m), lambda m: np.ones_like(m))
    assert abs(num / den - O.chi_beamed(mu, mu_bar)) < 1e-13
    if mu == mu_bar:
        assert abs(O.chi_beamed(mu, mu) - (1.0 - mu) ** 2 * (mu * mu + 4.0 * mu + 5.0) / 8.0) < 1e-15


def test_cone_extension_inside_the_neutrinosphere():
    """Eq. d22: outside R_nu the cone edge of Eq. d17; inside it falls to -1 (chi_2 = 1, isotropic),
    so chi = chi_1 there (Eq. d21)."""
    R_nu = 5e6
    assert abs(O.pair_mu(R_nu, 1e7) - np.sqrt(1.0 - 0.25)) < 1e-15
    assert O.pair_mu(R_nu, 4.9e6) < -0.04 and O.pair_mu(R_nu, 1e6) == -1.0
    assert O.chi_beamed(-1.0, -1.0) == 1.0
    eta = np.full((1, 4, 2, 3), 0.3)
    r_nu = np.full((1, 4, 3), R_nu)
    chi = O.pair_chi(eta, r_nu, np.array([[1e6, 5e7]]))
    assert np.allclose(chi[0, :, 0], O.chi_isotropic(0.3, 0.3), rtol=0, atol=1e-15)
    assert np.all(chi[0, :, 1] < O.chi_isotropic(0.3, 0.3))


def _with_chi(pair=30.0):
    inp = SP.strong(n_ray=2, n_r=12, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True, pair=pair)
    p = dict(inp['problem'], pair_chi=True)
    rc = 0.5 * (p['r_edge'][:, 1:] + p['r_edge'][:, :-1])
    p['eta1'] = np.broadcast_to(np.clip(rc / rc[:, -1:], 0.0, 1.0)[:, None, :, None], inp['psi0'].shape).copy()
    return dict(inp, problem=p)


def test_step_with_the_angular_correction():
    inp = _with_chi()
    out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    plain = O.step(dict(inp['problem'], pair_chi=False), inp['psi0'], inp['ye0'], inp['T0'])
    L = out['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-13 * np.abs(L[:, 1]))
    assert np.all(np.abs(L[:, 7]) <= 1e-12 * np.abs(L[:, 5]))
    assert np.max(O.rel_change(out['psi'] - plain['psi'], plain['psi'])) > 1e-6
    f = O.setup_step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    assert f.chi is not None and np.all(f.chi <= 1.0) and np.all(f.chi > 0.0)


def test_jacobian_with_the_angular_correction():
    inp = _with_chi()
    f = O.setup_step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    rng = np.random.default_rng(2)
    psi = np.clip(f.psi_n * (1 + 0.3 * rng.uniform(-1, 1, f.psi_n.shape)), 0, 1)
    ye = f.ye_n.copy()
    A, Bm, Bp = O.jacobian(f, psi, ye)
    r = 0
    J = O.dense_matrix(A[r], Bm[r], Bp[r])
    u0 = O.pack(psi, ye)
    M = u0.shape[-1]
    cols = range(0, u0[r].size, 7)
    for c in cols:
        h = 1e-6 * abs(u0[r].flat[c]) if c % M == M - 1 else 1e-2
        up = u0.copy(); up[r].flat[c] += h
        um = u0.copy(); um[r].flat[c] -= h
        gp = O.pack(*O.residual(f, *O.unpack(up, f.n_e)))[r]
        gm = O.pack(*O.residual(f, *O.unpack(um, f.n_e)))[r]
        col = ((gp - gm) / (2 * h)).reshape(-1)
        scale = np.maximum(np.abs(J[:, c]).max(), np.abs(col).max())
        assert np.max(np.abs(J[:, c] - col)) < 1e-6 * scale
