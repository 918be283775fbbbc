"""The synthetic pair process (Eq. d14, reading P1; angular correction Eqs. d16-d22, reading P2) on
the GPU: mgfld_step with pair_coef solves the coupled (nu, antinu) systems (2 n_e x 2 n_e zone
blocks), checked through the C ABI against the oracle's fully coupled Newton (tests/test_pair_oracle.py
pins the oracle's pair terms).

Gates as for the plain step: FP64 at 1e-12 on the benchmark-family rays and at the problem's
rounding floor on the deliberately stiff strong-coupling problems, the mixed path at 1e-10, each
step against the oracle's step from the same state; lepton number and energy balanced to rounding;
equilibrium with pairs a fixed point."""
import numpy as np
import pytest

from oracle import mgfld_oracle as O
from paper_1809_05608_gb300 import problems
from tests import parity_measures as PM
from tests import small_problems as SP

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

M = None


@pytest.fixture(scope='module', autouse=True)
def _lib():
    global M
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1809_05608_gb300 import mgfld
    M = mgfld
    M.lib()


def _with_chi(inp):
    """The problem with the angular correction on and a flux factor rising outward."""
    p = dict(inp['problem'], pair_chi=True)
    rc = 0.5 * (p['r_edge'][:, 1:] + p['r_edge'][:, :-1])
    p['eta1'] = np.broadcast_to(np.clip(rc / rc[:, -1:], 0.0, 1.0)[:, None, :, None], inp['psi0'].shape).copy()
    return dict(inp, problem=p)


def _benchmark_rays(rays=(0, 511, 1023), pair=1.0):
    """Rays of the 1024-ray 2D workload with the pair kernel at `pair` x the NES scale (1e-41 rho)."""
    inp = problems.make_problem(3, rays=list(rays))
    p = dict(inp['problem'])
    p['pair_coef'] = 1e-41 * pair * p['rho']
    return dict(inp, problem=p)


def _ledgers_balanced(rep, lep=1e-13, en=1e-12):
    L = rep['ledger']
    assert np.all(np.abs(L[:, 3]) <= lep * np.abs(L[:, 1]))
    assert np.all(np.abs(L[:, 7]) <= en * np.abs(L[:, 5]))


@pytest.mark.parametrize('precision', [0, 1])
@pytest.mark.parametrize('pair,chi', [(1.0, False), (30.0, False), (30.0, True)])
def test_strong_coupling_with_pairs(precision, pair, chi):
    inp = SP.strong(n_ray=2, n_r=12, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True, pair=pair)
    if chi:
        inp = _with_chi(inp)
    gate = SP.fp64_tolerance(inp) if precision == 0 else 1e-10
    _, codes, rep, _ = PM.stepwise(M, torch, inp, precision, 2, gate,
                                   f'strong, pair {pair}, chi {chi}, precision {precision}', tol=1e-11, max_iter=40)
    assert codes == [M.MGFLD_OK] * 2
    _ledgers_balanced(rep)
    print(f'  iterations {rep["iters"].tolist()}, factorisations {rep["factorizations"].tolist()}')


@pytest.mark.parametrize('precision,gate,tol', [(0, 1e-12, 1e-12), (1, 1e-10, 1e-11)])
def test_benchmark_rays_with_pairs(precision, gate, tol):
    """The pair process moves much energy between the neutrinos and the matter on these rays, so T
    (from the sources of every group, weighted by eps^3) follows the convergence of psi less
    tightly than psi does: the mixed path iterates to 1e-11 here to hold T at its 1e-10."""
    inp = _benchmark_rays()
    _, codes, rep, _ = PM.stepwise(M, torch, inp, precision, 2, gate, f'3 benchmark rays with pairs, {precision}',
                                   tol=tol, max_iter=40)
    assert codes == [M.MGFLD_OK] * 2
    _ledgers_balanced(rep, en=1e-12 if precision == 0 else 1e-10)
    # the process is not inert on these rays
    plain = problems.make_problem(3, rays=[0, 511, 1023])
    st = M.Stepper(plain, precision, tol=1e-12 if precision == 0 else 1e-10, max_iter=40)
    psi, ye, T = st.state_to_device(plain['psi0'], plain['ye0'], plain['T0'])
    assert st.step(psi, ye, T) == M.MGFLD_OK
    st2 = M.Stepper(inp, precision, tol=1e-12 if precision == 0 else 1e-10, max_iter=40)
    psi2, ye2, T2 = st2.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    assert st2.step(psi2, ye2, T2) == M.MGFLD_OK
    torch.cuda.synchronize()
    assert PM.normwise(psi2.cpu().numpy(), psi.cpu().numpy()) > 1e-8


def test_full_launch_with_pairs_sampled():
    """The 1024-ray launch with the pair process and its angular correction (mixed, tol 1e-10):
    sampled rays against the oracle, every ray converged and balanced."""
    full = _with_chi(_benchmark_rays(rays=range(1024)))
    st = M.Stepper(full, M.MGFLD_MIXED, tol=1e-10, max_iter=60)
    psi, ye, T = st.state_to_device(full['psi0'], full['ye0'], full['T0'])
    rc = st.step(psi, ye, T)
    torch.cuda.synchronize()
    rep = {k: v.cpu().numpy() for k, v in st.report.items()}
    assert rc == M.MGFLD_OK and np.all(rep['ray_status'] == 0)
    # lepton number balances to rounding; the energy to the iteration's tolerance (the sources of
    # Eq. a62b are those of the last iterate, whose residual is set by tol)
    _ledgers_balanced(rep, lep=1e-12, en=1e-10)
    rays = [5, 600, 1000]
    sub = problems.subset_rays(full, rays)
    out = O.step(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'])
    PM.report('1024-ray launch with pairs and chi (mixed), sampled rays', psi[rays].cpu().numpy(), out['psi'], 1e-10)
    print(f'  iterations {np.bincount(rep["iters"]).tolist()}')


def test_equilibrium_with_pairs_is_a_fixed_point():
    """Uniform matter at beta equilibrium, Fermi-Dirac occupations (mu_nubar = -mu_nu, so creation
    balances annihilation group by group) and a reflecting edge: the step leaves it unchanged,
    with pairs, NES and absorption together."""
    for precision in (0, 1):
        inp = SP.strong(n_ray=2, n_r=10, n_e=6, kabs=1e17, kscat=1e15, nes=20.0, bc=M.MGFLD_BC_REFLECT, pair=20.0)
        p = inp['problem']
        p['rho'] = np.full_like(p['rho'], 4e12)
        p['nes_coef'] = 1e-41 * p['rho'] * 20.0
        p['pair_coef'] = 1e-41 * p['rho'] * 20.0
        T = np.full_like(inp['T0'], 6.0)
        ye = np.full_like(inp['ye0'], 0.28)
        mu_q, _ = O.species_mu(p['rho'], T, ye, O.EosParams())
        eps, _ = O.local_energies(p['e_edge'], np.ones_like(T))
        psi0 = 1.0 / (1.0 + np.exp((eps[:, None] - mu_q[:, :, :, None]) / T[:, None, :, None]))
        inp = dict(inp, psi0=psi0, ye0=ye, T0=T)
        st = M.Stepper(inp, precision, tol=1e-12, max_iter=40)
        psi, ye1, T1 = st.state_to_device(psi0, ye, T)
        assert st.step(psi, ye1, T1) == M.MGFLD_OK
        torch.cuda.synchronize()
        assert PM.normwise(psi.cpu().numpy(), psi0) < 1e-13
        assert np.max(np.abs(T1.cpu().numpy() / T - 1)) < 1e-13


@pytest.mark.parametrize('n_e', [3, 7, 24])
def test_pair_block_widths(n_e):
    """Ragged and widest coupled blocks (2 n_e = 6, 14, 48 rows; padded to 8, 16, 48)."""
    inp = SP.strong(n_ray=2, n_r=9, n_e=n_e, kabs=1e13, kscat=1e14, nes=5.0, pair=5.0)
    _, codes, rep, _ = PM.stepwise(M, torch, inp, 0, 1, SP.fp64_tolerance(inp), f'pairs, n_e {n_e}', tol=1e-11,
                                   max_iter=40)
    assert codes == [M.MGFLD_OK]
    _ledgers_balanced(rep)
