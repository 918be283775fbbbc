"""GPU (libmgfld through the C ABI) vs the CPU oracle, on seeded synthetic inputs.

Error measure (reading of "relative in psi0"): per ray and species, the max-norm
of psi_gpu - psi_oracle over all zones and groups divided by the max-norm of
psi_oracle.  Tolerances: FP64 path 1e-12, mixed path 1e-10 (as stated for the
method) on the single ray and every ray of the benchmark configurations, with the per-group
zone-max measure and the elementwise error printed beside (tests/parity_measures.py); only the
deliberately stiff strong-coupling problems take their FP64 rounding floor, ~1e-11 (NES rates
~1e4/(a c dt) amplify residual rounding)."""
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


def run_gpu(inp, precision=0, steps=1, **kw):
    kw.setdefault('tol', 1e-12 if precision == 0 else 1e-11)
    kw.setdefault('max_iter', 40)
    st = M.Stepper(inp, precision, **kw)
    psi, ye, T = st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    codes = [st.step(psi, ye, T) for _ in range(steps)]
    torch.cuda.synchronize()
    rep = {k: v.cpu().numpy() for k, v in st.report.items()}
    return psi.cpu().numpy(), ye.cpu().numpy(), T.cpu().numpy(), codes, rep


def run_oracle(inp, steps=1):
    psi, ye, T, outs = O.run_steps(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], steps)
    return psi, ye, T, outs


def normwise(a, b):
    return float(np.max(O.rel_change(a - b, b)))


def backward_error(inp, psi_prev, ye_prev, T_prev, psi, ye):
    """The oracle's own residual of Eqs. a58/a62a evaluated at a candidate root, scaled by
    a c dt and normalised per ray and species by max |psi| (rounding level ~1e-15)."""
    f = O.setup_step(inp['problem'], psi_prev, ye_prev, T_prev)
    G, GY = O.residual(f, psi, ye)
    scaled = G * (f.lapse * O.C_LIGHT * f.dt)[:, None, :, None]
    return float(np.max(np.max(np.abs(scaled), axis=(2, 3)) / np.max(np.abs(psi), axis=(2, 3))))


def fp64_gate(inp):
    """1e-12 (the stated FP64 parity target), widened to the problem's FP64 rounding floor
    max(1e-12, 1e-14 x stiffness) where the stiff NES terms make the root itself uncertain
    at that level (see small_problems.fp64_tolerance)."""
    return SP.fp64_tolerance(inp)


def test_single_ray_fp64_matches_oracle():
    inp = problems.make_problem(1)
    psi, ye, T, codes, rep = run_gpu(inp)
    psi_o, ye_o, T_o, outs = run_oracle(inp)
    assert codes == [M.MGFLD_OK]
    fwd = PM.report('single ray fp64', psi, psi_o, 1e-12)
    bwd = backward_error(inp, inp['psi0'], inp['ye0'], inp['T0'], psi, ye)
    bwd_o = backward_error(inp, inp['psi0'], inp['ye0'], inp['T0'], psi_o, ye_o)
    print(f'single ray fp64: forward {fwd:.2e}, backward {bwd:.2e} (oracle at its root {bwd_o:.2e})')
    assert fwd < 1e-12
    assert bwd < 10 * max(bwd_o, 1e-15)
    assert np.max(np.abs(ye - ye_o)) < 1e-14
    assert np.max(np.abs(T / T_o - 1)) < 1e-12
    L, Lo = rep['ledger'], outs[0]['ledger']
    assert np.allclose(L[:, [0, 1, 4, 5]], Lo[:, [0, 1, 4, 5]], rtol=1e-12, atol=0)
    assert np.all(np.abs(L[:, 3]) <= 1e-13 * np.abs(L[:, 1]))
    assert np.all(np.abs(L[:, 7]) <= 1e-13 * np.abs(L[:, 5]))


def test_2d_full_size_ray_subset_fp64_two_steps():
    """256-ray 512x20 profile family; rays are independent, so a subset is exact parity.
    Each step against the oracle's step from the same state at 1e-12, the two-step drift at
    2e-12, and the backward error (the oracle's residual at the GPU result) at rounding level."""
    inp = problems.make_problem(2, rays=[0, 101, 255])
    (psi, ye, T), codes, rep, (psi_o, ye_o, T_o) = PM.stepwise(M, torch, inp, 0, 2, 1e-12, '2d rays fp64',
                                                               tol=1e-12, max_iter=40)
    assert codes == [M.MGFLD_OK] * 2
    psi1, ye1, T1, _, _ = run_gpu(inp, steps=1)
    bwd = backward_error(inp, psi1, ye1, T1, psi, ye)
    o1 = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    bwd_o = backward_error(inp, o1['psi'], o1['ye'], o1['T'], psi_o, ye_o)
    print(f'  backward {bwd:.2e} (oracle {bwd_o:.2e})')
    assert bwd < 10 * max(bwd_o, 1e-15)
    assert np.max(np.abs(ye - ye_o)) < 1e-14


def test_full_launch_256_rays_sampled_against_oracle():
    """The full 256-ray launch of the 2D FP64 configuration; sampled rays vs the oracle at 1e-12."""
    full = problems.make_problem(2)
    psi, ye, T, codes, rep = run_gpu(full)
    assert codes == [M.MGFLD_OK]
    rays = [3, 128, 200]
    sub = problems.subset_rays(full, rays)
    psi_o, ye_o, T_o, _ = run_oracle(sub)
    PM.report('256-ray launch, sampled rays', psi[rays], psi_o, 1e-12)
    bwd = backward_error(sub, sub['psi0'], sub['ye0'], sub['T0'], psi[rays], ye[rays])
    bwd_o = backward_error(sub, sub['psi0'], sub['ye0'], sub['T0'], psi_o, ye_o)
    print(f'  backward {bwd:.2e} (oracle {bwd_o:.2e})')
    assert bwd < 10 * max(bwd_o, 1e-15)
    assert np.max(np.abs(T[rays] / T_o - 1)) < 1e-12
    assert np.all(rep['ray_status'] == 0) and np.all(rep['iters'] >= 2)


@pytest.mark.parametrize('kind', ['2d', 'strong'])
def test_fp64_modified_newton_matches_oracle(kind):
    """FP64 factors reused while the iteration contracts (refactor_ratio 0.1): the same root as
    the oracle's Newton, with fewer factorisations than iterations; each step against the
    oracle's step from the same state."""
    if kind == '2d':
        inp = problems.make_problem(2, rays=[0, 101, 255])
        tol, gate = 1e-12, 1e-12
    else:
        inp = SP.strong(n_ray=2, n_r=16, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True)
        tol, gate = 1e-11, fp64_gate(inp)
    _, codes, rep, _ = PM.stepwise(M, torch, inp, 0, 2, gate, f'fp64 modified Newton ({kind})', tol=tol,
                                   max_iter=40, refactor_ratio=0.1)
    assert codes == [M.MGFLD_OK] * 2
    print(f'  iterations {rep["iters"].tolist()}, factorisations {rep["factorizations"].tolist()}')
    assert np.all(rep['factorizations'] < rep['iters'])


@pytest.mark.parametrize('lapse', [False, True])
def test_strong_coupling_fp64(lapse):
    inp = SP.strong(n_ray=2, n_r=16, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=lapse)
    psi, ye, T, codes, rep = run_gpu(inp, steps=2, tol=1e-11)
    psi_o, ye_o, T_o, outs = run_oracle(inp, steps=2)
    assert codes == [M.MGFLD_OK] * 2
    assert normwise(psi, psi_o) < SP.fp64_tolerance(inp)
    assert np.max(np.abs(ye / ye_o - 1)) < 1e-12
    assert np.max(np.abs(T / T_o - 1)) < 1e-11
    L = rep['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-13 * np.abs(L[:, 1]))
    assert np.all(np.abs(L[:, 7]) <= 1e-12 * np.abs(L[:, 5]))


@pytest.mark.parametrize('n_e', [1, 3, 7, 12, 24, 32])
def test_ragged_group_counts(n_e):
    """Every padded block size (4, 8, 12, 24, 32) including ragged n_e < padded size."""
    inp = SP.strong(n_ray=3, n_r=9, n_e=n_e, kabs=1e13, kscat=1e14, nes=5.0)
    psi, ye, T, codes, _ = run_gpu(inp, tol=1e-11)
    psi_o, ye_o, T_o, _ = run_oracle(inp)
    assert codes == [M.MGFLD_OK]
    tol = SP.fp64_tolerance(inp)
    assert normwise(psi, psi_o) < tol
    assert np.max(np.abs(T / T_o - 1)) < tol


def test_single_zone_and_reflecting_equilibrium():
    """Uniform matter at beta equilibrium with a reflecting outer edge is a fixed point."""
    inp = SP.strong(n_ray=2, n_r=6, n_e=6, kabs=1e17, kscat=1e15, nes=20.0, bc=M.MGFLD_BC_REFLECT)
    p = inp['problem']
    p['rho'] = np.full_like(p['rho'], 4e12)
    p['nes_coef'] = 1e-41 * p['rho'] * 20.0
    T = np.full_like(inp['T0'], 6.0)
    ye = np.full_like(inp['ye0'], 0.28)
    mu_q, _ = O.species_mu(p['rho'], T, ye, O.EosParams())
    eps, _ = O.local_energies(p['e_edge'], np.ones_like(T))
    psi0 = 1.0 / (1.0 + np.exp((eps[:, None] - mu_q[:, :, :, None]) / T[:, None, :, None]))
    inp = dict(inp, psi0=psi0, ye0=ye, T0=T)
    psi, ye1, T1, codes, _ = run_gpu(inp)
    assert codes == [M.MGFLD_OK]
    assert normwise(psi, psi0) < 1e-13
    assert np.max(np.abs(T1 / T - 1)) < 1e-13
    one = SP.strong(n_ray=2, n_r=1, n_e=4)
    psi, _, T1, codes, _ = run_gpu(one)
    psi_o, _, T_o, _ = run_oracle(one)
    assert codes == [M.MGFLD_OK] and normwise(psi, psi_o) < 1e-12


def test_mixed_precision_matches_oracle_to_1e10():
    inp = problems.make_problem(3, rays=[0, 511, 1023])
    _, codes, rep, _ = PM.stepwise(M, torch, inp, 1, 2, 1e-10, 'mixed 1024-ray config rays', tol=1e-10, max_iter=40)
    assert codes == [M.MGFLD_OK] * 2
    assert np.all(rep['factorizations'] >= 1)


def test_mixed_strong_coupling():
    inp = SP.strong(n_ray=2, n_r=16, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True)
    psi, ye, T, codes, rep = run_gpu(inp, precision=1, steps=2, tol=1e-11)
    psi_o, ye_o, T_o, _ = run_oracle(inp, steps=2)
    assert codes == [M.MGFLD_OK] * 2
    assert normwise(psi, psi_o) < 1e-10


def test_assemble_matches_oracle_jacobian_and_residual():
    inp = SP.strong(n_ray=2, n_r=7, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True)
    n_ray, _, n_r, n_e = inp['psi0'].shape
    st = M.Stepper(inp)
    psi, ye, T = st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    dims = M.Dims(n_ray, n_r, n_e, 4)
    sys = dict(diag=torch.zeros(n_ray, 4, n_r, n_e, n_e, dtype=torch.float64, device='cuda'),
               lower=torch.zeros(n_ray, 4, n_r, n_e, dtype=torch.float64, device='cuda'),
               upper=torch.zeros(n_ray, 4, n_r, n_e, dtype=torch.float64, device='cuda'),
               rhs=torch.zeros(n_ray, 4, n_r, n_e, dtype=torch.float64, device='cuda'))
    assert M.mgfld_assemble(dims, st.prob.struct, psi, ye, T, sys, st.ws) == M.MGFLD_OK
    torch.cuda.synchronize()
    f = O.setup_step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    A, Bm, Bp = O.jacobian(f, f.psi_n, f.ye_n)
    G, _ = O.residual(f, f.psi_n, f.ye_n)
    D = sys['diag'].cpu().numpy()
    # The NES self-scattering term enters the diagonal twice with opposite signs (it
    # cancels exactly), so rounding is measured against the size of the summed terms.
    mu_q, _ = O.species_mu(f.rho, f.T_n, f.ye_n, f.eos)
    j, _ = O.emissivity(f.kappa_abs, f.eps, mu_q, f.T_n)
    terms = O.nes_inverse_mfp(f.psi_n, f.w, f.phi_out, f.phi_in) + j + f.kappa_abs
    for q in range(4):
        blk = A[:, :, q * n_e:(q + 1) * n_e, q * n_e:(q + 1) * n_e]
        scale = np.maximum(np.abs(blk).max(axis=-1), terms[:, q])[..., None]
        assert np.max(np.abs(D[:, q] - blk) / scale) < 1e-13
        lo = Bm[:, :, q * n_e:(q + 1) * n_e]
        up = Bp[:, :, q * n_e:(q + 1) * n_e]
        assert np.allclose(sys['lower'].cpu().numpy()[:, q], lo, rtol=1e-13, atol=0)
        assert np.allclose(sys['upper'].cpu().numpy()[:, q], up, rtol=1e-13, atol=0)
    rate = terms + 1.0 / (f.lapse[:, None, :, None] * O.C_LIGHT * f.dt)
    rscale = np.max(rate, axis=(2, 3), keepdims=True) * np.max(np.abs(f.psi_n), axis=(2, 3), keepdims=True)
    assert np.max(np.abs(sys['rhs'].cpu().numpy() + G) / rscale) < 1e-13


@pytest.mark.parametrize('precision,unit', [(0, 2.2e-16), (1, 1.2e-7)])
def test_factor_solve_matches_dense_lu(precision, unit):
    """mgfld_factor + mgfld_solve on random block-tridiagonal systems (some needing
    pivoting) against LAPACK on the dense matrix of each system."""
    rng = np.random.default_rng(11)
    for n_e, n_r in ((5, 6), (20, 9), (12, 4), (7, 1), (6, 2), (4, 3), (20, 64)):
        n_ray = 3
        # Block-diagonally dominant systems (the regime of the transport blocks), one of them
        # with its dominant entries off the diagonal so that every block needs row exchanges.
        diag = rng.standard_normal((n_ray, 4, n_r, n_e, n_e))
        diag[0] += 4 * n_e * np.eye(n_e)
        perm = np.roll(np.eye(n_e), 1, axis=0)
        diag[1] = diag[1] * 0.5 + 4 * n_e * perm
        diag[2] += 2.5 * n_e * np.eye(n_e)
        lower = rng.standard_normal((n_ray, 4, n_r, n_e)); lower[:, :, 0] = 0
        upper = rng.standard_normal((n_ray, 4, n_r, n_e)); upper[:, :, -1] = 0
        rhs = rng.standard_normal((n_ray, 4, n_r, n_e))
        dev = {k: torch.as_tensor(v, device='cuda') for k, v in
               dict(diag=diag, lower=lower, upper=upper, rhs=rhs).items()}
        dims = M.Dims(n_ray, n_r, n_e, 4)
        fac = torch.empty(M.mgfld_factor_bytes(dims, precision), dtype=torch.uint8, device='cuda')
        x = torch.empty_like(dev['rhs'])
        assert M.mgfld_factor(dims, dev, precision, fac) == M.MGFLD_OK
        assert M.mgfld_solve(dims, dev, precision, fac, dev['rhs'], x) == M.MGFLD_OK
        torch.cuda.synchronize()
        x = x.cpu().numpy()
        for r in range(n_ray):
            for q in range(4):
                J = O.dense_matrix(diag[r, q], lower[r, q], upper[r, q])
                xd = np.linalg.solve(J, rhs[r, q].reshape(-1))
                err = np.max(np.abs(x[r, q].reshape(-1) - xd)) / np.max(np.abs(xd))
                # backward-stable elimination: forward error <= O(n) unit roundoff x condition
                assert err < 50 * unit * np.linalg.cond(J), (n_e, r, q, err)


def test_nonconvergence_and_nan_are_reported_per_ray():
    inp = SP.strong(n_ray=3, n_r=8, n_e=4, kabs=1e16, nes=10.0)
    _, _, _, codes, rep = run_gpu(inp, max_iter=1)
    assert codes == [M.MGFLD_ENOCONV]
    assert np.all(rep['ray_status'] == M.MGFLD_ENOCONV) and np.all(rep['iters'] == 1)
    bad = dict(inp)
    psi0 = inp['psi0'].copy()
    psi0[1, 0, 3, 2] = np.nan
    bad['psi0'] = psi0
    _, _, _, codes, rep = run_gpu(bad)
    assert codes == [M.MGFLD_ENAN]
    assert rep['ray_status'][1] == M.MGFLD_ENAN
    assert rep['ray_status'][0] == M.MGFLD_OK and rep['ray_status'][2] == M.MGFLD_OK


def test_chunked_rays_give_identical_results():
    inp = problems.make_problem(2, n_ray=6, n_r=40, n_e=8)
    a = run_gpu(inp)[0]
    per_ray = M.mgfld_workspace_bytes(M.Dims(1, 40, 8, 4), 0)
    b = run_gpu(inp, max_ws_bytes=2 * per_ray + 100)[0]
    assert np.array_equal(a, b)


def test_reported_heating_equals_the_matter_energy_gain():
    """The library's gain-region heating (mgfld_step_report.heating) pinned like the oracle's
    (tests/test_heating_pin.py): with the heavy-lepton species off it equals the matter energy
    gain sum rho V (e_int(T^{n+1}, Ye^{n+1}) - e_int(T^n, Ye^n)) / m_B over 100-300 km computed from
    the GPU's own T and Ye; with the electron flavours off it is zero."""
    from tests import test_heating_pin as HP
    for precision in (0, 1):
        inp = HP._species_off(HP._problem(True), off=(2, 3))
        psi, ye, T, codes, rep = run_gpu(inp, precision=precision, tol=1e-11)
        assert codes == [M.MGFLD_OK]
        gain, size = HP._matter_energy_gain(inp, dict(T=T, ye=ye))
        tol = 1e-14 * size + 1e-12 * np.abs(gain)
        print(f'precision {precision}: heating {rep["heating"]}, matter energy gain {gain}')
        assert np.all(np.abs(gain) > 1e3 * tol)
        assert np.all(np.abs(rep['heating'] - gain) <= tol)
    inp = HP._species_off(HP._problem(True), off=(0, 1))
    _, _, _, codes, rep = run_gpu(inp, tol=1e-11)
    assert codes == [M.MGFLD_OK] and np.all(rep['heating'] == 0.0)
