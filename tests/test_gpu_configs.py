"""The largest workloads at their full sizes, in the launch configuration a user runs them:

* the 2D mixed-precision step, 1024 rays x 512 zones x 20 groups x 4 species, one launch of all
  rays as the benchmark times it (mixed, tol 1e-10): sampled rays match the oracle to 1e-10, and
  the same launch in FP64 at the parity tolerance matches to 1e-12 (no widening);
* the 3D-scale mixed-precision step, 4096 rays (64 theta x 64 phi) x 540 zones x 20 groups x 4
  species, one launch of all rays: every ray converges to 1e-10 (each with its own iteration
  count; on this workload they all take 5), sampled rays match the oracle, lepton number balances
  in every ray;
* the adjoint workload, 512 rays x 512 x 20, 20 FP64 steps with a checkpoint every 5: the
  gradient of the gain-region heating with respect to the six opacity scales and the three psi^0
  entries that carry the most of it matches central differences of the GPU forward map itself
  to 1e-6 relative per entry (the oracle cannot run 512 rays x 20 steps in a test).  The
  opacities are raised 1e13-fold: at the synthetic values (~20 orders below physical ones) the
  heating depends on the scales below FP64 resolution, so central differences read zero there."""
import numpy as np
import pytest

from oracle import mgfld_oracle as O
from paper_1809_05608_gb300 import problems
from tests import parity_measures as PM
from tests import small_problems as SP

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

M = None
ADJ = None


@pytest.fixture(scope='module', autouse=True)
def _lib():
    global M, ADJ
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1809_05608_gb300 import adjoint, mgfld
    M, ADJ = mgfld, adjoint
    M.lib()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device='cuda')


@pytest.mark.parametrize('precision,tol,gate', [(1, 1e-10, 1e-10), (0, 1e-12, 1e-12)], ids=['mixed', 'fp64'])
def test_2d_full_launch_1024_rays_sampled_against_oracle(precision, tol, gate):
    full = problems.make_problem(3)
    n_ray, _, n_r, n_e = full['psi0'].shape
    assert (n_ray, n_r, n_e) == (1024, 512, 20)
    st = M.Stepper(full, precision, tol=tol, max_iter=60)
    psi, ye, T = st.state_to_device(full['psi0'], full['ye0'], full['T0'])
    rc = st.step(psi, ye, T)
    torch.cuda.synchronize()
    rep = {k: v.cpu().numpy() for k, v in st.report.items()}
    assert rc == M.MGFLD_OK and np.all(rep['ray_status'] == 0)
    L = rep['ledger']
    lep = float(np.max(np.abs(L[:, 3]) / np.abs(L[:, 1])))
    assert lep <= 1e-12
    rays = [0, 511, 1023]
    sub = problems.subset_rays(full, rays)
    out = O.step(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'])
    got = psi[rays].cpu().numpy()
    PM.report(f'1024 x 512 x 20 launch, precision {precision}, sampled rays', got, out['psi'], gate)
    print(f'  iterations {np.bincount(rep["iters"]).tolist()}, lepton residual max {lep:.1e}')
    assert np.max(np.abs(T[rays].cpu().numpy() / out['T'] - 1.0)) < gate
    assert np.max(np.abs(ye[rays].cpu().numpy() - out['ye'])) < (1e-14 if precision == 0 else 1e-12)


def test_3d_scale_mixed_full_launch():
    full = problems.make_problem(4)
    n_ray, _, n_r, n_e = full['psi0'].shape
    assert (n_ray, n_r, n_e) == (4096, 540, 20)
    st = M.Stepper(full, M.MGFLD_MIXED, tol=1e-10, max_iter=60)
    psi, ye, T = st.state_to_device(full['psi0'], full['ye0'], full['T0'])
    rc = st.step(psi, ye, T)
    torch.cuda.synchronize()
    rep = {k: v.cpu().numpy() for k, v in st.report.items()}
    assert rc == M.MGFLD_OK and np.all(rep['ray_status'] == 0)
    assert np.all(rep['iters'] >= 2)                  # each ray's own count (converged rays leave the lists)
    L = rep['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-12 * np.abs(L[:, 1]))
    rays = [0, 2079, 4095]
    sub = problems.subset_rays(full, rays)
    out = O.step(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'])
    got = psi[rays].cpu().numpy()
    PM.report('4096 x 540 x 20 mixed, sampled rays', got, out['psi'], 1e-10)
    print(f'  iterations {np.bincount(rep["iters"]).tolist()}, chunks of {st.chunk} rays')
    assert np.max(np.abs(T[rays].cpu().numpy() / out['T'] - 1.0)) < 1e-10


def test_adjoint_workload_full_size_against_central_differences():
    inp = SP.strong(n_ray=512, n_r=512, n_e=20, config=5, kabs=1e13, kscat=1e13, nes=1.0)
    n_ray, _, n_r, n_e = inp['psi0'].shape
    assert (n_ray, n_r, n_e) == (512, 512, 20)
    n_steps = 20
    runner = ADJ.AdjointRunner(inp, checkpoint_every=5)
    s_np = np.ones((4, n_e)) * (1.0 + 0.1 * np.arange(4 * n_e).reshape(4, n_e) / (4 * n_e))
    scale = _dev(s_np).requires_grad_()
    psi0, ye0, T0 = _dev(inp['psi0']).requires_grad_(), _dev(inp['ye0']), _dev(inp['T0'])
    J = ADJ.heating_objective(scale, psi0, ye0, T0, runner, n_steps)
    gs, gp = torch.autograd.grad(J, [scale, psi0])
    gs, gp = gs.cpu().numpy(), gp.cpu().numpy()
    psi_np = inp['psi0']

    def J_of(sc, ps=None):
        with torch.no_grad():
            v, _ = runner.forward(_dev(sc), psi0.detach() if ps is None else _dev(ps), ye0, T0, n_steps)
        return float(v)

    J = float(J)
    assert J > 0.0 and np.max(np.abs(gs)) > 1e-6 * J       # the scales matter at these opacities
    # the scale entries carrying the most of J, and the three psi^0 entries carrying the most of
    # it, each 1e-6 relative at h = 1e-3 of the entry (truncation ~1e-10; forward noise
    # ~1e-13 |J| / (h |g|) <= 1e-7 of |g| for the scales)
    order = np.argsort(-(s_np * np.abs(gs)).ravel())[:6]
    for q, k in zip(*np.unravel_index(order, gs.shape)):
        assert s_np[q, k] * abs(gs[q, k]) >= 1e-3 * J
        h = 1e-3 * s_np[q, k]
        sp, sm = s_np.copy(), s_np.copy()
        sp[q, k] += h
        sm[q, k] -= h
        fd = (J_of(sp) - J_of(sm)) / (2 * h)
        print(f'dJ/dscale[{q},{k}]: adjoint {gs[q, k]:.9e}, central differences {fd:.9e}')
        assert abs(fd - gs[q, k]) <= 1e-6 * abs(gs[q, k])
    # psi^0 carries less of J here (at most ~3e-4 of it per entry): the forward noise term is
    # then ~1e-13 |J| / (h |g|) ~ 3e-7 of |g|, still inside 1e-6
    wp = np.abs(gp * psi_np)
    for flat in np.argsort(-wp.ravel())[:3]:
        idx = np.unravel_index(flat, wp.shape)
        assert wp[idx] >= 1e-4 * J
        h = 1e-3 * psi_np[idx]
        pp, pm = psi_np.copy(), psi_np.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (J_of(s_np, pp) - J_of(s_np, pm)) / (2 * h)
        print(f'dJ/dpsi0{tuple(int(i) for i in idx)}: adjoint {gp[idx]:.9e}, central differences {fd:.9e}')
        assert abs(fd - gp[idx]) <= 1e-6 * abs(gp[idx])
