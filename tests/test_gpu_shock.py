"""Transport through a shock on the GPU (problem fields u, eta1 through the C ABI) against the
oracle, on the imposed accretion-shock velocity profile (problems.make_shock_problem).

The shock terms are constants of the step (formed at psi^n), so the Newton system, its
convergence and its rounding floor are those of the shock-free step: the gates are the same as
for the plain step (normwise max over zones and groups per ray and species)."""
import ctypes

import numpy as np
import pytest

from oracle import mgfld_oracle as O
from paper_1809_05608_gb300 import problems
from tests import parity_measures as PM
from tests import small_problems as SP

torch = pytest.importorskip('torch')

M = None


def _load():
    global M
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


def normwise(a, b):
    return float(np.max(O.rel_change(a - b, b)))


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    _load()


@pytest.mark.gpu
def test_single_ray_shock_fp64_matches_oracle():
    _gpu()
    inp = problems.make_shock_problem(1)
    psi, ye, T, codes, rep = run_gpu(inp)
    psi_o, ye_o, T_o, outs = O.run_steps(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], 1)
    plain = O.step(dict(inp['problem'], u=None), inp['psi0'], inp['ye0'], inp['T0'])['psi']
    assert codes == [M.MGFLD_OK]
    fwd = normwise(psi, psi_o)
    print(f'single ray with shock, fp64: forward {fwd:.2e}; shock moved psi by {normwise(plain, psi_o):.2e}')
    assert normwise(plain, psi_o) > 1e-3            # the shock terms matter in this case
    assert fwd < 1e-12
    assert np.max(np.abs(ye - ye_o)) < 1e-14
    assert np.max(np.abs(T / T_o - 1)) < 1e-12
    L, Lo = rep['ledger'], outs[0]['ledger']
    assert np.allclose(L[:, [0, 1, 4, 5]], Lo[:, [0, 1, 4, 5]], rtol=1e-12, atol=0)
    # the frame terms carry no neutrino number: lepton number still balances
    assert np.all(np.abs(L[:, 3]) <= 1e-13 * np.abs(L[:, 1]))


@pytest.mark.gpu
@pytest.mark.parametrize('precision', [0, 1])
def test_full_size_shock_rays(precision):
    """Three 512 x 20 rays of the 1024-ray benchmark workload with the shock, two steps, each
    against the oracle's step from the same state: FP64 at 1e-12, mixed at 1e-10."""
    _gpu()
    inp = problems.make_shock_problem(3, rays=[0, 511, 1023])
    gate = 1e-12 if precision == 0 else 1e-10
    (psi, ye, T), codes, rep, (psi_o, ye_o, T_o) = PM.stepwise(
        M, torch, inp, precision, 2, gate, f'3 shock rays, precision {precision}',
        tol=1e-12 if precision == 0 else 1e-10, max_iter=40)
    assert codes == [M.MGFLD_OK] * 2
    assert np.max(np.abs(ye - ye_o)) < (1e-14 if precision == 0 else 1e-12)


@pytest.mark.gpu
def test_full_launch_with_shock_sampled():
    """The 1024-ray launch with the shock in the mixed path (the benchmark's shock line):
    sampled rays vs the oracle, every ray converged, lepton number balanced."""
    _gpu()
    full = problems.make_shock_problem(3)
    psi, ye, T, codes, rep = run_gpu(full, precision=1, tol=1e-10)
    assert codes == [M.MGFLD_OK]
    rays = [7, 512, 1020]
    sub = problems.subset_rays(full, rays)
    psi_o, _, T_o, _ = O.run_steps(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'], 1)
    fwd = normwise(psi[rays], psi_o)
    print(f'1024-ray shock launch (mixed), sampled rays: forward {fwd:.2e}')
    assert fwd < 1e-10
    assert np.all(rep['ray_status'] == 0)
    L = rep['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-12 * np.abs(L[:, 1]))


@pytest.mark.gpu
def test_zero_velocity_reproduces_the_plain_step():
    _gpu()
    inp = problems.make_shock_problem(2, n_ray=2, n_r=40, n_e=7)
    still = dict(inp, problem=dict(inp['problem'], u=np.zeros_like(inp['problem']['u'])))
    plain = dict(inp, problem=dict(inp['problem'], u=None, eta1=None))
    a = run_gpu(still, steps=2)
    b = run_gpu(plain, steps=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_adjoint_rejects_shock_terms_before_touching_the_device():
    """mgfld_adjoint does not differentiate the shock terms: a problem carrying u is refused by
    the argument checks (host only; the fake pointers are never dereferenced)."""
    _load()
    fake = ctypes.c_void_p(0x10000)
    prob = M.Problem(*[fake] * 8, M.lib().mgfld_eos_default(), 1e-6, 0, fake, None)
    st = M.State(fake, fake, fake)
    io = M.AdjointIO(None, None, None, 1.0, fake, fake, fake, None, 0, 0.0, 0, 0.0)
    dims = M.Dims(1, 8, 4, 4)
    rc = M.lib().mgfld_adjoint(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st), ctypes.byref(st),
                               ctypes.byref(io), ctypes.c_void_p(0x100000), 1 << 30, None)
    assert rc == M.MGFLD_EINVAL
    prob.u = None
    # without u the same call passes the checks up to the workspace size
    rc = M.lib().mgfld_adjoint(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st), ctypes.byref(st),
                               ctypes.byref(io), ctypes.c_void_p(0x100000), 16, None)
    assert rc == M.MGFLD_ENOMEM


@pytest.mark.gpu
@pytest.mark.parametrize('case', ['jump at the last interior edge', 'reflecting edge, 7 groups', 'one zone'])
def test_shock_edge_cases(case):
    """Shock terms where the roll-in weight sits at the grid's ends, with a reflecting outer edge and
    ragged groups, and on one-zone rays (no interior edge: the terms vanish)."""
    _gpu()
    if case == 'jump at the last interior edge':
        inp = SP.strong(n_ray=2, n_r=12, n_e=5, kabs=1e15, kscat=1e15, nes=10.0, lapse=True)
        u = np.zeros_like(inp['problem']['rho'])
        u[:, -1] = -0.05 * O.C_LIGHT
        u[:, 0] = 0.015 * O.C_LIGHT                   # half rolled in at the innermost edge
    elif case == 'reflecting edge, 7 groups':
        inp = SP.strong(n_ray=2, n_r=10, n_e=7, kabs=1e15, kscat=1e15, nes=10.0, bc=M.MGFLD_BC_REFLECT)
        u = -0.03 * O.C_LIGHT * (np.arange(10)[None, :] >= 5) * np.ones((2, 1))
    else:
        inp = SP.strong(n_ray=2, n_r=1, n_e=4)
        u = np.full_like(inp['problem']['rho'], -0.1 * O.C_LIGHT)
    eta1 = np.broadcast_to(np.linspace(0.1, 0.9, inp['psi0'].shape[3]), inp['psi0'].shape).copy()
    inp = dict(inp, problem=dict(inp['problem'], u=u, eta1=eta1))
    psi, ye, T, codes, rep = run_gpu(inp, tol=1e-11)
    out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    assert codes == [M.MGFLD_OK]
    assert normwise(psi, out['psi']) < SP.fp64_tolerance(inp)
    L = rep['ledger']
    assert np.all(np.abs(L[:, 3]) <= 1e-12 * np.abs(L[:, 1]))
