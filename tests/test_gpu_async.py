"""mgfld_step is asynchronous on its stream: the whole step is one CUDA graph whose outer iteration is
a device-side loop, so the call returns before the GPU has run it and nothing waits on the host.
Its results are bit-identical to the host-driven loop (the profiling mode), which runs the same
kernels in the same order; the step's status arrives in the report."""
import ctypes
import time

import numpy as np
import pytest

from paper_1809_05608_gb300 import problems
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


def _state(st, inp):
    return st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])


def test_the_call_returns_before_the_step_has_run():
    inp = problems.make_problem(3, rays=range(64))
    st = M.Stepper(inp, M.MGFLD_MIXED, tol=1e-10, max_iter=60)
    psi, ye, T = _state(st, inp)
    assert st.step(psi, ye, T) == M.MGFLD_OK           # builds and caches this argument set's graph
    psi, ye, T = _state(st, inp)
    ref = M.Stepper(inp, M.MGFLD_MIXED, tol=1e-10, max_iter=60)
    a = _state(ref, inp)
    torch.cuda.synchronize()
    st.status.fill_(-1)
    torch.cuda._sleep(int(5e8))                        # the stream is busy for a while first
    t0 = time.perf_counter()
    rc = st.step(psi, ye, T, wait=False)
    host_ms = (time.perf_counter() - t0) * 1e3
    busy = torch.cuda.current_stream().query()
    torch.cuda.synchronize()
    print(f'host time of the call {host_ms:.3f} ms; stream idle right after the call: {busy}')
    assert rc == M.MGFLD_OK and not busy and host_ms < 20.0
    assert st.worst_status() == M.MGFLD_OK
    assert ref.step(*a) == M.MGFLD_OK
    torch.cuda.synchronize()
    for x, y in zip((psi, ye, T), a):
        assert torch.equal(x, y)


def _host_loop_step(st, psi, ye, T):
    prof = (ctypes.c_double * (2 * M.PROF_N))()
    st.opts.profile = ctypes.cast(prof, ctypes.c_void_p)
    rc = st.step(psi, ye, T)
    st.opts.profile = None
    return rc


@pytest.mark.parametrize('case', ['mixed_uneven', 'fp64_newton', 'pair', 'coef', 'shock'])
def test_graph_and_host_loop_agree_bitwise(case):
    """Rays that converge after different numbers of iterations (the lists shrink on the device),
    Newton with a factorisation every iteration, the pair systems, the n+1 coefficients, the shock
    terms: two steps each way, every output and report bit for bit."""
    kw = dict(tol=1e-11, max_iter=40)
    prec = M.MGFLD_MIXED
    if case == 'mixed_uneven':
        a = SP.strong(n_ray=3, n_r=16, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True)
        b = problems.make_problem(3, rays=[0, 1, 2], n_r=16, n_e=5)
        inp = dict(a)
        for k in ('psi0', 'ye0', 'T0'):
            inp[k] = np.concatenate([a[k], b[k]])
        p = dict(a['problem'])
        for k in ('r_edge', 'lapse', 'rho', 'kappa_abs', 'kappa_scat', 'nes_coef'):
            pb = b['problem'][k] if b['problem'][k] is not None else np.sqrt(1.0 - 0.0 * b['problem']['rho'])
            p[k] = np.concatenate([a['problem'][k], pb])
        inp['problem'] = p
    elif case == 'fp64_newton':
        inp = problems.make_problem(2, rays=[3, 40], n_r=64, n_e=12)
        prec = M.MGFLD_FP64
        kw = dict(tol=1e-12, max_iter=40, refactor_ratio=0.0)
    elif case == 'pair':
        inp = SP.strong(n_ray=2, n_r=12, n_e=5, kabs=3e16, kscat=1e15, nes=30.0, lapse=True, pair=30.0)
    elif case == 'coef':
        inp = problems.make_problem(3, rays=[5, 6], n_r=64, n_e=12)
        kw['coef_iterate'] = True
    else:
        inp = problems.make_shock_problem(3, rays=[5, 700])
    g = M.Stepper(inp, prec, **kw)
    h = M.Stepper(inp, prec, **kw)
    sg, sh = _state(g, inp), _state(h, inp)
    for _ in range(2):
        assert g.step(*sg) == M.MGFLD_OK
        assert _host_loop_step(h, *sh) == M.MGFLD_OK
        torch.cuda.synchronize()
        for x, y in zip(sg, sh):
            assert torch.equal(x, y)
        for k in ('iters', 'ray_status', 'ledger', 'heating', 'factorizations'):
            assert torch.equal(g.report[k], h.report[k]), k
    its = g.report['iters'].cpu().numpy()
    print(f'{case}: iterations {its.tolist()}')
    if case == 'mixed_uneven':
        assert its.min() < its.max()                   # the rays did leave the lists at different times


def test_status_in_the_report_without_waiting():
    """Non-convergence and non-finite values reach the caller through the report's status (and the
    per-ray statuses) once the stream has run the step."""
    inp = SP.strong(n_ray=3, n_r=8, n_e=4, kabs=1e16, nes=10.0)
    st = M.Stepper(inp, M.MGFLD_FP64, tol=1e-12, max_iter=1)
    psi, ye, T = _state(st, inp)
    assert st.step(psi, ye, T, wait=False) == M.MGFLD_OK
    torch.cuda.synchronize()
    assert int(st.status[0]) == M.MGFLD_ENOCONV
    assert np.all(st.report['ray_status'].cpu().numpy() == M.MGFLD_ENOCONV)
    bad = dict(inp)
    psi0 = inp['psi0'].copy()
    psi0[1, 0, 3, 2] = np.nan
    bad['psi0'] = psi0
    st = M.Stepper(bad, M.MGFLD_FP64, tol=1e-12, max_iter=40)
    psi, ye, T = _state(st, bad)
    assert st.step(psi, ye, T, wait=False) == M.MGFLD_OK
    torch.cuda.synchronize()
    assert int(st.status[0]) == M.MGFLD_ENAN
    rs = st.report['ray_status'].cpu().numpy()
    assert rs[1] == M.MGFLD_ENAN and rs[0] == M.MGFLD_OK and rs[2] == M.MGFLD_OK


def test_consecutive_steps_without_synchronisation():
    """Ten steps queued back to back on the stream give what ten synchronised steps give."""
    inp = problems.make_problem(3, rays=range(8))
    a = M.Stepper(inp, M.MGFLD_MIXED, tol=1e-10, max_iter=60)
    b = M.Stepper(inp, M.MGFLD_MIXED, tol=1e-10, max_iter=60)
    sa, sb = _state(a, inp), _state(b, inp)
    for _ in range(10):
        assert a.step(*sa, wait=False) == M.MGFLD_OK
    for _ in range(10):
        assert b.step(*sb) == M.MGFLD_OK
    torch.cuda.synchronize()
    assert a.worst_status() == M.MGFLD_OK
    for x, y in zip(sa, sb):
        assert torch.equal(x, y)
