"""GPU discrete adjoint (mgfld_adjoint through the C ABI) vs the CPU oracle's adjoint.

Single step: both sides get the same start state and the same root (the oracle's), so
the comparison isolates the adjoint arithmetic.  Measure: per output array, max |gpu -
oracle| / max |oracle|.  Tolerance 1e-9: the transposed solve amplifies FP64 rounding by
the block condition number (~1e3-1e5 on these stiff problems), and the oracle's
automatic differentiation sums the same terms in another order.

Multi-step: the GPU objective and gradients (checkpointed recomputation) against the
oracle's objective_and_gradients, and the GPU gradient against central differences of
the GPU forward map."""
import numpy as np
import pytest

from oracle import mgfld_adjoint_oracle as A
from oracle import mgfld_oracle as O
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


def _scale(n_e):
    return np.ones((4, n_e)) * (1.0 + 0.1 * np.arange(4 * n_e).reshape(4, n_e) / (4 * n_e))


def _rel(g, o):
    return float(np.max(np.abs(g - o)) / max(np.max(np.abs(o)), 1e-300))


CASES = {
    'strong_lapse': lambda: SP.strong(n_ray=1, n_r=12, n_e=4, kabs=1e16, kscat=1e15, nes=10.0, lapse=True),
    'reflect': lambda: SP.strong(n_ray=1, n_r=10, n_e=6, kabs=1e16, kscat=1e15, nes=10.0, bc=1),
    'odd_groups': lambda: SP.strong(n_ray=2, n_r=9, n_e=7, kabs=1e15, kscat=1e14, nes=3.0),
    'tiles_weak': lambda: SP.strong(n_ray=3, n_r=40, n_e=8, kabs=1.0, kscat=1.0, nes=1.0, dt=1e-5),
}


@pytest.mark.parametrize('case', sorted(CASES))
def test_step_vjp_matches_oracle(case):
    inp = CASES[case]()
    prob = inp['problem']
    n_ray, _, n_r, n_e = inp['psi0'].shape
    scale = _scale(n_e)
    p = dict(prob, scale=scale)
    o = O.step(p, inp['psi0'], inp['ye0'], inp['T0'], rtol=1e-15)
    rng = np.random.default_rng(11)
    psi_bar = rng.standard_normal(inp['psi0'].shape) * 1e3
    ye_bar = rng.standard_normal(inp['ye0'].shape) * 1e2
    T_bar = rng.standard_normal(inp['T0'].shape)
    hw = 0.7
    ref = A.step_vjp(prob, inp['psi0'], inp['ye0'], inp['T0'], scale, o['psi'], o['ye'], psi_bar, ye_bar, T_bar,
                     heat_weight=hw)
    dp = M.DeviceProblem(p)
    dims = M.Dims(n_ray, n_r, n_e, 4)
    ws = torch.empty(M.mgfld_adjoint_workspace_bytes(dims), dtype=torch.uint8, device='cuda')
    s0 = (_dev(inp['psi0']), _dev(inp['ye0']), _dev(inp['T0']))
    s1 = (_dev(o['psi']), _dev(o['ye']))
    out = (torch.empty_like(s0[0]), torch.empty_like(s0[1]), torch.empty_like(s0[2]))
    s_bar = torch.zeros(4, n_e, dtype=torch.float64, device='cuda')
    rc, sweeps, change = M.mgfld_adjoint(dims, dp.struct, s0, s1, (_dev(psi_bar), _dev(ye_bar), _dev(T_bar)), out,
                                         ws, hw, s_bar)
    torch.cuda.synchronize()
    assert rc == M.MGFLD_OK, (M.status_str(rc), sweeps, change)
    got = [t.cpu().numpy() for t in out] + [s_bar.cpu().numpy()]
    # dL/dpsi^n is compared as psi^n dL/dpsi^n (the effect of a relative perturbation).  The
    # limiter is invariant under psi -> c psi, so d alpha/d psi_i ~ alpha / psi_i is
    # astronomically large (up to ~1e250 here) where psi^n_i is tiny, and both sides carry
    # errors of that size relative to alpha: the oracle's automatic differentiation forms it
    # as the difference of two terms ~ alpha / psi_i (through psi_e and |d psi|) that cancel
    # where psi_{i+1} << psi_i, and the adjoint values mu it multiplies are determined by any
    # FP64 transposed solve only to ~eps max|mu| (they can sit 40 orders of magnitude below
    # max|mu|).  Weighted by psi_i, both errors are ~eps relative to the weighted gradient.
    psi0 = inp['psi0']
    assert np.all(np.isfinite(got[0]))
    errs = [_rel(got[0] * psi0, ref[0] * psi0)]
    errs += [_rel(g, r) for g, r in zip(got[1:], ref[1:])]
    print(f'{case}: sweeps {sweeps} (change {change:.1e}); rel err psi-weighted {errs[0]:.2e} ye {errs[1]:.2e} '
          f'T {errs[2]:.2e} scale {errs[3]:.2e}; unweighted psi {_rel(got[0], ref[0]):.2e} (max |dL/dpsi| '
          f'{np.max(np.abs(ref[0])):.1e}, not asserted)')
    for name, e in zip(('psi-weighted', 'ye', 'T', 'scale'), errs):
        assert e < 1e-9, (name, e)


def test_adjoint_zero_bars_give_zero():
    """No upstream gradient and no heating weight: every output is exactly zero."""
    inp = CASES['odd_groups']()
    n_ray, _, n_r, n_e = inp['psi0'].shape
    dp = M.DeviceProblem(inp['problem'])
    dims = M.Dims(n_ray, n_r, n_e, 4)
    ws = torch.empty(M.mgfld_adjoint_workspace_bytes(dims), dtype=torch.uint8, device='cuda')
    s0 = (_dev(inp['psi0']), _dev(inp['ye0']), _dev(inp['T0']))
    o = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    out = tuple(torch.full_like(t, 7.0) for t in s0)
    s_bar = torch.zeros(4, n_e, dtype=torch.float64, device='cuda')
    rc, _, _ = M.mgfld_adjoint(dims, dp.struct, s0, (_dev(o['psi']), _dev(o['ye'])), (None, None, None), out, ws,
                               0.0, s_bar)
    torch.cuda.synchronize()
    assert rc == M.MGFLD_OK
    for t in out + (s_bar,):
        assert float(t.abs().max()) == 0.0


def test_adjoint_rejects_bad_arguments():
    inp = CASES['odd_groups']()
    n_ray, _, n_r, n_e = inp['psi0'].shape
    dp = M.DeviceProblem(inp['problem'])
    dims = M.Dims(n_ray, n_r, n_e, 4)
    need = M.mgfld_adjoint_workspace_bytes(dims)
    ws = torch.empty(need, dtype=torch.uint8, device='cuda')
    s0 = (_dev(inp['psi0']), _dev(inp['ye0']), _dev(inp['T0']))
    out = tuple(torch.empty_like(t) for t in s0)
    small = ws[:need - 256]
    rc, _, _ = M.mgfld_adjoint(dims, dp.struct, s0, s0[:2], (None, None, None), out, small)
    assert rc == M.MGFLD_ENOMEM
    rc, _, _ = M.mgfld_adjoint(dims, dp.struct, s0, s0[:2], (None, None, None), (out[0], None, out[2]), ws)
    assert rc == M.MGFLD_EINVAL
    assert M.mgfld_adjoint_workspace_bytes(M.Dims(1, 4, 33, 4)) == 0


def _runner(inp, every):
    return ADJ.AdjointRunner(inp, checkpoint_every=every, tol=1e-12)


def test_multistep_gradients_match_oracle_and_checkpointing_is_exact():
    inp = CASES['strong_lapse']()
    n_e = inp['psi0'].shape[3]
    scale = _scale(n_e)
    n_steps = 5
    J_o, gpsi_o, gs_o = A.objective_and_gradients(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], scale,
                                                  n_steps)
    res = {}
    for every in (1, 2, 5):
        r = _runner(inp, every)
        sc = _dev(scale)
        J, ck = r.forward(sc, _dev(inp['psi0']), _dev(inp['ye0']), _dev(inp['T0']), n_steps)
        g = r.reverse(sc, ck, n_steps)
        torch.cuda.synchronize()
        res[every] = (float(J), [t.cpu().numpy() for t in g])
        assert len(ck) == (n_steps + every - 1) // every
    J1, g1 = res[1]
    for every in (2, 5):
        Je, ge = res[every]
        assert Je == J1
        for a, b in zip(ge, g1):
            assert np.array_equal(a, b)            # recomputation reproduces the stored states bit for bit
    eJ = abs(J1 / J_o.sum() - 1)
    ep, es = _rel(g1[0] * inp['psi0'], gpsi_o * inp['psi0']), _rel(g1[3], gs_o)   # psi-weighted, as above
    print(f'5 steps: J rel {eJ:.2e}, dJ/dpsi0 {ep:.2e}, dJ/dscale {es:.2e}')
    assert eJ < 1e-11
    assert ep < 1e-8
    assert es < 1e-8


def test_autograd_function_and_central_differences():
    """Gradients through the autograd function against central differences of the GPU forward
    map, 1e-6 relative per entry.  Checked: every opacity scale with s |dJ/ds| >= 1e-3 |J| and five
    psi^0 entries with psi |dJ/dpsi| >= 1e-2 |J|, at h = 1e-3 of the entry.  At that h the
    truncation error is ~1e-10 (measured with the oracle) and the forward map's convergence noise
    (~1e-13 |J|) contributes 1e-13 |J| / (h |g|) <= 1e-7 of |g|; entries carrying less of J are
    below what central differences of a forward map at that accuracy resolve to 1e-6, and are
    checked against the oracle adjoint instead (test_multistep_gradients_match_oracle...)."""
    inp = CASES['odd_groups']()
    n_e = inp['psi0'].shape[3]
    n_steps = 3
    r = _runner(inp, 2)
    scale = _dev(_scale(n_e)).requires_grad_()
    psi0 = _dev(inp['psi0']).requires_grad_()
    ye0, T0 = _dev(inp['ye0']), _dev(inp['T0'])
    J = ADJ.heating_objective(scale, psi0, ye0, T0, r, n_steps)
    gs, gp = torch.autograd.grad(2.0 * J, [scale, psi0])
    gs, gp = gs.cpu().numpy() / 2.0, gp.cpu().numpy() / 2.0
    J = float(J)

    def J_of(sc, ps):
        with torch.no_grad():
            v, _ = r.forward(_dev(sc), _dev(ps), ye0, T0, n_steps)
        return float(v)

    s_np = _scale(n_e)
    big = np.argwhere(s_np * np.abs(gs) >= 1e-3 * abs(J))
    assert len(big) >= 4
    worst = 0.0
    for q, k in big:
        h = 1e-3 * s_np[q, k]
        sp, sm = s_np.copy(), s_np.copy()
        sp[q, k] += h
        sm[q, k] -= h
        fd = (J_of(sp, inp['psi0']) - J_of(sm, inp['psi0'])) / (2 * h)
        worst = max(worst, abs(fd - gs[q, k]) / abs(gs[q, k]))
        assert abs(fd - gs[q, k]) <= 1e-6 * abs(gs[q, k]), (q, k, fd, gs[q, k])
    wp = np.abs(gp * inp['psi0'])
    cand = np.argwhere(wp >= 1e-2 * abs(J))
    rng = np.random.default_rng(3)
    worst_p = 0.0
    for idx in cand[rng.choice(len(cand), size=min(5, len(cand)), replace=False)]:
        idx = tuple(idx)
        h = 1e-3 * inp['psi0'][idx]
        pp, pm = inp['psi0'].copy(), inp['psi0'].copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (J_of(s_np, pp) - J_of(s_np, pm)) / (2 * h)
        worst_p = max(worst_p, abs(fd - gp[idx]) / abs(gp[idx]))
        assert abs(fd - gp[idx]) <= 1e-6 * abs(gp[idx]), (idx, fd, gp[idx])
    print(f'central differences: {len(big)} scale entries, worst {worst:.1e}; 5 psi0 entries, worst {worst_p:.1e} '
          f'(per entry, relative)')
