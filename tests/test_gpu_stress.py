"""Neutrino stress and lapse update on the GPU (mgfld_stress_lapse through the C ABI) against the
oracle (Eqs. a62e-a62l), on the transport workloads with the matter pressure and inner mass of
problems.stress_inputs.

Error measures.  The edge stress is a difference of neighbouring zones' eps^3 d eps psi sums, so
its rounding is relative to the size of the terms, not of the difference: per edge the bound is
1e-13 x scale, scale = (4 pi/(hc)^3)/3 sum_q N_q sum_k F (|X_{i+1}| + |X_i|) A / Delta M.  The
lapse is a product of n_r exponentials (the GPU forms one exponential of a suffix sum): relative
1e-12."""

import numpy as np
import pytest

from oracle import mgfld_oracle as O
from oracle import stress_lapse_oracle as S
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device='cuda')


def run_gpu(prob, psi, ye, T, p, m_inner):
    n_ray, _, n_r, n_e = psi.shape
    dims = M.Dims(n_ray, n_r, n_e, 4)
    dp = M.DeviceProblem(prob)
    ws = torch.empty(M.mgfld_workspace_bytes(dims, M.MGFLD_FP64), dtype=torch.uint8, device='cuda')
    out = {k: torch.empty(n_ray, n_r, dtype=torch.float64, device='cuda') for k in ('f_edge', 'f_zone', 'lapse')}
    rc = M.mgfld_stress_lapse(dims, dp.struct, _dev(psi), _dev(ye), _dev(T), ws, p=_dev(p), m_inner=_dev(m_inner),
                              **out)
    torch.cuda.synchronize()
    assert rc == M.MGFLD_OK, M.status_str(rc)
    return {k: v.cpu().numpy() for k, v in out.items()}


def stress_scale(prob, psi, ye, T):
    f = O.setup_step(prob, psi, ye, T)
    X = (f.eps**3 * f.deps)[:, None] * np.abs(psi) * S.MEV_ERG
    X_r = np.empty_like(X)
    X_r[:, :, :-1] = X[:, :, 1:]
    X_r[:, :, -1] = f.ghost * X[:, :, -1]
    dM = f.rho * f.vol
    dM_e = np.append(0.5 * (dM[:, :-1] + dM[:, 1:]), dM[:, -1:], axis=1)
    s = np.einsum('q,rqik->ri', O.STAT_WEIGHT, np.abs(f.F) * (X_r + X))
    return O.FOUR_PI_HC3 / 3.0 * s * f.area[:, 1:] / dM_e


def check(prob, psi, ye, T, p, m_inner):
    ref = S.stress_and_lapse(prob, psi, ye, T, p, m_inner)
    got = run_gpu(prob, psi, ye, T, p, m_inner)
    scale = stress_scale(prob, psi, ye, T)
    e_err = np.max(np.abs(got['f_edge'] - ref['f_edge']) / np.maximum(scale, 1e-300))
    lap = np.max(np.abs(got['lapse'] / ref['lapse'] - 1.0))
    print(f'stress error / term scale {e_err:.2e}, lapse relative {lap:.2e}')
    assert e_err < 1e-13
    zscale = 0.5 * (scale + np.concatenate([np.zeros_like(scale[:, :1]), scale[:, :-1]], axis=1))
    assert np.max(np.abs(got['f_zone'] - ref['f_zone']) / np.maximum(zscale, 1e-300)) < 1e-13
    assert lap < 1e-12
    return got, ref


def test_single_ray_stress_and_lapse():
    inp = problems.make_problem(1)
    p, m = problems.stress_inputs(inp)
    check(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], p, m)


def test_full_size_rays_after_a_step_with_lapse():
    """Three 512 x 20 rays, the state after one oracle step with the lapse on, strong opacities."""
    inp = SP.strong(n_ray=3, n_r=512, n_e=20, kabs=1e3, kscat=1e3, nes=3.0, lapse=True)
    out = O.step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    p, m = problems.stress_inputs(dict(inp, ye0=out['ye'], T0=out['T']))
    got, ref = check(inp['problem'], out['psi'], out['ye'], out['T'], p, m)
    assert np.all(np.isfinite(got['lapse'])) and np.all(got['lapse'] > 0.0) and np.all(got['lapse'] < 1.0)


def test_full_launch_sampled():
    full = problems.make_problem(3)
    p, m = problems.stress_inputs(full)
    pr = full['problem']
    got = run_gpu(pr, full['psi0'], full['ye0'], full['T0'], p, m)
    rays = [0, 300, 1023]
    sub = problems.subset_rays(full, rays)
    ref = S.stress_and_lapse(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'], p[rays], m[rays])
    scale = stress_scale(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'])
    assert np.max(np.abs(got['f_edge'][rays] - ref['f_edge']) / np.maximum(scale, 1e-300)) < 1e-13
    assert np.max(np.abs(got['lapse'][rays] / ref['lapse'] - 1.0)) < 1e-12
    # the lapse rises outward wherever the pressure falls outward
    falls = np.diff(p, axis=1) < 0.0
    assert np.all(np.diff(got['lapse'], axis=1)[falls] > 0.0) and falls.mean() > 0.8


def test_reflecting_edge_and_bad_arguments():
    inp = SP.strong(n_ray=2, n_r=9, n_e=6, kabs=1e13, kscat=1e14, nes=5.0, bc=M.MGFLD_BC_REFLECT)
    p, m = problems.stress_inputs(inp)
    got, _ = check(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], p, m)
    assert np.all(got['f_edge'][:, -1] == 0.0)
    n_ray, _, n_r, n_e = inp['psi0'].shape
    dims = M.Dims(n_ray, n_r, n_e, 4)
    dp = M.DeviceProblem(inp['problem'])
    ws = torch.empty(M.mgfld_workspace_bytes(dims, M.MGFLD_FP64), dtype=torch.uint8, device='cuda')
    psi, ye, T = _dev(inp['psi0']), _dev(inp['ye0']), _dev(inp['T0'])
    lap = torch.empty(n_ray, n_r, dtype=torch.float64, device='cuda')
    assert M.mgfld_stress_lapse(dims, dp.struct, psi, ye, T, ws, lapse=lap) == M.MGFLD_EINVAL     # no p
    assert M.mgfld_stress_lapse(dims, dp.struct, psi, ye, T, ws[:1024], p=_dev(p), lapse=lap) == M.MGFLD_ENOMEM


def test_one_zone_rays():
    inp = SP.strong(n_ray=2, n_r=1, n_e=4)
    p, m = problems.stress_inputs(inp)
    got, _ = check(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'], p, m)
    assert np.all(got['lapse'] > 0.0)
