"""mgfld_step_noalloc: the step for callers that cannot allocate device memory.

Such callers (a host code using this solver as a black box without a GPU allocator
of its own, a process whose device memory is reserved by another framework's pool,
or a loop that cannot pay cudaMalloc's synchronisation) get the same step with the
scratch held in a fixed array inside the library.  This file is collected last so
that a stop-at-first-failure run has executed every other test before it."""
import ctypes

import numpy as np
import pytest

from oracle import mgfld_oracle as O
from paper_1809_05608_gb300 import mgfld as M
from paper_1809_05608_gb300 import problems

torch = pytest.importorskip('torch')


def test_noalloc_rejects_oversize_and_profiling_before_touching_the_gpu():
    big = M.Dims(64, 512, 20, 4)
    assert M.mgfld_workspace_bytes(big, 0) > M.NOALLOC_SCRATCH_BYTES
    prob = M.Problem(*[ctypes.c_void_p(0x10000)] * 8, M.lib().mgfld_eos_default(), 1e-6, 0)
    st = M.State(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000))
    L = M.lib()
    assert L.mgfld_step_noalloc(ctypes.byref(big), ctypes.byref(prob), ctypes.byref(st),
                                ctypes.byref(M.step_opts()), None, None) == M.MGFLD_ENOMEM
    prof = (ctypes.c_double * (2 * M.PROF_N))()
    small = M.Dims(1, 8, 4, 4)
    assert L.mgfld_step_noalloc(ctypes.byref(small), ctypes.byref(prob), ctypes.byref(st),
                                ctypes.byref(M.step_opts(profile=prof)), None, None) == M.MGFLD_EINVAL


@pytest.mark.gpu
def test_noalloc_step_matches_workspace_step_on_two_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    inp = problems.make_problem(2, rays=[5, 250])               # 2 full-size rays: 512 zones x 20 groups
    n_ray, _, n_r, n_e = inp['psi0'].shape
    dims = M.Dims(n_ray, n_r, n_e, 4)
    assert M.mgfld_workspace_bytes(dims, M.MGFLD_FP64) <= M.NOALLOC_SCRATCH_BYTES
    ref = M.Stepper(inp, M.MGFLD_FP64, tol=1e-12, max_iter=40)
    a = ref.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    b = ref.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    opts = M.step_opts(M.MGFLD_FP64, tol=1e-12, max_iter=40)
    for _ in range(2):
        assert ref.step(*a) == M.MGFLD_OK
        assert M.mgfld_step_noalloc(dims, ref.prob.struct, *b, opts) == M.MGFLD_OK
        torch.cuda.synchronize()
        pa, pb = a[0].cpu().numpy(), b[0].cpu().numpy()
        assert np.max(O.rel_change(pb - pa, pa)) < 1e-12
        assert np.max(np.abs(b[1].cpu().numpy() - a[1].cpu().numpy())) < 1e-14
        assert np.max(np.abs(b[2].cpu().numpy() / a[2].cpu().numpy() - 1)) < 1e-12
