"""Host-side checks of the C ABI (no GPU needed: nothing here reaches a CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_1809_05608_gb300 import mgfld as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def L():
    if not os.path.exists(M.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return M.lib()


def _declared():
    names = set()
    inc = os.path.join(ROOT, 'include')
    for f in os.listdir(inc):
        if f.endswith('.h'):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
            names |= set(re.findall(r'\b(mgfld_\w+)\s*\(', src))
    return names


def test_every_declared_symbol_is_exported(L):
    declared = _declared()
    assert {'mgfld_step', 'mgfld_assemble', 'mgfld_factor', 'mgfld_solve'} <= declared
    for name in declared:
        assert hasattr(L, name), name


def test_workspace_query(L):
    d = M.Dims(256, 512, 20, 4)
    b64 = M.mgfld_workspace_bytes(d, M.MGFLD_FP64)
    b32 = M.mgfld_workspace_bytes(d, M.MGFLD_MIXED)
    blocks = 256 * 4 * 512 * 20 * 20
    assert b64 > 16 * blocks and b32 < b64 and b64 - b32 >= 4 * blocks
    assert M.mgfld_workspace_bytes(M.Dims(1, 1, 33, 4), 0) == 0
    assert M.mgfld_workspace_bytes(M.Dims(1, 4, 4, 3), 0) == 0
    assert M.mgfld_factor_bytes(M.Dims(2, 3, 5, 4), M.MGFLD_MIXED) == 2 * 4 * 3 * 25 * 4


class _Fake:
    """A stand-in tensor: a pointer value that validation never dereferences."""
    def __init__(self, ptr, nbytes=8):
        self.ptr, self.nbytes = ptr, nbytes

    def data_ptr(self):
        return self.ptr

    def numel(self):
        return self.nbytes

    def element_size(self):
        return 1


def _call_step(L, dims, prob, opts, ws, ws_bytes):
    st = M.State(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000))
    return L.mgfld_step(ctypes.byref(dims), ctypes.byref(prob), ctypes.byref(st), ctypes.byref(opts), None,
                        ctypes.c_void_p(ws), ws_bytes, None)


def _prob(dt=1e-6, bc=0, null_rho=False):
    p = [ctypes.c_void_p(0x10000 * (i + 1)) for i in range(8)]
    if null_rho:
        p[3] = None
    return M.Problem(*p, M.lib().mgfld_eos_default(), dt, bc)


def test_argument_errors_are_reported_before_any_launch(L):
    d = M.Dims(2, 8, 5, 4)
    need = M.mgfld_workspace_bytes(d, 0)
    ok_opts = M.step_opts()
    base = 0x7f0000000000
    assert _call_step(L, d, _prob(), ok_opts, base, need - 1) == M.MGFLD_ENOMEM
    assert _call_step(L, d, _prob(), ok_opts, base + 8, need) == M.MGFLD_EINVAL       # misaligned
    assert _call_step(L, d, _prob(), ok_opts, 0, need) == M.MGFLD_EINVAL              # NULL workspace
    assert _call_step(L, M.Dims(2, 8, 33, 4), _prob(), ok_opts, base, 1 << 40) == M.MGFLD_EINVAL
    assert _call_step(L, M.Dims(2, 8, 5, 3), _prob(), ok_opts, base, 1 << 40) == M.MGFLD_EINVAL
    assert _call_step(L, M.Dims(0, 8, 5, 4), _prob(), ok_opts, base, 1 << 40) == M.MGFLD_EINVAL
    assert _call_step(L, d, _prob(dt=0.0), ok_opts, base, need) == M.MGFLD_EINVAL
    assert _call_step(L, d, _prob(bc=7), ok_opts, base, need) == M.MGFLD_EINVAL
    assert _call_step(L, d, _prob(null_rho=True), ok_opts, base, need) == M.MGFLD_EINVAL
    assert _call_step(L, d, _prob(), M.step_opts(max_iter=0), base, need) == M.MGFLD_EINVAL
    assert _call_step(L, d, _prob(), M.step_opts(precision=5), base, need) == M.MGFLD_EINVAL
    assert _call_step(L, d, _prob(), M.step_opts(tol=0.0), base, need) == M.MGFLD_EINVAL


def test_status_strings(L):
    assert M.status_str(M.MGFLD_OK) == 'ok'
    assert 'converge' in M.status_str(M.MGFLD_ENOCONV)
    assert M.status_str(99) == 'unknown status'
