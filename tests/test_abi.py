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
    # FP64 keeps FP64 blocks and inverses (16 B per block entry); MIXED FP32 ones (8 B) plus the
    # NES kernels as FP32 pairs (16 B per kernel entry and zone: 4 B per block entry)
    assert b64 > 16 * blocks and b32 < b64 and b64 - b32 >= 2 * blocks
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


def test_pair_process_arguments(L):
    """The pair process: coupled (nu, antinu) blocks need the pair workspace, at most 24 groups, and
    the frozen flux coefficients; refused on the host before any launch otherwise."""
    d = M.Dims(2, 8, 5, 4)
    base = 0x7f0000000000
    for prec in (M.MGFLD_FP64, M.MGFLD_MIXED):
        plain, paired = M.mgfld_workspace_bytes(d, prec), M.mgfld_workspace_bytes_pair(d, prec)
        # twice the dense blocks and factors, plus the creation and four annihilation kernels per zone
        blk = (8 if prec == M.MGFLD_FP64 else 4) * 2 * 4 * 8 * 5 * 5
        assert paired >= plain + 2 * blk + 8 * 2 * 8 * 5 * 5 * 5
    assert M.mgfld_workspace_bytes_pair(M.Dims(1, 4, 25, 4), 0) == 0
    assert M.mgfld_workspace_bytes_pair(M.Dims(1, 4, 24, 4), 0) > 0
    p = _prob()
    p.pair_coef = ctypes.c_void_p(0x90000)
    need = M.mgfld_workspace_bytes_pair(d, 0)
    assert _call_step(L, d, p, M.step_opts(), base, need - 1) == M.MGFLD_ENOMEM
    assert _call_step(L, d, p, M.step_opts(coef_iterate=True), base, need) == M.MGFLD_EINVAL
    assert _call_step(L, M.Dims(2, 8, 25, 4), p, M.step_opts(), base, 1 << 40) == M.MGFLD_EINVAL


def test_status_strings(L):
    assert M.status_str(M.MGFLD_OK) == 'ok'
    assert 'converge' in M.status_str(M.MGFLD_ENOCONV)
    assert M.status_str(99) == 'unknown status'


def _fake(n):
    return ctypes.c_void_p(0x7e0000000000 + 0x100000 * n)


def test_other_entry_points_check_their_arguments_before_any_launch(L):
    """mgfld_assemble, mgfld_factor, mgfld_solve, mgfld_stress_lapse and mgfld_energy_advect refuse
    missing buffers, bad sizes, precisions and workspaces with a status code, on the host, before
    any CUDA call (the fake pointers are never dereferenced)."""
    d = M.Dims(2, 8, 5, 4)
    need = M.mgfld_workspace_bytes(d, M.MGFLD_FP64)
    ws = 0x7f0000000000
    st = M.State(_fake(1), _fake(2), _fake(3))
    sysm = M.System(_fake(4), _fake(5), _fake(6), _fake(7))
    R = ctypes.byref

    def assemble(dims=d, prob=None, system=sysm, w=ws, nbytes=need):
        return L.mgfld_assemble(R(dims), R(prob or _prob()), R(st), R(system), ctypes.c_void_p(w), nbytes, None)

    assert assemble(nbytes=need - 1) == M.MGFLD_ENOMEM
    assert assemble(w=ws + 16) == M.MGFLD_EINVAL
    assert assemble(dims=M.Dims(2, 8, 33, 4)) == M.MGFLD_EINVAL
    assert assemble(prob=_prob(null_rho=True)) == M.MGFLD_EINVAL
    assert assemble(system=M.System(_fake(4), None, _fake(6), _fake(7))) == M.MGFLD_EINVAL
    paired = _prob()
    paired.pair_coef = _fake(9)
    assert assemble(prob=paired) == M.MGFLD_EINVAL            # its system is per species: use mgfld_step

    for prec in (-1, 2):
        assert L.mgfld_factor(R(d), R(sysm), prec, _fake(8), None) == M.MGFLD_EINVAL
        assert L.mgfld_solve(R(d), R(sysm), prec, _fake(8), _fake(9), _fake(10), None) == M.MGFLD_EINVAL
    assert L.mgfld_factor(R(d), R(sysm), M.MGFLD_FP64, None, None) == M.MGFLD_EINVAL
    assert L.mgfld_factor(R(M.Dims(2, 8, 5, 3)), R(sysm), M.MGFLD_FP64, _fake(8), None) == M.MGFLD_EINVAL
    assert L.mgfld_solve(R(d), R(sysm), M.MGFLD_MIXED, _fake(8), None, _fake(10), None) == M.MGFLD_EINVAL
    assert L.mgfld_solve(R(d), R(sysm), M.MGFLD_MIXED, _fake(8), _fake(9), None, None) == M.MGFLD_EINVAL

    def stress(io, w=ws, nbytes=need, state=st):
        return L.mgfld_stress_lapse(R(d), R(_prob()), R(state), R(io), ctypes.c_void_p(w), nbytes, None)

    io = M.StressIO(_fake(11), None, _fake(12), None, _fake(13))
    assert stress(io, nbytes=need - 1) == M.MGFLD_ENOMEM
    assert stress(io, w=ws + 8) == M.MGFLD_EINVAL
    assert stress(M.StressIO(None, None, _fake(12), None, _fake(13))) == M.MGFLD_EINVAL   # lapse needs p
    assert stress(io, state=M.State(_fake(1), None, _fake(3))) == M.MGFLD_EINVAL

    def eadv(prob, dims=d, psi=_fake(14)):
        return L.mgfld_energy_advect(R(dims), R(prob), psi, None, None)

    full = [_fake(20 + i) for i in range(8)]
    ok = M.EadvProblem(*full, 1, None)
    assert eadv(ok, dims=M.Dims(2, 8, 2, 4)) == M.MGFLD_EINVAL        # the PPM stencil needs 3 groups
    assert eadv(ok, dims=M.Dims(2, 8, 5, 2)) == M.MGFLD_EINVAL
    assert eadv(ok, psi=None) == M.MGFLD_EINVAL
    for field in ('r_edge_n', 'r_edge_np1', 'rho_n', 'rho_np1', 'e_edge'):
        bad = M.EadvProblem(*full, 1, None)
        setattr(bad, field, None)
        assert eadv(bad) == M.MGFLD_EINVAL, field
