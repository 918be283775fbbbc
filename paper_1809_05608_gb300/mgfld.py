"""Thin Python binding of libmgfld (include/mgfld.h).

The functions named like the C entry points only marshal arguments (torch
tensors -> device pointers, the current CUDA stream) and call the library; every
step of the transport computation runs in the library's CUDA kernels.  There is
no CPU or PyTorch fallback: if the shared library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, '_build', 'libmgfld.so')

MGFLD_OK, MGFLD_EINVAL, MGFLD_ENOMEM, MGFLD_ENOCONV, MGFLD_ENAN, MGFLD_ECUDA = range(6)
MGFLD_FP64, MGFLD_MIXED = 0, 1
MGFLD_BC_GHOST, MGFLD_BC_REFLECT = 0, 1
N_SPECIES = 4

EXPORTED = ('mgfld_eos_default', 'mgfld_workspace_bytes', 'mgfld_workspace_bytes_pair', 'mgfld_step', 'mgfld_assemble',
            'mgfld_factor_bytes', 'mgfld_factor', 'mgfld_solve', 'mgfld_status_str', 'mgfld_step_noalloc',
            'mgfld_adjoint_workspace_bytes', 'mgfld_adjoint', 'mgfld_energy_advect', 'mgfld_stress_lapse',
            'mgfld_arith_check')
NOALLOC_SCRATCH_BYTES = 64 << 20


class Dims(ctypes.Structure):
    _fields_ = [('n_ray', ctypes.c_int), ('n_r', ctypes.c_int), ('n_e', ctypes.c_int), ('n_s', ctypes.c_int)]


class EosParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ('gamma1', 'gamma2', 'e_coef', 'g_n', 'g_p', 'rho_nuc', 'rho_0', 'mb_c2', 'm_b')]


class Problem(ctypes.Structure):
    _fields_ = [('r_edge', ctypes.c_void_p), ('lapse', ctypes.c_void_p), ('e_edge', ctypes.c_void_p),
                ('rho', ctypes.c_void_p), ('kappa_abs', ctypes.c_void_p), ('kappa_scat', ctypes.c_void_p),
                ('nes_coef', ctypes.c_void_p), ('scale', ctypes.c_void_p), ('eos', EosParams),
                ('dt', ctypes.c_double), ('outer_bc', ctypes.c_int), ('u', ctypes.c_void_p),
                ('eta1', ctypes.c_void_p), ('pair_coef', ctypes.c_void_p), ('pair_chi', ctypes.c_int)]


class State(ctypes.Structure):
    _fields_ = [('psi', ctypes.c_void_p), ('ye', ctypes.c_void_p), ('T', ctypes.c_void_p)]


class StepOpts(ctypes.Structure):
    _fields_ = [('precision', ctypes.c_int), ('tol', ctypes.c_double), ('tolmin_psi', ctypes.c_double),
                ('tol_ye', ctypes.c_double), ('tolmin_ye', ctypes.c_double), ('max_iter', ctypes.c_int),
                ('refactor_ratio', ctypes.c_double), ('profile', ctypes.c_void_p), ('coef_iterate', ctypes.c_int)]


class StepReport(ctypes.Structure):
    _fields_ = [('iters', ctypes.c_void_p), ('ray_status', ctypes.c_void_p), ('ledger', ctypes.c_void_p),
                ('heating', ctypes.c_void_p), ('factorizations', ctypes.c_void_p), ('status', ctypes.c_void_p)]


class System(ctypes.Structure):
    _fields_ = [('diag', ctypes.c_void_p), ('lower', ctypes.c_void_p), ('upper', ctypes.c_void_p),
                ('rhs', ctypes.c_void_p)]


class AdjointIO(ctypes.Structure):
    _fields_ = [('psi_bar', ctypes.c_void_p), ('ye_bar', ctypes.c_void_p), ('T_bar', ctypes.c_void_p),
                ('heat_weight', ctypes.c_double), ('psi_bar_out', ctypes.c_void_p),
                ('ye_bar_out', ctypes.c_void_p), ('T_bar_out', ctypes.c_void_p), ('scale_bar', ctypes.c_void_p),
                ('max_sweeps', ctypes.c_int), ('sweep_tol', ctypes.c_double), ('sweeps_used', ctypes.c_int),
                ('sweep_change', ctypes.c_double)]


class EadvProblem(ctypes.Structure):
    _fields_ = [('r_edge_n', ctypes.c_void_p), ('r_edge_np1', ctypes.c_void_p), ('rho_n', ctypes.c_void_p),
                ('rho_np1', ctypes.c_void_p), ('lapse_n', ctypes.c_void_p), ('lapse_np1', ctypes.c_void_p),
                ('e_edge', ctypes.c_void_p), ('eta1', ctypes.c_void_p), ('limit', ctypes.c_int),
                ('u', ctypes.c_void_p)]


class StressIO(ctypes.Structure):
    _fields_ = [('p', ctypes.c_void_p), ('m_inner', ctypes.c_void_p), ('f_edge', ctypes.c_void_p),
                ('f_zone', ctypes.c_void_p), ('lapse', ctypes.c_void_p)]


_lib = None


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f'libmgfld is not built ({LIB_PATH} missing); run '
                           '`python -c "import __graft_entry__ as g; g.build()"` first')
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.mgfld_eos_default.restype = EosParams
    L.mgfld_eos_default.argtypes = []
    L.mgfld_workspace_bytes.restype = ctypes.c_size_t
    L.mgfld_workspace_bytes.argtypes = [P(Dims), ctypes.c_int]
    L.mgfld_workspace_bytes_pair.restype = ctypes.c_size_t
    L.mgfld_workspace_bytes_pair.argtypes = [P(Dims), ctypes.c_int]
    L.mgfld_factor_bytes.restype = ctypes.c_size_t
    L.mgfld_factor_bytes.argtypes = [P(Dims), ctypes.c_int]
    L.mgfld_step.restype = ctypes.c_int
    L.mgfld_step.argtypes = [P(Dims), P(Problem), P(State), P(StepOpts), P(StepReport),
                             ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.mgfld_assemble.restype = ctypes.c_int
    L.mgfld_assemble.argtypes = [P(Dims), P(Problem), P(State), P(System), ctypes.c_void_p,
                                 ctypes.c_size_t, ctypes.c_void_p]
    L.mgfld_factor.restype = ctypes.c_int
    L.mgfld_factor.argtypes = [P(Dims), P(System), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.mgfld_solve.restype = ctypes.c_int
    L.mgfld_solve.argtypes = [P(Dims), P(System), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p]
    L.mgfld_step_noalloc.restype = ctypes.c_int
    L.mgfld_step_noalloc.argtypes = [P(Dims), P(Problem), P(State), P(StepOpts), P(StepReport), ctypes.c_void_p]
    L.mgfld_adjoint_workspace_bytes.restype = ctypes.c_size_t
    L.mgfld_adjoint_workspace_bytes.argtypes = [P(Dims)]
    L.mgfld_adjoint.restype = ctypes.c_int
    L.mgfld_adjoint.argtypes = [P(Dims), P(Problem), P(State), P(State), P(AdjointIO), ctypes.c_void_p,
                                ctypes.c_size_t, ctypes.c_void_p]
    L.mgfld_stress_lapse.restype = ctypes.c_int
    L.mgfld_stress_lapse.argtypes = [P(Dims), P(Problem), P(State), P(StressIO), ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p]
    L.mgfld_energy_advect.restype = ctypes.c_int
    L.mgfld_energy_advect.argtypes = [P(Dims), P(EadvProblem), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.mgfld_status_str.restype = ctypes.c_char_p
    L.mgfld_status_str.argtypes = [ctypes.c_int]
    L.mgfld_arith_check.restype = ctypes.c_int
    L.mgfld_arith_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    _lib = L
    return L


def status_str(code: int) -> str:
    return lib().mgfld_status_str(int(code)).decode()


def arith_check(a, b, stream=None):
    """mgfld_arith_check on two equal-length FP64 device tensors: returns a [count, 8] device tensor
    (library quotient, CUDA quotient, library reciprocal, CUDA reciprocal, reciprocal seed,
    integer-pipe x < y, CUDA x < y, integer-pipe x == 0)."""
    import torch
    a = a.contiguous()
    b = b.contiguous()
    out = torch.empty((a.numel(), 8), dtype=torch.float64, device=a.device)
    rc = lib().mgfld_arith_check(_ptr(a), _ptr(b), a.numel(), _ptr(out), _stream(stream))
    if rc != MGFLD_OK:
        raise MgfldError(rc, 'mgfld_arith_check')
    return out


class MgfldError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f'{where}: {status_str(code)} ({code})')
        self.code = code


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def dims_of(psi):
    n_ray, n_s, n_r, n_e = psi.shape
    return Dims(n_ray, n_r, n_e, n_s)


# ---------------------------------------------------------------------------- device data

class DeviceProblem:
    """Device-resident (torch, FP64, contiguous) copy of a problem description and
    the matching C struct.  `prob` is a dict with the fields of mgfld_problem."""

    FIELDS = ('r_edge', 'lapse', 'e_edge', 'rho', 'kappa_abs', 'kappa_scat', 'nes_coef', 'scale')
    OPTIONAL_FIELDS = ('u', 'eta1', 'pair_coef')

    def __init__(self, prob, device='cuda'):
        import torch
        self.t = {}
        for f in self.FIELDS + self.OPTIONAL_FIELDS:
            v = prob.get(f)
            self.t[f] = None if v is None else torch.as_tensor(
                np.array(v, dtype=np.float64, order='C'), device=device)
        self.dt = float(prob['dt'])
        self.outer_bc = int(prob.get('outer_bc', MGFLD_BC_GHOST))
        self.pair_chi = 1 if prob.get('pair_chi') else 0
        self.eos = lib().mgfld_eos_default()
        self.struct = Problem(*[_ptr(self.t[f]) for f in self.FIELDS], self.eos, self.dt, self.outer_bc,
                              *[_ptr(self.t[f]) for f in self.OPTIONAL_FIELDS], self.pair_chi)

    def rays(self, lo, hi, n_r, n_e):
        """C struct viewing rays [lo, hi) only (rays are independent; used for chunking)."""
        def off(name, per_ray):
            t = self.t[name]
            return None if t is None else ctypes.c_void_p(t.data_ptr() + 8 * lo * per_ray)
        return Problem(off('r_edge', n_r + 1), off('lapse', n_r), _ptr(self.t['e_edge']), off('rho', n_r),
                       off('kappa_abs', N_SPECIES * n_r * n_e), off('kappa_scat', N_SPECIES * n_r * n_e),
                       off('nes_coef', n_r), _ptr(self.t['scale']), self.eos, self.dt, self.outer_bc,
                       off('u', n_r), off('eta1', N_SPECIES * n_r * n_e), off('pair_coef', n_r), self.pair_chi)


PROF_NAMES = ('setup', 'assemble', 'factor', 'solve', 'update', 'finish', 'residual')
PROF_N = len(PROF_NAMES)


def step_opts(precision=MGFLD_FP64, tol=1e-10, tolmin_psi=1.0, tol_ye=None, tolmin_ye=0.1, max_iter=40,
              refactor_ratio=None, profile=None, coef_iterate=False):
    """`refactor_ratio`: None gives 0.1 for MIXED and Newton (0) for FP64; a positive value makes
    FP64 reuse its factors too.  `profile`: optional ctypes (c_double * (2 * PROF_N)) array accumulating
    per-category (milliseconds, launches) for the categories of PROF_NAMES.  `coef_iterate`: the
    flux coefficients of Eq. a59 at the outer iterate (n+1) instead of at psi^n."""
    if refactor_ratio is None:
        refactor_ratio = 0.1 if precision == MGFLD_MIXED else 0.0
    return StepOpts(int(precision), float(tol), float(tolmin_psi), float(tol if tol_ye is None else tol_ye),
                    float(tolmin_ye), int(max_iter), float(refactor_ratio),
                    None if profile is None else ctypes.cast(profile, ctypes.c_void_p), 1 if coef_iterate else 0)


# ---------------------------------------------------------------------------- entry points

def mgfld_workspace_bytes(dims: Dims, precision: int) -> int:
    return int(lib().mgfld_workspace_bytes(ctypes.byref(dims), int(precision)))


def mgfld_workspace_bytes_pair(dims: Dims, precision: int) -> int:
    return int(lib().mgfld_workspace_bytes_pair(ctypes.byref(dims), int(precision)))


def mgfld_factor_bytes(dims: Dims, precision: int) -> int:
    return int(lib().mgfld_factor_bytes(ctypes.byref(dims), int(precision)))


def mgfld_step(dims, problem_struct, psi, ye, T, opts, ws, report=None, stream=None):
    """One implicit step in place on (psi, ye, T) (torch CUDA FP64 tensors), asynchronous on the
    stream unless opts.profile is set.  `report` is a dict of optional device tensors: iters,
    ray_status (int32), ledger [n_ray, 8], heating [n_ray] (float64), factorizations (int32),
    status [1] (int32, the step's worst status once it has run)."""
    rep = None
    if report is not None:
        rep = StepReport(_ptr(report.get('iters')), _ptr(report.get('ray_status')),
                         _ptr(report.get('ledger')), _ptr(report.get('heating')),
                         _ptr(report.get('factorizations')), _ptr(report.get('status')))
    st = State(_ptr(psi), _ptr(ye), _ptr(T))
    return lib().mgfld_step(ctypes.byref(dims), ctypes.byref(problem_struct), ctypes.byref(st),
                            ctypes.byref(opts), ctypes.byref(rep) if rep is not None else None,
                            _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))


def mgfld_step_noalloc(dims, problem_struct, psi, ye, T, opts, report=None, stream=None):
    """mgfld_step with the library's own fixed device scratch (no workspace argument) for
    callers that cannot allocate device memory; at most NOALLOC_SCRATCH_BYTES of workspace."""
    rep = None
    if report is not None:
        rep = StepReport(_ptr(report.get('iters')), _ptr(report.get('ray_status')),
                         _ptr(report.get('ledger')), _ptr(report.get('heating')),
                         _ptr(report.get('factorizations')), _ptr(report.get('status')))
    st = State(_ptr(psi), _ptr(ye), _ptr(T))
    return lib().mgfld_step_noalloc(ctypes.byref(dims), ctypes.byref(problem_struct), ctypes.byref(st),
                                    ctypes.byref(opts), ctypes.byref(rep) if rep is not None else None,
                                    _stream(stream))


def mgfld_assemble(dims, problem_struct, psi, ye, T, sys, ws, stream=None):
    """Linearisation at the start of the step; `sys` is a dict diag/lower/upper/rhs of tensors."""
    st = State(_ptr(psi), _ptr(ye), _ptr(T))
    s = System(_ptr(sys['diag']), _ptr(sys['lower']), _ptr(sys['upper']), _ptr(sys['rhs']))
    return lib().mgfld_assemble(ctypes.byref(dims), ctypes.byref(problem_struct), ctypes.byref(st),
                                ctypes.byref(s), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))


def mgfld_factor(dims, sys, precision, factor, stream=None):
    s = System(_ptr(sys['diag']), _ptr(sys['lower']), _ptr(sys['upper']), _ptr(sys.get('rhs')))
    return lib().mgfld_factor(ctypes.byref(dims), ctypes.byref(s), int(precision), _ptr(factor),
                              _stream(stream))


def mgfld_solve(dims, sys, precision, factor, rhs, x, stream=None):
    s = System(_ptr(sys.get('diag')), _ptr(sys['lower']), _ptr(sys['upper']), _ptr(sys.get('rhs')))
    return lib().mgfld_solve(ctypes.byref(dims), ctypes.byref(s), int(precision), _ptr(factor), _ptr(rhs),
                             _ptr(x), _stream(stream))


def mgfld_adjoint_workspace_bytes(dims: Dims) -> int:
    return int(lib().mgfld_adjoint_workspace_bytes(ctypes.byref(dims)))


def mgfld_adjoint(dims, problem_struct, state_n, state_np1, bars, out, ws, heat_weight=1.0, scale_bar=None,
                  max_sweeps=0, sweep_tol=0.0, stream=None):
    """Reverse of one step.  state_n = (psi, ye, T) at the step's start, state_np1 = (psi, ye)
    at its root; bars = (psi_bar, ye_bar, T_bar) of the step's outputs (entries may be None);
    out = (psi_bar_out, ye_bar_out, T_bar_out) tensors to overwrite; scale_bar [4, n_e] is
    accumulated into.  Returns (status, sweeps used, last relative mu_Ye change)."""
    s0 = State(_ptr(state_n[0]), _ptr(state_n[1]), _ptr(state_n[2]))
    s1 = State(_ptr(state_np1[0]), _ptr(state_np1[1]), None)
    io = AdjointIO(_ptr(bars[0]), _ptr(bars[1]), _ptr(bars[2]), float(heat_weight), _ptr(out[0]), _ptr(out[1]),
                   _ptr(out[2]), _ptr(scale_bar), int(max_sweeps), float(sweep_tol), 0, 0.0)
    rc = lib().mgfld_adjoint(ctypes.byref(dims), ctypes.byref(problem_struct), ctypes.byref(s0), ctypes.byref(s1),
                             ctypes.byref(io), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))
    return rc, io.sweeps_used, io.sweep_change


# ---------------------------------------------------------------------------- convenience

class Stepper:
    """Owns the device copies of one problem and a workspace; steps a device state.

    Rays are independent, so a problem whose workspace would exceed `max_ws_bytes`
    is processed in ray chunks that each fit (same results as one call)."""

    def __init__(self, inp, precision=MGFLD_FP64, device='cuda', max_ws_bytes=None, **opt_kw):
        import torch
        prob = inp['problem']
        self.n_ray, _, self.n_r, self.n_e = inp['psi0'].shape
        self.prob = DeviceProblem(prob, device)
        self.precision = precision
        self.opts = step_opts(precision, **opt_kw)
        wsb = mgfld_workspace_bytes_pair if prob.get('pair_coef') is not None else mgfld_workspace_bytes
        per_ray = wsb(Dims(1, self.n_r, self.n_e, N_SPECIES), precision)
        if max_ws_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            max_ws_bytes = free // 2
        self.chunk = max(1, min(self.n_ray, int(max_ws_bytes // max(per_ray, 1))))
        nbytes = wsb(Dims(self.chunk, self.n_r, self.n_e, N_SPECIES), precision)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.report = dict(iters=torch.zeros(self.n_ray, dtype=torch.int32, device=device),
                           ray_status=torch.zeros(self.n_ray, dtype=torch.int32, device=device),
                           ledger=torch.zeros(self.n_ray, 8, dtype=torch.float64, device=device),
                           heating=torch.zeros(self.n_ray, dtype=torch.float64, device=device),
                           factorizations=torch.zeros(self.n_ray, dtype=torch.int32, device=device))
        self.n_chunks = (self.n_ray + self.chunk - 1) // self.chunk
        self.status = torch.zeros(self.n_chunks, dtype=torch.int32, device=device)

    def state_to_device(self, psi, ye, T, device='cuda'):
        import torch
        return tuple(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
                     for a in (psi, ye, T))

    def step(self, psi, ye, T, stream=None, wait=True):
        """Advance (psi, ye, T) in place by one step.  The step runs asynchronously on the stream;
        with wait (default) the call then reads the step's status back (one synchronisation) and
        returns the worst mgfld status, without it it returns at once (MGFLD_OK: launched) and the
        status stays in self.status (one entry per chunk of rays) for the caller to read."""
        for c, lo in enumerate(range(0, self.n_ray, self.chunk)):
            hi = min(self.n_ray, lo + self.chunk)
            d = Dims(hi - lo, self.n_r, self.n_e, N_SPECIES)
            ps = self.prob.struct if (lo == 0 and hi == self.n_ray) else self.prob.rays(lo, hi, self.n_r, self.n_e)
            rep = {k: v[lo:hi] for k, v in self.report.items()}
            rep['status'] = self.status[c:c + 1]
            rc = mgfld_step(d, ps, psi[lo:hi], ye[lo:hi], T[lo:hi], self.opts, self.ws, rep, stream)
            if rc in (MGFLD_EINVAL, MGFLD_ENOMEM, MGFLD_ECUDA):
                raise MgfldError(rc, 'mgfld_step')
            if self.opts.profile:                  # the host-driven loop: rc is the step's status
                self.status[c] = rc
        if not wait:
            return MGFLD_OK
        return self.worst_status()

    def worst_status(self):
        """The worst status of the last step over its chunks (synchronises)."""
        codes = self.status.cpu().tolist()
        if MGFLD_ECUDA in codes:
            raise MgfldError(MGFLD_ECUDA, 'mgfld_step (bounded wait)')
        if MGFLD_ENAN in codes:
            return MGFLD_ENAN
        return MGFLD_ENOCONV if MGFLD_ENOCONV in codes else MGFLD_OK


def eadv_problem(t, limit=True):
    """C struct for mgfld_energy_advect from a dict of device tensors: r_edge_n, r_edge_np1
    [n_ray, n_r+1], rho_n, rho_np1 [n_ray, n_r], optional lapse_n, lapse_np1 [n_ray, n_r],
    e_edge [n_e+1], optional eta1 [n_ray, 4, n_r, n_e], optional u [n_ray, n_r] (the zone velocity
    that rolls energy advection out at a shock) (FP64, contiguous; kept alive by the caller)."""
    return EadvProblem(_ptr(t['r_edge_n']), _ptr(t['r_edge_np1']), _ptr(t['rho_n']), _ptr(t['rho_np1']),
                       _ptr(t.get('lapse_n')), _ptr(t.get('lapse_np1')), _ptr(t['e_edge']), _ptr(t.get('eta1')),
                       1 if limit else 0, _ptr(t.get('u')))


def mgfld_stress_lapse(dims, problem_struct, psi, ye, T, ws, p=None, m_inner=None, f_edge=None, f_zone=None,
                       lapse=None, stream=None):
    """Neutrino stress (edge and zone values) and the lapse of a device state; `ws` a uint8 device
    tensor of at least mgfld_workspace_bytes(dims, MGFLD_FP64) bytes; outputs [n_ray, n_r] FP64
    device tensors or None.  Returns the mgfld status."""
    st = State(_ptr(psi), _ptr(ye), _ptr(T))
    io = StressIO(_ptr(p), _ptr(m_inner), _ptr(f_edge), _ptr(f_zone), _ptr(lapse))
    return lib().mgfld_stress_lapse(ctypes.byref(dims), ctypes.byref(problem_struct), ctypes.byref(st),
                                    ctypes.byref(io), _ptr(ws), ws.numel(), _stream(stream))


def mgfld_energy_advect(dims, eadv_struct, psi, xi=None, stream=None):
    """One energy-advection step in place on psi [n_ray, 4, n_r, n_e] (device FP64); xi [n_ray, 4,
    n_r] (optional) receives each system's energy-fixing factor.  Returns the mgfld status."""
    return lib().mgfld_energy_advect(ctypes.byref(dims), ctypes.byref(eadv_struct), _ptr(psi), _ptr(xi),
                                     _stream(stream))
