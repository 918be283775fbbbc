"""Benchmark of the implicit MGFLD transport step on synthetic post-bounce profiles.

Headline workload: the 2D mixed-precision configuration, 1024 rays (2D, per-ray angular
perturbations) x 512 radial zones x 20 energy groups x 4 species, dt = 1e-6 s, outer tolerance
1e-10 (tolmin_psi = 1), with the seeds of that configuration.  A "step" is one implicit transport
step of every ray (mgfld_step).  Metric: zone*group*species updates per second (n_ray * n_r *
n_e * 4 per step / time) for the mixed-precision path (FP32 block factorisation, FP64 residual
refinement), with the FP64 path at the same tolerance on the same inputs beside it.  A second
line (`config4`) times the 3D-scale mixed configuration, 4096 rays (64 theta x 64 phi) x 540 x 20
x 4, 10 steps.

Under torchrun each rank steps its own 1024 rays of a larger 2D ray set (rays are independent: no
collective on the data path); `value` is the total over ranks.  The 3D-scale line shards its 4096
rays over the ranks.  `--impl reference` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1809_05608_gb300 import problems  # noqa: E402

CONFIG_ID = 3                                   # 2D mixed: 1024 rays x 512 x 20 x 4, 20 steps
RAYS_PER_RANK = problems.CONFIGS[CONFIG_ID].n_ray
C4_ID = 4                                       # 3D-scale mixed: 4096 rays x 540 x 20 x 4, 10 steps
C4_STEPS = problems.CONFIGS[C4_ID].steps
TOL = 1e-10
METRIC = 'MGFLD step zone*group*species updates/s (mixed FP32-factor/FP64-refined at 1e-10; FP64 path beside)'
UNIT = 'updates/s'
FP64_FLOP_PER_CLK_SM = 4.0      # 2 DFMA lanes per clock per SM (1.25 TFLOP/s nominal at 2.07 GHz x 152 SMs)
FP32_FLOP_PER_CLK_SM = 256.0    # 128 FFMA lanes per clock per SM
N_SM = 152
SM_HZ = 2.070e9
PEAK_FP64_TFS = FP64_FLOP_PER_CLK_SM * N_SM * SM_HZ / 1e12
PEAK_FP32_TFS = FP32_FLOP_PER_CLK_SM * N_SM * SM_HZ / 1e12
PEAK_SOURCE = 'derived: %g flop/clk/SM x 152 SMs x 2070 MHz max SM clock'


def _measured_hbm_gbs():
    """The measured HBM copy bandwidth of this machine's GPUs, else the recorded fallback."""
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            return float(json.load(f)['hbm_gbs']), 'measured copy bandwidth (of measured)'
    except (OSError, ValueError, KeyError):
        return 6800.0, 'fallback copy bandwidth 6.8 TB/s (of fallback)'


PEAK_HBM_GBS, HBM_SOURCE = _measured_hbm_gbs()
# FP64 operations of one energy-advection update (+, x, /, sqrt one each, FMA two), counted from
# the formulas the step evaluates per (system, group): Minerbo eta2 16, shifted edge 10, Eq. a78
# and the cell average 25, slope 27, interface value 45, parabola 14, flux 16, energy sums 7,
# Eq. p6 and the new psi 7, the zone constants shared over the groups 1.
EADV_FLOPS_PER_UPDATE = 168


def dist_info():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


def shard(n_gpus, rank, rays_per_rank=RAYS_PER_RANK):
    """Rays of rank `rank`: a contiguous block of a 2D ray set of rays_per_rank * n_gpus rays
    (rays are independent within a step, so ranks exchange nothing on the data path)."""
    return slice(rank * rays_per_rank, (rank + 1) * rays_per_rank)


def workload(n_gpus, rank, rays_per_rank=RAYS_PER_RANK):
    inp = problems.make_problem(CONFIG_ID, n_ray=rays_per_rank * n_gpus)
    if n_gpus > 1:
        inp = problems.subset_rays(inp, shard(n_gpus, rank, rays_per_rank))
    return inp


def shock_workload(n_gpus, rank, rays_per_rank=RAYS_PER_RANK):
    """The same rays with an imposed accretion-shock velocity profile and a flux factor."""
    inp = problems.make_shock_problem(CONFIG_ID, n_ray=rays_per_rank * n_gpus)
    if n_gpus > 1:
        inp = problems.subset_rays(inp, shard(n_gpus, rank, rays_per_rank))
    return inp


def pair_workload(n_gpus, rank, rays_per_rank=RAYS_PER_RANK):
    """The same rays with the synthetic pair process at the NES scale and its angular correction."""
    inp = problems.make_pair_problem(CONFIG_ID, n_ray=rays_per_rank * n_gpus)
    if n_gpus > 1:
        inp = problems.subset_rays(inp, shard(n_gpus, rank, rays_per_rank))
    return inp


def c4_shard(n_gpus, rank, n_ray=None):
    """Contiguous block of the 3D-scale configuration's rays for rank `rank` (its rays are a
    fixed 64 x 64 set, so more ranks each take fewer of them)."""
    n_ray = n_ray or problems.CONFIGS[C4_ID].n_ray
    lo = (n_ray * rank) // n_gpus
    hi = (n_ray * (rank + 1)) // n_gpus
    return slice(lo, hi)


def job_throughput(updates_per_rank_step, world, ms_per_step_max):
    """Whole-job updates/s: every rank's rays over the slowest rank's time per step."""
    return updates_per_rank_step * world / (ms_per_step_max * 1e-3)


def updates_per_step(inp):
    n_ray, n_s, n_r, n_e = inp['psi0'].shape
    return n_ray * n_s * n_r * n_e


def workload_name(inp, steps=None):
    n_ray, n_s, n_r, n_e = inp['psi0'].shape
    s = f'{n_ray} rays x {n_r} zones x {n_e} groups x {n_s} species, dt 1e-6 s, tol 1e-10'
    return s + (f', {steps} steps' if steps else '')


# ------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling every 200 ms; started before the warm-up so that its start-up
    never falls inside a timed region, and filtered to the timed window by its own
    sample timestamps."""
    FIELDS = ('timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.windows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.index), f'--query-gpu={self.FIELDS}',
                 '--format=csv,noheader,nounits', '-lms', '200'],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return
        # nvidia-smi's start-up (NVML initialisation) perturbs the GPU for a moment: wait for
        # its first sample before anything is timed.
        t0 = time.time()
        while not self.lines and time.time() - t0 < 15.0 and self.proc.poll() is None:
            time.sleep(0.05)
        time.sleep(0.5)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=['nvidia-smi unavailable'])
        time.sleep(0.5)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        import datetime
        sm, smax, reasons = [], [], set()
        names = ('hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap')
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(',')]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], '%Y/%m/%d %H:%M:%S.%f').timestamp()
                clk, cmax = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if not any(a - 0.25 <= ts <= b + 0.25 for a, b in self.windows):
                continue
            sm.append(clk)
            smax.append(cmax)
            for name, val in zip(names, parts[5:9]):
                if val.lower() == 'active':
                    reasons.add(name)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=['no samples inside the timed window'])
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                    samples=len(sm))


# ------------------------------------------------------------------------- traffic record

def traffic_record(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, 'profiles', 'ncu_traffic.txt')
    if not os.path.exists(path):
        return None
    src = open(os.path.join(ROOT, 'paper_1809_05608_gb300', 'csrc', 'blocktri.cu'), 'rb').read()
    src += open(os.path.join(ROOT, 'paper_1809_05608_gb300', 'csrc', 'assemble.cu'), 'rb').read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith('#') and parts[0] == kernel and parts[3] == digest:
            return dict(bytes=float(parts[1]), units=float(parts[2]))
    return None


# ------------------------------------------------------------------------- GPU arm

def run_path(M, torch, inp, precision, steps, warmup, barrier, clocks=None, refactor_ratio=None,
             coef_iterate=False, keep=False):
    """Time `steps` implicit steps of one path after `warmup` untimed ones.  The timed loop calls
    mgfld_step as a user does: asynchronous on the stream (the whole step one CUDA graph, its outer
    iteration a device-side loop), no host synchronisation between steps, CUDA events on the
    stream around the loop.  A second pass of `steps` steps then runs with per-category CUDA events
    (mgfld_step_opts.profile, which drives the outer iteration from the host) for the kernel times
    of the rooflines.  The stepper (workspace) is released unless `keep`."""
    st = M.Stepper(inp, precision, tol=TOL, max_iter=60, refactor_ratio=refactor_ratio, coef_iterate=coef_iterate)
    if clocks:
        clocks.start()
    psi, ye, T = st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    stream = torch.cuda.current_stream()
    nfact = torch.zeros_like(st.report['factorizations'])
    iters = torch.zeros_like(st.report['iters'])
    for _ in range(warmup):
        # the same calls as the timed loop (the first builds and caches the step's graph; the
        # counters' first additions load their kernels, which a cold page cache makes slow)
        rc = st.step(psi, ye, T, wait=False)
        assert rc == M.MGFLD_OK, M.status_str(rc)
        nfact += st.report['factorizations']
        iters += st.report['iters']
    assert st.worst_status() == M.MGFLD_OK
    nfact.zero_()
    iters.zero_()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    t_start = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rc = st.step(psi, ye, T, wait=False)
        assert rc == M.MGFLD_OK, M.status_str(rc)
        nfact += st.report['factorizations']
        iters += st.report['iters']
    e1.record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    clk = None
    if clocks:
        clocks.mark(t_start, t_end)
        clk = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    assert st.worst_status() == M.MGFLD_OK
    # the profiled pass: per-category kernel times (and the unit counts they belong to)
    prof = (ctypes.c_double * (2 * M.PROF_N))()
    st.opts.profile = ctypes.cast(prof, ctypes.c_void_p)
    rc = st.step(psi, ye, T)                      # event creation outside the counted pass
    assert rc == M.MGFLD_OK, M.status_str(rc)
    for c in range(2 * M.PROF_N):
        prof[c] = 0.0
    pfact = torch.zeros_like(nfact)
    piters = torch.zeros_like(iters)
    hist = torch.zeros(61, dtype=torch.int64, device=iters.device)
    hist += torch.bincount(st.report['iters'].long(), minlength=61)[:61]   # its kernels loaded, then reset
    hist.zero_()
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    for _ in range(steps):
        rc = st.step(psi, ye, T)
        assert rc == M.MGFLD_OK, M.status_str(rc)
        pfact += st.report['factorizations']
        piters += st.report['iters']
        hist += torch.bincount(st.report['iters'].long(), minlength=61)[:61]
    torch.cuda.synchronize()
    p_ms = (time.perf_counter() - p0) * 1e3
    st.opts.profile = None
    prof = {name: dict(ms=prof[2 * c], launches=int(prof[2 * c + 1])) for c, name in enumerate(M.PROF_NAMES)}
    ws_gb = (st.ws.numel() + sum(t.numel() * 8 for t in st.prob.t.values() if t is not None)) / 1e9
    out = dict(ms=ms, steps=steps, prof=prof, nfact=int(pfact.sum()), iters=int(piters.sum()),
               timed_nfact=int(nfact.sum()), timed_iters=int(iters.sum()),
               max_iters=int(st.report['iters'].max()), iters_hist=np.trim_zeros(hist.cpu().numpy(), 'b').tolist(),
               clocks=clk, chunk=st.chunk, ws_gb=ws_gb, n_ray=st.n_ray, profiled_ms=p_ms, coef=coef_iterate)
    if keep:
        out['stepper'] = st
        out['state'] = (psi, ye, T)
    else:
        del st, psi, ye, T
        torch.cuda.empty_cache()
    return out


def algorithmic_work(inp, kernel, nfact, iters, precision, coef=False, steps=0):
    """Algorithmic flop count over the timed steps for one kernel category.

    factor: per (zone, system) factorisation, N^3 FMAs of in-place Gauss-Jordan plus
    2 N^2 for the diagonal Schur scaling: 2 N^3 + 2 N^2 flops (FP64 or FP32).
    assemble (FP64 pipe only): per (zone, system, iteration) residual, two length-N NES sums
    per row (4 N^2) + 16 N of transport/absorption terms; with a fresh FP64 Jacobian one FMA
    per entry (2 N^2).  The mixed path's Jacobian rows are FP32 and are not counted.  With the
    flux coefficients formed at every iterate (coef) the NES sums arrive from the coefficient
    pass and the residual forms its rows from the coefficients and the limiter's derivatives
    (32 N)."""
    n_ray, n_s, n_r, n = inp['psi0'].shape
    if kernel == 'factor':
        per = 2.0 * n**3 + 2.0 * n**2
        return per * n_s * n_r * nfact
    if kernel == 'assemble':
        if precision == 1 and not coef:           # the first outer iteration only
            return n_s * n_r * n_ray * steps * 24.0 * n
        per_res = 32.0 * n if coef else 4.0 * n**2 + 16.0 * n
        per_jac = 2.0 * n**2 if precision == 0 else 0.0
        return n_s * n_r * (per_res * iters + per_jac * nfact)
    raise ValueError(kernel)


def residual_roofline(res, inp):
    """HBM roofline of the mixed path's later residual passes (k_resid_ff): per (zone, system,
    outer iteration after the first) the FP32-pair NES kernels (16 B per entry and zone, shared by
    the four systems: 4 N^2 B) and 96 B per row (the kept sums read and written, the four step
    constants, psi, j, the last correction, -G written)."""
    n_ray, n_s, n_r, n = inp['psi0'].shape
    prof = res['prof']['residual']
    launches = max(prof['launches'], 1)
    units = n_s * n_r * (res['iters'] - n_ray * res['steps'])
    per_unit = 4 * n * n + 96 * n
    gbs = per_unit * units / (prof['ms'] * 1e-3) / 1e9 if prof['ms'] > 0 else 0.0
    tr = traffic_record('k_resid_ff')
    traffic = None if tr is None else tr['bytes'] / tr['units'] * (units / n_r / launches)
    return dict(bound='hbm', kernel='k_resid_ff', achieved=gbs, peak=PEAK_HBM_GBS, unit='GB/s',
                frac=gbs / PEAK_HBM_GBS, traffic=traffic, peak_source=HBM_SOURCE, bytes_per_zone_system=per_unit,
                kernel_ms_per_launch=prof['ms'] / launches, kernel_share=prof['ms'] / res['ms'])


def roofline_for(res, inp, precision):
    """Roofline of the dominant kernel of the residual/Jacobian and factor categories."""
    prof = res['prof']
    cands = ('assemble', 'factor', 'residual') if prof.get('residual', {}).get('launches') else ('assemble', 'factor')
    dom = max(cands, key=lambda k: prof[k]['ms'])
    if dom == 'residual':
        return residual_roofline(res, inp)
    flops = algorithmic_work(inp, dom, res['nfact'], res['iters'], precision, coef=res.get('coef', False),
                             steps=res['steps'])
    achieved = flops / (prof[dom]['ms'] * 1e-3) / 1e12
    fp32 = dom == 'factor' and precision == 1
    per_clk = FP32_FLOP_PER_CLK_SM if fp32 else FP64_FLOP_PER_CLK_SM
    peak = per_clk * N_SM * SM_HZ / 1e12
    launches = max(prof[dom]['launches'], 1)
    kname = {'factor': 'k_factor_row2' if fp32 else 'k_factor', 'assemble': 'k_assemble'}[dom]
    tr = traffic_record(kname)
    traffic = None
    if tr is not None:
        units_per_launch = (res['nfact'] if dom == 'factor' else res['iters']) * inp['psi0'].shape[1] / launches
        traffic = tr['bytes'] / tr['units'] * units_per_launch
    return dict(bound='alu', kernel=kname, pipe='fp32' if fp32 else 'fp64', achieved=achieved, peak=peak,
                unit='TFLOP/s', frac=achieved / peak, traffic=traffic, peak_source=PEAK_SOURCE % per_clk,
                kernel_ms_per_launch=prof[dom]['ms'] / launches, kernel_share=prof[dom]['ms'] / res['ms'])


def factor_roofline(res, inp):
    """HBM roofline of the mixed path's FP32 block factorisation (k_factor_row2), the kernel that
    moves the FP32 blocks: per (zone, system) factorisation the N x N Jacobian block read and its
    N x N inverse written (2 x 4 N^2 B) plus the two FP32 couplings (8 N B).  Its FP32 flops
    (2 N^3 + 2 N^2) are reported beside it as a fraction of the derived FP32 peak."""
    n_ray, n_s, n_r, n = inp['psi0'].shape
    prof = res['prof']['factor']
    launches = max(prof['launches'], 1)
    units = n_s * n_r * res['nfact']
    per_unit = 8 * n * n + 8 * n
    gbs = per_unit * units / (prof['ms'] * 1e-3) / 1e9
    tfs = (2.0 * n**3 + 2.0 * n**2) * units / (prof['ms'] * 1e-3) / 1e12
    tr = traffic_record('k_factor_row2')
    traffic = None if tr is None else tr['bytes'] / tr['units'] * (units / n_r / launches)
    return dict(bound='hbm', kernel='k_factor_row2', achieved=gbs, peak=PEAK_HBM_GBS, unit='GB/s',
                frac=gbs / PEAK_HBM_GBS, traffic=traffic, peak_source=HBM_SOURCE, bytes_per_zone_system=per_unit,
                fp32_tflops=tfs, fp32_frac=tfs / PEAK_FP32_TFS, fp32_peak_source=PEAK_SOURCE % FP32_FLOP_PER_CLK_SM,
                kernel_ms_per_launch=prof['ms'] / launches, kernel_share=prof['ms'] / res['ms'])


def solve_roofline(res, inp):
    """HBM roofline of the mixed path's FP32 substitution (k_sysmax + k_solve_tma per solve).

    Bytes per (zone, system) and solve: every FP32 inverse block read by the inward and by the
    outward sweep (2 N^2 x 4 B; the blocks of the workload do not stay in the 129 MB L2 between
    the sweeps), plus the vectors: rhs read (8 N), its FP32 copy written and read (2 x 4 N), the
    two couplings (2 x 4 N), the forward result written and read (2 x 4 N) and x written (8 N)."""
    n_ray, n_s, n_r, n = inp['psi0'].shape
    prof = res['prof']['solve']
    solves = prof['launches']
    per_unit = 2 * n * n * 4 + 8 * n + 8 * n + 8 * n + 8 * n + 8 * n
    # iterations of the active rays: res['iters'] counts (ray, iteration) pairs over the timed steps
    nbytes = per_unit * n_s * n_r * res['iters']
    achieved = nbytes / (prof['ms'] * 1e-3) / 1e9
    tr = traffic_record('k_solve_tma')
    traffic = None
    if tr is not None and solves:
        traffic = tr['bytes'] / tr['units'] * (res['iters'] * n_s / solves)
    return dict(bound='hbm', kernel='k_solve_tma', achieved=achieved, peak=PEAK_HBM_GBS, unit='GB/s',
                frac=achieved / PEAK_HBM_GBS, traffic=traffic, peak_source=HBM_SOURCE,
                bytes_per_zone_system=per_unit, kernel_ms_per_launch=prof['ms'] / max(solves, 1),
                kernel_share=prof['ms'] / res['ms'])


def category_work(n, precision, coef=False):
    """Algorithmic work of each kernel category, per unit, for N = n groups.

    Returns {category: (unit, fp64 flop, fp32 flop, HBM bytes)} with units:
      'step'  per (zone, system) and step;
      'iter'  per (zone, system) and outer iteration of its ray;
      'citer' per (zone, system) and outer iteration after the first (coef only);
      'fact'  per (zone, system) and factorisation;
    and a second entry '<category>_<unit>' for a further part of a category.
    FP64 (precision 0) vs mixed (1) as the two paths compute; coef: the flux coefficients formed
    again at every outer iterate.  Counted from the formulas (not from the instructions the
    kernels issue): see the work table of the design notes."""
    N = float(n)
    mixed = precision == 1
    blk = 4.0 if mixed else 8.0
    w = {
        # NES rows (1.5 N^2 per zone over 4 systems) and the NES sums at psi^n (16 N^2 per zone),
        # emissivity, mean free path, neutrinosphere, ghost factor and limiter (~40 per element);
        # psi^n, kappa_a, kappa_s read, five per-element coefficient arrays written, the NES
        # kernels written once (FP64 in and out, plus two FP32 copies or the FP64 difference).
        'setup': ('step', 4.4 * N * N + 40 * N, 0.0, 64 * N + 6 * N * N),
        # residual: two N-term NES sums per row + 16 N; NES kernels read once per zone and
        # iteration (4 N^2 per system), psi, psi^n, j, kappa_a, alpha read and -G written (48 N)
        'assemble': ('iter', 4 * N * N + 16 * N, 0.0, 4 * N * N + 48 * N),
        # a fresh Jacobian: one FMA per entry (FP64) or FP32, its block written, the FP32 / FP64
        # in-minus-out kernel read (2 N^2 per system)
        'assemble_fact': ('fact', 0.0 if mixed else 2 * N * N, 2 * N * N if mixed else 0.0,
                          blk * N * N + 2 * N * N),
        # in-place Gauss-Jordan (2 N^3) + the diagonal Schur scaling (2 N^2); block in, inverse out
        'factor': ('fact', 0.0 if mixed else 2 * N ** 3 + 2 * N * N, 2 * N ** 3 + 2 * N * N if mixed else 0.0,
                   2 * blk * N * N + (8 if mixed else 16) * N),
        # two sweeps, each a matrix-vector product with the inverse block read (2 blk N^2 B)
        'solve': ('iter', 0.0 if mixed else 4 * N * N, 4 * N * N if mixed else 0.0,
                  2 * blk * N * N + 40 * N),
        # psi += dpsi and the tolerance test (x, psi read, psi written); Ye Newton per zone on the
        # two electron-flavour systems (kappa_a, j, psi read, j written)
        'update': ('iter', 8 * N, 0.0, 24 * N + 16 * N),
        # the converged sources (FP64 residual pass, or the kept sums plus an FP32 product), Eq.
        # a62b, T and the ledgers: NES kernels read once, psi, psi^n, sources read/written
        'finish': ('step', 16 * N + (0.0 if mixed else 4 * N * N), 2 * N * N if mixed else 0.0,
                   (2 if mixed else 4) * N * N + 40 * N),
    }
    if coef:
        # the coefficients at the iterate: the NES sums (4 N^2, handed on to the residual), the
        # mean free path, the neutrinosphere scan and the limiter with its two derivatives (~50 N);
        # NES kernels read (4 N^2 B), psi and sqrt(lambda) read, seven coefficient arrays written
        w['setup_citer'] = ('citer', 4 * N * N + 50 * N, 0.0, 4 * N * N + 96 * N)
        # the residual rows from the kept sums, the coefficients and the limiter's derivatives
        w['assemble'] = ('iter', 32 * N, 0.0, 88 * N)
    elif mixed:
        # the first outer iteration: the step constants and the row from the setup's NES sums
        # (~24 FP64 flop per row); psi, psi^n, j, kappa_a, alpha, the sums read, the four step
        # constants and -G written
        w['assemble'] = ('step', 24 * N, 0.0, 104 * N)
        # the later ones (k_resid_ff): the two increments phin.dpsi, phout.dpsi (4 N^2 flop at
        # FP32-pair precision) added to the kept sums and the row formed (16 N FP64); the kernels
        # in FP32 pairs (16 B per entry and zone: 4 N^2 B per system), and per row the sums read
        # and written, the four step constants, psi, j, the correction, -G (96 B)
        w['residual'] = ('citer', 16 * N, 4 * N * N, 4 * N * N + 96 * N)
    return w


def step_roofline(res, inp, precision):
    """Whole-step roofline of one path: per kernel category, the time its algorithmic FP64 flops,
    FP32 flops and HBM bytes need at the peaks (the largest of the three binds), summed over the
    categories, against the measured time per step.  Units are counted from the timed run's
    per-ray iteration and factorisation counts."""
    n_ray, n_s, n_r, n = inp['psi0'].shape
    zs = n_s * n_r                               # (zone, system) pairs per ray
    units = dict(step=zs * n_ray * res['steps'], iter=zs * res['iters'], fact=zs * res['nfact'],
                 citer=zs * (res['iters'] - n_ray * res['steps']))
    cats = {}
    tot64 = tot32 = totb = t_roof = 0.0
    for name, (unit, f64, f32, b) in category_work(n, precision, coef=res.get('coef', False)).items():
        u = units[unit]
        F64, F32, B = f64 * u, f32 * u, b * u
        t64 = F64 / (PEAK_FP64_TFS * 1e12)
        t32 = F32 / (PEAK_FP32_TFS * 1e12)
        tb = B / (PEAK_HBM_GBS * 1e9)
        base = name.split('_')[0]
        c = cats.setdefault(base, dict(fp64_gflop=0.0, fp32_gflop=0.0, hbm_gb=0.0, t64=0.0, t32=0.0, tb=0.0))
        c['fp64_gflop'] += F64 / 1e9
        c['fp32_gflop'] += F32 / 1e9
        c['hbm_gb'] += B / 1e9
        c['t64'] += t64
        c['t32'] += t32
        c['tb'] += tb
        tot64 += F64
        tot32 += F32
        totb += B
    steps = res['steps']
    # per-step scale of the profiled pass's units (the timed pass ran the same workload)
    for base, c in cats.items():
        bound = max(('fp64', c['t64']), ('fp32', c['t32']), ('hbm', c['tb']), key=lambda v: v[1])
        c['bound'] = bound[0]
        c['roofline_ms_per_step'] = bound[1] * 1e3 / steps
        meas = res['prof'].get(base, {}).get('ms', 0.0) / steps
        c['measured_ms_per_step'] = meas
        c['frac'] = c['roofline_ms_per_step'] / meas if meas > 0 else None
        for k in ('t64', 't32', 'tb'):
            c.pop(k)
        for k in ('fp64_gflop', 'fp32_gflop', 'hbm_gb'):
            c[k] /= steps
        t_roof += c['roofline_ms_per_step']
    ms = res['ms'] / steps
    return dict(roofline_ms_per_step=t_roof, ms_per_step=ms, frac=t_roof / ms,
                fp64_gflop_per_step=tot64 / 1e9 / steps, fp32_gflop_per_step=tot32 / 1e9 / steps,
                hbm_gb_per_step=totb / 1e9 / steps, categories=cats,
                peaks=dict(fp64_tflops=PEAK_FP64_TFS, fp32_tflops=PEAK_FP32_TFS, hbm_gbs=PEAK_HBM_GBS),
                method='sum over kernel categories of max(FP64 flop / FP64 peak, FP32 flop / FP32 peak, '
                       'HBM bytes / HBM peak), algorithmic counts per unit from the formulas')


def e2e_run(M, torch, inp, precision, steps, parts=2):
    """Same metric through the public API from pinned HOST buffers: every step uploads that
    step's inputs (matter, opacities, NES scale, grid, state), runs mgfld_step and reads the new
    state back.  The rays are processed in `parts` contiguous blocks, each with its own Stepper;
    the blocks' steps run one after another on one compute stream, and each block's copies run on
    its own copy streams while the other blocks compute: its state is read back (device -> host)
    as soon as its step ends and uploaded again (host -> device) for its next step, and its
    problem arrays of step s+1 go into a second device copy while step s runs (double buffering)."""
    n_ray = inp['psi0'].shape[0]
    names = ('r_edge', 'rho', 'kappa_abs', 'kappa_scat', 'nes_coef')
    main = torch.cuda.current_stream()
    comp = torch.cuda.Stream()
    blocks = []
    h2d = d2h = 0
    for c in range(parts):
        sub = problems.subset_rays(inp, slice(n_ray * c // parts, n_ray * (c + 1) // parts))
        st = M.Stepper(sub, precision, tol=TOL, max_iter=60)
        prob = sub['problem']
        host = {k: torch.from_numpy(np.ascontiguousarray(prob[k], dtype=np.float64)).pin_memory() for k in names}
        hs = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
              for a in (sub['psi0'], sub['ye0'], sub['T0'])]
        blk = dict(st=st, host=host, hs=hs, dev=[torch.empty_like(h, device='cuda') for h in hs],
                   out=[torch.empty_like(h).pin_memory() for h in hs], bufs=[st.prob, M.DeviceProblem(prob)],
                   copy=torch.cuda.Stream(), back=torch.cuda.Stream(),
                   ready=[torch.cuda.Event(), torch.cuda.Event()], free=[torch.cuda.Event(), torch.cuda.Event()],
                   state=torch.cuda.Event(), done=torch.cuda.Event(), read=torch.cuda.Event())
        h2d += sum(v.numel() * 8 for v in host.values()) + sum(h.numel() * 8 for h in hs)
        d2h += sum(h.numel() * 8 for h in hs)
        blocks.append(blk)

    def upload(blk, b):
        with torch.cuda.stream(blk['copy']):
            for k in names:
                blk['bufs'][b].t[k].copy_(blk['host'][k], non_blocking=True)
            blk['ready'][b].record(blk['copy'])

    def upload_state(blk, src):
        with torch.cuda.stream(blk['copy']):
            for d, h in zip(blk['dev'], src):
                d.copy_(h, non_blocking=True)
            blk['state'].record(blk['copy'])

    def run(n_steps, e0, e1, first):
        e0.record(main)
        comp.wait_event(e0)
        for blk in blocks:
            blk['copy'].wait_event(e0)
            blk['back'].wait_event(e0)
            upload(blk, 0)
            upload_state(blk, blk['hs'] if first else blk['out'])
        for s in range(n_steps):
            b = s % 2
            for blk in blocks:
                if s + 1 < n_steps:
                    if s >= 1:
                        blk['copy'].wait_event(blk['free'][1 - b])
                    upload(blk, 1 - b)
                comp.wait_event(blk['ready'][b])
                comp.wait_event(blk['state'])
                blk['st'].prob = blk['bufs'][b]
                with torch.cuda.stream(comp):
                    rc = blk['st'].step(*blk['dev'], stream=comp, wait=False)
                    assert rc == M.MGFLD_OK, M.status_str(rc)
                    blk['free'][b].record(comp)
                    blk['done'].record(comp)
                # the new state back to the host, then up again for the block's next step
                blk['back'].wait_event(blk['done'])
                with torch.cuda.stream(blk['back']):
                    for o, d in zip(blk['out'], blk['dev']):
                        o.copy_(d, non_blocking=True)
                    blk['read'].record(blk['back'])
                if s + 1 < n_steps:
                    blk['copy'].wait_event(blk['read'])
                    upload_state(blk, blk['out'])
        for blk in blocks:
            main.wait_stream(blk['back'])
            main.wait_stream(blk['copy'])
        main.wait_stream(comp)
        e1.record(main)
        torch.cuda.synchronize()

    # two untimed steps (each block's step graphs for both problem buffers built and cached); the
    # timed steps continue from their state, read back to the host
    torch.cuda.synchronize()
    run(2, torch.cuda.Event(), torch.cuda.Event(), True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    run(steps, e0, e1, False)
    ms = e0.elapsed_time(e1)
    for blk in blocks:
        assert blk['st'].worst_status() == M.MGFLD_OK
        blk['st'].prob = blk['bufs'][0]
    del blocks
    torch.cuda.empty_cache()
    return dict(ms=ms, h2d=h2d, d2h=d2h, parts=parts)


# ------------------------------------------------------------------------- CPU oracle

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(job):
    """One pool task: the oracle's implicit step(s) on one ray (arrays passed in)."""
    sub, n_steps, kw = job
    from oracle import mgfld_oracle as O
    O.run_steps(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'], n_steps, **kw)
    return 0


def _init_worker(barrier):
    """Pool start-up: the oracle's imports, then a wait until every worker has done them, so that
    no worker is still starting (and taking host cores) once the pool is handed over."""
    from oracle import mgfld_oracle  # noqa: F401
    try:
        barrier.wait(timeout=600)
    except Exception:
        pass


def _warm_worker(_):
    return os.getpid()


class OraclePool:
    """A process pool over rays for the CPU oracle (rays are independent), started with `spawn`
    and with one BLAS thread per process, so that each worker is one host core.  Every worker is
    started and has imported the oracle before the constructor returns."""

    def __init__(self, cores=None):
        import multiprocessing
        self.cores = cores or host_cores()
        saved = {k: os.environ.get(k) for k in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS')}
        for k in saved:
            os.environ[k] = '1'
        try:
            ctx = multiprocessing.get_context('spawn')
            barrier = ctx.Barrier(self.cores)
            self.ex = ctx.Pool(self.cores, initializer=_init_worker, initargs=(barrier,))
            self.ex.map(_warm_worker, range(self.cores), chunksize=1)   # start-up outside any timing
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def time_rays(self, inp, rays, n_steps=1, **kw):
        """Wall time of the oracle on the given rays, one pool task per ray."""
        jobs = [(problems.subset_rays(inp, slice(r, r + 1)), n_steps, kw) for r in rays]
        w0 = time.perf_counter()
        self.ex.map(_oracle_worker, jobs, chunksize=1)
        return time.perf_counter() - w0

    def close(self):
        self.ex.close()
        self.ex.join()


def oracle_sample(inp, n_rays, n_steps=1, **step_kw):
    """Time the CPU oracle, as it stands, on the first n_rays rays for n_steps steps, in this
    process (one core)."""
    from oracle import mgfld_oracle as O
    sub = problems.subset_rays(inp, slice(0, n_rays))
    c0, w0 = time.process_time(), time.perf_counter()
    O.run_steps(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'], n_steps, **step_kw)
    wall = time.perf_counter() - w0
    cpu = time.process_time() - c0
    ups = updates_per_step(sub) * n_steps / wall
    n_all = inp['psi0'].shape[0]
    return dict(value=ups, unit=UNIT, cores=max(1, int(round(cpu / wall))), kind='oracle',
                sample=f'{n_rays} of the {n_all} rays x {n_steps} implicit step(s), FP64 numpy/LAPACK, '
                       f'{wall:.1f} s wall', wall_s=wall)


def oracle_pool_sample(pool, inp, rays_per_core=2, n_steps=1, **kw):
    """The oracle on a process pool of the host cores: rays_per_core rays per core,
    spread over the workload, one task per ray."""
    n_all = inp['psi0'].shape[0]
    n = min(n_all, pool.cores * rays_per_core)
    rays = np.unique(np.linspace(0, n_all - 1, n).round().astype(int)).tolist()
    wall = pool.time_rays(inp, rays, n_steps, **kw)
    per_ray = updates_per_step(inp) // n_all
    return dict(value=per_ray * len(rays) * n_steps / wall, unit=UNIT, cores=pool.cores, kind='oracle',
                sample=f'{len(rays)} of the {n_all} rays (evenly spaced) x {n_steps} implicit step(s), one ray '
                       f'per task on a spawn process pool of {pool.cores} host cores (one BLAS thread each), '
                       f'FP64 numpy/LAPACK, {wall:.1f} s wall', wall_s=wall)


def stress_oracle_sample(inp, n_rays):
    """Time the stress-and-lapse oracle, as it stands, on the first n_rays rays' state."""
    from oracle import stress_lapse_oracle as S
    sub = problems.subset_rays(inp, slice(0, n_rays))
    p, m = problems.stress_inputs(sub)
    c0, w0 = time.process_time(), time.perf_counter()
    S.stress_and_lapse(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'], p, m)
    wall = time.perf_counter() - w0
    return dict(value=updates_per_step(sub) / wall, unit=UNIT, kind='oracle',
                cores=max(1, int(round((time.process_time() - c0) / wall))),
                sample=f'{n_rays} of the {inp["psi0"].shape[0]} rays, one call, FP64 numpy, {wall:.2f} s wall')


def energy_advection_run(M, torch, n_gpus, rank, steps, warmup, cpu_rays=0):
    """The energy-advection step (mgfld_energy_advect) on the same rays: device-resident inputs,
    `warmup` untimed steps, then `steps` steps timed with CUDA events on the launching stream
    (psi is advanced in place; the zone changes repeat every step).  Algorithmic traffic per
    update: psi read and written, eta1 read (24 B; the per-zone arrays are < 1 %)."""
    from paper_1809_05608_gb300 import problems as P
    inp = P.make_energy_advection(CONFIG_ID, n_ray=RAYS_PER_RANK * n_gpus)
    if n_gpus > 1:
        sl = shard(n_gpus, rank)
        for key in ('r_edge_n', 'r_edge_np1', 'rho_n', 'rho_np1', 'lapse_n', 'lapse_np1', 'psi', 'eta1'):
            inp[key] = np.ascontiguousarray(inp[key][sl])
    dev = {k: torch.as_tensor(np.ascontiguousarray(v), device='cuda') for k, v in inp.items()
           if isinstance(v, np.ndarray)}
    n_ray, n_s, n_r, n_e = inp['psi'].shape
    dims = M.Dims(n_ray, n_r, n_e, n_s)
    st = M.eadv_problem(dev)
    psi = dev['psi'].clone()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        assert M.mgfld_energy_advect(dims, st, psi, None, stream) == M.MGFLD_OK
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        M.mgfld_energy_advect(dims, st, psi, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ups = n_ray * n_s * n_r * n_e
    gbs = 24.0 * ups / (ms * 1e-3) / 1e9
    tfs = EADV_FLOPS_PER_UPDATE * ups / (ms * 1e-3) / 1e12
    mb = ups * 16 / 1e6
    # The kernel is bound by the FP64 pipe (divisions, square roots and the PPM arithmetic on
    # 24 B per update), not by HBM; both figures are reported, the FP64 one as the roofline.
    out = dict(metric='energy-advection updates/s', value=ups / (ms * 1e-3), unit=UNIT, ms_per_step=ms,
               steps=steps, warmup=warmup, dtype='f64',
               config=dict(workload=f'{n_ray} rays x {n_r} zones x {n_e} groups x {n_s} species, one step per '
                                    'launch, psi advanced in place',
                           l2=f'reads {mb:.0f} MB (psi, eta1) and writes {mb / 2:.0f} MB per step, larger than '
                              'the 129 MB L2'),
               roofline=dict(bound='alu', pipe='fp64', kernel='k_energy_advect', achieved=tfs, peak=PEAK_FP64_TFS,
                             unit='TFLOP/s', frac=tfs / PEAK_FP64_TFS, traffic=None,
                             flops_per_update=EADV_FLOPS_PER_UPDATE, peak_source=PEAK_SOURCE % FP64_FLOP_PER_CLK_SM),
               roofline_hbm=dict(bound='hbm', achieved=gbs, peak=PEAK_HBM_GBS, unit='GB/s', frac=gbs / PEAK_HBM_GBS,
                                 bytes_per_update=24, peak_source=HBM_SOURCE))
    if cpu_rays:
        from oracle import energy_advection_oracle as EO
        sub = {k: (np.ascontiguousarray(v[:cpu_rays]) if isinstance(v, np.ndarray) and v.ndim > 1 else v)
               for k, v in inp.items()}
        rc0 = 0.5 * (sub['r_edge_n'][:, 1:] + sub['r_edge_n'][:, :-1])
        rc1 = 0.5 * (sub['r_edge_np1'][:, 1:] + sub['r_edge_np1'][:, :-1])
        b = lambda a: np.broadcast_to(a[:, None, :], (a.shape[0], n_s, a.shape[1]))
        c0, w0 = time.process_time(), time.perf_counter()
        EO.step(sub['e_edge'], b(sub['lapse_n']), b(sub['lapse_np1']), b(rc0), b(rc1), b(sub['rho_n']),
                b(sub['rho_np1']), sub['psi'], sub['eta1'])
        wall = time.perf_counter() - w0
        out['cpu_baseline'] = dict(value=cpu_rays * n_s * n_r * n_e / wall, unit=UNIT,
                                   cores=max(1, int(round((time.process_time() - c0) / wall))), kind='oracle',
                                   sample=f'{cpu_rays} of the {n_ray} rays x 1 step, FP64 numpy, {wall:.2f} s wall')
    del dev, psi
    torch.cuda.empty_cache()
    return out


def stress_lapse_run(M, torch, inp, steps, warmup):
    """mgfld_stress_lapse (the neutrino stress and the lapse, Eqs. a62e-a62l) on the benchmark rays'
    state: device-resident inputs, `warmup` untimed calls, `steps` calls timed with CUDA events on
    the launching stream.  Each call forms the transport coefficients of the state (the setup
    kernels of the step) before the stress and lapse kernels, which the setup dominates."""
    p, m = problems.stress_inputs(inp)
    n_ray, n_s, n_r, n_e = inp['psi0'].shape
    dims = M.Dims(n_ray, n_r, n_e, n_s)
    dp = M.DeviceProblem(inp['problem'])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device='cuda')
    psi, ye, T, pd, md = dev(inp['psi0']), dev(inp['ye0']), dev(inp['T0']), dev(p), dev(m)
    ws = torch.empty(M.mgfld_workspace_bytes(dims, M.MGFLD_FP64), dtype=torch.uint8, device='cuda')
    out = {k: torch.empty(n_ray, n_r, dtype=torch.float64, device='cuda') for k in ('f_edge', 'f_zone', 'lapse')}
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        assert M.mgfld_stress_lapse(dims, dp.struct, psi, ye, T, ws, p=pd, m_inner=md, stream=stream, **out) == 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        M.mgfld_stress_lapse(dims, dp.struct, psi, ye, T, ws, p=pd, m_inner=md, stream=stream, **out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ups = n_ray * n_s * n_r * n_e
    del ws, dp, out, psi, ye, T, pd, md
    torch.cuda.empty_cache()
    return dict(metric='stress-and-lapse updates/s', value=ups / (ms * 1e-3), unit=UNIT, ms_per_call=ms,
                steps=steps, warmup=warmup, dtype='f64', launches_per_call=9,
                note='one call = the 7 setup kernels of the transport step on the state, k_stress, k_lapse')


def reference_arm(args, n_gpus, rank):
    """The oracle, as it stands, on the host cores, on this arm's workload: each step is the
    oracle's implicit step of one ray per core (a bounded sample; rays are independent, so
    updates/s scale per ray)."""
    if rank != 0:
        return 0
    inp = workload(1, 0)
    pool = OraclePool()
    n_all = inp['psi0'].shape[0]
    per_step = []
    rays_all = np.linspace(0, n_all - 1, pool.cores * (args.warmup + args.steps)).round().astype(int)
    for s in range(args.warmup + args.steps):
        rays = rays_all[s * pool.cores:(s + 1) * pool.cores].tolist()
        wall = pool.time_rays(inp, rays)
        if s >= args.warmup:
            per_step.append(wall)
    pool.close()
    ms = 1e3 * float(np.mean(per_step))
    per_ray = updates_per_step(inp) // n_all
    value = per_ray * pool.cores / (ms * 1e-3)
    sample = (f'{pool.cores} rays per timed step (one per host core, a spawn process pool with one BLAS thread '
              f'per process), evenly spaced over the {n_all} rays, one FP64 implicit step each')
    line = dict(impl='reference', metric=METRIC, value=value, unit=UNIT, n_gpus=n_gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling='weak', vs_baseline=None,
                dtype='f64', data='synthetic',
                config=dict(workload='2d ' + workload_name(inp), oracle_rays_per_step=pool.cores),
                cpu_baseline=dict(value=value, unit=UNIT, cores=pool.cores, kind='oracle', sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------- main

def profile_step(path, n_rays, config, zones=None):
    """One implicit step of the first n_rays rays of a workload (FP64 Newton, the mixed path, the
    mixed path with the shock terms or with the flux coefficients formed at every outer iterate),
    two energy-advection steps, or one stress-and-lapse call, for ncu captures of single launches
    (the step with its outer iteration driven from the host, whose kernels are ordinary launches);
    `zones` builds the rays with that many zones over the same radial range (a launch with the
    workload's systems per SM at a fraction of its memory); exits non-zero on a failed step."""
    import torch
    from paper_1809_05608_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_1809_05608_gb300 import mgfld as M
    if path == 'eadv':
        inp = problems.make_energy_advection(config, rays=slice(0, n_rays))
        dev = {k: torch.as_tensor(np.ascontiguousarray(v), device='cuda') for k, v in inp.items()
               if isinstance(v, np.ndarray)}
        n_ray, n_s, n_r, n_e = inp['psi'].shape
        rc = 0
        for _ in range(2):
            rc = rc or M.mgfld_energy_advect(M.Dims(n_ray, n_r, n_e, n_s), M.eadv_problem(dev), dev['psi'])
        torch.cuda.synchronize()
        print(f'profile step eadv: {n_rays} rays, status {M.status_str(rc)}', flush=True)
        return 0 if rc == M.MGFLD_OK else 1
    if path == 'stress':
        inp = problems.make_problem(config, rays=slice(0, n_rays))
        res = stress_lapse_run(M, torch, inp, 1, 1)
        print(f'profile step stress: {n_rays} rays, {res["ms_per_call"]:.3f} ms', flush=True)
        return 0
    if path == 'shock':
        inp = problems.make_shock_problem(config, rays=slice(0, n_rays), n_r=zones)
    elif path == 'pair':
        inp = problems.make_pair_problem(config, rays=slice(0, n_rays), n_r=zones)
    else:
        inp = problems.make_problem(config, rays=slice(0, n_rays), n_r=zones)
    prec = M.MGFLD_FP64 if path == 'fp64' else M.MGFLD_MIXED
    st = M.Stepper(inp, prec, tol=TOL, max_iter=60, coef_iterate=path == 'coef')
    psi, ye, T = st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    # the host-driven outer iteration (per-category events): ncu profiles the kernels of ordinary
    # launches, not those inside a graph with a conditional node
    prof = (ctypes.c_double * (2 * M.PROF_N))()
    st.opts.profile = ctypes.cast(prof, ctypes.c_void_p)
    rc = st.step(psi, ye, T)
    torch.cuda.synchronize()
    print(f'profile step {path}: {n_rays} rays, status {M.status_str(rc)}, '
          f'iterations {int(st.report["iters"].max())}', flush=True)
    return 0 if rc == M.MGFLD_OK else 1


def path_summary(res, inp, precision, ws, world_ms, ups, n_rays_rank, rooflines=True, **extra):
    out = dict(value=job_throughput(ups, ws, world_ms), unit=UNIT, ms_per_step=world_ms,
               kernel_ms={k: v['ms'] for k, v in res['prof'].items()},
               outer_iterations_per_step=res['max_iters'], iterations_histogram=res['iters_hist'],
               factorizations_per_ray_step=res['nfact'] / (n_rays_rank * res['steps']),
               gpu_launches=sum(v['launches'] for v in res['prof'].values()))
    if rooflines:
        out.update(roofline=roofline_for(res, inp, precision), roofline_step=step_roofline(res, inp, precision))
    out.update(extra)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=20)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='mgfld', choices=['mgfld', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-extra', action='store_true',
                    help='headline and its FP64 comparison only (no 3D-scale, shock, n+1, pair, stress, '
                         'energy-advection lines)')
    ap.add_argument('--profile-step', choices=['mixed', 'fp64', 'shock', 'coef', 'pair', 'eadv', 'stress'],
                    help='profiling target: one implicit step of this path (shock: the mixed path with '
                         'the shock terms; pair: the mixed path with the pair process and its angular '
                         'correction; coef: the mixed path with the flux coefficients formed at '
                         'every outer iterate; eadv: two energy-advection steps; stress: two stress-and-lapse '
                         'calls) on --rays rays of --config, no timing')
    ap.add_argument('--rays', type=int, default=64)
    ap.add_argument('--config', type=int, default=CONFIG_ID)
    ap.add_argument('--zones', type=int, default=None,
                    help='profiling target: the rays built with ZONES zones over the same radial range')
    args = ap.parse_args()
    if args.profile_step:
        return profile_step(args.profile_step, args.rays, args.config, args.zones)
    ws, rank, local = dist_info()
    n_gpus = max(args.gpus, ws)
    if args.impl == 'reference':
        return reference_arm(args, n_gpus, rank)

    # The oracle's process pool starts (spawn) before the first CUDA call of this process.
    pool = OraclePool() if (rank == 0 and ws == 1 and not args.no_cpu_baseline) else None

    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device='cuda')
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    from paper_1809_05608_gb300 import build as B
    if not os.path.exists(B.LIB) and rank == 0:
        B.build()
    barrier()
    from paper_1809_05608_gb300 import mgfld as M

    inp = workload(n_gpus, rank)
    n_rays_rank = inp['psi0'].shape[0]
    ups = updates_per_step(inp)
    clocks = ClockSampler(local)
    mixed = run_path(M, torch, inp, M.MGFLD_MIXED, args.steps, args.warmup, barrier, clocks)
    # FP64 beside it at the same tolerance: the same modified-Newton policy with FP64 factors (the
    # like-for-like baseline), and Newton with a new FP64 factorisation every iteration.
    fp64 = run_path(M, torch, inp, M.MGFLD_FP64, args.steps, args.warmup, barrier, refactor_ratio=0.1)
    newton = run_path(M, torch, inp, M.MGFLD_FP64, args.steps, args.warmup, barrier, refactor_ratio=0.0)
    ms_mixed = max_over_ranks(mixed['ms']) / args.steps
    ms_fp64 = max_over_ranks(fp64['ms']) / args.steps
    ms_newton = max_over_ranks(newton['ms']) / args.steps
    value = job_throughput(ups, ws, ms_mixed)
    value64 = job_throughput(ups, ws, ms_fp64)
    e2e = e2e_run(M, torch, inp, M.MGFLD_MIXED, args.steps)
    e2e_ms = max_over_ranks(e2e['ms']) / args.steps
    roof = roofline_for(mixed, inp, M.MGFLD_MIXED)
    # library kernels in the timed region: those of the profiled pass (the same kernels per
    # iteration), plus the graph's loop-condition kernel per iteration and its status kernel per step
    launches = sum(v['launches'] for v in mixed['prof'].values()) + args.steps * (mixed['max_iters'] + 1)
    extra = {}
    if not args.no_extra:
        # the 3D-scale configuration: 4096 rays x 540 x 20, its rays sharded over the ranks
        c4 = problems.make_problem(C4_ID, rays=c4_shard(n_gpus, rank))
        c4_ups = updates_per_step(c4)
        c4_res = run_path(M, torch, c4, M.MGFLD_MIXED, C4_STEPS, args.warmup, barrier)
        c4_ms = max_over_ranks(c4_res['ms']) / C4_STEPS
        c4_total = updates_per_step(problems.make_problem(C4_ID, rays=slice(0, 1))) * problems.CONFIGS[C4_ID].n_ray
        extra['config4'] = dict(
            metric=METRIC, value=c4_total / (c4_ms * 1e-3), unit=UNIT, ms_per_step=c4_ms, steps=C4_STEPS,
            warmup=args.warmup, scaling='strong', dtype='f32 factor + f64 residual/update',
            config=dict(workload='3d 64x64 ' + workload_name(c4, C4_STEPS).replace(f'{c4["psi0"].shape[0]} rays',
                                                                                  '4096 rays'),
                        rays_per_gpu=c4['psi0'].shape[0], chunk_rays=c4_res['chunk'],
                        l2='working set %.1f GB per GPU, larger than the 129 MB L2' % c4_res['ws_gb']),
            **{k: v for k, v in path_summary(c4_res, c4, M.MGFLD_MIXED, 1, c4_ms, c4_ups,
                                              c4['psi0'].shape[0]).items()
               if k not in ('value', 'unit', 'ms_per_step')},
            roofline_factor=factor_roofline(c4_res, c4), roofline_solve=solve_roofline(c4_res, c4))
        del c4
        # the same step with the shock-transport terms (Eqs. a90-a99) on the imposed shock profile
        shock = run_path(M, torch, shock_workload(n_gpus, rank), M.MGFLD_MIXED, args.steps, args.warmup, barrier)
        ms_shock = max_over_ranks(shock['ms']) / args.steps
        # the paper-literal n+1 flux coefficients of Eq. a59, formed again at every outer iterate
        lit = run_path(M, torch, inp, M.MGFLD_MIXED, args.steps, args.warmup, barrier, coef_iterate=True)
        ms_lit = max_over_ranks(lit['ms']) / args.steps
        extra['shock_path'] = dict(
            path_summary(shock, inp, M.MGFLD_MIXED, ws, ms_shock, ups, n_rays_rank),
            dtype='f32 factor + f64 residual/update',
            workload='the same rays with the imposed accretion-shock velocity (zero inside r_s - 15 km, -0.2c at '
                     'r_s ~ 150 km, -0.2c (r_s/r)^2 outside) and a synthetic flux factor; shock terms of Eqs. '
                     'a91-a99 at the shock',
            dominant_category=max(shock['prof'], key=lambda c: shock['prof'][c]['ms']))
        extra['coef_iterate_path'] = dict(
            path_summary(lit, inp, M.MGFLD_MIXED, ws, ms_lit, ups, n_rays_rank),
            dtype='f32 factor + f64 residual/update',
            workload='the same rays with the flux coefficients of Eq. a59 (mean free path, limiter, '
                     'neutrinosphere) formed again at every outer iterate',
            dominant_category=max(lit['prof'], key=lambda c: lit['prof'][c]['ms']))
        # the pair process (Eq. d14 with the angular correction of Eqs. d16-d22): coupled (nu, nubar)
        # systems of 2 n_e x 2 n_e zone blocks
        pr = run_path(M, torch, pair_workload(n_gpus, rank), M.MGFLD_MIXED, args.steps, args.warmup, barrier)
        ms_pair = max_over_ranks(pr['ms']) / args.steps
        extra['pair_path'] = dict(
            path_summary(pr, inp, M.MGFLD_MIXED, ws, ms_pair, ups, n_rays_rank, rooflines=False),
            dtype='f32 factor + f64 residual/update',
            workload='the same rays with the synthetic pair process at the NES scale (pair_coef = 1e-41 rho) '
                     'and its angular correction (pair_chi, the synthetic flux factor): coupled (nu, nubar) '
                     'systems of 40 x 40 zone blocks',
            dominant_category=max(pr['prof'], key=lambda c: pr['prof'][c]['ms']))
        del pr
        extra['stress_lapse'] = stress_lapse_run(M, torch, inp, args.steps, args.warmup)
        extra['energy_advection'] = energy_advection_run(
            M, torch, n_gpus, rank, args.steps, args.warmup,
            cpu_rays=0 if (rank != 0 or args.no_cpu_baseline) else 64)
    cpu = None
    if pool is not None:
        cpu = oracle_pool_sample(pool, inp)
        cpu.pop('wall_s')
        one = oracle_sample(inp, 4)
        cpu['single_core'] = dict(value=one['value'], cores=one['cores'], sample=one['sample'])
        if not args.no_extra:
            # the oracle on 2 rays per core of the other step lines (rays are independent)
            c = oracle_pool_sample(pool, shock_workload(n_gpus, rank), rays_per_core=1)
            c.pop('wall_s')
            extra['shock_path']['cpu_baseline'] = c
            c = oracle_pool_sample(pool, inp, rays_per_core=1, coef_iterate=True)
            c.pop('wall_s')
            extra['coef_iterate_path']['cpu_baseline'] = c
            c = oracle_pool_sample(pool, pair_workload(n_gpus, rank), rays_per_core=1)
            c.pop('wall_s')
            extra['pair_path']['cpu_baseline'] = c
            extra['stress_lapse']['cpu_baseline'] = stress_oracle_sample(inp, 16)
            c4 = problems.make_problem(C4_ID)
            c = oracle_pool_sample(pool, c4, rays_per_core=1)
            c.pop('wall_s')
            extra['config4']['cpu_baseline'] = c
            del c4
        pool.close()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=n_gpus, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms_mixed, higher_is_better=True, scaling='weak', vs_baseline=None,
        dtype='f32 factor + f64 residual/update', data='synthetic',
        config=dict(workload='2d ' + workload_name(inp, args.steps) + ' per GPU (the 2D mixed-precision '
                             'configuration, its seeds)',
                    n_ray_per_gpu=n_rays_rank, n_r=inp['psi0'].shape[2], n_e=inp['psi0'].shape[3], n_s=4,
                    precision='mixed',
                    l2='working set %.1f GB per GPU, larger than the 129 MB L2 (no flush needed)' % mixed['ws_gb'],
                    outer_iterations_per_step=mixed['max_iters'],
                    factorizations_per_ray_step=mixed['nfact'] / (n_rays_rank * args.steps)),
        roofline=roof, roofline_factor=factor_roofline(mixed, inp), roofline_solve=solve_roofline(mixed, inp),
        roofline_step=step_roofline(mixed, inp, M.MGFLD_MIXED),
        cpu_baseline=cpu, clocks=mixed['clocks'],
        e2e=dict(value=job_throughput(ups, ws, e2e_ms), unit=UNIT, h2d_bytes_per_step=e2e['h2d'],
                 d2h_bytes_per_step=e2e['d2h']),
        gpu_launches=launches,
        timing='mgfld_step as a user calls it: asynchronous on the stream (one CUDA graph per step, its outer '
               'iteration a device-side while loop), no host synchronisation inside the timed loop; kernel_ms and '
               'the rooflines from a second pass of the same number of steps with per-category CUDA events',
        profiled_ms_per_step=mixed['profiled_ms'] / args.steps,
        kernel_ms={k: v['ms'] for k, v in mixed['prof'].items()},
        iterations_histogram=mixed['iters_hist'],
        fp64_path=path_summary(fp64, inp, M.MGFLD_FP64, ws, ms_fp64, ups, n_rays_rank, dtype='f64',
                               iteration='modified Newton, refactor when a correction shrinks by less than 10x'),
        fp64_newton_path=path_summary(newton, inp, M.MGFLD_FP64, ws, ms_newton, ups, n_rays_rank, dtype='f64',
                                      iteration='Newton, new factors every iteration'),
        mixed_over_fp64=value / value64,
        **extra)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == '__main__':
    sys.exit(main())
