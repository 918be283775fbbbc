"""Benchmark of the implicit MGFLD transport step on synthetic post-bounce profiles.

Workload: 256 rays (2D, per-ray angular perturbations) x 512 radial zones x 20
energy groups x 4 species, dt = 1e-6 s, outer tolerance 1e-10 (tolmin_psi = 1):
the 2D ray-by-ray configuration.  A "step" is one implicit transport step of
every ray (mgfld_step).  Metric: zone*group*species updates per second
(n_ray * n_r * n_e * 4 per step / time), for the mixed-precision path (FP32
block factorisation, FP64 residual refinement) with the plain FP64 path on the
same inputs reported beside it.

Under torchrun each rank steps its own 256 rays of a larger 2D ray set (rays are
independent: no collective on the data path); `value` is the total over ranks.
`--impl reference` times the CPU oracle on host cores instead.
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

RAYS_PER_RANK = 256
CONFIG_ID = 2
TOL = 1e-10
METRIC = 'MGFLD step zone*group*species updates/s (mixed FP32-factor/FP64-refined at 1e-10; FP64 path beside)'
UNIT = 'updates/s'
FP64_FLOP_PER_CLK_SM = 4.0      # 2 DFMA lanes per clock per SM (1.25 TFLOP/s nominal at 2.07 GHz x 152 SMs)
FP32_FLOP_PER_CLK_SM = 256.0    # 128 FFMA lanes per clock per SM
N_SM = 152


def _measured_hbm_gbs():
    """The measured HBM copy bandwidth of this machine's GPUs, else the recorded fallback."""
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            return float(json.load(f)['hbm_gbs'])
    except (OSError, ValueError, KeyError):
        return 6800.0


PEAK_HBM_GBS = _measured_hbm_gbs()
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


def job_throughput(updates_per_rank_step, world, ms_per_step_max):
    """Whole-job updates/s: every rank's rays over the slowest rank's time per step."""
    return updates_per_rank_step * world / (ms_per_step_max * 1e-3)


def updates_per_step(inp):
    n_ray, n_s, n_r, n_e = inp['psi0'].shape
    return n_ray * n_s * n_r * n_e


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
             coef_iterate=False):
    st = M.Stepper(inp, precision, tol=TOL, max_iter=60, refactor_ratio=refactor_ratio, coef_iterate=coef_iterate)
    if clocks:
        clocks.start()
    psi, ye, T = st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    stream = torch.cuda.current_stream()
    prof = (ctypes.c_double * 12)()
    nfact = torch.zeros_like(st.report['factorizations'])
    iters = torch.zeros_like(st.report['iters'])
    for wi in range(warmup):
        # The warm-up runs exactly what the timed loop runs (profiling events, report sums),
        # so that one-time costs (lazy module loading, event creation) stay outside the timing.
        st.opts.profile = ctypes.cast(prof, ctypes.c_void_p) if wi == warmup - 1 else None
        rc = st.step(psi, ye, T)
        assert rc == M.MGFLD_OK, M.status_str(rc)
        nfact += st.report['factorizations']
        iters += st.report['iters']
    torch.cuda.synchronize()
    for c in range(12):
        prof[c] = 0.0
    nfact.zero_()
    iters.zero_()
    st.opts.profile = ctypes.cast(prof, ctypes.c_void_p)
    barrier()
    torch.cuda.synchronize()
    t_start = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rc = st.step(psi, ye, T)
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
    st.opts.profile = None
    prof = {name: dict(ms=prof[2 * c], launches=int(prof[2 * c + 1])) for c, name in enumerate(M.PROF_NAMES)}
    return dict(ms=ms, prof=prof, nfact=int(nfact.sum()), iters=int(iters.sum()),
                max_iters=int(st.report['iters'].max()), clocks=clk, stepper=st,
                state=(psi, ye, T))


def algorithmic_work(inp, kernel, nfact, iters, precision):
    """Algorithmic flop count over the timed steps for one kernel category.

    factor: per (zone, system) factorisation, N^3 FMAs of in-place Gauss-Jordan plus
    2 N^2 for the diagonal Schur scaling: 2 N^3 + 2 N^2 flops (FP64 or FP32).
    assemble (FP64 pipe only): per (zone, system, iteration) residual, two length-N NES sums
    per row (4 N^2) + 16 N of transport/absorption terms; with a fresh FP64 Jacobian one FMA
    per entry (2 N^2).  The mixed path's Jacobian rows are FP32 and are not counted."""
    n_ray, n_s, n_r, n = inp['psi0'].shape
    if kernel == 'factor':
        per = 2.0 * n**3 + 2.0 * n**2
        return per * n_s * n_r * nfact
    if kernel == 'assemble':
        per_res = 4.0 * n**2 + 16.0 * n
        per_jac = 2.0 * n**2 if precision == 0 else 0.0
        return n_s * n_r * (per_res * iters + per_jac * nfact)
    raise ValueError(kernel)


def roofline_for(res, inp, precision, clk):
    prof = res['prof']
    dom = max(('assemble', 'factor'), key=lambda k: prof[k]['ms'])
    flops = algorithmic_work(inp, dom, res['nfact'], res['iters'], precision)
    achieved = flops / (prof[dom]['ms'] * 1e-3) / 1e12
    fp32 = dom == 'factor' and precision == 1
    per_clk = FP32_FLOP_PER_CLK_SM if fp32 else FP64_FLOP_PER_CLK_SM
    peak = per_clk * N_SM * 2.070e9 / 1e12
    launches = max(prof[dom]['launches'], 1)
    kname = {'factor': 'k_factor', 'assemble': 'k_assemble'}[dom]
    tr = traffic_record(kname + ('_f32' if fp32 else ''))
    traffic = None
    if tr is not None:
        units_per_launch = (res['nfact'] if dom == 'factor' else res['iters']) * inp['psi0'].shape[1] / launches
        traffic = tr['bytes'] / tr['units'] * units_per_launch
    return dict(bound='alu', kernel=kname, pipe='fp32' if fp32 else 'fp64', achieved=achieved, peak=peak,
                unit='TFLOP/s', frac=achieved / peak, traffic=traffic,
                peak_source='derived: %g flop/clk/SM x 152 SMs x 2070 MHz max SM clock' % per_clk,
                kernel_ms_per_launch=prof[dom]['ms'] / launches, kernel_share=prof[dom]['ms'] / res['ms'])


def solve_roofline(res, inp):
    """HBM roofline of the mixed path's FP32 substitution (k_sysmax + k_solve_tma per solve).

    Bytes per (zone, system) and solve: every FP32 inverse block read by the inward and by the
    outward sweep (2 N^2 x 4 B; the 839 MB of blocks of the 256-ray workload do not stay in the
    129 MB L2 between the sweeps), plus the vectors: rhs read (8 N), its FP32 copy written and
    read (2 x 4 N), the two couplings (2 x 4 N), the forward result written and read (2 x 4 N)
    and x written (8 N)."""
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
                frac=achieved / PEAK_HBM_GBS, traffic=traffic, peak_source='measured copy bandwidth (of measured)',
                bytes_per_zone_system=per_unit, kernel_ms_per_launch=prof['ms'] / max(solves, 1),
                kernel_share=prof['ms'] / res['ms'])


def e2e_run(M, torch, inp, precision, steps):
    """Same metric through the public API from pinned HOST buffers: every step uploads
    that step's inputs (matter, opacities, NES scale, grid, state), runs mgfld_step and
    reads the new state back.  The problem arrays of step s+1 are uploaded on a second
    stream into a second device copy while step s runs (double buffering); the state goes
    host -> device -> host on the compute stream, in order."""
    st = M.Stepper(inp, precision, tol=TOL, max_iter=60)
    prob = inp['problem']
    names = ('r_edge', 'rho', 'kappa_abs', 'kappa_scat', 'nes_coef')
    host = {k: torch.from_numpy(np.ascontiguousarray(prob[k], dtype=np.float64)).pin_memory() for k in names}
    hs = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
          for a in (inp['psi0'], inp['ye0'], inp['T0'])]
    dev = [torch.empty_like(h, device='cuda') for h in hs]
    out = [torch.empty_like(h).pin_memory() for h in hs]
    bufs = [st.prob, M.DeviceProblem(prob)]
    h2d = sum(v.numel() * 8 for v in host.values()) + sum(h.numel() * 8 for h in hs)
    d2h = sum(h.numel() * 8 for h in hs)
    stream = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]     # buffer b uploaded
    free = [torch.cuda.Event(), torch.cuda.Event()]      # buffer b no longer read by a step

    def upload(b):
        with torch.cuda.stream(copy):
            for k in names:
                bufs[b].t[k].copy_(host[k], non_blocking=True)
            ready[b].record(copy)

    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy.wait_event(e0)
    upload(0)
    for s in range(steps):
        b = s % 2
        if s + 1 < steps:
            if s >= 1:
                copy.wait_event(free[1 - b])
            upload(1 - b)
        stream.wait_event(ready[b])
        st.prob = bufs[b]
        src = hs if s == 0 else out
        for d, h in zip(dev, src):
            d.copy_(h, non_blocking=True)
        rc = st.step(*dev)
        assert rc == M.MGFLD_OK, M.status_str(rc)
        free[b].record(stream)
        for o, d in zip(out, dev):
            o.copy_(d, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st.prob = bufs[0]
    return dict(ms=ms, h2d=h2d, d2h=d2h)


# ------------------------------------------------------------------------- CPU oracle

def oracle_sample(inp, n_rays, n_steps=1, **step_kw):
    """Time the CPU oracle, as it stands, on the first n_rays rays for n_steps steps."""
    from oracle import mgfld_oracle as O
    sub = problems.subset_rays(inp, slice(0, n_rays))
    c0, w0 = time.process_time(), time.perf_counter()
    O.run_steps(sub['problem'], sub['psi0'], sub['ye0'], sub['T0'], n_steps, **step_kw)
    wall = time.perf_counter() - w0
    cpu = time.process_time() - c0
    ups = updates_per_step(sub) * n_steps / wall
    return dict(value=ups, unit=UNIT, cores=max(1, int(round(cpu / wall))), kind='oracle',
                sample=f'{n_rays} of the 256 rays x {n_steps} implicit step(s), FP64 numpy/LAPACK, '
                       f'{wall:.1f} s wall', wall_s=wall)


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
                sample=f'{n_rays} of the 256 rays, one call, FP64 numpy, {wall:.2f} s wall')


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
    peak64 = FP64_FLOP_PER_CLK_SM * N_SM * 2.070e9 / 1e12
    # The kernel is bound by the FP64 pipe (divisions, square roots and the PPM arithmetic on
    # 24 B per update), not by HBM; both figures are reported, the FP64 one as the roofline.
    out = dict(metric='energy-advection updates/s', value=ups / (ms * 1e-3), unit=UNIT, ms_per_step=ms,
               steps=steps, warmup=warmup, dtype='f64',
               config=dict(workload=f'{n_ray} rays x {n_r} zones x {n_e} groups x {n_s} species, one step per '
                                    'launch, psi advanced in place',
                           l2='reads 168 MB (psi, eta1) and writes 84 MB per step, larger than the 129 MB L2'),
               roofline=dict(bound='alu', pipe='fp64', kernel='k_energy_advect', achieved=tfs, peak=peak64,
                             unit='TFLOP/s', frac=tfs / peak64, traffic=None,
                             flops_per_update=EADV_FLOPS_PER_UPDATE,
                             peak_source='derived: %g flop/clk/SM x 152 SMs x 2070 MHz max SM clock'
                                         % FP64_FLOP_PER_CLK_SM),
               roofline_hbm=dict(bound='hbm', achieved=gbs, peak=PEAK_HBM_GBS, unit='GB/s', frac=gbs / PEAK_HBM_GBS,
                                 bytes_per_update=24, peak_source='measured copy bandwidth (of measured)'))
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
    return dict(metric='stress-and-lapse updates/s', value=ups / (ms * 1e-3), unit=UNIT, ms_per_call=ms,
                steps=steps, warmup=warmup, dtype='f64', launches_per_call=9,
                note='one call = the 7 setup kernels of the transport step on the state, k_stress, k_lapse')


def reference_arm(args, n_gpus, rank):
    if rank != 0:
        return 0
    inp = workload(1, 0)
    rays = 4
    per_step = []
    for s in range(args.warmup + args.steps):
        r = oracle_sample(inp, rays)
        if s >= args.warmup:
            per_step.append(r['wall_s'])
    ms = 1e3 * float(np.mean(per_step))
    value = updates_per_step(problems.subset_rays(inp, slice(0, rays))) / (ms * 1e-3)
    line = dict(impl='reference', metric=METRIC, value=value, unit=UNIT, n_gpus=n_gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling='weak', vs_baseline=None,
                dtype='f64', data='synthetic',
                config=dict(workload='2d 256 rays x 512 zones x 20 groups x 4 species, dt 1e-6 s, tol 1e-10',
                            oracle_rays_per_step=rays),
                cpu_baseline=dict(value=value, unit=UNIT, cores=r['cores'], kind='oracle',
                                  sample=f'{rays} of the 256 rays, one implicit step per timed step'),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------- main

def profile_step(path, n_rays):
    """One implicit step of the first n_rays rays of the benchmark workload (FP64 Newton, the
    mixed path, the mixed path with the shock terms or with the flux coefficients formed at every
    outer iterate), two energy-advection steps, or one stress-and-lapse call, for ncu captures of
    single launches; exits non-zero on a failed step."""
    import torch
    from paper_1809_05608_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_1809_05608_gb300 import mgfld as M
    if path == 'eadv':
        inp = problems.make_energy_advection(CONFIG_ID, rays=slice(0, n_rays))
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
        inp = problems.make_problem(CONFIG_ID, rays=slice(0, n_rays))
        res = stress_lapse_run(M, torch, inp, 1, 1)
        print(f'profile step stress: {n_rays} rays, {res["ms_per_call"]:.3f} ms', flush=True)
        return 0
    if path == 'shock':
        inp = problems.make_shock_problem(CONFIG_ID, rays=slice(0, n_rays))
    else:
        inp = problems.make_problem(CONFIG_ID, rays=slice(0, n_rays))
    prec = M.MGFLD_FP64 if path == 'fp64' else M.MGFLD_MIXED
    st = M.Stepper(inp, prec, tol=TOL, max_iter=60, coef_iterate=path == 'coef')
    psi, ye, T = st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    rc = st.step(psi, ye, T)
    torch.cuda.synchronize()
    print(f'profile step {path}: {n_rays} rays, status {M.status_str(rc)}, '
          f'iterations {int(st.report["iters"].max())}', flush=True)
    return 0 if rc == M.MGFLD_OK else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=10)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='mgfld', choices=['mgfld', 'reference'])
    ap.add_argument('--oracle-rays', type=int, default=12)
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--profile-step', choices=['mixed', 'fp64', 'shock', 'coef', 'eadv', 'stress'],
                    help='profiling target: one implicit step of this path (shock: the mixed path with '
                         'the shock terms; coef: the mixed path with the flux coefficients formed at '
                         'every outer iterate; eadv: two energy-advection steps; stress: two stress-and-lapse '
                         'calls) on --rays rays, no timing')
    ap.add_argument('--rays', type=int, default=64)
    args = ap.parse_args()
    if args.profile_step:
        return profile_step(args.profile_step, args.rays)
    ws, rank, local = dist_info()
    n_gpus = max(args.gpus, ws)
    if args.impl == 'reference':
        return reference_arm(args, n_gpus, rank)

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
    ups = updates_per_step(inp)
    clocks = ClockSampler(local)
    mixed = run_path(M, torch, inp, M.MGFLD_MIXED, args.steps, args.warmup, barrier, clocks)
    # FP64 beside it: the same modified-Newton policy with FP64 factors (the like-for-like
    # baseline), and Newton with a new FP64 factorisation every iteration.
    fp64 = run_path(M, torch, inp, M.MGFLD_FP64, args.steps, args.warmup, barrier, refactor_ratio=0.1)
    newton = run_path(M, torch, inp, M.MGFLD_FP64, args.steps, args.warmup, barrier, refactor_ratio=0.0)
    ms_mixed = max_over_ranks(mixed['ms']) / args.steps
    ms_fp64 = max_over_ranks(fp64['ms']) / args.steps
    ms_newton = max_over_ranks(newton['ms']) / args.steps
    value = job_throughput(ups, ws, ms_mixed)
    value64 = job_throughput(ups, ws, ms_fp64)
    # the same step with the shock-transport terms (Eqs. a90-a99) on the imposed shock profile
    shock = run_path(M, torch, shock_workload(n_gpus, rank), M.MGFLD_MIXED, args.steps, args.warmup, barrier)
    ms_shock = max_over_ranks(shock['ms']) / args.steps
    # the paper-literal n+1 flux coefficients of Eq. a59, formed again at every outer iterate
    lit = run_path(M, torch, inp, M.MGFLD_MIXED, args.steps, args.warmup, barrier, coef_iterate=True)
    ms_lit = max_over_ranks(lit['ms']) / args.steps
    e2e = e2e_run(M, torch, inp, M.MGFLD_MIXED, args.steps)
    e2e_ms = max_over_ranks(e2e['ms']) / args.steps
    roof = roofline_for(mixed, inp, M.MGFLD_MIXED, mixed['clocks'])
    roof64 = roofline_for(fp64, inp, M.MGFLD_FP64, None)
    roof_newton = roofline_for(newton, inp, M.MGFLD_FP64, None)
    launches = sum(v['launches'] for v in mixed['prof'].values())
    stress = stress_lapse_run(M, torch, inp, args.steps, args.warmup)
    eadv = energy_advection_run(M, torch, n_gpus, rank, args.steps, args.warmup,
                                cpu_rays=0 if (rank != 0 or args.no_cpu_baseline) else 64)
    cpu = cpu_shock = cpu_lit = cpu_stress = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_sample(inp, args.oracle_rays)
        cpu.pop('wall_s')
        # the oracle on 2-ray samples of the other step lines (rays are independent)
        cpu_shock = oracle_sample(shock_workload(n_gpus, rank), 2)
        cpu_shock.pop('wall_s')
        cpu_lit = oracle_sample(inp, 2, coef_iterate=True)
        cpu_lit.pop('wall_s')
        cpu_stress = stress_oracle_sample(inp, 16)
    if rank != 0:
        return 0
    work_gb = (mixed['stepper'].ws.numel() + sum(t.numel() * 8 for t in mixed['stepper'].prob.t.values()
                                                 if t is not None)) / 1e9
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=n_gpus, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms_mixed, higher_is_better=True, scaling='weak', vs_baseline=None,
        dtype='f32 factor + f64 residual/update', data='synthetic',
        config=dict(workload='2d 256 rays x 512 zones x 20 groups x 4 species per GPU, dt 1e-6 s, tol 1e-10',
                    n_ray_per_gpu=RAYS_PER_RANK, n_r=512, n_e=20, n_s=4, precision='mixed',
                    l2='working set %.1f GB per GPU, larger than the 129 MB L2 (no flush needed)' % work_gb,
                    outer_iterations_per_step=mixed['max_iters'],
                    factorizations_per_ray_step=mixed['nfact'] / (RAYS_PER_RANK * args.steps)),
        roofline=roof, roofline_solve=solve_roofline(mixed, inp), cpu_baseline=cpu, clocks=mixed['clocks'],
        e2e=dict(value=job_throughput(ups, ws, e2e_ms), unit=UNIT, h2d_bytes_per_step=e2e['h2d'],
                 d2h_bytes_per_step=e2e['d2h']),
        gpu_launches=launches,
        kernel_ms={k: v['ms'] for k, v in mixed['prof'].items()},
        fp64_path=dict(value=value64, unit=UNIT, ms_per_step=ms_fp64, roofline=roof64, dtype='f64',
                       iteration='modified Newton, refactor when a correction shrinks by less than 10x',
                       kernel_ms={k: v['ms'] for k, v in fp64['prof'].items()},
                       outer_iterations_per_step=fp64['max_iters'],
                       factorizations_per_ray_step=fp64['nfact'] / (RAYS_PER_RANK * args.steps),
                       gpu_launches=sum(v['launches'] for v in fp64['prof'].values())),
        fp64_newton_path=dict(value=job_throughput(ups, ws, ms_newton), unit=UNIT, ms_per_step=ms_newton,
                              roofline=roof_newton, dtype='f64', iteration='Newton, new factors every iteration',
                              kernel_ms={k: v['ms'] for k, v in newton['prof'].items()},
                              outer_iterations_per_step=newton['max_iters'],
                              factorizations_per_ray_step=newton['nfact'] / (RAYS_PER_RANK * args.steps)),
        shock_path=dict(value=job_throughput(ups, ws, ms_shock), unit=UNIT, ms_per_step=ms_shock,
                        dtype='f32 factor + f64 residual/update',
                        workload='the same rays with the imposed accretion-shock velocity (zero inside '
                                 'r_s - 15 km, -0.2c at r_s ~ 150 km, -0.2c (r_s/r)^2 outside) and a '
                                 'synthetic flux factor; shock terms of Eqs. a91-a99 at the shock',
                        kernel_ms={k: v['ms'] for k, v in shock['prof'].items()},
                        roofline=roofline_for(shock, inp, M.MGFLD_MIXED, None), cpu_baseline=cpu_shock,
                        dominant_category=max(shock['prof'], key=lambda c: shock['prof'][c]['ms']),
                        outer_iterations_per_step=shock['max_iters'],
                        gpu_launches=sum(v['launches'] for v in shock['prof'].values())),
        coef_iterate_path=dict(value=job_throughput(ups, ws, ms_lit), unit=UNIT, ms_per_step=ms_lit,
                               dtype='f32 factor + f64 residual/update',
                               workload='the same rays with the flux coefficients of Eq. a59 (mean free path, '
                                        'limiter, neutrinosphere) formed again at every outer iterate',
                               kernel_ms={k: v['ms'] for k, v in lit['prof'].items()},
                               roofline=roofline_for(lit, inp, M.MGFLD_MIXED, None), cpu_baseline=cpu_lit,
                               dominant_category=max(lit['prof'], key=lambda c: lit['prof'][c]['ms']),
                               outer_iterations_per_step=lit['max_iters'],
                               gpu_launches=sum(v['launches'] for v in lit['prof'].values())),
        mixed_over_fp64=value / value64,
        energy_advection=eadv,
        stress_lapse=dict(stress, cpu_baseline=cpu_stress))
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == '__main__':
    sys.exit(main())
