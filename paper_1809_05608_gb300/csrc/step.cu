// Outer iteration of the implicit transport step and the C ABI (include/mgfld.h).
//
// Per outer iteration (Eq. a62aa) and per still-active ray:
//   1. residual (and, when the ray needs one, a fresh Jacobian) of Eq. a58 at the iterate;
//   2. block-Thomas factorisation (every iteration in FP64; in MIXED only when the
//      correction stopped contracting fast, the FP32 factors being reused otherwise, so
//      that the FP64 residual drives an iterative refinement);
//   3. forward/back substitution for the correction of psi;
//   4. psi += correction; one Newton step of the zone-local Ye equation (Eq. a62a) at the
//      new psi (the Ye column of Eq. a62ae is taken by outer block Gauss-Seidel, which
//      converges to the same root); the convergence test of Eq. a62ab.
// After convergence: Eq. a62b for the internal energy, T from the EoS, and the lepton and
// energy ledgers of Eqs. a60-a62.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "mgfld_internal.cuh"

namespace mgfld {

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

Layout make_layout(int n_ray, int n_r, int n, int precision, int pair) {
  Layout L{};
  L.mixed = precision == MGFLD_MIXED;
  L.pair = pair != 0;
  const size_t R = (size_t)n_ray, Z = R * n_r, F = Z * NS * n, B = F * n;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.groups = take(sizeof(double) * 3 * MAX_NE);
  L.phout = take(sizeof(double) * Z * n * n);
  L.phin = take(sizeof(double) * Z * n * n);
  L.phd = take(precision == MGFLD_MIXED ? 0 : sizeof(double) * Z * n * n);
  L.rsum = take(sizeof(double) * Z * n);
  L.phin32 = take(precision == MGFLD_MIXED ? sizeof(float) * Z * n * n : 0);
  L.phd32 = take(precision == MGFLD_MIXED ? sizeof(float) * Z * n * n : 0);
  L.nesff = take(precision == MGFLD_MIXED ? sizeof(float4) * Z * n * n : 0);
  L.nessc = take(precision == MGFLD_MIXED ? sizeof(int2) * Z * n : 0);
  L.lam = take(sizeof(double) * F);
  L.alpha = take(sizeof(double) * F);
  L.ghost = take(sizeof(double) * R * NS * n);
  L.rnu = take(sizeof(double) * R * NS * n);
  L.jbuf = take(sizeof(double) * F);
  L.psi_n = take(sizeof(double) * F);
  L.ye_n = take(sizeof(double) * Z);
  L.e_n = take(sizeof(double) * Z);
  L.zone = take(sizeof(double) * Z * ZC_N);
  L.src = take(sizeof(double) * F);
  L.shock = take(sizeof(double) * F);
  L.cdiag = take(sizeof(double) * F);
  L.cup = take(sizeof(double) * F);
  L.clow = take(sizeof(double) * F);
  L.cb = take(sizeof(double) * F);
  // pair systems: per ray two (2n x 2n) blocks per zone, twice the four species' n x n blocks
  const size_t Bs = pair ? 2 * B : B;
  L.diag = take((precision == MGFLD_MIXED ? sizeof(float) : sizeof(double)) * Bs);
  L.lower = take(sizeof(double) * F);
  L.upper = take(sizeof(double) * F);
  L.rhs = take(sizeof(double) * F);
  L.x = take(sizeof(double) * F);
  L.dinv = take((precision == MGFLD_MIXED ? sizeof(float) : sizeof(double)) * Bs);
  L.zled = take(sizeof(double) * Z * 8);
  L.sscale = take(sizeof(int) * R * NS);
  L.lower32 = take(precision == MGFLD_MIXED ? sizeof(float) * F : 0);
  L.upper32 = take(precision == MGFLD_MIXED ? sizeof(float) * F : 0);
  L.g32 = take(precision == MGFLD_MIXED ? sizeof(float) * F : 0);
  L.rhs32 = take(precision == MGFLD_MIXED ? sizeof(float) * F : 0);
  L.kinv = take(sizeof(double) * F);
  L.viol = take(sizeof(unsigned long long) * R);
  L.vprev = take(sizeof(double) * R);
  L.active = take(sizeof(int) * R);
  L.iters = take(sizeof(int) * R);
  L.status = take(sizeof(int) * R);
  L.refac = take(sizeof(int) * R);
  L.nfact = take(sizeof(int) * R);
  L.nanflag = take(sizeof(int) * R);
  L.list_act = take(sizeof(int) * R);
  L.list_ref = take(sizeof(int) * R);
  L.counters = take(sizeof(int) * 8);
  L.pmake = take(pair ? sizeof(double) * Z * n * n : 0);
  L.pmsum = take(pair ? sizeof(double) * Z * n : 0);
  L.pkill = take(pair ? sizeof(double) * Z * NS * n * n : 0);
  // Setup-only arrays share storage with buffers that are first written after the setup has
  // consumed them: sqrt(lambda) (read by the limiter kernel) lives in rhs, and (FP64) the NES
  // sums at psi^n (read by the first residual, before the first solve or the final sources) in
  // x and src.
  L.slam = L.rhs;
  if (precision == MGFLD_MIXED) {
    // MIXED keeps the NES sums of each ray's latest residual for the final sources.
    L.g0 = take(sizeof(double) * F);
    L.l0 = take(sizeof(double) * F);
  } else {
    L.g0 = L.src;
    L.l0 = L.x;
  }
  L.total = off;
  return L;
}

Ws resolve(void *base, const Layout &L) {
  char *b = (char *)base;
  Ws w;
  w.E = (double *)(b + L.groups);
  w.W = w.E + MAX_NE;
  w.WE = w.W + MAX_NE;
  w.phout = (double *)(b + L.phout);
  w.phin = (double *)(b + L.phin);
  w.phd = L.mixed ? nullptr : (double *)(b + L.phd);
  w.rsum = (double *)(b + L.rsum);
  w.phin32 = L.mixed ? (float *)(b + L.phin32) : nullptr;
  w.phd32 = L.mixed ? (float *)(b + L.phd32) : nullptr;
  w.nesff = L.mixed ? (float4 *)(b + L.nesff) : nullptr;
  w.nessc = L.mixed ? (int2 *)(b + L.nessc) : nullptr;
  w.lam = (double *)(b + L.lam);
  w.slam = (double *)(b + L.slam);
  w.g0 = (double *)(b + L.g0);
  w.l0 = (double *)(b + L.l0);
  w.alpha = (double *)(b + L.alpha);
  w.ghost = (double *)(b + L.ghost);
  w.rnu = (double *)(b + L.rnu);
  w.jbuf = (double *)(b + L.jbuf);
  w.psi_n = (double *)(b + L.psi_n);
  w.ye_n = (double *)(b + L.ye_n);
  w.e_n = (double *)(b + L.e_n);
  w.zone = (double *)(b + L.zone);
  w.src = (double *)(b + L.src);
  w.shock = (double *)(b + L.shock);
  w.cdiag = (double *)(b + L.cdiag);
  w.cup = (double *)(b + L.cup);
  w.clow = (double *)(b + L.clow);
  w.cb = (double *)(b + L.cb);
  w.pmake = L.pair ? (double *)(b + L.pmake) : nullptr;
  w.pmsum = L.pair ? (double *)(b + L.pmsum) : nullptr;
  w.pkill = L.pair ? (double *)(b + L.pkill) : nullptr;
  w.lim = nullptr;
  w.jl = w.jr = nullptr;       // set by mgfld_step when the coefficients follow the iterate
  w.diag = (double *)(b + L.diag);
  w.lower = (double *)(b + L.lower);
  w.upper = (double *)(b + L.upper);
  w.rhs = (double *)(b + L.rhs);
  w.x = (double *)(b + L.x);
  w.dinv = (void *)(b + L.dinv);
  w.zled = (double *)(b + L.zled);
  w.sscale = (int *)(b + L.sscale);
  w.lower32 = L.mixed ? (float *)(b + L.lower32) : nullptr;
  w.upper32 = L.mixed ? (float *)(b + L.upper32) : nullptr;
  w.g32 = L.mixed ? (float *)(b + L.g32) : nullptr;
  w.rhs32 = L.mixed ? (float *)(b + L.rhs32) : nullptr;
  w.kinv = (double *)(b + L.kinv);
  w.viol = (unsigned long long *)(b + L.viol);
  w.vprev = (double *)(b + L.vprev);
  w.active = (int *)(b + L.active);
  w.iters = (int *)(b + L.iters);
  w.status = (int *)(b + L.status);
  w.refac = (int *)(b + L.refac);
  w.nfact = (int *)(b + L.nfact);
  w.nanflag = (int *)(b + L.nanflag);
  w.list_act = (int *)(b + L.list_act);
  w.list_ref = (int *)(b + L.list_ref);
  w.counters = (int *)(b + L.counters);
  return w;
}

struct Tol {
  double tol, tolmin, tol_ye, tolmin_ye, refactor_ratio;
  int max_iter, mixed, chord;   // chord: reuse factors while the iteration contracts fast enough
  float tolm, tolm_ye;      // tol = tolm 2^tole (for tol_ratio)
  int tole, tole_ye;
};

__global__ void k_init(int n_ray, Ws w) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_ray) return;
  w.active[r] = 1;
  w.iters[r] = 0;
  w.status[r] = MGFLD_OK;
  w.refac[r] = 1;
  w.nfact[r] = 1;
  w.nanflag[r] = 0;
  w.viol[r] = 0ull;
  w.vprev[r] = INFINITY;
  w.list_act[r] = r;
  w.list_ref[r] = r;
}

// Largest violation ratio of a warp's lanes reported once per ray (lanes of one warp may
// belong to two rays at a boundary, then each lane reports for itself).  Ratios are
// non-negative floats, so their bit patterns order like their values.
__device__ inline void report_violation(Ws &w, int ray, float viol) {
  const unsigned full = 0xffffffffu;
  const int ray0 = __shfl_sync(full, ray, 0);
  if (__all_sync(full, ray == ray0)) {
    for (int off = 16; off > 0; off >>= 1) viol = fmaxf(viol, __shfl_down_sync(full, viol, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&w.viol[ray], (unsigned long long)__float_as_uint(viol));
  } else {
    atomicMax(&w.viol[ray], (unsigned long long)__float_as_uint(viol));
  }
}

// The same for a whole block (every thread of the block calls it): one atomic per block when
// the block lies in one ray, per warp otherwise.
__device__ inline void report_violation_block(Ws &w, int ray, float viol) {
  __shared__ float wmax[32];
  __shared__ int wray[32];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const int ray0 = __shfl_sync(full, ray, 0);
  const bool one = __all_sync(full, ray == ray0);
  if (one) {
    for (int off = 16; off > 0; off >>= 1) viol = fmaxf(viol, __shfl_down_sync(full, viol, off));
  } else {
    atomicMax(&w.viol[ray], (unsigned long long)__float_as_uint(viol));
  }
  if (lane == 0) {
    wmax[wid] = one ? viol : 0.f;
    wray[wid] = one ? ray : -1;
  }
  __syncthreads();
  if (wid == 0) {
    const float v = lane < nw ? wmax[lane] : 0.f;
    const int rr = lane < nw ? wray[lane] : wray[0];
    const bool same = __all_sync(full, rr == wray[0]) && wray[0] >= 0;
    if (same) {
      float m = v;
      for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(full, m, off));
      if (lane == 0) atomicMax(&w.viol[rr], (unsigned long long)__float_as_uint(m));
    } else if (lane < nw && rr >= 0) {
      atomicMax(&w.viol[rr], (unsigned long long)__float_as_uint(v));
    }
  }
}

// psi += dpsi (Eq. a62aa) and the per-element convergence ratio |d psi| / (tol max(|psi|, tolmin))
// of Eq. a62ab, one thread per (ray, q, i, k) of the active rays.  All 32 lanes of a warp reach
// the reduction (out-of-range lanes carry ratio 0).
__global__ void k_update_psi(Prob p, Ws w, Tol tl, double *__restrict__ psi, const int *__restrict__ list,
                             int n_list, const int *__restrict__ n_dev) {
  const unsigned per_ray = (unsigned)(NS * p.n_r * p.n);
  const unsigned total = (unsigned)listed(n_list, n_dev) * per_ray;
  if (blockIdx.x * blockDim.x >= total) return;          // the whole block
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = t < total;
  const unsigned rl = t / per_ray;
  const int ray = in ? list[rl] : list[0];
  float viol = 0.f;
  if (in) {
    const unsigned local = t - rl * per_ray;
    const size_t g = (size_t)ray * per_ray + local;
    size_t gx = g;
    if (p.pair) {
      // the correction of the coupled pair systems, [ray][pair][zone][2 n]
      const unsigned zq = local / (unsigned)p.n, k = local - zq * p.n;
      const unsigned q = zq / (unsigned)p.n_r, i = zq - q * p.n_r;
      gx = (((size_t)ray * 2 + (q >> 1)) * p.n_r + i) * (2 * p.n) + (q & 1) * p.n + k;
    }
    const double d = w.x[gx];
    const double v = psi[g] + d;
    psi[g] = v;
    // |d| / max(|v|, tolmin) and the finiteness test on the bit patterns (non-negative doubles
    // order as their integer patterns), so the FP64 pipe only takes the addition
    const long long ad = __double_as_longlong(d) & 0x7fffffffffffffffll;
    const long long av = __double_as_longlong(v) & 0x7fffffffffffffffll;
    const long long tm = __double_as_longlong(tl.tolmin);
    viol = tol_ratio_bits(ad, av > tm ? av : tm, tl.tolm, tl.tole);
    if (av >= 0x7ff0000000000000ll) {
      atomicExch(&w.nanflag[ray], 1);
      viol = INFINITY;
    }
  }
  report_violation_block(w, ray, viol);
}

// The same for two consecutive elements per thread (no pair process, an even group count, 16-byte
// aligned psi): the rows read and written 16 bytes at a time.
__device__ inline float psi_ratio(double d, double v, const Tol &tl, bool &bad) {
  const long long ad = __double_as_longlong(d) & 0x7fffffffffffffffll;
  const long long av = __double_as_longlong(v) & 0x7fffffffffffffffll;
  const long long tm = __double_as_longlong(tl.tolmin);
  bad = bad || av >= 0x7ff0000000000000ll;
  return tol_ratio_bits(ad, av > tm ? av : tm, tl.tolm, tl.tole);
}
__global__ void k_update_psi2(Prob p, Ws w, Tol tl, double *__restrict__ psi, const int *__restrict__ list,
                              int n_list, const int *__restrict__ n_dev) {
  const unsigned per_ray2 = (unsigned)(NS * p.n_r * p.n) / 2;
  const unsigned total = (unsigned)listed(n_list, n_dev) * per_ray2;
  if (blockIdx.x * blockDim.x >= total) return;          // the whole block
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = t < total;
  const unsigned rl = t / per_ray2;
  const int ray = in ? list[rl] : list[0];
  float viol = 0.f;
  if (in) {
    const size_t g = ((size_t)ray * per_ray2 + (t - rl * per_ray2)) * 2;
    const double2 d = *reinterpret_cast<const double2 *>(w.x + g);
    double2 v = *reinterpret_cast<const double2 *>(psi + g);
    v.x += d.x;
    v.y += d.y;
    *reinterpret_cast<double2 *>(psi + g) = v;
    bool bad = false;
    viol = fmaxf(psi_ratio(d.x, v.x, tl, bad), psi_ratio(d.y, v.y, tl, bad));
    if (bad) {
      atomicExch(&w.nanflag[ray], 1);
      viol = INFINITY;
    }
  }
  report_violation_block(w, ray, viol);
}

// One Newton step of the zone-local Ye equation (Eq. a62a) at the updated psi, with T held at
// T^n (Sec. "Lagrangian Transport Step"), then the nu_e / nubar_e emissivities at the new Ye.
// A change dmu of the chemical potential rescales j = kappa_a e^{(mu - eps)/T} by e^{dmu/T},
// one exponential per species (direct evaluation where the exponent cap is involved).  The cap
// is tested once per species at the lowest group energy, where mu - eps is largest: in the
// usual case no group reaches it and the per-group sums share their products,
//   sum w j (1 - psi) - sum w kappa psi  and  sum w j (1 - psi)  (the Ye derivative).
__global__ void k_update_ye(Prob p, Ws w, Tol tl, const double *__restrict__ psi, double *__restrict__ ye,
                            const double *__restrict__ T, const int *__restrict__ list, int n_list,
                            const int *__restrict__ n_dev) {
  const int n = p.n;
  const unsigned total = (unsigned)(listed(n_list, n_dev) * p.n_r);
  if (blockIdx.x * blockDim.x >= total) return;          // the whole block
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = t < total;
  const unsigned rl = t / (unsigned)p.n_r;
  const int ray = in ? list[rl] : list[0];
  float viol = 0.f;
  if (in) {
    const int i = (int)(t - rl * p.n_r);
    const size_t zi = (size_t)ray * p.n_r + i;
    const double *z = w.zone + zi * ZC_N;
    const double inv_a = z[ZC_INV_A];
    const double inv_a3 = inv_a * inv_a * inv_a;
    const double inv_acdt = z[ZC_INV_ACDT];
    const double Ti = T[zi], rho = p.rho[zi];
    // MIXED: the quotients by T^n as products with the zone's 1/T^n, the others from a reciprocal
    // seed with a Newton correction (within an ulp; the iteration converges to 1e-10); the FP64 path
    // divides
    const bool fast = w.phin32 != nullptr;
    const double iT = z[ZC_INV_T];
    const double cy = fast ? quot(kFourPiHC3 * p.eos.mb, rho) : kFourPiHC3 * p.eos.mb / rho;
    const double capT = kExpCap * Ti;
    const double eps0 = w.E[0] * inv_a;
    // rows of an even number of groups in 16-byte aligned arrays are read in 16-byte pieces
    const bool vec = (n % 2 == 0) &&
                     ((((uintptr_t)psi | (uintptr_t)p.kabs | (uintptr_t)w.jbuf) & 15u) == 0);
    double Y = ye[zi];
    double mu, dmu;
    if (fast) mu_nue_zone_q(p.eos, z[ZC_MUA], z[ZC_MUB], Ti, Y, mu, dmu);
    else mu_nue_zone(p.eos, z[ZC_MUA], z[ZC_MUB], Ti, Y, mu, dmu);
    double sG = 0.0, sdG = 0.0;
    for (int q = 0; q < 2; ++q) {
      const double sg = lepton_sign(q);
      const double muq = species_mu(q, mu), dmuq_T = fast ? sg * dmu * iT : sg * dmu / Ti;
      const size_t g0 = (((size_t)ray * NS + q) * p.n_r + i) * n;
      double a0, a1 = 0.0, c = 0.0;
      if (muq - eps0 < capT) {                    // no group at the cap
        if (vec) {
          // the same sums in the same order, the rows read 16 bytes at a time
          for (int k = 0; k < n; k += 2) {
            const double2 kp2 = *reinterpret_cast<const double2 *>(p.kabs + g0 + k);
            const double2 ps2 = *reinterpret_cast<const double2 *>(psi + g0 + k);
            const double2 jb2 = *reinterpret_cast<const double2 *>(w.jbuf + g0 + k);
            const double w0 = w.W[k], w1 = w.W[k + 1];
            const double k0 = p.scale ? kp2.x * p.scale[q * n + k] : kp2.x;
            const double k1 = p.scale ? kp2.y * p.scale[q * n + k + 1] : kp2.y;
            const double wj0 = w0 * jb2.x, wj1 = w1 * jb2.y;
            a1 += fma(-wj0, ps2.x, wj0);
            c = fma(w0 * k0, ps2.x, c);
            a1 += fma(-wj1, ps2.y, wj1);
            c = fma(w1 * k1, ps2.y, c);
          }
        } else {
          for (int k = 0; k < n; ++k) {
            const double wk = w.W[k];
            const double kap = p.scale ? p.kabs[g0 + k] * p.scale[q * n + k] : p.kabs[g0 + k];
            const double pk = psi[g0 + k];
            const double wj = wk * w.jbuf[g0 + k];
            a1 += fma(-wj, pk, wj);               // w j (1 - psi)
            c = fma(wk * kap, pk, c);             // w kappa psi
          }
        }
        a0 = a1 - c;
      } else {
        a0 = 0.0;
        for (int k = 0; k < n; ++k) {
          const double wk = w.W[k];
          const double kap = p.scale ? p.kabs[g0 + k] * p.scale[q * n + k] : p.kabs[g0 + k];
          const double pk = psi[g0 + k];
          const double wj = wk * w.jbuf[g0 + k];
          const double tj = fma(-wj, pk, wj);
          a0 += tj - wk * kap * pk;
          if (muq - w.E[k] * inv_a < capT) a1 += tj;
        }
      }
      sG += sg * a0 * inv_a3;
      sdG += sg * a1 * inv_a3 * dmuq_T;
    }
    const double GY = (Y - w.ye_n[zi]) * inv_acdt + cy * sG;
    const double dGY = inv_acdt + cy * sdG;
    const double dY = fast ? -quot(GY, dGY) : -GY / dGY;
    Y += dY;
    ye[zi] = Y;
    viol = tol_ratio(fabs(dY), fmax(fabs(Y), tl.tolmin_ye), tl.tolm_ye, tl.tole_ye);
    double mu1, dmu1;
    if (fast) mu_nue_zone_q(p.eos, z[ZC_MUA], z[ZC_MUB], Ti, Y, mu1, dmu1);
    else mu_nue_zone(p.eos, z[ZC_MUA], z[ZC_MUB], Ti, Y, mu1, dmu1);
    for (int q = 0; q < 2; ++q) {
      const double m0 = species_mu(q, mu), m1 = species_mu(q, mu1);
      const double ratio = exp(fast ? (m1 - m0) * iT : (m1 - m0) / Ti);
      const size_t g0 = (((size_t)ray * NS + q) * p.n_r + i) * n;
      if (m0 - eps0 < capT && m1 - eps0 < capT) {
        if (vec) {
          for (int k = 0; k < n; k += 2) {
            double2 *jb = reinterpret_cast<double2 *>(w.jbuf + g0 + k);
            double2 v = *jb;
            v.x *= ratio;
            v.y *= ratio;
            *jb = v;
          }
        } else {
          for (int k = 0; k < n; ++k) w.jbuf[g0 + k] *= ratio;
        }
      } else {
        for (int k = 0; k < n; ++k) {
          const double eps = w.E[k] * inv_a;
          if (m0 - eps < capT && m1 - eps < capT) {
            w.jbuf[g0 + k] *= ratio;
          } else {
            bool live;
            w.jbuf[g0 + k] = emissivity(scaled(p, p.kabs, g0 + k, q, k), m1, eps, Ti, live);
          }
        }
      }
    }
    if (!isfinite(Y)) {
      atomicExch(&w.nanflag[ray], 1);
      viol = INFINITY;
    }
  }
  report_violation(w, ray, viol);
}

// Per ray: close the iteration, decide convergence / failure / refactorisation and build the
// compacted lists of rays that continue (counters[0]) and that need new factors (counters[1]).
__global__ void k_check(int n_ray, Ws w, Tol tl) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_ray || !w.active[r]) return;
  const int it = ++w.iters[r];
  const double v = (double)__uint_as_float((unsigned)w.viol[r]);
  w.viol[r] = 0ull;
  int st = -1;
  if (w.nanflag[r]) st = MGFLD_ENAN;
  else if (v <= 1.0) st = MGFLD_OK;
  else if (it >= tl.max_iter) st = MGFLD_ENOCONV;
  if (st >= 0) {
    w.status[r] = st;
    w.active[r] = 0;
    return;
  }
  const int a = atomicAdd(&w.counters[0], 1);
  w.list_act[a] = r;
  int ref = 1;
  if (tl.chord) ref = v > tl.refactor_ratio * w.vprev[r];
  w.vprev[r] = v;
  w.refac[r] = ref;
  if (ref) {
    const int b = atomicAdd(&w.counters[1], 1);
    w.list_ref[b] = r;
    w.nfact[r] += 1;
  }
}

// Eq. a62b with the converged sources (w.src), T from the EoS, and per-zone ledger terms:
// [0] lepton number before, [1] after, [2] lepton number lost at R_{I+1/2} (last zone only),
// [3] energy at infinity before, [4] after, [5] energy lost, [6] gain-region heating.
// The group sums run over the grid at infinity (W_k = E_k^2 dE_k, W_k E_k) and take the zone's
// lapse factors once: eps^2 d eps = W / a^3 and eps^3 d eps = W E / a^4 on the comoving grid.
__global__ void k_finish(Prob p, Ws w, const double *__restrict__ psi, const double *__restrict__ ye,
                         double *__restrict__ T) {
  const int n = p.n;
  const size_t zi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (zi >= (size_t)p.n_ray * p.n_r) return;
  const int ray = (int)(zi / p.n_r), i = (int)(zi % p.n_r);
  const int last = p.n_r - 1;
  const double *z = w.zone + zi * ZC_N;
  const double inv_a = z[ZC_INV_A], a = z[ZC_A];
  const double inv_a3 = inv_a * inv_a * inv_a, inv_a4 = inv_a3 * inv_a;
  const double vol = z[ZC_VOL];
  const double rho = p.rho[zi], Y = ye[zi], Yn = w.ye_n[zi];
  const double acdt = z[ZC_ACDT];
  double sum_e = 0.0, heat = 0.0, nu_lep_a = 0.0, nu_lep_b = 0.0, nu_en_a = 0.0, nu_en_b = 0.0;
  double lep_loss = 0.0, en_loss = 0.0;
  for (int q = 0; q < NS; ++q) {
    const size_t g0 = (((size_t)ray * NS + q) * p.n_r + i) * n;
    double sS = 0.0, eA = 0.0, eB = 0.0, nA = 0.0, nB = 0.0;
    for (int k = 0; k < n; ++k) {
      const double we = w.WE[k];
      const double pk = psi[g0 + k], pn = w.psi_n[g0 + k];
      sS = fma(we, w.src[g0 + k], sS);
      eA = fma(we, pk, eA);
      eB = fma(we, pn, eB);
      if (q < 2) {
        nA = fma(w.W[k], pk, nA);
        nB = fma(w.W[k], pn, nB);
      }
    }
    const double sw = stat_weight(q), sl = lepton_sign(q);
    sum_e += sw * sS;
    if (q < 2) {
      heat += sS;
      nu_lep_a += sl * nA;
      nu_lep_b += sl * nB;
    }
    nu_en_a += sw * eA;
    nu_en_b += sw * eB;
    if (i == last) {
      for (int k = 0; k < n; ++k) {
        const double pk = psi[g0 + k];
        const double gh = w.ghost[((size_t)ray * NS + q) * n + k];
        const double fb = -w.alpha[g0 + k] * (gh * pk - pk);       // A psi1 / a^2 at R_{I+1/2}
        lep_loss += lepton_sign(q) * w.W[k] * fb;
        en_loss += stat_weight(q) * w.WE[k] * fb;
      }
    }
  }
  sum_e *= inv_a4;
  heat *= inv_a4;
  nu_lep_a *= inv_a3;
  nu_lep_b *= inv_a3;
  nu_en_a *= inv_a4;
  nu_en_b *= inv_a4;
  const double e_new = w.e_n[zi] - acdt * kFourPiHC3 * (p.eos.mb / rho) * sum_e;
  T[zi] = (e_new - eos_e_cold(p.eos, rho, Y)) / p.eos.ec;
  double *zl = w.zled + zi * 8;
  zl[0] = rho * vol * Yn / p.eos.mb + vol * kFourPiHC3 * nu_lep_b;
  zl[1] = rho * vol * Y / p.eos.mb + vol * kFourPiHC3 * nu_lep_a;
  zl[2] = (i == last) ? kC * p.dt * kFourPiHC3 * lep_loss : 0.0;
  zl[3] = a * (rho * vol * w.e_n[zi] / p.eos.mb + vol * kFourPiHC3 * nu_en_b);
  zl[4] = a * (rho * vol * e_new / p.eos.mb + vol * kFourPiHC3 * nu_en_a);
  zl[5] = (i == last) ? kC * p.dt * kFourPiHC3 * en_loss : 0.0;
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const double rc = 0.5 * (re[i] + re[i + 1]);
  zl[6] = (rc >= 1.0e7 && rc <= 3.0e7) ? -acdt * vol * kFourPiHC3 * heat : 0.0;
  zl[7] = 0.0;
  if (!isfinite(T[zi])) atomicExch(&w.nanflag[ray], 1);
}

// Per ray, fixed-order reduction of the per-zone ledger terms (deterministic).
__global__ void k_ledger(int n_r, Ws w, double *ledger, double *heating, int *status) {
  __shared__ double red[7][128];
  const int ray = blockIdx.x;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < n_r; i += blockDim.x) {
    const double *z = w.zled + ((size_t)ray * n_r + i) * 8;
    for (int c = 0; c < 7; ++c) acc[c] += z[c];
  }
  for (int c = 0; c < 7; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int c = 0; c < 7; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double lb = red[0][0], la = red[1][0], ll = red[2][0];
    const double eb = red[3][0], ea = red[4][0], el = red[5][0];
    if (ledger) {
      double *L = ledger + (size_t)ray * 8;
      L[0] = lb; L[1] = la; L[2] = ll; L[3] = la + ll - lb;
      L[4] = eb; L[5] = ea; L[6] = el; L[7] = ea + el - eb;
    }
    if (heating) heating[ray] = red[6][0];
    if (w.nanflag[ray]) w.status[ray] = MGFLD_ENAN;
    // Worst status over rays: ENAN dominates ENOCONV.
    const int st = w.status[ray];
    if (st == MGFLD_ENAN) atomicMax(&w.counters[2], 2);
    else if (st == MGFLD_ENOCONV) atomicMax(&w.counters[2], 1);
    if (status) status[ray] = w.status[ray];
  }
}

// Outer loop of the graph path: continue while some ray is still active and no bounded wait of
// the substitution gave up (counters[0]: active rays, counters[3]: the wait flag).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int *__restrict__ counters) {
  cudaGraphSetConditional(h, (counters[0] > 0 && counters[3] == 0) ? 1u : 0u);
}

// The step's status for the caller's report: ECUDA if a bounded wait gave up, else the worst ray
// status (ENAN before ENOCONV), else OK.
__global__ void k_status(const int *__restrict__ counters, int *__restrict__ status) {
  *status = counters[3] != 0 ? MGFLD_ECUDA
                             : (counters[2] == 2 ? MGFLD_ENAN : (counters[2] == 1 ? MGFLD_ENOCONV : MGFLD_OK));
}

// Optional per-category timing: a pair of CUDA events per category, read back after the host
// synchronisations the outer iteration already performs.  The events are created on the
// first profiled call on each device and kept for the life of the process (creating and
// destroying events on every call perturbed the host-synchronised loop).
struct Prof {
  double *out;
  cudaStream_t s;
  cudaEvent_t (*ev)[2];
  int pending[MGFLD_PROF_N];
  Prof(double *o, cudaStream_t st) : out(o), s(st), ev(nullptr) {
    for (int c = 0; c < MGFLD_PROF_N; ++c) pending[c] = 0;
    if (!out) return;
    static std::mutex lock;
    static cudaEvent_t cache[64][MGFLD_PROF_N][2];
    static bool made[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
      out = nullptr;
      return;
    }
    std::lock_guard<std::mutex> g(lock);
    if (!made[dev]) {
      for (int c = 0; c < MGFLD_PROF_N; ++c) {
        cudaEventCreate(&cache[dev][c][0]);
        cudaEventCreate(&cache[dev][c][1]);
      }
      made[dev] = true;
    }
    ev = cache[dev];
  }
  void begin(int c) { if (out) cudaEventRecord(ev[c][0], s); }
  void end(int c, int launches) {
    if (!out) return;
    cudaEventRecord(ev[c][1], s);
    pending[c] = launches;
  }
  void collect() {
    if (!out) return;
    for (int c = 0; c < MGFLD_PROF_N; ++c) {
      if (!pending[c]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[c][0], ev[c][1]) == cudaSuccess) {
        out[2 * c] += ms;
        out[2 * c + 1] += pending[c];
      }
      pending[c] = 0;
    }
  }
};

static Eos make_eos(const mgfld_eos_params &e) {
  Eos d;
  d.g1 = e.gamma1; d.g2 = e.gamma2; d.ec = e.e_coef; d.gn = e.g_n; d.gp = e.g_p;
  d.rho0 = e.rho_0; d.mbc2 = e.mb_c2; d.mb = e.m_b;
  d.f1 = 0.75 * std::cbrt(3.0 / (8.0 * kPi)) * kHC;
  d.rho_fac = std::pow(e.m_b / e.rho_0, e.gamma1 - 4.0 / 3.0);
  d.f2 = (e.gamma1 - 1.0) / (e.gamma2 - 1.0) * d.f1 * std::pow(0.5 * e.rho_nuc / e.m_b, e.gamma1 - e.gamma2) *
         d.rho_fac;
  d.log_gn_gp = std::log(e.g_n / e.g_p);
  d.g1_is_4_3 = e.gamma1 == 4.0 / 3.0;
  d.g2_is_5_2 = e.gamma2 == 2.5;
  return d;
}

bool dims_ok(const mgfld_dims *d) {
  if (!d || d->n_ray < 1 || d->n_r < 1 || d->n_e < 1 || d->n_e > MAX_NE || d->n_s != NS) return false;
  // Kernels decompose element indices in 32-bit arithmetic.
  return (long long)d->n_ray * NS * d->n_r * d->n_e < (1ll << 31);
}

bool prob_ok(const mgfld_problem *p) {
  return p && p->r_edge && p->e_edge && p->rho && p->kappa_abs && p->kappa_scat && p->dt > 0.0 &&
         (p->outer_bc == MGFLD_BC_GHOST || p->outer_bc == MGFLD_BC_REFLECT);
}

Prob make_prob(const mgfld_dims *d, const mgfld_problem *p) {
  Prob q;
  q.n_ray = d->n_ray; q.n_r = d->n_r; q.n = d->n_e; q.bc = p->outer_bc; q.dt = p->dt;
  q.r_edge = p->r_edge; q.lapse = p->lapse; q.e_edge = p->e_edge; q.rho = p->rho;
  q.kabs = p->kappa_abs; q.kscat = p->kappa_scat; q.nes = p->nes_coef; q.scale = p->scale;
  q.u = p->u; q.eta1 = p->eta1;
  q.pair = p->pair_coef; q.pair_chi = p->pair_chi;
  q.eos = make_eos(p->eos);
  return q;
}

static inline unsigned nblk(size_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

#define MGFLD_CUDA(x)                                  \
  do {                                                 \
    if ((x) != cudaSuccess) return MGFLD_ECUDA;        \
  } while (0)

}  // namespace mgfld

using namespace mgfld;

extern "C" {

mgfld_eos_params mgfld_eos_default(void) {
  mgfld_eos_params e;
  e.gamma1 = 4.0 / 3.0; e.gamma2 = 2.5; e.e_coef = 1.5; e.g_n = 2.0; e.g_p = 2.0;
  e.rho_nuc = 2.5e14; e.rho_0 = 2.5e14; e.mb_c2 = 939.565; e.m_b = 1.674927e-24;
  return e;
}

size_t mgfld_workspace_bytes(const mgfld_dims *dims, int precision) {
  if (!dims_ok(dims)) return 0;
  return make_layout(dims->n_ray, dims->n_r, dims->n_e, precision).total;
}

size_t mgfld_workspace_bytes_pair(const mgfld_dims *dims, int precision) {
  if (!dims_ok(dims) || 2 * dims->n_e > 48) return 0;
  return make_layout(dims->n_ray, dims->n_r, dims->n_e, precision, 1).total;
}

size_t mgfld_factor_bytes(const mgfld_dims *dims, int precision) {
  if (!dims_ok(dims)) return 0;
  const size_t blocks = (size_t)dims->n_ray * NS * dims->n_r * dims->n_e * dims->n_e;
  return blocks * (precision == MGFLD_MIXED ? sizeof(float) : sizeof(double));
}

const char *mgfld_status_str(mgfld_status s) {
  switch (s) {
    case MGFLD_OK: return "ok";
    case MGFLD_EINVAL: return "invalid argument";
    case MGFLD_ENOMEM: return "workspace too small";
    case MGFLD_ENOCONV: return "outer iteration did not converge";
    case MGFLD_ENAN: return "non-finite value";
    case MGFLD_ECUDA: return "CUDA error";
  }
  return "unknown status";
}

}  // extern "C"

namespace mgfld {

// Everything one call of the step needs, resolved from its arguments.
struct StepCall {
  Layout L;
  Ws w;
  Prob p;
  Tol tl;
  int pair, R, n, NR, coef_iterate, precision;
  mgfld_state st;
  mgfld_step_report rep;
};

static mgfld_status step_prepare(const mgfld_dims *dims, const mgfld_problem *prob, mgfld_state *state,
                                 const mgfld_step_opts *opts, mgfld_step_report *report, void *ws, size_t ws_bytes,
                                 StepCall &c) {
  if (!dims_ok(dims) || !prob_ok(prob) || !state || !state->psi || !state->ye || !state->T || !opts || !ws)
    return MGFLD_EINVAL;
  if ((opts->precision != MGFLD_FP64 && opts->precision != MGFLD_MIXED) || opts->max_iter < 1 ||
      !(opts->tol > 0.0) || !(opts->tol_ye > 0.0) || !(opts->tolmin_psi >= 0.0) || !(opts->tolmin_ye >= 0.0))
    return MGFLD_EINVAL;
  if (opts->coef_iterate && prob->u) return MGFLD_EINVAL;
  c.pair = prob->pair_coef != nullptr;
  // the pair process: coupled blocks of 2 n_e <= 48 rows, with the coefficients frozen for the step
  if (c.pair && (2 * dims->n_e > 48 || opts->coef_iterate)) return MGFLD_EINVAL;
  if (((uintptr_t)ws & 255u) != 0) return MGFLD_EINVAL;
  c.L = make_layout(dims->n_ray, dims->n_r, dims->n_e, opts->precision, c.pair);
  if (ws_bytes < c.L.total) return MGFLD_ENOMEM;
  c.w = resolve(ws, c.L);
  if (opts->coef_iterate) {
    // the limiter's derivatives take the storage of 1/lambda and lambda, which the neutrinosphere
    // scan has consumed before the limiter kernel writes them (setup and every iteration)
    c.w.jl = c.w.kinv;
    c.w.jr = c.w.lam;
  }
  c.p = make_prob(dims, prob);
  Tol &tl = c.tl;
  tl.tol = opts->tol; tl.tolmin = opts->tolmin_psi; tl.tol_ye = opts->tol_ye; tl.tolmin_ye = opts->tolmin_ye;
  tl.refactor_ratio = opts->refactor_ratio > 0.0 ? opts->refactor_ratio : 0.1;
  tl.max_iter = opts->max_iter; tl.mixed = opts->precision == MGFLD_MIXED;
  tl.chord = tl.mixed || opts->refactor_ratio > 0.0;
  tl.tolm = (float)std::frexp(opts->tol, &tl.tole);
  tl.tolm_ye = (float)std::frexp(opts->tol_ye, &tl.tole_ye);
  c.R = dims->n_ray; c.n = dims->n_e; c.NR = dims->n_r;
  c.coef_iterate = opts->coef_iterate;
  c.precision = opts->precision;
  c.st = *state;
  c.rep = report ? *report : mgfld_step_report{};
  return MGFLD_OK;
}

// The set-up of the step: frozen coefficients, per-ray bookkeeping, cleared counters.
static cudaError_t enqueue_setup(const StepCall &c, cudaStream_t s) {
  cudaError_t e = launch_setup(c.p, c.w, c.st.psi, c.st.ye, c.st.T, s);
  if (e != cudaSuccess) return e;
  k_init<<<nblk(c.R, 128), 128, 0, s>>>(c.R, c.w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaMemsetAsync(c.w.counters, 0, sizeof(int) * 8, s);
}

// One outer iteration (Eq. a62aa): residual / Jacobian of the listed rays, factorisation of the
// rays that need it, substitution, psi and Ye updates, convergence test and the next lists.  The
// listed counts are the host's (n_act, n_ref) or, with device_counts, counters[0] and [1] on the
// device (the grids then cover all rays and blocks past the counts return at once).
static cudaError_t enqueue_iteration(const StepCall &c, int it, int n_act, int n_ref, bool device_counts, Prof *prof,
                                     cudaStream_t s) {
  const Prob &p = c.p;
  const Ws &w = c.w;
  const Tol &tl = c.tl;
  const int n = c.n, NR = c.NR, R = c.R, pair = c.pair;
  const int *cnt_act = device_counts ? w.counters : nullptr;
  const int *cnt_ref = device_counts ? (tl.chord ? w.counters + 1 : w.counters) : nullptr;
  const int *jac = tl.chord ? w.refac : nullptr;
  cudaError_t e = cudaSuccess;
#define MGFLD_ENQ(x)                          \
  do {                                        \
    if ((e = (x)) != cudaSuccess) return e;   \
  } while (0)
  if (c.coef_iterate && it > 0) {
    // the flux coefficients of Eq. a59 at the current iterate (psi and Ye updated in place)
    if (prof) prof->begin(MGFLD_PROF_SETUP);
    MGFLD_ENQ(launch_coef_iterate(p, w, c.st.psi, w.list_act, n_act, cnt_act, s));
    if (prof) prof->end(MGFLD_PROF_SETUP, 3);
  }
  const bool incremental = !pair && it > 0 && tl.mixed && !c.coef_iterate;
  if (prof) prof->begin(incremental ? MGFLD_PROF_RESIDUAL : MGFLD_PROF_ASSEMBLE);
  if (pair)
    MGFLD_ENQ(launch_assemble_pair(p, w, c.st.psi, w.diag, tl.mixed, w.lower, w.upper, w.rhs, w.list_act, n_act, jac,
                                   s, nullptr, it == 0, cnt_act));
  else if (incremental)
    MGFLD_ENQ(launch_resid_ff(p, w, c.st.psi, (float *)w.diag, w.lower, w.upper, w.rhs, w.list_act, n_act, jac,
                              tl.tolmin, s, cnt_act));
  else
    MGFLD_ENQ(launch_assemble(p, w, c.st.psi, w.diag, tl.mixed, w.lower, w.upper, w.rhs, w.list_act, n_act, jac, s,
                              nullptr, it == 0 || c.coef_iterate, cnt_act));
  if (prof) prof->end(incremental ? MGFLD_PROF_RESIDUAL : MGFLD_PROF_ASSEMBLE, 1);
  const int *flist = tl.chord ? w.list_ref : w.list_act;
  const int nf = tl.chord ? n_ref : n_act;
  if (nf > 0) {
    if (prof) prof->begin(MGFLD_PROF_FACTOR);
    if (pair)
      MGFLD_ENQ(launch_factor_rows(2 * n, NR, nf * 2, 2, w.diag, tl.mixed ? (const void *)w.lower32 : w.lower,
                                   tl.mixed ? (const void *)w.upper32 : w.upper, w.dinv, tl.mixed, flist, s, cnt_ref));
    else if (tl.mixed)
      MGFLD_ENQ(launch_factor_f32(n, NR, nf * NS, (const float *)w.diag, w.lower32, w.upper32, (float *)w.dinv, flist,
                                  s, cnt_ref));
    else
      MGFLD_ENQ(launch_factor(n, NR, nf * NS, w.diag, 0, w.lower, w.upper, w.dinv, c.precision, flist, s, cnt_ref));
    if (prof) prof->end(MGFLD_PROF_FACTOR, 1);
  }
  if (prof) prof->begin(MGFLD_PROF_SOLVE);
  if (pair)
    MGFLD_ENQ(launch_solve_rows(2 * n, NR, n_act * 2, 2, w.dinv, tl.mixed ? (const void *)w.lower32 : w.lower,
                                tl.mixed ? (const void *)w.upper32 : w.upper, w.rhs, w.rhs32, w.sscale, w.x, tl.mixed,
                                w.list_act, s, cnt_act));
  else if (tl.mixed && n % 2 == 0)
    MGFLD_ENQ(launch_solve_tma(n, NR, n_act * NS, w.dinv, w.lower32, w.upper32, w.rhs, w.rhs32, w.x, w.g32,
                               w.list_act, w.sscale, w.counters + 3, s, cnt_act));
  else
    MGFLD_ENQ(launch_solve(n, NR, n_act * NS, w.dinv, w.lower, w.upper, w.rhs, w.x, c.precision, w.list_act, s,
                           cnt_act));
  if (prof) prof->end(MGFLD_PROF_SOLVE, 1);
  if (prof) prof->begin(MGFLD_PROF_UPDATE);
  if (!pair && n % 2 == 0 && ((uintptr_t)c.st.psi & 15u) == 0)
    k_update_psi2<<<nblk((size_t)n_act * NS * NR * n / 2, 256), 256, 0, s>>>(p, w, tl, c.st.psi, w.list_act, n_act,
                                                                        cnt_act);
  else
    k_update_psi<<<nblk((size_t)n_act * NS * NR * n, 256), 256, 0, s>>>(p, w, tl, c.st.psi, w.list_act, n_act,
                                                                       cnt_act);
  MGFLD_ENQ(cudaGetLastError());
  k_update_ye<<<nblk((size_t)n_act * NR, 128), 128, 0, s>>>(p, w, tl, c.st.psi, c.st.ye, c.st.T, w.list_act, n_act,
                                                            cnt_act);
  MGFLD_ENQ(cudaGetLastError());
  MGFLD_ENQ(cudaMemsetAsync(w.counters, 0, sizeof(int) * 2, s));
  k_check<<<nblk(R, 128), 128, 0, s>>>(R, w, tl);
  MGFLD_ENQ(cudaGetLastError());
  if (prof) prof->end(MGFLD_PROF_UPDATE, 3);
  return cudaSuccess;
}

// After the iteration: Eq. a62b with the converged sources, T, the ledgers, the report.
static cudaError_t enqueue_finish(const StepCall &c, Prof *prof, cudaStream_t s) {
  const Ws &w = c.w;
  const int R = c.R, NR = c.NR;
  cudaError_t e = cudaSuccess;
  if (prof) prof->begin(MGFLD_PROF_FINISH);
  if (c.pair)
    MGFLD_ENQ(launch_assemble_pair(c.p, w, c.st.psi, w.diag, c.tl.mixed, w.lower, w.upper, w.rhs, nullptr, R, nullptr,
                                   s, w.src, 0));
  else if (c.tl.mixed)
    MGFLD_ENQ(launch_src_mixed(c.p, w, c.st.psi, w.src, s));
  else
    MGFLD_ENQ(launch_assemble(c.p, w, c.st.psi, w.diag, c.tl.mixed, w.lower, w.upper, w.rhs, nullptr, R, nullptr, s,
                              w.src));
  k_finish<<<nblk((size_t)R * NR, 128), 128, 0, s>>>(c.p, w, c.st.psi, c.st.ye, c.st.T);
  MGFLD_ENQ(cudaGetLastError());
  MGFLD_ENQ(cudaMemsetAsync(w.counters + 2, 0, sizeof(int), s));
  k_ledger<<<R, 128, 0, s>>>(NR, w, c.rep.ledger, c.rep.heating, c.rep.ray_status);
  MGFLD_ENQ(cudaGetLastError());
  if (prof) prof->end(MGFLD_PROF_FINISH, 3);
  if (c.rep.iters)
    MGFLD_ENQ(cudaMemcpyAsync(c.rep.iters, w.iters, sizeof(int) * R, cudaMemcpyDeviceToDevice, s));
  if (c.rep.factorizations)
    MGFLD_ENQ(cudaMemcpyAsync(c.rep.factorizations, w.nfact, sizeof(int) * R, cudaMemcpyDeviceToDevice, s));
  if (c.rep.status) {
    k_status<<<1, 1, 0, s>>>(w.counters, c.rep.status);
    MGFLD_ENQ(cudaGetLastError());
  }
  return cudaSuccess;
#undef MGFLD_ENQ
}

// The step with the outer iteration driven from the host: one stream synchronisation per
// iteration (the convergence counters), per-category timing when requested.
static mgfld_status step_host_loop(const StepCall &c, double *profile, cudaStream_t s) {
  Prof prof(profile, s);
  Prof *pp = profile ? &prof : nullptr;
  if (pp) prof.begin(MGFLD_PROF_SETUP);
  MGFLD_CUDA(enqueue_setup(c, s));
  if (pp) prof.end(MGFLD_PROF_SETUP, 7 + (c.p.u ? 1 : 0) + (c.pair ? 1 : 0));
  int n_act = c.R, n_ref = c.R;
  int host_counters[8];
  for (int it = 0; it < c.tl.max_iter && n_act > 0; ++it) {
    MGFLD_CUDA(enqueue_iteration(c, it, n_act, n_ref, false, pp, s));
    MGFLD_CUDA(cudaMemcpyAsync(host_counters, c.w.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    MGFLD_CUDA(cudaStreamSynchronize(s));
    prof.collect();
    if (host_counters[3] != 0) return MGFLD_ECUDA;      // a bounded wait in the solve gave up
    n_act = host_counters[0];
    n_ref = host_counters[1];
  }
  MGFLD_CUDA(enqueue_finish(c, pp, s));
  MGFLD_CUDA(cudaMemcpyAsync(host_counters + 2, c.w.counters + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  MGFLD_CUDA(cudaStreamSynchronize(s));
  prof.collect();
  if (host_counters[2] == 2) return MGFLD_ENAN;
  if (host_counters[2] == 1) return MGFLD_ENOCONV;
  return MGFLD_OK;
}

// ------------------------------------------------------------------ the graph path
//
// The whole step as one CUDA graph: the set-up and the first iteration, then a while-conditional
// node whose body is one iteration with device-resident counts, its condition set on the device
// by k_loop_cond after every convergence test, then the finish.  Nothing waits on the host, so the
// call is asynchronous on the caller's stream.  The instantiated graph of each distinct set of
// arguments (pointers, sizes, options) is kept for the life of the process and launched again
// when the same arguments come back.

static void key_put(std::string &k, const void *v, size_t n) { k.append((const char *)v, n); }
template <typename T> static void key_put(std::string &k, const T &v) { key_put(k, &v, sizeof(T)); }

static std::string graph_key(int dev, const mgfld_dims *d, const mgfld_problem *pr, const mgfld_state *st,
                             const mgfld_step_opts *o, const mgfld_step_report &rep, const void *ws, size_t ws_bytes) {
  std::string k;
  key_put(k, dev);
  key_put(k, d->n_ray); key_put(k, d->n_r); key_put(k, d->n_e); key_put(k, d->n_s);
  const void *ptrs[] = {pr->r_edge, pr->lapse, pr->e_edge, pr->rho, pr->kappa_abs, pr->kappa_scat, pr->nes_coef,
                        pr->scale, pr->u, pr->eta1, pr->pair_coef, st->psi, st->ye, st->T, rep.iters, rep.ray_status,
                        rep.ledger, rep.heating, rep.factorizations, rep.status, ws};
  key_put(k, ptrs, sizeof(ptrs));
  const double eos[] = {pr->eos.gamma1, pr->eos.gamma2, pr->eos.e_coef, pr->eos.g_n, pr->eos.g_p, pr->eos.rho_nuc,
                        pr->eos.rho_0, pr->eos.mb_c2, pr->eos.m_b, pr->dt, o->tol, o->tolmin_psi, o->tol_ye,
                        o->tolmin_ye, o->refactor_ratio};
  key_put(k, eos, sizeof(eos));
  const int ints[] = {pr->outer_bc, pr->pair_chi, o->precision, o->max_iter, o->coef_iterate};
  key_put(k, ints, sizeof(ints));
  key_put(k, ws_bytes);
  return k;
}

struct GraphCache {
  std::mutex lock;
  std::unordered_map<std::string, cudaGraphExec_t> execs;
  cudaStream_t cap[64][2] = {};      // per device: the streams the graphs are captured on
};
static GraphCache &graph_cache() {
  static GraphCache *c = new GraphCache();     // kept for the life of the process
  return *c;
}

static cudaError_t build_step_graph(const StepCall &c, cudaStream_t cs, cudaStream_t bs, cudaGraphExec_t *out) {
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr, body = nullptr, done = nullptr;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle h{};
  cudaGraphNodeParams cp{};
  cudaGraphNode_t cn{};
  bool body_open = false;
  auto fail = [&](cudaError_t err) {
    if (body_open) {
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(bs, &tmp);
    }
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(cs, &tmp);
    if (tmp) cudaGraphDestroy(tmp);
    return err;
  };
  if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g)) != cudaSuccess) return fail(e);
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return fail(e);
  if ((e = enqueue_setup(c, cs)) != cudaSuccess) return fail(e);
  if ((e = enqueue_iteration(c, 0, c.R, c.R, false, nullptr, cs)) != cudaSuccess) return fail(e);
  k_loop_cond<<<1, 1, 0, cs>>>(h, c.w.counters);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess) return fail(e);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&cn, g, deps, nullptr, nd, &cp)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
    return fail(e);
  body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
    return fail(e);
  body_open = true;
  if ((e = enqueue_iteration(c, 1, c.R, c.R, true, nullptr, bs)) != cudaSuccess) return fail(e);
  k_loop_cond<<<1, 1, 0, bs>>>(h, c.w.counters);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaStreamEndCapture(bs, &body)) != cudaSuccess) return fail(e);
  body_open = false;
  if ((e = enqueue_finish(c, nullptr, cs)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamEndCapture(cs, &done)) != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, done, 0);
  cudaGraphDestroy(done);
  return e;
}

static mgfld_status step_graph(const StepCall &c, const mgfld_dims *dims, const mgfld_problem *prob,
                               const mgfld_step_opts *opts, void *ws, size_t ws_bytes, cudaStream_t s) {
  int dev = 0;
  MGFLD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return MGFLD_ECUDA;
  const std::string key = graph_key(dev, dims, prob, &c.st, opts, c.rep, ws, ws_bytes);
  GraphCache &gc = graph_cache();
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> guard(gc.lock);
    auto it = gc.execs.find(key);
    if (it != gc.execs.end()) {
      exec = it->second;
    } else {
      for (int k = 0; k < 2; ++k)
        if (!gc.cap[dev][k]) MGFLD_CUDA(cudaStreamCreateWithFlags(&gc.cap[dev][k], cudaStreamNonBlocking));
      MGFLD_CUDA(build_step_graph(c, gc.cap[dev][0], gc.cap[dev][1], &exec));
      gc.execs.emplace(key, exec);
    }
  }
  MGFLD_CUDA(cudaGraphLaunch(exec, s));
  return MGFLD_OK;
}

mgfld_status step_host_synchronised(const mgfld_dims *dims, const mgfld_problem *prob, mgfld_state *state,
                                    const mgfld_step_opts *opts, mgfld_step_report *report, void *ws,
                                    size_t ws_bytes, void *stream) {
  StepCall c;
  const mgfld_status st = step_prepare(dims, prob, state, opts, report, ws, ws_bytes, c);
  if (st != MGFLD_OK) return st;
  return step_host_loop(c, opts->profile, (cudaStream_t)stream);
}

}  // namespace mgfld

extern "C" {

mgfld_status mgfld_step(const mgfld_dims *dims, const mgfld_problem *prob, mgfld_state *state,
                        const mgfld_step_opts *opts, mgfld_step_report *report, void *ws, size_t ws_bytes,
                        void *stream) {
  StepCall c;
  const mgfld_status st = step_prepare(dims, prob, state, opts, report, ws, ws_bytes, c);
  if (st != MGFLD_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (opts->profile) return step_host_loop(c, opts->profile, s);
  return step_graph(c, dims, prob, opts, ws, ws_bytes, s);
}

mgfld_status mgfld_assemble(const mgfld_dims *dims, const mgfld_problem *prob, const mgfld_state *state,
                            mgfld_system *sys, void *ws, size_t ws_bytes, void *stream) {
  if (!dims_ok(dims) || !prob_ok(prob) || !state || !state->psi || !state->ye || !state->T || !sys ||
      !sys->diag || !sys->lower || !sys->upper || !sys->rhs || !ws || prob->pair_coef)
    return MGFLD_EINVAL;
  if (((uintptr_t)ws & 255u) != 0) return MGFLD_EINVAL;
  const Layout L = make_layout(dims->n_ray, dims->n_r, dims->n_e, MGFLD_FP64);
  if (ws_bytes < L.total) return MGFLD_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  const Ws w = resolve(ws, L);
  const Prob p = make_prob(dims, prob);
  MGFLD_CUDA(launch_setup(p, w, state->psi, state->ye, state->T, s));
  MGFLD_CUDA(launch_assemble(p, w, state->psi, sys->diag, 0, sys->lower, sys->upper, sys->rhs, nullptr,
                             dims->n_ray, nullptr, s, nullptr, 1));
  return MGFLD_OK;
}

mgfld_status mgfld_factor(const mgfld_dims *dims, const mgfld_system *sys, int precision, void *factor,
                          void *stream) {
  if (!dims_ok(dims) || !sys || !sys->diag || !sys->lower || !sys->upper || !factor ||
      (precision != MGFLD_FP64 && precision != MGFLD_MIXED))
    return MGFLD_EINVAL;
  MGFLD_CUDA(launch_factor(dims->n_e, dims->n_r, dims->n_ray * NS, sys->diag, 0, sys->lower, sys->upper,
                           factor, precision, nullptr, (cudaStream_t)stream));
  return MGFLD_OK;
}

mgfld_status mgfld_solve(const mgfld_dims *dims, const mgfld_system *sys, int precision, const void *factor,
                         const double *rhs, double *x, void *stream) {
  if (!dims_ok(dims) || !sys || !sys->lower || !sys->upper || !factor || !rhs || !x ||
      (precision != MGFLD_FP64 && precision != MGFLD_MIXED))
    return MGFLD_EINVAL;
  MGFLD_CUDA(launch_solve(dims->n_e, dims->n_r, dims->n_ray * NS, factor, sys->lower, sys->upper, rhs, x,
                          precision, nullptr, (cudaStream_t)stream));
  return MGFLD_OK;
}

}  // extern "C"
