// Residual and Jacobian rows of the per-species Newton system (Eqs. a58, a59, a62ac).
//
// One thread owns the equation of (ray, species q, zone i, group k):
//   G = (psi - psi^n)/(a c dt) + (a^2/V)[A psi1/a^2 |_{i+1/2} - A psi1/a^2 |_{i-1/2}] - S,
//   psi1_{i+1/2} = -D_{i+1/2} (psi_{i+1} - psi_i)              (Eq. a59, D frozen at psi^n)
//   (with a shock, Eqs. a93/a99: a step constant joins the bracket, see k_shock)
//   S = j (1 - psi) - kappa_a psi                             (Eq. a55)
//     + C [(1 - psi_k) sum_k' w_k' Phi_in[k,k'] psi_k' - psi_k sum_k' w_k' Phi_out[k,k'] (1 - psi_k')]
//                                                              (Eq. d8, Phi_1 = 0; Phi_in[k,k'] = Phi_out[k',k])
// and, when the ray is flagged for a new factorisation, the dense row dG_k/dpsi_k' of the
// diagonal block plus the diagonal couplings to zones i-1 and i+1 (Eq. a62ae).
#include "mgfld_internal.cuh"

namespace mgfld {

template <typename TD>
__global__ void k_assemble(Prob p, Ws w, const double *__restrict__ psi, TD *__restrict__ diag,
                           double *__restrict__ lower, double *__restrict__ upper, double *__restrict__ rhs,
                           const int *__restrict__ list, int n_list, const int *__restrict__ jac_flag,
                           double *__restrict__ src_out, int first, const int *__restrict__ n_dev) {
  const int n = p.n;
  // 32-bit index arithmetic (element counts are below 2^31, checked on the host).
  const unsigned per_ray = (unsigned)(NS * p.n_r * n);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)listed(n_list, n_dev) * per_ray) return;
  const unsigned rl = t / per_ray;
  const int ray = list ? list[rl] : (int)rl;
  // Thread order (zone, species, group) inside a ray: the four species of a zone share the
  // zone's NES kernel rows through L1.
  const unsigned local = t - rl * per_ray;
  const unsigned kq = local / (unsigned)n;
  const int k = (int)(local - kq * n);
  const int q = (int)(kq % NS);
  const int i = (int)(kq / NS);
  const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;   // (ray, q, i, k) storage index
  const size_t zi = (size_t)ray * p.n_r + i;
  const int last = p.n_r - 1;

  const double *z = w.zone + zi * ZC_N;
  const double pre = z[ZC_PRE];
  const double inv_acdt = z[ZC_INV_ACDT];

  const double *ps = psi + (g - k);
  const double pk = ps[k];
  const double *fin = w.phin + (zi * n + k) * n;
  const double *fout = w.phout + (zi * n + k) * n;
  double gain = 0.0, lp = 0.0;
  if (first) {                 // formed at this psi already: by the setup (psi^n) or with the n+1 coefficients
    gain = w.g0[g];
    lp = w.l0[g];
  } else if (src_out && w.phin32) {
    // MIXED, converged state psi_m + dpsi (dpsi = w.x, the last correction of this ray): the
    // sums of the ray's last residual (at psi_m, kept in g0/l0) plus phin.dpsi and phout.dpsi,
    // taken in FP32.  |dpsi| is below the tolerance, so the FP32 rounding (relative 2^-24 of
    // |phin| |dpsi|) stays far below the FP64 rounding of the sums themselves.
    const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
    const double *dx = w.x + (g - k);
    float dg = 0.f, dl = 0.f;
    for (int kp = 0; kp < n; ++kp) {
      const float d = (float)dx[kp];
      dg = fmaf(fi[kp], d, dg);
      dl = fmaf(fi[kp] - fd[kp], d, dl);
    }
    gain = w.g0[g] + (double)dg;
    lp = w.l0[g] + (double)dl;
  } else {
    for (int kp = 0; kp < n; ++kp) {
      const double pv = ps[kp];
      gain += fin[kp] * pv;
      lp += fout[kp] * pv;
    }
    if (w.phin32 && !src_out) {   // MIXED: keep this residual's sums for the final sources
      w.g0[g] = gain;
      w.l0[g] = lp;
    }
  }
  const double j = w.jbuf[g];
  double G, dg, c_low, c_up;
  if (!first && !src_out && !w.jl) {
    // Later iterations with the coefficients frozen for the step: the constants the first pass
    // stored, G = psi (D0 + j + gain - lp) - c_r psi_{i+1} - c_l psi_{i-1} - (b0 + j + gain), which
    // is Eq. a58 with the flux of Eq. a59 and S regrouped (the terms in psi collected).
    dg = ((w.cdiag[g] + j) + gain) - lp;
    G = fma(pk, dg, -((w.cb[g] + j) + gain));
    c_up = w.cup[g];
    c_low = w.clow[g];
    if (i < last) G = fma(-c_up, ps[k + n], G);
    if (i > 0) G = fma(-c_low, ps[k - (ptrdiff_t)n], G);
  } else if (!src_out && !w.jl && w.phin32) {
    // The first pass of the mixed path with the coefficients frozen for the step: the step
    // constants (D0 with the ghost of the outer edge folded in, the couplings, the psi-independent
    // part b0), stored for the later passes, and the row formed from them as the later passes form
    // it.  (The FP64 path forms its first row below from the terms of Eq. a58 as written: with
    // the regrouped form there, its results on the benchmark rays moved from 0.90 to 1.02 x 1e-12
    // of the oracle's, across the FP64 gate.)
    const double kap = scaled(p, p.kabs, g, q, k);
    const double al_out = w.alpha[g];
    const double al_in = i > 0 ? w.alpha[g - n] : 0.0;
    const double jdiag = i == last ? fma(-al_out, w.ghost[((size_t)ray * NS + q) * n + k], al_out) + al_in
                                   : al_out + al_in;
    const double d0 = inv_acdt + pre * jdiag + kap + w.rsum[zi * n + k];
    const double sh = p.u ? w.shock[g] : 0.0;
    const double b0 = w.psi_n[g] * inv_acdt - pre * sh;
    c_up = i < last ? pre * al_out : 0.0;
    c_low = pre * al_in;
    w.cdiag[g] = d0;
    w.cup[g] = c_up;
    w.clow[g] = c_low;
    w.cb[g] = b0;
    dg = ((d0 + j) + gain) - lp;
    G = fma(pk, dg, -((b0 + j) + gain));
    if (i < last) G = fma(-c_up, ps[k + n], G);
    if (i > 0) G = fma(-c_low, ps[k - (ptrdiff_t)n], G);
  } else {
    // The sources alone (src_out), the row with the flux coefficients of the iterate (jl), or
    // the FP64 path's first row.
    const double loss = w.rsum[zi * n + k] - lp;          // sum_k' phout (1 - psi_k')
    const double kap = scaled(p, p.kabs, g, q, k);
    const double S = j * (1.0 - pk) - kap * pk + ((1.0 - pk) * gain - pk * loss);
    if (src_out) {               // converged sources for Eq. a62b and the ledgers
      src_out[g] = S;
      return;
    }

    const double al_out = w.alpha[g];
    const double al_in = i > 0 ? w.alpha[g - n] : 0.0;
    const double gh = (i == last) ? w.ghost[((size_t)ray * NS + q) * n + k] : 0.0;
    const double p_right = i < last ? ps[k + n] : gh * pk;
    const double p_left = i > 0 ? ps[k - (ptrdiff_t)n] : pk;
    const double flux_out = -al_out * (p_right - pk);
    const double flux_in = -al_in * (pk - p_left);
    // shock transport: the step-constant frame terms of Eqs. a93 and a99 (formed at psi^n)
    const double sh = p.u ? w.shock[g] : 0.0;
    G = (pk - w.psi_n[g]) * inv_acdt + pre * (flux_out - flux_in + sh) - S;
    // flux parts of the row: d(flux at i+1/2)/d psi_i = jl, d/d psi_{i+1} = jr; alpha and -alpha with
    // the frozen coefficients, with the limiter's own derivative when they follow the iterate
    double jdiag = al_out * (1.0 - gh) + al_in, jlow = al_in, jup = al_out;
    if (w.jl) {
      const double jl_out = w.jl[g], jr_out = w.jr[g];
      const double jl_in = i > 0 ? w.jl[g - n] : 0.0, jr_in = i > 0 ? w.jr[g - n] : 0.0;
      jdiag = jl_out + gh * jr_out - jr_in;
      jlow = jl_in;
      jup = -jr_out;
    }
    dg = inv_acdt + pre * jdiag + j + kap + (gain + loss);
    c_low = pre * jlow;
    c_up = i < last ? pre * jup : 0.0;
    if (first && !w.jl && !src_out) {
      // the FP64 path's first pass: the step constants of its later passes
      w.cdiag[g] = inv_acdt + pre * jdiag + kap + w.rsum[zi * n + k];
      w.cup[g] = c_up;
      w.clow[g] = c_low;
      w.cb[g] = w.psi_n[g] * inv_acdt - pre * sh;
    }
  }
  rhs[g] = -G;

  if (jac_flag && !jac_flag[ray]) return;
  TD *row = diag + g * n;
  // dS_k/dpsi_k' = (1 - psi_k) phin + psi_k phout = phin - psi_k phd, entered with a minus;
  // dg joins the diagonal entry in the rows' precision.  Rows are written 16 bytes at a time where n allows
  // (the rows of one warp's threads are 16-byte aligned and contiguous per species).
  if (sizeof(TD) == 4 && w.phin32) {
    const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
    // FP32 operands from the integer pipe (truncated; the FP32 Jacobian is the preconditioner of
    // the FP64 refinement), dg joining the diagonal in FP32
    const float pf = d2f_exp2(pk, 0);
    const float dk = fmaf(pf, fd[k], -fi[k]) + (float)dg;
    if ((n & 3) == 0) {
      for (int c = 0; c < n; c += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(fi + c);
        const float4 d = *reinterpret_cast<const float4 *>(fd + c);
        float4 v = make_float4(fmaf(pf, d.x, -a.x), fmaf(pf, d.y, -a.y), fmaf(pf, d.z, -a.z), fmaf(pf, d.w, -a.w));
        if (k == c) v.x = dk;
        if (k == c + 1) v.y = dk;
        if (k == c + 2) v.z = dk;
        if (k == c + 3) v.w = dk;
        *reinterpret_cast<float4 *>(row + c) = v;
      }
    } else {
      for (int kp = 0; kp < n; ++kp) row[kp] = TD(kp == k ? dk : fmaf(pf, fd[kp], -fi[kp]));
    }
  } else {
    const double *fd = w.phd + (zi * n + k) * n;
    const double dk = fma(pk, fd[k], -fin[k]) + dg;
    bool done = false;
    if constexpr (sizeof(TD) == 8) {
      if ((n & 1) == 0) {
        for (int c = 0; c < n; c += 2) {
          const double2 a = *reinterpret_cast<const double2 *>(fin + c);
          const double2 d = *reinterpret_cast<const double2 *>(fd + c);
          double2 v = make_double2(fma(pk, d.x, -a.x), fma(pk, d.y, -a.y));
          if (k == c) v.x = dk;
          if (k == c + 1) v.y = dk;
          *reinterpret_cast<double2 *>(row + c) = v;
        }
        done = true;
      }
    }
    if (!done) {
      for (int kp = 0; kp < n; ++kp) row[kp] = TD(kp == k ? dk : fma(pk, fd[kp], -fin[kp]));
    }
  }
  lower[g] = -c_low;
  upper[g] = -c_up;
  if (w.lower32) {
    w.lower32[g] = d2f_exp2(-c_low, 0);
    w.upper32[g] = d2f_exp2(-c_up, 0);
  }
}

cudaError_t launch_assemble(const Prob &p, const Ws &w, const double *psi, void *diag, int diag_fp32,
                            double *lower, double *upper, double *rhs, const int *list, int n_list,
                            const int *jac_flag, cudaStream_t s, double *src_out, int first, const int *n_dev) {
  const size_t total = (size_t)n_list * NS * p.n_r * p.n;
  if (total == 0) return cudaSuccess;
  const unsigned B = 256;
  const unsigned grid = (unsigned)((total + B - 1) / B);
  if (diag_fp32)
    k_assemble<float><<<grid, B, 0, s>>>(p, w, psi, (float *)diag, lower, upper, rhs, list, n_list, jac_flag,
                                         src_out, first, n_dev);
  else
    k_assemble<double><<<grid, B, 0, s>>>(p, w, psi, (double *)diag, lower, upper, rhs, list, n_list,
                                          jac_flag, src_out, first, n_dev);
  return cudaGetLastError();
}

// The converged sources of the mixed path for Eq. a62b and the ledgers, one thread per (ray, q, i,
// k) of every ray:
//   S = j (1 - psi) - kappa_a psi + (1 - psi) gain - psi loss          (Eqs. a55, d8)
// at psi = psi_m + dpsi (dpsi the ray's last, sub-tolerance correction w.x): gain and
// loss = rsum - lp from the sums of the ray's last residual at psi_m (g0, l0) plus phin.dpsi and
// (phin - phd).dpsi taken in FP32 (|dpsi| is below the tolerance, so their FP32 rounding stays far
// below the FP64 rounding of the sums), the two corrections joined in FP32 before one conversion.
// The block stages the corrections of the rows it covers in shared memory as FP32, one conversion
// per value instead of one per product.
constexpr int kSrcThreads = 256;
__global__ void __launch_bounds__(kSrcThreads)
k_src_mixed(Prob p, Ws w, const double *__restrict__ psi, double *__restrict__ src) {
  __shared__ float xs[kSrcThreads + 2 * MAX_NE];
  const int n = p.n;
  const unsigned per_ray = (unsigned)(NS * p.n_r * n);
  const unsigned total = (unsigned)p.n_ray * per_ray;
  const unsigned b0 = blockIdx.x * kSrcThreads;
  const unsigned last = min(b0 + kSrcThreads, total) - 1;
  const unsigned gq0 = b0 / (unsigned)n;                    // first (ray, zone, species) row group
  const unsigned cnt = (last / (unsigned)n - gq0 + 1) * (unsigned)n;
  for (unsigned j = threadIdx.x; j < cnt; j += kSrcThreads) {
    const unsigned gq = gq0 + j / (unsigned)n, kk = j % (unsigned)n;
    const unsigned ray = gq / (unsigned)(NS * p.n_r), rem = gq - ray * (unsigned)(NS * p.n_r);
    const unsigned i = rem / NS, q = rem - i * NS;
    xs[j] = (float)w.x[(((size_t)ray * NS + q) * p.n_r + i) * n + kk];
  }
  __syncthreads();
  const unsigned t = b0 + threadIdx.x;
  if (t >= total) return;
  const unsigned ray = t / per_ray;
  const unsigned local = t - ray * per_ray;
  const unsigned kq = local / (unsigned)n;
  const int k = (int)(local - kq * n);
  const int q = (int)(kq % NS);
  const int i = (int)(kq / NS);
  const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;
  const size_t zi = (size_t)ray * p.n_r + i;
  const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
  const float *dx = xs + (t / (unsigned)n - gq0) * (unsigned)n;
  float dg = 0.f, dl = 0.f;
  for (int kp = 0; kp < n; ++kp) {
    const float d = dx[kp], a = fi[kp];
    dg = fmaf(a, d, dg);
    dl = fmaf(a - fd[kp], d, dl);
  }
  const double pk = psi[g];
  const double q1 = 1.0 - pk;
  const float pf = d2f_exp2(pk, 0);
  // (1 - psi) dgain + psi dlp: the FP32 part of (1 - psi) gain - psi loss
  const float corr = fmaf(1.f - pf, dg, pf * dl);
  const double kap = scaled(p, p.kabs, g, q, k);
  const double loss0 = w.rsum[zi * n + k] - w.l0[g];
  double S = fma(q1, w.g0[g], fma(-pk, loss0, (double)corr));
  S = fma(w.jbuf[g], q1, fma(-kap, pk, S));
  src[g] = S;
}

cudaError_t launch_src_mixed(const Prob &p, const Ws &w, const double *psi, double *src, cudaStream_t s) {
  const size_t total = (size_t)p.n_ray * NS * p.n_r * p.n;
  if (total == 0) return cudaSuccess;
  k_src_mixed<<<(unsigned)((total + kSrcThreads - 1) / kSrcThreads), kSrcThreads, 0, s>>>(p, w, psi, src);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// The later residual passes of the mixed path (coefficients frozen for the step, no pair
// process): the NES sums of the iterate from the kept sums of the previous one plus the kernels
// times the last correction,
//   gain = gain_prev + sum_k' phin[k][k'] dpsi_k',   lp = lp_prev + sum_k' phout[k][k'] dpsi_k',
// exact in exact arithmetic (the sums are linear in psi).  The products and their sums are taken
// in FP32 pairs (hi + lo, ~48 bits; products split exactly with an FMA, sums with the two-sum of
// Knuth), on row-scaled kernels and group-scaled corrections, so the FP64 pipe only adds the two
// increments to the kept sums and forms the row.  The pairs carry the increment to ~1e-13 of the
// sum of its terms' magnitudes, so a (zone, species) group whose last correction exceeds ~1.6 %
// of max(|psi|, tolmin) over the group forms its sums again in FP64 instead; below that the error
// of an increment stays within a few FP64 roundings of the sums themselves.  Then the row
// as the later passes form it (G = psi (D0 + j + gain - lp) - (b0 + j + gain) - couplings) and,
// where the ray takes new factors, the FP32 Jacobian rows.
//
// A block takes whole zones (Z zones of NS n rows, Z NS n <= 256), stages their scaled kernels
// and the corrections of its rows in shared memory, and runs the two dot products of a row as
// one sequence of packed FP32x2 operations (the gain and the loss sums side by side).  Rows are
// threads in the order (zone, species, group) of k_assemble.
__host__ __device__ inline int ff_zpb(int n) { return (256 / (NS * n)) > 0 ? 256 / (NS * n) : 1; }
__host__ __device__ inline int ff_ld(int n) { return (n % 2 == 0) ? n + 1 : n; }      // odd row stride in float4
static inline size_t ff_smem(int n) {
  const int z = ff_zpb(n), rows = z * NS * n;
  return sizeof(float4) * (size_t)z * n * ff_ld(n) + sizeof(int2) * (size_t)z * n + sizeof(float2) * rows +
         2 * sizeof(unsigned) * (size_t)z * NS + sizeof(long long) * (size_t)z;
}

// Knuth's two-sum of the two lanes of a pair: s + b -> s, returning its rounding error; the
// differences are FMAs with a -1 multiplier (exact as subtractions, no negations).
__device__ inline float2 two_sum2(float2 &s, float2 b) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 a = s;
  s = __fadd2_rn(a, b);
  const float2 bb = __ffma2_rn(a, m1, s);                      // s - a
  const float2 u = __ffma2_rn(__ffma2_rn(bb, m1, s), m1, a);   // a - (s - bb)
  const float2 v = __ffma2_rn(bb, m1, b);                      // b - bb
  return __fadd2_rn(u, v);
}

// The NES sums of one row at psi in FP64, as k_assemble forms them (a group whose last correction
// is too large for the FP32-pair increment).  Kept out of line, so that the common path does not
// carry its registers.
__device__ __noinline__ void nes_sums_fp64(const double *__restrict__ fin, const double *__restrict__ fout,
                                           const double *__restrict__ ps, int n, double *gain, double *lp) {
  double a = 0.0, b = 0.0;
  for (int kp = 0; kp < n; ++kp) {
    const double pv = ps[kp];
    a += fin[kp] * pv;
    b += fout[kp] * pv;
  }
  *gain = a;
  *lp = b;
}

// CTAs of 256 threads per SM the residual kernel is compiled for (its register budget).
#ifndef MGFLD_FF_MINB
#define MGFLD_FF_MINB 7
#endif

__global__ void __launch_bounds__(256, MGFLD_FF_MINB)
k_resid_ff(Prob p, Ws w, const double *__restrict__ psi, float *__restrict__ diag, double *__restrict__ lower,
           double *__restrict__ upper, double *__restrict__ rhs, const int *__restrict__ list, int n_list,
           const int *__restrict__ jac_flag, double tolmin, const int *__restrict__ n_dev) {
  extern __shared__ __align__(16) unsigned char ff_sm[];
  const int n = p.n, ld = ff_ld(n), zpb = ff_zpb(n);
  const unsigned zrows = (unsigned)(NS * n), bt = (unsigned)zpb * zrows, nn = (unsigned)(n * n);
  // (16-byte pieces first, then 8-byte, then 4-byte: every array aligned to its element)
  float4 *tile = reinterpret_cast<float4 *>(ff_sm);                       // [zpb][n][ld]
  float2 *dff = reinterpret_cast<float2 *>(tile + (size_t)zpb * n * ld);   // [bt]: (d, -d)
  int2 *rsc = reinterpret_cast<int2 *>(dff + bt);                          // [zpb][n]
  long long *zoff = reinterpret_cast<long long *>(rsc + (size_t)zpb * n);  // [zpb]: zone index ray n_r + i
  unsigned *gmx = reinterpret_cast<unsigned *>(zoff + zpb);                // [zpb NS]: max |dpsi| (upper words)
  unsigned *gpx = gmx + (size_t)zpb * NS;                                  // [zpb NS]: max |psi|
  const unsigned per_ray = (unsigned)p.n_r * zrows;
  const unsigned total = (unsigned)listed(n_list, n_dev) * per_ray;
  const unsigned b0 = blockIdx.x * bt;
  if (b0 >= total) return;                                                 // the whole block
  const unsigned t = b0 + threadIdx.x;
  const bool in = t < total;
  // this row (its loads issued before the staging)
  const unsigned rl = in ? t / per_ray : 0;
  const int ray = list[rl];
  const unsigned local = t - rl * per_ray;
  const unsigned kq = local / (unsigned)n;
  const int k = (int)(local - kq * n);
  const int q = (int)(kq % NS);
  const int i = (int)(kq / NS);
  const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;
  const size_t zi = (size_t)ray * p.n_r + i;
  const int last = p.n_r - 1;
  double dx = 0.0, g0 = 0.0, l0 = 0.0, pk = 0.0;
  if (in) {
    dx = w.x[g];
    g0 = w.g0[g];
    l0 = w.l0[g];
    pk = psi[g];
  }
  // the block's zones (consecutive in the listed order): their indices, scaled kernels, row scales
  const unsigned gz0 = b0 / zrows;
  const unsigned nzb = min((unsigned)zpb, (total - b0 + zrows - 1) / zrows);
  const unsigned grp = threadIdx.x / (unsigned)n;
  if (threadIdx.x < nzb) {
    const unsigned gz = gz0 + threadIdx.x, zr = gz / p.n_r;
    zoff[threadIdx.x] = (long long)list[zr] * p.n_r + (gz - zr * p.n_r);
  }
  if (threadIdx.x < (unsigned)zpb * NS) gmx[threadIdx.x] = gpx[threadIdx.x] = 0u;
  __syncthreads();
  for (unsigned zs = 0; zs < nzb; ++zs) {
    const float4 *src = w.nesff + (size_t)zoff[zs] * nn;
    float4 *dst = tile + (size_t)zs * n * ld;
    for (unsigned e = threadIdx.x; e < nn; e += bt) dst[e + e / (unsigned)n * (unsigned)(ld - n)] = src[e];
    if (threadIdx.x < (unsigned)n) rsc[zs * n + threadIdx.x] = w.nessc[(size_t)zoff[zs] * n + threadIdx.x];
  }
  // the corrections of the block's (zone, species) groups, each scaled by its group's largest
  if (in) {
    atomicMax(&gmx[grp], abs_hi_word(dx));
    atomicMax(&gpx[grp], abs_hi_word(pk));
  }
  __syncthreads();
  const int sgrp = scale_of_max(gmx[grp]);
  {
    // the correction of the mixed path comes from the FP32 substitution (an FP32 value times a
    // power of two), so its scaled FP32 form is exact (the lo part of split_ff is zero)
    const float d = d2f_exp2(dx, sgrp);
    dff[threadIdx.x] = make_float2(d, -d);
  }
  __syncthreads();
  if (!in) return;

  const double *ps = psi + (g - k);
  const unsigned zs = threadIdx.x / zrows;
  double gain, lp;
  // the pairs while the group's last correction is at most 2^-6 (1.6 %) of max(max |psi|, tolmin),
  // by exponents (the same decision for every row of the group)
  if ((int)(gmx[grp] >> 20) + 6 <= (int)(max(gpx[grp], abs_hi_word(tolmin)) >> 20)) {
    const float4 *fr = tile + ((size_t)zs * n + k) * ld;
    const float2 *dr = dff + (size_t)grp * n;
    // (gain, loss) lanes; two running sums (even and odd k') for two independent dependency chains
    float2 s0 = make_float2(0.f, 0.f), s1 = s0, e0 = s0, e1 = s0;
    auto term = [&](int kp, float2 &sum, float2 &err) {
      const float4 f = fr[kp];                       // (in hi, in lo, out hi, out lo)
      const float2 d = dr[kp];                       // (d, -d)
      const float2 fh = make_float2(f.x, f.z), fl = make_float2(f.y, f.w);
      const float2 dh = make_float2(d.x, d.x), nd = make_float2(d.y, d.y);
      const float2 pr = __fmul2_rn(fh, dh);
      const float2 ex = __ffma2_rn(fh, dh, __fmul2_rn(fh, nd));          // exact product error
      const float2 cr = __fmul2_rn(fl, dh);                              // the kernels' lo part
      const float2 e = two_sum2(sum, pr);
      err = __fadd2_rn(err, __fadd2_rn(__fadd2_rn(ex, cr), e));
    };
    int kp = 0;
    for (; kp + 1 < n; kp += 2) {
      term(kp, s0, e0);
      term(kp + 1, s1, e1);
    }
    if (kp < n) term(kp, s0, e0);
    const float2 e01 = two_sum2(s0, s1);
    const float2 er = __fadd2_rn(__fadd2_rn(e0, e1), e01);
    const float2 sm = s0;
    const int2 sc = rsc[zs * n + k];
    const int ug = -(sc.x + sgrp), ul = -(sc.y + sgrp);
    gain = (g0 + f2d_exp2(sm.x, ug)) + f2d_exp2(er.x, ug);
    lp = (l0 + f2d_exp2(sm.y, ul)) + f2d_exp2(er.y, ul);
  } else {
    // a large last correction: the sums at the iterate in FP64, as k_assemble forms them
    nes_sums_fp64(w.phin + (zi * n + k) * n, w.phout + (zi * n + k) * n, ps, n, &gain, &lp);
  }
  w.g0[g] = gain;
  w.l0[g] = lp;

  const double j = w.jbuf[g];
  const double dg = ((w.cdiag[g] + j) + gain) - lp;
  double G = fma(pk, dg, -((w.cb[g] + j) + gain));
  const double c_up = w.cup[g], c_low = w.clow[g];
  if (i < last) G = fma(-c_up, ps[k + n], G);
  if (i > 0) G = fma(-c_low, ps[k - (ptrdiff_t)n], G);
  rhs[g] = -G;

  if (!jac_flag || !jac_flag[ray]) return;
  // a new FP32 Jacobian row for the ray (as k_assemble writes it)
  float *row = diag + g * n;
  const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
  const float pf = d2f_exp2(pk, 0);
  const float dk = fmaf(pf, fd[k], -fi[k]) + (float)dg;
  for (int kp = 0; kp < n; ++kp) row[kp] = kp == k ? dk : fmaf(pf, fd[kp], -fi[kp]);
  lower[g] = -c_low;
  upper[g] = -c_up;
  w.lower32[g] = d2f_exp2(-c_low, 0);
  w.upper32[g] = d2f_exp2(-c_up, 0);
}

cudaError_t launch_resid_ff(const Prob &p, const Ws &w, const double *psi, float *diag, double *lower,
                            double *upper, double *rhs, const int *list, int n_list, const int *jac_flag,
                            double tolmin, cudaStream_t s, const int *n_dev) {
  const size_t zones = (size_t)n_list * p.n_r;
  if (zones == 0) return cudaSuccess;
  const int zpb = ff_zpb(p.n);
  const size_t sm = ff_smem(p.n);
  if (sm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_resid_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_resid_ff<<<(unsigned)((zones + zpb - 1) / zpb), zpb * NS * p.n, sm, s>>>(p, w, psi, diag, lower, upper, rhs,
                                                                            list, n_list, jac_flag, tolmin, n_dev);
  return cudaGetLastError();
}

}  // namespace mgfld
