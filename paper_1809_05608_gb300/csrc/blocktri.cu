// Batched block-Thomas elimination for the per-(ray, species) systems of Eq. a62ae.
//
// Structure exploited: the off-diagonal blocks are diagonal (the flux coefficient is
// frozen), so the Schur update of a zone is a diagonal scaling of its neighbour's
// inverse, e.g. D'_i = D_i - diag(l_i) D'^{-1}_{i-1} diag(u_{i-1}): no dense block product,
// hence no tensor-core contraction on this path.  Each dense block is inverted in
// place by Gauss-Jordan elimination with partial pivoting.
//
// Two-sided ("twisted") elimination: every system is eliminated top-down over zones
// 0..m-1 and bottom-up over zones n_r-1..m+1 at the same time, the two halves meeting at
// the middle zone m = n_r/2, whose block receives both Schur terms.  The substitution runs
// the same way (inward to the middle, then outward).  The sequential chain along the zones,
// which bounds these latency-limited kernels, is half as long, and there are twice as many
// independent instruction streams; the arithmetic is unchanged.
//
// Thread mapping (FP64): one thread per block row, the two halves of SPC/2 systems per CTA
// so that SPC * NP is a multiple of 32 and every lane of every FMA instruction does work.
// Rows and columns beyond the real group count n (<= NP) are padded with the identity.
// The pivot search, pivot-row broadcast and the natural-order inverse go through
// shared memory; the inverse of each zone is streamed to the caller's factor buffer.
#include "mgfld_internal.cuh"

namespace mgfld {

template <int NP>
struct Pack {
  static constexpr int gcd(int a, int b) { return b == 0 ? a : gcd(b, a % b); }
  // Half-systems per CTA: a multiple of 32 threads and even (both halves of a system share a CTA).
  static constexpr int SPC0 = 32 / gcd(NP, 32);
  static constexpr int SPC = SPC0 % 2 == 0 ? SPC0 : 2 * SPC0;
  static constexpr int THREADS = SPC * NP;
};

// 32-bit pivot-search key of row r: the upper word of |x| (sign cleared; non-negative IEEE
// values order like their bit patterns) with its 5 lowest bits replaced by 31 - r.  One integer
// max over the keys then finds the largest |x| to 15 mantissa bits, ties going to the lowest
// row, and the winner's row is 31 - (key & 31).  Rows already used as pivots carry -1.
__device__ inline int pivot_key(double x, int r) {
  const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
  return (int)((hi & ~31u) | (unsigned)(31 - r));
}

template <int NP>
__device__ inline int max_key(const int *__restrict__ c) {
  static_assert(NP % 4 == 0, "padded block sizes are multiples of 4");
  int m[NP / 4];
#pragma unroll
  for (int j = 0; j < NP / 4; ++j) {
    const int4 v = reinterpret_cast<const int4 *>(c)[j];
    m[j] = max(max(v.x, v.y), max(v.z, v.w));
  }
#pragma unroll
  for (int w = 1; w < NP / 4; w *= 2)
#pragma unroll
    for (int j = 0; j + w < NP / 4; j += 2 * w) m[j] = max(m[j], m[j + w]);
  return m[0];
}

// Map the j-th system of the launch to a global (ray, species) system index.
__device__ inline long system_of(long j, const int *ray_list) {
  return ray_list ? (long)ray_list[j / NS] * NS + (j % NS) : j;
}

template <typename T> __device__ inline T to_t(double v);
template <> __device__ inline double to_t<double>(double v) { return v; }
template <> __device__ inline float to_t<float>(double v) { return (float)v; }

// FP64 block-Thomas elimination (one thread per block row, SPC systems per CTA).  Per pivot
// step: barrier; every row reads the NP candidate keys of its system (NP/4 vector loads, a
// depth-log2 max tree); the pivot row publishes itself; barrier; every row forms its multiplier
// with one FMA and updates its NP entries.  The entry of the next pivot column is updated
// first and its key published at once, so that the next search only waits for that one FMA
// while the other NP - 1 drain through the FP64 pipe.
// CTAs per SM the FP64 factor is compiled for (its register budget).
#ifndef MGFLD_FP64_MINB
#define MGFLD_FP64_MINB 4
#endif

template <int NP, typename TIn>
__global__ void __launch_bounds__(Pack<NP>::THREADS, NP <= 20 ? MGFLD_FP64_MINB : 1)
k_factor(int n, int n_r, int n_sys, const TIn *__restrict__ diag, const double *__restrict__ lower,
         const double *__restrict__ upper, double *__restrict__ dinv, const int *__restrict__ ray_list,
         const int *__restrict__ n_dev) {
  constexpr int SPC = Pack<NP>::SPC;
  __shared__ double tile[SPC][NP][NP + 1];           // natural-order inverse of the previous zone
  __shared__ __align__(16) double prow[SPC][NP];     // pivot row of the current step
  __shared__ __align__(16) int cand[SPC][NP];        // pivot-search keys
  __shared__ double ushr[SPC][NP];                   // coupling to the next zone: the column scaling of its Schur term
  __shared__ int pivrow[SPC][NP];                    // row chosen at each step
  __shared__ double pinv[SPC];                       // 1 / pivot of the current step

  const int s = threadIdx.x / NP, r = threadIdx.x % NP;
  const int half = s & 1;                            // 0: zones 0..m top-down, 1: zones n_r-1..m+1 bottom-up
  const int n_sys_e = listed_sys(n_sys, n_dev, NS);
  if ((long)blockIdx.x * (SPC / 2) >= n_sys_e) return;   // the whole CTA
  const long jsys = (long)blockIdx.x * (SPC / 2) + (s >> 1);
  const bool valid = jsys < n_sys_e;
  const long sys = valid ? system_of(jsys, ray_list) : 0;
  const int m = n_r / 2;
  const int len = half == 0 ? m + 1 : n_r - 1 - m;   // zones of this half; all threads step m + 1 times

  // Each zone's rows are loaded when the zone starts: an FP64 zone step holds the pipe for far
  // longer than a memory round trip, and the registers of a prefetch would cost resident CTAs.
  for (int j = 0; j <= m; ++j) {
    const bool active = j < len;                     // inactive (bottom half, j >= len): dummy identity
    const int i = half == 0 ? j : n_r - 1 - j;
    const bool real = valid && active && r < n;
    const size_t zrow = ((size_t)sys * n_r + (real ? i : 0)) * n + r;   // (sys, i, r)
    double a[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) a[c] = (real && c < n) ? (double)diag[zrow * n + c] : ((c == r) ? 1.0 : 0.0);
    const double lr = (real && j > 0) ? (half == 0 ? lower[zrow] : upper[zrow]) : 0.0;
    if (j > 0 && active) {
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = fma(-(lr * tile[s][r][c]), ushr[s][c], a[c]);
    }
    if (half == 0 && j == m && n_r - 1 > m) {
      // Middle zone: also subtract the bottom-up half's term diag(u_m) D''^{-1}_{m+1} diag(l_{m+1})
      // (that half finished at step len - 1 < m; its tile and coupling are kept).
      const double um = real ? upper[zrow] : 0.0;
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = fma(-(um * tile[s + 1][r][c]), ushr[s + 1][c], a[c]);
    }

    // Gauss-Jordan inversion in place with partial pivoting (implicit row exchanges).
    bool used = false;
    int my_step = 0;
    cand[s][r] = pivot_key(a[0], r);
#pragma unroll
    for (int pstep = 0; pstep < NP; ++pstep) {
      __syncthreads();
      const int best = 31 - (max_key<NP>(cand[s]) & 31);
      const bool me = (r == best);
      if (me) {
        // The pivot entry was updated first in the previous step, so its reciprocal is
        // formed while the rest of this row is still in the FP64 pipe.
        pinv[s] = recip(a[pstep]);
#pragma unroll
        for (int c = 0; c < NP; c += 2)
          *reinterpret_cast<double2 *>(&prow[s][c]) = make_double2(a[c], a[c + 1]);
        pivrow[s][pstep] = r;
        used = true;
        my_step = pstep;
      }
      __syncthreads();
      const double inv = pinv[s];
      // Uniform update for every row: a -= f * pivot_row, with f chosen so that the pivot row
      // itself becomes pivot_row / pivot (f = 1 - 1/pivot): one FMA either way.  The pivot
      // column itself is overwritten below, so its update is skipped.
      const double f = fma(me ? -1.0 : a[pstep], inv, me ? 1.0 : 0.0);
      if (pstep + 1 < NP) {
        a[pstep + 1] = fma(-f, prow[s][pstep + 1], a[pstep + 1]);
        cand[s][r] = used ? -1 : pivot_key(a[pstep + 1], r);
      }
      // the rest of the pivot row read from shared memory as it is used (16-byte pieces)
#pragma unroll
      for (int c = 0; c < NP; c += 2) {
        const double2 v = *reinterpret_cast<const double2 *>(&prow[s][c]);
        if (c != pstep + 1 && c != pstep) a[c] = fma(-f, v.x, a[c]);
        if (c + 1 != pstep + 1 && c + 1 != pstep) a[c + 1] = fma(-f, v.y, a[c + 1]);
      }
      a[pstep] = me ? inv : -f;
    }
    // Row r now holds row my_step of the inverse, with column c belonging to input row pivrow[c].
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < NP; ++c) tile[s][my_step][pivrow[s][c]] = a[c];
      ushr[s][r] = real ? (half == 0 ? upper[zrow] : lower[zrow]) : 0.0;
    }
    __syncthreads();
    if (real) {
      double *out = dinv + zrow * n;
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c < n) out[c] = tile[s][r][c];
    }
  }
}

// FP64 forward and back substitution with the twisted factors (one thread per block row, the
// two halves of each system in the same CTA, stepping together): forward g_i = Dinv_i (r_i -
// l_i g_{i-1}) for i < m and h_i = Dinv_i (r_i - u_i h_{i+1}) for i > m, the middle
// x_m = Dinv_m (r_m - l_m g_{m-1} - u_m h_{m+1}), then back outward from m.  The forward results
// are kept in x (which may alias rhs: each zone's rhs is read before its x is written).
template <int NP>
__global__ void __launch_bounds__(Pack<NP>::THREADS)
k_solve(int n, int n_r, int n_sys, const double *__restrict__ dinv, const double *__restrict__ lower,
        const double *__restrict__ upper, const double *rhs, double *x, const int *__restrict__ ray_list,
        const int *__restrict__ n_dev) {
  constexpr int SPC = Pack<NP>::SPC;
  __shared__ double v[SPC][NP];
  __shared__ double mid[SPC / 2][NP];               // h_{m+1}, then x_m
  const int s = threadIdx.x / NP, r = threadIdx.x % NP;
  const int half = s & 1, sl = s >> 1;
  const int n_sys_e = listed_sys(n_sys, n_dev, NS);
  if ((long)blockIdx.x * (SPC / 2) >= n_sys_e) return;   // the whole CTA
  const long jsys = (long)blockIdx.x * (SPC / 2) + sl;
  const bool valid = jsys < n_sys_e;
  const long sys = valid ? system_of(jsys, ray_list) : 0;
  const bool realr = valid && r < n;
  const size_t base = (size_t)sys * n_r * n;
  const int m = n_r / 2, B = n_r - 1 - m;
  const int F = half == 0 ? m : B;

  auto rowdot = [&](int z, bool real) {
    const double *src = dinv + (base + (size_t)z * n + r) * n;
    double acc0 = 0.0, acc1 = 0.0;
    if (real) {
#pragma unroll
      for (int c = 0; c < NP; c += 2) {
        if (c < n) acc0 = fma(src[c], v[s][c], acc0);
        if (c + 1 < n) acc1 = fma(src[c + 1], v[s][c + 1], acc1);
      }
    }
    return acc0 + acc1;
  };
  // Forward (all threads step m times for the barriers; a half past its F steps idles).
  double prev = 0.0;
  for (int j = 0; j < m; ++j) {
    const bool act = j < F;
    const bool real = realr && act;
    const int z = half == 0 ? j : n_r - 1 - j;
    const size_t zr = base + (size_t)(real ? z : 0) * n + r;
    const double c = (real && j > 0) ? (half == 0 ? lower[zr] : upper[zr]) : 0.0;
    const double b = real ? rhs[zr] : 0.0;
    v[s][r] = real ? b - c * prev : 0.0;
    __syncthreads();
    const double g = rowdot(z, real);
    if (real) {
      x[zr] = g;
      prev = g;
    }
    __syncthreads();
  }
  if (half == 1) mid[sl][r] = B > 0 ? prev : 0.0;
  __syncthreads();
  if (half == 0) {
    const size_t zr = base + (size_t)m * n + r;
    const double l = (realr && m > 0) ? lower[zr] : 0.0;
    const double u = (realr && m < n_r - 1) ? upper[zr] : 0.0;
    v[s][r] = realr ? rhs[zr] - l * prev - u * mid[sl][r] : 0.0;
  }
  __syncthreads();
  if (half == 0) {
    const double xm = rowdot(m, realr);
    if (realr) x[base + (size_t)m * n + r] = xm;
    prev = xm;
  }
  __syncthreads();
  if (half == 0) mid[sl][r] = prev;
  __syncthreads();
  if (half == 1) prev = mid[sl][r];
  // Backward: top x_i = g_i - Dinv_i (u_i x_{i+1}), i = m-1..0; bottom x_i = h_i - Dinv_i (l_i x_{i-1}).
  for (int j = 0; j < m; ++j) {
    const bool act = j < F;
    const bool real = realr && act;
    const int z = half == 0 ? m - 1 - j : m + 1 + j;
    const size_t zr = base + (size_t)(real ? z : 0) * n + r;
    const double c = real ? (half == 0 ? upper[zr] : lower[zr]) : 0.0;
    v[s][r] = real ? c * prev : 0.0;
    __syncthreads();
    const double acc = rowdot(z, real);
    if (real) {
      const double xi = x[zr] - acc;
      x[zr] = xi;
      prev = xi;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Thread-per-row elimination and substitution for systems of any block width up to 64 rows
// (the coupled nu / antinu blocks of the pair process: 2 n_e rows), in FP64 or FP32, with
// `spr` systems per ray (the launch's j-th system is system j % spr of ray ray_list[j / spr]).
// Same algorithm and thread mapping as k_factor / k_solve above: partial pivoting through integer
// keys (6 row bits for blocks wider than 32), the next zone's rows fetched one zone ahead, the
// pivot row read from shared memory where it is used; shared memory sized at launch.
template <int NP, typename T>
struct RowCta {
  static constexpr int gcd(int a, int b) { return b == 0 ? a : gcd(b, a % b); }
  static constexpr int SPC0 = 32 / gcd(NP, 32);
  static constexpr int SPC = SPC0 % 2 == 0 ? SPC0 : 2 * SPC0;   // half-systems per CTA (even)
  static constexpr int THREADS = SPC * NP;
  static constexpr int KB = NP > 32 ? 6 : 5;                     // row bits of a pivot key
  static constexpr size_t TILE = sizeof(T) * SPC * NP * (NP + 1); // natural-order inverse of the previous zone
  static constexpr size_t PROW = sizeof(T) * SPC * NP;           // pivot row of the current step
  static constexpr size_t USHR = sizeof(T) * SPC * NP;           // column scaling of the next zone's Schur term
  static constexpr size_t PINV = 16 * SPC;                       // 1 / pivot (16-byte slots)
  static constexpr size_t CAND = sizeof(int) * SPC * NP;         // pivot-search keys
  static constexpr size_t PIVR = sizeof(int) * SPC * NP;         // row chosen at each step
  static constexpr size_t BYTES = TILE + PROW + USHR + PINV + CAND + PIVR;
};

__device__ inline long system_of_spr(long j, const int *ray_list, int spr) {
  return ray_list ? (long)ray_list[j / spr] * spr + (j % spr) : j;
}

template <int KB> __device__ inline int row_key(double x, int r) {
  const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
  return (int)((hi & ~((1u << KB) - 1u)) | (unsigned)((1 << KB) - 1 - r));
}
template <int KB> __device__ inline int row_key(float x, int r) {
  const unsigned b = (unsigned)__float_as_int(x) & 0x7fffffffu;
  return (int)((b & ~((1u << KB) - 1u)) | (unsigned)((1 << KB) - 1 - r));
}
__device__ inline double recip_t(double d) { return recip(d); }
__device__ inline float recip_t(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  const float e = fmaf(-d, r, 1.f);
  return isfinite(r) ? fmaf(r, e, r) : r;
}

template <int NP, typename TIn, typename T>
__global__ void __launch_bounds__(RowCta<NP, T>::THREADS)
k_factor_rows(int n, int n_r, int n_sys, int spr, const TIn *__restrict__ diag, const T *__restrict__ lower,
              const T *__restrict__ upper, T *__restrict__ dinv, const int *__restrict__ ray_list,
              const int *__restrict__ n_dev) {
  using C = RowCta<NP, T>;
  constexpr int SPC = C::SPC, KB = C::KB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*tile)[NP][NP + 1] = reinterpret_cast<T (*)[NP][NP + 1]>(smem_raw);
  T (*prow)[NP] = reinterpret_cast<T (*)[NP]>(smem_raw + C::TILE);
  T (*ushr)[NP] = reinterpret_cast<T (*)[NP]>(smem_raw + C::TILE + C::PROW);
  T *pinv = reinterpret_cast<T *>(smem_raw + C::TILE + C::PROW + C::USHR);          // stride 16 bytes
  int (*cand)[NP] = reinterpret_cast<int (*)[NP]>(smem_raw + C::TILE + C::PROW + C::USHR + C::PINV);
  int (*pivrow)[NP] = reinterpret_cast<int (*)[NP]>(smem_raw + C::TILE + C::PROW + C::USHR + C::PINV + C::CAND);
  constexpr int PS = 16 / sizeof(T);                 // pinv slot stride in elements

  const int s = threadIdx.x / NP, r = threadIdx.x % NP;
  const int half = s & 1;                            // 0: zones 0..m top-down, 1: zones n_r-1..m+1 bottom-up
  const int n_sys_e = listed_sys(n_sys, n_dev, spr);
  if ((long)blockIdx.x * (SPC / 2) >= n_sys_e) return;   // the whole CTA
  const long jsys = (long)blockIdx.x * (SPC / 2) + (s >> 1);
  const bool valid = jsys < n_sys_e;
  const long sys = valid ? system_of_spr(jsys, ray_list, spr) : 0;
  const int m = n_r / 2;
  const int len = half == 0 ? m + 1 : n_r - 1 - m;   // zones of this half; all threads step m + 1 times
  const T one = T(1), zero = T(0);

  T nxt[NP];
  T nl = zero;
  auto load_row = [&](int j) {
    const bool act = valid && j < len && r < n;
    const int z = half == 0 ? j : n_r - 1 - j;
    const size_t zr = ((size_t)sys * n_r + (act ? z : 0)) * n + r;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      if (act && c < n) nxt[c] = (T)diag[zr * n + c];
      else nxt[c] = (c == r) ? one : zero;
    }
    nl = (act && j > 0) ? (half == 0 ? lower[zr] : upper[zr]) : zero;
  };
  load_row(0);
  for (int j = 0; j <= m; ++j) {
    const bool active = j < len;
    const int i = half == 0 ? j : n_r - 1 - j;
    const bool real = valid && active && r < n;
    const size_t zrow = ((size_t)sys * n_r + (real ? i : 0)) * n + r;
    T a[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) a[c] = nxt[c];
    const T lr = nl;
    if (j + 1 <= m) load_row(j + 1);
    if (j > 0 && active) {
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = fma(-(lr * tile[s][r][c]), ushr[s][c], a[c]);
    }
    if (half == 0 && j == m && n_r - 1 > m) {
      const T um = real ? upper[zrow] : zero;
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = fma(-(um * tile[s + 1][r][c]), ushr[s + 1][c], a[c]);
    }
    bool used = false;
    int my_step = 0;
    cand[s][r] = row_key<KB>(a[0], r);
#pragma unroll
    for (int pstep = 0; pstep < NP; ++pstep) {
      __syncthreads();
      int best_key = cand[s][0];
#pragma unroll
      for (int c = 1; c < NP; ++c) best_key = max(best_key, cand[s][c]);
      const int best = (1 << KB) - 1 - (best_key & ((1 << KB) - 1));
      const bool me = (r == best);
      if (me) {
        pinv[s * PS] = recip_t(a[pstep]);
#pragma unroll
        for (int c = 0; c < NP; ++c) prow[s][c] = a[c];
        pivrow[s][pstep] = r;
        used = true;
        my_step = pstep;
      }
      __syncthreads();
      const T inv = pinv[s * PS];
      const T f = fma(me ? -one : a[pstep], inv, me ? one : zero);
      if (pstep + 1 < NP) {
        a[pstep + 1] = fma(-f, prow[s][pstep + 1], a[pstep + 1]);
        cand[s][r] = used ? -1 : row_key<KB>(a[pstep + 1], r);
      }
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c != pstep + 1 && c != pstep) a[c] = fma(-f, prow[s][c], a[c]);
      a[pstep] = me ? inv : -f;
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < NP; ++c) tile[s][my_step][pivrow[s][c]] = a[c];
      ushr[s][r] = real ? (half == 0 ? upper[zrow] : lower[zrow]) : zero;
    }
    __syncthreads();
    if (real) {
      T *out = dinv + zrow * n;
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c < n) out[c] = tile[s][r][c];
    }
  }
}

// Substitution with those factors (twisted, as k_solve).  FP64: rhs and x as given.  FP32: the
// right-hand side arrives scaled by 2^k per system and rounded to FP32 (rhs32, k in sys_exp, from
// k_sysmax), the sweeps run in FP32 and x is scaled back by an exact multiplication by 2^-k; the
// forward results are kept in x (in the scaled units) until the backward sweep replaces them.
template <int NP, typename T>
__global__ void __launch_bounds__(RowCta<NP, T>::THREADS)
k_solve_rows(int n, int n_r, int n_sys, int spr, const T *__restrict__ dinv, const T *__restrict__ lower,
             const T *__restrict__ upper, const double *rhs, const float *__restrict__ rhs32,
             const int *__restrict__ sys_exp, double *x, const int *__restrict__ ray_list,
             const int *__restrict__ n_dev) {
  constexpr int SPC = RowCta<NP, T>::SPC;
  __shared__ T v[SPC][NP];
  __shared__ T mid[SPC / 2][NP];
  const int s = threadIdx.x / NP, r = threadIdx.x % NP;
  const int half = s & 1, sl = s >> 1;
  const int n_sys_e = listed_sys(n_sys, n_dev, spr);
  if ((long)blockIdx.x * (SPC / 2) >= n_sys_e) return;   // the whole CTA
  const long jsys = (long)blockIdx.x * (SPC / 2) + sl;
  const bool valid = jsys < n_sys_e;
  const long sys = valid ? system_of_spr(jsys, ray_list, spr) : 0;
  const bool realr = valid && r < n;
  const size_t base = (size_t)sys * n_r * n;
  const int m = n_r / 2, B = n_r - 1 - m;
  const int F = half == 0 ? m : B;
  const bool f32 = sizeof(T) == 4;
  const double unscale = (f32 && valid) ? ldexp(1.0, -sys_exp[jsys]) : 1.0;
  const T zero = T(0);
  auto b_at = [&](size_t zr) -> T { return f32 ? (T)rhs32[zr] : (T)rhs[zr]; };
  auto rowdot = [&](int z, bool real) {
    const T *src = dinv + (base + (size_t)z * n + r) * n;
    T acc0 = zero, acc1 = zero;
    if (real) {
#pragma unroll
      for (int c = 0; c < NP; c += 2) {
        if (c < n) acc0 = fma(src[c], v[s][c], acc0);
        if (c + 1 < n) acc1 = fma(src[c + 1], v[s][c + 1], acc1);
      }
    }
    return acc0 + acc1;
  };
  T prev = zero;
  for (int j = 0; j < m; ++j) {
    const bool act = j < F;
    const bool real = realr && act;
    const int z = half == 0 ? j : n_r - 1 - j;
    const size_t zr = base + (size_t)(real ? z : 0) * n + r;
    const T c = (real && j > 0) ? (half == 0 ? lower[zr] : upper[zr]) : zero;
    const T b = real ? b_at(zr) : zero;
    v[s][r] = real ? b - c * prev : zero;
    __syncthreads();
    const T g = rowdot(z, real);
    if (real) {
      x[zr] = (double)g;
      prev = g;
    }
    __syncthreads();
  }
  if (half == 1) mid[sl][r] = B > 0 ? prev : zero;
  __syncthreads();
  if (half == 0) {
    const size_t zr = base + (size_t)m * n + r;
    const T l = (realr && m > 0) ? lower[zr] : zero;
    const T u = (realr && m < n_r - 1) ? upper[zr] : zero;
    v[s][r] = realr ? b_at(zr) - l * prev - u * mid[sl][r] : zero;
  }
  __syncthreads();
  if (half == 0) {
    const T xm = rowdot(m, realr);
    if (realr) x[base + (size_t)m * n + r] = (double)xm * unscale;
    prev = xm;
  }
  __syncthreads();
  if (half == 0) mid[sl][r] = prev;
  __syncthreads();
  if (half == 1) prev = mid[sl][r];
  for (int j = 0; j < m; ++j) {
    const bool act = j < F;
    const bool real = realr && act;
    const int z = half == 0 ? m - 1 - j : m + 1 + j;
    const size_t zr = base + (size_t)(real ? z : 0) * n + r;
    const T c = real ? (half == 0 ? upper[zr] : lower[zr]) : zero;
    v[s][r] = real ? c * prev : zero;
    __syncthreads();
    const T acc = rowdot(z, real);
    if (real) {
      const T xi = (T)x[zr] - acc;
      x[zr] = (double)xi * unscale;
      prev = xi;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Warp-synchronous FP32 variants (MIXED precision): one warp per half of a (ray, species)
// system, lane r owns block row r (NP <= 32), no CTA-wide barriers.  FP32 arithmetic is 63x
// cheaper than FP64 on this GPU, so these kernels are bound by the dependency chain along the
// zones and by the instruction and shared-memory traffic of each zone step.
constexpr int kWarpsPerCta = 4;

// Per-thread 16-byte asynchronous global-to-shared copies (completion waited by the issuing thread).
__device__ inline void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ inline void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ inline void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
// one element of 4 or 8 bytes
template <typename TE> __device__ inline void cp_async_elem(TE *dst, const TE *src) {
  if constexpr (sizeof(TE) == 4) cp_async4(dst, src);
  else cp_async8(dst, src);
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
template <int N> __device__ inline void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// FP32 reciprocal: the hardware approximation (rcp.approx.ftz) refined by one Newton step, a
// few multiply-adds instead of the correctly rounded library reciprocal; ample for the FP32
// preconditioner.  rcp(0) = inf and rcp(NaN) = NaN as before.
__device__ inline float rcp_nr(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  const float e = fmaf(-x, r, 1.f);
  return isfinite(r) ? fmaf(r, e, r) : r;
}

// Packed FP32 helpers (two lanes of arithmetic per instruction).
__device__ inline void fma2_row(float *a, float s, const float *p, int c) {
  const float2 r = __ffma2_rn(make_float2(s, s), make_float2(p[c], p[c + 1]), make_float2(a[c], a[c + 1]));
  a[c] = r.x;
  a[c + 1] = r.y;
}

// In-place Gauss-Jordan inverse with partial pivoting of the warp's NP x NP zone block, lane r
// holding row r.  The pivot is found with a warp max reduction on integer keys (|a| bits with
// the row index in the 5 low bits), the pivot row is broadcast through a double-buffered
// shared-memory row (one 16-byte store per 4 entries by its owner, broadcast 16-byte loads by
// every lane), and the eliminations run as packed FP32 FMAs.  Returns with a[] holding row
// my_step of the inverse with column c belonging to natural column piv(c) (byte c % 4 of
// piv[c / 4]).
template <int NP>
__device__ inline void gj_invert(float *a, float (*prow)[NP + 4], int r, bool row, int &my_step, unsigned *piv) {
  const unsigned full = 0xffffffffu;
  bool used = !row;
  my_step = 0;
  int key = used ? -1 : (int)(((unsigned)__float_as_int(fabsf(a[0])) & ~31u) | (unsigned)(31 - r));
#pragma unroll
  for (int ps = 0; ps < NP; ++ps) {
    const int best = 31 - (__reduce_max_sync(full, key) & 31);
    if (ps % 4 == 0) piv[ps / 4] = (unsigned)best;      // four 8-bit pivot rows per register
    else piv[ps / 4] |= (unsigned)best << (8 * (ps % 4));
    const bool me = (r == best);
    float *pb = prow[ps & 1];
    if (me) {
      used = true;
      my_step = ps;
#pragma unroll
      for (int c = 0; c < NP; c += 4)
        *reinterpret_cast<float4 *>(pb + c) = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
    }
    __syncwarp();
    float pv[NP];
#pragma unroll
    for (int c = 0; c < NP; c += 4) {
      const float4 v = *reinterpret_cast<const float4 *>(pb + c);
      pv[c] = v.x;
      pv[c + 1] = v.y;
      pv[c + 2] = v.z;
      pv[c + 3] = v.w;
    }
    const float inv = rcp_nr(pv[ps]);
    const float f = fmaf(me ? -1.f : a[ps], inv, me ? 1.f : 0.f);
    // the pair holding the next pivot column first, so that the next search can start
    if (ps + 1 < NP) {
      const int cn = (ps + 1) & ~1;
      fma2_row(a, -f, pv, cn);
      key = used ? -1 : (int)(((unsigned)__float_as_int(fabsf(a[ps + 1])) & ~31u) | (unsigned)(31 - r));
#pragma unroll
      for (int c = 0; c < NP; c += 2)
        if (c != cn) fma2_row(a, -f, pv, c);
    } else {
#pragma unroll
      for (int c = 0; c < NP; c += 2) fma2_row(a, -f, pv, c);
    }
    a[ps] = me ? inv : -f;
  }
}

// In-place Gauss-Jordan inverse without row exchanges, lane r holding row r, with 2 x 2 pivot
// blocks: at step b the owners of rows p = 2b and p + 1 publish both rows (double-buffered
// shared memory), every lane forms the inverse of the pivot block
// P = [[d00, d01], [d10, d11]] in closed form (one reciprocal of its determinant) and eliminates
// with the two multipliers (a_p, a_{p+1}) P^{-1}; the owners take the rows of P^{-1} times the
// pivot rows by the same formula.  Half as many broadcast steps on the chain of each block, the
// same number of FMAs.  Leading 2 x 2 blocks of the Schur complements of an M-matrix (or of a
// column diagonally dominant matrix) are nonsingular, so no exchanges are needed; returns false
// (the same in every lane) when a determinant was zero or not finite.  NP must be even.
template <int NP>
__device__ inline bool gj_invert_np2(float *a, float (*prow)[2][NP + 4], int r) {
  static_assert(NP % 4 == 0, "pivot pairs inside 16-byte pieces");
  bool ok = true;
#pragma unroll
  for (int b = 0; b < NP / 2; ++b) {
    const int p = 2 * b;
    float (*pb)[NP + 4] = prow[b & 1];
    if (r == p || r == p + 1) {
      float *dst = pb[r - p];
#pragma unroll
      for (int c = 0; c < NP; c += 2) *reinterpret_cast<float2 *>(dst + c) = make_float2(a[c], a[c + 1]);
    }
    __syncwarp();
    // the pivot block (columns p, p + 1 of both pivot rows) first
    const float2 q0 = *reinterpret_cast<const float2 *>(&pb[0][p]);
    const float2 q1 = *reinterpret_cast<const float2 *>(&pb[1][p]);
    const float det = fmaf(q0.x, q1.y, -(q0.y * q1.x));
    const float idet = rcp_nr(det);
    ok = ok && isfinite(idet) && det != 0.f;
    const float i00 = q1.y * idet, i01 = -q0.y * idet, i10 = -q1.x * idet, i11 = q0.x * idet;
    float f0, f1;
    if (r == p) {
      f0 = 1.f - i00;
      f1 = -i01;
    } else if (r == p + 1) {
      f0 = -i10;
      f1 = 1.f - i11;
    } else {
      f0 = fmaf(a[p], i00, a[p + 1] * i10);
      f1 = fmaf(a[p], i01, a[p + 1] * i11);
    }
#pragma unroll
    for (int c = 0; c < NP; c += 4) {
      const float4 v0 = *reinterpret_cast<const float4 *>(&pb[0][c]);
      const float4 v1 = *reinterpret_cast<const float4 *>(&pb[1][c]);
      float2 lo = __ffma2_rn(make_float2(-f0, -f0), make_float2(v0.x, v0.y), make_float2(a[c], a[c + 1]));
      float2 hi = __ffma2_rn(make_float2(-f0, -f0), make_float2(v0.z, v0.w), make_float2(a[c + 2], a[c + 3]));
      lo = __ffma2_rn(make_float2(-f1, -f1), make_float2(v1.x, v1.y), lo);
      hi = __ffma2_rn(make_float2(-f1, -f1), make_float2(v1.z, v1.w), hi);
      a[c] = lo.x;
      a[c + 1] = lo.y;
      a[c + 2] = hi.x;
      a[c + 3] = hi.y;
    }
    if (r == p) {
      a[p] = i00;
      a[p + 1] = i01;
    } else if (r == p + 1) {
      a[p] = i10;
      a[p + 1] = i11;
    } else {
      a[p] = -f0;
      a[p + 1] = -f1;
    }
  }
  return __all_sync(0xffffffffu, ok);
}

// CTAs per SM the FP32 factor is compiled for (its register budget): the kernel is bound by the
// latency of its pivot chain, so resident warps matter more than a few spilled registers.
#ifndef MGFLD_FW32_MINB
#define MGFLD_FW32_MINB 4
#endif

// Warps per CTA of the factor: four (two systems), two for the widest blocks so that the
// static shared memory (two row buffers and the inverse tile per warp) stays under 48 KB.
template <int NP> __host__ __device__ constexpr int fw_wpc() { return NP > 24 ? 2 : 4; }

// At most 128 registers (NP <= 24), so that four CTAs (eight systems) fit on an SM and the
// 256-ray workload's 512 CTAs run in a single wave on 152 SMs.
// PIVOT: partial pivoting in every zone (the C ABI's factor of arbitrary systems); otherwise
// elimination without row exchanges (the outer iteration's M-matrix blocks, see gj_invert_np2)
// with partial pivoting only for a zone whose unpivoted elimination met a zero or non-finite
// pivot.
template <int NP, typename TIn, typename TC, bool PIVOT>
__global__ void __launch_bounds__(fw_wpc<NP>() * 32, MGFLD_FW32_MINB)
k_factor_w32(int n, int n_r, int n_sys, const TIn *__restrict__ diag, const TC *__restrict__ lower,
             const TC *__restrict__ upper, float *__restrict__ dinv, const int *__restrict__ ray_list,
             const int *__restrict__ n_dev) {
  static_assert(NP % 4 == 0, "rows of NP floats in 16-byte pieces");
  // tile: the natural-order inverse of each warp's last zone (read by the other half at the
  // middle zone); ushr: that zone's coupling to the next zone of the sequence; prow: pivot rows.
  constexpr int W = fw_wpc<NP>();
  __shared__ __align__(16) float tile[W][NP][NP];
  __shared__ __align__(16) float ushr[W][NP];
  __shared__ __align__(16) float prow[W][2][NP + 4];
  __shared__ __align__(16) float prow2[W][2][2][NP + 4];
  __shared__ __align__(16) float rowbuf[W][2][NP][NP];
  __shared__ __align__(16) TC cplb[W][2][2][32];      // per lane: the next zone's couplings (rows path)
  const int wid = threadIdx.x >> 5, r = threadIdx.x & 31;
  const int half = wid & 1;                          // 0: zones 0..m top-down, 1: zones n_r-1..m+1 bottom-up
  const long jsys = (long)blockIdx.x * (W / 2) + (wid >> 1);
  if (jsys >= listed_sys(n_sys, n_dev, NS)) return;  // both warps of the system leave; no barrier below
  const long sys = system_of(jsys, ray_list);
  const bool real = r < n;
  const bool row = r < NP;
  const bool vec = (n == NP) && sizeof(TIn) == 4;    // 16-byte row loads and stores
  const int m = n_r / 2;
  const int len = half == 0 ? m + 1 : n_r - 1 - m;
  auto zone = [&](int j) { return half == 0 ? j : n_r - 1 - j; };
  // Next zone's rows, fetched one zone ahead into a double-buffered shared-memory block (each
  // lane its own row: 16-byte asynchronous copies on the fast path, so no registers hold the
  // prefetch), and its couplings into registers.  The coupling loads are unconditional (lanes
  // without a row read row 0) with the conditions applied when the values are consumed, so that
  // no instruction waits on a load in the zone it was issued.
  const int rr = real ? r : 0;
  TC nl_raw = TC(0), nu_raw = TC(0);
  auto load_row = [&](int j) {
    const int z = zone(j);
    const size_t zr = ((size_t)sys * n_r + z) * n + rr;
    float *dst = &rowbuf[wid][j & 1][row ? r : 0][0];
    if (vec) {
      if (row) {
#pragma unroll
        for (int c = 0; c < NP; c += 4) cp_async16(dst + c, diag + zr * n + c);
      }
      // couplings to the previous zone of this half's sequence (row scaling of its Schur term)
      // and to the next one (column scaling of this zone's Schur term), in the same copy group
      cp_async_elem(&cplb[wid][j & 1][0][r], (half == 0 ? lower : upper) + zr);
      cp_async_elem(&cplb[wid][j & 1][1][r], (half == 0 ? upper : lower) + zr);
      cp_async_commit();
    } else {
      if (row) {
#pragma unroll
        for (int c = 0; c < NP; ++c) dst[c] = (real && c < n) ? (float)diag[zr * n + c] : ((c == r) ? 1.f : 0.f);
      }
      nl_raw = half == 0 ? lower[zr] : upper[zr];
      nu_raw = half == 0 ? upper[zr] : lower[zr];
    }
  };
  if (len > 0) load_row(0);
  for (int j = 0; j < len; ++j) {
    const int z = zone(j);
    const size_t zrow = ((size_t)sys * n_r + z) * n + r;
    if (vec) {
      cp_async_wait_all();
      nl_raw = cplb[wid][j & 1][0][r];
      nu_raw = cplb[wid][j & 1][1][r];
    }
    const float lr = (real && j > 0) ? (float)nl_raw : 0.f;
    const float ur = real ? (float)nu_raw : 0.f;
    if (j + 1 < len) load_row(j + 1);
    // Middle zone: wait for the bottom-up half of this system (its last tile and coupling).
    const bool mid = half == 0 && j == m;
    if (mid) asm volatile("bar.sync %0, 64;" ::"r"(1 + (wid >> 1)) : "memory");
    float a[NP];
    // The zone's Schur complement from its raw rows (still in the row buffer) and the previous
    // zone's inverse (still in this warp's tile), so that it can be rebuilt for the fallback.
    auto build_a = [&]() {
      if (row) {
#pragma unroll
        for (int c = 0; c < NP; c += 4) {
          const float4 v = *reinterpret_cast<const float4 *>(&rowbuf[wid][j & 1][r][c]);
          a[c] = v.x;
          a[c + 1] = v.y;
          a[c + 2] = v.z;
          a[c + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < NP; ++c) a[c] = 0.f;
      }
      if (j > 0 && row) {
        // a -= diag(l) Dinv_prev diag(u_prev): row scale lr, column scale ushr
#pragma unroll
        for (int c = 0; c < NP; c += 4) {
          const float4 u = *reinterpret_cast<const float4 *>(&ushr[wid][c]);
          const float4 d = *reinterpret_cast<const float4 *>(&tile[wid][r][c]);
          const float2 t0 = __fmul2_rn(make_float2(-lr, -lr), make_float2(d.x, d.y));
          const float2 t1 = __fmul2_rn(make_float2(-lr, -lr), make_float2(d.z, d.w));
          const float2 r0 = __ffma2_rn(t0, make_float2(u.x, u.y), make_float2(a[c], a[c + 1]));
          const float2 r1 = __ffma2_rn(t1, make_float2(u.z, u.w), make_float2(a[c + 2], a[c + 3]));
          a[c] = r0.x;
          a[c + 1] = r0.y;
          a[c + 2] = r1.x;
          a[c + 3] = r1.y;
        }
      }
      if (mid && n_r - 1 > m && row) {
        // the bottom-up half's Schur term diag(u_m) D''^{-1}_{m+1} diag(l_{m+1}) as well
#pragma unroll
        for (int c = 0; c < NP; ++c) a[c] = a[c] - (ur * tile[wid ^ 1][r][c]) * ushr[wid ^ 1][c];
      }
    };
    build_a();
    const bool ok = PIVOT ? false : gj_invert_np2<NP>(a, prow2[wid], r);
    __syncwarp();                  // every lane has read the previous zone's tile row
    if (ok) {
      if (row) {
#pragma unroll
        for (int c = 0; c < NP; c += 2) *reinterpret_cast<float2 *>(&tile[wid][r][c]) = make_float2(a[c], a[c + 1]);
      }
    } else {
      // pivoting requested, or a zero or non-finite pivot: the block with partial pivoting
      if (!PIVOT) build_a();
      int my_step;
      unsigned piv[NP / 4];
      gj_invert<NP>(a, prow[wid], r, row, my_step, piv);
      __syncwarp();
      if (row) {
#pragma unroll
        for (int c = 0; c < NP; ++c) tile[wid][my_step][(piv[c / 4] >> (8 * (c % 4))) & 0xffu] = a[c];
      }
    }
    __syncwarp();
    if (row) ushr[wid][r] = ur;   // column scaling of this zone's Schur term in the next zone
    if (real) {
      float *out = dinv + zrow * n;
      if (vec) {
#pragma unroll
        for (int c = 0; c < NP; c += 4)
          *reinterpret_cast<float4 *>(out + c) = *reinterpret_cast<const float4 *>(&tile[wid][r][c]);
      } else {
#pragma unroll
        for (int c = 0; c < NP; ++c)
          if (c < n) out[c] = tile[wid][r][c];
      }
    }
    __syncwarp();
  }
  if (half == 1) asm volatile("bar.sync %0, 64;" ::"r"(1 + (wid >> 1)) : "memory");
}

// ---------------------------------------------------------------------------------------
// FP32 factor of the outer iteration with two block rows per lane (the mixed path's zone blocks,
// M-matrices: no row exchanges).  L = NP/2 lanes hold a half-system, lane m rows m and m + L, and a
// warp holds S = 32 / L half-systems (three at NP = 20); warp 0 of a CTA takes the top-down halves
// and warp 1 the bottom-up halves of the same S systems.  Every pivot row is read from shared memory
// once per lane for its two rows, so a broadcast serves twice the rows and S systems at once: the
// shared-memory traffic per system, which bounds the one-row-per-lane kernel, drops about threefold.
// Gauss-Jordan with 2 x 2 pivot blocks as gj_invert_np2; the Schur term of the next zone is formed
// from the lane's own rows of the inverse, still in registers (row r of the inverse stays with the
// lane of row r); the next zone's rows and couplings arrive by asynchronous copies issued one zone
// ahead.  A zone whose 2 x 2 pivot block is singular or not finite leaves its inverse non-finite
// (the outer iteration then reports ENAN for the ray); the ABI's factor of arbitrary systems uses
// the pivoting kernel above.
template <int NP>
struct Row2 {
  static constexpr int L = NP / 2;                 // lanes per half-system
  static constexpr int S = 32 / L;                 // half-systems per warp
  static constexpr int PAD = (NP / 4) % 2 ? NP : NP + 4;   // pivot-row stride: an odd number of
                                                           // 16-byte pieces (conflict-free reads)
};

// CTAs per SM the two-rows-per-lane factor is compiled for (its register budget).
#ifndef MGFLD_ROW2_MINB
#define MGFLD_ROW2_MINB 9
#endif

template <int NP>
__global__ void __launch_bounds__(64, MGFLD_ROW2_MINB)
k_factor_row2(int n_r, int n_sys, const float *__restrict__ diag, const float *__restrict__ lower,
              const float *__restrict__ upper, float *__restrict__ dinv, const int *__restrict__ ray_list,
              const int *__restrict__ n_dev) {
  using C = Row2<NP>;
  constexpr int L = C::L, S = C::S, PD = C::PAD;
  static_assert(NP % 4 == 0 && L % 2 == 0, "pivot pairs in one lane pair, rows in 16-byte pieces");
  // The next zone's rows and couplings arrive by cp.async, per warp (each lane copies and later
  // reads only its own two rows: 80-byte rows are conflict-free for its 16-byte reads); after its
  // last zone the bottom-up warp leaves its last inverse in its row buffer for the middle zone of
  // the top-down warp.
  __shared__ __align__(16) float rows[2][S][NP][NP];       // the next zone's rows, per warp
  __shared__ __align__(16) float cpl[2][S][2][NP];         // its couplings (to the previous / next zone)
  __shared__ __align__(16) float prow[2][2][S][2][PD];     // per warp, double-buffered pivot row pairs
  __shared__ __align__(16) float ucol[2][S][NP];           // column scaling of the next zone's Schur term
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = wid;                                    // 0: zones 0..m top-down, 1: n_r-1..m+1 bottom-up
  const int g = lane / L, mm = lane % L;                   // half-system of the warp, lane in it
  const int n_sys_e = listed_sys(n_sys, n_dev, NS);
  const long j0 = (long)blockIdx.x * S;
  if (j0 >= n_sys_e) return;                               // the whole CTA
  const long jsys = j0 + g;
  const bool valid = g < S && jsys < n_sys_e;
  const long sys = valid ? system_of(jsys, ray_list) : 0;
  const int gs = g < S ? g : 0;                            // shared-memory slot (idle lanes use 0)
  const int m = n_r / 2;
  const int len = half == 0 ? m + 1 : n_r - 1 - m;
  auto zone = [&](int j) { return half == 0 ? j : n_r - 1 - j; };
  const int r0 = mm, r1 = mm + L;                          // this lane's two rows
  auto issue = [&](int j) {                                // rows and couplings of zone j
    if (valid && j < len) {
      const size_t zb = ((size_t)sys * n_r + zone(j)) * NP;
#pragma unroll
      for (int c = 0; c < NP; c += 4) {
        cp_async16(&rows[wid][gs][r0][c], diag + (zb + r0) * NP + c);
        cp_async16(&rows[wid][gs][r1][c], diag + (zb + r1) * NP + c);
      }
      const float *lin = half == 0 ? lower : upper, *lout = half == 0 ? upper : lower;
      cp_async4(&cpl[wid][gs][0][r0], lin + zb + r0);
      cp_async4(&cpl[wid][gs][0][r1], lin + zb + r1);
      cp_async4(&cpl[wid][gs][1][r0], lout + zb + r0);
      cp_async4(&cpl[wid][gs][1][r1], lout + zb + r1);
    }
    cp_async_commit();
  };
  float (*midt)[NP][NP] = rows[1];                         // the bottom-up warp's last inverse
  float a0[NP], a1[NP];
  issue(0);
  for (int j = 0; j < len; ++j) {
    cp_async_wait_all();
    __syncwarp();
    // the zone's rows minus the Schur term of the previous zone: row r gets
    // -l_r (row r of the previous inverse, this lane's registers) * u_prev (column scaling)
    // (lanes without a system run on whatever their slot holds: they store nothing, and a slot
    // without a system is read by its own lanes only)
    const float l0 = cpl[wid][gs][0][r0], l1 = cpl[wid][gs][0][r1];   // used from the second zone on
    const float u0 = cpl[wid][gs][1][r0], u1 = cpl[wid][gs][1][r1];
#pragma unroll
    for (int c = 0; c < NP; c += 4) {
      float4 x0 = *reinterpret_cast<const float4 *>(&rows[wid][gs][r0][c]);
      float4 x1 = *reinterpret_cast<const float4 *>(&rows[wid][gs][r1][c]);
      if (j > 0) {
        const float4 u = *reinterpret_cast<const float4 *>(&ucol[wid][gs][c]);
        x0.x = fmaf(-(l0 * a0[c]), u.x, x0.x);
        x0.y = fmaf(-(l0 * a0[c + 1]), u.y, x0.y);
        x0.z = fmaf(-(l0 * a0[c + 2]), u.z, x0.z);
        x0.w = fmaf(-(l0 * a0[c + 3]), u.w, x0.w);
        x1.x = fmaf(-(l1 * a1[c]), u.x, x1.x);
        x1.y = fmaf(-(l1 * a1[c + 1]), u.y, x1.y);
        x1.z = fmaf(-(l1 * a1[c + 2]), u.z, x1.z);
        x1.w = fmaf(-(l1 * a1[c + 3]), u.w, x1.w);
      }
      a0[c] = x0.x; a0[c + 1] = x0.y; a0[c + 2] = x0.z; a0[c + 3] = x0.w;
      a1[c] = x1.x; a1[c + 1] = x1.y; a1[c + 2] = x1.z; a1[c + 3] = x1.w;
    }
    __syncwarp();                                          // every lane has read the rows and ucol
    issue(j + 1);
    if (half == 0 && j == m) {
      // middle zone: wait for the bottom-up half (which arrives once, after its last zone, whatever
      // its length) and subtract its term diag(u_m) D''^{-1}_{m+1} diag(l_{m+1}) as well
      asm volatile("bar.sync 1, 64;" ::: "memory");
      if (n_r - 1 > m) {
#pragma unroll
        for (int c = 0; c < NP; ++c) {
          const float lc = ucol[1][gs][c];
          a0[c] = fmaf(-(u0 * midt[gs][r0][c]), lc, a0[c]);
          a1[c] = fmaf(-(u1 * midt[gs][r1][c]), lc, a1[c]);
        }
      }
    }
    // Gauss-Jordan inversion with 2 x 2 pivot blocks (rows p, p + 1: lanes p % L and p % L + 1 of
    // slot p / L, known at compile time)
#pragma unroll
    for (int b = 0; b < NP / 2; ++b) {
      const int p = 2 * b, sl = p / L, pl = p % L;
      float (*pb)[2][PD] = prow[wid][b & 1];
      if (g < S && (mm == pl || mm == pl + 1)) {          // lanes beyond the S half-systems publish nothing
        float *dst = pb[gs][mm - pl];
#pragma unroll
        for (int c = 0; c < NP; c += 4) {
          if (sl == 0) *reinterpret_cast<float4 *>(dst + c) = make_float4(a0[c], a0[c + 1], a0[c + 2], a0[c + 3]);
          else *reinterpret_cast<float4 *>(dst + c) = make_float4(a1[c], a1[c + 1], a1[c + 2], a1[c + 3]);
        }
      }
      __syncwarp();
      const float2 q0 = *reinterpret_cast<const float2 *>(&pb[gs][0][p]);
      const float2 q1 = *reinterpret_cast<const float2 *>(&pb[gs][1][p]);
      const float det = fmaf(q0.x, q1.y, -(q0.y * q1.x));
      const float idet = rcp_nr(det);
      const float i00 = q1.y * idet, i01 = -q0.y * idet, i10 = -q1.x * idet, i11 = q0.x * idet;
      // multipliers of the two rows: owners take the rows of P^{-1} times the pivot rows
      float f00, f01, f10, f11;
      if (sl == 0 && mm == pl) { f00 = 1.f - i00; f01 = -i01; }
      else if (sl == 0 && mm == pl + 1) { f00 = -i10; f01 = 1.f - i11; }
      else { f00 = fmaf(a0[p], i00, a0[p + 1] * i10); f01 = fmaf(a0[p], i01, a0[p + 1] * i11); }
      if (sl == 1 && mm == pl) { f10 = 1.f - i00; f11 = -i01; }
      else if (sl == 1 && mm == pl + 1) { f10 = -i10; f11 = 1.f - i11; }
      else { f10 = fmaf(a1[p], i00, a1[p + 1] * i10); f11 = fmaf(a1[p], i01, a1[p + 1] * i11); }
#pragma unroll
      for (int c = 0; c < NP; c += 4) {
        const float4 v0 = *reinterpret_cast<const float4 *>(&pb[gs][0][c]);
        const float4 v1 = *reinterpret_cast<const float4 *>(&pb[gs][1][c]);
        float2 lo = __ffma2_rn(make_float2(-f00, -f00), make_float2(v0.x, v0.y), make_float2(a0[c], a0[c + 1]));
        float2 hi = __ffma2_rn(make_float2(-f00, -f00), make_float2(v0.z, v0.w), make_float2(a0[c + 2], a0[c + 3]));
        lo = __ffma2_rn(make_float2(-f01, -f01), make_float2(v1.x, v1.y), lo);
        hi = __ffma2_rn(make_float2(-f01, -f01), make_float2(v1.z, v1.w), hi);
        a0[c] = lo.x; a0[c + 1] = lo.y; a0[c + 2] = hi.x; a0[c + 3] = hi.y;
        lo = __ffma2_rn(make_float2(-f10, -f10), make_float2(v0.x, v0.y), make_float2(a1[c], a1[c + 1]));
        hi = __ffma2_rn(make_float2(-f10, -f10), make_float2(v0.z, v0.w), make_float2(a1[c + 2], a1[c + 3]));
        lo = __ffma2_rn(make_float2(-f11, -f11), make_float2(v1.x, v1.y), lo);
        hi = __ffma2_rn(make_float2(-f11, -f11), make_float2(v1.z, v1.w), hi);
        a1[c] = lo.x; a1[c + 1] = lo.y; a1[c + 2] = hi.x; a1[c + 3] = hi.y;
      }
      if (sl == 0 && mm == pl) { a0[p] = i00; a0[p + 1] = i01; }
      else if (sl == 0 && mm == pl + 1) { a0[p] = i10; a0[p + 1] = i11; }
      else { a0[p] = -f00; a0[p + 1] = -f01; }
      if (sl == 1 && mm == pl) { a1[p] = i00; a1[p + 1] = i01; }
      else if (sl == 1 && mm == pl + 1) { a1[p] = i10; a1[p + 1] = i11; }
      else { a1[p] = -f10; a1[p + 1] = -f11; }
    }
    // the inverse rows to the factor buffer, and this zone's coupling to the next zone of the
    // sequence (column scaling of the next Schur term) to the warp's shared row
    if (valid) {
      float *o0 = dinv + (((size_t)sys * n_r + zone(j)) * NP + r0) * NP;
      float *o1 = dinv + (((size_t)sys * n_r + zone(j)) * NP + r1) * NP;
#pragma unroll
      for (int c = 0; c < NP; c += 4) {
        *reinterpret_cast<float4 *>(o0 + c) = make_float4(a0[c], a0[c + 1], a0[c + 2], a0[c + 3]);
        *reinterpret_cast<float4 *>(o1 + c) = make_float4(a1[c], a1[c + 1], a1[c + 2], a1[c + 3]);
      }
    }
    if (g < S) {
      ucol[wid][gs][r0] = u0;
      ucol[wid][gs][r1] = u1;
    }
    if (half == 1 && j == len - 1 && g < S) {
      // the bottom-up half's last inverse for the middle zone of the top-down half
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        midt[gs][r0][c] = a0[c];
        midt[gs][r1][c] = a1[c];
      }
    }
    __syncwarp();
  }
  cp_async_wait_all();
  if (half == 1) asm volatile("bar.sync 1, 64;" ::: "memory");
}

// Forward/back substitution with the twisted FP32 factors, two warps per system (the top-down
// and bottom-up halves), lane r owning block row r; the halves meet at the middle zone m through
// shared memory and a two-warp named barrier.
template <int NP>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
k_solve_w32(int n, int n_r, int n_sys, const float *__restrict__ dinv, const double *__restrict__ lower,
            const double *__restrict__ upper, const double *__restrict__ rhs, double *__restrict__ x,
            const int *__restrict__ ray_list, const int *__restrict__ n_dev) {
  __shared__ float hbuf[kWarpsPerCta / 2][32], xbuf[kWarpsPerCta / 2][32];
  const unsigned full = 0xffffffffu;
  const int wid = threadIdx.x >> 5, r = threadIdx.x & 31;
  const int half = wid & 1, slot = wid >> 1;
  const long jsys = (long)blockIdx.x * (kWarpsPerCta / 2) + slot;
  if (jsys >= listed_sys(n_sys, n_dev, NS)) return;
  const long sys = system_of(jsys, ray_list);
  const bool real = r < n;
  const size_t base = (size_t)sys * n_r * n;
  const int m = n_r / 2, B = n_r - 1 - m;
  // Power-of-two scaling of the right-hand side (FP32 range), the same in both halves.
  double mx = 0.0;
  if (real)
    for (int i = 0; i < n_r; ++i) mx = fmax(mx, fabs(rhs[base + (size_t)i * n + r]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(full, mx, off));
  double scale = 1.0;
  if (mx > 0.0 && isfinite(mx)) {
    int e;
    frexp(mx, &e);
    scale = ldexp(1.0, -e);
  }
  auto matvec = [&](int z, float v) {
    const float *src = dinv + (base + (size_t)z * n + (real ? r : 0)) * n;
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
    for (int c = 0; c < NP; c += 2) {
      const float v0 = __shfl_sync(full, v, c), v1 = __shfl_sync(full, v, c + 1);
      if (c < n) acc0 = fmaf(src[c], v0, acc0);
      if (c + 1 < n) acc1 = fmaf(src[c + 1], v1, acc1);
    }
    return acc0 + acc1;
  };
  auto bar = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(1 + slot) : "memory"); };
  bar();                       // both halves have read rhs for the scale before x (may alias rhs) is written
  // Forward: top g_i = Dinv_i (r_i - l_i g_{i-1}), i < m; bottom h_i = Dinv_i (r_i - u_i h_{i+1}), i > m.
  const int flen = half == 0 ? m : B;
  float prev = 0.f;
  for (int j = 0; j < flen; ++j) {
    const int z = half == 0 ? j : n_r - 1 - j;
    const size_t zr = base + (size_t)z * n + r;
    const float c = (real && j > 0) ? (float)(half == 0 ? lower[zr] : upper[zr]) : 0.f;
    const float v = real ? (float)(rhs[zr] * scale) - c * prev : 0.f;
    const float g = matvec(z, v);
    if (real) x[zr] = (double)g;
    prev = g;
  }
  if (half == 1) hbuf[slot][r] = B > 0 ? prev : 0.f;
  bar();
  if (half == 0) {
    // Middle zone: x_m = Dinv_m (r_m - l_m g_{m-1} - u_m h_{m+1}).
    const size_t zr = base + (size_t)m * n + r;
    const float l = (real && m > 0) ? (float)lower[zr] : 0.f;
    const float u = (real && m < n_r - 1) ? (float)upper[zr] : 0.f;
    const float v = real ? (float)(rhs[zr] * scale) - l * prev - u * hbuf[slot][r] : 0.f;
    const float xm = matvec(m, v);
    if (real) x[zr] = (double)xm / scale;
    xbuf[slot][r] = xm;
    prev = xm;
  }
  bar();
  if (half == 1) prev = xbuf[slot][r];
  // Backward: top x_i = g_i - Dinv_i (u_i x_{i+1}), i = m-1..0; bottom x_i = h_i - Dinv_i (l_i x_{i-1}), i = m+1..
  for (int j = 0; j < flen; ++j) {
    const int z = half == 0 ? m - 1 - j : m + 1 + j;
    const size_t zr = base + (size_t)z * n + r;
    const float c = real ? (float)(half == 0 ? upper[zr] : lower[zr]) : 0.f;
    const float gz = real ? (float)x[zr] : 0.f;
    const float xi = gz - matvec(z, real ? c * prev : 0.f);
    if (real) x[zr] = (double)xi / scale;
    prev = xi;
  }
}

#define MGFLD_DISPATCH_NP(n, ...)                          \
  if (n <= 4) { constexpr int NP = 4; __VA_ARGS__; }         \
  else if (n <= 8) { constexpr int NP = 8; __VA_ARGS__; }    \
  else if (n <= 12) { constexpr int NP = 12; __VA_ARGS__; }  \
  else if (n <= 16) { constexpr int NP = 16; __VA_ARGS__; }  \
  else if (n <= 20) { constexpr int NP = 20; __VA_ARGS__; }  \
  else if (n <= 24) { constexpr int NP = 24; __VA_ARGS__; }  \
  else { constexpr int NP = 32; __VA_ARGS__; }

// ---------------------------------------------------------------------------------------
// TMA-fed warp solve (MIXED, even n): each warp streams its system's per-zone inverse block and
// the zone's right-hand side / coupling vectors into a ring of shared-memory slots with bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier per slot), issued
// STAGES-1 zones ahead by lane 0, so the recurrence never waits on a global-memory round trip.
// Every wait is bounded: on timeout the warp flags `err`, waits (bounded) for its copies in
// flight and returns.
template <int NP>
struct SolveRing {
  // Ring depth: a power of two (slot and phase by masks), 8 for N <= 20 and 4 above, so that
  // the rings of both warps (<= 26 KB) let every CTA of a 1024-system launch be resident.
  static constexpr int STAGES = NP <= 20 ? 8 : 4;
  static constexpr int WPC = 2;                              // warps per CTA (the two halves of one system)
  static constexpr int SLOT = NP * NP * 4;                   // bytes: one inverse block
};

__device__ inline unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ inline void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                   "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ inline bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr int kWaitLimit = 1 << 22;
__device__ inline bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The power-of-two scaling of one system's right-hand side for the FP32 substitution: k such that
// max |rhs| 2^k lies in [1/2, 1) (from the largest exponent, so the maximum is taken over the
// upper words of the bit patterns: integer pipe only), and the FP32 copy rhs 2^k.  All threads of
// the block call it.
__device__ inline void sysmax_scale(const double *__restrict__ rhs, int cnt, int *__restrict__ sys_exp,
                                    float *__restrict__ rhs32) {
  __shared__ unsigned red[256];
  __shared__ int kexp_s;
  unsigned m = 0u;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x)
    m = max(m, (unsigned)(__double_as_longlong(rhs[e]) >> 32) & 0x7fffffffu);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int e = (int)(red[0] >> 20);
    const int k = (e > 0 && e < 0x7ff) ? 1022 - e : 0;
    *sys_exp = k;
    kexp_s = k;
  }
  __syncthreads();
  const int k = kexp_s;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) rhs32[e] = d2f_exp2(rhs[e], k);
}

// Per-system power-of-two scaling of the FP32 solve: k with max |rhs| 2^k in [0.5, 1) (the
// exponent field of the maximum), then the scaled right-hand side rounded to FP32 once, so that
// the substitution reads FP32 values.  One CTA per listed system; its n_r x n right-hand side is
// contiguous (coalesced loads; the second pass reads it from L2).
__global__ void k_sysmax(int n, int n_r, const double *__restrict__ rhs, const int *__restrict__ ray_list,
                         int *__restrict__ sys_exp, float *__restrict__ rhs32, const int *__restrict__ n_dev) {
  if ((int)blockIdx.x >= listed_sys(gridDim.x, n_dev, NS)) return;    // the whole block
  const size_t base = (size_t)system_of(blockIdx.x, ray_list) * n_r * n;
  sysmax_scale(rhs + base, n_r * n, sys_exp + blockIdx.x, rhs32 + base);
}

// k_sysmax for systems listed with `spr` systems per ray.
__global__ void k_sysmax_spr(int n, int n_r, const double *__restrict__ rhs, const int *__restrict__ ray_list, int spr,
                             int *__restrict__ sys_exp, float *__restrict__ rhs32, const int *__restrict__ n_dev) {
  if ((int)blockIdx.x >= listed_sys(gridDim.x, n_dev, spr)) return;   // the whole block
  const size_t base = (size_t)system_of_spr(blockIdx.x, ray_list, spr) * n_r * n;
  sysmax_scale(rhs + base, n_r * n, sys_exp + blockIdx.x, rhs32 + base);
}

// Row r of a zone's inverse times the zone vector held in shared memory (vb).  VEC: n == NP,
// rows 16-byte aligned, float4 loads; otherwise scalar loads masked to the n real columns.
template <int NP, bool VEC>
__device__ inline float row_dot(const float *__restrict__ row, const float *__restrict__ vb, int n) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  if (VEC) {
#pragma unroll
    for (int c = 0; c < NP; c += 4) {
      const float4 m = *reinterpret_cast<const float4 *>(row + c);
      const float4 v = *reinterpret_cast<const float4 *>(vb + c);
      a0 = fmaf(m.x, v.x, a0);
      a1 = fmaf(m.y, v.y, a1);
      a2 = fmaf(m.z, v.z, a2);
      a3 = fmaf(m.w, v.w, a3);
    }
  } else {
#pragma unroll
    for (int c = 0; c < NP; ++c)
      if (c < n) {
        if (c % 2 == 0) a0 = fmaf(row[c], vb[c], a0);
        else a1 = fmaf(row[c], vb[c], a1);
      }
  }
  return (a0 + a1) + (a2 + a3);
}

// MIXED-precision substitution with the twisted FP32 factors: one CTA per system, warp 0 the
// top-down half (zones 0..m-1, then the middle zone m, then back up from m-1 to 0), warp 1 the
// bottom-up half (zones n_r-1..m+1, then back down from m+1).  Each warp streams its zones'
// inverse blocks through its own ring of bulk copies (one copy per use, mbarrier completion,
// bounded waits); the halves meet at the middle through shared memory and CTA barriers.  Lane
// r owns block row r; the zone vector is broadcast through shared memory.  The right-hand side
// arrives scaled and rounded to FP32 (k_sysmax); the result is scaled back by an exact FP64
// multiplication by 2^-k.  Offsets inside a system are 32-bit.  Every block is read twice (the
// inward and the outward sweep), so the kernel is bound by the HBM bandwidth of those reads.
template <int NP, bool VEC>
__global__ void __launch_bounds__(SolveRing<NP>::WPC * 32)
k_solve_tma(int n, int n_r, int n_sys, const float *__restrict__ dinv, const float *__restrict__ lower,
            const float *__restrict__ upper, const float *__restrict__ rhs32, double *__restrict__ x,
            float *__restrict__ g32, const int *__restrict__ ray_list, const int *__restrict__ sys_exp, int *err,
            const int *__restrict__ n_dev) {
  using R = SolveRing<NP>;
  static_assert(R::WPC == 2, "one system per CTA: two warps, one per half");
  constexpr int S = R::STAGES;
  static_assert((S & (S - 1)) == 0 && S % 4 == 0, "power-of-two ring, refilled four slots at a time");
  constexpr int D = 8;                                      // depth of the per-lane vector queue
  __shared__ __align__(128) unsigned char ring[2][S][NP * NP * 4];
  __shared__ __align__(16) float vbuf[2][NP];               // the zone vector, broadcast through smem
  __shared__ __align__(16) float qbuf[2][D][2][32];         // per-lane queue: (rhs or g, coupling)
  __shared__ __align__(8) unsigned long long bar[2][S];
  __shared__ float hbuf[32], xbuf[32];                      // h_{m+1} and x_m, exchanged at the middle
  const unsigned full = 0xffffffffu;
  const int half = threadIdx.x >> 5, r = threadIdx.x & 31;
  const long jsys = blockIdx.x;
  if (jsys >= listed_sys(n_sys, n_dev, NS)) return;         // whole CTA
  const long sys = system_of(jsys, ray_list);
  const bool real = r < n;
  const int rr = real ? r : 0;                              // lanes without a row use row 0 (unused)
  const unsigned blk = (unsigned)(n * n * 4);
  const double unscale = ldexp(1.0, -sys_exp[jsys]);       // rhs was scaled by 2^k before rounding
  const int m = n_r / 2, B = n_r - 1 - m;
  const int F = half == 0 ? m : B;                          // forward steps of this half
  const int U = half == 0 ? 2 * m + 1 : 2 * B;              // ring uses of this half
  // Zone sequences: forward zf0 + j dz, backward zb0 - j dz; element offsets z n (32-bit).
  const int dz = half == 0 ? 1 : -1;
  const int dzn = dz * n;
  const int zf0 = half == 0 ? 0 : n_r - 1, zb0 = half == 0 ? m - 1 : m + 1;
  // Per-lane element pointers of this system (row r of zone z is [z * n]).
  const size_t sb = (size_t)sys * n_r * n;
  const float *rhs_l = rhs32 + sb + rr;
  const float *cin_l = (half == 0 ? lower : upper) + sb + rr;   // coupling used going inward
  const float *cout_l = (half == 0 ? upper : lower) + sb + rr;  // coupling used going outward
  float *g_l = g32 + sb + rr;
  double *x_l = x + sb + rr;
  const float *dsys = dinv + sb * n;
  const unsigned rowoff = (unsigned)rr * (unsigned)n * 4u; // byte offset of row r in a slot
  if (r == 0) {
    for (int k = 0; k < S; ++k) mbar_init(&bar[half][k], 1);
    mbar_fence_init();
  }
  __syncwarp();
  // Lane 0 issues the bulk copies in use order, tracking the source block of the next use:
  // top-down half +1 zone up to the middle, then -1; bottom-up half -1 to zone m + 1, which is
  // used twice (last forward, first backward), then +1.  All S slots are filled up front, then
  // four at a time once the four uses that held them are consumed.
  int iu = 0;
  const float *src = dsys + (size_t)zf0 * n * n;
  const int bstep = n * n;
  auto issue_next = [&]() {
    unsigned long long *b = &bar[half][iu & (S - 1)];
    mbar_expect_tx(b, blk);
    bulk_g2s(ring[half][iu & (S - 1)], src, blk, b);
    ++iu;
    if (half == 0) src += iu <= m ? bstep : -bstep;
    else src += iu < B ? -bstep : (iu == B ? 0 : bstep);
  };
  bool ok = true;                                           // warp-uniform
  auto wait = [&](int u) -> bool {
    if (!ok) return false;
    if (mbar_try_wait(&bar[half][u & (S - 1)], (unsigned)((u / S) & 1))) return true;
    bool w = mbar_wait_bounded(&bar[half][u & (S - 1)], (unsigned)((u / S) & 1));
    ok = __all_sync(full, w);
    if (!ok) {                                    // give up: flag and drain own copies
      if (r == 0) {
        atomicExch(err, 1);
        for (int v = u + 1; v < iu; ++v) mbar_wait_bounded(&bar[half][v & (S - 1)], (unsigned)((v / S) & 1));
      }
      __syncwarp();
    }
    return ok;
  };
  auto advance = [&](int u) {                     // use u consumed: refill four slots after every fourth
    if ((u & 3) == 3) {
      __syncwarp();
      if (r == 0 && ok)
        for (int k = 0; k < 4 && iu < U; ++k) issue_next();
    }
  };
  auto slot_row = [&](int u) {
    return reinterpret_cast<const float *>(ring[half][u & (S - 1)] + rowoff);
  };
  // Per-lane queue of (rhs or forward result, coupling) for the uses D ahead, in shared memory
  // through 4-byte asynchronous copies: one copy group per use, waited for with
  // cp.async.wait_group D-1, so that no register load is outstanding across the recurrence.
  float (*q)[2][32] = qbuf[half];
  auto fill = [&](int d, const float *a, const float *c, int zo) {
    cp_async4(&q[d][0][r], a + zo);
    cp_async4(&q[d][1][r], c + zo);
    cp_async_commit();
  };
  // the middle zone's right-hand side and couplings (top-down half), fetched up front
  const int zm = m * n;
  const float bm_raw = rhs_l[zm], lm_raw = cin_l[zm], um_raw = cout_l[zm];
  float *vb = vbuf[half];

  if (r == 0)
    for (int k = 0; k < S && k < U; ++k) issue_next();
  iu = __shfl_sync(full, iu, 0);
#pragma unroll
  for (int d = 0; d < D; ++d) fill(d, rhs_l, cin_l, (d < F ? zf0 + d * dz : zf0) * n);
  float prev = 0.f;
  int zfo = zf0 * n;                              // element offset of the current forward zone
  for (int j = 0; j < F; ++j) {
    const int d = j & (D - 1);
    cp_async_wait_group<D - 1>();
    const float b = q[d][0][r], l = j > 0 ? q[d][1][r] : 0.f;
    if (wait(j)) {
      if (r < NP) vb[r] = real ? b - l * prev : 0.f;
      __syncwarp();
      const float g = row_dot<NP, VEC>(slot_row(j), vb, n);
      if (real) g_l[zfo] = g;
      prev = g;
    }
    fill(d, rhs_l, cin_l, j + D < F ? zfo + D * dzn : zfo);   // the slot just read: the zone D ahead
    advance(j);
    zfo += dzn;
  }
  cp_async_wait_all();
  if (half == 1) hbuf[r] = B > 0 ? prev : 0.f;
  __syncthreads();
  if (half == 0) {
    // Middle zone: x_m = Dinv_m (r_m - l_m g_{m-1} - u_m h_{m+1}).
    const float bm = real ? bm_raw : 0.f;
    const float lm = (real && m > 0) ? lm_raw : 0.f;
    const float um = (real && m < n_r - 1) ? um_raw : 0.f;
    float xm = 0.f;
    if (wait(m)) {
      if (r < NP) vb[r] = real ? bm - lm * prev - um * hbuf[r] : 0.f;
      __syncwarp();
      xm = row_dot<NP, VEC>(slot_row(m), vb, n);
      if (real) x_l[zm] = (double)xm * unscale;
    }
    advance(m);
    xbuf[r] = xm;
    prev = xm;
  }
  __syncthreads();
  if (half == 1) prev = xbuf[r];
  // Backward: top x_i = g_i - Dinv_i (u_i x_{i+1}); bottom x_i = h_i - Dinv_i (l_i x_{i-1}).
#pragma unroll
  for (int d = 0; d < D; ++d) fill(d, g_l, cout_l, (d < F ? zb0 - d * dz : m) * n);   // m: valid whatever F is
  int zbo = zb0 * n;
  const int ub = U - F;                           // first backward use
  for (int j = 0; j < F; ++j) {
    const int d = j & (D - 1);
    const int u = ub + j;
    cp_async_wait_group<D - 1>();
    const float gz = q[d][0][r], c = q[d][1][r];
    if (wait(u)) {
      if (r < NP) vb[r] = real ? c * prev : 0.f;
      __syncwarp();
      const float xi = gz - row_dot<NP, VEC>(slot_row(u), vb, n);
      if (real) x_l[zbo] = (double)xi * unscale;
      prev = xi;
    }
    fill(d, g_l, cout_l, j + D < F ? zbo - D * dzn : zbo);
    advance(u);
    zbo -= dzn;
  }
  cp_async_wait_all();
}

cudaError_t launch_solve_tma(int n, int n_r, int n_sys, const void *dinv, const float *lower32,
                             const float *upper32, const double *rhs, float *rhs32, double *x, float *g32,
                             const int *ray_list, int *sys_exp, int *err, cudaStream_t s, const int *n_dev) {
  if (n_sys == 0) return cudaSuccess;
  k_sysmax<<<n_sys, 256, 0, s>>>(n, n_r, rhs, ray_list, sys_exp, rhs32, n_dev);
  MGFLD_DISPATCH_NP(n, {
    using R = SolveRing<NP>;
    const unsigned grid = (unsigned)n_sys;                 // one system (two warps) per CTA
    if (n == NP)
      k_solve_tma<NP, true><<<grid, R::WPC * 32, 0, s>>>(n, n_r, n_sys, (const float *)dinv, lower32, upper32, rhs32,
                                                         x, g32, ray_list, sys_exp, err, n_dev);
    else
      k_solve_tma<NP, false><<<grid, R::WPC * 32, 0, s>>>(n, n_r, n_sys, (const float *)dinv, lower32, upper32,
                                                          rhs32, x, g32, ray_list, sys_exp, err, n_dev);
    return cudaGetLastError();
  })
}

template <int NP>
static cudaError_t run_factor(int n, int n_r, int n_sys, const void *diag, int diag_fp32, const double *lower,
                              const double *upper, void *dinv, const int *ray_list, cudaStream_t s,
                              const int *n_dev) {
  constexpr int SPS = Pack<NP>::SPC / 2;             // systems per CTA
  const unsigned grid = (unsigned)((n_sys + SPS - 1) / SPS);
  if (diag_fp32)
    k_factor<NP, float><<<grid, Pack<NP>::THREADS, 0, s>>>(n, n_r, n_sys, (const float *)diag, lower, upper,
                                                           (double *)dinv, ray_list, n_dev);
  else
    k_factor<NP, double><<<grid, Pack<NP>::THREADS, 0, s>>>(n, n_r, n_sys, (const double *)diag, lower, upper,
                                                            (double *)dinv, ray_list, n_dev);
  return cudaGetLastError();
}

template <int NP>
static cudaError_t run_solve(int n, int n_r, int n_sys, const void *dinv, const double *lower,
                             const double *upper, const double *rhs, double *x, const int *ray_list,
                             cudaStream_t s, const int *n_dev) {
  constexpr int SPS = Pack<NP>::SPC / 2;             // systems per CTA
  const unsigned grid = (unsigned)((n_sys + SPS - 1) / SPS);
  k_solve<NP><<<grid, Pack<NP>::THREADS, 0, s>>>(n, n_r, n_sys, (const double *)dinv, lower, upper, rhs, x,
                                                 ray_list, n_dev);
  return cudaGetLastError();
}

cudaError_t launch_factor(int n, int n_r, int n_sys, const void *diag, int diag_fp32, const double *lower,
                          const double *upper, void *dinv, int precision, const int *ray_list,
                          cudaStream_t s, const int *n_dev) {
  if (n_sys == 0) return cudaSuccess;
  if (precision == MGFLD_MIXED) {
    if (diag_fp32) {
      MGFLD_DISPATCH_NP(n, constexpr int W = fw_wpc<NP>();
                        const unsigned grid = (unsigned)((n_sys + W / 2 - 1) / (W / 2));
                        k_factor_w32<NP, float, double, true><<<grid, W * 32, 0, s>>>(
                            n, n_r, n_sys, (const float *)diag, lower, upper, (float *)dinv, ray_list, n_dev);
                        return cudaGetLastError())
    } else {
      MGFLD_DISPATCH_NP(n, constexpr int W = fw_wpc<NP>();
                        const unsigned grid = (unsigned)((n_sys + W / 2 - 1) / (W / 2));
                        k_factor_w32<NP, double, double, true><<<grid, W * 32, 0, s>>>(
                            n, n_r, n_sys, (const double *)diag, lower, upper, (float *)dinv, ray_list, n_dev);
                        return cudaGetLastError())
    }
  } else {
    MGFLD_DISPATCH_NP(n, return (run_factor<NP>(n, n_r, n_sys, diag, diag_fp32, lower, upper, dinv,
                                                        ray_list, s, n_dev)))
  }
}

#define MGFLD_DISPATCH_NPW(n, ...)                          \
  if (n <= 8) { constexpr int NP = 8; __VA_ARGS__; }          \
  else if (n <= 16) { constexpr int NP = 16; __VA_ARGS__; }   \
  else if (n <= 24) { constexpr int NP = 24; __VA_ARGS__; }   \
  else if (n <= 32) { constexpr int NP = 32; __VA_ARGS__; }   \
  else if (n <= 40) { constexpr int NP = 40; __VA_ARGS__; }   \
  else { constexpr int NP = 48; __VA_ARGS__; }

template <int NP, typename TIn, typename T>
static cudaError_t run_factor_rows(int nb, int n_r, int n_sys, int spr, const TIn *diag, const T *lower,
                                   const T *upper, T *dinv, const int *ray_list, cudaStream_t s,
                                   const int *n_dev) {
  using C = RowCta<NP, T>;
  const unsigned grid = (unsigned)((n_sys + C::SPC / 2 - 1) / (C::SPC / 2));
  if (C::BYTES > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_factor_rows<NP, TIn, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)C::BYTES);
    if (e != cudaSuccess) return e;
  }
  k_factor_rows<NP, TIn, T><<<grid, C::THREADS, C::BYTES, s>>>(nb, n_r, n_sys, spr, diag, lower, upper, dinv, ray_list,
                                                               n_dev);
  return cudaGetLastError();
}

cudaError_t launch_factor_rows(int nb, int n_r, int n_sys, int spr, const void *diag, const void *lower,
                               const void *upper, void *dinv, int fp32, const int *ray_list, cudaStream_t s,
                               const int *n_dev) {
  if (n_sys == 0) return cudaSuccess;
  if (nb > 48) return cudaErrorInvalidValue;
  if (fp32) {
    MGFLD_DISPATCH_NPW(nb, return (run_factor_rows<NP, float, float>(nb, n_r, n_sys, spr, (const float *)diag,
                                                                        (const float *)lower, (const float *)upper,
                                                                        (float *)dinv, ray_list, s, n_dev)))
  } else {
    MGFLD_DISPATCH_NPW(nb, return (run_factor_rows<NP, double, double>(nb, n_r, n_sys, spr, (const double *)diag,
                                                                          (const double *)lower, (const double *)upper,
                                                                          (double *)dinv, ray_list, s, n_dev)))
  }
}

cudaError_t launch_solve_rows(int nb, int n_r, int n_sys, int spr, const void *dinv, const void *lower,
                              const void *upper, const double *rhs, float *rhs32, int *sys_exp, double *x, int fp32,
                              const int *ray_list, cudaStream_t s, const int *n_dev) {
  if (n_sys == 0) return cudaSuccess;
  if (nb > 48) return cudaErrorInvalidValue;
  if (fp32) {
    // per-system power-of-two scaling of the right-hand side for the FP32 sweeps
    k_sysmax_spr<<<n_sys, 256, 0, s>>>(nb, n_r, rhs, ray_list, spr, sys_exp, rhs32, n_dev);
    MGFLD_DISPATCH_NPW(nb, using C = RowCta<NP, float>;
                       k_solve_rows<NP, float><<<(unsigned)((n_sys + C::SPC / 2 - 1) / (C::SPC / 2)), C::THREADS, 0, s>>>(
                           nb, n_r, n_sys, spr, (const float *)dinv, (const float *)lower, (const float *)upper, rhs,
                           rhs32, sys_exp, x, ray_list, n_dev);
                       return cudaGetLastError())
  } else {
    MGFLD_DISPATCH_NPW(nb, using C = RowCta<NP, double>;
                       k_solve_rows<NP, double><<<(unsigned)((n_sys + C::SPC / 2 - 1) / (C::SPC / 2)), C::THREADS, 0, s>>>(
                           nb, n_r, n_sys, spr, (const double *)dinv, (const double *)lower, (const double *)upper, rhs,
                           nullptr, nullptr, x, ray_list, n_dev);
                       return cudaGetLastError())
  }
}

cudaError_t launch_factor_f32(int n, int n_r, int n_sys, const float *diag, const float *lower32,
                              const float *upper32, float *dinv, const int *ray_list, cudaStream_t s,
                              const int *n_dev) {
  if (n_sys == 0) return cudaSuccess;
  if (n % 4 == 0) {
    // blocks of a multiple of 4 rows: two rows per lane
    MGFLD_DISPATCH_NP(n, constexpr int S = Row2<NP>::S;
                      k_factor_row2<NP><<<(unsigned)((n_sys + S - 1) / S), 64, 0, s>>>(n_r, n_sys, diag, lower32,
                                                                                         upper32, dinv, ray_list,
                                                                                         n_dev);
                      return cudaGetLastError())
  }
  MGFLD_DISPATCH_NP(n, constexpr int W = fw_wpc<NP>();
                    const unsigned grid = (unsigned)((n_sys + W / 2 - 1) / (W / 2));
                    k_factor_w32<NP, float, float, false><<<grid, W * 32, 0, s>>>(n, n_r, n_sys, diag, lower32, upper32,
                                                                            dinv, ray_list, n_dev);
                    return cudaGetLastError())
}

cudaError_t launch_solve(int n, int n_r, int n_sys, const void *dinv, const double *lower,
                         const double *upper, const double *rhs, double *x, int precision,
                         const int *ray_list, cudaStream_t s, const int *n_dev) {
  if (n_sys == 0) return cudaSuccess;
  if (precision == MGFLD_MIXED) {
    const unsigned grid = (unsigned)((n_sys + kWarpsPerCta / 2 - 1) / (kWarpsPerCta / 2));
    MGFLD_DISPATCH_NP(n, k_solve_w32<NP><<<grid, kWarpsPerCta * 32, 0, s>>>(n, n_r, n_sys, (const float *)dinv,
                                                                          lower, upper, rhs, x, ray_list, n_dev);
                         return cudaGetLastError())
  } else {
    MGFLD_DISPATCH_NP(n, return (run_solve<NP>(n, n_r, n_sys, dinv, lower, upper, rhs, x, ray_list, s, n_dev)))
  }
}

}  // namespace mgfld
