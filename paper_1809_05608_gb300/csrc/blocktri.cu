// Batched block-Thomas elimination for the per-(ray, species) systems of Eq. a62ae.
//
// Structure exploited: the off-diagonal blocks are diagonal (the flux coefficient is
// frozen), so the Schur update of zone i is a diagonal scaling of the previous
// inverse, D'_i = D_i - diag(l_i) D'^{-1}_{i-1} diag(u_{i-1}): no dense block product,
// hence no tensor-core contraction on this path.  Each dense block is inverted in
// place by Gauss-Jordan elimination with partial pivoting.
//
// Thread mapping: one thread per block row; SPC systems (rays x species) share a CTA so
// that SPC * NP is a multiple of 32 and every lane of every FMA instruction does work.
// Rows and columns beyond the real group count n (<= NP) are padded with the identity.
// The pivot search, pivot-row broadcast and the natural-order inverse go through
// shared memory; the inverse of each zone is streamed to the caller's factor buffer.
#include "mgfld_internal.cuh"

namespace mgfld {

template <int NP>
struct Pack {
  static constexpr int gcd(int a, int b) { return b == 0 ? a : gcd(b, a % b); }
  static constexpr int SPC = 32 / gcd(NP, 32);   // systems per CTA
  static constexpr int THREADS = SPC * NP;
};

// 1/d for the pivot of a Gauss-Jordan step without FP64-pipe conversions or compares: the
// mantissa of d, rounded to 24 bits, becomes an FP32 value m in [1, 2] by bit manipulation
// (integer pipe), its reciprocal is taken in FP32, the exponent of 1/d is rebuilt from the two
// exponents, and one Newton-Raphson step x1 = x0 + x0 (1 - d x0) (two FMAs on the FP64 pipe)
// takes the ~2^-23 seed to ~2^-46 relative.  Zero, subnormal, non-finite and extreme-exponent
// pivots take a plain division (rare; a zero pivot means a singular block).  The factors only
// steer the outer iteration, whose fixed point is set by the FP64 residual.
__device__ inline double recip(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned m23 = (unsigned)((b >> 29) & 0x7fffff);
  const float up = ((b >> 28) & 1ull) ? 1.1920928955078125e-7f : 0.f;     // round the dropped bits
  const float m = __uint_as_float(0x3f800000u | m23) + up;                 // exact; may be 2.0
  const unsigned rb = __float_as_uint(__frcp_rn(m));                      // 1/m in (0.5, 1]
  const int ed = (int)(rb >> 23) - 127 + 2046 - e;                         // biased exponent of 1/|d|
  if (e == 0 || e == 0x7ff || ed <= 0 || ed >= 0x7ff) return 1.0 / d;
  const double x = __longlong_as_double((long long)((b & 0x8000000000000000ull) |
                                                    ((unsigned long long)ed << 52) |
                                                    ((unsigned long long)(rb & 0x7fffff) << 29)));
  return fma(x, fma(-d, x, 1.0), x);
}

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
template <int NP, typename TIn>
__global__ void __launch_bounds__(Pack<NP>::THREADS)
k_factor(int n, int n_r, int n_sys, const TIn *__restrict__ diag, const double *__restrict__ lower,
         const double *__restrict__ upper, double *__restrict__ dinv, const int *__restrict__ ray_list) {
  constexpr int SPC = Pack<NP>::SPC;
  __shared__ double tile[SPC][NP][NP + 1];           // natural-order inverse of the previous zone
  __shared__ __align__(16) double prow[SPC][NP];     // pivot row of the current step
  __shared__ __align__(16) int cand[SPC][NP];        // pivot-search keys
  __shared__ double ushr[SPC][NP];                   // upper_{i-1}, the column scaling of the Schur update
  __shared__ int pivrow[SPC][NP];                    // row chosen at each step
  __shared__ double pinv[SPC];                       // 1 / pivot of the current step

  const int s = threadIdx.x / NP, r = threadIdx.x % NP;
  const long jsys = (long)blockIdx.x * SPC + s;
  const bool valid = jsys < n_sys;
  const long sys = valid ? system_of(jsys, ray_list) : 0;
  const bool real = valid && r < n;

  // Rows of the next zone are fetched one zone ahead (registers) to hide memory latency.
  double nxt[NP];
  double nl = 0.0;
  auto load_row = [&](int i) {
    const size_t zr = ((size_t)sys * n_r + i) * n + r;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      if (real && c < n) nxt[c] = (double)diag[zr * n + c];
      else nxt[c] = (c == r) ? 1.0 : 0.0;
    }
    nl = (real && i > 0) ? lower[zr] : 0.0;
  };
  load_row(0);
  for (int i = 0; i < n_r; ++i) {
    const size_t zrow = ((size_t)sys * n_r + i) * n + r;   // (sys, i, r)
    double a[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) a[c] = nxt[c];
    const double lr = nl;
    if (i + 1 < n_r) load_row(i + 1);
    if (i > 0) {
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = fma(-(lr * tile[s][r][c]), ushr[s][c], a[c]);
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
      double pr[NP];
#pragma unroll
      for (int c = 0; c < NP; c += 2) {
        const double2 v = *reinterpret_cast<const double2 *>(&prow[s][c]);
        pr[c] = v.x;
        pr[c + 1] = v.y;
      }
      const double inv = pinv[s];
      // Uniform update for every row: a -= f * pivot_row, with f chosen so that the pivot row
      // itself becomes pivot_row / pivot (f = 1 - 1/pivot): one FMA either way.  The pivot
      // column itself is overwritten below, so its update is skipped.
      const double f = fma(me ? -1.0 : a[pstep], inv, me ? 1.0 : 0.0);
      if (pstep + 1 < NP) {
        a[pstep + 1] = fma(-f, pr[pstep + 1], a[pstep + 1]);
        cand[s][r] = used ? -1 : pivot_key(a[pstep + 1], r);
      }
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c != pstep + 1 && c != pstep) a[c] = fma(-f, pr[c], a[c]);
      a[pstep] = me ? inv : -f;
    }
    // Row r now holds row my_step of the inverse, with column c belonging to input row pivrow[c].
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NP; ++c) tile[s][my_step][pivrow[s][c]] = a[c];
    ushr[s][r] = real ? upper[zrow] : 0.0;
    __syncthreads();
    if (real) {
      double *out = dinv + zrow * n;
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c < n) out[c] = tile[s][r][c];
    }
  }
}

// Forward and back substitution with the stored inverses (one thread per block row).
// MIXED (T = float): the right-hand side of each system is scaled by a power of two so
// that its largest entry is O(1) before rounding to FP32, and unscaled on output.
template <int NP, typename T>
__global__ void __launch_bounds__(Pack<NP>::THREADS)
k_solve(int n, int n_r, int n_sys, const T *__restrict__ dinv, const double *__restrict__ lower,
        const double *__restrict__ upper, const double *__restrict__ rhs, double *__restrict__ x,
        const int *__restrict__ ray_list) {
  constexpr int SPC = Pack<NP>::SPC;
  __shared__ T v[SPC][NP];
  __shared__ double red[SPC][NP];
  const int s = threadIdx.x / NP, r = threadIdx.x % NP;
  const long jsys = (long)blockIdx.x * SPC + s;
  const bool valid = jsys < n_sys;
  const long sys = valid ? system_of(jsys, ray_list) : 0;
  const bool real = valid && r < n;
  const size_t base = (size_t)sys * n_r * n;

  double scale = 1.0;
  if (sizeof(T) == 4) {
    double m = 0.0;
    if (real)
      for (int i = 0; i < n_r; ++i) m = fmax(m, fabs(rhs[base + (size_t)i * n + r]));
    red[s][r] = m;
    __syncthreads();
    m = 0.0;
    for (int c = 0; c < NP; ++c) m = fmax(m, red[s][c]);
    if (m > 0.0 && isfinite(m)) {
      int e;
      frexp(m, &e);
      scale = ldexp(1.0, -e);
    }
  }

  // The next zone's inverse row, rhs and coupling are loaded one zone ahead so that their
  // memory latency overlaps the current zone's arithmetic (the recurrence is sequential).
  T row[NP], nrow[NP];
#pragma unroll
  for (int c = 0; c < NP; ++c) nrow[c] = T(0);
  double nb = 0.0, nc = 0.0;
  auto load_fwd = [&](int i) {
    const size_t zr = base + (size_t)i * n + r;
    const T *src = dinv + zr * n;
#pragma unroll
    for (int c = 0; c < NP; ++c) nrow[c] = (c < n) ? src[c] : T(0);
    nb = rhs[zr];
    nc = i > 0 ? lower[zr] : 0.0;
  };
  if (real) load_fwd(0);
  T g_prev = T(0);
  for (int i = 0; i < n_r; ++i) {
    const size_t zr = base + (size_t)i * n + r;
#pragma unroll
    for (int c = 0; c < NP; ++c) row[c] = nrow[c];
    const double b = nb, l = nc;
    if (real && i + 1 < n_r) load_fwd(i + 1);
    v[s][r] = real ? to_t<T>(b * scale) - to_t<T>(l) * g_prev : T(0);
    __syncthreads();
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < NP; ++c) acc = acc + row[c] * v[s][c];
    if (real) x[zr] = (double)acc;
    g_prev = acc;
    __syncthreads();
  }
  auto load_bwd = [&](int i) {
    const size_t zr = base + (size_t)i * n + r;
    const T *src = dinv + zr * n;
#pragma unroll
    for (int c = 0; c < NP; ++c) nrow[c] = (c < n) ? src[c] : T(0);
    nb = x[zr];
    nc = i < n_r - 1 ? upper[zr] : 0.0;
  };
  if (real) load_bwd(n_r - 1);
  T x_next = T(0);
  for (int i = n_r - 1; i >= 0; --i) {
    const size_t zr = base + (size_t)i * n + r;
#pragma unroll
    for (int c = 0; c < NP; ++c) row[c] = nrow[c];
    const double g = nb, u = nc;
    if (real && i > 0) load_bwd(i - 1);
    v[s][r] = real ? to_t<T>(u) * x_next : T(0);
    __syncthreads();
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < NP; ++c) acc = acc + row[c] * v[s][c];
    const T xi = to_t<T>(g) - acc;
    if (real) x[zr] = (double)xi / scale;
    x_next = xi;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Warp-synchronous FP32 variants (MIXED precision): one warp per (ray, species) system, lane r
// owns block row r (NP <= 32), no CTA-wide barriers.  The pivot is found with a warp max
// reduction on integer keys, the pivot row is broadcast with shuffles, and the per-zone
// natural-order inverse goes through a per-warp shared-memory tile.  FP32 arithmetic is 63x
// cheaper than FP64 on this GPU, so these kernels are bound by the dependency chain along
// the zones, which the warp form shortens.
constexpr int kWarpsPerCta = 4;

template <int NP, typename TIn, typename TC>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
k_factor_w32(int n, int n_r, int n_sys, const TIn *__restrict__ diag, const TC *__restrict__ lower,
             const TC *__restrict__ upper, float *__restrict__ dinv, const int *__restrict__ ray_list) {
  __shared__ float tile[kWarpsPerCta][NP][NP + 1];
  __shared__ float ushr[kWarpsPerCta][NP];
  const unsigned full = 0xffffffffu;
  const int wid = threadIdx.x >> 5, r = threadIdx.x & 31;
  const long jsys = (long)blockIdx.x * kWarpsPerCta + wid;
  if (jsys >= n_sys) return;                        // whole warp leaves; no CTA barrier below
  const long sys = system_of(jsys, ray_list);
  const bool real = r < n;
  const bool row = r < NP;
  float nxt[NP];
  float nl = 0.f;
  auto load_row = [&](int i) {
    const size_t zr = ((size_t)sys * n_r + i) * n + r;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      if (real && c < n) nxt[c] = (float)diag[zr * n + c];
      else nxt[c] = (c == r) ? 1.f : 0.f;
    }
    nl = (real && i > 0) ? (float)lower[zr] : 0.f;
  };
  load_row(0);
  for (int i = 0; i < n_r; ++i) {
    const size_t zrow = ((size_t)sys * n_r + i) * n + r;
    float a[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) a[c] = nxt[c];
    const float lr = nl;
    if (i + 1 < n_r) load_row(i + 1);
    if (i > 0 && row) {
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = a[c] - (lr * tile[wid][r][c]) * ushr[wid][c];
    }
    bool used = !row;
    int my_step = 0;
    int piv[NP];
    // Pivot-search key as in the FP64 factor: |a| bits with the row index in the 5 low bits, so
    // one warp max names the pivot row.  The pivot and next-pivot-column entries of the pivot
    // row are broadcast first and the next pivot column is updated first, so that the next
    // search overlaps the broadcast and update of the other columns.
    int key = used ? -1 : (int)(((unsigned)__float_as_int(fabsf(a[0])) & ~31u) | (unsigned)(31 - r));
#pragma unroll
    for (int pstep = 0; pstep < NP; ++pstep) {
      const int best = 31 - (__reduce_max_sync(full, key) & 31);
      piv[pstep] = best;
      const bool me = (r == best);
      if (me) {
        used = true;
        my_step = pstep;
      }
      const float pp = __shfl_sync(full, a[pstep], best);
      const float inv = __frcp_rn(pp);
      const float f = fmaf(me ? -1.f : a[pstep], inv, me ? 1.f : 0.f);
      if (pstep + 1 < NP) {
        const float pn = __shfl_sync(full, a[pstep + 1], best);
        a[pstep + 1] = fmaf(-f, pn, a[pstep + 1]);
        key = used ? -1 : (int)(((unsigned)__float_as_int(fabsf(a[pstep + 1])) & ~31u) | (unsigned)(31 - r));
      }
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c != pstep + 1 && c != pstep) a[c] = fmaf(-f, __shfl_sync(full, a[c], best), a[c]);
      a[pstep] = me ? inv : -f;
    }
    __syncwarp();
    if (row) {
#pragma unroll
      for (int c = 0; c < NP; ++c) tile[wid][my_step][piv[c]] = a[c];
      ushr[wid][r] = real ? (float)upper[zrow] : 0.f;
    }
    __syncwarp();
    if (real) {
      float *out = dinv + zrow * n;
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c < n) out[c] = tile[wid][r][c];
    }
  }
}

template <int NP>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
k_solve_w32(int n, int n_r, int n_sys, const float *__restrict__ dinv, const double *__restrict__ lower,
            const double *__restrict__ upper, const double *__restrict__ rhs, double *__restrict__ x,
            const int *__restrict__ ray_list) {
  const unsigned full = 0xffffffffu;
  const int wid = threadIdx.x >> 5, r = threadIdx.x & 31;
  const long jsys = (long)blockIdx.x * kWarpsPerCta + wid;
  if (jsys >= n_sys) return;
  const long sys = system_of(jsys, ray_list);
  const bool real = r < n;
  const size_t base = (size_t)sys * n_r * n;
  // Power-of-two scaling of the right-hand side (FP32 range), as in the CTA kernel.
  double m = 0.0;
  if (real)
    for (int i = 0; i < n_r; ++i) m = fmax(m, fabs(rhs[base + (size_t)i * n + r]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(full, m, off));
  double scale = 1.0;
  if (m > 0.0 && isfinite(m)) {
    int e;
    frexp(m, &e);
    scale = ldexp(1.0, -e);
  }
  float nrow[NP], rowv[NP];
#pragma unroll
  for (int c = 0; c < NP; ++c) nrow[c] = 0.f;
  double nb = 0.0, nc = 0.0;
  auto load = [&](int i, bool fwd) {
    const size_t zr = base + (size_t)i * n + r;
    const float *src = dinv + zr * n;
#pragma unroll
    for (int c = 0; c < NP; ++c) nrow[c] = (c < n) ? src[c] : 0.f;
    nb = fwd ? rhs[zr] : x[zr];
    nc = fwd ? (i > 0 ? lower[zr] : 0.0) : (i < n_r - 1 ? upper[zr] : 0.0);
  };
  if (real) load(0, true);
  float g_prev = 0.f;
  for (int i = 0; i < n_r; ++i) {
#pragma unroll
    for (int c = 0; c < NP; ++c) rowv[c] = nrow[c];
    const double b = nb, l = nc;
    if (real && i + 1 < n_r) load(i + 1, true);
    const float v = real ? (float)(b * scale) - (float)l * g_prev : 0.f;
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
    for (int c = 0; c < NP; c += 2) {
      acc0 = fmaf(rowv[c], __shfl_sync(full, v, c), acc0);
      if (c + 1 < NP) acc1 = fmaf(rowv[c + 1], __shfl_sync(full, v, c + 1), acc1);
    }
    const float g = acc0 + acc1;
    if (real) x[base + (size_t)i * n + r] = (double)g;
    g_prev = g;
  }
  if (real) load(n_r - 1, false);
  float x_next = 0.f;
  for (int i = n_r - 1; i >= 0; --i) {
#pragma unroll
    for (int c = 0; c < NP; ++c) rowv[c] = nrow[c];
    const double gz = nb, u = nc;
    if (real && i > 0) load(i - 1, false);
    const float v = real ? (float)u * x_next : 0.f;
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
    for (int c = 0; c < NP; c += 2) {
      acc0 = fmaf(rowv[c], __shfl_sync(full, v, c), acc0);
      if (c + 1 < NP) acc1 = fmaf(rowv[c + 1], __shfl_sync(full, v, c + 1), acc1);
    }
    const float xi = gz - (acc0 + acc1);
    if (real) x[base + (size_t)i * n + r] = (double)xi / scale;
    x_next = xi;
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
  // Ring depth: up to 12 zones ahead, with the ring of both warps under 44 KB of static smem.
  static constexpr int FIT = 45056 / (2 * NP * NP * 4);
  static constexpr int STAGES = FIT < 12 ? FIT : 12;
  static constexpr int WPC = 2;                              // warps (systems) per CTA
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

// Per-system max |rhs| (for the power-of-two scaling of the FP32 solve), one CTA per system,
// coalesced over the system's contiguous n_r x n right-hand side.
__global__ void k_sysmax(int n, int n_r, const double *__restrict__ rhs, const int *__restrict__ ray_list,
                         int *__restrict__ sys_exp) {
  __shared__ double red[256];
  const long sys = system_of(blockIdx.x, ray_list);
  const size_t base = (size_t)sys * n_r * n, cnt = (size_t)n_r * n;
  double m = 0.0;
  for (size_t e = threadIdx.x; e < cnt; e += blockDim.x) m = fmax(m, fabs(rhs[base + e]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // k with max |rhs| 2^k in [0.5, 1): the exponent field read off the bit pattern.
    m = red[0];
    const long long b = __double_as_longlong(m);
    const int e = (int)((b >> 52) & 0x7ff);
    sys_exp[blockIdx.x] = (m > 0.0 && e < 0x7ff) ? 1022 - e : 0;
  }
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

template <int NP, bool VEC>
__global__ void __launch_bounds__(SolveRing<NP>::WPC * 32)
k_solve_tma(int n, int n_r, int n_sys, const float *__restrict__ dinv, const float *__restrict__ lower,
            const float *__restrict__ upper, const double *__restrict__ rhs, double *__restrict__ x,
            float *__restrict__ g32, const int *__restrict__ ray_list, const int *__restrict__ sys_exp, int *err) {
  using R = SolveRing<NP>;
  constexpr int S = R::STAGES;
  constexpr int D = 8;                                      // depth of the per-lane vector queue
  __shared__ __align__(128) unsigned char ring[R::WPC][S][NP * NP * 4];
  __shared__ __align__(16) float vbuf[R::WPC][NP];          // the zone vector, broadcast through smem
  __shared__ __align__(8) unsigned long long bar[R::WPC][S];
  const unsigned full = 0xffffffffu;
  const int wid = threadIdx.x >> 5, r = threadIdx.x & 31;
  const long jsys = (long)blockIdx.x * R::WPC + wid;
  if (jsys >= n_sys) return;
  const long sys = system_of(jsys, ray_list);
  const bool real = r < n;
  const size_t base = (size_t)sys * n_r * n;
  const unsigned blk = (unsigned)(n * n * 4);
  const int kexp = sys_exp[jsys];             // rhs is scaled by 2^kexp before rounding to FP32
  if (r == 0) {
    for (int k = 0; k < S; ++k) mbar_init(&bar[wid][k], 1);
    mbar_fence_init();
  }
  __syncwarp();

  // Use u < n_r is forward zone u, u >= n_r backward zone 2 n_r - 1 - u; one bulk copy (the
  // zone's inverse block) per use.
  auto zone_of = [&](int u) { return u < n_r ? u : 2 * n_r - 1 - u; };
  auto issue = [&](int u) {
    unsigned long long *b = &bar[wid][u % S];
    mbar_expect_tx(b, blk);
    bulk_g2s(ring[wid][u % S], dinv + (base + (size_t)zone_of(u) * n) * n, blk, b);
  };
  auto wait = [&](int u, int issued_to) -> bool {
    bool ok = mbar_wait_bounded(&bar[wid][u % S], (unsigned)((u / S) & 1));
    ok = __all_sync(full, ok);
    if (!ok) {                                    // give up: flag, drain own copies, return
      if (r == 0) {
        atomicExch(err, 1);
        for (int v = u + 1; v <= issued_to; ++v) mbar_wait_bounded(&bar[wid][v % S], (unsigned)((v / S) & 1));
      }
      __syncwarp();
    }
    return ok;
  };
  // Per-lane queue of the zone vectors (own row), D uses ahead in a ring of registers indexed
  // by compile-time slots (the zone loop is unrolled by D), all in FP32: the rhs is rescaled by
  // exponent arithmetic, so no FP64-pipe work sits on the recurrence.
  // The loaded values are queued as loaded (the rhs as FP64) and converted when consumed, so
  // each load has D zone steps to arrive.
  double qa[D];
  float qb[D];
  auto fetch = [&](int u, double &va, float &vb) {
    va = 0.0;
    vb = 0.f;
    if (!real || u >= 2 * n_r) return;
    const int i = zone_of(u);
    const size_t zr = base + (size_t)i * n + r;
    if (u < n_r) {
      va = rhs[zr];
      vb = i > 0 ? lower[zr] : 0.f;
    } else {
      va = (double)g32[zr];                         // forward result written by this lane
      vb = i < n_r - 1 ? upper[zr] : 0.f;
    }
  };
  float *vb = vbuf[wid];
  const int rr = real ? r : 0;                      // lanes without a row read row 0 (result unused)

  int issued = -1;
  if (r == 0)
    for (int u = 0; u < S - 1 && u < n_r; ++u) issue(u);
  issued = (S - 1 < n_r ? S - 1 : n_r) - 1;
#pragma unroll
  for (int d = 0; d < D; ++d) fetch(d < n_r ? d : 2 * n_r, qa[d], qb[d]);
  float g_prev = 0.f;
  for (int i0 = 0; i0 < n_r; i0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int i = i0 + d;
      if (i >= n_r) break;
      const float b = d2f_exp2(qa[d], kexp), l = qb[d];
      fetch(i + D < n_r ? i + D : 2 * n_r, qa[d], qb[d]);
      if (!wait(i, issued)) return;
      if (r < NP) vb[r] = real ? b - l * g_prev : 0.f;
      __syncwarp();
      const float g = row_dot<NP, VEC>((const float *)ring[wid][i % S] + (size_t)rr * n, vb, n);
      if (real) g32[base + (size_t)i * n + r] = g;
      g_prev = g;
      __syncwarp();
      const int nu = i + S - 1;
      if (nu < n_r) {
        if (r == 0) issue(nu);
        issued = nu;
      }
    }
  }
  if (r == 0)
    for (int u = n_r; u < n_r + S - 1 && u < 2 * n_r; ++u) issue(u);
  issued = (n_r + S - 1 < 2 * n_r ? n_r + S - 1 : 2 * n_r) - 1;
#pragma unroll
  for (int d = 0; d < D; ++d) fetch(n_r + d, qa[d], qb[d]);
  float x_next = 0.f;
  for (int k0 = 0; k0 < n_r; k0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int k = k0 + d;
      if (k >= n_r) break;
      const int u = n_r + k, i = n_r - 1 - k;
      const float gz = (float)qa[d], uu = qb[d];
      fetch(u + D, qa[d], qb[d]);
      if (!wait(u, issued)) return;
      if (r < NP) vb[r] = real ? uu * x_next : 0.f;
      __syncwarp();
      const float xi = gz - row_dot<NP, VEC>((const float *)ring[wid][u % S] + (size_t)rr * n, vb, n);
      if (real) x[base + (size_t)i * n + r] = f2d_exp2(xi, -kexp);
      x_next = xi;
      __syncwarp();
      const int nu = u + S - 1;
      if (nu < 2 * n_r) {
        if (r == 0) issue(nu);
        issued = nu;
      }
    }
  }
}

cudaError_t launch_solve_tma(int n, int n_r, int n_sys, const void *dinv, const float *lower32,
                             const float *upper32, const double *rhs, double *x, float *g32,
                             const int *ray_list, int *sys_exp, int *err, cudaStream_t s) {
  if (n_sys == 0) return cudaSuccess;
  k_sysmax<<<n_sys, 256, 0, s>>>(n, n_r, rhs, ray_list, sys_exp);
  MGFLD_DISPATCH_NP(n, {
    using R = SolveRing<NP>;
    const unsigned grid = (unsigned)((n_sys + R::WPC - 1) / R::WPC);
    if (n == NP)
      k_solve_tma<NP, true><<<grid, R::WPC * 32, 0, s>>>(n, n_r, n_sys, (const float *)dinv, lower32, upper32, rhs,
                                                         x, g32, ray_list, sys_exp, err);
    else
      k_solve_tma<NP, false><<<grid, R::WPC * 32, 0, s>>>(n, n_r, n_sys, (const float *)dinv, lower32, upper32,
                                                          rhs, x, g32, ray_list, sys_exp, err);
    return cudaGetLastError();
  })
}

template <int NP>
static cudaError_t run_factor(int n, int n_r, int n_sys, const void *diag, int diag_fp32, const double *lower,
                              const double *upper, void *dinv, const int *ray_list, cudaStream_t s) {
  constexpr int SPC = Pack<NP>::SPC;
  const unsigned grid = (unsigned)((n_sys + SPC - 1) / SPC);
  if (diag_fp32)
    k_factor<NP, float><<<grid, Pack<NP>::THREADS, 0, s>>>(n, n_r, n_sys, (const float *)diag, lower, upper,
                                                           (double *)dinv, ray_list);
  else
    k_factor<NP, double><<<grid, Pack<NP>::THREADS, 0, s>>>(n, n_r, n_sys, (const double *)diag, lower, upper,
                                                            (double *)dinv, ray_list);
  return cudaGetLastError();
}

template <int NP, typename T>
static cudaError_t run_solve(int n, int n_r, int n_sys, const void *dinv, const double *lower,
                             const double *upper, const double *rhs, double *x, const int *ray_list,
                             cudaStream_t s) {
  constexpr int SPC = Pack<NP>::SPC;
  const unsigned grid = (unsigned)((n_sys + SPC - 1) / SPC);
  k_solve<NP, T><<<grid, Pack<NP>::THREADS, 0, s>>>(n, n_r, n_sys, (const T *)dinv, lower, upper, rhs, x,
                                                    ray_list);
  return cudaGetLastError();
}

cudaError_t launch_factor(int n, int n_r, int n_sys, const void *diag, int diag_fp32, const double *lower,
                          const double *upper, void *dinv, int precision, const int *ray_list,
                          cudaStream_t s) {
  if (n_sys == 0) return cudaSuccess;
  if (precision == MGFLD_MIXED) {
    const unsigned grid = (unsigned)((n_sys + kWarpsPerCta - 1) / kWarpsPerCta);
    if (diag_fp32) {
      MGFLD_DISPATCH_NP(n, k_factor_w32<NP, float, double><<<grid, kWarpsPerCta * 32, 0, s>>>(
                               n, n_r, n_sys, (const float *)diag, lower, upper, (float *)dinv, ray_list);
                           return cudaGetLastError())
    } else {
      MGFLD_DISPATCH_NP(n, k_factor_w32<NP, double, double><<<grid, kWarpsPerCta * 32, 0, s>>>(
                               n, n_r, n_sys, (const double *)diag, lower, upper, (float *)dinv, ray_list);
                           return cudaGetLastError())
    }
  } else {
    MGFLD_DISPATCH_NP(n, return (run_factor<NP>(n, n_r, n_sys, diag, diag_fp32, lower, upper, dinv,
                                                        ray_list, s)))
  }
}

cudaError_t launch_factor_f32(int n, int n_r, int n_sys, const float *diag, const float *lower32,
                              const float *upper32, float *dinv, const int *ray_list, cudaStream_t s) {
  if (n_sys == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n_sys + kWarpsPerCta - 1) / kWarpsPerCta);
  MGFLD_DISPATCH_NP(n, k_factor_w32<NP, float, float><<<grid, kWarpsPerCta * 32, 0, s>>>(
                           n, n_r, n_sys, diag, lower32, upper32, dinv, ray_list);
                       return cudaGetLastError())
}

cudaError_t launch_solve(int n, int n_r, int n_sys, const void *dinv, const double *lower,
                         const double *upper, const double *rhs, double *x, int precision,
                         const int *ray_list, cudaStream_t s) {
  if (n_sys == 0) return cudaSuccess;
  if (precision == MGFLD_MIXED) {
    const unsigned grid = (unsigned)((n_sys + kWarpsPerCta - 1) / kWarpsPerCta);
    MGFLD_DISPATCH_NP(n, k_solve_w32<NP><<<grid, kWarpsPerCta * 32, 0, s>>>(n, n_r, n_sys, (const float *)dinv,
                                                                          lower, upper, rhs, x, ray_list);
                         return cudaGetLastError())
  } else {
    MGFLD_DISPATCH_NP(n, return (run_solve<NP, double>(n, n_r, n_sys, dinv, lower, upper, rhs, x, ray_list, s)))
  }
}

}  // namespace mgfld
