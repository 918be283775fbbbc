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

// 1/x for x of either precision.  FP64: FP32 seed refined by two Newton-Raphson steps
// x_{m+1} = x_m (2 - d x_m) (quadratic convergence: 24 -> 48 -> full bits), which keeps
// the FP64 pipe to four fused multiply-adds; outside the FP32 range a plain division.
__device__ inline double recip(double d) {
  const double ad = fabs(d);
  if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
  double x = (double)__frcp_rn((float)d);
  double e = fma(-d, x, 1.0);
  x = fma(x, e, x);
  e = fma(-d, x, 1.0);
  return fma(x, e, x);
}
__device__ inline float recip(float d) { return __frcp_rn(d); }

template <typename T> __device__ inline T to_t(double v);
template <> __device__ inline double to_t<double>(double v) { return v; }
template <> __device__ inline float to_t<float>(double v) { return (float)v; }

// Map the j-th system of the launch to a global (ray, species) system index.
__device__ inline long system_of(long j, const int *ray_list) {
  return ray_list ? (long)ray_list[j / NS] * NS + (j % NS) : j;
}

template <int NP, typename T>
__global__ void __launch_bounds__(Pack<NP>::THREADS)
k_factor(int n, int n_r, int n_sys, const double *__restrict__ diag, const double *__restrict__ lower,
         const double *__restrict__ upper, T *__restrict__ dinv, const int *__restrict__ ray_list) {
  constexpr int SPC = Pack<NP>::SPC;
  __shared__ T tile[SPC][NP][NP + 1];   // natural-order inverse of the previous zone
  __shared__ T prow[SPC][NP];           // pivot row of the current step
  __shared__ T cand[SPC][NP];           // pivot candidates (|a|, -1 once used)
  __shared__ T ushr[SPC][NP];           // upper_{i-1}, the column scaling of the Schur update
  __shared__ int pivrow[SPC][NP];       // row chosen at each step

  const int s = threadIdx.x / NP, r = threadIdx.x % NP;
  const long jsys = (long)blockIdx.x * SPC + s;
  const bool valid = jsys < n_sys;
  const long sys = valid ? system_of(jsys, ray_list) : 0;
  const bool real = valid && r < n;

  // Rows of the next zone are fetched one zone ahead (registers) to hide memory latency.
  T nxt[NP];
  double nl = 0.0;
  auto load_row = [&](int i) {
    const size_t zr = ((size_t)sys * n_r + i) * n + r;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      if (real && c < n) nxt[c] = to_t<T>(diag[zr * n + c]);
      else nxt[c] = (c == r) ? T(1) : T(0);
    }
    nl = (real && i > 0) ? lower[zr] : 0.0;
  };
  load_row(0);
  for (int i = 0; i < n_r; ++i) {
    const size_t zrow = ((size_t)sys * n_r + i) * n + r;   // (sys, i, r)
    T a[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) a[c] = nxt[c];
    const T lr = to_t<T>(nl);
    if (i + 1 < n_r) load_row(i + 1);
    if (i > 0) {
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = a[c] - (lr * tile[s][r][c]) * ushr[s][c];
    }

    // Gauss-Jordan inversion in place with partial pivoting (implicit row exchanges).
    bool used = false;
    int my_step = 0;
#pragma unroll
    for (int pstep = 0; pstep < NP; ++pstep) {
      cand[s][r] = used ? T(-1) : fabs(a[pstep]);
      __syncthreads();
      int best = 0;
      T bv = cand[s][0];
#pragma unroll
      for (int c = 1; c < NP; ++c) {
        const T v = cand[s][c];
        if (v > bv) { bv = v; best = c; }
      }
      const bool me = (r == best);
      if (me) {
#pragma unroll
        for (int c = 0; c < NP; ++c) prow[s][c] = a[c];
        pivrow[s][pstep] = r;
        used = true;
        my_step = pstep;
      }
      __syncthreads();
      const T inv = recip(prow[s][pstep]);
      // Uniform update for every row: a -= f * pivot_row, with f chosen so that the
      // pivot row itself becomes pivot_row / pivot (f = 1 - 1/pivot).
      const T f = me ? (T(1) - inv) : a[pstep] * inv;
#pragma unroll
      for (int c = 0; c < NP; ++c) a[c] = a[c] - f * prow[s][c];
      a[pstep] = me ? inv : -f;
    }
    // Row r now holds row my_step of the inverse, with column c belonging to input row pivrow[c].
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NP; ++c) tile[s][my_step][pivrow[s][c]] = a[c];
    ushr[s][r] = real ? to_t<T>(upper[zrow]) : T(0);
    __syncthreads();
    if (real) {
      T *out = dinv + zrow * n;
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

template <int NP, typename T>
static cudaError_t run_factor(int n, int n_r, int n_sys, const double *diag, const double *lower,
                              const double *upper, void *dinv, const int *ray_list, cudaStream_t s) {
  constexpr int SPC = Pack<NP>::SPC;
  const unsigned grid = (unsigned)((n_sys + SPC - 1) / SPC);
  k_factor<NP, T><<<grid, Pack<NP>::THREADS, 0, s>>>(n, n_r, n_sys, diag, lower, upper, (T *)dinv, ray_list);
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

#define MGFLD_DISPATCH_NP(n, CALL)            \
  if (n <= 4) { constexpr int NP = 4; CALL; }      \
  else if (n <= 8) { constexpr int NP = 8; CALL; } \
  else if (n <= 12) { constexpr int NP = 12; CALL; } \
  else if (n <= 16) { constexpr int NP = 16; CALL; } \
  else if (n <= 20) { constexpr int NP = 20; CALL; } \
  else if (n <= 24) { constexpr int NP = 24; CALL; } \
  else { constexpr int NP = 32; CALL; }

cudaError_t launch_factor(int n, int n_r, int n_sys, const double *diag, const double *lower,
                          const double *upper, void *dinv, int precision, const int *ray_list,
                          cudaStream_t s) {
  if (n_sys == 0) return cudaSuccess;
  if (precision == MGFLD_MIXED) {
    MGFLD_DISPATCH_NP(n, return (run_factor<NP, float>(n, n_r, n_sys, diag, lower, upper, dinv, ray_list, s)))
  } else {
    MGFLD_DISPATCH_NP(n, return (run_factor<NP, double>(n, n_r, n_sys, diag, lower, upper, dinv, ray_list, s)))
  }
}

cudaError_t launch_solve(int n, int n_r, int n_sys, const void *dinv, const double *lower,
                         const double *upper, const double *rhs, double *x, int precision,
                         const int *ray_list, cudaStream_t s) {
  if (n_sys == 0) return cudaSuccess;
  if (precision == MGFLD_MIXED) {
    MGFLD_DISPATCH_NP(n, return (run_solve<NP, float>(n, n_r, n_sys, dinv, lower, upper, rhs, x, ray_list, s)))
  } else {
    MGFLD_DISPATCH_NP(n, return (run_solve<NP, double>(n, n_r, n_sys, dinv, lower, upper, rhs, x, ray_list, s)))
  }
}

}  // namespace mgfld
