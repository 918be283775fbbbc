// Neutrino stress and lapse update (Sec. "Solution of the Transport Equations", Eqs. a62e-a62l).
//
// mgfld_stress_lapse evaluates the transport step's coefficients at the state it is given (the
// same setup kernels; the flux limiter of every edge is kept), then
//   k_stress: a thread per (ray, edge i+1/2): f = -(4 pi/(hc)^3)/3 sum_q N_q sum_k F (X_{i+1} - X_i)
//             A_{i+1/2} / Delta M_{i+1/2}, X = eps^3 d eps psi0 on each zone's comoving grid
//             (Eqs. a62e-a62f), and the zone value, the mean of its two edges (Eq. a62i);
//   k_lapse:  a warp per ray: the enclosed rest mass (warp reduction), the exterior lapse at the
//             outer edge (Eq. a62k), and the inward product of Eq. a62l written as one exponential
//             of a suffix sum, a_i = a_I exp(sum_{j >= i} x_j), x_j the bracket over rho c^2.
// Readings: the stress term of Eq. a62l is Delta M f / (4 pi R^2) (a force per area, as the
// pressure difference beside it); Eq. a62k carries the square root of the Schwarzschild lapse;
// the scan starts with a_I = a_{I+1/2}; the outer edge uses the transport's ghost zone and the
// centre edge carries no stress; the enclosed mass adds the caller's mass inside the innermost
// edge to sum rho V.
#include "mgfld_internal.cuh"

namespace mgfld {

constexpr double kG = 6.67430e-8;            // cm^3 g^-1 s^-2
constexpr double kMeVErg = 1.602176634e-6;

cudaError_t launch_setup(const Prob &p, const Ws &w, const double *psi, const double *ye, const double *T,
                         cudaStream_t s);

__global__ void k_stress(Prob p, Ws w, const double *__restrict__ psi, double *__restrict__ f_edge,
                         double *__restrict__ f_zone) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)(p.n_ray * p.n_r)) return;
  const int n = p.n, last = p.n_r - 1;
  const int ray = (int)(t / (unsigned)p.n_r), i = (int)(t - (unsigned)ray * p.n_r);
  const size_t zi = t;
  // f at edge e (e = i - 1 or i) of this ray, from zones e and e+1 (ghost beyond the last zone)
  auto edge = [&](int e) -> double {
    const double *z = w.zone + ((size_t)ray * p.n_r + e) * ZC_N;
    const double ia = z[ZC_INV_A], ia4 = ia * ia * ia * ia;
    const double dM = p.rho[(size_t)ray * p.n_r + e] * z[ZC_VOL];
    double ia4r = ia4, dMr = dM;
    if (e < last) {
      const double *zr = z + ZC_N;
      const double iar = zr[ZC_INV_A];
      ia4r = iar * iar * iar * iar;
      dMr = p.rho[(size_t)ray * p.n_r + e + 1] * zr[ZC_VOL];
    }
    double s = 0.0;
    for (int q = 0; q < NS; ++q) {
      const size_t row = (((size_t)ray * NS + q) * p.n_r + e) * n;
      double sq = 0.0;
      for (int k = 0; k < n; ++k) {
        const double x = psi[row + k] * ia4;
        const double xr = e < last ? psi[row + n + k] * ia4r : w.ghost[((size_t)ray * NS + q) * n + k] * x;
        sq += w.lim[row + k] * (xr - x) * (w.E[k] * w.W[k]);
      }
      s += stat_weight(q) * sq;
    }
    const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
    const double A = 4.0 * kPi * re[e + 1] * re[e + 1];
    const double dMe = e < last ? 0.5 * (dM + dMr) : dM;
    return -kFourPiHC3 / 3.0 * kMeVErg * s * A / dMe;
  };
  const double fo = edge(i);
  const double fi = i > 0 ? edge(i - 1) : 0.0;
  if (f_edge) f_edge[zi] = fo;
  if (f_zone) f_zone[zi] = 0.5 * (fo + fi);
}

// One warp per ray.  Lane l takes the contiguous zones [l c, (l + 1) c), c = ceil(n_r / 32).
__global__ void k_lapse(Prob p, const double *__restrict__ pres, const double *__restrict__ m_inner,
                        const double *__restrict__ f_edge, const double *__restrict__ vol_src, int vol_stride,
                        double *__restrict__ lapse) {
  const int ray = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (ray >= p.n_ray) return;
  const int nr = p.n_r, c = (nr + 31) / 32;
  const int lo = lane * c, hi = min(lo + c, nr);
  const double *rho = p.rho + (size_t)ray * nr, *pr = pres + (size_t)ray * nr, *fe = f_edge + (size_t)ray * nr;
  const double *re = p.r_edge + (size_t)ray * (nr + 1);
  const double *vol = vol_src + (size_t)ray * nr * vol_stride;
  // enclosed rest mass
  double m = 0.0;
  for (int i = lo; i < hi; ++i) m += rho[i] * vol[(size_t)i * vol_stride];
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  m += m_inner ? m_inner[ray] : 0.0;
  const double a_out = sqrt(1.0 - 2.0 * kG * m / (kC * kC * re[nr]));
  // x_j for the edges j + 1/2 below the last zone; local suffix sums inside the lane's chunk
  double acc = 0.0;
  for (int i = hi - 1; i >= lo; --i) {
    if (i < nr - 1) {
      const double rho_e = 0.5 * (rho[i] + rho[i + 1]);
      const double dM_e = 0.5 * (rho[i] * vol[(size_t)i * vol_stride] + rho[i + 1] * vol[(size_t)(i + 1) * vol_stride]);
      const double R = re[i + 1];
      acc += (pr[i + 1] - pr[i] - dM_e / (4.0 * kPi * R * R) * fe[i]) / (rho_e * kC * kC);
    }
  }
  // exclusive suffix sum of the lanes' totals (lanes above this one)
  double above = 0.0, v = acc;
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v += u;
  }
  above = v - acc;
  // second pass: each zone's suffix sum and its lapse
  double run = above;
  for (int i = hi - 1; i >= lo; --i) {
    if (i < nr - 1) {
      const double rho_e = 0.5 * (rho[i] + rho[i + 1]);
      const double dM_e = 0.5 * (rho[i] * vol[(size_t)i * vol_stride] + rho[i + 1] * vol[(size_t)(i + 1) * vol_stride]);
      const double R = re[i + 1];
      run += (pr[i + 1] - pr[i] - dM_e / (4.0 * kPi * R * R) * fe[i]) / (rho_e * kC * kC);
    }
    lapse[(size_t)ray * nr + i] = a_out * exp(run);
  }
}

}  // namespace mgfld

using namespace mgfld;

extern "C" mgfld_status mgfld_stress_lapse(const mgfld_dims *dims, const mgfld_problem *prob,
                                           const mgfld_state *state, const mgfld_stress_io *io, void *ws,
                                           size_t ws_bytes, void *stream) {
  if (!dims_ok(dims) || !prob_ok(prob) || !state || !state->psi || !state->ye || !state->T || !io || !ws)
    return MGFLD_EINVAL;
  if (io->lapse && !io->p) return MGFLD_EINVAL;
  if (((uintptr_t)ws & 255u) != 0) return MGFLD_EINVAL;
  const Layout L = make_layout(dims->n_ray, dims->n_r, dims->n_e, MGFLD_FP64);
  if (ws_bytes < L.total) return MGFLD_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  Ws w = resolve(ws, L);
  w.lim = w.lower;                       // the limiter of every edge (lower is free here)
  Prob p = make_prob(dims, prob);
  p.u = nullptr;                         // the shock terms do not enter the stress
  if (launch_setup(p, w, state->psi, state->ye, state->T, s) != cudaSuccess) return MGFLD_ECUDA;
  const size_t nz = (size_t)dims->n_ray * dims->n_r;
  // the edge stress is needed by the lapse even when the caller does not keep it
  double *fe = io->f_edge ? io->f_edge : w.rhs;
  k_stress<<<(unsigned)((nz + 127) / 128), 128, 0, s>>>(p, w, state->psi, fe, io->f_zone);
  if (cudaGetLastError() != cudaSuccess) return MGFLD_ECUDA;
  if (io->lapse) {
    k_lapse<<<(unsigned)((dims->n_ray + 3) / 4), 128, 0, s>>>(p, io->p, io->m_inner, fe, w.zone + ZC_VOL, ZC_N,
                                                             io->lapse);
    if (cudaGetLastError() != cudaSuccess) return MGFLD_ECUDA;
  }
  return MGFLD_OK;
}
