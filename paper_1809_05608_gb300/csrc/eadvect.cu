// Energy-advection step (Sec. "Neutrino Energy Advection Step" and its appendix on the lapse):
// the Lagrangian shift of each group in energy (Eqs. a78-a80, eta2 from the Minerbo closure,
// Eqs. a86-a87), the parabolic remap of eps^2 psi back to the grid tied to the new lapse with the
// energy-fixing factor (Eqs. a81, h9-h17, h22-h24, h31-h35 in Cartesian form, p5-p8), and the
// occupation limiter (Eqs. a81a-a81d).
//
// A block takes SPB consecutive (ray, species, zone) systems and one thread per (system, group):
// the systems' rows of psi (and eta1) are contiguous, so loads and stores are coalesced; each
// phase of the remap (shifted edges, cell averages, slopes, interface values, parabolas, fluxes)
// runs over the elements in shared memory between block barriers, and the per-system parts (the
// zone's constants, the three energy sums of xi, the sequential limiter) run on the system's
// first thread.  All arithmetic is FP64.  The PPM limiters are continuous in their inputs, so
// rounding differences against a CPU evaluation (FMA contraction) move results by rounding only.
#include "mgfld_internal.cuh"

namespace mgfld {

constexpr int kEadvThreads = 256;

__device__ inline double cube_moment(double lo, double hi) { return (hi * hi * hi - lo * lo * lo) / 3.0; }
__device__ inline double centre(double lo, double hi) { return sqrt((hi * hi + hi * lo + lo * lo) / 3.0); }

// Minerbo closure (Eqs. a86-a87) with eta2_thick = 1/3 and eta2_thin = 1.
__device__ inline double minerbo_eta2(double eta1) {
  const double x = fmin(fmax(eta1, 0.0), 1.0);
  const double p = 1.0 / 3.0 + 2.0 * x * x / 15.0 * (3.0 - x + 3.0 * x * x);
  return 1.5 * (1.0 - p) * (1.0 / 3.0) + 0.5 * (3.0 * p - 1.0);
}

struct EadvArgs {
  int n_ray, n_r, n, spb, limit;
  const double *r_n, *r_np1, *rho_n, *rho_np1, *a_n, *a_np1, *e_edge, *eta1;
  double *psi, *xi;
};

// Shared-memory layout per system (stride per array, in doubles):
//   E_d[n+1] shifted edges at infinity, eps_t[n+1] target edges, nd[n] numbers on the shifted
//   groups, A[n+4], X[n+4] cell averages and widths with two ghost groups at each end, dm[n+4]
//   monotonised slopes, face[n+4] interface values, aL/aR/a6[n], F[n+1] fluxes, eta2[n], zc[4]
//   zone constants (da/a - dR/R, db/b - dR/R, a^{n+1}, the number factor of Eq. a78), sums[4].
__host__ __device__ inline int eadv_stride(int n) { return 13 * (n + 5) + 8; }

__global__ void __launch_bounds__(kEadvThreads) k_energy_advect(EadvArgs g) {
  extern __shared__ double sh[];
  const int n = g.n, spb = g.spb, st = eadv_stride(n);
  const unsigned n_sys = (unsigned)g.n_ray * NS * (unsigned)g.n_r;
  const unsigned s0 = blockIdx.x * (unsigned)spb;
  const int tid = threadIdx.x;
  const int sl = tid / n, k = tid - sl * n;
  const unsigned sg = s0 + (unsigned)sl;
  const bool live = sl < spb && sg < n_sys;
  double *base = sh + (size_t)(live ? sl : 0) * st;
  double *E_d = base, *eps_t = E_d + (n + 5), *nd = eps_t + (n + 5), *A = nd + (n + 5), *X = A + (n + 5);
  double *dm = X + (n + 5), *face = dm + (n + 5), *aL = face + (n + 5), *aR = aL + (n + 5), *a6 = aR + (n + 5);
  double *F = a6 + (n + 5), *eta2 = F + (n + 5), *epsd_c = eta2 + (n + 5), *zc = epsd_c + (n + 5);
  // system (ray, q, i) and its zone
  const unsigned ray = live ? sg / (NS * (unsigned)g.n_r) : 0;
  const unsigned i = live ? sg % (unsigned)g.n_r : 0;
  const size_t zi = (size_t)ray * g.n_r + i;
  const size_t el = (size_t)sg * n + k;
  double psi0 = 0.0;
  // Phase 1: the zone's constants (first thread of the system) and eta2 per group.
  if (live) {
    psi0 = g.psi[el];
    eta2[k] = g.eta1 ? minerbo_eta2(g.eta1[el]) : 1.0 / 3.0;
    if (k == 0) {
      const double *re0 = g.r_n + ray * (size_t)(g.n_r + 1) + i, *re1 = g.r_np1 + ray * (size_t)(g.n_r + 1) + i;
      const double r0 = 0.5 * (re0[0] + re0[1]), r1 = 0.5 * (re1[0] + re1[1]);
      const double rho0 = g.rho_n[zi], rho1 = g.rho_np1[zi];
      const double a0 = g.a_n ? g.a_n[zi] : 1.0, a1 = g.a_np1 ? g.a_np1[zi] : 1.0;
      const double b0 = 1.0 / (4.0 * kPi * r0 * r0 * rho0), b1 = 1.0 / (4.0 * kPi * r1 * r1 * rho1);
      const double da_a = (a1 - a0) / a0, dr_r = (r1 - r0) / r0, db_b = (b1 - b0) / b0;
      zc[0] = da_a - dr_r;
      zc[1] = db_b - dr_r;
      zc[2] = a1;
      zc[3] = (rho1 * a1 * a1 * a1) / (rho0 * a0 * a0 * a0);
    }
  }
  __syncthreads();
  // Phase 2: shifted edges (Eq. a79 at the edges, eta2 the mean of the adjacent groups) and the
  // target edges E / a^{n+1} (Eq. p1); thread k takes edge k, the last group also edge n.
  if (live) {
    const double a1 = zc[2];
    const double e2k = k == 0 ? eta2[0] : 0.5 * (eta2[k - 1] + eta2[k]);
    const double Ek = g.e_edge[k];
    E_d[k] = (1.0 + zc[0] - zc[1] * e2k) * Ek;
    eps_t[k] = Ek / a1;
    if (k == n - 1) {
      const double En = g.e_edge[n];
      E_d[n] = (1.0 + zc[0] - zc[1] * eta2[n - 1]) * En;
      eps_t[n] = En / a1;
    }
  }
  __syncthreads();
  // Phase 3: Eq. a78 (psi on the shifted group, its number nd) and the cell averages eps^2 psi
  // of the parabolic remap, with two zero-slope ghost groups at each end.
  if (live) {
    const double a1 = zc[2];
    const double El = g.e_edge[k], Eh = g.e_edge[k + 1];
    const double psi_d = zc[3] * (cube_moment(El, Eh) / cube_moment(E_d[k], E_d[k + 1])) * psi0;
    const double lo = E_d[k] / a1, hi = E_d[k + 1] / a1;
    const double num = psi_d * cube_moment(lo, hi);
    const double dx = hi - lo;
    nd[k] = num;
    epsd_c[k] = centre(lo, hi);
    A[k + 2] = num / dx;
    X[k + 2] = dx;
    if (k == 0) {
      A[0] = A[1] = num / dx;
      X[0] = X[1] = dx;
    }
    if (k == n - 1) {
      A[n + 2] = A[n + 3] = num / dx;
      X[n + 2] = X[n + 3] = dx;
    }
  }
  __syncthreads();
  // Phase 4: average slopes (Eq. h9) monotonised (Eq. h11) at extended groups 1..n+2.
  auto slope = [&](int j) {
    const double xl = X[j - 1], x0 = X[j], xr = X[j + 1];
    const double dp = A[j + 1] - A[j], dn = A[j] - A[j - 1];
    const double s = x0 / (xl + x0 + xr) * ((2.0 * xl + x0) / (xr + x0) * dp + (x0 + 2.0 * xr) / (xl + x0) * dn);
    const double lim = fmin(fabs(s), fmin(2.0 * fabs(dp), 2.0 * fabs(dn)));
    dm[j] = dp * dn > 0.0 ? copysign(lim, s) : 0.0;
  };
  if (live) {
    slope(k + 1);
    if (k < 2) slope(n + 1 + k);
  }
  __syncthreads();
  // Phase 5: interface values between extended groups j and j+1, j = 1..n+1 (Eq. h12, the cubic
  // through the group integrals), limited to the range of the two averages (Eqs. h15-h16).
  auto interface = [&](int j) {
    const double xl = X[j - 1], x0 = X[j], x1 = X[j + 1], x2 = X[j + 2];
    const double d = A[j + 1] - A[j];
    const double tot = xl + x0 + x1 + x2;
    double t = (2.0 * x1 * x0 / (x0 + x1)) * ((xl + x0) / (2.0 * x0 + x1) - (x2 + x1) / (2.0 * x1 + x0)) * d;
    t = t - x0 * (xl + x0) / (2.0 * x0 + x1) * dm[j + 1] + x1 * (x1 + x2) / (x0 + 2.0 * x1) * dm[j];
    double f = A[j] + x0 / (x0 + x1) * d + t / tot;
    f = fmax(f, fmin(A[j], A[j + 1]));
    f = fmin(f, fmax(A[j], A[j + 1]));
    face[j] = f;
  };
  if (live) {
    interface(k + 1);
    if (k == 0) interface(n + 1);
  }
  __syncthreads();
  // Phase 6: the parabola of each shifted group (Eqs. h17, h22-h24) with the monotonicity
  // corrections (Eqs. h31-h35, Cartesian form).
  if (live) {
    const double a = A[k + 2];
    double l = face[k + 1], r = face[k + 2];
    const double d = r - l, s6 = 6.0 * (a - 0.5 * (l + r));
    const bool lm = d * d < d * s6, rm = d * d < -d * s6;
    const double l2 = lm ? 3.0 * a - 2.0 * r : l;
    const double r2 = rm ? 3.0 * a - 2.0 * l : r;
    aL[k] = l2;
    aR[k] = r2;
    a6[k] = 6.0 * (a - 0.5 * (l2 + r2));
  }
  __syncthreads();
  // Phase 7: the flux across target edge k (Eq. p5): the number in the slice between the shifted
  // and the target edge, from the parabola of the group the slice belongs to; zero at the two
  // outer edges.  Also the target group centres (eta2 is no longer needed: its storage is reused).
  double *ct = eta2;
  if (live) {
    const double a1 = zc[2];
    ct[k] = centre(eps_t[k], eps_t[k + 1]);
    if (k == 0) {
      F[0] = 0.0;
      F[n] = 0.0;
    } else {
      const double d = eps_t[k] - E_d[k] / a1;
      double f = 0.0;
      if (d < 0.0) {                  // top of group k-1 moves up into target group k
        const double dx = X[k + 1];
        const double y = fmin(fmax(-d / dx, 0.0), 1.0);
        const double avg = aR[k - 1] - 0.5 * y * ((aR[k - 1] - aL[k - 1]) - (1.0 - 2.0 * y / 3.0) * a6[k - 1]);
        f = avg * y * dx;
      } else if (d > 0.0) {           // bottom of group k moves down into target group k-1
        const double dx = X[k + 2];
        const double y = fmin(fmax(d / dx, 0.0), 1.0);
        const double avg = aL[k] + 0.5 * y * ((aR[k] - aL[k]) + (1.0 - 2.0 * y / 3.0) * a6[k]);
        f = -avg * y * dx;
      }
      F[k] = f;
    }
  }
  __syncthreads();
  // Phase 8: xi (Eqs. p6-p8): the factor on the flux divergence that gives the target groups the
  // energy the shifted groups hold (1 without flux).
  double *sums = zc + 4;
  if (live && k == 0) {
    double eb = 0.0, s1 = 0.0, s2 = 0.0;
    for (int kk = 0; kk < n; ++kk) {
      eb += nd[kk] * epsd_c[kk];
      s1 += nd[kk] * ct[kk];
      s2 += (F[kk] - F[kk + 1]) * ct[kk];
    }
    sums[0] = s2 != 0.0 ? (eb - s1) / s2 : 1.0;
  }
  __syncthreads();
  // Phase 9: Eq. p6 and psi on the target groups (kept in nd).
  if (live) {
    const double xi = sums[0];
    const double num = nd[k] + xi * (F[k] - F[k + 1]);
    nd[k] = num / cube_moment(eps_t[k], eps_t[k + 1]);
  }
  __syncthreads();
  // Phase 10: the occupation limiter (Eqs. a81a-a81d), sequential over groups k = 0..n-3.
  if (live && g.limit && k == 0) {
    bool over = false;
    for (int kk = 0; kk < n - 2; ++kk) over |= nd[kk] > 1.0;
    if (over) {
      for (int kk = 0; kk < n - 2; ++kk) {
        double d = nd[kk] - 1.0;
        if (!(d > 0.0)) continue;
        const double e0 = ct[kk], e1 = ct[kk + 1], e2 = ct[kk + 2];
        const double w0 = e0 * e0 * (eps_t[kk + 1] - eps_t[kk]);
        const double w1 = e1 * e1 * (eps_t[kk + 2] - eps_t[kk + 1]);
        const double w2 = e2 * e2 * (eps_t[kk + 3] - eps_t[kk + 2]);
        const double c_up = (e2 - e0) * w0 / ((e2 - e1) * w1);
        const double c_dn = (e1 - e0) * w0 / ((e2 - e1) * w2);
        d = fmin(d, fmax(nd[kk + 2], 0.0) / c_dn);   // never take group k + 2 below zero
        nd[kk] -= d;
        nd[kk + 1] += c_up * d;
        nd[kk + 2] -= c_dn * d;
      }
    }
  }
  __syncthreads();
  if (live) {
    g.psi[el] = nd[k];
    if (k == 0 && g.xi) g.xi[sg] = sums[0];
  }
}

}  // namespace mgfld

using namespace mgfld;

extern "C" mgfld_status mgfld_energy_advect(const mgfld_dims *dims, const mgfld_eadv_problem *prob, double *psi,
                                            double *xi, void *stream) {
  if (!dims_ok(dims) || dims->n_e < 3 || !prob || !psi || !prob->r_edge_n || !prob->r_edge_np1 || !prob->rho_n ||
      !prob->rho_np1 || !prob->e_edge)
    return MGFLD_EINVAL;
  EadvArgs g;
  g.n_ray = dims->n_ray;
  g.n_r = dims->n_r;
  g.n = dims->n_e;
  g.spb = kEadvThreads / g.n;
  g.limit = prob->limit != 0;
  g.r_n = prob->r_edge_n;
  g.r_np1 = prob->r_edge_np1;
  g.rho_n = prob->rho_n;
  g.rho_np1 = prob->rho_np1;
  g.a_n = prob->lapse_n;
  g.a_np1 = prob->lapse_np1;
  g.e_edge = prob->e_edge;
  g.eta1 = prob->eta1;
  g.psi = psi;
  g.xi = xi;
  const size_t n_sys = (size_t)g.n_ray * NS * g.n_r;
  const unsigned grid = (unsigned)((n_sys + g.spb - 1) / g.spb);
  const unsigned threads = (unsigned)((g.spb * g.n + 31) / 32 * 32);
  const size_t smem = sizeof(double) * (size_t)g.spb * eadv_stride(g.n);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_energy_advect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MGFLD_ECUDA;
  k_energy_advect<<<grid, threads, smem, (cudaStream_t)stream>>>(g);
  return cudaGetLastError() == cudaSuccess ? MGFLD_OK : MGFLD_ECUDA;
}
