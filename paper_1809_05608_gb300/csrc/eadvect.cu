// Energy-advection step (Sec. "Neutrino Energy Advection Step" and its appendix on the lapse):
// the Lagrangian shift of each group in energy (Eqs. a78-a80, eta2 from the Minerbo closure,
// Eqs. a86-a87), the parabolic remap of eps^2 psi back to the grid tied to the new lapse with the
// energy-fixing factor (Eqs. a81, h9-h17, h22-h24, h31-h35 in Cartesian form, p5-p8), and the
// occupation limiter (Eqs. a81a-a81d).
//
// A block takes SPB consecutive (ray, species, zone) systems and one thread per (system, group):
// the systems' rows of psi (and eta1) are contiguous, so loads and stores are coalesced; each
// phase of the remap (shifted edges, cell averages, slopes, interface values, parabolas, fluxes)
// runs over the elements in shared memory between block barriers.  All arithmetic is FP64, and
// the FP64 pipe bounds the kernel (every FP64 warp instruction occupies it for the same time,
// however few lanes are active), so the work is arranged to keep FP64 instructions few and
// warp-wide: the zone's constants are spread over the system's first threads; quotients are
// formed from a reciprocal seeded on the integer and FP32 pipes and refined by Newton steps
// (a few FP64 FMAs instead of a division), the quotients that share a denominator from one of
// them (slopes, interface values), and a group's slope and interface from one reciprocal of the
// product of their denominators; the number on a shifted group needs no quotient (Eq. a78 times
// its moment); cube moments use the factored form (hi^3 - lo^3)/(hi - lo) = hi^2 + hi lo + lo^2;
// the grid at infinity (moments, centres) is formed once per block; and the two sums of xi are
// a tree reduction over the system's threads.  Only the occupation limiter, rarely active, is
// sequential.  The PPM limiters are continuous in their inputs, so these rearrangements move
// results by rounding only.
#include "mgfld_internal.cuh"

namespace mgfld {

constexpr int kEadvThreads = 256;
constexpr double kThird = 1.0 / 3.0;

// eta2 of the Minerbo closure (Eqs. a86-a87): the weighting of the thick (1/3) and thin (1)
// limits by the closure's factor p, (1 - p)/2 + (3p - 1)/2, is p itself.
__device__ inline double eddington_p(double eta1) {
  const double x = fmin(fmax(eta1, 0.0), 1.0);
  return kThird + 2.0 * x * x / 15.0 * (3.0 - x + 3.0 * x * x);
}

struct EadvArgs {
  int n_ray, n_r, n, spb, limit;
  const double *r_n, *r_np1, *rho_n, *rho_np1, *a_n, *a_np1, *e_edge, *eta1, *u;
  double *psi, *xi;
};

// Shared memory: a block header of 3 MAX_NE doubles (per group of the grid at infinity: the
// moment E^2 dE = (E_+^3 - E_-^3)/3, its reciprocal, the centre E_k of Eq. a01b), then per
// system (stride per array, in doubles): E_d[n+1] shifted edges at infinity, nd[n] numbers on
// the shifted groups, A[n+4], X[n+4] cell averages and widths with two ghost groups at each end,
// dm[n+4] monotonised slopes, face[n+4] interface values, aL/aR/a6[n], F[n+1] fluxes, eta2[n]
// (later the target centres), epsd_c[n] shifted centres, red[3][n+5] reduction scratch, zc[10]
// zone constants (a^{n+1}/a^n, R^{n+1}/R^n, b^{n+1}/b^n, the number factor of Eq. a78, 1/a^{n+1},
// the kept fraction of the displacement, xi, the limiter flag, (a^{n+1})^3).
constexpr int kEadvHeader = 3 * MAX_NE;
__host__ __device__ inline int eadv_stride(int n) { return 15 * (n + 5) + 10; }
__host__ __device__ inline size_t eadv_smem(int spb, int n) {
  return sizeof(double) * ((size_t)kEadvHeader + (size_t)spb * eadv_stride(n));
}

__global__ void __launch_bounds__(kEadvThreads) k_energy_advect(EadvArgs g) {
  extern __shared__ double sh[];
  const int n = g.n, spb = g.spb, st = eadv_stride(n);
  const unsigned n_sys = (unsigned)g.n_ray * NS * (unsigned)g.n_r;
  const unsigned s0 = blockIdx.x * (unsigned)spb;
  const int tid = threadIdx.x;
  const int sl = tid / n, k = tid - sl * n;
  const unsigned sg = s0 + (unsigned)sl;
  const bool live = sl < spb && sg < n_sys;
  double *cmE = sh, *icmE = sh + MAX_NE, *Ec = sh + 2 * MAX_NE;
  double *base = sh + kEadvHeader + (size_t)(live ? sl : 0) * st;
  double *E_d = base, *nd = E_d + (n + 5), *A = nd + (n + 5), *X = A + (n + 5);
  double *dm = X + (n + 5), *face = dm + (n + 5), *aL = face + (n + 5), *aR = aL + (n + 5), *a6 = aR + (n + 5);
  double *F = a6 + (n + 5), *eta2 = F + (n + 5), *epsd_c = eta2 + (n + 5), *red = epsd_c + (n + 5);
  double *zc = red + 3 * (n + 5);
  // system (ray, q, i) and its zone
  const unsigned ray = live ? sg / (NS * (unsigned)g.n_r) : 0;
  const unsigned i = live ? sg % (unsigned)g.n_r : 0;
  const size_t zi = (size_t)ray * g.n_r + i;
  const size_t el = (size_t)sg * n + k;
  double psi0 = 0.0;
  // Phase 1: the grid at infinity (block), eta2 per group, and the zone's constants, the
  // system's threads sharing the five divisions: a^{n+1}/a^n, 1/a^{n+1}, R^{n+1}/R^n (R the
  // zone-centre areal radius, the mean of its edges), b^{n+1}/b^n with b = 1/(4 pi R^2 rho), and
  // the number factor (rho a^3)^{n+1}/(rho a^3)^n of Eq. a78; the first thread adds the kept
  // fraction of the displacement.
  if (tid < n) {
    const double lo = g.e_edge[tid], hi = g.e_edge[tid + 1];
    const double q = hi * hi + hi * lo + lo * lo;
    cmE[tid] = (hi - lo) * q * kThird;
    icmE[tid] = recip2(cmE[tid]);
    Ec[tid] = sqrt(q * kThird);
  }
  if (live) {
    psi0 = g.psi[el];
    eta2[k] = g.eta1 ? eddington_p(g.eta1[el]) : kThird;
    // quotient j of the zone (every thread of the system takes one or two, same code path):
    // 0 a^{n+1}/a^n, 1 1/a^{n+1}, 2 R^{n+1}/R^n, 3 b^{n+1}/b^n, 4 the number factor
    const double *re0 = g.r_n + ray * (size_t)(g.n_r + 1) + i, *re1 = g.r_np1 + ray * (size_t)(g.n_r + 1) + i;
    const double a0 = g.a_n ? g.a_n[zi] : 1.0, a1 = g.a_np1 ? g.a_np1[zi] : 1.0;
    const double rho0 = g.rho_n[zi], rho1 = g.rho_np1[zi];
    const double r0 = re0[0] + re0[1], r1 = re1[0] + re1[1];
    for (int j = k; j < 5; j += n) {
      const double num = j == 0 ? a1 : j == 1 ? 1.0 : j == 2 ? r1 : j == 3 ? r0 * r0 * rho0 : rho1 * a1 * a1 * a1;
      const double den = j == 0 ? a0 : j == 1 ? a1 : j == 2 ? r0 : j == 3 ? r1 * r1 * rho1 : rho0 * a0 * a0 * a0;
      zc[j < 2 ? 4 * j : j - 1] = quot(num, den);    // slots 0, 4, 1, 2, 3
    }
    if (k == 0) {
      zc[7] = 0.0;
      zc[8] = a1 * a1 * a1;
      // at a shock the displacement is rolled out by the roll-in weights of the zone's edges
      double keep = 1.0;
      if (g.u) {
        const double *u = g.u + (size_t)ray * g.n_r;
        double wmax = 0.0;
        for (int e = -1; e <= 0; ++e) {               // edges i-1/2 and i+1/2
          const int lo = (int)i + e;
          if (lo < 0 || lo + 1 >= g.n_r) continue;
          const double beta = (u[lo + 1] - u[lo]) / kC;
          wmax = fmax(wmax, fmin(fmax((fabs(beta) - kShockOn) / (kShockFull - kShockOn), 0.0), 1.0));
        }
        keep = 1.0 - wmax;
      }
      zc[5] = keep;
    }
  }
  __syncthreads();
  // Phase 2: shifted edges (Eq. a79 at the edges, eta2 the mean of the adjacent groups):
  // E_d = E (1 + keep [(da/a - dR/R) - (db/b - dR/R) eta2]); thread k takes edge k, the last
  // group also edge n.
  if (live) {
    const double tr = zc[1], keep = zc[5];
    const double c0 = keep * (zc[0] - tr), c1 = keep * (zc[2] - tr);
    const double e2k = k == 0 ? eta2[0] : 0.5 * (eta2[k - 1] + eta2[k]);
    E_d[k] = (1.0 + c0 - c1 * e2k) * g.e_edge[k];
    if (k == n - 1) E_d[n] = (1.0 + c0 - c1 * eta2[n - 1]) * g.e_edge[n];
  }
  __syncthreads();
  // Phase 3: Eq. a78 (psi on the shifted group), its number nd and the cell average eps^2 psi
  // of the parabolic remap (number per unit comoving energy), with two zero-slope ghost groups at
  // each end; the shifted group centre (Eq. a01b).  psi on the shifted group times that group's
  // moment is the number of Eq. a78, so nd = (the number factor) E^2 dE psi^n / (a^{n+1})^3 takes
  // no quotient; the cell average is nd over the comoving width, and 1/(Dh - Dl) serves the
  // fluxes of phase 7 as well (kept in the reduction scratch, free until phase 8).
  double *iw = red + 2 * (n + 5);
  if (live) {
    const double ia1 = zc[4];
    const double Dl = E_d[k], Dh = E_d[k + 1];
    const double dD = Dh - Dl, rw = recip2(dD);
    const double qD = Dh * Dh + Dh * Dl + Dl * Dl;
    const double b2 = zc[3] * cmE[k] * psi0 * (ia1 * ia1);
    iw[k] = rw;
    const double dx = dD * ia1;
    const double avg = b2 * rw;
    nd[k] = b2 * ia1;
    epsd_c[k] = ia1 * sqrt(qD * kThird);
    A[k + 2] = avg;
    X[k + 2] = dx;
    if (k == 0) {
      A[0] = A[1] = avg;
      X[0] = X[1] = dx;
    }
    if (k == n - 1) {
      A[n + 2] = A[n + 3] = avg;
      X[n + 2] = X[n + 3] = dx;
    }
  }
  __syncthreads();
  // Phase 4: average slopes (Eq. h9) monotonised (Eq. h11) at the groups (extended index
  // 2..n+1), the two quotients of Eq. h9 over a common denominator.  The ghost groups copy their
  // neighbour, so one of their two differences is zero and the limiter makes their slopes zero.
  // Thread k takes slope and interface k + 2 (phase 5): one reciprocal of the product of the two
  // denominators serves both (each is the other times it), and the interface's terms that do not
  // involve the slopes are formed here from the same widths.
  double fb = 0.0, cR = 0.0, cL = 0.0, flo = 0.0, fhi = 0.0;
  if (live) {
    const int j = k + 2;
    const double xl = X[j - 1], x0 = X[j], x1 = X[j + 1], x2 = X[j + 2];
    const double sl_ = xl + x0, s01 = x0 + x1, s3 = sl_ + x1;
    const double P = 2.0 * x0 + x1, Q = x0 + 2.0 * x1, tot = s3 + x2;
    const double d4 = s3 * s01 * sl_;
    const double d5 = s01 * P * Q * tot;
    const double r45 = recip2(d4 * d5);
    const double inv5 = d4 * r45;
    const double dp = A[j + 1] - A[j], dn = A[j] - A[j - 1];
    const double s = x0 * ((2.0 * xl + x0) * sl_ * dp + (x0 + 2.0 * x1) * s01 * dn) * (d5 * r45);
    // (minima of non-negative values by their bit patterns, on the integer pipe: fmin's result,
    // NaN operands included)
    const double adp = fabs(dp), adn = fabs(dn), as = fabs(s);
    const double m2d = 2.0 * (dbits(adp) < dbits(adn) ? adp : adn);
    const double lim = dbits(as) < dbits(m2d) ? as : m2d;
    dm[j] = dp * dn > 0.0 ? copysign(lim, s) : 0.0;
    if (k < 2) dm[k == 0 ? 1 : n + 2] = 0.0;
    // Phase 5's interface j (Eq. h12): f = A_j + [x0 d P Q tot + 2 x0 x1 ((xl + x0) Q - (x2 + x1) P) d
    //   - s01 (x0 (xl + x0) Q dm_{j+1} - x1 (x1 + x2) P dm_j)] / (s01 P Q tot), d = A_{j+1} - A_j
    fb = A[j] + (x0 * dp * P * Q * tot + 2.0 * x0 * x1 * (sl_ * Q - (x2 + x1) * P) * dp) * inv5;
    cR = -(s01 * x0 * sl_ * Q * inv5);
    cL = s01 * x1 * (x1 + x2) * P * inv5;
    flo = fmin(A[j], A[j + 1]);
    fhi = fmax(A[j], A[j + 1]);
  }
  __syncthreads();
  // Phase 5: interface values between extended groups j and j+1, j = 1..n+1 (Eq. h12, the cubic
  // through the group integrals), limited to the range of the two averages (Eqs. h15-h16).  At
  // the two end interfaces the ghost's average equals the group's, so the limiter returns it.
  if (live) {
    if (k < n - 1) {
      const int j = k + 2;
      face[j] = fmin(fmax(fma(cR, dm[j + 1], fma(cL, dm[j], fb)), flo), fhi);
    } else {
      face[1] = A[2];
    }
    if (k == 0) face[n + 1] = A[n + 1];
  }
  __syncthreads();
  // Phase 6: the parabola of each shifted group (Eqs. h17, h22-h24) with the monotonicity
  // corrections (Eqs. h31-h35, Cartesian form).
  if (live) {
    const double a = A[k + 2];
    double l = face[k + 1], r = face[k + 2];
    const double d = r - l, s6 = 6.0 * (a - 0.5 * (l + r));
    const double dd = d * d, ds = d * s6;
    const bool lm = ord_key(dd) < ord_key(ds), rm = ord_key(dd) < ord_key(-ds);   // integer pipe
    const double l2 = lm ? 3.0 * a - 2.0 * r : l;
    const double r2 = rm ? 3.0 * a - 2.0 * l : r;
    aL[k] = l2;
    aR[k] = r2;
    a6[k] = 6.0 * (a - 0.5 * (l2 + r2));
  }
  __syncthreads();
  // Phase 7: the flux across target edge k (Eq. p5): the number in the slice between the shifted
  // and the target edge, from the parabola of the group the slice belongs to; zero at the two
  // outer edges.  Also the target group centres E_k / a^{n+1} (eta2's storage is reused).
  double *ct = eta2;
  if (live) {
    const double ia1 = zc[4];
    ct[k] = Ec[k] * ia1;
    if (k == 0) {
      F[0] = 0.0;
      F[n] = 0.0;
    } else {
      // d < 0: the top of group k-1 moves up into target group k (slice from its right end);
      // d > 0: the bottom of group k moves down into target group k-1 (from its left end).  The
      // slice's fraction of its group is |d| / (Dh - Dl) at infinity (the factor 1/a^{n+1} of
      // both cancels), with 1/(Dh - Dl) from phase 3.
      const double d = g.e_edge[k] - E_d[k];
      const bool up = ord_key(d) < ord_key(-0.0);     // d < 0, on the integer pipe
      const int gsrc = up ? k - 1 : k;
      const double dir = up ? -1.0 : 1.0;
      const double dx = X[gsrc + 2];
      const double yr = fabs(d) * iw[gsrc];
      const double y = dbits(yr) < dbits(1.0) ? yr : 1.0;
      const double end = up ? aR[gsrc] : aL[gsrc];
      const double avg = end + dir * 0.5 * y * ((aR[gsrc] - aL[gsrc]) + dir * (1.0 - 2.0 * kThird * y) * a6[gsrc]);
      F[k] = -dir * avg * y * dx;
    }
  }
  __syncthreads();
  // Phase 8: the sums of xi (Eqs. p6-p8) over the system's groups by a tree over its threads:
  // the energy the shifted groups' numbers lose when they move to the target centres (the energy
  // held by the shifted groups minus the same numbers at the target centres, taken per group), and
  // the flux divergence at the target centres.
  double *r0 = red, *r2 = red + (n + 5);
  double div = 0.0;
  if (live) {
    div = F[k] - F[k + 1];
    r0[k] = nd[k] * (epsd_c[k] - ct[k]);
    r2[k] = div * ct[k];
  }
  int top = 1;
  while (top * 2 < n) top *= 2;
  for (int s = top; s >= 1; s >>= 1) {
    __syncthreads();
    if (live && k < s && k + s < n) {
      r0[k] += r0[k + s];
      r2[k] += r2[k + s];
    }
  }
  __syncthreads();
  // Phase 9: xi (1 without flux), Eq. p6 and psi on the target groups, whose moment is
  // E^2 dE / (a^{n+1})^3; groups below the top two that end above one flag the limiter.
  if (live) {
    const double s2 = r2[0];
    const double xi = !is_zero(s2) ? quot(r0[0], s2) : 1.0;
    const double num = nd[k] + xi * div;
    const double v = num * zc[8] * icmE[k];
    nd[k] = v;
    if (k == 0) zc[6] = xi;
    if (k < n - 2 && ord_key(v) > ord_key(1.0)) zc[7] = 1.0;     // benign race: every writer stores 1
  }
  __syncthreads();
  // Phase 10: the occupation limiter (Eqs. a81a-a81d), sequential over groups k = 0..n-3, only
  // in systems that have an overfilled group.
  if (live && g.limit && k == 0 && zc[7] != 0.0) {
    const double ia1 = zc[4];
    for (int kk = 0; kk < n - 2; ++kk) {
      double d = nd[kk] - 1.0;
      if (!(d > 0.0)) continue;
      const double e0 = ct[kk], e1 = ct[kk + 1], e2 = ct[kk + 2];
      const double w0 = e0 * e0 * (g.e_edge[kk + 1] - g.e_edge[kk]) * ia1;
      const double w1 = e1 * e1 * (g.e_edge[kk + 2] - g.e_edge[kk + 1]) * ia1;
      const double w2 = e2 * e2 * (g.e_edge[kk + 3] - g.e_edge[kk + 2]) * ia1;
      const double c_up = (e2 - e0) * w0 / ((e2 - e1) * w1);
      const double c_dn = (e1 - e0) * w0 / ((e2 - e1) * w2);
      d = fmin(d, fmax(nd[kk + 2], 0.0) / c_dn);   // never take group k + 2 below zero
      nd[kk] -= d;
      nd[kk + 1] += c_up * d;
      nd[kk + 2] -= c_dn * d;
    }
  }
  __syncthreads();
  if (live) {
    g.psi[el] = nd[k];
    if (k == 0 && g.xi) g.xi[sg] = zc[6];
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
  // systems per block: the most that fill whole warps (spb n a multiple of 32; every FP64 warp
  // instruction costs the pipe the same however many of its lanes work), else as many as fit
  g.spb = kEadvThreads / g.n;
  for (int sp = kEadvThreads / g.n; sp >= 1; --sp)
    if ((sp * g.n) % 32 == 0) {
      g.spb = sp;
      break;
    }
  g.limit = prob->limit != 0;
  g.r_n = prob->r_edge_n;
  g.r_np1 = prob->r_edge_np1;
  g.rho_n = prob->rho_n;
  g.rho_np1 = prob->rho_np1;
  g.a_n = prob->lapse_n;
  g.a_np1 = prob->lapse_np1;
  g.e_edge = prob->e_edge;
  g.eta1 = prob->eta1;
  g.u = prob->u;
  g.psi = psi;
  g.xi = xi;
  const size_t n_sys = (size_t)g.n_ray * NS * g.n_r;
  const unsigned grid = (unsigned)((n_sys + g.spb - 1) / g.spb);
  const unsigned threads = (unsigned)((g.spb * g.n + 31) / 32 * 32);
  const size_t smem = eadv_smem(g.spb, g.n);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_energy_advect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MGFLD_ECUDA;
  k_energy_advect<<<grid, threads, smem, (cudaStream_t)stream>>>(g);
  return cudaGetLastError() == cudaSuccess ? MGFLD_OK : MGFLD_ECUDA;
}
