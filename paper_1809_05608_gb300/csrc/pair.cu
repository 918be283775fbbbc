// The synthetic pair process (Eq. d14, zeroth moment, Legendre order 0) in the implicit step.
//
// Each neutrino species q is made and destroyed together with its partner qbar (nu_e with
// nubar_e, nu_mu,tau with nubar_mu,tau), group by group:
//   S_pair,k = C [(1 - psi_k) sum_k' w_k' Phi^p(eps_k, eps_k') (1 - psibar_k')
//                 - psi_k sum_k' w_k' chi_q(k, k') Phi^a(eps_k, eps_k') psibar_k'],
// the annihilation kernel Phi^a = pair_coef per zone, the creation kernel Phi^p =
// e^{-(eps + eps')/T} Phi^a (Eq. d12 with the pair energy eps + eps' given to the e-e+ pair), and
// chi the angular correction of the annihilation kernel (Eqs. d16-d22; 1 unless enabled).  The
// process couples the two species of a pair in every zone, so the Newton system is solved per
// (ray, pair) with coupled 2 n x 2 n zone blocks: rows and columns (s n + k), s = 0 for the
// neutrino and 1 for the antineutrino of the pair; the couplings to the neighbouring zones stay
// diagonal.  Vectors of that system are laid out [ray][pair][zone][2 n].
#include "mgfld_internal.cuh"

namespace mgfld {

// Shared memory of k_pair per zone: e^{-eps/T} and eps^2 d eps of each group, and the flux
// factor and cone edge (Eqs. d17, d22) of every species and group.
__host__ __device__ inline size_t pair_zone_doubles(int n) { return (size_t)(2 + 3 * NS) * n; }
static inline int pair_zones_per_block(int n) {
  const int z = 256 / (NS * n);
  return z < 1 ? 1 : z;
}

// One thread per (zone, species q, group k): row k of species q's weighted annihilation kernel
//   pkill[q][k][k'] = C w_k' chi_q(k, k') Phi^a,
// and (q = 0) row k of the weighted creation kernel, shared by the species,
//   pmake[k][k'] = C w_k' Phi^p(eps_k, eps_k') = C w_k' Phi^a e^{-eps_k/T} e^{-eps_k'/T},
// with its row sum.  chi = min(chi_1, chi_2) (Eq. d21): chi_1 = 1 - eta eta' / 6 (Eq. d16, the
// flux factors eta of species q at eps_k and of its partner at eps_k', the input eta1 clamped to
// [0, 1]), chi_2 = (8 + (mu mu' - 3)(1 + mu)(1 + mu')) / 8 (Eq. d19) with the cone edges
// mu = max(sign(x) sqrt|x|, -1), x = 1 - (R_nu / R_i)^2 (Eqs. d17, d22), R_nu each species' and
// group's neutrinosphere at psi^n and R_i the zone centre.
__global__ void k_pair(Prob p, Ws w, const double *__restrict__ T, int zpb) {
  extern __shared__ double sm[];
  const int n = p.n, per = NS * n;
  const int zl = threadIdx.x / per, rem = threadIdx.x % per, q = rem / n, k = rem % n;
  const unsigned nz = (unsigned)(p.n_ray * p.n_r);
  const unsigned zi = blockIdx.x * (unsigned)zpb + zl;
  const bool live = zl < zpb && zi < nz;
  double *ez = sm + (size_t)(live ? zl : 0) * pair_zone_doubles(n);
  double *wl = ez + n, *eta = wl + n, *mu = eta + NS * n, *mu1 = mu + NS * n;
  int ray = 0, i = 0;
  if (live) {
    ray = (int)(zi / (unsigned)p.n_r);
    i = (int)(zi - (unsigned)ray * p.n_r);
    const double inv_a = 1.0 / lapse_at(p, ray, i);
    if (q == 0) {
      ez[k] = exp(-(w.E[k] * inv_a) / T[zi]);
      wl[k] = kCNes * p.pair[zi] * (w.W[k] * inv_a * inv_a * inv_a);
    }
    const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;
    eta[q * n + k] = p.eta1 ? fmin(fmax(p.eta1[g], 0.0), 1.0) : 0.0;
    const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
    const double rc = 0.5 * (re[i] + re[i + 1]);
    const double rr = w.rnu[((size_t)ray * NS + q) * n + k] / rc;
    const double x = 1.0 - rr * rr;
    const double m = fmax(x > 0.0 ? sqrt(x) : (x < 0.0 ? -sqrt(-x) : 0.0), -1.0);
    mu[q * n + k] = m;
    mu1[q * n + k] = 1.0 + m;
  }
  __syncthreads();
  if (!live) return;
  const int qb = q ^ 1;
  double *kill = w.pkill + (((size_t)zi * NS + q) * n + k) * n;
  if (p.pair_chi) {
    // the factors of this row taken out of the loop: chi_1 = 1 - (eta / 6) eta', and
    // chi_2 = 1 + (mu mu' - 3) ((1 + mu) / 8) (1 + mu') (the 1/8 exact)
    const double e6 = eta[q * n + k] / 6.0, mt = mu[q * n + k], m8 = 0.125 * mu1[q * n + k];
    for (int kp = 0; kp < n; ++kp) {
      const double c1 = fma(-e6, eta[qb * n + kp], 1.0);
      const double c2 = fma(fma(mt, mu[qb * n + kp], -3.0) * m8, mu1[qb * n + kp], 1.0);
      kill[kp] = wl[kp] * fmin(c1, c2);
    }
  } else {
    for (int kp = 0; kp < n; ++kp) kill[kp] = wl[kp];
  }
  if (q == 0) {
    double *make = w.pmake + ((size_t)zi * n + k) * n;
    const double ek = ez[k];
    double ms = 0.0;
    for (int kp = 0; kp < n; ++kp) {
      const double v = wl[kp] * (ek * ez[kp]);
      make[kp] = v;
      ms += v;
    }
    w.pmsum[(size_t)zi * n + k] = ms;
  }
}

cudaError_t launch_pair(const Prob &p, const Ws &w, const double *T, cudaStream_t s) {
  const int zpb = pair_zones_per_block(p.n);
  const size_t nz = (size_t)p.n_ray * p.n_r;
  const size_t sm = sizeof(double) * zpb * pair_zone_doubles(p.n);
  k_pair<<<(unsigned)((nz + zpb - 1) / zpb), zpb * NS * p.n, sm, s>>>(p, w, T, zpb);
  return cudaGetLastError();
}

// Residual and Jacobian rows of the coupled pair systems (Eqs. a58, a59 with the sources of
// Eqs. a55, d8 and d14), one thread per (ray, species q, zone i, group k) equation, as k_assemble
// with the frozen flux coefficients, plus the pair sums
//   make = sum_k' pmake[k][k'] (1 - psibar_k') = pmsum_k - sum pmake psibar,  kill = sum pkill psibar,
// S += (1 - psi_k) make - psi_k kill.  Row (s n + k) of the zone's 2 n x 2 n block: the species'
// own NES block with the diagonal, and the partner's columns
//   dG_k / d psibar_k' = (1 - psi_k) pmake[k][k'] + psi_k pkill[k][k'].
// src_out: the converged sources (psi layout) for Eq. a62b and the ledgers.
template <typename TD>
__global__ void k_assemble_pair(Prob p, Ws w, const double *__restrict__ psi, TD *__restrict__ diag,
                                double *__restrict__ lower, double *__restrict__ upper, double *__restrict__ rhs,
                                const int *__restrict__ list, int n_list, const int *__restrict__ jac_flag,
                                double *__restrict__ src_out, int first, const int *__restrict__ n_dev) {
  const int n = p.n, n2 = 2 * n;
  const unsigned per_ray = (unsigned)(NS * p.n_r * n);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)listed(n_list, n_dev) * per_ray) return;
  const unsigned rl = t / per_ray;
  const int ray = list ? list[rl] : (int)rl;
  const unsigned local = t - rl * per_ray;
  const unsigned kq = local / (unsigned)n;
  const int k = (int)(local - kq * n);
  const int q = (int)(kq % NS);
  const int i = (int)(kq / NS);
  const int pq = q >> 1, sq = q & 1, qb = q ^ 1;
  const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;
  const size_t gc = (((size_t)ray * 2 + pq) * p.n_r + i) * n2 + (size_t)sq * n + k;
  const size_t zi = (size_t)ray * p.n_r + i;
  const int last = p.n_r - 1;
  const double *z = w.zone + zi * ZC_N;
  const double pre = z[ZC_PRE];
  const double inv_acdt = z[ZC_INV_ACDT];

  const double *ps = psi + (g - k);
  const double *pb = psi + (((size_t)ray * NS + qb) * p.n_r + i) * n;
  const double pk = ps[k];
  const double *fin = w.phin + (zi * n + k) * n;
  const double *fout = w.phout + (zi * n + k) * n;
  double gain = 0.0, lp = 0.0;
  if (first) {
    gain = w.g0[g];
    lp = w.l0[g];
  } else {
    for (int kp = 0; kp < n; ++kp) {
      const double pv = ps[kp];
      gain += fin[kp] * pv;
      lp += fout[kp] * pv;
    }
  }
  const double *mk = w.pmake + (zi * n + k) * n;
  const double *kl = w.pkill + ((zi * NS + q) * n + k) * n;
  double mb = 0.0, kb = 0.0;
  for (int kp = 0; kp < n; ++kp) {
    const double v = pb[kp];
    mb = fma(mk[kp], v, mb);
    kb = fma(kl[kp], v, kb);
  }
  const double make = w.pmsum[zi * n + k] - mb, kill = kb;
  const double loss = w.rsum[zi * n + k] - lp;
  const double kap = scaled(p, p.kabs, g, q, k);
  const double j = w.jbuf[g];
  const double S = j * (1.0 - pk) - kap * pk + ((1.0 - pk) * gain - pk * loss) + ((1.0 - pk) * make - pk * kill);
  if (src_out) {
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
  const double sh = p.u ? w.shock[g] : 0.0;
  const double G = (pk - w.psi_n[g]) * inv_acdt + pre * (flux_out - flux_in + sh) - S;
  rhs[gc] = -G;
  if (jac_flag && !jac_flag[ray]) return;
  const double jdiag = al_out * (1.0 - gh) + al_in;
  const double dg = inv_acdt + pre * jdiag + j + kap + (gain + loss) + (make + kill);
  TD *row = diag + gc * n2;
  const int own = sq * n, part = (1 - sq) * n;
  if (sizeof(TD) == 4 && w.phin32) {
    // FP32 rows (the preconditioner of the FP64 refinement): operands converted on the integer
    // pipe (truncated), the partner's columns from FP32 copies of the pair kernels
    const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
    const float pf = d2f_exp2(pk, 0);
    const float dgf = (float)dg;
    for (int kp = 0; kp < n; ++kp) {
      const float e = fmaf(pf, fd[kp], -fi[kp]);
      row[own + kp] = TD(kp == k ? e + dgf : e);
    }
    for (int kp = 0; kp < n; ++kp) {
      const float m = d2f_exp2(mk[kp], 0);
      row[part + kp] = TD(fmaf(pf, d2f_exp2(kl[kp], 0) - m, m));
    }
  } else {
    const double *fd = w.phd + (zi * n + k) * n;
    for (int kp = 0; kp < n; ++kp) {
      const double e = fma(pk, fd[kp], -fin[kp]);
      row[own + kp] = TD(kp == k ? e + dg : e);
    }
    for (int kp = 0; kp < n; ++kp) row[part + kp] = TD(fma(pk, kl[kp] - mk[kp], mk[kp]));
  }
  const double c_low = pre * al_in, c_up = i < last ? pre * al_out : 0.0;
  lower[gc] = -c_low;
  upper[gc] = -c_up;
  if (w.lower32) {
    w.lower32[gc] = d2f_exp2(-c_low, 0);
    w.upper32[gc] = d2f_exp2(-c_up, 0);
  }
}

cudaError_t launch_assemble_pair(const Prob &p, const Ws &w, const double *psi, void *diag, int diag_fp32,
                                 double *lower, double *upper, double *rhs, const int *list, int n_list,
                                 const int *jac_flag, cudaStream_t s, double *src_out, int first, const int *n_dev) {
  const size_t total = (size_t)n_list * NS * p.n_r * p.n;
  if (total == 0) return cudaSuccess;
  const unsigned B = 256;
  const unsigned grid = (unsigned)((total + B - 1) / B);
  if (diag_fp32)
    k_assemble_pair<float><<<grid, B, 0, s>>>(p, w, psi, (float *)diag, lower, upper, rhs, list, n_list, jac_flag,
                                              src_out, first, n_dev);
  else
    k_assemble_pair<double><<<grid, B, 0, s>>>(p, w, psi, (double *)diag, lower, upper, rhs, list, n_list, jac_flag,
                                               src_out, first, n_dev);
  return cudaGetLastError();
}

}  // namespace mgfld
