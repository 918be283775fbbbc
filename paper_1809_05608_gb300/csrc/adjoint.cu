// Discrete adjoint of one implicit transport step (FP64).
//
// One step maps p = (psi^n, Ye^n, T^n, s) to x = (psi^{n+1}, Ye^{n+1}) through G(x; p) = 0
// (Eqs. a58, a59, a62a with the coefficients frozen at p), then to T^{n+1} (Eq. a62b and the
// EoS) and to the gain-region heating H.  With upstream gradients x_bar, T_bar and a weight on
// H, the implicit-function theorem gives
//     J^T mu = x_bar + T_bar dT/dx + w_H dH/dx,      p_bar = T_bar dT/dp + w_H dH/dp - mu^T dG/dp.
// J^T is block-tridiagonal in radius with per-species transposed blocks and a zone-local Ye
// column and row; it is solved by block Gauss-Seidel on (psi, Ye), each psi half being a
// block-Thomas solve of the transposed per-species system (factor kernel shared with the
// forward step).  dG/dp is taken analytically through every frozen coefficient: NES kernels
// and emissivities (T^n, Ye^n, s), mean free path lambda (psi^n, Ye^n, T^n, s), limited
// diffusion coefficient (Eqs. a20-a26a, branch by branch), neutrinosphere (the tau = 2/3
// scan) and outer ghost (Eq. a62af).
#include <cmath>
#include <cstring>

#include "mgfld_internal.cuh"

namespace mgfld {

struct AdjWs {
  double *j1;     // emissivity at Ye^{n+1}
  double *zadj;   // per zone [8]: mu1, dmu1, muT1, dmun, muTn, muY, bY, dYY
  double *b;      // psi part of the adjoint right-hand side
  double *lamb;   // gradient with respect to lambda^(t)
  double *ktb;    // gradient with respect to 1/lambda^(t)
  double *rbar;   // neutrinosphere gradient per edge
  double *psinb;  // flux-coefficient part of the psi^n gradient
  double *tT;     // per-element contributions to the T^n gradient
  double *sS;     // per-element contributions to the scale gradient
  double *yY;     // per-element contributions to the Ye^n gradient
  double *gbar;   // ghost-factor gradient per (ray, q, k)
  unsigned long long *conv;  // [2] bits of max|d mu_Y| and max|mu_Y| of the current sweep
};
enum { ZA_MU1 = 0, ZA_DMU1, ZA_MUT1, ZA_DMUN, ZA_MUTN, ZA_MUY, ZA_BY, ZA_DYY };

struct AdjLayout {
  Layout fwd;
  size_t j1, zadj, b, lamb, ktb, rbar, psinb, tT, sS, yY, gbar, conv, total;
};

static size_t aup(size_t v) { return (v + 255) & ~(size_t)255; }

static AdjLayout make_adj_layout(int n_ray, int n_r, int n) {
  AdjLayout A;
  A.fwd = make_layout(n_ray, n_r, n, MGFLD_FP64);
  const size_t F = (size_t)n_ray * NS * n_r * n, Z = (size_t)n_ray * n_r;
  size_t off = A.fwd.total;
  auto take = [&](size_t bytes) { size_t o = off; off = aup(off + bytes); return o; };
  A.j1 = take(8 * F);
  A.zadj = take(8 * Z * 8);
  A.b = take(8 * F);
  A.lamb = take(8 * F);
  A.ktb = take(8 * F);
  A.rbar = take(8 * F);
  A.psinb = take(8 * F);
  A.tT = take(8 * F);
  A.sS = take(8 * F);
  A.yY = take(8 * F);
  A.gbar = take(8 * (size_t)n_ray * NS * n);
  A.conv = take(16);
  A.total = off;
  return A;
}

static AdjWs resolve_adj(void *base, const AdjLayout &A) {
  char *b = (char *)base;
  AdjWs a;
  a.j1 = (double *)(b + A.j1);
  a.zadj = (double *)(b + A.zadj);
  a.b = (double *)(b + A.b);
  a.lamb = (double *)(b + A.lamb);
  a.ktb = (double *)(b + A.ktb);
  a.rbar = (double *)(b + A.rbar);
  a.psinb = (double *)(b + A.psinb);
  a.tT = (double *)(b + A.tT);
  a.sS = (double *)(b + A.sS);
  a.yY = (double *)(b + A.yY);
  a.gbar = (double *)(b + A.gbar);
  a.conv = (unsigned long long *)(b + A.conv);
  return a;
}

// Decomposition of a global (ray, q, i, k) element index.
struct Elem {
  int ray, q, i, k;
  size_t g, zi;
};
__device__ inline Elem elem_of(const Prob &p, size_t t) {
  Elem e;
  const int n = p.n;
  e.k = (int)(t % n);
  size_t u = t / n;
  e.i = (int)(u % p.n_r);
  u /= p.n_r;
  e.q = (int)(u % NS);
  e.ray = (int)(u / NS);
  e.g = t;
  e.zi = (size_t)e.ray * p.n_r + e.i;
  return e;
}

// Exponent magnitude of the synthetic NES out-kernel: Phi_out(k, m) ~ e^{-eo(k, m)/T}.
__device__ inline double nes_exponent(double ek, double em, bool down) { return down ? ek - em : 2.0 * (em - ek); }

__device__ inline bool in_gain(const Prob &p, int ray, int i) {
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const double rc = 0.5 * (re[i] + re[i + 1]);
  return rc >= 1.0e7 && rc <= 3.0e7;
}

// Weight of dS_{q,k}/d(.) in the explicit outputs: T^{n+1} (Eq. a62b) and the heating H.
__device__ inline double omega(const Prob &p, const Ws &w, int q, int k, double inv_a, const double *z, double rho,
                               double Tb, double hcoef) {
  const double inv_a3 = inv_a * inv_a * inv_a;
  const double we = w.W[k] * inv_a3 * w.E[k] * inv_a;
  double om = Tb * (-z[ZC_ACDT] * kFourPiHC3 * (p.eos.mb / rho) / p.eos.ec) * stat_weight(q) * we;
  if (q < 2) om += hcoef * we;
  return om;
}

__global__ void k_adj_zone1(Prob p, Ws w, AdjWs a, const double *__restrict__ ye1, const double *__restrict__ Tn) {
  const size_t zi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (zi >= (size_t)p.n_ray * p.n_r) return;
  const int n = p.n;
  const int ray = (int)(zi / p.n_r), i = (int)(zi % p.n_r);
  const double *z = w.zone + zi * ZC_N;
  const double T = Tn[zi];
  double mu1, dmu1, mun, dmun;
  mu_nue_zone(p.eos, z[ZC_MUA], z[ZC_MUB], T, ye1[zi], mu1, dmu1);
  mu_nue_zone(p.eos, z[ZC_MUA], z[ZC_MUB], T, w.ye_n[zi], mun, dmun);
  double *za = a.zadj + zi * 8;
  za[ZA_MU1] = mu1;
  za[ZA_DMU1] = dmu1;
  za[ZA_MUT1] = log(ye1[zi] / (1.0 - ye1[zi])) + p.eos.log_gn_gp;
  za[ZA_DMUN] = dmun;
  za[ZA_MUTN] = log(w.ye_n[zi] / (1.0 - w.ye_n[zi])) + p.eos.log_gn_gp;
  za[ZA_MUY] = 0.0;
  const double inv_a = z[ZC_INV_A];
  for (int q = 0; q < NS; ++q) {
    const size_t g0 = (((size_t)ray * NS + q) * p.n_r + i) * n;
    for (int k = 0; k < n; ++k) {
      const double sc = p.scale ? p.scale[q * n + k] : 1.0;
      bool live;
      a.j1[g0 + k] = emissivity(p.kabs[g0 + k] * sc, species_mu(q, mu1), w.E[k] * inv_a, T, live);
    }
  }
}

// b_psi = psi_bar + sum_k omega_k dS_k/dpsi_k' at x (transposed source Jacobian).
__global__ void k_adj_rhs(Prob p, Ws w, AdjWs a, const double *__restrict__ psi1, const double *__restrict__ psib1,
                          const double *__restrict__ Tb1, double hw) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * NS * p.n_r * p.n) return;
  const Elem e = elem_of(p, t);
  const int n = p.n;
  const double *z = w.zone + e.zi * ZC_N;
  const double inv_a = z[ZC_INV_A];
  const double rho = p.rho[e.zi];
  const double Tb = Tb1 ? Tb1[e.zi] : 0.0;
  const double hcoef = in_gain(p, e.ray, e.i) ? hw * (-z[ZC_ACDT] * z[ZC_VOL] * kFourPiHC3) : 0.0;
  const double *ps = psi1 + (t - e.k);
  const size_t zrow = e.zi * n;
  double acc = 0.0, gain = 0.0, lp = 0.0;
  for (int k = 0; k < n; ++k) {
    const double om = omega(p, w, e.q, k, inv_a, z, rho, Tb, hcoef);
    acc += om * (w.phin[(zrow + k) * n + e.k] - ps[k] * w.phd[(zrow + k) * n + e.k]);
    gain += w.phin[(zrow + e.k) * n + k] * ps[k];
    lp += w.phout[(zrow + e.k) * n + k] * ps[k];
  }
  const double loss = w.rsum[zrow + e.k] - lp;
  const double sc = p.scale ? p.scale[e.q * n + e.k] : 1.0;
  const double kap = p.kabs[t] * sc;
  const double om_k = omega(p, w, e.q, e.k, inv_a, z, rho, Tb, hcoef);
  acc -= om_k * (a.j1[t] + kap + gain + loss);
  a.b[t] = (psib1 ? psib1[t] : 0.0) + acc;
}

// Ye part of the right-hand side and the Ye diagonal of J.
__global__ void k_adj_rhsY(Prob p, Ws w, AdjWs a, const double *__restrict__ psi1, const double *__restrict__ ye1,
                           const double *__restrict__ yeb1, const double *__restrict__ Tb1,
                           const double *__restrict__ Tn, double hw) {
  const size_t zi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (zi >= (size_t)p.n_ray * p.n_r) return;
  const int n = p.n;
  const int ray = (int)(zi / p.n_r), i = (int)(zi % p.n_r);
  const double *z = w.zone + zi * ZC_N;
  double *za = a.zadj + zi * 8;
  const double inv_a = z[ZC_INV_A], inv_a3 = inv_a * inv_a * inv_a;
  const double rho = p.rho[zi], T = Tn[zi];
  const double Tb = Tb1 ? Tb1[zi] : 0.0;
  const double hcoef = in_gain(p, ray, i) ? hw * (-z[ZC_ACDT] * z[ZC_VOL] * kFourPiHC3) : 0.0;
  const double cy = kFourPiHC3 * p.eos.mb / rho;
  const double capT = kExpCap * T;
  double sb = 0.0, sd = 0.0;
  for (int q = 0; q < 2; ++q) {
    const double mq = species_mu(q, za[ZA_MU1]);
    const double djq = lepton_sign(q) * za[ZA_DMU1] / T;          // d ln j / dYe
    const size_t g0 = (((size_t)ray * NS + q) * p.n_r + i) * n;
    for (int k = 0; k < n; ++k) {
      if (mq - w.E[k] * inv_a >= capT) continue;
      const double dS = (1.0 - psi1[g0 + k]) * a.j1[g0 + k] * djq;   // dS_qk/dYe
      sb += omega(p, w, q, k, inv_a, z, rho, Tb, hcoef) * dS;
      sd += lepton_sign(q) * w.W[k] * inv_a3 * dS;
    }
  }
  const double y1 = ye1[zi], yn1 = 1.0 - y1;
  const Eos &E = p.eos;
  const double mu_e = z[ZC_MUA] * (E.g1_is_4_3 ? cbrt(y1) : pow(y1, E.g1 - 1.0));
  const double mu_nn = z[ZC_MUB] * (E.g2_is_5_2 ? yn1 * sqrt(yn1) : pow(yn1, E.g2 - 1.0));
  za[ZA_BY] = (yeb1 ? yeb1[zi] : 0.0) + sb - Tb * (mu_e - mu_nn) / E.ec;     // d e_cold/dYe = mu_e - mu_nn
  za[ZA_DYY] = z[ZC_INV_ACDT] + cy * sd;
}

// Transposed diagonal blocks (row k of D^T = column k of D) and couplings of J_psi^T.
__global__ void k_adj_assembleT(Prob p, Ws w, AdjWs a, const double *__restrict__ psi1) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * NS * p.n_r * p.n) return;
  const Elem e = elem_of(p, t);
  const int n = p.n, last = p.n_r - 1;
  const double *z = w.zone + e.zi * ZC_N;
  const double *ps = psi1 + (t - e.k);
  const size_t zrow = e.zi * n;
  double gain = 0.0, lp = 0.0;
  for (int k = 0; k < n; ++k) {
    gain += w.phin[(zrow + e.k) * n + k] * ps[k];
    lp += w.phout[(zrow + e.k) * n + k] * ps[k];
  }
  const double loss = w.rsum[zrow + e.k] - lp;
  const double sc = p.scale ? p.scale[e.q * n + e.k] : 1.0;
  const double kap = p.kabs[t] * sc;
  const double al_out = w.alpha[t];
  const double al_in = e.i > 0 ? w.alpha[t - n] : 0.0;
  const double gh = (e.i == last) ? w.ghost[((size_t)e.ray * NS + e.q) * n + e.k] : 0.0;
  const double pre = z[ZC_PRE];
  const double dg = z[ZC_INV_ACDT] + pre * (al_out * (1.0 - gh) + al_in) + a.j1[t] + kap + gain + loss;
  double *row = w.diag + t * n;
  for (int kp = 0; kp < n; ++kp)                       // D[kp][k] = -(phin - psi_kp phd)[kp][k]
    row[kp] = -(w.phin[(zrow + kp) * n + e.k] - ps[kp] * w.phd[(zrow + kp) * n + e.k]);
  row[e.k] += dg;
  // J^T couples zone i to i-1 through upper_{i-1} and to i+1 through lower_{i+1}.
  w.lower[t] = e.i > 0 ? -w.zone[(e.zi - 1) * ZC_N + ZC_PRE] * w.alpha[t - n] : 0.0;
  w.upper[t] = e.i < last ? -w.zone[(e.zi + 1) * ZC_N + ZC_PRE] * al_out : 0.0;
}

// rhs_psi = b_psi - (dG_Y/dpsi)^T mu_Y.
__global__ void k_adj_mix(Prob p, Ws w, AdjWs a) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * NS * p.n_r * p.n) return;
  const Elem e = elem_of(p, t);
  double r = a.b[t];
  if (e.q < 2) {
    const double *z = w.zone + e.zi * ZC_N;
    const double inv_a = z[ZC_INV_A];
    const double cy = kFourPiHC3 * p.eos.mb / p.rho[e.zi];
    const double sc = p.scale ? p.scale[e.q * p.n + e.k] : 1.0;
    const double kap = p.kabs[t] * sc;
    const double wk = w.W[e.k] * inv_a * inv_a * inv_a;
    r += cy * lepton_sign(e.q) * wk * (a.j1[t] + kap) * a.zadj[e.zi * 8 + ZA_MUY];
  }
  w.rhs[t] = r;
}

// mu_Y = (b_Y - (dG_psi/dYe)^T mu_psi) / (dG_Y/dYe), one zone per thread.
__global__ void k_adj_muY(Prob p, Ws w, AdjWs a, const double *__restrict__ psi1, const double *__restrict__ Tn) {
  const size_t zi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (zi >= (size_t)p.n_ray * p.n_r) return;
  const int n = p.n;
  const int ray = (int)(zi / p.n_r), i = (int)(zi % p.n_r);
  double *za = a.zadj + zi * 8;
  const double inv_a = w.zone[zi * ZC_N + ZC_INV_A];
  const double T = Tn[zi], capT = kExpCap * T;
  double s = 0.0;
  for (int q = 0; q < 2; ++q) {
    const double mq = species_mu(q, za[ZA_MU1]);
    const double djq = lepton_sign(q) * za[ZA_DMU1] / T;
    const size_t g0 = (((size_t)ray * NS + q) * p.n_r + i) * n;
    for (int k = 0; k < n; ++k) {
      if (mq - w.E[k] * inv_a >= capT) continue;
      s += -(1.0 - psi1[g0 + k]) * a.j1[g0 + k] * djq * w.x[g0 + k];   // dG_psi/dYe = -dS/dYe
    }
  }
  const double mu = (za[ZA_BY] - s) / za[ZA_DYY];
  atomicMax(a.conv, dbits(fabs(mu - za[ZA_MUY])));
  atomicMax(a.conv + 1, dbits(fabs(mu)));
  za[ZA_MUY] = mu;
}

// Gradient ab = dQ/d alpha_{i+1/2} carried back to the left/right psi^n and lambda and to the
// neutrinosphere radius through the limited coefficient (Eqs. a20-a26a with readings R3, R7;
// same branches as the forward edge kernel).  With psi_e = (pl + pr)/2, dpsi = pr - pl,
// s = sign(dpsi), c = lambda_e / (3 dR) and alpha = K lambda_e F (K = A / (3 dR a^2)):
//   F = psi_e / (psi_e + c|dpsi|):  d alpha/d pl =  K lambda_e c s pr / D^2,
//                                   d alpha/d pr = -K lambda_e c s pl / D^2   (D = psi_e + c|dpsi|),
//                                   d alpha/d lambda_e = K F^2;
//   F = h psi_e / (c|dpsi|):        d alpha/d pl =  (K h / i3) s pr / dpsi^2,
//                                   d alpha/d pr = -(K h / i3) s pl / dpsi^2,
//                                   d alpha/d h = (K / i3) psi_e / |dpsi|,  d alpha/d lambda_e = 0.
// These closed forms avoid the cancellation of the chain through psi_e and |dpsi| (two terms
// larger than their sum by pl/pr where pr << pl).  The limiter is invariant under psi -> c psi,
// so where psi^n is tiny the partials are huge (~ alpha / psi): the upstream factor ab is
// applied first and the small denominators divide last.
struct EdgeGrad {
  double dpl, dpr, dll, dlr, drnu;
};
__device__ inline EdgeGrad edge_grad(double ab, double pl, double pr, double ll, double lr, double i3, double geo,
                                    double r_e2inv, bool outside, double rnu) {
  EdgeGrad d = {0, 0, 0, 0, 0};
  const double le = sqrt(ll * lr);
  const double pe = 0.5 * (pl + pr), dp = pr - pl;
  const double K = i3 * geo;
  if (pe <= 1e-300 || ab == 0.0) return d;         // F = 0, or nothing to carry
  if (dp == 0.0) {                                  // F = 1: alpha = lambda_e K
    const double g = ab * K * le;
    d.dll = g / (2.0 * ll);
    d.dlr = g / (2.0 * lr);
    return d;
  }
  const double adp = fabs(dp), s = dp > 0.0 ? 1.0 : -1.0;
  const double c = le * i3;
  const double x = c * adp;
  double h = 1.0, sq = 0.0;
  bool geom = false;
  if (outside) {
    sq = sqrt(fmax(1.0 - rnu * rnu * r_e2inv, 0.0));
    h = 0.5 * (1.0 + sq);
    geom = h * pe < (1.0 - h) * x;
  }
  double g_le = 0.0;
  if (geom) {
    const double g = ab * geo * h;
    d.dpl = s * ((g * (pr / adp)) / adp);
    d.dpr = -s * ((g * (pl / adp)) / adp);
    if (sq > 0.0) d.drnu = (ab * geo * (pe / adp)) * (0.5 * (-rnu * r_e2inv) / sq);
  } else {
    const double D = pe + x;
    const double F = pe / D;
    const double g = ab * K * le * c;
    d.dpl = s * ((g * (pr / D)) / D);
    d.dpr = -s * ((g * (pl / D)) / D);
    g_le = ab * K * F * F;
  }
  d.dll = g_le * le / (2.0 * ll);
  d.dlr = g_le * le / (2.0 * lr);
  return d;
}

// Flux-coefficient adjoint: alpha_bar of the two edges of zone i from mu_psi (in w.x), then
// their partials into lambda_bar_i and the psi^n gradient of zone i; the neutrinosphere and
// ghost parts are collected for k_adj_rnu.
__global__ void k_adj_flux(Prob p, Ws w, AdjWs a, const double *__restrict__ psi1) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * NS * p.n_r * p.n) return;
  const Elem e = elem_of(p, t);
  const int n = p.n, last = p.n_r - 1;
  const double *re = p.r_edge + (size_t)e.ray * (p.n_r + 1);
  const int gq = (e.ray * NS + e.q) * n + e.k;
  const double rnu = w.rnu[gq];
  const double pre_i = w.zone[e.zi * ZC_N + ZC_PRE];
  const double mu_i = w.x[t];
  double lb = 0.0, pb = 0.0, rb = 0.0;
  // outer edge i+1/2 (zone i on its left)
  if (!(e.i == last && p.bc == MGFLD_BC_REFLECT)) {
    const double *z = w.zone + e.zi * ZC_N;
    const double pl = w.psi_n[t], ll = w.lam[t];
    double pr, lr, ab;
    const double gh = (e.i == last) ? w.ghost[gq] : 0.0;
    if (e.i < last) {
      pr = w.psi_n[t + n];
      lr = w.lam[t + n];
      const double pre_r = w.zone[(e.zi + 1) * ZC_N + ZC_PRE];
      ab = (mu_i * pre_i - w.x[t + n] * pre_r) * (psi1[t + n] - psi1[t]);
    } else {
      pr = gh * pl;
      lr = ll;
      ab = mu_i * pre_i * (gh - 1.0) * psi1[t];
    }
    const EdgeGrad d = edge_grad(ab, pl, pr, ll, lr, z[ZC_EI3DR], z[ZC_EGEO], z[ZC_EIR2], re[e.i + 1] > rnu, rnu);
    if (e.i < last) {
      lb += d.dll;
      pb += d.dpl;
    } else {
      lb += d.dll + d.dlr;                              // lambda_{I+1} = lambda_I
      pb += d.dpl + gh * d.dpr;                         // psi_{I+1} = g psi_I
      // ghost factor: through G (flux to the ghost) and through alpha's psi_r = g psi_I
      a.gbar[gq] = mu_i * pre_i * w.alpha[t] * psi1[t] + d.dpr * pl;
    }
    rb = d.drnu;
  }
  // inner edge i-1/2 (zone i on its right)
  if (e.i > 0) {
    const size_t tl = t - n;
    const double *z = w.zone + (e.zi - 1) * ZC_N;
    const double pl = w.psi_n[tl], ll = w.lam[tl];
    const double pr = w.psi_n[t], lr = w.lam[t];
    const double ab = (w.x[tl] * z[ZC_PRE] - mu_i * pre_i) * (psi1[t] - psi1[tl]);
    const EdgeGrad d = edge_grad(ab, pl, pr, ll, lr, z[ZC_EI3DR], z[ZC_EGEO], z[ZC_EIR2], re[e.i] > rnu, rnu);
    lb += d.dlr;
    pb += d.dpr;
  }
  a.lamb[t] = lb;
  a.psinb[t] = pb;
  a.rbar[t] = rb;
}

// Neutrinosphere adjoint per (ray, q, k): collect dJ/dR_nu from the geometric-limiter edges
// and the ghost factor, then distribute it over the lambda of the zones its tau scan used.
__global__ void k_adj_rnu(Prob p, Ws w, AdjWs a) {
  const int n = p.n;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n_ray * NS * n) return;
  const int k = t % n, q = (t / n) % NS, ray = t / (n * NS);
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const size_t off = ((size_t)ray * NS + q) * p.n_r * n + k;
  double R = 0.0;
  for (int i = 0; i < p.n_r; ++i) R += a.rbar[off + (size_t)i * n];
  if (p.bc == MGFLD_BC_GHOST) {
    const double rI = 0.5 * (re[p.n_r - 1] + re[p.n_r]);
    const double rg = 2.0 * re[p.n_r] - rI;
    const double rnu = w.rnu[t];
    if (rnu < rI) {
      const double den = rg * rg - 0.25 * rnu * rnu;
      R += a.gbar[t] * (0.5 * rnu) * (rI * rI - rg * rg) / (den * den);
    }
  }
  if (R == 0.0) return;
  double tau_out = 0.0;
  for (int i = p.n_r - 1; i >= 0; --i) {
    const double dtau = (re[i + 1] - re[i]) * w.kinv[off + (size_t)i * n];
    if (tau_out + dtau >= kTauNu) {
      const double li = w.lam[off + (size_t)i * n];
      a.lamb[off + (size_t)i * n] += R * (-(kTauNu - tau_out));
      for (int j = i + 1; j < p.n_r; ++j) {
        const double kj = w.kinv[off + (size_t)j * n];
        a.lamb[off + (size_t)j * n] += R * li * (-(re[j + 1] - re[j]) * kj * kj);
      }
      return;
    }
    tau_out += dtau;
  }
}

// Parameter gradients per element (ray, q, i, k): psi^n (time term, flux coefficients, mean
// free path through the NES sums), and the contributions to the scale, T^n and Ye^n gradients.
__global__ void k_adj_params(Prob p, Ws w, AdjWs a, const double *__restrict__ psi1, const double *__restrict__ Tn,
                             const double *__restrict__ Tb1, double hw, double *__restrict__ psib_out) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * NS * p.n_r * p.n) return;
  const Elem e = elem_of(p, t);
  const int n = p.n;
  const double *z = w.zone + e.zi * ZC_N;
  const double *za = a.zadj + e.zi * 8;
  const double inv_a = z[ZC_INV_A], inv_a3 = inv_a * inv_a * inv_a;
  const double T = Tn[e.zi], T2 = T * T, capT = kExpCap * T;
  const size_t zrow = e.zi * n;
  const size_t r0 = t - e.k;                        // (ray, q, i, 0)
  // kappa_t gradient of this zone-species row (the mean free path is 1/kappa_t)
  const double lam = w.lam[t];
  const double ktb_self = -lam * lam * a.lamb[t];
  // psi^n gradient: time term + flux coefficients + sum_k ktb_k d kappa_t,k / d psi^n_k' (= phd[k][k'])
  double pn = w.x[t] * z[ZC_INV_ACDT] + a.psinb[t];
  for (int k = 0; k < n; ++k) {
    const double lk = w.lam[r0 + k];
    pn += (-lk * lk * a.lamb[r0 + k]) * w.phd[(zrow + k) * n + e.k];
  }
  psib_out[t] = pn;
  // weights of dS/dp: theta (source in G_psi and in the outputs), theta_ae (abs/em in G_Y)
  const double rho = p.rho[e.zi];
  const double Tb = Tb1 ? Tb1[e.zi] : 0.0;
  const double hcoef = in_gain(p, e.ray, e.i) ? hw * (-z[ZC_ACDT] * z[ZC_VOL] * kFourPiHC3) : 0.0;
  const double theta = w.x[t] + omega(p, w, e.q, e.k, inv_a, z, rho, Tb, hcoef);
  const double wk = w.W[e.k] * inv_a3;
  const double cy = kFourPiHC3 * p.eos.mb / rho;
  const double theta_ae = -za[ZA_MUY] * cy * lepton_sign(e.q) * wk;
  const double eps = w.E[e.k] * inv_a;
  const double kin = p.kabs[t], ksin = p.kscat[t];
  const double pk = psi1[t];
  // at x: emissivity j1 = kappa e^{x1}, x1 = (mu_q(Ye1, T) - eps)/T
  const double m1 = species_mu(e.q, za[ZA_MU1]);
  const bool live1 = m1 - eps < capT;
  const double ex1 = live1 ? exp((m1 - eps) / T) : exp(kExpCap);
  const double dSae_ds = (ex1 * (1.0 - pk) - pk) * kin;                 // d S_ae / d s
  const double muT1 = e.q == 0 ? za[ZA_MUT1] : (e.q == 1 ? -za[ZA_MUT1] : 0.0);
  const double dx1dT = live1 ? muT1 / T - (m1 - eps) / T2 : 0.0;
  const double dSae_dT = (1.0 - pk) * a.j1[t] * dx1dT;
  // at psi^n: emissivity j_n and the NES rates of the mean free path
  const double mn = species_mu(e.q, z[ZC_MU]);
  const bool liven = mn - eps < capT;
  const double exn = liven ? exp((mn - eps) / T) : exp(kExpCap);
  const double muTn = e.q == 0 ? za[ZA_MUTN] : (e.q == 1 ? -za[ZA_MUTN] : 0.0);
  const double dxndT = liven ? muTn / T - (mn - eps) / T2 : 0.0;
  const double dkt_ds = kin * (1.0 + exn) + ksin;
  double dkt_dT = w.jbuf[t] * dxndT;
  // T-derivatives of the NES kernels: d phout[k][m]/dT = phout eo(k,m)/T^2, d phin[k][m]/dT = phin eo(m,k)/T^2
  double g1 = 0.0, l1 = 0.0;
  const double *ps1 = psi1 + r0;
  const double *psn = w.psi_n + r0;
  for (int m = 0; m < n; ++m) {
    const double em = w.E[m] * inv_a;
    const double eo_km = nes_exponent(eps, em, m <= e.k);
    const double eo_mk = nes_exponent(em, eps, e.k <= m);
    const double fin = w.phin[(zrow + e.k) * n + m] * eo_mk;
    const double fout = w.phout[(zrow + e.k) * n + m] * eo_km;
    g1 += fin * ps1[m];
    l1 += fout * (1.0 - ps1[m]);
    dkt_dT += (fin * psn[m] + fout * (1.0 - psn[m])) / T2;
  }
  const double dSnes_dT = ((1.0 - pk) * g1 - pk * l1) / T2;
  a.sS[t] = (theta + theta_ae) * dSae_ds + ktb_self * dkt_ds;
  a.tT[t] = theta * (dSae_dT + dSnes_dT) + theta_ae * dSae_dT + ktb_self * dkt_dT;
  a.yY[t] = (e.q < 2 && liven) ? ktb_self * w.jbuf[t] * lepton_sign(e.q) * za[ZA_DMUN] / T : 0.0;
}

// Per zone: T^n and Ye^n gradients.
__global__ void k_adj_zoneout(Prob p, Ws w, AdjWs a, const double *__restrict__ Tb1, double *__restrict__ Tb_out,
                              double *__restrict__ yeb_out) {
  const size_t zi = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (zi >= (size_t)p.n_ray * p.n_r) return;
  const int n = p.n;
  const int ray = (int)(zi / p.n_r), i = (int)(zi % p.n_r);
  const double *z = w.zone + zi * ZC_N;
  const double *za = a.zadj + zi * 8;
  double tt = 0.0, yy = 0.0;
  for (int q = 0; q < NS; ++q) {
    const size_t g0 = (((size_t)ray * NS + q) * p.n_r + i) * n;
    for (int k = 0; k < n; ++k) {
      tt += a.tT[g0 + k];
      yy += a.yY[g0 + k];
    }
  }
  const double Tb = Tb1 ? Tb1[zi] : 0.0;
  const double yn = w.ye_n[zi], ynn = 1.0 - yn;
  const Eos &E = p.eos;
  const double mu_e = z[ZC_MUA] * (E.g1_is_4_3 ? cbrt(yn) : pow(yn, E.g1 - 1.0));
  const double mu_nn = z[ZC_MUB] * (E.g2_is_5_2 ? ynn * sqrt(ynn) : pow(ynn, E.g2 - 1.0));
  Tb_out[zi] = Tb + tt;
  yeb_out[zi] = za[ZA_MUY] * z[ZC_INV_ACDT] + yy + Tb * (mu_e - mu_nn) / E.ec;
}

// scale_bar[q][k] += sum over rays and zones (one block per (q, k), fixed-order reduction).
__global__ void k_adj_scale(Prob p, AdjWs a, double *__restrict__ scale_bar) {
  __shared__ double red[256];
  const int n = p.n;
  const int qk = blockIdx.x, q = qk / n, k = qk % n;
  double acc = 0.0;
  const size_t cnt = (size_t)p.n_ray * p.n_r;
  for (size_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int ray = (int)(e / p.n_r), i = (int)(e % p.n_r);
    acc += a.sS[(((size_t)ray * NS + q) * p.n_r + i) * n + k];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) scale_bar[qk] += red[0];
}

static inline unsigned nb(size_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

#define ADJ_CUDA(x)                              \
  do {                                           \
    if ((x) != cudaSuccess) return MGFLD_ECUDA;  \
  } while (0)

static mgfld_status adjoint_step(const Prob &p, const mgfld_state *s0, const mgfld_state *s1, mgfld_adjoint_io *io,
                                 void *ws, cudaStream_t s) {
  const AdjLayout A = make_adj_layout(p.n_ray, p.n_r, p.n);
  const Ws w = resolve(ws, A.fwd);
  const AdjWs a = resolve_adj(ws, A);
  const size_t F = (size_t)p.n_ray * NS * p.n_r * p.n, Z = (size_t)p.n_ray * p.n_r;
  const unsigned B = 256;
  const double hw = io->heat_weight;
  ADJ_CUDA(launch_setup(p, w, s0->psi, s0->ye, s0->T, s));
  k_adj_zone1<<<nb(Z, 128), 128, 0, s>>>(p, w, a, s1->ye, s0->T);
  k_adj_rhs<<<nb(F, B), B, 0, s>>>(p, w, a, s1->psi, io->psi_bar, io->T_bar, hw);
  k_adj_rhsY<<<nb(Z, 128), 128, 0, s>>>(p, w, a, s1->psi, s1->ye, io->ye_bar, io->T_bar, s0->T, hw);
  k_adj_assembleT<<<nb(F, B), B, 0, s>>>(p, w, a, s1->psi);
  ADJ_CUDA(cudaGetLastError());
  ADJ_CUDA(launch_factor(p.n, p.n_r, p.n_ray * NS, w.diag, 0, w.lower, w.upper, w.dinv, MGFLD_FP64, nullptr, s));
  const int max_sweeps = io->max_sweeps > 0 ? io->max_sweeps : 30;
  const double tol = io->sweep_tol > 0.0 ? io->sweep_tol : 1e-15;
  mgfld_status st = MGFLD_ENOCONV;
  io->sweeps_used = 0;
  io->sweep_change = 0.0;
  for (int it = 0; it < max_sweeps; ++it) {
    k_adj_mix<<<nb(F, B), B, 0, s>>>(p, w, a);
    ADJ_CUDA(cudaGetLastError());
    ADJ_CUDA(launch_solve(p.n, p.n_r, p.n_ray * NS, w.dinv, w.lower, w.upper, w.rhs, w.x, MGFLD_FP64, nullptr, s));
    ADJ_CUDA(cudaMemsetAsync(a.conv, 0, 16, s));
    k_adj_muY<<<nb(Z, 128), 128, 0, s>>>(p, w, a, s1->psi, s0->T);
    ADJ_CUDA(cudaGetLastError());
    unsigned long long cv[2];
    ADJ_CUDA(cudaMemcpyAsync(cv, a.conv, sizeof(cv), cudaMemcpyDeviceToHost, s));
    ADJ_CUDA(cudaStreamSynchronize(s));
    double d, m;
    memcpy(&d, &cv[0], 8);
    memcpy(&m, &cv[1], 8);
    io->sweeps_used = it + 1;
    if (!std::isfinite(d) || !std::isfinite(m)) {
      io->sweep_change = NAN;
      st = MGFLD_ENAN;
      break;
    }
    io->sweep_change = m > 0.0 ? d / m : (d > 0.0 ? INFINITY : 0.0);
    // The first sweep starts from mu_Y = 0, so its change is the whole value.
    if (it > 0 && io->sweep_change <= tol) {
      st = MGFLD_OK;
      break;
    }
    if (it == 0 && m == 0.0) {           // no lepton coupling: mu_psi is already exact
      st = MGFLD_OK;
      break;
    }
  }
  // With the last sweep's mu_Y the psi half is one sweep behind; one more psi solve makes the
  // pair consistent with the mu_Y used in the parameter gradients.
  k_adj_mix<<<nb(F, B), B, 0, s>>>(p, w, a);
  ADJ_CUDA(cudaGetLastError());
  ADJ_CUDA(launch_solve(p.n, p.n_r, p.n_ray * NS, w.dinv, w.lower, w.upper, w.rhs, w.x, MGFLD_FP64, nullptr, s));
  k_adj_flux<<<nb(F, B), B, 0, s>>>(p, w, a, s1->psi);
  k_adj_rnu<<<nb((size_t)p.n_ray * NS * p.n, 128), 128, 0, s>>>(p, w, a);
  k_adj_params<<<nb(F, B), B, 0, s>>>(p, w, a, s1->psi, s0->T, io->T_bar, hw, io->psi_bar_out);
  k_adj_zoneout<<<nb(Z, 128), 128, 0, s>>>(p, w, a, io->T_bar, io->T_bar_out, io->ye_bar_out);
  if (io->scale_bar) k_adj_scale<<<NS * p.n, 256, 0, s>>>(p, a, io->scale_bar);
  ADJ_CUDA(cudaGetLastError());
  return st;
}

}  // namespace mgfld

using namespace mgfld;

extern "C" {

size_t mgfld_adjoint_workspace_bytes(const mgfld_dims *dims) {
  if (!dims_ok(dims)) return 0;
  return make_adj_layout(dims->n_ray, dims->n_r, dims->n_e).total;
}

mgfld_status mgfld_adjoint(const mgfld_dims *dims, const mgfld_problem *prob, const mgfld_state *state_n,
                           const mgfld_state *state_np1, mgfld_adjoint_io *io, void *ws, size_t ws_bytes,
                           void *stream) {
  if (!dims_ok(dims) || !prob_ok(prob) || !state_n || !state_n->psi || !state_n->ye || !state_n->T ||
      !state_np1 || !state_np1->psi || !state_np1->ye || !io || !io->psi_bar_out || !io->ye_bar_out ||
      !io->T_bar_out || !ws || !(io->sweep_tol >= 0.0) || io->max_sweeps < 0)
    return MGFLD_EINVAL;
  if (prob->u || prob->pair_coef) return MGFLD_EINVAL;   // shock and pair terms are not differentiated
  if (((uintptr_t)ws & 255u) != 0) return MGFLD_EINVAL;
  if (ws_bytes < make_adj_layout(dims->n_ray, dims->n_r, dims->n_e).total) return MGFLD_ENOMEM;
  return adjoint_step(make_prob(dims, prob), state_n, state_np1, io, ws, (cudaStream_t)stream);
}

}  // extern "C"
