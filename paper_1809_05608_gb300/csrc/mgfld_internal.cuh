// Internal declarations of the sm_103a MGFLD transport-step library.
//
// Layout conventions (all device arrays, C row-major):
//   per (ray, species, zone, group): index ((ray * NS + q) * n_r + i) * n + k
//   per (ray, zone):                 index ray * n_r + i
//   NES out-kernel Phi_out:          index ((ray * n_r + i) * n + k) * n + k'
//   dense block rows:                index (((ray * NS + q) * n_r + i) * n + k) * n + k'
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mgfld.h"

namespace mgfld {

constexpr int NS = 4;                       // nu_e, nubar_e, nu_mu/tau, nubar_mu/tau
constexpr int MAX_NE = 32;
constexpr double kC = 2.99792458e10;        // cm/s
constexpr double kHC = 1.23984198e-10;      // MeV cm
constexpr double kPi = 3.14159265358979323846;
constexpr double kFourPiHC3 = 4.0 * kPi / (kHC * kHC * kHC);          // number density per eps^2 d eps psi
constexpr double kCNes = 2.0 * kPi / (kC * kHC * kHC * kHC);          // Eq. d8 moment divided by c
constexpr double kExpCap = 700.0;           // cap on (mu - eps)/T in the emissivity
constexpr double kTauNu = 2.0 / 3.0;        // optical depth of the neutrinosphere

__host__ __device__ inline double stat_weight(int q) { return q < 2 ? 1.0 : 2.0; }
__host__ __device__ inline double lepton_sign(int q) { return q == 0 ? 1.0 : (q == 1 ? -1.0 : 0.0); }

// Double-gamma EoS constants with F1, F2 pre-evaluated on the host (Eqs. e4, e7).
struct Eos {
  double g1, g2, ec, gn, gp, rho0, mbc2, mb, f1, f2, rho_fac;  // rho_fac = (m_B/rho_0)^(g1-4/3)
  double log_gn_gp;         // ln(g_n / g_p)
  int g1_is_4_3, g2_is_5_2; // the default exponents, evaluated with cbrt / sqrt instead of pow
};

// Device view of one problem (pointers into caller memory and the workspace).
struct Prob {
  int n_ray, n_r, n, bc;
  double dt;
  const double *r_edge, *lapse, *e_edge, *rho, *kabs, *kscat, *nes, *scale;
  const double *u, *eta1;   // shock transport (Eqs. a90-a99): zone velocity and flux factor, or NULL
  const double *pair;       // synthetic pair process (Eq. d14): annihilation kernel per zone, or NULL
  int pair_chi;             // its angular correction (Eqs. d16-d22) on
  Eos eos;
};

// Workspace regions (byte offsets from the workspace base).
struct Layout {
  int mixed, pair;
  size_t groups, phout, phin, phd, rsum, phin32, phd32, nesff, nessc, lam, slam, g0, l0, alpha, ghost, rnu, jbuf, psi_n, ye_n, e_n,
      zone, src, shock, cdiag, cup, clow, cb, pmake, pmsum, pkill;
  size_t diag, lower, upper, rhs, x, dinv, zled, sscale, kinv, lower32, upper32, g32, rhs32;
  size_t viol, vprev, active, iters, status, refac, nfact, nanflag, list_act, list_ref, counters;
  size_t total;
};

// pair: the coupled nu / antinu systems of the pair process (wider blocks and the pair kernels).
Layout make_layout(int n_ray, int n_r, int n, int precision, int pair = 0);

// mgfld_step with the outer iteration driven from the host (one stream synchronisation per
// iteration; returns the worst ray status): what mgfld_step does when profiling is requested,
// and the path of the no-allocation entry point, which creates no graph.
mgfld_status step_host_synchronised(const mgfld_dims *dims, const mgfld_problem *prob, mgfld_state *state,
                                    const mgfld_step_opts *opts, mgfld_step_report *report, void *ws,
                                    size_t ws_bytes, void *stream);

// Argument checks and the device view of a caller's problem (shared by the C entry points).
bool dims_ok(const mgfld_dims *d);
bool prob_ok(const mgfld_problem *p);
Prob make_prob(const mgfld_dims *d, const mgfld_problem *p);

// Per-zone constants evaluated once per step: a^2/V (flux divergence prefactor of Eq. a58),
// 1/(a c dt), 1/a, V, mu_nue at (rho, T^n, Ye^n), a and a c dt.
// ZC_MUA, ZC_MUB: the Ye-independent factors of mu_e and of the nuclear part of mu_n, so that
// mu_nue(Ye) = A Ye^(g1-1) - B (1-Ye)^(g2-1) + T ln(Ye/(1-Ye)) + T ln(g_n/g_p) (Eqs. e11-e13; the
// thermal de Broglie terms of mu_p and mu_n cancel in mu_e + mu_p - mu_n).
// ZC_E*: constants of the outer edge i+1/2 of zone i (for the last zone, the edge to the
// ghost): 1/(3 (R_{i+1} - R_i)), 4 pi R_{i+1/2}^2 / a_{i+1/2}^2 and 1/R_{i+1/2}^2 (Eq. a59).
// ZC_INV_T = 1/T^n; ZC_EMU, ZC_EMUI = e^{+-mu/T^n} for the factored emissivity exponentials
// e^{(mu_q - eps)/T} = e^{mu_q/T} e^{-eps/T} of the mixed path (-1 where |mu/T| >= kEmuMax,
// which takes the direct form).  ZC_SHOCK: beta_{i+1/2} times its roll-in weight at the outer
// edge (Eq. a90; zero without velocities and at the outermost edge).
enum { ZC_PRE = 0, ZC_INV_ACDT = 1, ZC_INV_A = 2, ZC_VOL = 3, ZC_MU = 4, ZC_A = 5, ZC_ACDT = 6,
       ZC_MUA = 7, ZC_MUB = 8, ZC_EI3DR = 9, ZC_EGEO = 10, ZC_EIR2 = 11, ZC_INV_T = 12, ZC_EMU = 13,
       ZC_EMUI = 14, ZC_SHOCK = 15, ZC_N = 16 };
constexpr double kEmuMax = 600.0;

// Roll-in of the shock terms: |u_{i+1} - u_i| / c where they start and where they are whole.
constexpr double kShockOn = 0.01, kShockFull = 0.02;

// Minerbo closure (Eqs. a86-a87) with eta2_thick = 1/3 and eta2_thin = 1, eta1 clamped to [0, 1].
__device__ inline double minerbo_eta2(double eta1) {
  const double x = fmin(fmax(eta1, 0.0), 1.0);
  const double p = 1.0 / 3.0 + 2.0 * x * x / 15.0 * (3.0 - x + 3.0 * x * x);
  return 1.5 * (1.0 - p) * (1.0 / 3.0) + 0.5 * (3.0 * p - 1.0);
}

// Pointers resolved from a layout.
struct Ws {
  double *E, *W;            // group centre energy at infinity E_k and E_k^2 dE_k (Eq. a01b)
  double *WE;               // E_k^3 dE_k
  // Weighted NES kernels of each zone, [ray][zone][k][k'] (row k contiguous), with the moment
  // constant C = 2 pi / (c (hc)^3) and the group weight w_k' = eps_k'^2 d eps_k' folded in:
  //   phout[k][k'] = C w_k' Phi_out(eps_k, eps_k'),  phin[k][k'] = C w_k' Phi_in(eps_k, eps_k').
  double *phout, *phin;
  double *phd;              // phin - phout: the NES Jacobian row is -phin + psi_k phd (one FMA)
  double *rsum;             // [ray][zone][k] row sums of phout: sum_k' phout (1 - psi_k') = rsum - phout.psi
  float *phin32, *phd32;    // FP32 copies for the Jacobian of the mixed path
  // MIXED: the NES kernels as pairs of FP32 values (hi + lo, ~48 bits), each row scaled by a power
  // of two: nesff[k][k'] = (phin hi, phin lo, phout hi, phout lo) of phin[k][k'] 2^sin_k and
  // phout[k][k'] 2^sout_k, nessc[k] = (sin_k, sout_k); the later residual passes add the
  // kernels times the last correction to the kept sums in this form (FP32 pipe).
  float4 *nesff;
  int2 *nessc;
  double *lam, *alpha, *ghost, *rnu, *jbuf, *psi_n, *ye_n, *e_n;
  double *slam;             // per (ray, q, i, k): sqrt(lambda^(t)) at psi^n (edge mean free path = product)
  double *g0, *l0;          // per (ray, q, i, k): the NES sums phin.psi^n and phout.psi^n (first iteration)
  double *zone;             // per zone [n_ray][n_r][ZC_N]: see ZC_* below
  double *src;              // per (ray, q, i, k): total source S at the converged state
  double *shock;            // per (ray, q, i, k): the step-constant shock term of Eq. a99's bracket
  // Per (ray, q, i, k), written by the first residual pass when the flux coefficients are frozen
  // for the step: the psi coefficient of Eq. a58 without the iterate-dependent j and NES terms,
  // D0 = 1/(a c dt) + (a^2/V)(alpha_out (1 - ghost) + alpha_in) + kappa_a + sum_k' phout; the
  // couplings c_r = (a^2/V) alpha_out (0 in the last zone: the ghost is in D0) and c_l = (a^2/V)
  // alpha_in; and b0 = psi^n/(a c dt) - (a^2/V) shock.
  double *cdiag, *cup, *clow, *cb;
  // Pair process, or null: per zone the weighted creation kernel pmake[k][k'] = C w_k' Phi^p
  // ([ray][zone][k][k']) with its row sums pmsum, and per species the weighted annihilation kernel
  // pkill[q][k][k'] = C w_k' chi_q Phi^a ([ray][zone][q][k][k']).
  double *pmake, *pmsum, *pkill;
  double *lim;              // per (ray, q, i, k), or null: the flux limiter at the outer edge (kept
                            // by the setup for the neutrino stress)
  double *jl, *jr;          // per (ray, q, i, k), or null: d(edge flux A psi1/a^2)/d psi_i and
                            // d/d psi_{i+1} with the limiter's own dependence (coefficients at the
                            // outer iterate); null: the frozen coefficients' alpha and -alpha
  double *diag, *lower, *upper, *rhs, *x;
  void *dinv;
  double *zled;             // per-zone ledger terms [n_ray][n_r][8]
  int *sscale;              // per listed system: exponent k of the 2^k scaling of the FP32 solve
  float *lower32, *upper32; // FP32 copies of the (step-constant) coupling coefficients, MIXED only
  float *g32;               // forward-substitution results of the FP32 solve
  float *rhs32;             // the FP32 solve's scaled right-hand side
  double *kinv;             // per (ray, q, i, k): 1/lambda^(t) at psi^n (transport opacity)
  unsigned long long *viol; // per-ray max violation ratio (double bits, non-negative)
  double *vprev;
  int *active, *iters, *status, *refac, *nfact, *nanflag, *list_act, *list_ref, *counters;
};

Ws resolve(void *base, const Layout &L);

// ---------------------------------------------------------------- device helpers

__device__ inline double lapse_at(const Prob &p, int ray, int i) {
  return p.lapse ? p.lapse[(size_t)ray * p.n_r + i] : 1.0;
}

// Chemical potential of nu_e in beta equilibrium, mu_e + mu_p - mu_n (Eqs. e11-e13),
// and its Ye-derivative at fixed rho, T.
__device__ inline void eos_mu_nue(const Eos &e, double rho, double T, double ye, double &mu, double &dmu) {
  const double n_e = rho * ye / e.mb;
  const double n_n = rho * (1.0 - ye) / e.mb;
  const double lam3 = pow(kHC * kHC / (2.0 * kPi * e.mbc2 * T), e.ec);
  const double mu_e = e.g1 * e.f1 * pow(n_e, e.g1 - 1.0) * e.rho_fac;
  const double mu_nn = e.g2 * e.f2 * pow(n_n, e.g2 - 1.0);
  const double mu_n = mu_nn + T * log(n_n * lam3 / e.gn);
  const double mu_p = T * log(n_e * lam3 / e.gp);
  mu = mu_e + mu_p - mu_n;
  dmu = (e.g1 - 1.0) * mu_e / ye + T / ye + (e.g2 - 1.0) * mu_nn / (1.0 - ye) + T / (1.0 - ye);
}

// The same chemical potential from the per-zone factors A, B (see ZC_MUA) at temperature T.
__device__ inline void mu_nue_zone(const Eos &e, double A, double B, double T, double ye, double &mu, double &dmu) {
  const double yn = 1.0 - ye;
  const double mu_e = A * (e.g1_is_4_3 ? cbrt(ye) : pow(ye, e.g1 - 1.0));
  const double mu_nn = B * (e.g2_is_5_2 ? yn * sqrt(yn) : pow(yn, e.g2 - 1.0));
  mu = mu_e - mu_nn + T * (log(ye / yn) + e.log_gn_gp);
  dmu = ((e.g1 - 1.0) * mu_e + T) / ye + ((e.g2 - 1.0) * mu_nn + T) / yn;
}

// a / (tol b) for a, b >= 0 as a float, without an FP64 division: exponents by integer
// arithmetic, mantissas (the leading 23 bits) divided in FP32.  tol = tolm * 2^tole.
// Enough for convergence tests (ratio <= 1) and contraction ratios; +inf for non-finite a.
__device__ inline float tol_ratio_bits(long long ba, long long bb, float tolm, int tole);
__device__ inline float tol_ratio(double a, double b, float tolm, int tole) {
  return tol_ratio_bits(__double_as_longlong(a), __double_as_longlong(b), tolm, tole);
}
// The same from the bit patterns of the two non-negative values (integer and FP32 pipes only).
__device__ inline float tol_ratio_bits(long long ba, long long bb, float tolm, int tole) {
  if (ba == 0) return 0.f;
  if (bb == 0) return INFINITY;
  const int ea = (int)(ba >> 52), eb = (int)(bb >> 52);
  if (ea >= 2047) return INFINITY;
  const float ma = __int_as_float(0x3f800000 | (int)((ba >> 29) & 0x7fffff));
  const float mb = __int_as_float(0x3f800000 | (int)((bb >> 29) & 0x7fffff));
  const int e = ea - eb - tole;
  if (e > 120) return INFINITY;
  if (e < -120) return 0.f;
  return ldexpf(ma / (tolm * mb), e);
}

// Internal energy per baryon without its thermal part (Eq. e10 / N_B at T = 0).
__device__ inline double eos_e_cold(const Eos &e, double rho, double ye) {
  const double n_b = rho / e.mb;
  const double n_e = rho * ye / e.mb;
  const double n_n = rho * (1.0 - ye) / e.mb;
  const double pe = e.g1_is_4_3 ? n_e * cbrt(n_e) : pow(n_e, e.g1);
  const double pn = e.g2_is_5_2 ? n_n * n_n * sqrt(n_n) : pow(n_n, e.g2);
  return (e.f1 * pe * e.rho_fac + e.f2 * pn) / n_b;
}

__device__ inline double species_mu(int q, double mu_nue) {
  return q == 0 ? mu_nue : (q == 1 ? -mu_nue : 0.0);
}

// Emissivity j = kappa_a exp((mu - eps)/T) with the exponent capped (Kirchhoff, Eq. a55).
__device__ inline double emissivity(double kap, double mu, double eps, double T, bool &live) {
  const double x = (mu - eps) / T;
  live = x < kExpCap;
  return kap * exp(live ? x : kExpCap);
}

__device__ inline unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// ---------------------------------------------------------------- launchers

cudaError_t launch_groups(const Prob &p, const Ws &w, cudaStream_t s);
// The flux coefficients again at the state psi for the listed rays (mean free path with the NES
// rates at psi and the emissivity of the current Ye, neutrinosphere and ghost factor, limiter and
// its derivatives), and the NES sums at psi for the residual pass of the same iterate (g0, l0);
// the setup's other products (NES kernels, zone constants, psi^n) are kept.  Not combined with
// the shock terms (refused by mgfld_step).
cudaError_t launch_coef_iterate(const Prob &p, const Ws &w, const double *psi, const int *list, int n_list,
                                const int *n_dev, cudaStream_t s);
cudaError_t launch_setup(const Prob &p, const Ws &w, const double *psi, const double *ye, const double *T,
                         cudaStream_t s);
// diag is double (FP64 path, C ABI) or float (MIXED: the Jacobian feeds the FP32 factor only).
// first: the NES sums at psi are already in g0, l0 (psi^n in the first outer iteration, from the
// setup; the iterate with the n+1 coefficients, from launch_coef_iterate).
// The later residual passes of the mixed path (frozen coefficients, no pair process): the NES
// sums of the iterate from the kept ones plus the kernels times the last correction (FP32 pairs),
// or again in FP64 for the groups whose last correction is large against max(|psi|, tolmin); the
// row, and the FP32 Jacobian rows of the rays flagged in jac_flag.
cudaError_t launch_resid_ff(const Prob &p, const Ws &w, const double *psi, float *diag, double *lower,
                            double *upper, double *rhs, const int *list, int n_list, const int *jac_flag,
                            double tolmin, cudaStream_t s, const int *n_dev = nullptr);
// The converged sources of the mixed path (all rays) from the last residual's sums and the last
// correction, into src.
cudaError_t launch_src_mixed(const Prob &p, const Ws &w, const double *psi, double *src, cudaStream_t s);
cudaError_t launch_assemble(const Prob &p, const Ws &w, const double *psi, void *diag, int diag_fp32,
                            double *lower, double *upper, double *rhs, const int *list, int n_list,
                            const int *jac_flag, cudaStream_t s, double *src_out = nullptr, int first = 0,
                            const int *n_dev = nullptr);
cudaError_t launch_factor(int n, int n_r, int n_sys, const void *diag, int diag_fp32, const double *lower,
                          const double *upper, void *dinv, int precision, const int *ray_list,
                          cudaStream_t s, const int *n_dev = nullptr);
// MIXED-precision solve fed by bulk asynchronous copies; requires even n, 16-byte aligned
// arrays and rhs != x.  Sets *err on a bounded-wait timeout.
cudaError_t launch_solve_tma(int n, int n_r, int n_sys, const void *dinv, const float *lower32,
                             const float *upper32, const double *rhs, float *rhs32, double *x, float *g32,
                             const int *ray_list, int *sys_exp, int *err, cudaStream_t s,
                             const int *n_dev = nullptr);

// An opacity entry of (species q, group k) times the optional per-(q, k) scale (no multiplication
// without a scale: an FP64 operation saved per use, the same value).
__device__ inline double scaled(const Prob &p, const double *a, size_t g, int q, int k) {
  return p.scale ? a[g] * p.scale[q * p.n + k] : a[g];
}

// Count of a launch's listed rays: the host's n (the grid is sized for it) or, when the launch
// belongs to an outer iteration that runs without the host, the device-resident count n_dev
// (<= n; blocks past it return at once).
__device__ inline int listed(int n, const int *n_dev) { return n_dev ? *n_dev : n; }
// The same for a launch over systems, spr systems per listed ray.
__device__ inline int listed_sys(int n_sys, const int *n_dev, int spr) { return n_dev ? *n_dev * spr : n_sys; }

// Exact power-of-two rescaling between FP64 and FP32 by exponent arithmetic on the bit
// patterns (integer pipe only; mantissa truncated to 24 bits; results below the FP32 normal
// range flush to zero, above it become infinite).
__device__ inline float d2f_exp2(double v, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0.f;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ef = e == 0x7ff ? 255 : e - 1023 + k + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u | (e == 0x7ff ? (unsigned)((b >> 29) & 0x7fffff) : 0u));
  return __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7fffff));
}
__device__ inline double f2d_exp2(float v, int k) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xff);
  if (e == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned long long man = (unsigned long long)(b & 0x7fffffu) << 29;
  if (e == 255) return __longlong_as_double((long long)(sign | (0x7ffull << 52) | man));
  const long long ed = (long long)e - 127 + 1023 + k;
  if (ed <= 0) return __longlong_as_double((long long)sign);
  if (ed >= 0x7ff) return __longlong_as_double((long long)(sign | (0x7ffull << 52)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)ed << 52) | man));
}

// v 2^k as an unevaluated sum hi + lo of two FP32 values (integer pipe and two FP32
// multiplications): hi is d2f_exp2(v, k) (the leading 24 bits), lo the remaining 29 bits of the
// mantissa rounded to 24, so hi + lo carries ~48 bits of v.  Where lo would fall below the FP32
// normal range (v 2^k below ~2^-103) it is dropped; hi follows d2f_exp2.
__device__ inline float2 split_ff(double v, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const float hi = d2f_exp2(v, k);
  const int E = (int)((b >> 52) & 0x7ff);
  const int ef = E + k - 919;                  // exponent field of 2^(E - 1023 + k - 23)
  float lo = 0.f;
  if (E != 0 && E != 0x7ff && ef >= 1 && ef <= 254) {
    lo = __uint2float_rn((unsigned)(b & 0x1fffffffull)) * 0x1p-29f * __int_as_float(ef << 23);
    if (b >> 63) lo = -lo;
  }
  return make_float2(hi, lo);
}

// The power-of-two exponent k that brings max |v| of a set into [1/2, 1), from the maximum of
// the upper words of the bit patterns (0 for an all-zero or non-finite set).
__device__ inline int scale_of_max(unsigned hi_word_max) {
  const int e = (int)(hi_word_max >> 20);
  return (e > 0 && e < 0x7ff) ? 1022 - e : 0;
}
__device__ inline unsigned abs_hi_word(double v) {
  return (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
}
// 1/d without FP64-pipe conversions or compares (the pivots of the FP64 Gauss-Jordan steps; the
// seed of the energy remap's quotients): the mantissa of d, rounded to 24 bits, becomes an FP32
// value m in [1, 2] by bit manipulation (integer pipe), its reciprocal is taken in FP32, the
// exponent of 1/d is rebuilt from the two exponents, and one Newton-Raphson step
// x1 = x0 + x0 (1 - d x0) (two FMAs on the FP64 pipe) takes the ~2^-23 seed to ~2^-46 relative.
// Zero, subnormal, non-finite and extreme-exponent values take a plain division (rare; a zero
// pivot means a singular block).  The factors only steer the outer iteration, whose fixed point
// is set by the FP64 residual.
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

// n/d within about an ulp at a third of a division's FP64 instructions: the reciprocal seed of
// recip (~2^-46, its conversions on the integer pipe) and one Newton correction of the quotient,
// q = n x + x (n - d n x), whose error is of the order of the square of the seed's.  Zero,
// subnormal and non-finite divisors, and quotients that overflow, take the plain division (the
// tests on the integer pipe).
__device__ inline double quot(double n, double d) {
  const int ed = (int)((__double_as_longlong(d) >> 52) & 0x7ff);
  const double x = recip(d);
  const double q = n * x;
  const int eq = (int)((__double_as_longlong(q) >> 52) & 0x7ff);
  if (ed == 0 || ed == 0x7ff || eq == 0x7ff) return n / d;
  return fma(x, fma(-d, q, n), q);
}

// 1/d within about an ulp: recip and a second Newton-Raphson step (zero, subnormal and non-finite
// d: the plain division).
__device__ inline double recip2(double d) {
  const int ed = (int)((__double_as_longlong(d) >> 52) & 0x7ff);
  if (ed == 0 || ed == 0x7ff) return 1.0 / d;
  const double x = recip(d);
  return fma(x, fma(-d, x, 1.0), x);
}

// Order keys of doubles for comparisons on the integer pipe: the bit pattern of a non-negative
// value orders like the value, so two non-negative values compare by their patterns (dbits); ord_key
// maps every non-NaN value to an integer of the same order (-0 just below +0).
__device__ inline long long ord_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}
__device__ inline bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }

// mu_nue_zone with its three quotients (ye / yn, and the two terms of dmu over ye and yn) from one
// reciprocal of ye yn (recip2, within about an ulp): the mixed path's Ye update, whose iteration
// converges to 1e-10.
__device__ inline void mu_nue_zone_q(const Eos &e, double A, double B, double T, double ye, double &mu,
                                     double &dmu) {
  const double yn = 1.0 - ye;
  const double r = recip2(ye * yn);
  const double mu_e = A * (e.g1_is_4_3 ? cbrt(ye) : pow(ye, e.g1 - 1.0));
  const double mu_nn = B * (e.g2_is_5_2 ? yn * sqrt(yn) : pow(yn, e.g2 - 1.0));
  mu = mu_e - mu_nn + T * (log(ye * (ye * r)) + e.log_gn_gp);
  dmu = ((e.g1 - 1.0) * mu_e + T) * (yn * r) + ((e.g2 - 1.0) * mu_nn + T) * (ye * r);
}

// MIXED-precision factor with FP32 diagonal blocks and FP32 coupling coefficients.
cudaError_t launch_factor_f32(int n, int n_r, int n_sys, const float *diag, const float *lower32,
                              const float *upper32, float *dinv, const int *ray_list, cudaStream_t s,
                              const int *n_dev = nullptr);
// Pair process (pair.cu): the weighted kernels of every zone (after the neutrinosphere scan),
// and the residual / Jacobian of the coupled pair systems (blocks of 2 n rows, vectors
// [ray][pair][zone][2 n]; src_out in the psi layout).
cudaError_t launch_pair(const Prob &p, const Ws &w, const double *T, cudaStream_t s);
cudaError_t launch_assemble_pair(const Prob &p, const Ws &w, const double *psi, void *diag, int diag_fp32,
                                 double *lower, double *upper, double *rhs, const int *list, int n_list,
                                 const int *jac_flag, cudaStream_t s, double *src_out, int first,
                                 const int *n_dev = nullptr);

// Thread-per-row factor and substitution of systems of block width nb <= 48 with spr systems per
// ray (the coupled nu / antinu pair systems: nb = 2 n, spr = 2), FP64 or FP32 (fp32: float blocks,
// couplings and factors; the substitution scales each system's right-hand side by a power of two
// into rhs32 / sys_exp first).
cudaError_t launch_factor_rows(int nb, int n_r, int n_sys, int spr, const void *diag, const void *lower,
                               const void *upper, void *dinv, int fp32, const int *ray_list, cudaStream_t s,
                               const int *n_dev = nullptr);
cudaError_t launch_solve_rows(int nb, int n_r, int n_sys, int spr, const void *dinv, const void *lower,
                              const void *upper, const double *rhs, float *rhs32, int *sys_exp, double *x, int fp32,
                              const int *ray_list, cudaStream_t s, const int *n_dev = nullptr);
cudaError_t launch_solve(int n, int n_r, int n_sys, const void *dinv, const double *lower,
                         const double *upper, const double *rhs, double *x, int precision,
                         const int *ray_list, cudaStream_t s, const int *n_dev = nullptr);

}  // namespace mgfld
