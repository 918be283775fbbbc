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
};

// Device view of one problem (pointers into caller memory and the workspace).
struct Prob {
  int n_ray, n_r, n, bc;
  double dt;
  const double *r_edge, *lapse, *e_edge, *rho, *kabs, *kscat, *nes, *scale;
  Eos eos;
};

// Workspace regions (byte offsets from the workspace base).
struct Layout {
  size_t groups, phi, lam, alpha, ghost, rnu, jbuf, psi_n, ye_n, e_n, zone, src;
  size_t diag, lower, upper, rhs, x, dinv, zled;
  size_t viol, vprev, active, iters, status, refac, nfact, nanflag, list_act, list_ref, counters;
  size_t total;
};

Layout make_layout(int n_ray, int n_r, int n, int precision);

// Per-zone constants evaluated once per step: a^2/V (flux divergence prefactor of Eq. a58),
// 1/(a c dt), 1/a, V, mu_nue at (rho, T^n, Ye^n), a and a c dt.
enum { ZC_PRE = 0, ZC_INV_ACDT = 1, ZC_INV_A = 2, ZC_VOL = 3, ZC_MU = 4, ZC_A = 5, ZC_ACDT = 6, ZC_N = 8 };

// Pointers resolved from a layout.
struct Ws {
  double *E, *W;            // group centre energy at infinity E_k and E_k^2 dE_k (Eq. a01b)
  double *phi, *lam, *alpha, *ghost, *rnu, *jbuf, *psi_n, *ye_n, *e_n;
  double *zone;             // per zone [n_ray][n_r][ZC_N]: see ZC_* below
  double *src;              // per (ray, q, i, k): total source S at the converged state
  double *diag, *lower, *upper, *rhs, *x;
  void *dinv;
  double *zled;             // per-zone ledger terms [n_ray][n_r][8]
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

// Internal energy per baryon without its thermal part (Eq. e10 / N_B at T = 0).
__device__ inline double eos_e_cold(const Eos &e, double rho, double ye) {
  const double n_b = rho / e.mb;
  const double n_e = rho * ye / e.mb;
  const double n_n = rho * (1.0 - ye) / e.mb;
  return (e.f1 * pow(n_e, e.g1) * e.rho_fac + e.f2 * pow(n_n, e.g2)) / n_b;
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
cudaError_t launch_setup(const Prob &p, const Ws &w, const double *psi, const double *ye, const double *T,
                         cudaStream_t s);
cudaError_t launch_assemble(const Prob &p, const Ws &w, const double *psi, const double *ye, const double *T,
                            double *diag, double *lower, double *upper, double *rhs, const int *list,
                            int n_list, const int *jac_flag, cudaStream_t s, double *src_out = nullptr);
cudaError_t launch_factor(int n, int n_r, int n_sys, const double *diag, const double *lower,
                          const double *upper, void *dinv, int precision, const int *ray_list,
                          cudaStream_t s);
cudaError_t launch_solve(int n, int n_r, int n_sys, const void *dinv, const double *lower,
                         const double *upper, const double *rhs, double *x, int precision,
                         const int *ray_list, cudaStream_t s);

}  // namespace mgfld
