// Frozen coefficients of one implicit step, evaluated once at (psi^n, Ye^n, T^n).
//
// Group energies (Eq. a01b), NES kernels (Eqs. d3, d4, d7; synthetic out-kernel),
// emissivity and transport mean free path (Eqs. a17, a55, d8, d8c), the
// neutrinosphere and outer ghost (Eq. a62af) and the limited diffusion
// coefficients at zone edges (Eqs. a59, a20-a26a), held fixed over the outer
// iteration so that the off-diagonal blocks of Eq. a62ae stay diagonal.
#include "mgfld_internal.cuh"

namespace mgfld {

// E_k = sqrt((E+^2 + E+ E- + E-^2)/3) so that E_k^2 dE_k = (E+^3 - E-^3)/3 (Eq. a01b).
__global__ void k_groups(int n, const double *__restrict__ e_edge, double *E, double *W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double lo = e_edge[k], hi = e_edge[k + 1];
  const double ec = sqrt((hi * hi + hi * lo + lo * lo) / 3.0);
  E[k] = ec;
  W[k] = ec * ec * (hi - lo);
}

// Per zone: Ye^n copy, e_int(T^n, Ye^n) (Eq. e10), mu_nue(rho, T^n, Ye^n) (Eqs. e11-e13) and the
// geometric constants of Eq. a58 (a^2/V with V = 4 pi (R+^3 - R-^3)/3, 1/(a c dt), 1/a).
__global__ void k_zone(Prob p, Ws w, const double *__restrict__ ye, const double *__restrict__ T) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * p.n_r) return;
  const int ray = (int)(t / p.n_r), i = (int)(t % p.n_r);
  const double rho = p.rho[t];
  w.ye_n[t] = ye[t];
  w.e_n[t] = eos_e_cold(p.eos, rho, ye[t]) + p.eos.ec * T[t];
  double mu, dmu;
  eos_mu_nue(p.eos, rho, T[t], ye[t], mu, dmu);
  const double a = lapse_at(p, ray, i);
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const double rm = re[i], rp = re[i + 1];
  const double vol = 4.0 * kPi * (rp * rp * rp - rm * rm * rm) / 3.0;
  double *z = w.zone + t * ZC_N;
  z[ZC_PRE] = a * a / vol;
  z[ZC_INV_ACDT] = 1.0 / (a * kC * p.dt);
  z[ZC_INV_A] = 1.0 / a;
  z[ZC_VOL] = vol;
  z[ZC_MU] = mu;
  z[ZC_A] = a;
  z[ZC_ACDT] = a * kC * p.dt;
}

// Row k of the NES out-kernel of zone (ray, i): down/iso-scattering coef e^{-(eps_k - eps_k')/T}
// computed directly, up-scattering from detailed balance (Eq. d7up) as coef e^{-2(eps_k' - eps_k)/T}.
__global__ void k_phi(Prob p, Ws w, const double *__restrict__ T) {
  const int n = p.n;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * p.n_r * n) return;
  const int k = (int)(t % n);
  const size_t zi = t / n;                       // ray * n_r + i
  const int ray = (int)(zi / p.n_r), i = (int)(zi % p.n_r);
  double *row = w.phi + t * n;
  if (!p.nes) {
    for (int kp = 0; kp < n; ++kp) row[kp] = 0.0;
    return;
  }
  const double inv_a = 1.0 / lapse_at(p, ray, i);
  const double Ti = T[zi], coef = p.nes[zi];
  const double ek = w.E[k] * inv_a;
  for (int kp = 0; kp < n; ++kp) {
    const double d = ek - w.E[kp] * inv_a;
    row[kp] = coef * (kp <= k ? exp(-d / Ti) : exp(2.0 * d / Ti));
  }
}

// Emissivity at Ye^n and the transport mean free path at psi^n:
// 1/lambda = kappa_a + j + kappa_s + C sum_k' w_k' [Phi_in psi + Phi_out (1 - psi)].
__global__ void k_jlam(Prob p, Ws w, const double *__restrict__ psi, const double *__restrict__ ye,
                       const double *__restrict__ T) {
  const int n = p.n;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * NS * p.n_r * n) return;
  const int k = (int)(t % n);
  size_t u = t / n;
  const int i = (int)(u % p.n_r);
  u /= p.n_r;
  const int q = (int)(u % NS);
  const int ray = (int)(u / NS);
  const size_t zi = (size_t)ray * p.n_r + i;
  const double *z = w.zone + zi * ZC_N;
  const double inv_a = z[ZC_INV_A];
  const double Ti = T[zi];
  const double sc = p.scale ? p.scale[q * n + k] : 1.0;
  const double kap = p.kabs[t] * sc, ksc = p.kscat[t] * sc;
  bool live;
  const double j = emissivity(kap, species_mu(q, z[ZC_MU]), w.E[k] * inv_a, Ti, live);
  w.jbuf[t] = j;
  const double *ps = psi + (t - k);             // psi[ray][q][i][0]
  const double *ph = w.phi + zi * n * n;
  const double inv_a3 = inv_a * inv_a * inv_a;
  double nes = 0.0;
  for (int kp = 0; kp < n; ++kp) {
    const double wk = w.W[kp] * inv_a3;
    nes += wk * (ph[kp * n + k] * ps[kp] + ph[k * n + kp] * (1.0 - ps[kp]));
  }
  w.lam[t] = 1.0 / (kap + j + ksc + kCNes * nes);
  w.psi_n[t] = psi[t];
}

// Neutrinosphere radius per (ray, q, k): where the optical depth integrated inward from
// the outer edge reaches 2/3 (linear inside the zone), else the centre edge; then the
// outer ghost ratio of Eq. a62af with R_nu clamped to the last zone centre.
__global__ void k_nusphere(Prob p, Ws w) {
  const int n = p.n;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n_ray * NS * n) return;
  const int k = t % n, q = (t / n) % NS, ray = t / (n * NS);
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const double *lam = w.lam + ((size_t)ray * NS + q) * p.n_r * n + k;
  double tau_out = 0.0;
  double rnu = re[0];
  for (int i = p.n_r - 1; i >= 0; --i) {
    const double li = lam[(size_t)i * n];
    const double dtau = (re[i + 1] - re[i]) / li;
    if (tau_out + dtau >= kTauNu) {
      rnu = re[i + 1] - (kTauNu - tau_out) * li;
      break;
    }
    tau_out += dtau;
  }
  w.rnu[t] = rnu;
  const double rI = 0.5 * (re[p.n_r - 1] + re[p.n_r]);
  const double rg = 2.0 * re[p.n_r] - rI;
  const double rn = fmin(rnu, rI);
  w.ghost[t] = (rI * rI - 0.25 * rn * rn) / (rg * rg - 0.25 * rn * rn);
}

// alpha_{i+1/2} = A_{i+1/2} D_{i+1/2} / a_{i+1/2}^2 with D = lambda_e F / (3 (R_{i+1} - R_i)),
// lambda_e = sqrt(lambda_i lambda_{i+1}), F = min(F_intrp, F_geom) at psi^n.
__global__ void k_edges(Prob p, Ws w) {
  const int n = p.n;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.n_ray * NS * p.n_r * n) return;
  const int k = (int)(t % n);
  size_t u = t / n;
  const int i = (int)(u % p.n_r);
  u /= p.n_r;
  const int q = (int)(u % NS);
  const int ray = (int)(u / NS);
  const int last = p.n_r - 1;
  if (i == last && p.bc == MGFLD_BC_REFLECT) {
    w.alpha[t] = 0.0;
    return;
  }
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const int gq = (ray * NS + q) * n + k;
  const double psi_i = w.psi_n[t];
  const double lam_i = w.lam[t];
  const double r_i = 0.5 * (re[i] + re[i + 1]);
  const double a_i = lapse_at(p, ray, i);
  double psi_r, lam_r, r_r, a_r;
  if (i < last) {
    psi_r = w.psi_n[t + n];
    lam_r = w.lam[t + n];
    r_r = 0.5 * (re[i + 1] + re[i + 2]);
    a_r = lapse_at(p, ray, i + 1);
  } else {
    psi_r = w.ghost[gq] * psi_i;
    lam_r = lam_i;
    r_r = 2.0 * re[p.n_r] - r_i;
    a_r = a_i;
  }
  const double lam_e = sqrt(lam_i * lam_r);
  const double dpsi = psi_r - psi_i;
  const double dR = r_r - r_i;
  const double psi_e = 0.5 * (psi_i + psi_r);
  const double r_e = re[i + 1];
  double F;
  if (psi_e <= 1e-300) {
    F = 0.0;
  } else if (dpsi == 0.0) {
    F = 1.0;
  } else {
    const double x = lam_e * fabs(dpsi / dR) / 3.0;
    F = 1.0 / (1.0 + x / psi_e);
    const double rnu = w.rnu[gq];
    if (r_e > rnu) {
      const double s = rnu / r_e;
      const double mu = sqrt(fmax(1.0 - s * s, 0.0));
      F = fmin(F, 0.5 * (1.0 + mu) * psi_e / x);
    }
  }
  const double D = lam_e * F / (3.0 * dR);
  const double a_e = 0.5 * (a_i + a_r);
  w.alpha[t] = 4.0 * kPi * r_e * r_e * D / (a_e * a_e);
}

static inline unsigned nblk(size_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_groups(const Prob &p, const Ws &w, cudaStream_t s) {
  k_groups<<<1, MAX_NE, 0, s>>>(p.n, p.e_edge, w.E, w.W);
  return cudaGetLastError();
}

cudaError_t launch_setup(const Prob &p, const Ws &w, const double *psi, const double *ye, const double *T,
                         cudaStream_t s) {
  const unsigned B = 256;
  const size_t nz = (size_t)p.n_ray * p.n_r;
  const size_t nzk = nz * p.n;
  const size_t nall = nzk * NS;
  k_groups<<<1, MAX_NE, 0, s>>>(p.n, p.e_edge, w.E, w.W);
  k_zone<<<nblk(nz, B), B, 0, s>>>(p, w, ye, T);
  k_phi<<<nblk(nzk, B), B, 0, s>>>(p, w, T);
  k_jlam<<<nblk(nall, B), B, 0, s>>>(p, w, psi, ye, T);
  k_nusphere<<<nblk((size_t)p.n_ray * NS * p.n, B), B, 0, s>>>(p, w);
  k_edges<<<nblk(nall, B), B, 0, s>>>(p, w);
  return cudaGetLastError();
}

}  // namespace mgfld
