// Frozen coefficients of one implicit step, evaluated once at (psi^n, Ye^n, T^n).
//
// Group energies (Eq. a01b), NES kernels (Eqs. d3, d4, d7; synthetic out-kernel),
// emissivity and transport mean free path (Eqs. a17, a55, d8, d8c), the
// neutrinosphere and outer ghost (Eq. a62af) and the limited diffusion
// coefficients at zone edges (Eqs. a59, a20-a26a), held fixed over the outer
// iteration so that the off-diagonal blocks of Eq. a62ae stay diagonal.
#include "mgfld_internal.cuh"

namespace mgfld {

// E_k = sqrt((E+^2 + E+ E- + E-^2)/3) so that E_k^2 dE_k = (E+^3 - E-^3)/3 (Eq. a01b); W = E^2 dE
// and WE = E^3 dE per group (E, W, WE consecutive arrays of MAX_NE).
__global__ void k_groups(int n, const double *__restrict__ e_edge, double *E, double *W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double lo = e_edge[k], hi = e_edge[k + 1];
  const double ec = sqrt((hi * hi + hi * lo + lo * lo) / 3.0);
  E[k] = ec;
  W[k] = ec * ec * (hi - lo);
  W[MAX_NE + k] = W[k] * ec;
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
  const Eos &e = p.eos;
  const double nb = rho / e.mb;
  const double muA = e.g1 * e.f1 * (e.g1_is_4_3 ? cbrt(nb) : pow(nb, e.g1 - 1.0)) * e.rho_fac;
  const double muB = e.g2 * e.f2 * (e.g2_is_5_2 ? nb * sqrt(nb) : pow(nb, e.g2 - 1.0));
  double mu, dmu;
  mu_nue_zone(e, muA, muB, T[t], ye[t], mu, dmu);
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
  z[ZC_MUA] = muA;
  z[ZC_MUB] = muB;
  const int last = p.n_r - 1;
  const double r_i = 0.5 * (rm + rp);
  const double r_r = i < last ? 0.5 * (re[i + 1] + re[i + 2]) : 2.0 * rp - r_i;
  const double a_r = i < last ? lapse_at(p, ray, i + 1) : a;
  const double a_e = 0.5 * (a + a_r);
  z[ZC_EI3DR] = 1.0 / (3.0 * (r_r - r_i));
  z[ZC_EGEO] = 4.0 * kPi * rp * rp / (a_e * a_e);
  z[ZC_EIR2] = 1.0 / (rp * rp);
  if (p.u && i < last) {       // shock roll-in at the outer edge (Eq. a90)
    const double *u = p.u + (size_t)ray * p.n_r;
    const double beta = (u[i + 1] - u[i]) / kC;
    z[ZC_SHOCK] = beta * fmin(fmax((fabs(beta) - kShockOn) / (kShockFull - kShockOn), 0.0), 1.0);
  } else {
    z[ZC_SHOCK] = 0.0;
  }
  const double inv_T = 1.0 / T[t];
  const double xm = mu * inv_T;
  z[ZC_INV_T] = inv_T;
  if (fabs(xm) < kEmuMax) {
    const double em = exp(xm);
    z[ZC_EMU] = em;
    z[ZC_EMUI] = 1.0 / em;
  } else {
    z[ZC_EMU] = -1.0;
    z[ZC_EMUI] = -1.0;
  }
}

// Weighted NES kernels of zone (ray, i) (Eqs. d7down, d7up): down/iso-scattering
// Phi_out(eps_k, eps_k'<=k) = coef e^{-(eps_k - eps_k')/T} is built from the N-1 ratios
// g_m = e^{-(eps_m - eps_{m-1})/T} of consecutive groups (one exponential each, shared by the
// zone through shared memory) as a running product along the row; up-scattering is its square
// (coef e^{-2(eps_k' - eps_k)/T}) and Phi_in(eps_k, eps_k') = Phi_out(eps_k', eps_k).
// Rows k and n-1-k share a thread, so that every thread runs the same n-1 steps of the
// down-scattering chains and n-1 of the up-scattering chains (no divergent loop lengths).
// The running products (P along a row's down-scattering entries, Q along its up-scattering ones,
// 1 on the diagonal) are staged in shared memory with a padded stride (n + 1), and the copy-out
// forms each entry pair from its product with the chain's own two multiplications (a = cw_k' P,
// then a P: down-scattering (out, in) = (a, a P), up-scattering (in, out) = (a, a P)), so the
// values are those of the chains, bit for bit, from one staged FP64 per entry.
static inline int phi_threads_per_zone(int n) { return (n + 1) / 2; }
static inline size_t phi_zone_bytes(int n) {
  return sizeof(double) * ((size_t)n * (n + 1) + 2 * (size_t)n) + sizeof(int) * 2 * (size_t)n;
}
// Zones per block: zones * threads per zone a multiple of 32 where the staging fits in 75 KB
// (three blocks per SM), else as many zones as fit.
static inline int phi_zones_per_block(int n) {
  const int h = phi_threads_per_zone(n);
  int g = h, b = 32;
  while (b) { const int t = g % b; g = b; b = t; }
  const int full = 32 / g;
  const int fit = (int)((size_t)75 * 1024 / phi_zone_bytes(n));
  return full <= fit ? full : (fit < 1 ? 1 : fit);
}
static inline size_t phi_smem_bytes(int n) { return (size_t)phi_zones_per_block(n) * phi_zone_bytes(n); }

// Rows ka = t and kb = n-1-t of one zone's kernels: their running products into the staged tile
// sp (row stride ld), from the zone's consecutive-group ratios gap[m] and weights cw[m]; returns
// the two rows' sums of the out-kernel (equal rows of odd n: the middle row, both chains) and,
// with want_max, the largest upper words of |in| and |out| of each row (for the FP32-pair scales).
// Down-scattering entries run along a row as P = prod gap (one multiply per step) with the
// up-scattering partner o P = cw P^2; up-scattering entries likewise from Q = prod gap.
struct PhiRowMax {
  unsigned in_a, out_a, in_b, out_b;
};
__device__ inline void phi_chains(int n, int t, const double *gap, const double *cw, double *sp, int ld, bool want_max,
                                  double &rs_a, double &rs_b, PhiRowMax &mx) {
  const int ka = t, kb = n - 1 - t;                     // ka <= kb; equal for the middle row of odd n
  double *pa = sp + (size_t)ka * ld, *pb = sp + (size_t)kb * ld;
  double rsa = cw[ka], rsb = (ka == kb) ? 0.0 : cw[kb];
  pa[ka] = 1.0;
  pb[kb] = 1.0;
  mx.in_a = mx.out_a = abs_hi_word(cw[ka]);
  mx.in_b = mx.out_b = abs_hi_word(cw[kb]);
  // Down-scattering (k' < k): row ka's ka entries, then row kb's kb entries (n - 1 steps).
  double P = 1.0;
  for (int j = 0; j < n - 1; ++j) {
    const bool first = j < ka;
    if (!first && ka == kb) break;                      // middle row: its chain is already done
    const int kp = first ? ka - 1 - j : kb - 1 - (j - ka);
    if (j == ka) P = 1.0;
    P *= gap[kp + 1];                                   // e^{-(eps_k - eps_kp)/T}
    const double o = cw[kp] * P;                        // down-scattering k -> kp
    if (first) { pa[kp] = P; rsa += o; } else { pb[kp] = P; rsb += o; }
    if (want_max) {
      const unsigned ho = abs_hi_word(o), hv = abs_hi_word(o * P);   // in: cw e^{-2(eps_k - eps_kp)/T}
      if (first) { mx.out_a = max(mx.out_a, ho); mx.in_a = max(mx.in_a, hv); }
      else { mx.out_b = max(mx.out_b, ho); mx.in_b = max(mx.in_b, hv); }
    }
  }
  // Up-scattering (k' > k): row kb's n-1-kb entries, then row ka's n-1-ka entries.
  const int nb = n - 1 - kb;
  double Q = 1.0;
  for (int j = 0; j < n - 1; ++j) {
    const bool first = j < nb;
    if (!first && ka == kb) break;
    const int kp = first ? kb + 1 + j : ka + 1 + (j - nb);
    if (j == nb) Q = 1.0;
    Q *= gap[kp];                                       // e^{-(eps_kp - eps_k)/T}
    const double v = cw[kp] * Q;                        // down-scattering kp -> k
    const double o = v * Q;                             // up-scattering k -> kp
    if (first) { pb[kp] = Q; rsb += o; } else { pa[kp] = Q; rsa += o; }
    if (want_max) {
      const unsigned ho = abs_hi_word(o), hv = abs_hi_word(v);
      if (first) { mx.out_b = max(mx.out_b, ho); mx.in_b = max(mx.in_b, hv); }
      else { mx.out_a = max(mx.out_a, ho); mx.in_a = max(mx.in_a, hv); }
    }
  }
  if (kb != ka) {
    rs_a = rsa;
    rs_b = rsb;
  } else {
    rs_a = rs_b = rsa + rsb;
    mx.in_a = mx.in_b = max(mx.in_a, mx.in_b);
    mx.out_a = mx.out_b = max(mx.out_a, mx.out_b);
  }
}

// The consecutive-group ratios e^{-(eps_m - eps_{m-1})/T} and weights C w_m = C W_m / a^3 of one
// zone into shared memory, the zone's H threads striding over the groups.
__device__ inline void phi_zone_consts(const Ws &w, int n, int t, int H, double inv_a, double Ti, double nes,
                                       double *gap, double *cw) {
  const double cc = kCNes * inv_a * inv_a * inv_a * nes;
  for (int k = t; k < n; k += H) {
    if (k > 0) gap[k] = exp(-(w.E[k] - w.E[k - 1]) * inv_a / Ti);
    cw[k] = cc * w.W[k];
  }
}

__global__ void k_phi(Prob p, Ws w, const double *__restrict__ T, int zpb) {
  extern __shared__ double smem[];
  const int n = p.n, H = (n + 1) / 2, ld = n + 1;
  double *gapm = smem;                                   // [zpb][n]  e^{-(eps_m - eps_{m-1})/T}
  double *cwm = gapm + (size_t)zpb * n;                   // [zpb][n]  C w_m = C W_m / a^3
  double *sp = cwm + (size_t)zpb * n;                     // [zpb][n][n + 1]  running products
  int *rsc = reinterpret_cast<int *>(sp + (size_t)zpb * n * ld);   // [zpb][2][n]: in, out scales
  const int zl = threadIdx.x / H, t = threadIdx.x % H;
  const unsigned nz = (unsigned)(p.n_ray * p.n_r);
  const unsigned z0 = blockIdx.x * (unsigned)zpb;
  const unsigned zi = z0 + zl;
  const bool live = zl < zpb && zi < nz;
  double *gap = gapm + (size_t)(live ? zl : 0) * n;
  double *cw = cwm + (size_t)(live ? zl : 0) * n;
  if (live) {
    const int ray = (int)(zi / (unsigned)p.n_r), i = (int)(zi - (unsigned)ray * p.n_r);
    phi_zone_consts(w, n, t, H, 1.0 / lapse_at(p, ray, i), T[zi], p.nes ? p.nes[zi] : 0.0, gap, cw);
  }
  __syncthreads();
  const bool mixed = w.nesff != nullptr;
  if (live) {
    double rsa, rsb;
    PhiRowMax mx;
    phi_chains(n, t, gap, cw, sp + (size_t)zl * n * ld, ld, mixed, rsa, rsb, mx);
    w.rsum[(size_t)zi * n + t] = rsa;
    if (n - 1 - t != t) w.rsum[(size_t)zi * n + (n - 1 - t)] = rsb;
    if (mixed) {
      // MIXED: the power-of-two scale of every row of both kernels (its largest entry into
      // [1/2, 1)), for their FP32-pair form
      int *rz = rsc + (size_t)zl * 2 * n;
      rz[t] = scale_of_max(mx.in_a);
      rz[n + t] = scale_of_max(mx.out_a);
      rz[n - 1 - t] = scale_of_max(mx.in_b);
      rz[2 * n - 1 - t] = scale_of_max(mx.out_b);
    }
  }
  __syncthreads();
  const unsigned nzb = (z0 + zpb <= nz) ? (unsigned)zpb : nz - z0;
  if (mixed) {
    for (unsigned r = threadIdx.x; r < nzb * n; r += blockDim.x) {
      const unsigned zz = r / n, row = r - zz * n;
      w.nessc[(size_t)z0 * n + r] = make_int2(rsc[zz * 2 * n + row], rsc[zz * 2 * n + n + row]);
    }
  }
  // Coalesced copy of the block's zones (contiguous in [ray][zone][k][k'] order).
  const unsigned cnt = nzb * n * n;
  const size_t base = (size_t)z0 * n * n;
  for (unsigned e = threadIdx.x; e < cnt; e += blockDim.x) {
    const unsigned row = e / (unsigned)n, col = e - row * n;
    const unsigned zz = row / (unsigned)n, k = row - zz * n;
    const double P = sp[row * ld + col];
    const double a = cwm[zz * n + col] * P, b = a * P;
    const bool down = col <= k;                       // the diagonal: P = 1, a = b = cw_k
    const double o = down ? a : b, v = down ? b : a;
    w.phout[base + e] = o;
    w.phin[base + e] = v;
    if (w.phin32) {
      // FP32 copies for the mixed path's Jacobian by exponent/mantissa bit arithmetic (integer
      // pipe, truncating); in - out is taken in FP32 (a preconditioner entry).
      const float vf = d2f_exp2(v, 0);
      w.phin32[base + e] = vf;
      w.phd32[base + e] = __fsub_rn(vf, d2f_exp2(o, 0));
      const float2 fa = split_ff(v, rsc[zz * 2 * n + k]), fb = split_ff(o, rsc[zz * 2 * n + n + k]);
      w.nesff[base + e] = make_float4(fa.x, fa.y, fb.x, fb.y);
    } else {
      w.phd[base + e] = v - o;
    }
  }
}

// The NES sums of one (zone, group) row for the four species, sum_k' phin_k' psi_k' and
// sum_k' phout_k' psi_k' (psi of species q at ps0 + q qs), each row entry loaded once for all
// species; every sum runs over k' in ascending order.  The kernels that call it are bound by
// these 8N FP64 FMAs per thread, not by the row reads.
__device__ inline void nes_sums(const double *__restrict__ fin, const double *__restrict__ fout,
                                const double *__restrict__ ps0, size_t qs, int n, double gain[NS],
                                double lp[NS]) {
#pragma unroll
  for (int q = 0; q < NS; ++q) gain[q] = lp[q] = 0.0;
  for (int kp = 0; kp < n; ++kp) {
    const double a = fin[kp], b = fout[kp];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const double v = ps0[q * qs + kp];
      gain[q] += a * v;
      lp[q] += b * v;
    }
  }
}

// Emissivity at Ye^n and the transport mean free path at psi^n, one thread per (ray, zone,
// group) for the four species (which share the zone's NES rows and, for nu_mu/tau and their
// antiparticles with mu = 0, the exponential):
// 1/lambda = kappa_a + j + kappa_s + sum_k' [phin psi_k' + phout (1 - psi_k')].
__global__ void k_jlam(Prob p, Ws w, const double *__restrict__ psi, const double *__restrict__ T) {
  const int n = p.n;
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)(p.n_ray * p.n_r * n)) return;
  const unsigned zu = t / (unsigned)n;
  const int k = (int)(t - zu * n);
  const size_t zi = zu;
  const int ray = (int)(zu / (unsigned)p.n_r), i = (int)(zu - (unsigned)ray * p.n_r);
  const double *z = w.zone + zi * ZC_N;
  const double inv_a = z[ZC_INV_A];
  const double Ti = T[zi];
  const double eps = w.E[k] * inv_a;
  const double mu = z[ZC_MU];
  const double *fin = w.phin + (zi * n + k) * n;
  const double *fout = w.phout + (zi * n + k) * n;
  const double rs = w.rsum[zi * n + k];
  // MIXED: e^{(mu_q - eps)/T} = e^{mu_q/T} e^{-eps/T} with the zone's factors (one exponential
  // per thread); the FP64 path, and zones with |mu/T| too large for the factors, take the
  // direct form.
  const double emu = w.phin32 ? z[ZC_EMU] : -1.0;
  const double ex = emu > 0.0 ? exp(-eps * z[ZC_INV_T]) : 0.0;
  double gain[NS], lp[NS];
  nes_sums(fin, fout, psi + (((size_t)ray * NS) * p.n_r + i) * n, (size_t)p.n_r * n, n, gain, lp);
  double e_mu0 = 0.0;
  for (int q = 0; q < NS; ++q) {
    const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;
    const double kap = scaled(p, p.kabs, g, q, k), ksc = scaled(p, p.kscat, g, q, k);
    double e1;
    if (emu > 0.0) {
      e1 = q == 0 ? ex * emu : (q == 1 ? ex * z[ZC_EMUI] : ex);
    } else if (q == 3) {
      e1 = e_mu0;                          // same exponent as q = 2 (mu = 0)
    } else {
      bool live;
      e1 = emissivity(1.0, species_mu(q, mu), eps, Ti, live);
      if (q == 2) e_mu0 = e1;
    }
    const double j = kap * e1;
    w.jbuf[g] = j;
    const double kt = kap + j + ksc + gain[q] + (rs - lp[q]);
    const double y = rsqrt(kt);            // sqrt(lambda): the edge mean free path is a product
    w.kinv[g] = kt;
    w.slam[g] = y;
    w.lam[g] = y * y;
    w.g0[g] = gain[q];                        // reused by the first outer iteration's residual
    w.l0[g] = lp[q];
    w.psi_n[g] = psi[g];
  }
}

// Neutrinosphere radius per (ray, q, k): where the optical depth integrated inward from
// the outer edge reaches 2/3 (linear inside the zone), else the centre edge; then the
// outer ghost ratio of Eq. a62af with R_nu clamped to the last zone centre.
// One warp per (ray, q, k): lane c sums the optical depth of the c-th chunk of zones counted
// from the outer edge, an exclusive warp scan gives each chunk the depth above it, each lane
// looks for the crossing inside its chunk, and the outermost crossing wins.
// With a ray list (the outer iteration at the n+1 coefficients) only the listed rays are done.
__global__ void k_nusphere(Prob p, Ws w, const int *__restrict__ list, int n_list, const int *__restrict__ n_dev) {
  const unsigned full = 0xffffffffu;
  const int n = p.n;
  const int per_ray = NS * n;
  int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= (list ? listed(n_list, n_dev) : p.n_ray) * per_ray) return;   // whole warps leave together
  if (list) {
    const int rl = t / per_ray;
    t = list[rl] * per_ray + (t - rl * per_ray);
  }
  const int k = t % n, q = (t / n) % NS, ray = t / (n * NS);
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const size_t off = ((size_t)ray * NS + q) * p.n_r * n + k;
  const double *kt = w.kinv + off;                 // 1/lambda, so the scan needs no division
  const int L = (p.n_r + 31) / 32;                 // zones per chunk
  const int top = p.n_r - 1 - lane * L;            // outermost zone of this lane's chunk
  const int cnt = top < 0 ? 0 : (top + 1 < L ? top + 1 : L);
  double s = 0.0;
  for (int j = 0; j < cnt; ++j) {
    const int i = top - j;
    s += (re[i + 1] - re[i]) * kt[(size_t)i * n];
  }
  // exclusive prefix over lanes (outer chunks first)
  double above = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double v = __shfl_up_sync(full, above, o);
    if (lane >= o) above += v;
  }
  double tau_out = above - s;
  double rnu = 0.0;
  bool hit = false;
  for (int j = 0; j < cnt; ++j) {
    const int i = top - j;
    const double dtau = (re[i + 1] - re[i]) * kt[(size_t)i * n];
    if (dbits(tau_out + dtau) >= dbits(kTauNu)) {          // depths >= 0: compared on the integer pipe
      rnu = re[i + 1] - (kTauNu - tau_out) * w.lam[off + (size_t)i * n];
      hit = true;
      break;
    }
    tau_out += dtau;
  }
  const unsigned hits = __ballot_sync(full, hit);
  const int src = hits ? __ffs(hits) - 1 : 0;
  rnu = hits ? __shfl_sync(full, rnu, src) : re[0];
  if (lane == 0) {
    w.rnu[t] = rnu;
    const double rI = 0.5 * (re[p.n_r - 1] + re[p.n_r]);
    const double rg = 2.0 * re[p.n_r] - rI;
    const double rn = fmin(rnu, rI);
    w.ghost[t] = (rI * rI - 0.25 * rn * rn) / (rg * rg - 0.25 * rn * rn);
  }
}

// alpha_{i+1/2} = A_{i+1/2} D_{i+1/2} / a_{i+1/2}^2 with D = lambda_e F / (3 (R_{i+1} - R_i)),
// lambda_e = sqrt(lambda_i lambda_{i+1}) (the product of the stored square roots),
// F = min(F_intrp, F_geom) at psi^n.
// With a ray list (the outer iteration at the n+1 coefficients) only the listed rays are done.
__global__ void k_edges(Prob p, Ws w, const double *__restrict__ psi_src, const int *__restrict__ list, int n_list,
                        const int *__restrict__ n_dev) {
  const int n = p.n;
  const unsigned per_ray = (unsigned)(NS * p.n_r * n);
  unsigned tu = blockIdx.x * blockDim.x + threadIdx.x;
  if (tu >= (unsigned)(list ? listed(n_list, n_dev) : p.n_ray) * per_ray) return;
  if (list) {
    const unsigned rl = tu / per_ray;
    tu = (unsigned)list[rl] * per_ray + (tu - rl * per_ray);
  }
  const size_t t = tu;
  const unsigned u1 = tu / (unsigned)n;
  const int k = (int)(tu - u1 * n);
  const unsigned u2 = u1 / (unsigned)p.n_r;
  const int i = (int)(u1 - u2 * p.n_r);
  const int q = (int)(u2 % NS);
  const int ray = (int)(u2 / NS);
  const int last = p.n_r - 1;
  if (i == last && p.bc == MGFLD_BC_REFLECT) {
    w.alpha[t] = 0.0;
    if (w.lim) w.lim[t] = 0.0;
    if (w.jl) w.jl[t] = w.jr[t] = 0.0;
    return;
  }
  const double *re = p.r_edge + (size_t)ray * (p.n_r + 1);
  const int gq = (ray * NS + q) * n + k;
  const double psi_i = psi_src[t];
  const double sl_i = w.slam[t];
  double psi_r, sl_r;
  if (i < last) {
    psi_r = psi_src[t + n];
    sl_r = w.slam[t + n];
  } else {
    psi_r = w.ghost[gq] * psi_i;
    sl_r = sl_i;
  }
  const double lam_e = sl_i * sl_r;
  const double dpsi = psi_r - psi_i;
  const double psi_e = 0.5 * (psi_i + psi_r);
  const double *z = w.zone + ((size_t)ray * p.n_r + i) * ZC_N;
  double F;
  // derivatives of Phi = F (psi_r - psi_i) with respect to psi_i and psi_r on the branch the
  // limiter selects (lambda and R_nu held), for the coefficients at the outer iterate
  double dl = 0.0, dr = 0.0;
  // (the comparisons on the integer pipe, by order keys: the same outcomes as the FP64 ones)
  if (ord_key(psi_e) <= ord_key(1e-300)) {
    F = 0.0;
  } else if (is_zero(dpsi)) {
    F = 1.0;
    dl = -1.0;
    dr = 1.0;
  } else {
    const double b = lam_e * z[ZC_EI3DR];
    const double x = b * fabs(dpsi);                         // lambda |d psi/dR| / 3
    // F = min(F_intrp, F_geom) with F_intrp = psi_e/(psi_e + x) and, outside the
    // neutrinosphere, F_geom = h psi_e / x, h = (1 + mu_nu)/2, mu_nu = sqrt(1 - rho^2),
    // rho = R_nu / R_{i+1/2}.  F_geom is the smaller one exactly when h psi_e < (1 - h) x, i.e.
    // mu_nu (psi_e + x) < x - psi_e, tested without the square root as
    // x > psi_e and (1 - rho^2)(psi_e + x)^2 < (x - psi_e)^2; only the chosen quotient is formed.
    const double rnu = w.rnu[gq];
    bool geom = false;
    double m2 = 1.0;
    const double sp = psi_e + x;
    if (dbits(re[i + 1]) > dbits(rnu) && dbits(x) > dbits(psi_e)) {   // all of them >= 0 here
      m2 = fmax(1.0 - rnu * rnu * z[ZC_EIR2], 0.0);
      const double df = x - psi_e;
      geom = dbits(m2 * (sp * sp)) < dbits(df * df);
    }
    // one quotient for both branches: numerator and denominator selected first
    double num = psi_e, den = sp, h = 1.0;
    if (geom) {
      h = 0.5 * (1.0 + sqrt(m2));
      num = h * psi_e;
      den = x;
    }
    // MIXED (the coefficients steer an iteration converged to 1e-10): the quotient from the
    // integer-pipe reciprocal seed and one Newton correction, within an ulp; the FP64 path divides
    if (!w.jl) {
      F = w.phin32 ? quot(num, den) : num / den;
    } else {
      // the derivatives need 1/den as well: one reciprocal for F and both of them
      const double r = w.phin32 ? recip2(den) : 1.0 / den;
      F = num * r;
      if (geom) {                       // Phi = (h / b) psi_e s with 1/b = |d| / x
        dl = dr = 0.5 * h * dpsi * r;
      } else {                          // Phi = psi_e d / (psi_e + b |d|) = F d
        const double s = __double_as_longlong(dpsi) >= 0 ? 1.0 : -1.0;     // dpsi != 0 here
        const double phi = F * dpsi;
        dl = ((0.5 * dpsi - psi_e) - phi * (0.5 - b * s)) * r;
        dr = ((0.5 * dpsi + psi_e) - phi * (0.5 + b * s)) * r;
      }
    }
  }
  const double K = lam_e * z[ZC_EI3DR] * z[ZC_EGEO];
  w.alpha[t] = K * F;
  if (w.lim) w.lim[t] = F;
  if (w.jl) {
    w.jl[t] = -K * dl;
    w.jr[t] = -K * dr;
  }
}

// The transport mean free path at the outer iterate of the listed rays: as k_jlam with the NES
// rates at psi and the emissivity the iteration keeps at the current Ye (jbuf); psi^n and the
// emissivity are not touched.  The NES sums at psi, which the residual of the same iterate needs
// as well, are handed to it in g0 / l0 (the residual pass then reads them as it reads the setup's
// sums at psi^n in the first iteration).
__global__ void k_lam_iter(Prob p, Ws w, const double *__restrict__ psi, const int *__restrict__ list, int n_list,
                           const int *__restrict__ n_dev) {
  const int n = p.n;
  const unsigned per_ray = (unsigned)(p.n_r * n);
  unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)listed(n_list, n_dev) * per_ray) return;
  {
    const unsigned rl = t / per_ray;
    t = (unsigned)list[rl] * per_ray + (t - rl * per_ray);
  }
  const unsigned zu = t / (unsigned)n;
  const int k = (int)(t - zu * n);
  const size_t zi = zu;
  const int ray = (int)(zu / (unsigned)p.n_r), i = (int)(zu - (unsigned)ray * p.n_r);
  const double *fin = w.phin + (zi * n + k) * n;
  const double *fout = w.phout + (zi * n + k) * n;
  const double rs = w.rsum[zi * n + k];
  double gain[NS], lp[NS];
  nes_sums(fin, fout, psi + (((size_t)ray * NS) * p.n_r + i) * n, (size_t)p.n_r * n, n, gain, lp);
  for (int q = 0; q < NS; ++q) {
    const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;
    const double kap = scaled(p, p.kabs, g, q, k), ksc = scaled(p, p.kscat, g, q, k);
    const double kt = kap + w.jbuf[g] + ksc + gain[q] + (rs - lp[q]);
    const double y = rsqrt(kt);
    w.g0[g] = gain[q];
    w.l0[g] = lp[q];
    w.kinv[g] = kt;
    w.slam[g] = y;
    w.lam[g] = y * y;
  }
}

// Moment m_k = eta psi_k of one zone's row: eta = eta1 (psi1), or eta2(eta1) (psi2).
__device__ inline double shock_moment(const Prob &p, const double *psi, size_t row, int k, bool second) {
  const double x = p.eta1 ? fmin(fmax(p.eta1[row + k], 0.0), 1.0) : 0.0;
  return (second ? minerbo_eta2(x) : x) * psi[row + k];
}

// (E_+^3 m_{k+1/2} - E_-^3 m_{k-1/2}) / ((E_+^3 - E_-^3)/3) with m_{k+1/2} the mean of the adjacent
// groups (Eqs. a92, a98), zero at the lowest and highest group edge.  Written with the energies
// at infinity: the ratio is the same on every zone's comoving grid E/a.
__device__ inline double shock_ediv(const Prob &p, const double *psi, size_t row, int k, bool second) {
  const int n = p.n;
  const double mk = shock_moment(p, psi, row, k, second);
  const double up = k + 1 < n ? 0.5 * (mk + shock_moment(p, psi, row, k + 1, second)) : 0.0;
  const double dn = k > 0 ? 0.5 * (shock_moment(p, psi, row, k - 1, second) + mk) : 0.0;
  const double el = p.e_edge[k], eh = p.e_edge[k + 1];
  const double el3 = el * el * el, eh3 = eh * eh * eh;
  return (eh3 * up - el3 * dn) / ((eh3 - el3) / 3.0);
}

// Per (ray, q, i, k): the step constant that joins the bracket of Eq. a99 (times A/a^2 = the
// flux terms of Eq. a58),
//   shock = alpha_{i+1/2} dpsi0_i + (A/a^2)_{i+1/2} dpsi1_{i+1/2} - alpha_{i-1/2} dpsi0_{i-1},
// dpsi0_i = bw_{i+1/2} (-psi1_{i,k} + Ediv(psi1_i)_k)   (Eq. a91: zone i's psi0 seen from frame i+1,
// entering the flux of Eq. a93 at both zones sharing the edge), and
// dpsi1_{i+1/2} = -bw_{i+1/2} Ediv(psi2_{i+1})_k          (Eq. a97: the edge flux brought from
// frame i+1 back to frame i, for zone i only).  Formed at psi^n like the flux coefficients;
// bw = beta times its roll-in weight comes per edge from the zone constants (ZC_SHOCK), so the
// zones away from a shock only store a zero.
__global__ void k_shock(Prob p, Ws w, const double *__restrict__ psi) {
  const int n = p.n;
  const unsigned tu = blockIdx.x * blockDim.x + threadIdx.x;
  if (tu >= (unsigned)(p.n_ray * NS * p.n_r * n)) return;
  const size_t t = tu;
  const unsigned u1 = tu / (unsigned)n;
  const int k = (int)(tu - u1 * n);
  const unsigned u2 = u1 / (unsigned)p.n_r;
  const int i = (int)(u1 - u2 * p.n_r);
  const int ray = (int)(u2 / NS);
  const int last = p.n_r - 1;
  const size_t row = t - k;                      // zone i's group row
  const double *z = w.zone + ((size_t)ray * p.n_r + i) * ZC_N;
  double sh = 0.0;
  if (i < last) {
    const double bw = z[ZC_SHOCK];
    if (bw != 0.0) {
      const double d0 = bw * (-shock_moment(p, psi, row, k, false) + shock_ediv(p, psi, row, k, false));
      const double d1 = -bw * shock_ediv(p, psi, row + n, k, true);
      sh += w.alpha[t] * d0 + z[ZC_EGEO] * d1;
    }
  }
  if (i > 0) {
    const double bw = z[ZC_SHOCK - ZC_N];          // edge i-1/2, zone i-1's constant
    if (bw != 0.0) {
      const double d0 = bw * (-shock_moment(p, psi, row - n, k, false) + shock_ediv(p, psi, row - n, k, false));
      sh -= w.alpha[t - n] * d0;
    }
  }
  w.shock[t] = sh;
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
  {
    const int zpb = phi_zones_per_block(p.n);
    const size_t sm = phi_smem_bytes(p.n);
    if (sm > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k_phi<<<nblk(nz, zpb), zpb * phi_threads_per_zone(p.n), sm, s>>>(p, w, T, zpb);
  }
  k_jlam<<<nblk(nzk, B), B, 0, s>>>(p, w, psi, T);
  k_nusphere<<<nblk((size_t)p.n_ray * NS * p.n * 32, B), B, 0, s>>>(p, w, nullptr, 0, nullptr);   // a warp per (ray, q, k)
  k_edges<<<nblk(nall, B), B, 0, s>>>(p, w, w.psi_n, nullptr, 0, nullptr);
  if (p.u) k_shock<<<nblk(nall, B), B, 0, s>>>(p, w, w.psi_n);
  if (p.pair && w.pmake) {
    const cudaError_t e = launch_pair(p, w, T, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_coef_iterate(const Prob &p, const Ws &w, const double *psi, const int *list, int n_list,
                                const int *n_dev, cudaStream_t s) {
  if (n_list == 0) return cudaSuccess;
  const unsigned B = 256;
  const size_t nzk = (size_t)n_list * p.n_r * p.n;
  const size_t nall = nzk * NS;
  k_lam_iter<<<nblk(nzk, B), B, 0, s>>>(p, w, psi, list, n_list, n_dev);
  k_nusphere<<<nblk((size_t)n_list * NS * p.n * 32, B), B, 0, s>>>(p, w, list, n_list, n_dev);
  k_edges<<<nblk(nall, B), B, 0, s>>>(p, w, psi, list, n_list, n_dev);
  return cudaGetLastError();
}

}  // namespace mgfld
