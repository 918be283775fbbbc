// Residual and Jacobian rows of the per-species Newton system (Eqs. a58, a59, a62ac).
//
// One thread owns the equation of (ray, species q, zone i, group k):
//   G = (psi - psi^n)/(a c dt) + (a^2/V)[A psi1/a^2 |_{i+1/2} - A psi1/a^2 |_{i-1/2}] - S,
//   psi1_{i+1/2} = -D_{i+1/2} (psi_{i+1} - psi_i)              (Eq. a59, D frozen at psi^n)
//   (with a shock, Eqs. a93/a99: a step constant joins the bracket, see k_shock)
//   S = j (1 - psi) - kappa_a psi                             (Eq. a55)
//     + C [(1 - psi_k) sum_k' w_k' Phi_in[k,k'] psi_k' - psi_k sum_k' w_k' Phi_out[k,k'] (1 - psi_k')]
//                                                              (Eq. d8, Phi_1 = 0; Phi_in[k,k'] = Phi_out[k',k])
// and, when the ray is flagged for a new factorisation, the dense row dG_k/dpsi_k' of the
// diagonal block plus the diagonal couplings to zones i-1 and i+1 (Eq. a62ae).
#include "mgfld_internal.cuh"

namespace mgfld {

template <typename TD>
__global__ void k_assemble(Prob p, Ws w, const double *__restrict__ psi, TD *__restrict__ diag,
                           double *__restrict__ lower, double *__restrict__ upper, double *__restrict__ rhs,
                           const int *__restrict__ list, int n_list, const int *__restrict__ jac_flag,
                           double *__restrict__ src_out, int first, const int *__restrict__ n_dev) {
  const int n = p.n;
  // 32-bit index arithmetic (element counts are below 2^31, checked on the host).
  const unsigned per_ray = (unsigned)(NS * p.n_r * n);
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)listed(n_list, n_dev) * per_ray) return;
  const unsigned rl = t / per_ray;
  const int ray = list ? list[rl] : (int)rl;
  // Thread order (zone, species, group) inside a ray: the four species of a zone share the
  // zone's NES kernel rows through L1.
  const unsigned local = t - rl * per_ray;
  const unsigned kq = local / (unsigned)n;
  const int k = (int)(local - kq * n);
  const int q = (int)(kq % NS);
  const int i = (int)(kq / NS);
  const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;   // (ray, q, i, k) storage index
  const size_t zi = (size_t)ray * p.n_r + i;
  const int last = p.n_r - 1;

  const double *z = w.zone + zi * ZC_N;
  const double pre = z[ZC_PRE];
  const double inv_acdt = z[ZC_INV_ACDT];

  const double *ps = psi + (g - k);
  const double pk = ps[k];
  const double *fin = w.phin + (zi * n + k) * n;
  const double *fout = w.phout + (zi * n + k) * n;
  double gain = 0.0, lp = 0.0;
  if (first) {                 // formed at this psi already: by the setup (psi^n) or with the n+1 coefficients
    gain = w.g0[g];
    lp = w.l0[g];
  } else if (src_out && w.phin32) {
    // MIXED, converged state psi_m + dpsi (dpsi = w.x, the last correction of this ray): the
    // sums of the ray's last residual (at psi_m, kept in g0/l0) plus phin.dpsi and phout.dpsi,
    // taken in FP32.  |dpsi| is below the tolerance, so the FP32 rounding (relative 2^-24 of
    // |phin| |dpsi|) stays far below the FP64 rounding of the sums themselves.
    const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
    const double *dx = w.x + (g - k);
    float dg = 0.f, dl = 0.f;
    for (int kp = 0; kp < n; ++kp) {
      const float d = (float)dx[kp];
      dg = fmaf(fi[kp], d, dg);
      dl = fmaf(fi[kp] - fd[kp], d, dl);
    }
    gain = w.g0[g] + (double)dg;
    lp = w.l0[g] + (double)dl;
  } else {
    for (int kp = 0; kp < n; ++kp) {
      const double pv = ps[kp];
      gain += fin[kp] * pv;
      lp += fout[kp] * pv;
    }
    if (w.phin32 && !src_out) {   // MIXED: keep this residual's sums for the final sources
      w.g0[g] = gain;
      w.l0[g] = lp;
    }
  }
  const double j = w.jbuf[g];
  double G, dg, c_low, c_up;
  if (!first && !src_out && !w.jl) {
    // Later iterations with the coefficients frozen for the step: the constants the first pass
    // stored, G = psi (D0 + j + gain - lp) - c_r psi_{i+1} - c_l psi_{i-1} - (b0 + j + gain), which
    // is Eq. a58 with the flux of Eq. a59 and S regrouped (the terms in psi collected).
    dg = ((w.cdiag[g] + j) + gain) - lp;
    G = fma(pk, dg, -((w.cb[g] + j) + gain));
    c_up = w.cup[g];
    c_low = w.clow[g];
    if (i < last) G = fma(-c_up, ps[k + n], G);
    if (i > 0) G = fma(-c_low, ps[k - (ptrdiff_t)n], G);
  } else {
    const double loss = w.rsum[zi * n + k] - lp;          // sum_k' phout (1 - psi_k')
    const double kap = scaled(p, p.kabs, g, q, k);
    const double S = j * (1.0 - pk) - kap * pk + ((1.0 - pk) * gain - pk * loss);
    if (src_out) {               // converged sources for Eq. a62b and the ledgers
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
    // shock transport: the step-constant frame terms of Eqs. a93 and a99 (formed at psi^n)
    const double sh = p.u ? w.shock[g] : 0.0;
    G = (pk - w.psi_n[g]) * inv_acdt + pre * (flux_out - flux_in + sh) - S;
    // flux parts of the row: d(flux at i+1/2)/d psi_i = jl, d/d psi_{i+1} = jr; alpha and -alpha with
    // the frozen coefficients, with the limiter's own derivative when they follow the iterate
    double jdiag = al_out * (1.0 - gh) + al_in, jlow = al_in, jup = al_out;
    if (w.jl) {
      const double jl_out = w.jl[g], jr_out = w.jr[g];
      const double jl_in = i > 0 ? w.jl[g - n] : 0.0, jr_in = i > 0 ? w.jr[g - n] : 0.0;
      jdiag = jl_out + gh * jr_out - jr_in;
      jlow = jl_in;
      jup = -jr_out;
    }
    dg = inv_acdt + pre * jdiag + j + kap + (gain + loss);
    c_low = pre * jlow;
    c_up = i < last ? pre * jup : 0.0;
    if (first && !w.jl) {
      // the step constants of the later iterations (frozen coefficients): D0 with the ghost of
      // the outer edge folded in, the couplings, and the psi-independent part b0
      w.cdiag[g] = inv_acdt + pre * jdiag + kap + w.rsum[zi * n + k];
      w.cup[g] = c_up;
      w.clow[g] = c_low;
      w.cb[g] = w.psi_n[g] * inv_acdt - pre * sh;
    }
  }
  rhs[g] = -G;

  if (jac_flag && !jac_flag[ray]) return;
  TD *row = diag + g * n;
  // dS_k/dpsi_k' = (1 - psi_k) phin + psi_k phout = phin - psi_k phd, entered with a minus;
  // dg joins the diagonal entry in the rows' precision.  Rows are written 16 bytes at a time where n allows
  // (the rows of one warp's threads are 16-byte aligned and contiguous per species).
  if (sizeof(TD) == 4 && w.phin32) {
    const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
    // FP32 operands from the integer pipe (truncated; the FP32 Jacobian is the preconditioner of
    // the FP64 refinement), dg joining the diagonal in FP32
    const float pf = d2f_exp2(pk, 0);
    const float dk = fmaf(pf, fd[k], -fi[k]) + (float)dg;
    if ((n & 3) == 0) {
      for (int c = 0; c < n; c += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(fi + c);
        const float4 d = *reinterpret_cast<const float4 *>(fd + c);
        float4 v = make_float4(fmaf(pf, d.x, -a.x), fmaf(pf, d.y, -a.y), fmaf(pf, d.z, -a.z), fmaf(pf, d.w, -a.w));
        if (k == c) v.x = dk;
        if (k == c + 1) v.y = dk;
        if (k == c + 2) v.z = dk;
        if (k == c + 3) v.w = dk;
        *reinterpret_cast<float4 *>(row + c) = v;
      }
    } else {
      for (int kp = 0; kp < n; ++kp) row[kp] = TD(kp == k ? dk : fmaf(pf, fd[kp], -fi[kp]));
    }
  } else {
    const double *fd = w.phd + (zi * n + k) * n;
    const double dk = fma(pk, fd[k], -fin[k]) + dg;
    bool done = false;
    if constexpr (sizeof(TD) == 8) {
      if ((n & 1) == 0) {
        for (int c = 0; c < n; c += 2) {
          const double2 a = *reinterpret_cast<const double2 *>(fin + c);
          const double2 d = *reinterpret_cast<const double2 *>(fd + c);
          double2 v = make_double2(fma(pk, d.x, -a.x), fma(pk, d.y, -a.y));
          if (k == c) v.x = dk;
          if (k == c + 1) v.y = dk;
          *reinterpret_cast<double2 *>(row + c) = v;
        }
        done = true;
      }
    }
    if (!done) {
      for (int kp = 0; kp < n; ++kp) row[kp] = TD(kp == k ? dk : fma(pk, fd[kp], -fin[kp]));
    }
  }
  lower[g] = -c_low;
  upper[g] = -c_up;
  if (w.lower32) {
    w.lower32[g] = d2f_exp2(-c_low, 0);
    w.upper32[g] = d2f_exp2(-c_up, 0);
  }
}

cudaError_t launch_assemble(const Prob &p, const Ws &w, const double *psi, void *diag, int diag_fp32,
                            double *lower, double *upper, double *rhs, const int *list, int n_list,
                            const int *jac_flag, cudaStream_t s, double *src_out, int first, const int *n_dev) {
  const size_t total = (size_t)n_list * NS * p.n_r * p.n;
  if (total == 0) return cudaSuccess;
  const unsigned B = 256;
  const unsigned grid = (unsigned)((total + B - 1) / B);
  if (diag_fp32)
    k_assemble<float><<<grid, B, 0, s>>>(p, w, psi, (float *)diag, lower, upper, rhs, list, n_list, jac_flag,
                                         src_out, first, n_dev);
  else
    k_assemble<double><<<grid, B, 0, s>>>(p, w, psi, (double *)diag, lower, upper, rhs, list, n_list,
                                          jac_flag, src_out, first, n_dev);
  return cudaGetLastError();
}

// The converged sources of the mixed path for Eq. a62b and the ledgers, one thread per (ray, q, i,
// k) of every ray:
//   S = j (1 - psi) - kappa_a psi + (1 - psi) gain - psi loss          (Eqs. a55, d8)
// at psi = psi_m + dpsi (dpsi the ray's last, sub-tolerance correction w.x): gain and
// loss = rsum - lp from the sums of the ray's last residual at psi_m (g0, l0) plus phin.dpsi and
// (phin - phd).dpsi taken in FP32 (|dpsi| is below the tolerance, so their FP32 rounding stays far
// below the FP64 rounding of the sums), the two corrections joined in FP32 before one conversion.
// The block stages the corrections of the rows it covers in shared memory as FP32, one conversion
// per value instead of one per product.
constexpr int kSrcThreads = 256;
__global__ void __launch_bounds__(kSrcThreads)
k_src_mixed(Prob p, Ws w, const double *__restrict__ psi, double *__restrict__ src) {
  __shared__ float xs[kSrcThreads + 2 * MAX_NE];
  const int n = p.n;
  const unsigned per_ray = (unsigned)(NS * p.n_r * n);
  const unsigned total = (unsigned)p.n_ray * per_ray;
  const unsigned b0 = blockIdx.x * kSrcThreads;
  const unsigned last = min(b0 + kSrcThreads, total) - 1;
  const unsigned gq0 = b0 / (unsigned)n;                    // first (ray, zone, species) row group
  const unsigned cnt = (last / (unsigned)n - gq0 + 1) * (unsigned)n;
  for (unsigned j = threadIdx.x; j < cnt; j += kSrcThreads) {
    const unsigned gq = gq0 + j / (unsigned)n, kk = j % (unsigned)n;
    const unsigned ray = gq / (unsigned)(NS * p.n_r), rem = gq - ray * (unsigned)(NS * p.n_r);
    const unsigned i = rem / NS, q = rem - i * NS;
    xs[j] = (float)w.x[(((size_t)ray * NS + q) * p.n_r + i) * n + kk];
  }
  __syncthreads();
  const unsigned t = b0 + threadIdx.x;
  if (t >= total) return;
  const unsigned ray = t / per_ray;
  const unsigned local = t - ray * per_ray;
  const unsigned kq = local / (unsigned)n;
  const int k = (int)(local - kq * n);
  const int q = (int)(kq % NS);
  const int i = (int)(kq / NS);
  const size_t g = (((size_t)ray * NS + q) * p.n_r + i) * n + k;
  const size_t zi = (size_t)ray * p.n_r + i;
  const float *fi = w.phin32 + (zi * n + k) * n, *fd = w.phd32 + (zi * n + k) * n;
  const float *dx = xs + (t / (unsigned)n - gq0) * (unsigned)n;
  float dg = 0.f, dl = 0.f;
  for (int kp = 0; kp < n; ++kp) {
    const float d = dx[kp], a = fi[kp];
    dg = fmaf(a, d, dg);
    dl = fmaf(a - fd[kp], d, dl);
  }
  const double pk = psi[g];
  const double q1 = 1.0 - pk;
  const float pf = d2f_exp2(pk, 0);
  // (1 - psi) dgain + psi dlp: the FP32 part of (1 - psi) gain - psi loss
  const float corr = fmaf(1.f - pf, dg, pf * dl);
  const double kap = scaled(p, p.kabs, g, q, k);
  const double loss0 = w.rsum[zi * n + k] - w.l0[g];
  double S = fma(q1, w.g0[g], fma(-pk, loss0, (double)corr));
  S = fma(w.jbuf[g], q1, fma(-kap, pk, S));
  src[g] = S;
}

cudaError_t launch_src_mixed(const Prob &p, const Ws &w, const double *psi, double *src, cudaStream_t s) {
  const size_t total = (size_t)p.n_ray * NS * p.n_r * p.n;
  if (total == 0) return cudaSuccess;
  k_src_mixed<<<(unsigned)((total + kSrcThreads - 1) / kSrcThreads), kSrcThreads, 0, s>>>(p, w, psi, src);
  return cudaGetLastError();
}

}  // namespace mgfld
