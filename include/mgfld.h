/*
 * mgfld.h -- C ABI of the GB300 (sm_103a) implicit MGFLD transport step.
 *
 * The operation is the Lagrangian transport step of ray-by-ray multi-group
 * flux-limited diffusion (Bruenn et al., CHIMERA, Sec. "Lagrangian Transport
 * Step" and Sec. "Solution of the Transport Equations"):  for every radial ray,
 * the zeroth-moment equation (Eq. a58) with the flux-limited first moment
 * (Eq. a59, limiter Eqs. a20-a26a) and the electron-fraction equation (Eq. a62a)
 * are solved implicitly for psi^(0) at t^{n+1} and Ye^{n+1} by an outer Newton
 * iteration on a block-tridiagonal system in radius (Eqs. a62aa-a62ae, boundary
 * conditions Eq. a62af), then the internal energy (Eq. a62b) and temperature
 * are updated.  Sources: absorption/emission (Eq. a55), iso-energetic
 * scattering (Eq. d8c, in the mean free path only) and neutrino-electron
 * scattering with dense group coupling (Eqs. d1-d8).
 *
 * Conventions for every entry point:
 *   - All array pointers are DEVICE pointers unless stated, FP64, C row-major,
 *     owned by the caller.  The library never allocates or frees memory: the
 *     caller provides every buffer, including the workspace.
 *   - Sizes: n_ray rays, n_r radial zones, n_e energy groups (1..32), n_s = 4
 *     species in the order nu_e, nubar_e, nu_mu/tau, nubar_mu/tau, with
 *     n_ray * n_s * n_r * n_e < 2^31 (EINVAL otherwise; split the rays).
 *   - Units: cm, s, g/cm^3, MeV (T is kT in MeV).
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream) except where stated (mgfld_step with
 *     profiling, mgfld_step_noalloc and mgfld_adjoint synchronise it).
 *   - Errors are returned as mgfld_status; nothing aborts, throws or traps.
 *     Argument errors are detected on the host before any launch.
 */
#ifndef MGFLD_H
#define MGFLD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MGFLD_OK = 0,
  MGFLD_EINVAL = 1,   /* bad argument (sizes, NULL pointer, unsupported n_e) */
  MGFLD_ENOMEM = 2,   /* caller-provided workspace smaller than required      */
  MGFLD_ENOCONV = 3,  /* at least one ray did not converge within max_iter    */
  MGFLD_ENAN = 4,     /* a non-finite value appeared in at least one ray      */
  MGFLD_ECUDA = 5     /* a CUDA launch or runtime call failed                 */
} mgfld_status;

typedef enum { MGFLD_FP64 = 0, MGFLD_MIXED = 1 } mgfld_precision;
typedef enum { MGFLD_BC_GHOST = 0, MGFLD_BC_REFLECT = 1 } mgfld_outer_bc;

typedef struct { int n_ray, n_r, n_e, n_s; } mgfld_dims;

/* Double-gamma equation of state (Sec. "Double-gamma EoS", Eqs. e2-e13). */
typedef struct {
  double gamma1, gamma2, e_coef, g_n, g_p, rho_nuc, rho_0, mb_c2, m_b;
} mgfld_eos_params;

/* Default double-gamma constants: gamma1 = 4/3, gamma2 = 2.5, E_coef = 3/2,
 * g_n = g_p = 2, rho_nuc = rho_0 = 2.5e14 g/cm^3, m_B c^2 = 939.565 MeV,
 * m_B = 1.674927e-24 g.  Host function. */
mgfld_eos_params mgfld_eos_default(void);

/* Statement of one step's problem (Eqs. a58-a62a): given matter and grid. */
typedef struct {
  const double *r_edge;     /* [n_ray][n_r+1] zone-edge areal radii R_{i+1/2}, increasing, > 0 at the centre edge allowed 0 */
  const double *lapse;      /* [n_ray][n_r] lapse a_i at zone centres, or NULL for a = 1 (Eq. a8a) */
  const double *e_edge;     /* [n_e+1] group edges of the energy at infinity E = a eps (MeV), increasing */
  const double *rho;        /* [n_ray][n_r] rest-mass density */
  const double *kappa_abs;  /* [n_ray][n_s][n_r][n_e] absorption opacity 1/lambda_a at the local group energy (1/cm) */
  const double *kappa_scat; /* [n_ray][n_s][n_r][n_e] iso-energetic scattering opacity (Eq. d8c) (1/cm) */
  const double *nes_coef;   /* [n_ray][n_r] NES kernel scale (cm^3/s), or NULL for no NES */
  const double *scale;      /* [n_s][n_e] opacity scales multiplying kappa_abs and kappa_scat, or NULL */
  mgfld_eos_params eos;
  double dt;                /* time step (s) */
  int outer_bc;             /* mgfld_outer_bc */
  /* Transport through a shock (Sec. "Transport through a Shock", Eqs. a90-a99), both optional:
   * u     [n_ray][n_r] zone-centred fluid velocity (cm/s), or NULL for no shock terms.  At each
   *       interior edge i+1/2, beta = (u_{i+1} - u_i)/c; the frame corrections dpsi0_shock (Eq. a91,
   *       the flux of Eq. a93) and dpsi1_shock (Eq. a97, the bracket of Eq. a99) are weighted by a
   *       roll-in rising linearly from 0 at |beta| = 0.01 to 1 at |beta| = 0.02, and are formed
   *       at psi^n for the step (like the diffusion coefficient), so the Newton system keeps its
   *       block structure.  The outermost edge and the centre edge carry none.
   * eta1  [n_ray][n_s][n_r][n_e] flux factor psi1/psi0 at zone centres (clamped to [0, 1]) from
   *       which psi1 = eta1 psi^n and psi2 = eta2(eta1) psi^n (Minerbo closure, Eqs. a86-a87) are
   *       formed, or NULL for eta1 = 0.  Read only when u is set.
   * The shock terms are not differentiated: mgfld_adjoint returns MGFLD_EINVAL when u is set. */
  const double *u;
  const double *eta1;
  /* Synthetic pair process (Eq. d14, zeroth moment, Legendre order 0), optional:
   * pair_coef [n_ray][n_r] the annihilation kernel Phi^a (cm^3/s), or NULL for no pair process;
   *       the creation kernel is e^{-(eps + eps')/T^n} Phi^a (Eq. d12, the pair energy eps + eps'
   *       given to the e-e+ pair), nu_e paired with nubar_e and nu_mu,tau with nubar_mu,tau.  The
   *       process enters the sources (and so Eq. a62b) but not the transport mean free path, and
   *       leaves the lepton number (Eq. a62a) unchanged.  It couples each species to its partner
   *       group by group: mgfld_step then solves per (ray, pair) with coupled 2 n_e x 2 n_e zone
   *       blocks (n_e <= 24; FP64 or FP32 factors as opts->precision), and needs the workspace
   *       of mgfld_workspace_bytes_pair.  Not combined with opts->coef_iterate (EINVAL);
   *       mgfld_assemble and mgfld_adjoint return MGFLD_EINVAL when it is set.
   * pair_chi nonzero: the angular correction chi = min(chi_1, chi_2) of the annihilation kernel
   *       (Eqs. d16-d22) per (zone, eps, eps'): chi_1 = 1 - eta eta' / 6 with the flux factors of
   *       `eta1` (zero where eta1 is NULL), chi_2 from the cones of radiation emitted by each
   *       species' neutrinosphere at psi^n (Eqs. d17-d19), extended inside it by Eq. d22.  Read
   *       only when pair_coef is set. */
  const double *pair_coef;
  int pair_chi;
} mgfld_problem;

/* State at t^n on entry, t^{n+1} on exit (in place). */
typedef struct {
  double *psi;   /* [n_ray][n_s][n_r][n_e] zeroth angular moment psi^(0) */
  double *ye;    /* [n_ray][n_r] electron fraction */
  double *T;     /* [n_ray][n_r] temperature kT (MeV) */
} mgfld_state;

typedef struct {
  int precision;       /* mgfld_precision: FP64 Newton, or FP32 factor + FP64 residual refinement */
  double tol;          /* convergence: |d psi| <= tol * max(|psi|, tolmin_psi) for all (i,k,q) (Eq. a62ab) */
  double tolmin_psi;   /* typically 1 (Eq. a62ab) */
  double tol_ye;       /* |d Ye| <= tol_ye * max(Ye, tolmin_ye) */
  double tolmin_ye;    /* typically 0.1 */
  int max_iter;        /* outer-iteration cap per ray */
  double refactor_ratio; /* modified Newton: a ray keeps its factors while each correction is at most
                            this fraction of the previous one, and is refactored otherwise.  MIXED
                            always iterates this way (0 selects 0.1); FP64 does when > 0, and with 0
                            refactors every iteration (Newton, Eq. a62aa) */
  double *profile;     /* HOST pointer to double[MGFLD_PROF_N][2] or NULL.  When set, each kernel
                          category is bracketed by CUDA events on `stream` and its elapsed
                          milliseconds and launch count are ADDED to profile[c][0], profile[c][1]. */
  int coef_iterate;    /* 0: the flux coefficients of Eq. a59 (transport mean free path, limiter,
                          neutrinosphere, ghost factor) are formed once at psi^n, Ye^n.
                          Nonzero: the paper-literal n+1 coefficients of Eq. a59 - formed again at
                          every outer iterate (T held at T^n), the Jacobian adding the limiter's
                          derivative on the two zones of each edge (the mean free path's and the
                          neutrinosphere's dependence on psi are held within an iteration).  Not
                          combined with the shock terms: EINVAL when prob->u is set */
} mgfld_step_opts;

/* Kernel categories of mgfld_step_opts.profile. */
enum {
  MGFLD_PROF_SETUP = 0,    /* frozen coefficients: groups, EoS, NES kernels, mean free path, limiter, shock terms */
  MGFLD_PROF_ASSEMBLE = 1, /* residual and Jacobian rows (k_assemble; in MIXED its first outer iteration) */
  MGFLD_PROF_FACTOR = 2,   /* block-Thomas elimination with in-block Gauss-Jordan (k_factor) */
  MGFLD_PROF_SOLVE = 3,    /* forward/back substitution (k_solve) */
  MGFLD_PROF_UPDATE = 4,   /* psi and Ye update, convergence bookkeeping (k_update_psi, k_update_ye, k_check) */
  MGFLD_PROF_FINISH = 5,   /* energy/temperature update and ledgers (k_finish, k_ledger) */
  MGFLD_PROF_RESIDUAL = 6, /* MIXED, later outer iterations: residual rows from the kept NES sums and the
                              last correction (k_resid_ff) */
  MGFLD_PROF_N = 7
};

/* Per-step report, DEVICE pointers (any may be NULL). */
typedef struct {
  int *iters;          /* [n_ray] outer iterations used */
  int *ray_status;     /* [n_ray] mgfld_status of each ray (OK, ENOCONV, ENAN) */
  double *ledger;      /* [n_ray][8]: lepton number before, after, lost through R_{I+1/2},
                          residual (after + lost - before); energy at infinity (MeV) before,
                          after, lost, residual (Eqs. a60-a62 with a62a, a62b) */
  double *heating;     /* [n_ray] MeV deposited in matter by nu_e + nubar_e between 100 and 300 km */
  int *factorizations; /* [n_ray] number of block factorisations performed */
  int *status;         /* [1] the step's status once it has run on the stream: the worst ray status
                          (ENAN before ENOCONV), ECUDA if a bounded wait of the substitution gave
                          up, else OK.  mgfld_step returns before the step has run, so this is
                          where a caller reads non-convergence (after synchronising the stream) */
} mgfld_step_report;

/* Bytes of workspace mgfld_step needs for these dimensions and precision. */
size_t mgfld_workspace_bytes(const mgfld_dims *dims, int precision);

/* Bytes of workspace mgfld_step needs when the problem carries the pair process (pair_coef set):
 * the coupled 2 n_e x 2 n_e blocks and the pair kernels of every zone.  0 for invalid dims or
 * n_e > 24. */
size_t mgfld_workspace_bytes_pair(const mgfld_dims *dims, int precision);

/*
 * mgfld_step -- one implicit transport step for all rays (Eqs. a58, a59, a62a
 * solved together; then Eqs. a62b and the EoS inversion for T).
 *   dims, prob, opts: as above (host structs holding device pointers).
 *   state: psi^n, Ye^n, T^n on entry; psi^{n+1}, Ye^{n+1}, T^{n+1} on exit.
 *   report: optional per-ray outputs (device); may be NULL.
 *   ws, ws_bytes: device workspace of at least mgfld_workspace_bytes() bytes
 *   (mgfld_workspace_bytes_pair() with the pair process), 256-byte aligned; its
 *   contents are scratch.
 * Asynchronous on `stream`: the whole step (set-up, outer iteration, finish) is
 * one CUDA graph launched on the stream, its outer iteration a device-side loop
 * (a while-conditional node whose condition the convergence test sets after each
 * iteration), so nothing waits on the host and the call returns before the step
 * has run.  The graph of each distinct set of arguments (pointers, sizes,
 * options) is built on its first call, with a CUDA graph capture on streams of
 * the library's own, and kept for the life of the process; that first call must
 * not be made while the calling thread is capturing.  The call returns OK,
 * EINVAL, ENOMEM or ECUDA (argument and launch errors); the per-ray statuses,
 * iteration counts and ledgers, and the step's worst status (report->status:
 * ENAN before ENOCONV, ECUDA if a bounded wait gave up) are written on the
 * stream.  Rays that fail keep their last iterate.
 * With opts->profile set the outer iteration runs from the host instead (one
 * stream synchronisation per iteration, for the per-category events) and the
 * call returns the worst ray status as well.
 */
mgfld_status mgfld_step(const mgfld_dims *dims, const mgfld_problem *prob, mgfld_state *state,
                        const mgfld_step_opts *opts, mgfld_step_report *report,
                        void *ws, size_t ws_bytes, void *stream);

/*
 * Linear block-tridiagonal system of one outer iteration, per (ray, species):
 *   sum_k' diag[i][k][k'] x[i][k'] + lower[i][k] x[i-1][k] + upper[i][k] x[i+1][k] = rhs[i][k]
 * (Eq. a62ae with the Ye column moved to the outer iteration; the off-diagonal
 * blocks are diagonal because the limited diffusion coefficient is held at
 * psi^n).  Layout (device, FP64 unless noted):
 *   diag  [n_ray][n_s][n_r][n_e][n_e]  row k = equation of group k (Eq. a58 units, 1/cm)
 *   lower [n_ray][n_s][n_r][n_e]       zero for i = 0 (zero central flux)
 *   upper [n_ray][n_s][n_r][n_e]       zero for i = n_r-1 (ghost folded into diag, Eq. a62af)
 *   rhs   [n_ray][n_s][n_r][n_e]       -G (Eq. a58 residual) at the linearisation point
 */
typedef struct { double *diag, *lower, *upper, *rhs; } mgfld_system;

/*
 * mgfld_assemble -- linearise the step at its starting state: builds the
 * frozen coefficients from (psi^n, Ye^n, T^n) and writes the Newton system of
 * the first outer iteration (psi = psi^n, Ye = Ye^n) into `sys`.
 *   state is read only.  ws: as for mgfld_step.
 */
mgfld_status mgfld_assemble(const mgfld_dims *dims, const mgfld_problem *prob, const mgfld_state *state,
                            mgfld_system *sys, void *ws, size_t ws_bytes, void *stream);

/* Bytes of the factor buffer for these dimensions and precision (FP64: 8 n_e^2
 * per block; MIXED: 4 n_e^2 per block). */
size_t mgfld_factor_bytes(const mgfld_dims *dims, int precision);

/*
 * mgfld_factor -- two-sided ("twisted") block-Thomas elimination of `sys` (partial
 * pivoting inside each block), run from both ends towards the middle zone
 * m = n_r / 2 so that the sequential chain along the zones is half as long: writes,
 * for every (ray, species, zone), into `factor` ([n_ray][n_s][n_r][n_e][n_e], FP64 or
 * FP32 by `precision`):
 *   i < m:  D'_i^{-1},  D'_0 = diag_0,  D'_i = diag_i - lower_i D'_{i-1}^{-1} upper_{i-1};
 *   i > m:  D''_i^{-1}, D''_{n_r-1} = diag_{n_r-1}, D''_i = diag_i - upper_i D''_{i+1}^{-1} lower_{i+1};
 *   i = m:  (diag_m - lower_m D'_{m-1}^{-1} upper_{m-1} - upper_m D''_{m+1}^{-1} lower_{m+1})^{-1}
 * (lower_i, upper_i act as diagonal matrices).  sys->rhs is not used.  A singular
 * pivot gives non-finite factors (detected later by mgfld_solve's caller, not here).
 */
mgfld_status mgfld_factor(const mgfld_dims *dims, const mgfld_system *sys, int precision,
                          void *factor, void *stream);

/*
 * mgfld_solve -- solve the factored system (mgfld_factor's layout) for one right-hand
 * side: g_i = D'^{-1}_i (rhs_i - lower_i g_{i-1}) for i < m and
 * g_i = D''^{-1}_i (rhs_i - upper_i g_{i+1}) for i > m; x_m from the middle inverse
 * applied to rhs_m - lower_m g_{m-1} - upper_m g_{m+1}; then outward
 * x_i = g_i - D'^{-1}_i (upper_i x_{i+1}) (i < m), x_i = g_i - D''^{-1}_i (lower_i x_{i-1})
 * (i > m).  rhs, x: [n_ray][n_s][n_r][n_e] FP64 (x may alias rhs).  With MIXED precision
 * the substitution runs in FP32 on a per-system power-of-two scaling of rhs.
 * sys->diag and sys->rhs are not used.
 */
mgfld_status mgfld_solve(const mgfld_dims *dims, const mgfld_system *sys, int precision,
                         const void *factor, const double *rhs, double *x, void *stream);

/* Capacity of the device scratch array used by mgfld_step_noalloc: 64 MiB per GPU. */
#define MGFLD_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/*
 * mgfld_step_noalloc -- mgfld_step without a caller workspace.  (The paper has no
 * counterpart; this is a packaging choice of this library.)
 *
 * For callers that cannot allocate device memory for the library: a host code that
 * links this solver as a black box and has no GPU allocator of its own, a process
 * whose device memory is reserved in full by another framework's pool, or a loop
 * that cannot afford the device synchronisation of cudaMalloc/cudaFree.  The step's
 * scratch is a fixed array of MGFLD_NOALLOC_SCRATCH_BYTES in the library's device
 * image, kept by every GPU that loads the library until the process exits; nothing is
 * allocated or freed by this call, and no CUDA graph is created: the outer iteration runs
 * from the host (one stream synchronisation per iteration) and the call returns the worst
 * ray status, as mgfld_step does with profiling.  Inputs and outputs are the caller's, as
 * for mgfld_step.
 *   - Returns MGFLD_ENOMEM, before touching the GPU, when the step's workspace
 *     (mgfld_workspace_bytes, or mgfld_workspace_bytes_pair with the pair process) exceeds
 *     MGFLD_NOALLOC_SCRATCH_BYTES (at 512 zones x 20 groups: more than 2 rays in FP64, more
 *     than 3 in MIXED); split the rays into several calls.
 *   - Returns MGFLD_EINVAL if opts->profile is set (timing would create CUDA events).
 *   - Every call looks up the array's device address on the current device (nothing is
 *     cached, so a context reset between calls is harmless); the first call on a device
 *     also loads the library's device code there, so make it before any stream capture
 *     begins.
 *   - All calls on a device share the one array: calls that may overlap on the GPU
 *     (other streams, other host threads) race and must be serialised by the caller.
 *     Each call rewrites every part of the scratch it reads, so the contents left by
 *     a previous call never leak into a result.
 */
mgfld_status mgfld_step_noalloc(const mgfld_dims *dims, const mgfld_problem *prob, mgfld_state *state,
                                const mgfld_step_opts *opts, mgfld_step_report *report, void *stream);

/*
 * Discrete adjoint of one step (FP64).  The paper has no adjoint; it is the exact
 * derivative of the discrete step defined by Eqs. a58, a59, a62a, a62b with the
 * coefficients frozen at the start of the step (Eqs. a17, a20-a26a, a55, a62af, d7, d8).
 *
 * For a step p = (psi^n, Ye^n, T^n, scale) -> (psi^{n+1}, Ye^{n+1}, T^{n+1}, H), where
 * H[ray] is the heating of mgfld_step_report, and a scalar loss
 *   L = <psi_bar, psi^{n+1}> + <ye_bar, Ye^{n+1}> + <T_bar, T^{n+1}> + heat_weight sum(H),
 * mgfld_adjoint writes dL/dpsi^n, dL/dYe^n, dL/dT^n and adds dL/dscale.  The root
 * (psi^{n+1}, Ye^{n+1}) is the caller's (normally mgfld_step's output); the
 * implicit-function theorem turns the root condition G(x; p) = 0 into one
 * transposed solve J^T mu = dL/dx, J = dG/dx at the root, done by block
 * Gauss-Seidel between psi (block-Thomas on the transposed per-species system) and
 * Ye (zone-local), then p_bar = dL/dp - mu^T dG/dp.  T^{n+1} enters L through
 * Eq. a62b and the EoS inversion.  All pointers are DEVICE pointers; inputs (the
 * *_bar arrays) may be NULL for zero.  Shapes as the state arrays; scale_bar is
 * [n_s][n_e] and may be NULL (no scale gradient).
 */
typedef struct {
  const double *psi_bar, *ye_bar, *T_bar; /* dL/d(psi, Ye, T)^{n+1}, or NULL */
  double heat_weight;                     /* weight of sum(H) in L */
  double *psi_bar_out, *ye_bar_out, *T_bar_out; /* dL/d(psi, Ye, T)^n (overwritten; required) */
  double *scale_bar;                      /* dL/dscale is ADDED here, or NULL */
  int max_sweeps;                         /* Gauss-Seidel sweeps at most (0: 30) */
  double sweep_tol;                       /* stop when max|d mu_Ye| <= sweep_tol max|mu_Ye| (0: 1e-15) */
  int sweeps_used;                        /* out (host): sweeps performed */
  double sweep_change;                    /* out (host): relative mu_Ye change of the last sweep */
} mgfld_adjoint_io;

/* Bytes of workspace mgfld_adjoint needs (0 for invalid dims). */
size_t mgfld_adjoint_workspace_bytes(const mgfld_dims *dims);

/*
 * mgfld_adjoint -- reverse of one mgfld_step.
 *   prob: the step's problem (prob->scale as used in the step, or NULL for ones).
 *   state_n: (psi^n, Ye^n, T^n), the step's input.  state_np1: psi^{n+1}, Ye^{n+1}
 *   (T is not read).  ws: device workspace, 256-byte aligned, of at least
 *   mgfld_adjoint_workspace_bytes(); scratch.
 * Synchronises `stream` once per Gauss-Seidel sweep (the stopping test).
 * Returns OK, EINVAL (bad argument, psi_bar_out/ye_bar_out/T_bar_out missing),
 * ENOMEM (workspace too small), ENOCONV (the sweeps did not reach sweep_tol; the
 * outputs hold the last sweep's gradients), ENAN (a non-finite sweep change) or ECUDA.
 */
mgfld_status mgfld_adjoint(const mgfld_dims *dims, const mgfld_problem *prob, const mgfld_state *state_n,
                           const mgfld_state *state_np1, mgfld_adjoint_io *io, void *ws, size_t ws_bytes,
                           void *stream);

/* ----------------------------------------------------------------------------------------------
 * Energy advection (Sec. "Neutrino Energy Advection Step", Eqs. a78-a81d; the remap of App.
 * "Neutrino Energy Advection due to Changes in the Lapse", Eqs. p5-p8; the PPM interpolation of
 * Sec. "PPM Interpolation Scheme", Eqs. h9-h17, h22-h24, h31-h35, Cartesian form; the Minerbo
 * closure, Eqs. a86-a87).  The step that follows the transport step in the operator split: after a
 * hydrodynamics step changed rho, R and the lapse a of each zone, the occupations psi0 of each
 * (ray, species, zone) are
 *   1. shifted in energy (Eqs. a78-a80): every group edge E_{k+-1/2} moves by the factor
 *      1 + (da/a - dR/R) - (db/b - dR/R) eta2, b = 1/(4 pi R^2 rho), eta2 the Minerbo Eddington
 *      factor of the flux factor eta1 at the edge (mean of the two adjacent groups), with the
 *      neutrino number of every group kept (psi scaled by (rho a^3)^{n+1}/(rho a^3)^n x
 *      (E^2 dE)^n / (E^2 dE)^{shifted});
 *   2. remapped back to the grid E_{k+-1/2} / a^{n+1} (Eq. a81, p1): parabolic profiles of
 *      eps^2 psi over the shifted groups, the number in each slice swept across a target edge
 *      as the flux (zero at the lowest and highest edge, Eq. p5), all fluxes of the system
 *      scaled by one factor xi that keeps the energy (Eqs. p6-p8; xi = 1 without flux);
 *   3. optionally limited to psi <= 1 (Eqs. a81a-a81d), in increasing group order, moving the
 *      excess of group k to k+1 and k+2 with number and energy kept.
 * Neutrino number per comoving mass is conserved exactly; the remap conserves energy exactly.
 * The swept fraction of a group is clamped to [0, 1] (edges are assumed to move by less than a
 * group width in one step).
 * -------------------------------------------------------------------------------------------- */
typedef struct {
  const double *r_edge_n, *r_edge_np1;   /* [n_ray][n_r+1] areal radii of the zone edges before /
                                            after (cm); the zone's R is the mean of its edges */
  const double *rho_n, *rho_np1;         /* [n_ray][n_r] density before / after (g/cm^3) */
  const double *lapse_n, *lapse_np1;     /* [n_ray][n_r] lapse before / after, or NULL (= 1) */
  const double *e_edge;                  /* [n_e+1] group edges at infinity (MeV), increasing */
  const double *eta1;                    /* [n_ray][n_s][n_r][n_e] flux factors psi1/psi0 (clamped
                                            to [0, 1]), or NULL: eta2 = 1/3 (diffusion limit) */
  int limit;                             /* nonzero: apply step 3 */
  const double *u;                       /* [n_ray][n_r] zone-centred fluid velocity (cm/s), or NULL.
                                            At a shock the shock-transport terms of mgfld_problem.u
                                            replace energy advection: zone i's displacement (Eq.
                                            a79) is scaled by 1 - max(w_{i-1/2}, w_{i+1/2}), w the
                                            roll-in weights of its edges (0 at |u_{i+1} - u_i| =
                                            0.01c, 1 at 0.02c); the number factor of Eq. a78 stays */
} mgfld_eadv_problem;

/*
 * mgfld_energy_advect -- one energy-advection step, in place on psi [n_ray][n_s][n_r][n_e]
 * (device, FP64; n_s = 4, 3 <= n_e <= 32).  xi (device, [n_ray][n_s][n_r], or NULL) receives the
 * energy-fixing factor of each system.  All pointers are caller-owned device memory; no
 * workspace.  Asynchronous on `stream`.  Returns OK, EINVAL (bad dims or a required pointer
 * missing) or ECUDA (launch error).
 */
mgfld_status mgfld_energy_advect(const mgfld_dims *dims, const mgfld_eadv_problem *prob, double *psi,
                                 double *xi, void *stream);

/*
 * Neutrino stress and lapse update (Sec. "Solution of the Transport Equations", Eqs. a62e-a62l).
 *   p        [n_ray][n_r] matter pressure at zone centres (erg/cm^3); required when lapse is set.
 *   m_inner  [n_ray] rest mass inside the innermost edge R_{1/2} (g), or NULL for 0.
 *   f_edge   [n_ray][n_r] out: the stress (force per unit mass on the matter, cm/s^2, outward
 *            positive) at each zone's outer edge, Eq. a62e with the difference of Eq. a62f; the
 *            outermost edge uses the transport's ghost zone (Eq. a62af), none with a reflecting
 *            edge.  Or NULL.
 *   f_zone   [n_ray][n_r] out: the zone value, the mean of its two edges (Eq. a62i; the centre
 *            edge carries none), or NULL.
 *   lapse    [n_ray][n_r] out: the lapse at zone centres, Eqs. a62k-a62l: the exterior
 *            sqrt(1 - 2 G M / (c^2 R_{I+1/2})) of the enclosed rest mass M = m_inner + sum rho V in
 *            the last zone, then inward a_i = a_{i+1} exp[(p_{i+1} - p_i - Delta M_{i+1/2}
 *            f_{i+1/2} / (4 pi R_{i+1/2}^2)) / (rho_{i+1/2} c^2)] (edge values the means of the two
 *            zones), or NULL.
 * All device pointers, caller-owned.
 */
typedef struct {
  const double *p;
  const double *m_inner;
  double *f_edge, *f_zone, *lapse;
} mgfld_stress_io;

/*
 * mgfld_stress_lapse -- the neutrino stress of the state (psi, Ye, T) of problem `prob` and the
 * lapse it supports.  The flux limiter F^{n+1} of Eq. a62e is evaluated at this state with the
 * transport step's own coefficients (mean free path, neutrinosphere, ghost factor); energies are
 * each zone's comoving group energies E/a (prob->lapse is the lapse the state was computed on).
 * prob->u is ignored.  ws: at least mgfld_workspace_bytes(dims, MGFLD_FP64) bytes, 256-byte
 * aligned, scratch.  Asynchronous on `stream`.  Returns OK, EINVAL (bad arguments, or lapse
 * without p), ENOMEM (workspace too small) or ECUDA.
 */
mgfld_status mgfld_stress_lapse(const mgfld_dims *dims, const mgfld_problem *prob, const mgfld_state *state,
                                const mgfld_stress_io *io, void *ws, size_t ws_bytes, void *stream);

/* Human-readable name of a status code (static string). */
const char *mgfld_status_str(mgfld_status s);

/*
 * mgfld_arith_check -- self-check of the FP64 arithmetic the kernels use in place of FP64
 * divisions and comparisons (no paper counterpart; a diagnostic).  For i < count, with x = a[i],
 * y = b[i], writes out[8 i + 0..7] = the library's quotient x / y (a reciprocal seeded on the
 * integer and FP32 pipes with one Newton correction of the quotient), CUDA's x / y, the library's
 * reciprocal of y with two Newton steps, CUDA's 1 / y, the one-step reciprocal seed (~2^-46
 * relative), the integer-pipe comparison x < y by order keys (1 or 0), CUDA's x < y (1 or 0), and
 * the integer-pipe test x == 0 (1 or 0).  a, b: count device doubles; out: 8 count device doubles;
 * all caller-owned.  Asynchronous on `stream`.  Returns OK, EINVAL (count < 0 or a NULL pointer
 * with count > 0) or ECUDA.
 */
mgfld_status mgfld_arith_check(const double *a, const double *b, int count, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MGFLD_H */
