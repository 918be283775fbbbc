"""CPU oracle of the neutrino energy-advection step (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import this module; the
product path never does.  FP64 numpy, written from the paper's equations in their order:

  * Minerbo closure for the scalar Eddington factor eta2(eta1), Eqs. a86-a87;
  * step 1, the Lagrangian shift of the energy grid driven by the changes of the lapse a, the
    areal radius R and b = 1/(4 pi R^2 rho), Eqs. a78-a80 (number-conserving, Eq. a74);
  * step 2, the remap of the displaced grid back to the grid tied to the new lapse (Eq. a81):
    piecewise parabolic profiles of eps^2 psi in energy (Eqs. h9-h17, h22-h24, h31-h35 in their
    Cartesian form), fluxes of the swept slices across the target edges (Eq. p5), scaled by one
    factor xi per (ray, species, zone) that restores the energy (Eqs. p6-p8);
  * step 3, the occupation limiter psi <= 1 (Eqs. a81a-a81d).

Readings (the paper is silent or garbled here; the GPU path takes the same ones):
  E1  Each group edge E_{k+-1/2} moves by the factor of Eq. a79 evaluated with eta2 at the edge:
      the mean of the two adjacent groups' eta2 (the end edges take their group's), so that the
      displaced groups still partition the energy axis; the centres follow from the displaced
      edges by Eq. a01b.  Eq. a79's printed first-order form is used as is.
  E2  Energies are comoving, eps = E / a; the displaced grid lives at the new lapse (Eq. a80), the
      target grid is E_{k+-1/2} / a^{n+1} (Eq. p1).
  E3  PPM in energy is the Cartesian form (dV/d eps = 1) applied to the cell averages
      a_k = eps_k^2 psi_k (number per unit energy, Eq. a01b); two ghost groups at each end copy
      the end group's average and width (zero slope).
  E4  Fluxes at the lowest and highest edge are zero (Eq. p5); a slice swept across an interior
      edge is integrated over the parabola of the group it came from; the swept fraction of a
      group is clamped to [0, 1] (the step assumes edges move by less than a group).
  E5  xi = (E_before - sum_k n'_k eps_k) / sum_k (F_{k-1/2} - F_{k+1/2}) eps_k, the energy
      balance of Eq. p7 solved with the sum over k that the printed Eq. p8 drops; xi = 1 when the
      denominator vanishes (no flux).
  E6  The limiter runs k = 0 .. N-3 (0-based: every group that has two groups above it), in
      increasing k, with Eq. a81c/a81d's coefficients on the target grid, and acts only on an
      overfilled group; a removal that would drive psi_{k+2} below zero is scaled down to empty
      it exactly (no removal when psi_{k+2} <= 0).
  E7  eta1 (the flux factor psi1/psi0) is an input, clamped to [0, 1]; absent, eta2 = 1/3.
  E8  At a shock the shock-transport terms take over from energy advection (Sec. "Transport
      through a Shock": rolled in as energy advection is rolled out): zone i's displacement in
      Eq. a79 is scaled by 1 - max(w_{i-1/2}, w_{i+1/2}), w the roll-in weights of its two edges
      (mgfld_oracle.shock_beta); Eq. a78's number factor is kept, so number is still conserved.
"""
import numpy as np

FOUR_PI = 4.0 * np.pi


def minerbo_eta2(eta1):
    """Scalar Eddington factor of the Minerbo closure, Eqs. a86-a87 (eta2_thick = 1/3,
    eta2_thin = 1)."""
    x = np.clip(np.asarray(eta1, dtype=np.float64), 0.0, 1.0)
    p = 1.0 / 3.0 + 2.0 * x * x / 15.0 * (3.0 - x + 3.0 * x * x)
    return 1.5 * (1.0 - p) * (1.0 / 3.0) + 0.5 * (3.0 * p - 1.0) * 1.0


def cube_moment(lo, hi):
    """eps_k^2 d eps_k = (eps_+^3 - eps_-^3) / 3 (Eq. a01b / Eq. p4 without its 4 pi)."""
    return (hi * hi * hi - lo * lo * lo) / 3.0


def group_centres(lo, hi):
    """eps_k from Eq. a01b: eps_k^2 (hi - lo) = (hi^3 - lo^3) / 3."""
    return np.sqrt((hi * hi + hi * lo + lo * lo) / 3.0)


def edge_eddington(eta2):
    """Reading E1: eta2 at the N + 1 edges from the N groups (last axis)."""
    n = eta2.shape[-1]
    out = np.empty(eta2.shape[:-1] + (n + 1,))
    out[..., 0] = eta2[..., 0]
    out[..., n] = eta2[..., n - 1]
    out[..., 1:n] = 0.5 * (eta2[..., :-1] + eta2[..., 1:])
    return out


def shock_keep(u):
    """Reading E8: the fraction 1 - max(w_{i-1/2}, w_{i+1/2}) of the displacement kept in each
    zone, [n_ray, n_r], from zone-centred velocities u [n_ray, n_r]."""
    from oracle.mgfld_oracle import shock_beta
    _, w = shock_beta(u)
    lo = np.zeros(np.shape(u))
    hi = np.zeros(np.shape(u))
    lo[:, 1:] = w
    hi[:, :-1] = w
    return 1.0 - np.maximum(lo, hi)


def lagrangian_shift(e_edge, a_n, a_np1, r_n, r_np1, rho_n, rho_np1, eta2, psi, keep=None):
    """Step 1, Eqs. a78-a80, for systems along the leading axes and groups on the last axis.

    e_edge [N+1] are the group edges at infinity (MeV); a, r (zone-centre areal radius) and rho
    carry one value per system (broadcast over groups); eta2 and psi are [..., N].
    Returns (eps_d [..., N+1] displaced comoving edges, psi_d [..., N] occupation on them,
    nd [..., N] = psi_d eps_d-weights, i.e. the number per unit volume V^{n+1} per group)."""
    a_n, a_np1, r_n, r_np1, rho_n, rho_np1 = (np.asarray(v, dtype=np.float64)[..., None]
                                             for v in (a_n, a_np1, r_n, r_np1, rho_n, rho_np1))
    b_n = 1.0 / (FOUR_PI * r_n * r_n * rho_n)
    b_np1 = 1.0 / (FOUR_PI * r_np1 * r_np1 * rho_np1)
    da_a = (a_np1 - a_n) / a_n
    dr_r = (r_np1 - r_n) / r_n
    db_b = (b_np1 - b_n) / b_n
    # Eq. a79 at the edges (reading E1), rolled out at a shock (reading E8)
    disp = (da_a - dr_r) - (db_b - dr_r) * edge_eddington(eta2)
    if keep is not None:
        disp = np.asarray(keep, dtype=np.float64)[..., None] * disp
    s = 1.0 + disp
    E = np.broadcast_to(np.asarray(e_edge, dtype=np.float64), s.shape)
    E_d = s * E
    # Eq. a78: (rho a^3)^{n'+1} / (rho a^3)^n x (E^2 dE)^n / (E^2 dE)^{n'+1}, the group moments
    # E_k^2 dE_k of Eq. a01b on the group's own edges
    w_E_n = cube_moment(E[..., :-1], E[..., 1:])
    w_E_d = cube_moment(E_d[..., :-1], E_d[..., 1:])
    psi_d = (rho_np1 * a_np1 ** 3) / (rho_n * a_n ** 3) * (w_E_n / w_E_d) * psi
    # Eq. a80: comoving energies at the new lapse
    eps_d = E_d / a_np1
    nd = psi_d * cube_moment(eps_d[..., :-1], eps_d[..., 1:])
    return eps_d, psi_d, nd


def _with_ghosts(v):
    """Two ghost cells at each end of the last axis, copies of the end cells (reading E3)."""
    return np.concatenate([v[..., :1], v[..., :1], v, v[..., -1:], v[..., -1:]], axis=-1)


def ppm_profile(a, dxi):
    """Piecewise parabolic profiles of the cell averages a [..., N] on cells of widths dxi
    (Cartesian form): the average slopes (Eq. h9) monotonised (Eq. h11), the interface values
    of the cubic interpolating the cell integrals (Eq. h12, read as Colella & Woodward's Eq. 1.6,
    of which the printed one is a garbled copy) limited to the range of the two neighbours
    (Eqs. h15-h17), the parabola coefficients (Eqs. h22-h24) and the monotonicity corrections
    (Eqs. h31-h35).  Returns (aL, aR, a6), each [..., N]."""
    n = a.shape[-1]
    A = _with_ghosts(a)                  # A[j + 2] = a_j
    X = _with_ghosts(dxi)
    m = n + 4
    # Eq. h10 at the interfaces j - 1/2, j = 1..m-1 (extended indices)
    dA = A[..., 1:] - A[..., :-1]        # dA[j - 1] = A_j - A_{j-1}
    # Eq. h9 and h11 for extended cells j = 1..m-2
    da = np.zeros_like(A)
    dm = np.zeros_like(A)
    for j in range(1, m - 1):
        xl, x0, xr = X[..., j - 1], X[..., j], X[..., j + 1]
        dp, dn = dA[..., j], dA[..., j - 1]          # a_{j+1} - a_j, a_j - a_{j-1}
        s = x0 / (xl + x0 + xr) * ((2.0 * xl + x0) / (xr + x0) * dp + (x0 + 2.0 * xr) / (xl + x0) * dn)
        da[..., j] = s
        lim = np.minimum(np.abs(s), np.minimum(2.0 * np.abs(dp), 2.0 * np.abs(dn))) * np.sign(s)
        dm[..., j] = np.where(dp * dn > 0.0, lim, 0.0)
    # Eq. h12 at the interfaces j + 1/2 between extended cells j and j + 1, j = 1..m-3
    face = np.zeros(A.shape[:-1] + (m,))
    for j in range(1, m - 2):
        xl, x0, x1, x2 = X[..., j - 1], X[..., j], X[..., j + 1], X[..., j + 2]
        d = A[..., j + 1] - A[..., j]
        tot = xl + x0 + x1 + x2
        t = (2.0 * x1 * x0 / (x0 + x1)) * ((xl + x0) / (2.0 * x0 + x1) - (x2 + x1) / (2.0 * x1 + x0)) * d
        t = t - x0 * (xl + x0) / (2.0 * x0 + x1) * dm[..., j + 1] + x1 * (x1 + x2) / (x0 + 2.0 * x1) * dm[..., j]
        f = A[..., j] + x0 / (x0 + x1) * d + t / tot
        # Eqs. h15-h16: within the range of the two neighbouring averages
        f = np.maximum(f, np.minimum(A[..., j], A[..., j + 1]))
        f = np.minimum(f, np.maximum(A[..., j], A[..., j + 1]))
        face[..., j] = f
    # real cell i = extended j = i + 2: left face at j - 1 (face index j - 1), right face at j
    aR = face[..., 2:n + 2]
    aL = face[..., 1:n + 1]              # Eq. h17: a_L of cell i = a_R of cell i - 1
    # Eqs. h23-h24 and the monotonicity corrections h31-h35 (Cartesian forms)
    dA_c = aR - aL
    a6 = 6.0 * (a - 0.5 * (aL + aR))
    left_mon = dA_c * dA_c < dA_c * a6
    right_mon = dA_c * dA_c < -dA_c * a6
    aL2 = np.where(left_mon, 3.0 * a - 2.0 * aR, aL)
    aR2 = np.where(right_mon, 3.0 * a - 2.0 * aL, aR)
    a6 = 6.0 * (a - 0.5 * (aL2 + aR2))
    return aL2, aR2, a6


def parabola_average_right(aL, aR, a6, y):
    """Average of the parabola of Eq. h22 over the rightmost fraction y of its cell."""
    return aR - 0.5 * y * ((aR - aL) - (1.0 - 2.0 * y / 3.0) * a6)


def parabola_average_left(aL, aR, a6, y):
    """Average of the parabola of Eq. h22 over the leftmost fraction y of its cell."""
    return aL + 0.5 * y * ((aR - aL) + (1.0 - 2.0 * y / 3.0) * a6)


def remap_fluxes(eps_d, eps_t, aL, aR, a6):
    """Fluxes F_{k+1/2} [..., N+1] of Eq. p5: the number in the slice between the displaced edge
    eps_d and the target edge eps_t, counted from group k to group k+1, integrated over the
    parabola of the group the slice belongs to (reading E4; zero at the two outer edges)."""
    n = aL.shape[-1]
    dx = eps_d[..., 1:] - eps_d[..., :-1]
    F = np.zeros(eps_d.shape)
    for j in range(1, n):
        d = eps_t[..., j] - eps_d[..., j]          # target edge minus displaced edge
        # d < 0: slice [eps_t, eps_d] is the top of group j - 1 and moves up into target j
        yl = np.clip(-d / dx[..., j - 1], 0.0, 1.0)
        up = parabola_average_right(aL[..., j - 1], aR[..., j - 1], a6[..., j - 1], yl) * yl * dx[..., j - 1]
        # d > 0: slice [eps_d, eps_t] is the bottom of group j and moves down into target j - 1
        yr = np.clip(d / dx[..., j], 0.0, 1.0)
        down = parabola_average_left(aL[..., j], aR[..., j], a6[..., j], yr) * yr * dx[..., j]
        F[..., j] = np.where(d < 0.0, up, np.where(d > 0.0, -down, 0.0))
    return F


def energy_fix(nd, epsc_d, epsc_t, F):
    """xi of Eqs. p6-p8 (reading E5): the factor on the flux divergence that makes
    sum_k n_k eps_k on the target grid equal the energy sum_k n'_k eps'_k before the remap."""
    div = F[..., :-1] - F[..., 1:]                     # F_{k-1/2} - F_{k+1/2}
    e_before = np.sum(nd * epsc_d, axis=-1)
    s1 = np.sum(nd * epsc_t, axis=-1)
    s2 = np.sum(div * epsc_t, axis=-1)
    safe = np.where(s2 != 0.0, s2, 1.0)
    return np.where(s2 != 0.0, (e_before - s1) / safe, 1.0), div


def limit_occupation(psi, epsc, deps):
    """Step 3, Eqs. a81a-a81d (reading E6), on groups with centres epsc and widths deps."""
    psi = np.array(psi, dtype=np.float64, copy=True)
    w = epsc * epsc * deps
    n = psi.shape[-1]
    for k in range(n - 2):
        e0, e1, e2 = epsc[..., k], epsc[..., k + 1], epsc[..., k + 2]
        c_up = (e2 - e0) * w[..., k] / ((e2 - e1) * w[..., k + 1])          # Eq. a81c
        c_dn = (e1 - e0) * w[..., k] / ((e2 - e1) * w[..., k + 2])          # Eq. a81d
        d = np.maximum(psi[..., k] - 1.0, 0.0)
        # a removal from k + 2 larger than its (non-negative part of the) content is scaled down
        # to empty it; groups that are not overfilled are left alone
        d = np.minimum(d, np.maximum(psi[..., k + 2], 0.0) / c_dn)
        psi[..., k] -= d
        psi[..., k + 1] += c_up * d
        psi[..., k + 2] -= c_dn * d
    return psi


def step(e_edge, a_n, a_np1, r_n, r_np1, rho_n, rho_np1, psi, eta1=None, limit=True, keep=None):
    """One energy-advection step (Sec. "Neutrino Energy Advection Step"): psi [..., N] on the grid
    E / a^n in, psi on the grid E / a^{n+1} out.  The zone quantities (a, r, rho, and keep, the
    displacement fraction of reading E8) have the shape of psi without its last axis.
    Returns dict(psi, xi, psi_d, eps_d, eps_t, F)."""
    psi = np.asarray(psi, dtype=np.float64)
    eta2 = np.full(psi.shape, 1.0 / 3.0) if eta1 is None else minerbo_eta2(eta1)
    eps_d, psi_d, nd = lagrangian_shift(e_edge, a_n, a_np1, r_n, r_np1, rho_n, rho_np1, eta2, psi, keep)
    a_np1b = np.asarray(a_np1, dtype=np.float64)[..., None]
    eps_t = np.broadcast_to(np.asarray(e_edge, dtype=np.float64), eps_d.shape) / a_np1b
    dxd = eps_d[..., 1:] - eps_d[..., :-1]
    epsc_d = group_centres(eps_d[..., :-1], eps_d[..., 1:])
    aL, aR, a6 = ppm_profile(nd / dxd, dxd)           # cell averages eps^2 psi (reading E3)
    F = remap_fluxes(eps_d, eps_t, aL, aR, a6)
    epsc_t = group_centres(eps_t[..., :-1], eps_t[..., 1:])
    xi, div = energy_fix(nd, epsc_d, epsc_t, F)
    n_new = nd + xi[..., None] * div                  # Eq. p6
    psi_new = n_new / cube_moment(eps_t[..., :-1], eps_t[..., 1:])
    if limit:
        psi_new = limit_occupation(psi_new, epsc_t, eps_t[..., 1:] - eps_t[..., :-1])
    return dict(psi=psi_new, xi=xi, psi_d=psi_d, eps_d=eps_d, eps_t=eps_t, F=F)


def number_energy(psi, e_edge, a):
    """Number and energy per unit volume, sum_k psi eps_k^2 d eps_k and the same weighted by
    eps_k (Eqs. p2-p4 without the common factors), on the grid E / a."""
    a = np.asarray(a, dtype=np.float64)[..., None]
    eps = np.broadcast_to(np.asarray(e_edge, dtype=np.float64), np.shape(psi)[:-1] + (len(e_edge),)) / a
    w = cube_moment(eps[..., :-1], eps[..., 1:])
    c = group_centres(eps[..., :-1], eps[..., 1:])
    return np.sum(psi * w, axis=-1), np.sum(psi * w * c, axis=-1)
