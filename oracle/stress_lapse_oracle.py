"""CPU oracle of the neutrino stress and the lapse update (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import this module; the
product path never does.  FP64 numpy, written from the paper's equations in their order
(Sec. "Solution of the Transport Equations", after the energy equation):

  * the neutrino stress (force per unit mass on the matter) at every zone edge, Eq. a62e: the
    gradient of eps^3 d eps psi0 weighted by the flux limiter, differenced over the edge mass as
    Eq. a62f prescribes, summed over groups and species with the statistical weights; its zone
    value is the mean of the two edge values, Eq. a62i;
  * the lapse, Eqs. a62k-a62l: the exterior value at the outer edge from the enclosed rest mass,
    then inward zone by zone, a_i = a_{i+1} exp[(p_{i+1} - p_i - stress term) / (rho c^2)].

Readings (the GPU path takes the same ones):
  L1  Eq. a62l's stress term is the force per unit area Delta M_{i+1/2} f_{i+1/2} / (4 pi R^2):
      the printed extra 1/rho_{i+1/2} leaves the bracket with two different units (a pressure
      difference minus an acceleration times a length); with rho Delta R = Delta M / (4 pi R^2)
      the bracket is the integral of dp/dR - rho f over the zone spacing, as Eq. a46 requires.
  L2  Eq. a62k is printed without its square root: a = sqrt(1 - 2 G M / (c^2 R)) (the exterior
      Schwarzschild lapse; the paper's lapse test, Eq. t1, uses the root).
  L3  The inward scan starts at the last zone with a_I = a_{I+1/2}: no pressure or stress
      difference enters across the outer edge.
  L4  F^{n+1} in Eq. a62e is the flux limiter evaluated at the state passed in (the end-of-step
      psi, Ye, T), with lambda, R_nu and the ghost factor as the transport step forms them
      (readings R2-R5 applied to that state); the limiter value is min(F_intrp, F_geom).
  L5  The outermost edge uses the transport's ghost zone (Eq. a62af): psi_{I+1} = g psi_I,
      Delta M_{I+1} = Delta M_I, a_{I+1} = a_I; with a reflecting outer edge it carries no
      stress; the centre edge carries none (zero flux there).
  L6  M_{I+1/2} = M_inner + sum_i rho_i V_i (Eq. a62k's text sets M_g to the rest mass; M_inner,
      the mass inside the innermost edge, is an input); rho_{i+1/2} and p_{i+1/2} are arithmetic
      means of the two zones (text after Eq. a62l), Delta M_{i+1/2} = (Delta M_i + Delta M_{i+1})/2.
  L7  eps_k^3 Delta eps_k of zone i is taken on its comoving grid E / a_i (centres of Eq. a01b),
      in erg (MeV x 1.602176634e-6), so that the stress is in cm/s^2 with p in erg/cm^3.
"""
import numpy as np

from oracle import mgfld_oracle as O

G_NEWTON = 6.67430e-8            # cm^3 g^-1 s^-2
MEV_ERG = 1.602176634e-6


def edge_stress(f, psi, F):
    """f_{nu,r} at the outer edge of every zone, Eq. a62e (readings L4, L5, L7), [n_ray, n_r].

    f: the oracle's frozen coefficients of the state (setup_step); psi [n_ray, 4, n_r, n_e];
    F [n_ray, 4, n_r, n_e] the flux limiter at each zone's outer edge."""
    X = (f.eps**3 * f.deps)[:, None] * psi * MEV_ERG             # eps^3 d eps psi0 (erg)
    X_r = np.empty_like(X)
    X_r[:, :, :-1] = X[:, :, 1:]
    X_r[:, :, -1] = f.ghost * X[:, :, -1]                         # L5
    dM = f.rho * f.vol
    dM_e = np.empty_like(dM)
    dM_e[:, :-1] = 0.5 * (dM[:, :-1] + dM[:, 1:])
    dM_e[:, -1] = dM[:, -1]
    Fw = np.array(F, dtype=np.float64, copy=True)
    if f.outer_bc == O.BC_REFLECT:
        Fw[:, :, -1, :] = 0.0
    s = np.einsum('q,rqik->ri', O.STAT_WEIGHT, Fw * (X_r - X))
    return -O.FOUR_PI_HC3 / 3.0 * s * f.area[:, 1:] / dM_e


def zone_stress(f_edge):
    """Eq. a62i: the mean of the two edge values; the centre edge carries none (L5)."""
    inner = np.zeros_like(f_edge)
    inner[:, 1:] = f_edge[:, :-1]
    return 0.5 * (f_edge + inner)


def lapse(r_edge, rho, vol, p, f_edge, m_inner):
    """Eqs. a62k-a62l (readings L1-L3, L6): the lapse at zone centres, [n_ray, n_r]."""
    r_edge = np.asarray(r_edge, dtype=np.float64)
    n_ray, n_r = rho.shape
    dM = rho * vol
    M = np.asarray(m_inner, dtype=np.float64) + np.sum(dM, axis=1)
    R_out = r_edge[:, -1]
    a = np.empty((n_ray, n_r))
    a[:, -1] = np.sqrt(1.0 - 2.0 * G_NEWTON * M / (O.C_LIGHT**2 * R_out))
    for i in range(n_r - 2, -1, -1):
        rho_e = 0.5 * (rho[:, i] + rho[:, i + 1])
        dM_e = 0.5 * (dM[:, i] + dM[:, i + 1])
        Re = r_edge[:, i + 1]
        bracket = p[:, i + 1] - p[:, i] - dM_e / (4.0 * np.pi * Re * Re) * f_edge[:, i]
        a[:, i] = a[:, i + 1] * np.exp(bracket / (rho_e * O.C_LIGHT**2))
    return a


def stress_and_lapse(prob, psi, ye, T, p, m_inner):
    """The neutrino stress (edges and zones) and the new lapse for the state (psi, Ye, T) of
    problem `prob` (the transport step's problem dict), matter pressure p [n_ray, n_r] (erg/cm^3)
    and the mass inside the innermost edge m_inner [n_ray] (g).  Returns a dict."""
    f = O.setup_step(prob, psi, ye, T)
    fe = edge_stress(f, np.asarray(psi, dtype=np.float64), f.F)
    return dict(f_edge=fe, f_zone=zone_stress(fe),
                lapse=lapse(f.r_edge, f.rho, f.vol, np.asarray(p, dtype=np.float64), fe, m_inner))
