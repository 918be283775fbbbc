"""Small hand-built transport problems for pins and parity tests (inputs only)."""
import numpy as np

from paper_1809_05608_gb300 import problems


def strong(n_ray=2, n_r=8, n_e=5, kabs=1e16, kscat=1e14, nes=1.0, lapse=False, config=2,
           bc=0, dt=1e-6, pair=0.0):
    """The synthetic profile at reduced size with opacities scaled up so that
    absorption/emission, scattering and NES all matter within one step; pair > 0 adds the
    synthetic pair process with the annihilation kernel pair x 1e-41 rho (cm^3/s)."""
    inp = problems.make_problem(config, n_ray=n_ray, n_r=n_r, n_e=n_e)
    p = dict(inp['problem'])
    p['kappa_abs'] = p['kappa_abs'] * kabs
    p['kappa_scat'] = p['kappa_scat'] * kscat
    p['nes_coef'] = p['nes_coef'] * nes
    p['outer_bc'] = bc
    p['dt'] = dt
    if pair > 0.0:
        p['pair_coef'] = 1e-41 * pair * p['rho']
    if lapse:
        rc = 0.5 * (p['r_edge'][:, 1:] + p['r_edge'][:, :-1])
        p['lapse'] = np.sqrt(1.0 - 0.2 * rc[:, :1] / rc)   # 0.89 .. 1, varies along the ray
    inp = dict(inp)
    inp['problem'] = p
    return inp


def fp64_tolerance(inp):
    """Parity tolerance of the FP64 path for a problem: max(1e-12, 1e-14 * stiffness), where
    stiffness = max over (zone, group) of a c dt * (kappa_a + j + NES in/out rates) * |psi|,
    divided by max |psi| (per ray and species).  The residual's source terms, of size
    rate * psi, cancel at the root and each carries ~eps relative rounding, so two correct
    FP64 implementations differ by ~eps * stiffness in the normwise measure."""
    from oracle import mgfld_oracle as O
    f = O.setup_step(inp['problem'], inp['psi0'], inp['ye0'], inp['T0'])
    mu_q, _ = O.species_mu(f.rho, f.T_n, f.ye_n, f.eos)
    j, _ = O.emissivity(f.kappa_abs, f.eps, mu_q, f.T_n)
    rate = O.nes_inverse_mfp(f.psi_n, f.w, f.phi_out, f.phi_in) + j + f.kappa_abs
    weighted = rate * (f.lapse * O.C_LIGHT * f.dt)[:, None, :, None] * np.abs(f.psi_n)
    stiff = np.max(np.max(weighted, axis=(2, 3)) / np.max(np.abs(f.psi_n), axis=(2, 3)))
    return max(1e-12, 1e-14 * stiff)
