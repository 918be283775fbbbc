"""Small hand-built transport problems for pins and parity tests (inputs only)."""
import numpy as np

from paper_1809_05608_gb300 import problems


def strong(n_ray=2, n_r=8, n_e=5, kabs=1e16, kscat=1e14, nes=1.0, lapse=False, config=2,
           bc=0, dt=1e-6):
    """The synthetic profile at reduced size with opacities scaled up so that
    absorption/emission, scattering and NES all matter within one step."""
    inp = problems.make_problem(config, n_ray=n_ray, n_r=n_r, n_e=n_e)
    p = dict(inp['problem'])
    p['kappa_abs'] = p['kappa_abs'] * kabs
    p['kappa_scat'] = p['kappa_scat'] * kscat
    p['nes_coef'] = p['nes_coef'] * nes
    p['outer_bc'] = bc
    p['dt'] = dt
    if lapse:
        rc = 0.5 * (p['r_edge'][:, 1:] + p['r_edge'][:, :-1])
        p['lapse'] = np.sqrt(1.0 - 0.2 * rc[:, :1] / rc)   # 0.89 .. 1, varies along the ray
    inp = dict(inp)
    inp['problem'] = p
    return inp
