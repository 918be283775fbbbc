"""Error measures of a GPU result against the oracle's (test infrastructure).

normwise    per (ray, species): max |d| over all zones and groups / max |ref| over the same
            (the gate of "relative in psi0" used throughout the parity tests);
per_group   per (ray, species, group): max over zones of |d| / max over zones of |ref| (the
            zone-max measure of each group), with its bound implied by the normwise gate g:
            per_group <= g * max |ref| / max_zones |ref_group|;
elementwise max |d| / max(|ref|, 1e-30) over every element (reported, not gated: occupations
            span ~1e-40 ... 1 while the step's convergence test is absolute, tolmin_psi = 1)."""
import numpy as np


def normwise(a, b):
    num = np.max(np.abs(a - b), axis=(2, 3))
    den = np.maximum(np.max(np.abs(b), axis=(2, 3)), 1e-300)
    return float(np.max(num / den))


def per_group(a, b):
    num = np.max(np.abs(a - b), axis=2)
    den = np.maximum(np.max(np.abs(b), axis=2), 1e-300)
    return num / den


def per_group_bound(b, gate):
    whole = np.max(np.abs(b), axis=(2, 3))[:, :, None]
    grp = np.maximum(np.max(np.abs(b), axis=2), 1e-300)
    return gate * whole / grp


def elementwise(a, b, floor=1e-30):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def report(name, a, b, gate):
    """Print the three measures and check the normwise gate and the per-group bound it implies."""
    nw = normwise(a, b)
    pg = per_group(a, b)
    bound = per_group_bound(b, gate)
    ratio = float(np.max(pg / bound))
    el = elementwise(a, b)
    print(f'{name}: normwise {nw:.2e} (gate {gate:.1e}); per-group zone-max {float(np.max(pg)):.2e} '
          f'(median {float(np.median(pg)):.2e}, at most {ratio:.2f} of its implied bound); '
          f'elementwise (floor 1e-30) {el:.2e}')
    assert nw < gate, (name, nw, gate)
    assert ratio < 1.0, (name, ratio)
    return nw


def stepwise(M, torch, inp, precision, steps, gate, label, **step_kw):
    """`steps` GPU steps of `inp`, each compared with the oracle's step taken from the GPU's own
    previous state (the parity of one implicit step, gated at `gate`), and the final state with
    the oracle's own `steps` consecutive steps (states that differ by ~gate after a step give
    different next steps: the drift is gated at steps * gate).  Returns the final GPU state
    (psi, ye, T), the per-step codes, the last report and the oracle's final state."""
    from oracle import mgfld_oracle as O
    st = M.Stepper(inp, precision, **step_kw)
    psi, ye, T = st.state_to_device(inp['psi0'], inp['ye0'], inp['T0'])
    prob = inp['problem']
    prev = (inp['psi0'], inp['ye0'], inp['T0'])
    codes = []
    for s in range(steps):
        codes.append(st.step(psi, ye, T))
        torch.cuda.synchronize()
        got = (psi.cpu().numpy(), ye.cpu().numpy(), T.cpu().numpy())
        ref = O.step(prob, *prev)
        report(f'{label}, step {s + 1} from the same state', got[0], ref['psi'], gate)
        t_err = float(np.max(np.abs(got[2] / ref['T'] - 1.0)))
        print(f'  T relative {t_err:.2e}')
        assert t_err < gate
        prev = got
    rep = {k: v.cpu().numpy() for k, v in st.report.items()}
    psi_o, ye_o, T_o, _ = O.run_steps(prob, inp['psi0'], inp['ye0'], inp['T0'], steps)
    report(f'{label}, {steps} steps from the start (drift)', prev[0], psi_o, steps * gate)
    return prev, codes, rep, (psi_o, ye_o, T_o)
