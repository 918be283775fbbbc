"""Gradients of a multi-step transport run through the library's discrete adjoint.

The objective is the energy deposited in matter by nu_e and nubar_e between 100 and
300 km, summed over rays and over `n_steps` implicit steps (the heating that
mgfld_step reports per ray).  Parameters: the per-(species, group) opacity scales s
that multiply kappa_abs and kappa_scat, and the initial state (psi^0, Ye^0, T^0).

Forward: FP64 mgfld_step calls, keeping the state every `checkpoint_every` steps.
Reverse: each segment between checkpoints is stepped forward again from its
checkpoint (the states inside it are held only while the segment is reversed), then
mgfld_adjoint is applied step by step from the segment's end.  Memory: one state per
checkpoint plus one segment of states.  Every transport and adjoint operation runs in
the library's kernels; this module orders the calls and holds device buffers.
"""
from __future__ import annotations

import numpy as np

from . import mgfld as M


class AdjointRunner:
    """Forward/reverse driver for one problem (device-resident, FP64)."""

    def __init__(self, inp, checkpoint_every=5, device='cuda', tol=1e-12, max_iter=60, max_sweeps=0,
                 sweep_tol=0.0):
        import torch
        prob = inp['problem']
        self.n_ray, _, self.n_r, self.n_e = np.asarray(inp['psi0']).shape
        self.device = device
        self.prob = M.DeviceProblem(prob, device)
        self.dims = M.Dims(self.n_ray, self.n_r, self.n_e, M.N_SPECIES)
        self.opts = M.step_opts(M.MGFLD_FP64, tol=tol, tolmin_psi=1.0, tolmin_ye=0.1, max_iter=max_iter)
        nbytes = max(M.mgfld_adjoint_workspace_bytes(self.dims), M.mgfld_workspace_bytes(self.dims, M.MGFLD_FP64))
        if nbytes == 0:
            raise M.MgfldError(M.MGFLD_EINVAL, 'mgfld_adjoint_workspace_bytes')
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.heating = torch.zeros(self.n_ray, dtype=torch.float64, device=device)
        self.ray_status = torch.zeros(self.n_ray, dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.checkpoint_every = max(1, int(checkpoint_every))
        self.max_sweeps, self.sweep_tol = int(max_sweeps), float(sweep_tol)
        self.sweeps = []

    def _problem(self, scale):
        p = self.prob.struct
        return M.Problem(p.r_edge, p.lapse, p.e_edge, p.rho, p.kappa_abs, p.kappa_scat, p.nes_coef,
                         M._ptr(scale), p.eos, p.dt, p.outer_bc, p.u, p.eta1, p.pair_coef)

    def _step(self, ps, psi, ye, T):
        rc = M.mgfld_step(self.dims, ps, psi, ye, T, self.opts, self.ws,
                          dict(heating=self.heating, ray_status=self.ray_status, status=self.status))
        if rc == M.MGFLD_OK:
            rc = int(self.status.item())          # the step's own status (waits for it)
        if rc != M.MGFLD_OK:
            raise M.MgfldError(rc, 'mgfld_step')
        return self.heating.sum()

    def forward(self, scale, psi0, ye0, T0, n_steps):
        """Total heating J (device scalar) and the checkpoints [(step, psi, ye, T)]."""
        ps = self._problem(scale)
        psi, ye, T = psi0.clone(), ye0.clone(), T0.clone()
        ckpt = [(0, psi.clone(), ye.clone(), T.clone())]
        J = psi.new_zeros(())
        for n in range(n_steps):
            J = J + self._step(ps, psi, ye, T)
            if (n + 1) % self.checkpoint_every == 0 and n + 1 < n_steps:
                ckpt.append((n + 1, psi.clone(), ye.clone(), T.clone()))
        return J, ckpt

    def reverse(self, scale, ckpt, n_steps, heat_weight=1.0, bars=(None, None, None)):
        """Gradients (psi^0, Ye^0, T^0, scale) of heat_weight * J + <bars, state^{n_steps}>."""
        import torch
        ps = self._problem(scale)
        psi_bar, ye_bar, T_bar = bars
        s_bar = torch.zeros(M.N_SPECIES, self.n_e, dtype=torch.float64, device=self.device)
        out = None
        self.sweeps = []
        for c in range(len(ckpt) - 1, -1, -1):
            n0, psi, ye, T = ckpt[c]
            n1 = ckpt[c + 1][0] if c + 1 < len(ckpt) else n_steps
            states = [(psi.clone(), ye.clone(), T.clone())]
            for _ in range(n0, n1):
                p, y, t = (a.clone() for a in states[-1])
                self._step(ps, p, y, t)
                states.append((p, y, t))
            for m in range(n1 - n0 - 1, -1, -1):
                out = (torch.empty_like(states[m][0]), torch.empty_like(states[m][1]),
                       torch.empty_like(states[m][2]))
                rc, sweeps, change = M.mgfld_adjoint(self.dims, ps, states[m], states[m + 1][:2],
                                                     (psi_bar, ye_bar, T_bar), out, self.ws, heat_weight, s_bar,
                                                     self.max_sweeps, self.sweep_tol)
                if rc != M.MGFLD_OK:
                    raise M.MgfldError(rc, f'mgfld_adjoint (sweeps {sweeps}, change {change:.3e})')
                self.sweeps.append(sweeps)
                psi_bar, ye_bar, T_bar = out
            del states
        return psi_bar, ye_bar, T_bar, s_bar


def _heating_function():
    import torch

    class HeatingObjective(torch.autograd.Function):
        """J(scale, psi^0, Ye^0, T^0) = total gain-region heating over n_steps; backward by
        the discrete adjoint with checkpointed recomputation."""

        @staticmethod
        def forward(ctx, scale, psi0, ye0, T0, runner, n_steps):
            scale_c = scale.detach().contiguous()
            J, ckpt = runner.forward(scale_c, psi0.detach().contiguous(), ye0.detach().contiguous(),
                                     T0.detach().contiguous(), n_steps)
            ctx.runner, ctx.n_steps, ctx.ckpt, ctx.scale = runner, n_steps, ckpt, scale_c
            return J

        @staticmethod
        def backward(ctx, gJ):
            w = float(gJ.item())
            psi_b, ye_b, T_b, s_b = ctx.runner.reverse(ctx.scale, ctx.ckpt, ctx.n_steps, heat_weight=w)
            return s_b, psi_b, ye_b, T_b, None, None

    return HeatingObjective


_FN = None


def heating_objective(scale, psi0, ye0, T0, runner: AdjointRunner, n_steps: int):
    """Differentiable total heating: torch.autograd sees (scale, psi0, ye0, T0)."""
    global _FN
    if _FN is None:
        _FN = _heating_function()
    return _FN.apply(scale, psi0, ye0, T0, runner, n_steps)


def reduce_over_ranks(J, scale_grad, group=None):
    """Ray-sharded runs (contiguous ray blocks per rank): J is a sum over rays, so the whole-job
    objective and its gradient with respect to the shared [4, n_e] opacity scales are sums over
    the ranks' values, formed by one all-reduce of 1 + 4 n_e doubles (NCCL for device tensors,
    gloo for host ones).  The gradients with respect to psi^0, Ye^0 and T^0 belong to the rank's
    own rays and are not reduced.  Returns the summed (J, scale_grad)."""
    import torch
    import torch.distributed as dist
    g = torch.as_tensor(scale_grad, dtype=torch.float64)
    buf = torch.cat([torch.as_tensor(J, dtype=torch.float64, device=g.device).reshape(1), g.reshape(-1)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[0], buf[1:].reshape(g.shape)
