"""torch.autograd.Function wrappers of the solve and its adjoint (Eqs. 5-6).

Forward: node z coordinates and quad thicknesses -> (u, C) through
``sso_model_solve``.  Backward: with upstream gradients (gu, gC) the scalar
being differentiated is J = gC * C + gu^T u, whose sensitivity
``sso_model_gradient(w = gC, g = gu)`` returns directly (one adjoint solve if
gu is non-zero, none otherwise since K is symmetric).

A model holds one solution at a time: backward must run before the same model
is solved again.
"""
import torch

from . import model as _model


class SSOFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mdl, z, t, opts=None):
        mdl.set_design(z, t)
        mdl.solve(opts)
        r = mdl.result(device=z.device)
        ctx.mdl = mdl
        ctx.device = z.device
        C = torch.tensor(r["C"], dtype=torch.float64, device=z.device)
        return r["u"], C

    @staticmethod
    def backward(ctx, gu, gC):
        mdl = ctx.mdl
        w = float(gC) if gC is not None else 0.0
        g = None
        if gu is not None and bool(torch.any(gu != 0)):
            g = gu.to(torch.float64).contiguous()
        mdl.gradient(w, g)
        r = mdl.result(device=ctx.device)
        return None, r["dz"], r["dt"], None


class BatchSSOFunction(torch.autograd.Function):
    """Batched form: z [B, n_nodes], t [B, n_quads] over a Batch of models with
    one topology -> u [B, 6 n_nodes], C [B]."""

    @staticmethod
    def forward(ctx, batch, z, t, opts=None):
        for i, m in enumerate(batch.models):
            m.set_design(z[i], t[i] if t is not None else None)
        batch.solve(opts)
        us, Cs = [], []
        for m in batch.models:
            r = m.result(device=z.device)
            us.append(r["u"])
            Cs.append(r["C"])
        ctx.batch = batch
        ctx.device = z.device
        return torch.stack(us), torch.tensor(Cs, dtype=torch.float64, device=z.device)

    @staticmethod
    def backward(ctx, gu, gC):
        batch = ctx.batch
        n = len(batch.models)
        w = [0.0] * n if gC is None else [float(x) for x in gC.detach().cpu()]
        g = None
        if gu is not None and bool(torch.any(gu != 0)):
            g = [gu[i].to(torch.float64).contiguous() for i in range(n)]
        batch.gradient(w, g)
        dzs, dts = [], []
        for m in batch.models:
            r = m.result(device=ctx.device)
            dzs.append(r["dz"])
            dts.append(r["dt"])
        return None, torch.stack(dzs), torch.stack(dts), None
