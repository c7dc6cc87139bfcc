"""torch.autograd.Function wrappers of the solve and its adjoint (Eqs. 5-6).

Forward: node z coordinates and quad thicknesses -> (u, C, V) through
``sso_model_solve`` and ``sso_model_volume``: displacements, compliance
C = f^T u and the material volume V = sum A_e t_e of the quads (Sec. 3.3).
Backward: with upstream gradients (gu, gC, gV) the scalar being
differentiated is J = gC * C + gu^T u + gV * V.  ``sso_model_gradient(w = gC,
g = gu)`` gives the C and u part directly (one adjoint solve if gu is
non-zero, none otherwise since K is symmetric); the V part is gV times the
volume gradient computed in the forward pass.

With t = None the thicknesses stay as they are and backward returns no
gradient for them.

A model holds one solution at a time: backward must run before the same model
is solved again.
"""
import torch

from . import model as _model


def _grad_scalar(g):
    return 0.0 if g is None else float(g)


class SSOFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mdl, z, t, opts=None):
        mdl.set_design(z, t)
        mdl.solve(opts)
        r = mdl.result(device=z.device)
        vol = mdl.volume(device=z.device)
        ctx.mdl = mdl
        ctx.device = z.device
        ctx.t_given = t is not None
        ctx.vdz = vol["dz"]
        ctx.vdt = vol["dt"]
        C = torch.tensor(r["C"], dtype=torch.float64, device=z.device)
        return r["u"], C, vol["V"]

    @staticmethod
    def backward(ctx, gu, gC, gV):
        mdl = ctx.mdl
        w = _grad_scalar(gC)
        g = None
        if gu is not None and bool(torch.any(gu != 0)):
            g = gu.to(torch.float64).contiguous()
        mdl.gradient(w, g)
        r = mdl.result(device=ctx.device)
        dz, dt = r["dz"], r["dt"]
        if gV is not None:
            dz = dz + gV.to(torch.float64) * ctx.vdz
            dt = dt + gV.to(torch.float64) * ctx.vdt
        return None, dz, (dt if ctx.t_given else None), None


class BatchSSOFunction(torch.autograd.Function):
    """Batched form: z [B, n_nodes], t [B, n_quads] over a Batch of models with
    one topology -> u [B, 6 n_nodes], C [B], V [B]."""

    @staticmethod
    def forward(ctx, batch, z, t, opts=None):
        for i, m in enumerate(batch.models):
            m.set_design(z[i], t[i] if t is not None else None)
        batch.solve(opts)
        us, Cs, Vs, vdz, vdt = [], [], [], [], []
        for m in batch.models:
            r = m.result(device=z.device)
            v = m.volume(device=z.device)
            us.append(r["u"])
            Cs.append(r["C"])
            Vs.append(v["V"])
            vdz.append(v["dz"])
            vdt.append(v["dt"])
        ctx.batch = batch
        ctx.device = z.device
        ctx.t_given = t is not None
        ctx.vdz = torch.stack(vdz)
        ctx.vdt = torch.stack(vdt)
        return (torch.stack(us), torch.tensor(Cs, dtype=torch.float64, device=z.device),
                torch.stack(Vs))

    @staticmethod
    def backward(ctx, gu, gC, gV):
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
        dz, dt = torch.stack(dzs), torch.stack(dts)
        if gV is not None:
            gv = gV.to(torch.float64).reshape(n, 1)
            dz = dz + gv * ctx.vdz
            dt = dt + gv * ctx.vdt
        return None, dz, (dt if ctx.t_given else None), None
