"""The optimal dispatch as a differentiable function of the bus loads.

``optimal_dispatch(handle, Pd, Qd)`` solves the OPF of the handle's network
with the given loads (opf_set_loads + opf_solve), factors K_aug at the solution
(opf_vjp_prepare) and returns Pg for every generator (slack first).  Its
backward is opf_dispatch_vjp: the implicit-function derivative of the barrier
solution at the final barrier parameter, computed with the condensed
recoveries of Theorems 1 and 2 (one Cholesky solve with Kred and two solves
with G_x per cotangent).

Many cotangents at once: ``torch.func.vjp`` followed by ``torch.func.vmap`` of
the returned function runs one batched opf_dispatch_vjp for the whole batch
(the backward node has a vmap rule), and ``dispatch_vjp(handle, V)`` calls it
directly for a (k, ng) tensor of cotangents.  Second derivatives are not
provided.
"""
from __future__ import annotations

import torch

from .binding import OPF_OK, OPFError


def _device(handle):
    return getattr(handle, "device", None) or torch.device("cuda", torch.cuda.current_device())


def _vjp_call(handle, V):
    """V (..., ng) -> (grad_Pd, grad_Qd), each (..., nb), on V's device."""
    lead = V.shape[:-1]
    dev = _device(handle)
    v = V.detach().reshape(-1, handle.ng).to(device=dev, dtype=torch.float64).contiguous()
    gP = torch.empty((v.shape[0], handle.nb), dtype=torch.float64, device=dev)
    gQ = torch.empty_like(gP)
    handle.dispatch_vjp(v, gP, gQ)
    out = lambda t: t.reshape(*lead, handle.nb).to(V.device)  # noqa: E731
    return out(gP), out(gQ)


class _DispatchVJP(torch.autograd.Function):
    """grad_d = vbar^T dPg/dd; batched under vmap."""

    @staticmethod
    def forward(vbar, handle):
        return _vjp_call(handle, vbar)

    @staticmethod
    def setup_context(ctx, inputs, output):
        pass

    @staticmethod
    def vmap(info, in_dims, vbar, handle):
        bd = in_dims[0]
        if bd is None:
            v = vbar.unsqueeze(0).expand(info.batch_size, *vbar.shape)
        else:
            v = vbar.movedim(bd, 0)
        gP, gQ = _vjp_call(handle, v)
        return (gP, gQ), (0, 0)


class OptimalDispatch(torch.autograd.Function):
    """Pg*(Pd, Qd) of the handle's network (float64, every generator)."""

    @staticmethod
    def forward(Pd, Qd, handle, variant, tol):
        handle.set_loads(Pd.detach().cpu().numpy(), Qd.detach().cpu().numpy())
        out = handle.solve(variant=variant, tol=tol)
        if out["status"] != OPF_OK:
            raise OPFError(out["status"], "opf_solve")
        _, _, _, Pg = handle.solution()
        handle.vjp_prepare()
        return torch.as_tensor(Pg, dtype=torch.float64, device=Pd.device)

    @staticmethod
    def setup_context(ctx, inputs, output):
        ctx.handle = inputs[2]

    @staticmethod
    def backward(ctx, gPg):
        gP, gQ = _DispatchVJP.apply(gPg, ctx.handle)
        return gP, gQ, None, None, None


def optimal_dispatch(handle, Pd, Qd, variant="linred", tol=1e-8):
    """Differentiable Pg*(Pd, Qd); see the module docstring."""
    return OptimalDispatch.apply(Pd, Qd, handle, variant, tol)


def dispatch_vjp(handle, V):
    """vbar^T dPg/dd for cotangents V (k, ng) at the handle's prepared solution
    (after optimal_dispatch or opf_vjp_prepare); returns (grad_Pd, grad_Qd)."""
    return _vjp_call(handle, V)
