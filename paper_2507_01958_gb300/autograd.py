"""torch.autograd.Function over the C ABI: m(T) of the equilibrium reached by
the Chambolle-Pock solve, differentiable in (m0, V, W, nu or nu(x)) through
mfg_adjoint (implicit differentiation of the KKT conditions).

Forward runs mfg_solve from the standard start (m^k = m0, w = 0, z = 0);
backward runs one adjoint solve.  The gradient is exact for the converged
equilibrium, so the forward solve must be converged (enough CP iterations or a
CP tolerance in the problem).
"""
from __future__ import annotations

import torch

from . import _lib as L


class MFGEquilibrium(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m0, V, W, nu, problem, precision="mixed", adj_tol=1e-10):
        field = nu.dim() > 0
        if field:  # a viscosity field nu(x): the plan reads it on the host
            p = dict(problem, nu_field=nu.detach().to("cpu", torch.float64).numpy())
        else:
            p = dict(problem, nu=float(nu))
        plan = L.mfg_plan(p, precision=precision)
        nx, ny = p["n"]
        S = nx * ny
        nt = p["nt"]
        c = 1 + 2 * p["dim"]
        dev = m0.device
        y = torch.zeros(c * nt * S, dtype=torch.float64, device=dev)
        y[: nt * S] = m0.reshape(-1).repeat(nt)
        ybar = y.clone()
        z = torch.zeros(nt * S, dtype=torch.float64, device=dev)
        rc, st = L.mfg_solve(plan, m0.contiguous().reshape(-1), V.contiguous().reshape(-1),
                             W.contiguous().reshape(-1), y, ybar, z)
        if rc != L.MFG_OK:
            raise L.MfgError(rc, L.mfg_last_error())
        ctx.plan, ctx.shape, ctx.nt, ctx.adj_tol, ctx.field = plan, (nx, ny), nt, adj_tol, field
        ctx.stats = st[0]
        ctx.save_for_backward(y, z)
        return y[(nt - 1) * S: nt * S].reshape(nx, ny).clone()

    @staticmethod
    def backward(ctx, g_mT):
        y, z = ctx.saved_tensors
        nx, ny = ctx.shape
        S, nt = nx * ny, ctx.nt
        gy = torch.zeros_like(y)
        gy[(nt - 1) * S: nt * S] = g_mT.reshape(-1).to(torch.float64)
        dm0 = torch.empty(S, dtype=torch.float64, device=y.device)
        dV = torch.empty_like(dm0)
        dW = torch.empty_like(dm0)
        dnu = torch.empty(S if ctx.field else 1, dtype=torch.float64, device=y.device)
        L.mfg_adjoint(ctx.plan, 0, y, z, gy, dm0, dV, dW, dnu, tol=ctx.adj_tol)
        dnu = dnu.reshape(nx, ny) if ctx.field else dnu.reshape(())
        return dm0.reshape(nx, ny), dV.reshape(nx, ny), dW.reshape(nx, ny), dnu, None, None, None


def equilibrium_mT(m0, V, W, nu, problem, precision="mixed", adj_tol=1e-10):
    """m(T) as a differentiable function of m0, V, W (fields) and nu: a 0-d
    tensor (constant viscosity) or an (Nx, Ny) tensor (a viscosity field nu(x),
    whose gradient is taken node by node)."""
    return MFGEquilibrium.apply(m0, V, W, nu, problem, precision, adj_tol)
