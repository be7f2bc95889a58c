"""Accelerated Chambolle-Pock iteration for (VMFG_h) (Sec. 3 eq. pasosChamPock,
step sizes of Sec. 5), in the paper's notation and order:

  x_{l+1} = prox_{sigma psi*}(x_l + sigma ybar_l)
          = C^T (C C^T)^{-1} (C (x_l + sigma ybar_l) - sigma d)        (eq. CC*)
  y_{l+1} = prox_{tau phi}(y_l - tau x_{l+1})
  theta   = 1/sqrt(1 + 2 gamma tau_l); tau_{l+1} = theta tau_l;
  sigma_{l+1} = sigma_l/theta
  ybar_{l+1} = y_{l+1} + theta (y_{l+1} - y_l)
  r_l = ||m_{l+1} - m_l||_2; stop when r_l <= cp_tol (if cp_tol > 0).

The proxes of iteration l use (tau_l, sigma_l) and the step sizes are updated
afterwards (Chambolle-Pock 2011, Alg. 2).  C and C^T are sparse matrices, or on
grids too large to assemble (n > 2^22) the plane-by-plane applies of
operators.py, pinned against the sparse matrices.  The dual x is stored explicitly; the
solve with C C^T is exact (sparse LU or the spatially-diagonalised solver), or,
with method="pcg", inexact as in Sec. 5: preconditioned CG with the paper's P
(eq. prec; P = C C^T for l = 0), started from the previous z, stopped at the
fixed prob["cg_tol"] or at the adaptive min{1e-4, max{1e-6, 1e-4 r}} of Sec. 5
(prob["cg_rule"] = 1), relative either to the residual of the warm start
(cg_ref="resid") or to the right-hand side of the full system (cg_ref="rhs").
With a viscosity field nu(x) (prob["nu_field"]) the exact solve is sparse LU
and the PCG preconditioner is Alg. 1 with a sparse LU per time frequency.
Start: tau_0 = sigma_0 = 1, x_0 = 0, ybar_0 = y_0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import operators as ops
from . import solvers
from .prox import prox


class _PlaneOp:
    """C or C^T applied plane by plane (operators.apply_C_planes /
    apply_Ct_planes) for grids too large to assemble; supports `@`."""

    def __init__(self, prob, transpose):
        self.prob, self.transpose = prob, transpose

    def __matmul__(self, v):
        f = ops.apply_Ct_planes if self.transpose else ops.apply_C_planes
        return f(self.prob, v)


class Solver:
    def __init__(self, prob, m0, V, W, method="auto", cg_ref="resid", matrix_free=None):
        self.prob = prob
        s, n, c = ops.sizes(prob)
        self.n, self.c = n, c
        if matrix_free is None:
            matrix_free = n > (1 << 22)
        if matrix_free:
            self.C, self.CT = _PlaneOp(prob, False), _PlaneOp(prob, True)
        else:
            self.C = ops.constraint(prob)
            self.CT = self.C.T.tocsr()
        self.d = ops.rhs_d(prob, m0)
        self.V, self.W = V, W
        if method == "auto":
            method = "lu" if (n <= 40000 or ops.has_nu_field(prob)) else "modal"
        self.method = method
        self.cg_ref = cg_ref
        if method == "lu":
            self._lu = spla.splu(ops.AAt(prob, self.C).tocsc())

    def solve_AAt(self, b):
        if self.method == "lu":
            return self._lu.solve(b)
        return solvers.solve_AAt_modal(self.prob, b)

    def solve_AAt_pcg(self, b, z0, tol):
        """Inexact solve of C C^T z = b by PCG from z0 (Sec. 5); returns (z, iterations)."""
        p = self.prob
        apply_A = lambda v: self.C @ (self.CT @ v)
        if ops.has_nu_field(p):
            # a viscosity field: Alg. 1 with one sparse LU per time frequency
            apply_Minv = lambda r: solvers.precond_lu(p, r)
        elif p["l"] == 0:
            apply_Minv = lambda r: solvers.solve_AAt_modal(p, r)
        else:
            apply_Minv = lambda r: solvers.precond_modal(p, r)
        if self.cg_ref == "resid":
            dz, it = solvers.pcg(apply_A, apply_Minv, b - apply_A(z0), tol, maxiter=p["max_cg"])
            return z0 + dz, it
        return solvers.pcg(apply_A, apply_Minv, b, tol, x0=z0, maxiter=p["max_cg"])

    def run(self, y0, iters=None, ybar0=None, x0=None, tau0=None, sigma0=None, record=False):
        p = self.prob
        shp = (self.c,) + (p["nt"],) + tuple(p["n"])
        y = np.asarray(y0, dtype=np.float64).reshape(-1).copy()
        ybar = y.copy() if ybar0 is None else np.asarray(ybar0, dtype=np.float64).reshape(-1).copy()
        x = np.zeros_like(y) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()
        tau = p["tau0"] if tau0 is None else tau0
        sigma = p["sigma0"] if sigma0 is None else sigma0
        iters = p["max_cp"] if iters is None else iters
        # warm start of the inexact solve: the z whose C^T z is the given dual
        z = self.solve_AAt_modal_or_lu(x) if (self.method == "pcg" and x0 is not None) else np.zeros(self.n)
        hist, cg_hist = [], []
        r_prev = np.inf
        ell = 0
        for ell in range(1, iters + 1):
            b = self.C @ (x + sigma * ybar) - sigma * self.d
            if self.method == "pcg":
                tol = p["cg_tol"] if p["cg_rule"] == 0 else min(1e-4, max(1e-6, 1e-4 * r_prev))
                z, it = self.solve_AAt_pcg(b, z, tol)
                cg_hist.append(it)
            else:
                z = self.solve_AAt(b)
            x = self.CT @ z
            y_new = prox(p, tau, (y - tau * x).reshape(shp), self.V, self.W).reshape(-1)
            theta = 1.0 / np.sqrt(1.0 + 2.0 * p["gamma"] * tau)
            tau, sigma = theta * tau, sigma / theta
            ybar = y_new + theta * (y_new - y)
            r = np.linalg.norm(y_new[:self.n] - y[:self.n])
            r_prev = r
            y = y_new
            if record:
                hist.append(r)
            if p["cp_tol"] > 0 and r <= p["cp_tol"]:
                break
        return {"y": y.reshape(shp), "ybar": ybar.reshape(shp), "z": z.reshape(shp[1:]),
                "x": x.reshape(shp), "tau": tau, "sigma": sigma, "iters": ell, "r": hist, "cg": cg_hist}

    def solve_AAt_modal_or_lu(self, x):
        """z with C^T z = x for a given dual start x (least-squares: z = (C C^T)^{-1} C x)."""
        b = self.C @ x
        if self.method == "lu":
            return self._lu.solve(b)
        return solvers.solve_AAt_modal(self.prob, b)
