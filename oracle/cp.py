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
afterwards (Chambolle-Pock 2011, Alg. 2).  The dual x is stored explicitly; the
solve with C C^T is exact (sparse LU or the spatially-diagonalised solver).
Start: tau_0 = sigma_0 = 1, x_0 = 0, ybar_0 = y_0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import operators as ops
from . import solvers
from .prox import prox


class Solver:
    def __init__(self, prob, m0, V, W, method="auto"):
        self.prob = prob
        self.C = ops.constraint(prob)
        self.CT = self.C.T.tocsr()
        self.d = ops.rhs_d(prob, m0)
        self.V, self.W = V, W
        s, n, c = ops.sizes(prob)
        self.n, self.c = n, c
        if method == "auto":
            method = "lu" if n <= 40000 else "modal"
        self.method = method
        if method == "lu":
            self._lu = spla.splu(ops.AAt(prob, self.C).tocsc())

    def solve_AAt(self, b):
        if self.method == "lu":
            return self._lu.solve(b)
        return solvers.solve_AAt_modal(self.prob, b)

    def run(self, y0, iters=None, ybar0=None, x0=None, tau0=None, sigma0=None, record=False):
        p = self.prob
        shp = (self.c,) + (p["nt"],) + tuple(p["n"])
        y = np.asarray(y0, dtype=np.float64).reshape(-1).copy()
        ybar = y.copy() if ybar0 is None else np.asarray(ybar0, dtype=np.float64).reshape(-1).copy()
        x = np.zeros_like(y) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()
        tau = p["tau0"] if tau0 is None else tau0
        sigma = p["sigma0"] if sigma0 is None else sigma0
        iters = p["max_cp"] if iters is None else iters
        z = np.zeros(self.n)
        hist = []
        ell = 0
        for ell in range(1, iters + 1):
            b = self.C @ (x + sigma * ybar) - sigma * self.d
            z = self.solve_AAt(b)
            x = self.CT @ z
            y_new = prox(p, tau, (y - tau * x).reshape(shp), self.V, self.W).reshape(-1)
            theta = 1.0 / np.sqrt(1.0 + 2.0 * p["gamma"] * tau)
            tau, sigma = theta * tau, sigma / theta
            ybar = y_new + theta * (y_new - y)
            r = np.linalg.norm(y_new[:self.n] - y[:self.n])
            y = y_new
            if record:
                hist.append(r)
            if p["cp_tol"] > 0 and r <= p["cp_tol"]:
                break
        return {"y": y.reshape(shp), "ybar": ybar.reshape(shp), "z": z.reshape(shp[1:]),
                "x": x.reshape(shp), "tau": tau, "sigma": sigma, "iters": ell, "r": hist}
