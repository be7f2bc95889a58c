"""Implicit differentiation of the converged equilibrium (the KKT conditions of
(VMFG_h), Sec. 2-3), for the gradient of a loss on m(T) with respect to m0,
the potential field V (the coupling of f) and the viscosity nu.

At a solution (y, z) of the CP iteration, y = prox_{tau phi}(y - tau C^T z) and
C y = d(m0), i.e. on the active set A (cells with m > 0, flux components w_c
!= 0; inactive components are fixed at 0):
    R1 = grad phi_A(y) + (C^T z)_A = 0,     R2 = C_A y_A - d(m0) = 0.
With the KKT matrix K = [[H, C_A^T], [C_A, 0]], H = Hessian of phi on A
(per cell, derived from b_hat = |w|^2/(2m) and F), the adjoint
K [mu; eta] = [g_A; 0], g = dloss/dy, gives dloss/dtheta = -[mu; eta].dR/dtheta:
    d/dm0(x) = eta(plane 0, x)/dt                    (d = m0/dt on plane 0)
    d/dV(x)  = -sum_k mu_m(k, x)                      (V enters f_eff on every plane)
    d/dW(x)  = -mu_m(last, x)/dt                      (G/dt on the last plane)
    d/dnu    = -mu_m.(I (x) K) z - eta.(I (x) K) m     (L = nu K + I/dt in C)
Everything here is assembled as sparse matrices and solved by sparse LU.

`kkt_newton` refines a CP solution to the exact KKT point on its active set by
Newton's method (quadratic convergence), which makes finite differences of the
loss accurate enough to pin the gradient.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import operators as ops
from .prox import coupling


def active_mask(y):
    """(c, nt, Nx, Ny) boolean: m > 0 and, in such cells, w_c != 0."""
    y = np.asarray(y)
    m_on = y[0] > 0
    act = np.zeros(y.shape, dtype=bool)
    act[0] = m_on
    act[1:] = (y[1:] != 0) & m_on[None]
    return act


def grad_phi(prob, y, V, W):
    """Gradient of phi = b_hat + F_eff at y (valid where m > 0)."""
    y = np.asarray(y, dtype=np.float64)
    m, w = y[0], y[1:]
    a, b, c = coupling(prob, V, W)
    safe = np.where(m > 0, m, 1.0)
    w2 = (w * w).sum(axis=0)
    gm = -w2 / (2 * safe * safe) + a * m + b * m * m + c
    gw = w / safe[None]
    return np.concatenate([gm[None], gw], axis=0)


def hessian(prob, y):
    """Sparse block-diagonal Hessian of phi over all c*n components (cells with
    m = 0 get zero blocks; callers restrict to the active set)."""
    y = np.asarray(y, dtype=np.float64)
    c = y.shape[0]
    n = y[0].size
    m = y[0].reshape(-1)
    w = y[1:].reshape(c - 1, -1)
    a, b, _ = coupling(prob, np.zeros(prob["n"]), np.zeros(prob["n"]))
    ap = (a + 2 * b * y[0]).reshape(-1)
    safe = np.where(m > 0, m, 1.0)
    rows, cols, vals = [], [], []
    idx = np.arange(n)
    on = m > 0
    # mm
    rows.append(idx[on]); cols.append(idx[on])
    vals.append(((w * w).sum(0) / safe ** 3 + ap)[on])
    for q in range(c - 1):
        iq = (q + 1) * n + idx
        rows += [idx[on], iq[on], iq[on]]
        cols += [iq[on], idx[on], iq[on]]
        vals += [(-w[q] / safe ** 2)[on], (-w[q] / safe ** 2)[on], (1.0 / safe)[on]]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(c * n, c * n))


def kkt_residual(prob, y, z, m0, V, W, C=None, act=None):
    if C is None:
        C = ops.constraint(prob)
    if act is None:
        act = active_mask(y)
    a = act.reshape(-1)
    r1 = (grad_phi(prob, y, V, W).reshape(-1) + C.T @ np.asarray(z).reshape(-1))[a]
    r2 = C @ np.asarray(y).reshape(-1) - ops.rhs_d(prob, m0)
    return r1, r2


def kkt_newton(prob, y, z, m0, V, W, iters=8, tol=1e-14):
    """Newton's method on R1 = 0, R2 = 0 with the active set of y frozen."""
    C = ops.constraint(prob)
    act = active_mask(y)
    a = act.reshape(-1)
    y = np.asarray(y, dtype=np.float64).reshape(-1).copy()
    z = np.asarray(z, dtype=np.float64).reshape(-1).copy()
    shp = act.shape
    CA = C[:, a]
    for _ in range(iters):
        r1, r2 = kkt_residual(prob, y.reshape(shp), z, m0, V, W, C, act)
        scale = max(1.0, np.abs(grad_phi(prob, y.reshape(shp), V, W).reshape(-1)[a]).max())
        if max(np.abs(r1).max() / scale, np.abs(r2).max() / max(1.0, np.abs(ops.rhs_d(prob, m0)).max())) < tol:
            break
        H = hessian(prob, y.reshape(shp))[a][:, a]
        K = sp.bmat([[H, CA.T], [CA, None]]).tocsc()
        step = spla.splu(K).solve(-np.concatenate([r1, r2]))
        y[a] += step[:a.sum()]
        z += step[a.sum():]
    return y.reshape(shp), z.reshape(shp[1:])


def loss_mT(prob, y, m_target):
    """sum_ij (m^{N_t}_ij - m_target,ij)^2 dx^d and its gradient in y."""
    dx, dy = ops.spacing(prob)
    vol = dx * (dy if prob["dim"] == 2 else 1.0)
    y = np.asarray(y)
    diff = y[0, -1] - np.asarray(m_target).reshape(y.shape[2:])
    g = np.zeros_like(y)
    g[0, -1] = 2 * diff * vol
    return float((diff * diff).sum() * vol), g


def _nu_field_gradient(prob, mu_m, z, eta3, m):
    """dloss/dnu(x) at every node for a viscosity field.  nu enters only through
    K_nu = sum_axes D^1 diag(nu_face) (D^1)^T / dx^2 with nu_face the mean of the
    face's two nodes, so dK_nu/dnu_a = sum over the faces f of node a of
    (1/2) g_f g_f^T / dx^2 with g_f = (D^1)^T row f (the face difference), and
      dloss/dnu_a = -(1/2) sum_k sum_{f of a} [(g_f.mu_m^k)(g_f.z^k) + (g_f.eta^k)(g_f.m^k)] / dx^2,
    the same contraction as the scalar dnu with K split face by face."""
    nt = prob["nt"]
    nx, ny = prob["n"]
    dx = ops.spacing(prob)
    out = np.zeros((nx, ny))
    for ax in range(prob["dim"]):
        n_ax = (nx, ny)[ax]
        d1, _ = ops.div_blocks(n_ax, prob["bc"][ax])
        D = sp.kron(d1, sp.identity(ny)) if (prob["dim"] == 2 and ax == 0) else (
            sp.kron(sp.identity(nx), d1) if prob["dim"] == 2 else d1)
        cf = np.zeros(D.shape[1])
        for k in range(nt):
            g = lambda u: D.T @ np.asarray(u[k]).reshape(-1)
            cf += g(mu_m) * g(z) + g(eta3) * g(m)
        cf /= dx[ax] ** 2
        # face f joins node f and its plus neighbour; each takes half
        absD = abs(D).tocsr()
        out += (-0.5 * (absD @ cf)).reshape(nx, ny)
    return out


def adjoint_gradients(prob, y, z, gy):
    """Solve K [mu; eta] = [g_A; 0] and contract: returns dict of dm0 (Nx, Ny),
    dV (Nx, Ny), dW (Nx, Ny), dnu (float; with a viscosity field the (Nx, Ny)
    derivative in the node values nu(x)), plus mu, eta."""
    C = ops.constraint(prob)
    act = active_mask(y)
    a = act.reshape(-1)
    shp = act.shape
    H = hessian(prob, y)[a][:, a]
    CA = C[:, a]
    K = sp.bmat([[H, CA.T], [CA, None]]).tocsc()
    rhs = np.concatenate([np.asarray(gy).reshape(-1)[a], np.zeros(C.shape[0])])
    sol = spla.splu(K).solve(rhs)
    mu = np.zeros(a.size)
    mu[a] = sol[:a.sum()]
    eta = sol[a.sum():]
    mu = mu.reshape(shp)
    nt = prob["nt"]
    nx, ny = prob["n"]
    h = ops.dt(prob)
    eta3 = eta.reshape(nt, nx, ny)
    if ops.has_nu_field(prob):
        z3 = np.asarray(z).reshape(nt, nx, ny)
        dnu = _nu_field_gradient(prob, mu[0], z3, eta3, np.asarray(y)[0].reshape(nt, nx, ny))
    else:
        _, Ksp = ops.spatial(prob)
        Kz = np.stack([(Ksp @ np.asarray(z).reshape(nt, -1)[k]) for k in range(nt)]).reshape(nt, nx, ny)
        Km = np.stack([(Ksp @ np.asarray(y)[0].reshape(nt, -1)[k]) for k in range(nt)]).reshape(nt, nx, ny)
        dnu = float(-(mu[0] * Kz).sum() - (eta3 * Km).sum())
    return {
        "dm0": eta3[0] / h,
        "dV": -mu[0].sum(axis=0),
        "dW": -mu[0][-1] / h,
        "dnu": dnu,
        "mu": mu,
        "eta": eta3,
    }
