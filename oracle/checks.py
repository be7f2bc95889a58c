"""Diagnostics computed from definitions: mass, constraint residual, the
objective phi (Sec. 2 b_hat, calB, calF), its conjugate and the primal-dual gap.

The conjugate of the per-cell phi for f_eff(m) = a m + c (f_b = 0) is derived
from the definition of b_hat: for fixed m the sup over w in K of
beta.w - |w|^2/(2m) equals m |P_K beta|^2 / 2, so
phi*(alpha, beta) = ([alpha + |P_K beta|^2/2 - c]_+)^2 / (2a)   (a > 0).
It is pinned in the tests by numerical maximisation.
"""
from __future__ import annotations

import numpy as np

from . import operators as ops
from .prox import coupling, project_K


def mass(prob, y):
    """Sum_ij m^k_ij dx^d for every plane k (exactly 1 when C y = d, m0 normalised)."""
    dx, dy = ops.spacing(prob)
    vol = dx * (dy if prob["dim"] == 2 else 1.0)
    return np.asarray(y)[0].reshape(prob["nt"], -1).sum(axis=1) * vol


def constraint_residual(prob, y, m0):
    C = ops.constraint(prob)
    return C @ np.asarray(y).reshape(-1) - ops.rhs_d(prob, m0)


def objective_cells(prob, y, V, W):
    """phi per cell (nt, Nx, Ny), +inf outside the domain."""
    y = np.asarray(y, dtype=np.float64)
    m, w = y[0], y[1:]
    a, b, c = coupling(prob, V, W)
    F = 0.5 * a * m * m + b * m ** 3 / 3.0 + c * m
    inK = np.all(project_K(w) == w, axis=0)
    w2 = (w * w).sum(axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        bh = np.where(m > 0, w2 / (2.0 * np.where(m > 0, m, 1.0)), 0.0)
    ok = ((m > 0) & inK) | ((m == 0) & (w2 == 0))
    return np.where(ok, bh + F, np.inf)


def objective(prob, y, V, W):
    return float(objective_cells(prob, y, V, W).sum())


def conjugate_cells(prob, alpha, beta, V, W):
    """phi*(alpha, beta) per cell, f_b = 0 and a > 0."""
    a, b, c = coupling(prob, V, W)
    assert b == 0.0
    P = project_K(beta)
    s = np.maximum(alpha + 0.5 * (P * P).sum(axis=0) - c, 0.0)
    return s * s / (2.0 * a)


def gap(prob, y, z, m0, V, W):
    """phi(y) + phi*(-x) + <z, d> with x = C^T z (feasible y assumed)."""
    C = ops.constraint(prob)
    x = (C.T @ np.asarray(z).reshape(-1)).reshape(np.asarray(y).shape)
    d = ops.rhs_d(prob, m0)
    return objective(prob, y, V, W) + float(conjugate_cells(prob, -x[0], -x[1:], V, W).sum()) \
        + float(np.asarray(z).reshape(-1) @ d)
