"""Linear solvers for the oracle: direct LU, plain CG, and the exact
spatially-diagonalised solver.

The spatially-diagonalised solver follows Sec. 4.3: K = F^{-1} Lambda F with F a
DFT (periodic axis) or an orthonormal DCT-II (Neumann axis), eigenvalues
2 - 2cos(2 pi v/N)/dx^2 and 2 - 2cos(pi v/N)/dx^2 (Alg. 2), and B B^T = 2K
(eq. precstead).  Every block of AAt (eq. largeA) and of P (eq. prec) is then a
polynomial in K, so in K's eigenbasis each spatial mode leaves one symmetric
tridiagonal N_t x N_t system, solved here by Thomas elimination.  This is an
exact direct method, not the paper's preconditioned CG; it is pinned against
sparse LU on small grids.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operators import PERIODIC, Dtt, dt, has_nu_field, nu_faces, spacing, spatial, viscous


# threads of the FFT library (all host cores; the transforms are the same)
_WORKERS = os.cpu_count() or 1


def solve_direct(A, b):
    """Sparse LU solve (SuperLU through scipy)."""
    return spla.splu(A.tocsc()).solve(np.asarray(b, dtype=np.float64))


def solve_cg(A, b, tol=1e-12, x0=None, maxiter=100000):
    """Unpreconditioned conjugate gradients (Hestenes-Stiefel), stopping when
    ||b - A x||_2 <= tol ||b||_2.  Returns (x, iterations)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    p = r.copy()
    rr = r @ r
    bn = np.sqrt(b @ b)
    it = 0
    while np.sqrt(rr) > tol * bn and it < maxiter:
        q = A @ p
        alpha = rr / (p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def laplacian_eigs(prob):
    """Eigenvalues kappa_s of K on the (Nx, Ny) mode grid, in the order of the
    transforms used by `to_modes` (Alg. 2)."""
    out = []
    dims = 2 if prob["dim"] == 2 else 1
    for ax in range(dims):
        n = prob["n"][ax]
        h = spacing(prob)[ax]
        v = np.arange(n)
        if prob["bc"][ax] == PERIODIC:
            lam = 2.0 - 2.0 * np.cos(2.0 * np.pi * v / n)
        else:
            lam = 2.0 - 2.0 * np.cos(np.pi * v / n)
        out.append(lam / h ** 2)
    if dims == 1:
        return out[0][:, None]
    return out[0][:, None] + out[1][None, :]


def to_modes(prob, u):
    """Forward spatial transform of a (nt, Nx, Ny) array: DFT on periodic axes,
    orthonormal DCT-II on Neumann axes."""
    u = np.asarray(u)
    axes = [1, 2] if prob["dim"] == 2 else [1]
    for a in axes:
        if prob["bc"][a - 1] == PERIODIC:
            u = sfft.fft(u, axis=a, workers=_WORKERS)
        else:
            u = sfft.dct(u, type=2, norm="ortho", axis=a, workers=_WORKERS)
    return u


def from_modes(prob, u):
    axes = [2, 1] if prob["dim"] == 2 else [1]
    for a in axes:
        if prob["bc"][a - 1] == PERIODIC:
            u = sfft.ifft(u, axis=a, workers=_WORKERS)
        else:
            if np.iscomplexobj(u):
                u = sfft.idct(u.real, type=2, norm="ortho", axis=a, workers=_WORKERS) + \
                    1j * sfft.idct(u.imag, type=2, norm="ortho", axis=a, workers=_WORKERS)
            else:
                u = sfft.idct(u, type=2, norm="ortho", axis=a, workers=_WORKERS)
    return u


def thomas(diag, off, rhs):
    """Symmetric tridiagonal solve along axis 0 for every column at once.
    diag: (nt, ...), off: (...) constant off-diagonal, rhs: (nt, ...)."""
    nt = diag.shape[0]
    c = np.empty(diag.shape, dtype=np.result_type(diag, off))
    d = np.empty(rhs.shape, dtype=np.result_type(rhs, diag, off))
    c[0] = off / diag[0]
    d[0] = rhs[0] / diag[0]
    for k in range(1, nt):
        den = diag[k] - off * c[k - 1]
        c[k] = off / den
        d[k] = (rhs[k] - off * d[k - 1]) / den
    x = np.empty_like(d)
    x[nt - 1] = d[nt - 1]
    for k in range(nt - 2, -1, -1):
        x[k] = d[k] - c[k] * x[k + 1]
    return x


def _shape(prob):
    nx, ny = prob["n"]
    return prob["nt"], nx, ny


def _constant_nu(prob, what):
    if has_nu_field(prob):
        raise ValueError(what + " needs a constant viscosity (the spatial eigenbasis of K)")


def solve_AAt_modal(prob, b):
    """Exact solve of AAt z = b.  Per spatial mode s with eigenvalue kappa:
    L_s = nu kappa + 1/dt, C_s = L_s^2 + 2 kappa; diagonal (C_s, C_s + 1/dt^2, ...),
    off-diagonal -L_s/dt (eq. largeA with B B^T = 2K)."""
    _constant_nu(prob, "solve_AAt_modal")
    nt, nx, ny = _shape(prob)
    kap = laplacian_eigs(prob)
    h = dt(prob)
    Ls = prob["nu"] * kap + 1.0 / h
    Cs = Ls ** 2 + 2.0 * kap
    diag = np.broadcast_to(Cs, (nt,) + Cs.shape).copy()
    diag[1:] += 1.0 / h ** 2
    bh = to_modes(prob, np.asarray(b, dtype=np.float64).reshape(nt, nx, ny))
    zh = thomas(diag, -Ls / h, bh)
    return np.real(from_modes(prob, zh)).reshape(-1)


def precond_modal(prob, r):
    """Exact P^{-1} r for eq. prec: per spatial mode, C_hat_s = nu^2 kappa^2 + 2 kappa,
    L_hat_s = (nu kappa + 1/dt)/dt, diagonal (C_hat + l L_hat, C_hat + 2 L_hat, ...),
    off-diagonal -L_hat (no time transform involved)."""
    _constant_nu(prob, "precond_modal")
    nt, nx, ny = _shape(prob)
    kap = laplacian_eigs(prob)
    h = dt(prob)
    Lh = (prob["nu"] * kap + 1.0 / h) / h
    Ch = prob["nu"] ** 2 * kap ** 2 + 2.0 * kap
    diag = np.broadcast_to(Ch + 2.0 * Lh, (nt,) + Ch.shape).copy()
    diag[0] = Ch + prob["l"] * Lh
    rh = to_modes(prob, np.asarray(r, dtype=np.float64).reshape(nt, nx, ny))
    zh = thomas(diag, -Lh, rh)
    return np.real(from_modes(prob, zh)).reshape(-1)


def eig_range_AAt(prob):
    """Smallest and largest eigenvalue of AAt (eq. largeA).  In the spatial
    eigenbasis AAt splits into one symmetric tridiagonal N_t x N_t block per
    spatial mode (the blocks of solve_AAt_modal), so its spectrum is the union
    of theirs; each block's extreme eigenvalues come from LAPACK's tridiagonal
    eigensolver.  Modes with equal Laplacian eigenvalue share a block."""
    _constant_nu(prob, "eig_range_AAt")
    nt, kap, h = _modal_blocks(prob)
    lo, hi = np.inf, -np.inf
    for k in np.unique(kap):
        Ls = prob["nu"] * k + 1.0 / h
        d = np.full(nt, Ls ** 2 + 2.0 * k)
        d[1:] += 1.0 / h ** 2
        e = np.full(nt - 1, -Ls / h)
        lo = min(lo, sla.eigvalsh_tridiagonal(d, e, select="i", select_range=(0, 0))[0])
        hi = max(hi, sla.eigvalsh_tridiagonal(d, e, select="i", select_range=(nt - 1, nt - 1))[0])
    return float(lo), float(hi)


def cond_AAt(prob):
    """2-norm condition number of AAt, from eig_range_AAt."""
    lo, hi = eig_range_AAt(prob)
    return hi / lo


def tridiag_mult(diag, off, x):
    """y = T x along axis 0 for a symmetric tridiagonal T with constant off-diagonal."""
    y = diag * x
    y[:-1] += off * x[1:]
    y[1:] += off * x[:-1]
    return y


def _modal_blocks(prob):
    nt = prob["nt"]
    kap = laplacian_eigs(prob)
    h = dt(prob)
    return nt, kap, h


def apply_AAt_modal(prob, p):
    """AAt p through the spatial eigenbasis (same blocks as solve_AAt_modal,
    multiplied instead of solved): a matrix-free AAt for grids too large to
    assemble."""
    _constant_nu(prob, "apply_AAt_modal")
    nt, kap, h = _modal_blocks(prob)
    nx, ny = prob["n"]
    Ls = prob["nu"] * kap + 1.0 / h
    Cs = Ls ** 2 + 2.0 * kap
    diag = np.broadcast_to(Cs, (nt,) + Cs.shape).copy()
    diag[1:] += 1.0 / h ** 2
    ph = to_modes(prob, np.asarray(p, dtype=np.float64).reshape(nt, nx, ny))
    return np.real(from_modes(prob, tridiag_mult(diag, -Ls / h, ph))).reshape(-1)


def apply_P_modal(prob, z):
    """P z for the preconditioner of eq. prec, through the spatial eigenbasis;
    also returns the largest eigenvalue of P (its 2-norm)."""
    _constant_nu(prob, "apply_P_modal")
    nt, kap, h = _modal_blocks(prob)
    nx, ny = prob["n"]
    Lh = (prob["nu"] * kap + 1.0 / h) / h
    Ch = prob["nu"] ** 2 * kap ** 2 + 2.0 * kap
    diag = np.broadcast_to(Ch + 2.0 * Lh, (nt,) + Ch.shape).copy()
    diag[0] = Ch + prob["l"] * Lh
    zh = to_modes(prob, np.asarray(z, dtype=np.float64).reshape(nt, nx, ny))
    out = np.real(from_modes(prob, tridiag_mult(diag, -Lh, zh))).reshape(-1)
    lam_max = float((Ch + 4.0 * Lh).max())  # Gershgorin bound, attained up to O(1/nt^2)
    return out, lam_max


def pcg(apply_A, apply_Minv, b, tol, x0=None, maxiter=10000):
    """Preconditioned CG (Fletcher-Reeves beta), ||r|| <= tol ||b||; returns (x, it)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x)
    z = apply_Minv(r)
    p = z.copy()
    rz = r @ z
    bn = np.sqrt(b @ b)
    it = 0
    while np.sqrt(r @ r) > tol * bn and it < maxiter:
        q = apply_A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = apply_Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


# ------------------------------------------------------------ nu(x) field --
# With a viscosity field the spatial blocks are no longer polynomials in K, so
# the per-frequency systems of Alg. 1 are solved as sparse matrices.


def time_basis(nt, l):
    """Orthonormal eigenvectors Q (columns) and eigenvalues of D_tt with first
    entry l (Sec. 4.1: the DCT-VIII basis for l = 1, DST-I for l = 2), from
    LAPACK's symmetric eigensolver on the assembled N_t x N_t matrix."""
    lam, Q = np.linalg.eigh(Dtt(nt, l).toarray())
    return Q, lam


def _prec_blocks(prob):
    """C_hat = K_nu^2 + B B^T and L_hat = (K_nu + I/dt)/dt of eq. prec."""
    B, K = spatial(prob)
    Kv = viscous(prob, K)
    h = dt(prob)
    ident = sp.identity(Kv.shape[0])
    return (Kv @ Kv + B @ B.T).tocsc(), ((Kv + ident / h) / h).tocsc()


def precond_lu(prob, r):
    """P^{-1} r by Alg. 1: time transform (P = (Q (x) I) diag_k(C_hat +
    lambda_k L_hat) (Q^T (x) I) with D_tt = Q Lambda Q^T), one sparse LU solve
    per time frequency (the paper's first option for the per-step systems,
    Sec. 4.1 after Alg. 1), inverse time transform.  Any viscosity, l in {1, 2}."""
    if prob["l"] not in (1, 2):
        raise ValueError("precond_lu: l must be 1 or 2")
    nt = prob["nt"]
    Q, lam = time_basis(nt, prob["l"])
    Ch, Lh = _prec_blocks(prob)
    R = np.asarray(r, dtype=np.float64).reshape(nt, -1)
    Yh = Q.T @ R
    Xh = np.empty_like(Yh)
    for k in range(nt):
        Xh[k] = spla.splu((Ch + lam[k] * Lh).tocsc()).solve(Yh[k])
    return (Q @ Xh).reshape(-1)


def nu_ref(prob):
    """Reference viscosity of the constant-coefficient spatial solve that
    preconditions the per-frequency systems for a field nu(x): the geometric
    mean sqrt(min * max) of the live face viscosities (faces past a Neumann
    end excluded), the value that balances the extreme ratios nu_face/nu_ref."""
    vals = []
    for ax, f in enumerate(nu_faces(prob)):
        if prob["bc"][ax] != PERIODIC:
            idx = [slice(None), slice(None)]
            idx[ax] = slice(0, -1)
            f = f[tuple(idx)]
        vals.append(f.reshape(-1))
    v = np.concatenate(vals)
    return float(np.sqrt(v.min() * v.max()))


def _mbar_inv(prob, nub, lam_k, v):
    """(C_hat + lambda_k L_hat)^{-1} v for the constant viscosity nub: diagonal
    in the spatial eigenbasis of K (Alg. 2), eigenvalue
    nub^2 kappa^2 + 2 kappa + lambda_k (nub kappa + 1/dt)/dt."""
    nx, ny = prob["n"]
    kap = laplacian_eigs(prob)
    h = dt(prob)
    den = nub ** 2 * kap ** 2 + 2.0 * kap + lam_k * (nub * kap + 1.0 / h) / h
    vh = to_modes(prob, np.asarray(v, dtype=np.float64).reshape(1, nx, ny))
    return np.real(from_modes(prob, vh / den[None])).reshape(-1)


def precond_inner(prob, r, s):
    """Alg. 1 with inexact per-frequency solves: for each time frequency k,
    `s` steps of preconditioned CG on (C_hat + lambda_k L_hat) x = y_k from
    x = 0, preconditioned by the same block with the constant viscosity
    nu_ref(prob) (solved exactly in the spatial eigenbasis); s = 0 applies that
    constant-coefficient block alone.  A step whose curvature p.Mp is not
    positive, or whose r.z vanishes, contributes nothing (alpha = beta = 0).
    Exact for a constant field with s >= 1; tends to precond_lu as s grows."""
    nt = prob["nt"]
    Q, lam = time_basis(nt, prob["l"])
    Ch, Lh = _prec_blocks(prob)
    nub = nu_ref(prob)
    R = np.asarray(r, dtype=np.float64).reshape(nt, -1)
    Yh = Q.T @ R
    Xh = np.zeros_like(Yh)
    for k in range(nt):
        M = (Ch + lam[k] * Lh).tocsr()
        res = Yh[k].copy()
        z = _mbar_inv(prob, nub, lam[k], res)
        if s == 0:
            Xh[k] = z
            continue
        p = z.copy()
        rz = res @ z
        x = np.zeros_like(res)
        for i in range(s):
            q = M @ p
            pq = p @ q
            alpha = rz / pq if (pq > 0 and np.isfinite(pq)) else 0.0
            x += alpha * p
            if i == s - 1:
                break
            res -= alpha * q
            z = _mbar_inv(prob, nub, lam[k], res)
            rz_new = res @ z
            beta = rz_new / rz if rz > 0 else 0.0
            rz = rz_new
            p = z + beta * p
        Xh[k] = x
    return (Q @ Xh).reshape(-1)
