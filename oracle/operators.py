"""Sparse finite-difference operators, assembled straight from the paper.

Layout: a scalar field on one time plane is flattened (i, j) -> i*Ny + j (j
fastest, Sec. 4.3 ordering of y_k); a space-time field is (k, i, j) with k the
plane index 0..Nt-1.  The primal vector is c = 1 + 2*dim planes
(m, w1, w2[, w3, w4]) each of size n = Nt*Nx*Ny, where plane k of m holds
m^{k+1} and plane k of w holds w^k (pairing (m^{k+1}, w^k) of the scheme,
Sec. 2 eq. MFG_T2h).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

PERIODIC = "periodic"


def spacing(prob):
    """dx per axis: (b-a)/N periodic, (b-a)/(N+1) Neumann (Sec. 2, Sec. 4.3)."""
    res = []
    for ax in range(2):
        n, length, bc = prob["n"][ax], prob["len"][ax], prob["bc"][ax]
        res.append(length / n if bc == PERIODIC else length / (n + 1))
    return tuple(res)


def dt(prob):
    return prob["T"] / prob["nt"]


def div_blocks(n, bc):
    """Unscaled divergence blocks D^1, D^2 of Sec. 4.3 (N x N each).

    Periodic: D^1 has 1 on the diagonal, -1 below it and -1 in the top-right
    corner; D^2 = -(D^1)^T.  Neumann ("Dirichlet-type"): D^1 is the same without
    the corner and with a 0 in its last diagonal entry; D^2 has -1 on the diagonal
    except a 0 in its first entry, and 1 above it.
    """
    if bc == PERIODIC:
        d1 = sp.lil_matrix((n, n))
        for i in range(n):
            d1[i, i] = 1.0
            d1[i, (i - 1) % n] += -1.0
        d1 = d1.tocsr()
        d2 = (-d1.T).tocsr()
        return d1, d2
    d1 = sp.lil_matrix((n, n))
    d2 = sp.lil_matrix((n, n))
    for i in range(n):
        if i < n - 1:
            d1[i, i] = 1.0
        if i >= 1:
            d1[i, i - 1] = -1.0
        if i >= 1:
            d2[i, i] = -1.0
        if i + 1 < n:
            d2[i, i + 1] = 1.0
    return d1.tocsr(), d2.tocsr()


def spatial(prob):
    """Per-time-step spatial operators: (B, K) with B = div_h (Nx*Ny x (2*dim)*Nx*Ny,
    w components (w1, w2[, w3, w4]) stacked) and K the negative Laplacian built as
    D^1 (D^1)^T / dx^2 per axis, Kronecker-summed (Sec. 4.3)."""
    nx, ny = prob["n"]
    dx, dy = spacing(prob)
    d1x, d2x = div_blocks(nx, prob["bc"][0])
    kx = (d1x @ d1x.T) / dx ** 2
    if prob["dim"] == 1:
        B = sp.hstack([d1x / dx, d2x / dx]).tocsr()
        return B, sp.csr_matrix(kx)
    d1y, d2y = div_blocks(ny, prob["bc"][1])
    ky = (d1y @ d1y.T) / dy ** 2
    Ix, Iy = sp.identity(nx), sp.identity(ny)
    B = sp.hstack([sp.kron(d1x, Iy) / dx, sp.kron(d2x, Iy) / dx,
                   sp.kron(Ix, d1y) / dy, sp.kron(Ix, d2y) / dy]).tocsr()
    K = (sp.kron(kx, Iy) + sp.kron(Ix, ky)).tocsr()
    return B, K


def has_nu_field(prob):
    """True when the problem carries a viscosity field nu(x) (prob["nu_field"],
    one value per node, shape (Nx, Ny)) instead of the constant prob["nu"]."""
    return prob.get("nu_field") is not None


def nu_faces(prob):
    """Face viscosities of a field nu(x): on each active axis, face i sits
    between node i and node i+1 (wrapping on a periodic axis) and takes the
    arithmetic mean of the two node values; the face past the end of a Neumann
    axis joins no second node and carries 0.  Returns one (Nx, Ny) array per
    active axis (x, then y in 2-D)."""
    nx, ny = prob["n"]
    nu = np.asarray(prob["nu_field"], dtype=np.float64).reshape(nx, ny)
    out = []
    for ax in range(prob["dim"]):
        nb = np.roll(nu, -1, axis=ax)
        f = 0.5 * (nu + nb)
        if prob["bc"][ax] != PERIODIC:
            idx = [slice(None), slice(None)]
            idx[ax] = -1
            f[tuple(idx)] = 0.0
        out.append(f)
    return out


def K_nu(prob):
    """Variable-coefficient negative Laplacian -div(nu grad) in the paper's
    difference form: per axis D^1 diag(nu_face) (D^1)^T / dx^2 with the D^1
    blocks of Sec. 4.3 (columns = faces, face i between nodes i and i+1), summed
    over the axes as K is.  A constant field gives nu K exactly.  The paper
    allows nu(x) without fixing its discretisation (Sec. 4, before Sec. 4.1);
    this is the symmetric conservative reading, which keeps L symmetric so
    that C = L^2 + B B^T and the block forms of Sec. 4.1 hold unchanged."""
    nx, ny = prob["n"]
    dx, dy = spacing(prob)
    faces = nu_faces(prob)
    d1x, _ = div_blocks(nx, prob["bc"][0])
    if prob["dim"] == 1:
        return (d1x @ sp.diags(faces[0].reshape(-1)) @ d1x.T / dx ** 2).tocsr()
    d1y, _ = div_blocks(ny, prob["bc"][1])
    Dx = sp.kron(d1x, sp.identity(ny))
    Dy = sp.kron(sp.identity(nx), d1y)
    return (Dx @ sp.diags(faces[0].reshape(-1)) @ Dx.T / dx ** 2 +
            Dy @ sp.diags(faces[1].reshape(-1)) @ Dy.T / dy ** 2).tocsr()


def viscous(prob, K=None):
    """The viscous term of L: nu K for a constant nu, K_nu for a field."""
    if has_nu_field(prob):
        return K_nu(prob)
    if K is None:
        _, K = spatial(prob)
    return (prob["nu"] * K).tocsr()


def L_matrix(prob, K=None):
    """L = nu K + I/dt (Sec. 3, below the matrices A and B); K_nu + I/dt for a
    viscosity field."""
    Kv = viscous(prob, K)
    return (Kv + sp.identity(Kv.shape[0]) / dt(prob)).tocsr()


def constraint(prob):
    """Reduced constraint matrix C = [A_red | B_red] (Sec. 3 eq. ABC with the
    initial-condition block row eliminated): block row k (k = 0..Nt-1) reads
    L m^{k+1} - m^k/dt + div_h w^k, and the m^0 = m0 term moves to d."""
    nt = prob["nt"]
    B, K = spatial(prob)
    L = L_matrix(prob, K)
    s = K.shape[0]
    shift = sp.diags([np.ones(nt - 1)], [-1], shape=(nt, nt))
    A_red = sp.kron(sp.identity(nt), L) - sp.kron(shift, sp.identity(s)) / dt(prob)
    ncomp = B.shape[1] // s
    Bcols = [sp.kron(sp.identity(nt), B[:, c * s:(c + 1) * s]) for c in range(ncomp)]
    return sp.hstack([A_red] + Bcols).tocsr()


def apply_C_planes(prob, v):
    """C v without assembling C (for grids too large to assemble): plane by
    plane, row k = L m^{k+1} - m^k/dt + div_h w^k with the m^0 term excluded
    (it belongs to d), using the spatial blocks B, K of `spatial`.  Pinned
    against `constraint(prob) @ v` on small grids."""
    nt = prob["nt"]
    B, K = spatial(prob)
    s = K.shape[0]
    c = n_planes(prob)
    v = np.asarray(v, dtype=np.float64).reshape(c, nt, s)
    m = v[0]
    w = np.concatenate([v[q] for q in range(1, c)], axis=1)  # (nt, (c-1) s) in the w order of B
    h = dt(prob)
    Kv = viscous(prob, K)
    out = (Kv @ m.T).T + m / h + (B @ w.T).T
    out[1:] -= m[:-1] / h
    return out.reshape(-1)


def apply_Ct_planes(prob, p):
    """C^T p without assembling C: the m rows L p^k - p^{k+1}/dt (p^{Nt} = 0)
    and the w rows B^T p^k, plane by plane.  Pinned against
    `constraint(prob).T @ p` on small grids."""
    nt = prob["nt"]
    B, K = spatial(prob)
    s = K.shape[0]
    c = n_planes(prob)
    p = np.asarray(p, dtype=np.float64).reshape(nt, s)
    h = dt(prob)
    xm = (viscous(prob, K) @ p.T).T + p / h
    xm[:-1] -= p[1:] / h
    xw = (B.T @ p.T).T  # (nt, (c-1) s)
    out = np.empty((c, nt, s))
    out[0] = xm
    for q in range(1, c):
        out[q] = xw[:, (q - 1) * s:q * s]
    return out.reshape(-1)


def rhs_d(prob, m0):
    """d = (m0/dt, 0, ..., 0): the initial datum moved to the right-hand side."""
    nx, ny = prob["n"]
    d = np.zeros((prob["nt"], nx * ny))
    d[0] = np.asarray(m0, dtype=np.float64).reshape(-1) / dt(prob)
    return d.reshape(-1)


def AAt(prob, C=None):
    """The reduced SPD matrix C C^T, formed by a sparse product (eq. largeA is a check)."""
    if C is None:
        C = constraint(prob)
    return (C @ C.T).tocsr()


def Dtt(nt, l):
    """Negative second difference in time with first entry l (Sec. 4.1)."""
    D = sp.diags([-np.ones(nt - 1), 2.0 * np.ones(nt), -np.ones(nt - 1)], [-1, 0, 1]).tolil()
    D[0, 0] = float(l)
    return D.tocsr()


def precond(prob):
    """P = I_Nt (x) C_hat + D_tt (x) L_hat with C_hat = nu^2 K^2 + B B^T and
    L_hat = L/dt (Sec. 4.1 eq. prec and its Kronecker form); for a viscosity
    field nu K becomes K_nu, so C_hat = K_nu^2 + B B^T."""
    B, K = spatial(prob)
    L = L_matrix(prob, K)
    Kv = viscous(prob, K)
    C_hat = Kv @ Kv + B @ B.T
    L_hat = L / dt(prob)
    nt = prob["nt"]
    return (sp.kron(sp.identity(nt), C_hat) + sp.kron(Dtt(nt, prob["l"]), L_hat)).tocsr()


def n_planes(prob):
    return 1 + 2 * prob["dim"]


def sizes(prob):
    nx, ny = prob["n"]
    s = nx * ny
    return s, prob["nt"] * s, n_planes(prob)
