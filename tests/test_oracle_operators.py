"""Pins of the oracle's sparse operators against what the paper fixes."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import mfg_inputs as mi
from oracle import operators as ops

GOLD = os.path.join(os.path.dirname(__file__), "golden", "div_blocks_N5.txt")


def _golden():
    mats, name, rows = {}, None, []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            if name:
                mats[name] = np.array(rows, dtype=float)
            name, rows = line, []
        else:
            rows.append([float(t) for t in line.split()])
    mats[name] = np.array(rows, dtype=float)
    return mats


def test_div_blocks_match_printed_matrices():
    g = _golden()
    d1, d2 = ops.div_blocks(5, "periodic")
    np.testing.assert_array_equal(d1.toarray(), g["periodic_D1"])
    np.testing.assert_array_equal(d2.toarray(), -g["periodic_D1"].T)
    np.testing.assert_array_equal((d1 @ d1.T).toarray(), g["periodic_DDt"])
    np.testing.assert_array_equal((d2 @ d2.T).toarray(), g["periodic_DDt"])
    n1, n2 = ops.div_blocks(5, "neumann")
    np.testing.assert_array_equal(n1.toarray(), g["neumann_D1"])
    np.testing.assert_array_equal(n2.toarray(), g["neumann_D2"])
    np.testing.assert_array_equal((n1 @ n1.T).toarray(), g["neumann_DDt"])
    np.testing.assert_array_equal((n2 @ n2.T).toarray(), g["neumann_DDt"])


def test_div_matches_div_h_definition():
    """B w equals the Sec. 2 formula (div_h w)_ij on a periodic grid."""
    inst = mi.small(11, nx=7, ny=6, bc=("periodic", "periodic"))
    p = inst["problem"]
    B, _ = ops.spatial(p)
    dx, dy = ops.spacing(p)
    w = mi.random_field((4, 7, 6), 5)
    ref = ((w[0] - np.roll(w[0], 1, 0)) / dx + (np.roll(w[1], -1, 0) - w[1]) / dx
           + (w[2] - np.roll(w[2], 1, 1)) / dy + (np.roll(w[3], -1, 1) - w[3]) / dy)
    np.testing.assert_allclose(B @ w.reshape(-1), ref.reshape(-1), rtol=0, atol=1e-12)


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("neumann", "neumann"),
                                ("periodic", "neumann"), ("neumann", "periodic")])
@pytest.mark.parametrize("dim", [1, 2])
def test_BBt_is_2K_and_mass_conserving(bc, dim):
    inst = mi.small(3, dim=dim, nx=9, ny=7, bc=bc)
    B, K = ops.spatial(inst["problem"])
    assert abs(B @ B.T - 2 * K).max() < 1e-9 * abs(K).max()    # eq. precstead
    one = np.ones(K.shape[0])
    assert np.abs(one @ B).max() < 1e-9 * abs(B).max()
    assert np.abs(one @ K).max() < 1e-9 * abs(K).max()


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_laplacian_eigenvalues_textbook(bc):
    n = 11
    d1, _ = ops.div_blocks(n, bc)
    ev = np.sort(np.linalg.eigvalsh((d1 @ d1.T).toarray()))
    v = np.arange(n)
    ref = 2 - 2 * np.cos((2 if bc == "periodic" else 1) * np.pi * v / n)
    np.testing.assert_allclose(ev, np.sort(ref), atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_AAt_block_form(seed):
    """C C^T equals eq. largeA: C = L^2 + B B^T on the first diagonal block,
    C + I/dt^2 below it, -L/dt off the diagonal."""
    p = mi.small(seed)["problem"]
    A = ops.AAt(p).toarray()
    B, K = ops.spatial(p)
    L = ops.L_matrix(p, K).toarray()
    s = K.shape[0]
    h = ops.dt(p)
    Cb = L @ L + (B @ B.T).toarray()
    nt = p["nt"]
    ref = np.zeros((nt * s, nt * s))
    for k in range(nt):
        ref[k*s:(k+1)*s, k*s:(k+1)*s] = Cb + (np.eye(s) / h ** 2 if k > 0 else 0)
        if k + 1 < nt:
            ref[k*s:(k+1)*s, (k+1)*s:(k+2)*s] = -L / h
            ref[(k+1)*s:(k+2)*s, k*s:(k+1)*s] = -L / h
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_uniform_density_is_feasible():
    """m^k = m0 uniform, w = 0 satisfies the discrete Fokker-Planck constraint."""
    for seed in (1, 2, 5):
        inst = mi.small(seed)
        p = inst["problem"]
        nx, ny = p["n"]
        m0 = np.full((nx, ny), 1.0 / (nx * ny * mi.cell_volume(p)))
        y = mi.initial_iterate(p, m0)
        res = ops.constraint(p) @ y.reshape(-1) - ops.rhs_d(p, m0)
        assert np.abs(res).max() < 1e-10 * np.abs(ops.rhs_d(p, m0)).max()


@pytest.mark.parametrize("l", [1, 2])
@pytest.mark.parametrize("nt", [3, 8, 13])
def test_time_eigenvalues_formula(l, nt):
    """eq. eigs: lambda_k = 2 - 2 cos(pi (k-1+l/2)/(N_t+l/2))."""
    ev = np.sort(np.linalg.eigvalsh(ops.Dtt(nt, l).toarray()))
    k = np.arange(1, nt + 1)
    ref = 2 - 2 * np.cos(np.pi * (k - 1 + l / 2) / (nt + l / 2))
    np.testing.assert_allclose(ev, np.sort(ref), atol=1e-12)


def test_precond_exact_at_zero_viscosity():
    """Sec. 4.2: with nu = 0 and l = 1, P = AAt."""
    for seed in (1, 2, 3):
        p = dict(mi.small(seed, nu=0.0, l=1)["problem"])
        A = ops.AAt(p)
        P = ops.precond(p)
        assert abs(A - P).max() < 1e-10 * abs(A).max()


@pytest.mark.parametrize("l", [1, 2])
def test_lemma1_unit_eigenvalues(l):
    """Lemma 1: P^{-1} AAt has eigenvalue 1 with multiplicity >= (N_t-1) N_x N_y."""
    p = mi.small(7, nx=4, ny=3, nt=5, nu=0.3, l=l)["problem"]
    A = ops.AAt(p).toarray()
    P = ops.precond(p).toarray()
    ev = sla.eigvals(A, P).real
    s = 12
    assert np.sum(np.abs(ev - 1) < 1e-8) >= (p["nt"] - 1) * s
    assert ev.min() > 0


def test_nonunit_eigenvalues_closed_form():
    """Derived: per spatial mode, AAt_s - P_s = delta_s e1 e1^T with
    delta_s = nu kappa_s/dt (l = 1), so the non-unit eigenvalue is
    1 + delta_s * sum_k V_k1^2 / (C_hat_s + lambda_k L_hat_s); this is the
    spectrum of Fig. eigstime shifted by one."""
    p = mi.small(8, nx=6, ny=5, nt=6, nu=0.1, l=1, bc=("periodic", "neumann"))["problem"]
    A = ops.AAt(p).toarray()
    P = ops.precond(p).toarray()
    ev = np.sort(sla.eigvals(A, P).real)
    B, K = ops.spatial(p)
    kap = np.linalg.eigvalsh(K.toarray())
    h = ops.dt(p)
    lam, Vt = np.linalg.eigh(ops.Dtt(p["nt"], 1).toarray())
    Lh = (p["nu"] * kap + 1 / h) / h
    Ch = p["nu"] ** 2 * kap ** 2 + 2 * kap
    delta = p["nu"] * kap / h
    mu = 1 + delta * np.array([np.sum(Vt[0] ** 2 / (c + lam * lh)) for c, lh in zip(Ch, Lh)])
    ref = np.sort(np.concatenate([mu, np.ones((p["nt"] - 1) * K.shape[0])]))
    np.testing.assert_allclose(ev, ref, atol=1e-9)
    assert ev.max() <= 1.25 + 1e-9


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("neumann", "neumann"), ("periodic", "neumann")])
@pytest.mark.parametrize("dim", [1, 2])
def test_planewise_C_and_Ct_match_assembled(bc, dim):
    """The matrix-free plane-by-plane C and C^T (used at full size) equal the
    assembled reduced constraint matrix and its transpose."""
    p = mi.small(29, dim=dim, bc=bc, nx=7, ny=6, nt=5)["problem"]
    C = ops.constraint(p)
    v = mi.random_field(C.shape[1], 3)
    z = mi.random_field(C.shape[0], 4)
    np.testing.assert_allclose(ops.apply_C_planes(p, v), C @ v, rtol=0, atol=1e-12 * np.abs(C @ v).max())
    np.testing.assert_allclose(ops.apply_Ct_planes(p, z), C.T @ z, rtol=0, atol=1e-12 * np.abs(C.T @ z).max())
