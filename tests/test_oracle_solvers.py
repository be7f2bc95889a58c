"""Pins of the oracle's solvers: the spatially-diagonalised exact solver and the
exact P^{-1} against sparse LU, CG against LU, PCG behaviour fixed by the paper."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle import solvers

BCS = [("periodic", "periodic"), ("neumann", "neumann"), ("periodic", "neumann"),
       ("neumann", "periodic")]


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("dim", [1, 2])
def test_modal_AAt_solve_matches_lu(bc, dim):
    inst = mi.small(21, dim=dim, bc=bc, nx=9, ny=6, nt=7)
    p = inst["problem"]
    A = ops.AAt(p)
    b = mi.random_field(A.shape[0], 4)
    z_lu = solvers.solve_direct(A, b)
    z_md = solvers.solve_AAt_modal(p, b)
    assert np.linalg.norm(z_md - z_lu) <= 1e-9 * np.linalg.norm(z_lu)
    assert np.linalg.norm(A @ z_md - b) <= 1e-12 * np.linalg.norm(b) * 10


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("l", [1, 2])
def test_modal_precond_matches_lu(bc, l):
    p = mi.small(5, bc=bc, nx=8, ny=5, nt=6, l=l)["problem"]
    P = ops.precond(p)
    r = mi.random_field(P.shape[0], 9)
    z_lu = solvers.solve_direct(P, r)
    z_md = solvers.precond_modal(p, r)
    assert np.linalg.norm(z_md - z_lu) <= 1e-10 * np.linalg.norm(z_lu)


def test_cg_matches_lu():
    p = mi.small(2, nx=6, ny=5, nt=4, nu=0.05)["problem"]
    A = ops.AAt(p)
    b = mi.random_field(A.shape[0], 1)
    x, it = solvers.solve_cg(A, b, tol=1e-13)
    z = solvers.solve_direct(A, b)
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(x - z) <= 1e-7 * np.linalg.norm(z)


def test_modal_residual_medium_grid():
    """32 x 32 x 16 periodic/Neumann: residual of the exact solver at round-off."""
    for bc in [("periodic", "periodic"), ("neumann", "neumann")]:
        p = mi.small(4, nx=32, ny=32, nt=16, bc=bc, nu=0.1)["problem"]
        A = ops.AAt(p)
        b = mi.random_field(A.shape[0], 2)
        z = solvers.solve_AAt_modal(p, b)
        assert np.linalg.norm(A @ z - b) <= 1e-11 * np.linalg.norm(b)


def test_pcg_one_iteration_when_exact():
    """Sec. 4.2: nu = 0, l = 1 gives P = AAt, so PCG stops after one iteration."""
    p = mi.small(6, nu=0.0, l=1, nx=10, ny=8, nt=6)["problem"]
    A = ops.AAt(p)
    b = mi.random_field(A.shape[0], 3)
    x, it = solvers.pcg(lambda v: A @ v, lambda r: solvers.precond_modal(p, r), b, 1e-12)
    assert it == 1
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("l,cap", [(1, 12), (2, 60)])
def test_pcg_iterations_bounded(l, cap):
    """With the recursive preconditioner PCG needs few iterations (Tables 1-3:
    average CG counts of 2-6 for l = 1 and 7-40 for l = 2 at tolerances <= 1e-4)."""
    p = mi.small(6, nu=0.01, l=l, nx=16, ny=16, nt=32, bc=("periodic", "periodic"))["problem"]
    A = ops.AAt(p)
    b = mi.random_field(A.shape[0], 3)
    x, it = solvers.pcg(lambda v: A @ v, lambda r: solvers.precond_modal(p, r), b, 1e-10)
    assert it <= cap
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.0001


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("dim", [1, 2])
def test_modal_applies_match_sparse(bc, dim):
    """The matrix-free applies of AAt and P through the spatial eigenbasis equal
    the assembled sparse matrices."""
    p = mi.small(17, dim=dim, bc=bc, nx=9, ny=7, nt=6)["problem"]
    v = mi.random_field(ops.sizes(p)[1], 5)
    A = ops.AAt(p)
    P = ops.precond(p)
    assert np.linalg.norm(solvers.apply_AAt_modal(p, v) - A @ v) <= 1e-12 * np.linalg.norm(A @ v)
    Pv, lam = solvers.apply_P_modal(p, v)
    assert np.linalg.norm(Pv - P @ v) <= 1e-12 * np.linalg.norm(P @ v)
    assert lam >= np.abs(np.linalg.eigvalsh(P.toarray())).max() * (1 - 1e-12)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("dim", [1, 2])
def test_eig_range_matches_dense_spectrum(bc, dim):
    """The per-mode tridiagonal spectrum of AAt equals the dense eigenvalues of
    the assembled C C^T (extremes, to round-off)."""
    p = mi.small(23, dim=dim, bc=bc, nx=7, ny=6, nt=5)["problem"]
    ev = np.linalg.eigvalsh(ops.AAt(p).toarray())
    lo, hi = solvers.eig_range_AAt(p)
    assert abs(lo - ev.min()) <= 1e-9 * ev.min()
    assert abs(hi - ev.max()) <= 1e-12 * ev.max()
    assert abs(solvers.cond_AAt(p) - ev.max() / ev.min()) <= 1e-8 * ev.max() / ev.min()
