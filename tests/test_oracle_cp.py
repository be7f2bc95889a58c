"""Pins of the oracle Chambolle-Pock loop against facts fixed by the problem:
the trivial equilibrium, a vanishing duality gap and constraint residual, mass
conservation, and solver independence."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import checks
from oracle import operators as ops
from oracle.cp import Solver


def _uniform_instance(seed, bc, dim=2):
    inst = mi.small(seed, dim=dim, nx=6, ny=5, nt=5, bc=bc, nu=0.1, g_a=0.3)
    p = dict(inst["problem"], gamma=0.05)
    nx, ny = p["n"]
    m0 = np.full((nx, ny), 1.0 / (nx * ny * mi.cell_volume(p)))
    V = np.full((nx, ny), 0.4)
    W = np.full((nx, ny), -0.2)
    y0 = mi.initial_iterate(p, m0, eps=0.05, seed=seed)
    return p, m0, V, W, y0


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("neumann", "neumann")])
@pytest.mark.parametrize("dim", [1, 2])
def test_trivial_equilibrium(bc, dim):
    """Uniform m0 with x-independent f and g: the minimiser is m = m0, w = 0
    (mass is conserved and F is convex, so Jensen's inequality gives the bound;
    b_hat >= 0 vanishes only at w = 0)."""
    p, m0, V, W, y0 = _uniform_instance(3, bc, dim)
    res = Solver(p, m0, V, W).run(y0, iters=1500)
    y = res["y"]
    assert np.abs(y[0] - m0[None]).max() < 1e-6 * m0.max()
    assert np.abs(y[1:]).max() < 1e-6
    z = res["z"]
    # u ~ -z is spatially constant at the equilibrium
    assert np.abs(z - z.mean(axis=(1, 2), keepdims=True)).max() < 1e-5 * max(1, np.abs(z).max())


@pytest.mark.parametrize("seed", [1, 2])
def test_gap_and_feasibility_vanish(seed):
    inst = mi.small(seed, nx=5, ny=4, nt=4, nu=0.2, eps=0.0)
    p = dict(inst["problem"], gamma=0.05)
    s = Solver(p, inst["m0"], inst["V"], inst["W"])
    early = s.run(inst["y0"], iters=20)
    late = s.run(inst["y0"], iters=3000)
    for res, tol_gap, tol_c in ((late, 1e-6, 1e-7),):
        cres = checks.constraint_residual(p, res["y"], inst["m0"])
        dnorm = np.linalg.norm(ops.rhs_d(p, inst["m0"]))
        assert np.linalg.norm(cres) <= tol_c * dnorm
        g = checks.gap(p, res["y"], res["z"], inst["m0"], inst["V"], inst["W"])
        obj = checks.objective(p, res["y"], inst["V"], inst["W"])
        assert abs(g) <= tol_gap * max(1.0, abs(obj))
        np.testing.assert_allclose(checks.mass(p, res["y"]), 1.0, atol=1e-8)
    # residual and mass error decrease along the run
    c_early = np.linalg.norm(checks.constraint_residual(p, early["y"], inst["m0"]))
    c_late = np.linalg.norm(checks.constraint_residual(p, late["y"], inst["m0"]))
    assert c_late < 1e-3 * c_early


def test_conjugate_matches_numerical_sup():
    """phi*(alpha, beta) = sup_{m,w} alpha m + beta.w - phi(m, w), checked on a grid."""
    inst = mi.small(4, nx=1, ny=1, nt=2)
    p = dict(inst["problem"], n=(1, 1))
    rng = np.random.default_rng(0)
    from scipy.optimize import minimize_scalar
    V = np.array([[0.3]])
    W = np.array([[0.0]])
    from oracle.prox import coupling, project_K
    a, b, c = coupling(p, V, W)
    for _ in range(20):
        alpha = rng.normal() * 2
        beta = rng.normal(size=4)
        P2 = (project_K(beta) ** 2).sum()
        # sup over w in closed form m |P|^2/2, sup over m numerically
        f = lambda m: -(alpha * m + m * P2 / 2 - 0.5 * a[0, 0, 0] * m * m - c[0, 0, 0] * m)
        r = minimize_scalar(f, bounds=(0, 1e3), method="bounded", options={"xatol": 1e-12})
        num = max(-r.fun, 0.0)
        ours = checks.conjugate_cells(p, np.full((2, 1, 1), alpha),
                                      np.broadcast_to(beta[:, None, None, None], (4, 2, 1, 1)), V, W)[0, 0, 0]
        assert abs(ours - num) <= 1e-8 * max(1, num)


def test_lu_and_modal_agree():
    inst = mi.small(12, nx=8, ny=6, nt=5)
    p = inst["problem"]
    r1 = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=25)
    r2 = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=25)
    assert np.linalg.norm(r1["y"] - r2["y"]) <= 1e-10 * np.linalg.norm(r1["y"])


def _small_cp_problem(**kw):
    import mfg_inputs as mi
    inst = mi.small(7, dim=2, nx=8, ny=12, nt=10, bc=("periodic", "neumann"), **kw)
    return inst


def test_pcg_inner_solve_matches_exact_solve():
    """The inexact inner solve of Sec. 5 (PCG with the paper's P, warm start)
    reproduces the exact-solve iterate when its tolerance is at round-off, for
    both stop references and both time transforms."""
    import numpy as np
    from oracle.cp import Solver
    for l in (1, 2):
        inst = _small_cp_problem(l=l)
        p = dict(inst["problem"], cg_tol=1e-13, cg_rule=0)
        ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=15)
        for cg_ref in ("resid", "rhs"):
            got = Solver(p, inst["m0"], inst["V"], inst["W"], method="pcg", cg_ref=cg_ref).run(inst["y0"], iters=15)
            assert np.linalg.norm(got["y"] - ref["y"]) <= 1e-9 * np.linalg.norm(ref["y"])
            assert len(got["cg"]) == 15 and min(got["cg"]) >= 1


def test_pcg_inner_solve_counts():
    """Stop relative to the full right-hand side never needs more iterations
    than stop relative to the warm-start residual (the full right-hand side is
    the larger reference once z is warm); with nu = 0 and l = 1, P equals
    C C^T (Sec. 4.2) and every solve takes at most one iteration."""
    import numpy as np
    from oracle.cp import Solver
    inst = _small_cp_problem(l=1)
    p = dict(inst["problem"], cg_rule=1, cg_tol=1e-10)
    a = Solver(p, inst["m0"], inst["V"], inst["W"], method="pcg", cg_ref="resid").run(inst["y0"], iters=20)
    b = Solver(p, inst["m0"], inst["V"], inst["W"], method="pcg", cg_ref="rhs").run(inst["y0"], iters=20)
    assert sum(b["cg"]) <= sum(a["cg"])
    inst0 = _small_cp_problem(l=1, nu=0.0)
    p0 = dict(inst0["problem"], cg_rule=0, cg_tol=1e-12)
    c = Solver(p0, inst0["m0"], inst0["V"], inst0["W"], method="pcg").run(inst0["y0"], iters=5)
    assert max(c["cg"]) <= 1


def test_matrix_free_solver_matches_assembled():
    """The CP loop with the plane-by-plane C / C^T (used on grids too large to
    assemble) gives the assembled-matrix iterate to round-off, with any thread
    count."""
    import oracle
    inst = mi.small(7, nx=9, ny=8, nt=6, nu=0.1)
    p = inst["problem"]
    a = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=12)
    oracle.set_threads(1)
    try:
        b = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal", matrix_free=True).run(inst["y0"], iters=12)
    finally:
        oracle.set_threads()
    assert np.linalg.norm(a["y"] - b["y"]) <= 1e-12 * np.linalg.norm(a["y"])
    assert np.linalg.norm(a["x"] - b["x"]) <= 1e-12 * np.linalg.norm(a["x"])
