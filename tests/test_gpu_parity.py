"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs: operators, preconditioner, prox and the CP iterate.

Tolerances: operator applies are single FP64 stencil evaluations, compared in
relative l2 and l_inf at 1e-12.  The preconditioner solve z = P^{-1} r is
compared by its normwise backward error
  eta = ||P z - r||_inf / (||P||_inf ||z||_inf + ||r||_inf)
against the oracle's assembled P: orthonormal transforms make the apply
backward stable with eta = O(N u), u the unit round-off of the transforms
(1e-12 for FP64, 5e-5 for FP32), while the forward error also carries the
condition number of P (up to ~1e8 here), so it is checked only loosely.
The CP iterate after a fixed count is compared at 1e-8 relative l2 (the target
stated for the method, with PCG at relative tolerance 1e-10)."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle import solvers
from oracle.cp import Solver
from oracle.prox import prox as oracle_prox

from _gpu_helpers import cp_bound, dev, host, lib, linf_rel, rel

pytestmark = pytest.mark.gpu

# ragged sizes spanning several 8 x 32 stencil tiles and several time chunks
CASES = [
    dict(seed=1, dim=2, nx=19, ny=45, nt=11, bc=("periodic", "periodic")),
    dict(seed=2, dim=2, nx=17, ny=33, nt=9, bc=("neumann", "neumann")),
    dict(seed=3, dim=2, nx=10, ny=70, nt=7, bc=("periodic", "neumann")),
    dict(seed=4, dim=2, nx=25, ny=12, nt=13, bc=("neumann", "periodic")),
    dict(seed=5, dim=1, nx=67, nt=12, bc=("periodic", "periodic")),
    dict(seed=6, dim=1, nx=40, nt=9, bc=("neumann", "periodic")),
]


# power-of-two axes take the FFT spatial passes; N_t in {32, 64} the fixed-size time pass
POW2 = [
    dict(seed=21, dim=2, nx=16, ny=32, nt=32, bc=("periodic", "periodic")),
    dict(seed=22, dim=2, nx=32, ny=8, nt=64, bc=("neumann", "neumann")),
    dict(seed=23, dim=2, nx=8, ny=64, nt=16, bc=("periodic", "neumann")),
    dict(seed=24, dim=2, nx=64, ny=16, nt=8, bc=("neumann", "periodic")),
    dict(seed=25, dim=1, nx=128, nt=32, bc=("neumann", "periodic")),
    dict(seed=26, dim=1, nx=256, nt=32, bc=("periodic", "periodic")),
]


def _inst(case, **kw):
    c = dict(case)
    c.update(kw)
    return mi.small(**c)


def _backward_error(A, x, b):
    res = np.abs(A @ x - b).max()
    nA = np.abs(A).sum(axis=1).max()
    return res / (nA * np.abs(x).max() + np.abs(b).max())


def _plan(prob, precision="fp64"):
    return lib().mfg_plan(dict(prob), precision=precision)


@pytest.mark.parametrize("case", CASES)
def test_apply_C_Ct_AAt(case):
    import torch
    inst = _inst(case)
    p = inst["problem"]
    L = lib()
    plan = _plan(p)
    s, n, c = ops.sizes(p)
    C = ops.constraint(p)
    v = mi.random_field(c * n, 11)
    pv = mi.random_field(n, 12)
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    x = torch.empty(c * n, dtype=torch.float64, device="cuda")
    q = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_C(plan, 0, dev(v), r)
    L.mfg_apply_Ct(plan, 0, dev(pv), x)
    L.mfg_apply_AAt(plan, 0, dev(pv), q)
    torch.cuda.synchronize()
    ref_r, ref_x = C @ v, C.T @ pv
    ref_q = ops.AAt(p, C) @ pv
    for got, ref in ((host(r), ref_r), (host(x), ref_x), (host(q), ref_q)):
        assert rel(got, ref) <= 1e-12
        assert linf_rel(got, ref) <= 1e-12
    # the double-float stencil (about 48 significant bits) of MFG_MIXED_DF
    plan_df = _plan(p, "mixed_df")
    L.mfg_apply_AAt(plan_df, 0, dev(pv), q)
    torch.cuda.synchronize()
    assert rel(host(q), ref_q) <= 1e-12
    assert linf_rel(host(q), ref_q) <= 1e-12


@pytest.mark.parametrize("case", CASES + POW2)
@pytest.mark.parametrize("l", [0, 1, 2])
def test_precond_fp64(case, l):
    """l = 1, 2: the paper's P (eq. prec); l = 0: the exact variant, P = AAt."""
    import torch
    inst = _inst(case, l=l)
    p = inst["problem"]
    plan = _plan(p)
    n = ops.sizes(p)[1]
    r = mi.random_field(n, 21)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    lib().mfg_apply_precond(plan, 0, dev(r), z)
    torch.cuda.synchronize()
    P = ops.AAt(p) if l == 0 else ops.precond(p)
    zg = host(z)
    assert _backward_error(P, zg, r) <= 1e-12
    assert rel(zg, solvers.solve_direct(P, r)) <= 1e-6


@pytest.mark.parametrize("case", CASES[:4] + POW2)
def test_precond_fp32(case):
    import torch
    inst = _inst(case, l=1)
    p = inst["problem"]
    plan = _plan(p, "mixed")
    n = ops.sizes(p)[1]
    r = mi.random_field(n, 22)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    lib().mfg_apply_precond(plan, 0, dev(r), z)
    torch.cuda.synchronize()
    P = ops.precond(p)
    zg = host(z)
    assert _backward_error(P, zg, r) <= 5e-5
    assert rel(zg, solvers.solve_direct(P, r)) <= 1e-2


@pytest.mark.parametrize("case", CASES)
def test_prox(case):
    import torch
    inst = _inst(case)
    p = inst["problem"]
    plan = _plan(p)
    s, n, c = ops.sizes(p)
    v = mi.random_field((c, p["nt"]) + tuple(p["n"]), 31, -2.0, 2.0)
    v[0] += 0.5
    y = torch.empty(c * n, dtype=torch.float64, device="cuda")
    for tau in (0.05, 1.0):
        lib().mfg_prox(plan, 0, tau, dev(v), dev(inst["V"]), dev(inst["W"]), y)
        torch.cuda.synchronize()
        ref = oracle_prox(p, tau, v, inst["V"], inst["W"]).reshape(-1)
        got = host(y)
        assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
        assert np.all(got[:n] >= 0)


def _gpu_cp(inst, iters, precision="fp64", cg_tol=1e-10, **kw):
    import torch
    p = dict(inst["problem"], max_cp=iters, cg_tol=cg_tol, **kw)
    L = lib()
    plan = L.mfg_plan(p, precision=precision)
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    return rc, st[0], host(y), host(ybar), host(z)


@pytest.mark.parametrize("case", CASES + POW2[:3])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
def test_cp_iterate(case, precision):
    """PCG at 1e-12 so that the comparison isolates the implementation.

    Bound: max(1e-8, 10 kappa u) with kappa = cond(AAt) and u = 2^-53.  Every
    exact solve with AAt carries a relative error up to ~kappa u, and the oracle's
    own two exact solvers (LU and spatially diagonalised) already differ by that
    much on the stiffest case here (kappa ~ 1e8)."""
    inst = _inst(case)
    p = inst["problem"]
    iters = 25
    rc, st, y, ybar, z = _gpu_cp(inst, iters, precision, cg_tol=1e-12)
    assert rc == 0 and st.status == 0
    assert st.cp_iters == iters and st.ell == iters
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=iters)
    tol = cp_bound(p)
    n = ops.sizes(p)[1]
    assert rel(y, ref["y"]) <= tol
    assert rel(y[:n], ref["y"][0]) <= tol
    assert rel(ybar, ref["ybar"]) <= tol
    C = ops.constraint(p)
    assert rel(C.T @ z, ref["x"]) <= tol
    assert abs(st.tau - ref["tau"]) <= 1e-14 * ref["tau"]
    assert abs(st.sigma - ref["sigma"]) <= 1e-14 * ref["sigma"]


def test_cp_resume_matches_single_run():
    import torch
    inst = _inst(CASES[0])
    p = dict(inst["problem"], max_cp=10)
    L = lib()
    plan = L.mfg_plan(p)
    m0, V, W = dev(inst["m0"]), dev(inst["V"]), dev(inst["W"])
    y = dev(inst["y0"]); ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, m0, V, W, y, ybar, z)
    rc, st = L.mfg_solve(plan, m0, V, W, y, ybar, z, stats=st)
    assert st[0].ell == 20
    _, st2, y2, _, _ = _gpu_cp(inst, 20)
    assert rel(host(y), y2) <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
def test_config1_fixed_count(precision):
    """1-D periodic workload, 300 CP iterations, PCG at 1e-10: iterate vs oracle."""
    inst = mi.config1()
    p = inst["problem"]
    rc, st, y, ybar, z = _gpu_cp(inst, 300, precision, cg_tol=1e-10)
    assert rc == 0 and st.cp_iters == 300
    ref = Solver(p, inst["m0"], inst["V"], inst["W"]).run(inst["y0"], iters=300)
    err = rel(y, ref["y"])
    print(f"config1 {precision}: rel err {err:.3e}, PCG iterations {st.cg_iters}")
    assert err <= 1e-8


@pytest.mark.parametrize("case", CASES[:3] + POW2[:1])
def test_prox_quadratic_coupling(case):
    """f(x, m) = f_a m + f_b m^2 + V(x) with f_b > 0 (the crowd-aversion coupling
    of the paper's Problem 1): the prox equation is no longer concave."""
    import torch
    inst = _inst(case, f_a=0.0)
    p = dict(inst["problem"], f_b=0.5)
    plan = _plan(p)
    s, n, c = ops.sizes(p)
    v = mi.random_field((c, p["nt"]) + tuple(p["n"]), 61, -2.0, 2.0)
    v[0] += 0.5
    y = torch.empty(c * n, dtype=torch.float64, device="cuda")
    for tau in (0.05, 1.0, 7.0):
        lib().mfg_prox(plan, 0, tau, dev(v), dev(inst["V"]), dev(inst["W"]), y)
        torch.cuda.synchronize()
        ref = oracle_prox(p, tau, v, inst["V"], inst["W"]).reshape(-1)
        assert np.abs(host(y) - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


def test_problem1_shape_adaptive_tolerance():
    """Problem 1 of Sec. 5.1 on a small grid (16^2, N_t = 32): f = (m^2 - sin 2 pi y
    - sin 2 pi x - cos 4 pi x)/2, m0 = 1, gamma = 5e-4, nu = 0.01, the adaptive CG
    rule and the CP stop rule of Sec. 5.  The device run stops within a few
    iterations of the exact-solve oracle and lands on the same density."""
    import torch
    N, nt = 16, 32
    p = mi._problem(2, N, N, ("periodic", "periodic"), nt, 0.01, f_a=0.0, f_b=0.5, gamma=5e-4,
                    max_cp=1000, cg_rule=1)
    X, Y = mi.nodes(p)
    V = -0.5 * (np.sin(2 * np.pi * Y) + np.sin(2 * np.pi * X) + np.cos(4 * np.pi * X))
    m0 = np.ones((N, N))
    p["cp_tol"] = 1e-4 * np.linalg.norm(m0)
    W = np.zeros_like(V)
    y0 = mi.initial_iterate(p, m0)
    L = lib()
    plan = L.mfg_plan(p, precision="mixed")
    y = dev(y0)
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(m0), dev(V), dev(W), y, ybar, z)
    assert rc == 0 and st[0].status == 0
    ref = Solver(p, m0, V, W, method="modal").run(y0)
    assert abs(st[0].cp_iters - ref["iters"]) <= max(3, 0.05 * ref["iters"])
    assert st[0].r_last <= p["cp_tol"]
    n = ops.sizes(p)[1]
    assert rel(host(y)[:n], ref["y"][0]) <= 1e-3


@pytest.mark.parametrize("case", CASES[:2] + POW2[:2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cp_exact_time_solve(case, precision):
    """l = 0: the preconditioner is AAt itself (tridiagonal solves in time per
    spatial mode), so FP64 PCG stops after one iteration and the CP iterate
    matches the oracle like the paper's preconditioner does."""
    inst = _inst(case, l=0)
    p = inst["problem"]
    iters = 15
    rc, st, y, ybar, z = _gpu_cp(inst, iters, precision, cg_tol=1e-12)
    assert rc == 0 and st.status == 0
    if precision == "fp64":
        assert st.max_cg_in_solve <= 2
    ref = Solver(dict(p, l=1), inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=iters)
    tol = cp_bound(p)
    assert rel(y, ref["y"]) <= tol


@pytest.mark.parametrize("cg_ref", ["rhs", "resid"])
@pytest.mark.parametrize("case", [CASES[0], CASES[3], POW2[0]])
def test_pcg_stop_reference(case, cg_ref):
    """FP64 Fletcher-Reeves PCG with the paper's P against the oracle's PCG
    (same algorithm, warm start from z_l, tolerance 1e-10 relative to ||b||
    (MFG_CG_REF_RHS) or to the warm-start residual (MFG_CG_REF_RESID)): the same
    number of PCG iterations per solve, up to one at a tolerance boundary, and
    the same iterate."""
    inst = _inst(case)
    iters = 8
    rc, st, y, ybar, z = _gpu_cp(inst, iters, "fp64", cg_tol=1e-10, cg_ref=cg_ref)
    assert rc == 0 and st.status == 0
    p = dict(inst["problem"], max_cp=iters, cg_tol=1e-10)
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="pcg", cg_ref=cg_ref).run(inst["y0"], iters=iters)
    print(f"\n{cg_ref}: device {st.cg_iters} PCG iterations, oracle {sum(ref['cg'])} ({ref['cg']})")
    assert abs(st.cg_iters - sum(ref["cg"])) <= 1
    assert abs(st.max_cg_in_solve - max(ref["cg"])) <= 1
    assert rel(y, ref["y"]) <= 1e-7


@pytest.mark.parametrize("case", CASES)
def test_prox_step_matches_oracle(case):
    """The in-solve primal step (k_prox_cp: lift x = C^T z, prox of y - tau x,
    extrapolation) through mfg_prox_step, against the oracle's sparse C^T and
    bisection prox."""
    import torch
    inst = _inst(case)
    p = inst["problem"]
    plan = _plan(p)
    s, n, c = ops.sizes(p)
    y0 = mi.random_field((c, p["nt"]) + tuple(p["n"]), 81, -1.0, 1.0)
    y0[0] += 1.0
    zf = mi.random_field(n, 82, -0.5, 0.5)
    tau = 0.37
    y, ybar = dev(y0), torch.empty(c * n, dtype=torch.float64, device="cuda")
    lib().mfg_prox_step(plan, 0, tau, dev(zf), y, ybar, dev(inst["V"]), dev(inst["W"]))
    torch.cuda.synchronize()
    x = ops.constraint(p).T @ zf
    ref = oracle_prox(p, tau, (y0.reshape(-1) - tau * x).reshape(y0.shape), inst["V"], inst["W"]).reshape(-1)
    theta = 1.0 / np.sqrt(1.0 + 2.0 * p["gamma"] * tau)
    ref_bar = ref + theta * (ref - y0.reshape(-1))
    assert rel(host(y), ref) <= 1e-12
    assert np.abs(host(y) - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
    assert rel(host(ybar), ref_bar) <= 1e-12


@pytest.mark.parametrize("qp", [1.5, 3.0])
@pytest.mark.parametrize("case", CASES[:2] + CASES[4:5])
def test_prox_general_hamiltonian(case, qp):
    """prox for H = |p|^{q'}/q' (b_hat = |w|^q/(q m^{q-1}), Sec. 2) against the
    oracle's nested bisection."""
    import torch
    inst = _inst(case)
    p = dict(inst["problem"], qprime=qp)
    plan = _plan(p)
    s, n, c = ops.sizes(p)
    v = mi.random_field((c, p["nt"]) + tuple(p["n"]), 91, -2.0, 2.0)
    v[0] += 0.5
    y = torch.empty(c * n, dtype=torch.float64, device="cuda")
    for tau in (0.05, 1.0):
        lib().mfg_prox(plan, 0, tau, dev(v), dev(inst["V"]), dev(inst["W"]), y)
        torch.cuda.synchronize()
        ref = oracle_prox(p, tau, v, inst["V"], inst["W"]).reshape(-1)
        got = host(y)
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        assert np.all(got[:n] >= 0)


@pytest.mark.parametrize("qp", [1.5, 3.0])
@pytest.mark.parametrize("precision", ["fp64", "mixed_tc"])
def test_cp_iterate_general_hamiltonian(qp, precision):
    """The CP iterate with the general power Hamiltonian against the oracle."""
    inst = _inst(CASES[1])
    iters = 10
    rc, st, y, ybar, z = _gpu_cp(inst, iters, precision, cg_tol=1e-12, qprime=qp)
    assert rc == 0 and st.status == 0 and st.cp_iters == iters
    p = dict(inst["problem"], qprime=qp)
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=iters)
    err = rel(y, ref["y"])
    print(f"\nq' = {qp}, {precision}: rel err {err:.2e}")
    assert err <= cp_bound(p)
    assert rel(ybar, ref["ybar"]) <= cp_bound(p)
