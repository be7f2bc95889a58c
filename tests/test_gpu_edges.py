"""Edge cases of the hot path on the device against the oracle: the smallest
grids (N = 2 per axis, where a periodic axis's two neighbours coincide, and
N_t = 2), the largest N_t (256, the generic time pass; the tensor-core
precision falls back to the CUDA cores there), the longest FFT line (a 1-D
axis of 512 points), zero viscosity (Sec. 4.2: P = AAt for l = 1, so every PCG
solve stops after one iteration) and a zero initial density (the degenerate
feasible point m = 0, w = 0)."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle.cp import Solver

from _gpu_helpers import cp_bound, dev, host, lib, rel

pytestmark = pytest.mark.gpu

EDGES = [
    dict(seed=51, dim=2, nx=2, ny=2, nt=2, bc=("periodic", "periodic")),
    dict(seed=52, dim=2, nx=2, ny=3, nt=3, bc=("neumann", "neumann")),
    dict(seed=53, dim=2, nx=3, ny=2, nt=2, bc=("periodic", "neumann")),
    dict(seed=54, dim=1, nx=2, nt=2, bc=("periodic", "periodic")),
    dict(seed=55, dim=1, nx=2, nt=4, bc=("neumann", "neumann")),
    dict(seed=56, dim=2, nx=4, ny=6, nt=256, bc=("neumann", "periodic")),
    dict(seed=57, dim=1, nx=512, nt=8, bc=("neumann", "neumann"), nu=0.05),
    dict(seed=58, dim=1, nx=512, nt=6, bc=("periodic", "periodic"), nu=0.05),
]


def _inst(case, **kw):
    c = dict(case)
    c.update(kw)
    return mi.small(**c)


@pytest.mark.parametrize("case", EDGES)
def test_edge_operators(case):
    import torch
    inst = _inst(case)
    p = inst["problem"]
    L = lib()
    plan = L.mfg_plan(p)
    s, n, c = ops.sizes(p)
    Cm = ops.constraint(p)
    v = mi.random_field(c * n, 1)
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_C(plan, 0, dev(v), r)
    assert rel(host(r), Cm @ v) <= 1e-12
    q = mi.random_field(n, 2)
    x = torch.empty(c * n, dtype=torch.float64, device="cuda")
    L.mfg_apply_Ct(plan, 0, dev(q), x)
    assert rel(host(x), Cm.T @ q) <= 1e-12
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_AAt(plan, 0, dev(q), out)
    assert rel(host(out), ops.AAt(p, Cm) @ q) <= 1e-12


@pytest.mark.parametrize("case", EDGES)
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-12), ("mixed_tc", 5e-5)])
def test_edge_precond_backward_error(case, precision, bar):
    """Normwise backward error of P^{-1} r against the assembled P (the bars of
    the other preconditioner tests)."""
    import torch
    inst = _inst(case)
    p = inst["problem"]
    L = lib()
    plan = L.mfg_plan(p, precision=precision)
    n = ops.sizes(p)[1]
    r = mi.random_field(n, 3)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_precond(plan, 0, dev(r), z)
    P = ops.precond(p)
    zh = host(z)
    eta = np.abs(r - P @ zh).max() / (abs(P).sum(axis=1).max() * np.abs(zh).max() + np.abs(r).max())
    assert eta <= bar


def _run(p, inst, precision):
    import torch
    L = lib()
    plan = L.mfg_plan(p, precision=precision)
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    return rc, st[0], host(y)


@pytest.mark.parametrize("case", EDGES)
@pytest.mark.parametrize("precision", ["fp64", "mixed_tc"])
def test_edge_cp_iterate(case, precision):
    inst = _inst(case)
    p = dict(inst["problem"], max_cp=8, cg_tol=1e-12)
    rc, st, y = _run(p, inst, precision)
    assert rc == 0 and st.status == 0 and st.cp_iters == 8
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=8)
    assert rel(y, ref["y"]) <= cp_bound(p)


@pytest.mark.parametrize("case", [EDGES[1], EDGES[5], dict(seed=59, dim=2, nx=16, ny=32, nt=32,
                                                            bc=("periodic", "neumann"))])
def test_zero_viscosity_pcg_stops_after_one_iteration(case):
    """nu = 0, l = 1: the preconditioner equals AAt (Sec. 4.2), so each PCG
    solve ends after one iteration (FP64, tolerance 1e-10)."""
    inst = _inst(case, nu=0.0, l=1)
    p = dict(inst["problem"], max_cp=6, cg_tol=1e-10, cg_ref="resid")
    rc, st, y = _run(p, inst, "fp64")
    assert rc == 0 and st.status == 0
    assert st.max_cg_in_solve <= 1
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=6)
    assert rel(y, ref["y"]) <= cp_bound(p)


@pytest.mark.parametrize("precision", ["fp64", "mixed_tc"])
def test_zero_initial_density(precision):
    """m0 = 0: the iterate stays finite and matches the oracle."""
    inst = _inst(dict(seed=60, dim=2, nx=12, ny=16, nt=8, bc=("neumann", "periodic")))
    inst["m0"] = np.zeros_like(inst["m0"])
    inst["y0"] = mi.initial_iterate(inst["problem"], inst["m0"])
    p = dict(inst["problem"], max_cp=10, cg_tol=1e-12)
    rc, st, y = _run(p, inst, precision)
    assert rc == 0 and st.status == 0 and np.isfinite(y).all()
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=10)
    nrm = max(np.linalg.norm(ref["y"]), 1e-300)
    assert np.linalg.norm(y - ref["y"].reshape(-1)) / nrm <= cp_bound(p)
