"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times: the 2-D periodic 128^2 x 64 workload and the 2-D Neumann
512^2 x 128 workload (n = 33.5 M).  Assembling sparse matrices at these sizes
is impractical, so the oracle side uses its matrix-free applies through the
spatial eigenbasis (pinned against the sparse matrices on small grids), its
exact spatially-diagonalised solve, and the prox on sampled cells."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle import solvers
from oracle.cp import Solver
from oracle.prox import coupling, prox_cells

from _gpu_helpers import dev, host, lib, rel

pytestmark = pytest.mark.gpu


def _inst(which):
    return mi.config2(nu=1e-2) if which == "config2" else mi.config3()


@pytest.mark.parametrize("which", ["config2", "config3"])
def test_fullsize_AAt_and_precond(which):
    import torch
    inst = _inst(which)
    p = inst["problem"]
    n = ops.sizes(p)[1]
    L = lib()
    pv = mi.random_field(n, 51)
    ref_q = solvers.apply_AAt_modal(p, pv)
    for prec in ("fp64", "mixed_df"):
        plan = L.mfg_plan(p, precision=prec)
        q = torch.empty(n, dtype=torch.float64, device="cuda")
        L.mfg_apply_AAt(plan, 0, dev(pv), q)
        torch.cuda.synchronize()
        assert rel(host(q), ref_q) <= 1e-11, prec
    r = mi.random_field(n, 52)
    for prec, eta_max in (("fp64", 1e-12), ("mixed", 5e-5)):
        plan = L.mfg_plan(p, precision=prec)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        L.mfg_apply_precond(plan, 0, dev(r), z)
        torch.cuda.synchronize()
        zh = host(z)
        Pz, lam = solvers.apply_P_modal(p, zh)
        eta = np.linalg.norm(Pz - r) / (lam * np.linalg.norm(zh) + np.linalg.norm(r))
        assert eta <= eta_max, (prec, eta)


@pytest.mark.parametrize("which", ["config2", "config3"])
def test_fullsize_prox_sampled(which):
    import torch
    inst = _inst(which)
    p = inst["problem"]
    s, n, c = ops.sizes(p)
    L = lib()
    plan = L.mfg_plan(p)
    v = mi.random_field((c, p["nt"]) + tuple(p["n"]), 53, -2.0, 2.0)
    v[0] += 0.5
    y = torch.empty(c * n, dtype=torch.float64, device="cuda")
    tau = 0.37
    L.mfg_prox(plan, 0, tau, dev(v), dev(inst["V"]), dev(inst["W"]), y)
    torch.cuda.synchronize()
    got = host(y).reshape(v.shape)
    rng = np.random.default_rng(3)
    cells = rng.integers(0, n, size=20000)
    cells[:500] = np.arange(n - 500, n)  # include the terminal plane (g/dt)
    a, b, cc = coupling(p, inst["V"], inst["W"])
    flat = lambda arr: arr.reshape(arr.shape[0], -1) if arr.ndim == 4 else arr.reshape(-1)
    ref = prox_cells(tau, flat(v)[:, cells], a.reshape(-1)[cells], b, cc.reshape(-1)[cells])
    assert np.abs(flat(got)[:, cells] - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
def test_fullsize_cp_config2(precision):
    """Three CP iterations on the 128^2 x 64 workload (nu = 1e-2) against the
    oracle; cond(AAt) ~ 1e6 here, so the bound is 1e-8."""
    import torch
    inst = mi.config2(nu=1e-2)
    p = dict(inst["problem"], max_cp=3, cg_tol=1e-12)
    L = lib()
    plan = L.mfg_plan(p, precision=precision)
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    assert rc == 0 and st[0].cp_iters == 3
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=3)
    assert rel(host(y), ref["y"]) <= 1e-8
    assert rel(host(ybar), ref["ybar"]) <= 1e-8


def test_fullsize_cp_config3_first_iteration():
    """One CP iteration on the 512^2 x 128 Neumann workload (mixed precision, the
    benchmark's configuration): the dual update is the exact solve of eq. CC* up to
    the PCG tolerance (energy-norm error), and the new primal equals the oracle's
    prox of y0 - tau C^T z on sampled cells."""
    import torch
    inst = mi.config3()
    p = dict(inst["problem"], max_cp=1, cg_tol=1e-12)
    s, n, c = ops.sizes(p)
    L = lib()
    plan = L.mfg_plan(p, precision="mixed")
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    assert rc == 0 and st[0].status == 0
    # with x0 = 0, z0 = 0 and ybar0 = y0 (w = 0, m^k = m0): C y0 - d = nu K m0 on every plane
    _, K = ops.spatial(p)
    Km0 = (K @ inst["m0"].reshape(-1)).reshape(p["n"])
    b = p["sigma0"] * p["nu"] * np.broadcast_to(Km0, (p["nt"],) + tuple(p["n"])).reshape(-1)
    zs = solvers.solve_AAt_modal(p, b)
    zh = host(z)
    e = zh - zs
    en = np.sqrt(e @ solvers.apply_AAt_modal(p, e))
    ref_n = np.sqrt(zs @ solvers.apply_AAt_modal(p, zs))
    assert en <= 1e-7 * ref_n
    # primal: prox of y0 - tau0 C^T z (C^T z from the device, parity-tested on small grids)
    x = torch.empty(c * n, dtype=torch.float64, device="cuda")
    L.mfg_apply_Ct(plan, 0, z, x)
    torch.cuda.synchronize()
    vv = inst["y0"].reshape(c, -1) - p["tau0"] * host(x).reshape(c, -1)
    rng = np.random.default_rng(4)
    cells = rng.integers(0, n, size=20000)
    a, bb, cc = coupling(p, inst["V"], inst["W"])
    ref = prox_cells(p["tau0"], vv[:, cells], a.reshape(-1)[cells], bb, cc.reshape(-1)[cells])
    got = host(y).reshape(c, -1)[:, cells]
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    assert np.all(np.isfinite(host(y))) and host(y)[:n].min() >= 0.0
