"""Parity of the benchmark's solver path (MFG_MIXED_TC: FP32 preconditioner
with its time transforms on the tensor cores inside FP64 flexible PCG, PCG
relative tolerance 1e-10 against ||b||, one graph launch per solve) with the
FP64 oracle at the workloads' full sizes and iteration counts.

  * 2-D periodic 128^2 x 64: 300 CP iterations for nu = 1 (the stiffest,
    cond(AAt) ~ 7e9) and nu = 1e-3, 30 for nu = 1e-2 and 1e-1; y, ybar and
    the dual x = C^T z against the oracle's exact-solve run, relative l2 <= 1e-8
    (the target stated for the method).  Each case prints its errors.
  * 2-D Neumann 512^2 x 128 (n = 33.5 M, the benchmark's headline workload):
    three CP iterations, each step checked against the oracle from the state
    before it: the dual update against the exact solve of eq. CC* in the
    energy norm (bound tol sqrt(cond(AAt)), what a relative residual of tol
    guarantees), the new primal against the oracle's prox of y - tau C^T z on
    every cell, the extrapolation and the step sizes.
  * The smallest and the largest instance of the 64-instance uneven batch,
    solved together in one batch plan, each against its own oracle run.
  * The adjoint on the 32^2 x 16 copy of the adjoint workload against the
    oracle's sparse-LU KKT gradient at the same converged point."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import adjoint as oadj
from oracle import operators as ops
from oracle import solvers
from oracle.cp import Solver
from oracle.prox import prox

from _gpu_helpers import cp_bound, dev, host, lib, rel

pytestmark = pytest.mark.gpu

CG_TOL = 1e-10


def _solve(p, inst, precision="mixed_tc"):
    import torch
    L = lib()
    plan = L.mfg_plan(p, precision=precision)
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    return rc, st[0], host(y), host(ybar), host(z)


@pytest.mark.parametrize("nu,iters", [(1.0, 300), (1e-3, 300), (1e-2, 30), (1e-1, 30)])
def test_config2_fixed_count_mixed_tc(nu, iters):
    inst = mi.config2(nu=nu)
    p = dict(inst["problem"], max_cp=iters, cg_tol=CG_TOL)
    rc, st, y, ybar, z = _solve(p, inst)
    assert rc == 0 and st.status == 0 and st.cp_iters == iters
    s, n, c = ops.sizes(p)
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=iters)
    x = ops.apply_Ct_planes(p, z)
    errs = {"y": rel(y, ref["y"]), "m": rel(y[:n], ref["y"][0]), "w": rel(y[n:], ref["y"][1:]),
            "ybar": rel(ybar, ref["ybar"]), "x": rel(x, ref["x"])}
    print(f"\n128^2x64 nu={nu:g}, {iters} CP, mixed_tc, PCG {CG_TOL:g}: "
          + ", ".join(f"{k} {v:.2e}" for k, v in errs.items())
          + f"; {st.cg_iters / iters:.2f} PCG per CP, cond(AAt) {solvers.cond_AAt(p):.2e}")
    for k, v in errs.items():
        assert v <= 1e-8, (k, v)
    assert abs(st.tau - ref["tau"]) <= 1e-13 * ref["tau"]


def test_config3_three_iterations_mixed_tc():
    import torch
    inst = mi.config3()
    p = dict(inst["problem"], max_cp=1, cg_tol=CG_TOL)
    s, n, c = ops.sizes(p)
    L = lib()
    plan = L.mfg_plan(p, precision="mixed_tc")
    m0d, Vd, Wd = dev(inst["m0"]), dev(inst["V"]), dev(inst["W"])
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    d = ops.rhs_d(p, inst["m0"])
    lo, hi = solvers.eig_range_AAt(p)
    bound = 2.0 * CG_TOL * np.sqrt(hi / lo)
    st = None
    for it in range(3):
        y_l, ybar_l, z_l = host(y), host(ybar), host(z)
        tau, sigma = (p["tau0"], p["sigma0"]) if st is None else (st[0].tau, st[0].sigma)
        rc, st = L.mfg_solve(plan, m0d, Vd, Wd, y, ybar, z, stats=st)
        assert rc == 0 and st[0].status == 0 and st[0].ell == it + 1
        # dual: exact solve of AAt z = AAt z_l + sigma (C ybar_l - d) (eq. CC* with x_l = C^T z_l)
        b = solvers.apply_AAt_modal(p, z_l) + sigma * (ops.apply_C_planes(p, ybar_l) - d)
        zs = solvers.solve_AAt_modal(p, b)
        zh = host(z)
        e = zh - zs
        err_A = np.sqrt(e @ solvers.apply_AAt_modal(p, e)) / np.sqrt(zs @ b)
        # primal: prox of y_l - tau C^T z_{l+1} on every cell
        v = y_l.reshape(c, -1) - tau * ops.apply_Ct_planes(p, zh).reshape(c, -1)
        y_ref = prox(p, tau, v.reshape((c, p["nt"]) + tuple(p["n"])), inst["V"], inst["W"]).reshape(-1)
        yh = host(y)
        err_y = rel(yh, y_ref)
        theta = 1.0 / np.sqrt(1.0 + 2.0 * p["gamma"] * tau)
        ybar_ref = yh + theta * (yh - y_l)
        err_bar = rel(host(ybar), ybar_ref)
        print(f"\n512^2x128 CP iteration {it + 1}: dual energy-norm error {err_A:.2e} (bound {bound:.1e}), "
              f"primal {err_y:.2e}, extrapolation {err_bar:.2e}, {st[0].cg_iters} PCG")
        assert err_A <= bound
        assert err_y <= 1e-11
        assert err_bar <= 1e-13
        assert abs(st[0].tau - theta * tau) <= 1e-15 * tau
        assert abs(st[0].sigma - sigma / theta) <= 1e-15 * sigma / theta
        assert yh[:n].min() >= 0.0 and np.isfinite(yh).all()


def test_uneven_batch_extremes_mixed_tc():
    """Seed 103 (64^2 x 32, periodic) and seed 141 (256^2 x 128, Neumann,
    nu = 1e-3) of the uneven batch in one plan and one graph launch."""
    import torch
    L = lib()
    iters = 20
    insts = [mi.config5_instance(s) for s in (103, 141)]
    probs = [dict(i["problem"], max_cp=iters, cg_tol=CG_TOL, precision="mixed_tc") for i in insts]
    plan = L.mfg_plan(probs)
    cat = lambda k: dev(np.concatenate([np.asarray(i[k]).reshape(-1) for i in insts]))
    y = cat("y0")
    ybar = y.clone()
    z = torch.zeros(L.mfg_sizes(plan)["dual"], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, cat("m0"), cat("V"), cat("W"), y, ybar, z)
    assert rc == 0
    yh = host(y)
    for b, inst in enumerate(insts):
        lay = L.mfg_layout(plan, b)
        yb = yh[lay["primal_off"]:lay["primal_off"] + lay["c"] * lay["n"]]
        p = probs[b]
        assert st[b].status == 0 and st[b].cp_iters == iters
        ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=iters)
        err = rel(yb, ref["y"])
        print(f"\nbatch instance {p['n'][0]}^2 x {p['nt']} ({p['bc'][0]}, nu={p['nu']:.3g}): rel err {err:.2e}, "
              f"{st[b].cg_iters / iters:.2f} PCG per CP")
        assert err <= cp_bound(p)


def test_adjoint_config4_copy():
    """The adjoint workload (periodic, nu = 0.05, loss ||m(T) - m_target||^2)
    on its 32^2 x 16 copy: the device gradient against the oracle's sparse-LU
    KKT gradient at the same converged point.  The acceleration constant is
    0.05 so that CP reaches r <= 1e-9 ||m0|| within the cap; it changes the
    path to the equilibrium, not the equilibrium."""
    import torch
    L = lib()
    inst = mi.config4(n=32, nt=16)
    p = dict(inst["problem"], gamma=0.05, max_cp=40000, cg_tol=1e-12,
             cp_tol=1e-9 * np.linalg.norm(inst["m0"]))
    plan = L.mfg_plan(p, precision="fp64")
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    assert rc == 0 and st[0].r_last <= p["cp_tol"], st[0].r_last
    c = 1 + 2 * p["dim"]
    yh = host(y).reshape((c, p["nt"]) + tuple(p["n"]))
    _, g = oadj.loss_mT(p, yh, inst["m_target"])
    ref = oadj.adjoint_gradients(p, yh, host(z).reshape(p["nt"], *p["n"]), g)
    S = p["n"][0] * p["n"][1]
    dm0, dV, dW = (torch.empty(S, dtype=torch.float64, device="cuda") for _ in range(3))
    dnu = torch.empty(1, dtype=torch.float64, device="cuda")
    rc, sa = L.mfg_adjoint(plan, 0, y, z, dev(g), dm0, dV, dW, dnu, tol=1e-12, max_iter=20000)
    assert rc == 0 and sa.status == 0
    errs = {"dm0": rel(host(dm0), ref["dm0"]), "dV": rel(host(dV), ref["dV"]), "dW": rel(host(dW), ref["dW"]),
            "dnu": abs(host(dnu)[0] - ref["dnu"]) / max(1.0, abs(ref["dnu"]))}
    print(f"\nadjoint 32^2x16: {st[0].cp_iters} CP to r {st[0].r_last:.1e}, {sa.cg_iters} adjoint PCG, "
          + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v <= 1e-7, (k, v)
