"""The paper's two test problems (Sec. 5.1 Problem 1, periodic crowd aversion;
Sec. 5.2 Problem 2, Gaussian target on the Neumann square) at N = 16 with
N_t = 8N, the CP stop rule CPtol = 1e-4 ||m0|| and the adaptive CG rule
min{1e-4, max{1e-6, 1e-4 r}} of Sec. 5, solved on the device and by the
oracle's inexact solve (the same PCG with the paper's preconditioner, warm
start and stop reference).  The device must stop within a few CP iterations
of the oracle, need about as many PCG iterations per solve, and land on the
same density.  Each case prints its counts next to the paper's (Tables 1 and
3: soft pins; the paper leaves the scaling conventions that fix them open)."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle.cp import Solver

from _gpu_helpers import dev, host, lib, rel

pytestmark = pytest.mark.gpu

# (problem, paper's CP count and average CG with the DCT-VIII preconditioner at nu = 0.01, N = 16)
CASES = [("problem1", mi.problem1, 77, 2.4), ("problem2", mi.problem2, 354, 3.8)]


@pytest.mark.parametrize("name,fn,paper_cp,paper_cg", CASES)
@pytest.mark.parametrize("cg_ref", ["resid", "rhs"])
def test_paper_problem_device_vs_oracle(name, fn, paper_cp, paper_cg, cg_ref):
    import torch
    inst = fn(N=16, nu=0.01)
    p = dict(inst["problem"], cg_ref=cg_ref)
    L = lib()
    plan = L.mfg_plan(p, precision="mixed_tc")
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    assert rc == 0 and st[0].status == 0
    assert st[0].r_last <= p["cp_tol"]
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="pcg", cg_ref=cg_ref).run(inst["y0"])
    dev_cg = st[0].cg_iters / st[0].cp_iters
    ora_cg = float(np.mean(ref["cg"]))
    n = ops.sizes(p)[1]
    err = rel(host(y)[:n], ref["y"][0])
    print(f"\n{name} 16^2 x 128, nu = 0.01, stop reference {cg_ref}: device {st[0].cp_iters} CP, "
          f"{dev_cg:.2f} PCG per CP; oracle {ref['iters']} CP, {ora_cg:.2f}; paper {paper_cp} CP, {paper_cg} "
          f"(DCT); density rel diff {err:.1e}")
    assert abs(st[0].cp_iters - ref["iters"]) <= max(3, 0.02 * ref["iters"])
    assert abs(dev_cg - ora_cg) <= 0.25 * ora_cg + 0.2
    assert err <= 1e-3
