"""Batched solves (several uneven instances in one plan, one graph launch):
every instance matches the oracle and, bit for bit, its own single-instance
solve, whatever its neighbours in the batch."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle.cp import Solver

from _gpu_helpers import cp_bound, dev, host, lib, rel

pytestmark = pytest.mark.gpu

BATCH = [
    dict(seed=11, dim=2, nx=24, ny=40, nt=8, bc=("periodic", "periodic"), nu=0.05),
    dict(seed=12, dim=2, nx=17, ny=21, nt=12, bc=("neumann", "neumann"), nu=0.3),
    dict(seed=13, dim=1, nx=50, nt=6, bc=("periodic", "periodic"), nu=0.01),
    dict(seed=14, dim=2, nx=9, ny=70, nt=5, bc=("neumann", "periodic"), nu=0.002),
]


def _solve(insts, iters, precision):
    import torch
    L = lib()
    probs = [dict(i["problem"], max_cp=iters, cg_tol=1e-12, precision=precision) for i in insts]
    plan = L.mfg_plan(probs)
    cat = lambda k: dev(np.concatenate([np.asarray(i[k]).reshape(-1) for i in insts]))
    y = cat("y0")
    ybar = y.clone()
    z = torch.zeros(L.mfg_sizes(plan)["dual"], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, cat("m0"), cat("V"), cat("W"), y, ybar, z)
    assert rc == 0
    outs = []
    for b in range(len(insts)):
        lay = L.mfg_layout(plan, b)
        cn = lay["c"] * lay["n"]
        outs.append((host(y)[lay["primal_off"]:lay["primal_off"] + cn],
                     host(z)[lay["dual_off"]:lay["dual_off"] + lay["n"]], st[b]))
    return outs


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
def test_batch_matches_solo_and_oracle(precision):
    insts = [mi.small(**c) for c in BATCH]
    iters = 15
    batched = _solve(insts, iters, precision)
    for inst, (yb, zb, st) in zip(insts, batched):
        assert st.status == 0 and st.cp_iters == iters
        ys, zs, _ = _solve([inst], iters, precision)[0]
        assert np.array_equal(yb, ys) and np.array_equal(zb, zs)
        p = inst["problem"]
        ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=iters)
        tol = cp_bound(p)
        assert rel(yb, ref["y"]) <= tol


def test_batch_mixed_precisions_and_zero_iterations():
    """Instances may differ in precision; an instance with max_cp = 0 is left untouched."""
    import torch
    L = lib()
    insts = [mi.small(**c) for c in BATCH[:2]]
    probs = [dict(insts[0]["problem"], max_cp=5, precision="fp64"),
             dict(insts[1]["problem"], max_cp=0, precision="mixed")]
    plan = L.mfg_plan(probs)
    cat = lambda k: dev(np.concatenate([np.asarray(i[k]).reshape(-1) for i in insts]))
    y = cat("y0")
    y_in = host(y).copy()
    ybar = y.clone()
    z = torch.zeros(L.mfg_sizes(plan)["dual"], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, cat("m0"), cat("V"), cat("W"), y, ybar, z)
    assert rc == 0 and st[0].cp_iters == 5 and st[1].cp_iters == 0
    lay = L.mfg_layout(plan, 1)
    sl = slice(lay["primal_off"], lay["primal_off"] + lay["c"] * lay["n"])
    assert np.array_equal(host(y)[sl], y_in[sl])
