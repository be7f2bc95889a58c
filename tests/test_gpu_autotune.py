"""The autotuner: it picks among measured launch variants (vector grid,
preconditioner pass kinds, AAt chunking) without changing the operators, so a
tuned solve still matches the oracle at the CP bar; the choice is cached per
instance shape and a second plan of the same shape takes it untimed."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle.cp import Solver

from _gpu_helpers import cp_bound, dev, host, lib, rel

pytestmark = pytest.mark.gpu

CASES = [
    (dict(seed=81, dim=2, nx=32, ny=64, nt=32, bc=("periodic", "neumann")), "mixed_tc"),
    (dict(seed=82, dim=2, nx=19, ny=45, nt=11, bc=("neumann", "periodic")), "mixed"),
    (dict(seed=83, dim=1, nx=128, nt=64, bc=("neumann", "periodic")), "fp64"),
]


@pytest.mark.parametrize("case,precision", CASES)
def test_tuned_solve_matches_oracle(case, precision):
    import torch
    L = lib()
    inst = mi.small(**case)
    p = dict(inst["problem"], max_cp=15, cg_tol=1e-12)
    plan = L.mfg_plan(p, precision=precision)
    before = L.mfg_get_schedule(plan, 0)
    assert before["tuned"] == 0
    L.mfg_autotune(plan)
    sch = L.mfg_get_schedule(plan, 0)
    print(f"\n{case['nx']}x{case.get('ny', 1)}x{case['nt']} {precision}: {sch}")
    assert sch["tuned"] == 1
    assert sch["vec_blocks"] in (152, 304, 608)
    assert sch["precond_us"] > 0 and sch["aat_us"] > 0
    if precision != "mixed_tc":
        assert sch["time_pass"] == "cuda_cores"
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    assert rc == 0 and st[0].status == 0 and st[0].cp_iters == 15
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=15)
    assert rel(host(y), ref["y"]) <= cp_bound(p)
    # a second plan of the same shape takes the cached choice without timing
    plan2 = L.mfg_plan(p, precision=precision)
    L.mfg_autotune(plan2)
    sch2 = L.mfg_get_schedule(plan2, 0)
    assert sch2["tuned"] == 1 and sch2["measured"] == 0
    for k in ("time_pass", "fft", "aat_blocks", "vec_blocks"):
        assert sch2[k] == sch[k]


def test_tuned_batch_matches_untuned_to_roundoff():
    """Every instance of a batch, tuned, against the same batch untuned: the
    launch choices only reorder floating-point operations."""
    import torch
    L = lib()
    insts = [mi.small(**c) for c, _ in CASES[:2]]
    probs = [dict(i["problem"], max_cp=10, cg_tol=1e-12, precision="mixed_tc") for i in insts]
    outs = []
    for tune in (False, True):
        plan = L.mfg_plan(probs)
        if tune:
            L.mfg_autotune(plan)
        cat = lambda k: dev(np.concatenate([np.asarray(i[k]).reshape(-1) for i in insts]))
        y = cat("y0")
        ybar = y.clone()
        z = torch.zeros(L.mfg_sizes(plan)["dual"], dtype=torch.float64, device="cuda")
        rc, st = L.mfg_solve(plan, cat("m0"), cat("V"), cat("W"), y, ybar, z)
        assert rc == 0
        outs.append(host(y))
    assert rel(outs[1], outs[0]) <= 1e-9
