"""The tensor-core time pass (MFG_MIXED_TC: tcgen05 TF32 products, operands
split in three for ~FP32 accuracy) against the oracle's assembled P and the CP
iterate, at the FP32 path's bars.

Cases cover N_t = 32, 64 and 128 (the sizes the tensor-core kernel takes; 128
stages its K dimension in two rounds), ragged strips (S not a multiple of the
128-mode strip, S below one strip), both time transforms (l = 1 DCT-VIII, l = 2
DST-I), both boundary conditions and the FFT and dense spatial passes."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle.cp import Solver

from _gpu_helpers import cp_bound, dev, host, lib, rel

pytestmark = pytest.mark.gpu

TC_CASES = [
    dict(seed=41, dim=2, nx=19, ny=45, nt=32, bc=("periodic", "periodic")),   # S = 855: 7 strips, ragged
    dict(seed=42, dim=2, nx=16, ny=32, nt=64, bc=("neumann", "neumann")),     # S = 512: 4 full strips, FFT
    dict(seed=43, dim=2, nx=10, ny=70, nt=128, bc=("periodic", "neumann")),   # S = 700, two K rounds
    dict(seed=44, dim=2, nx=32, ny=32, nt=128, bc=("periodic", "periodic")),  # FFT, two K rounds
    dict(seed=45, dim=1, nx=40, nt=64, bc=("neumann", "periodic")),           # S = 40 < one strip
    dict(seed=46, dim=1, nx=128, nt=32, bc=("periodic", "periodic")),         # S = 128: one strip
]


def _backward_error(A, x, b):
    res = np.abs(A @ x - b).max()
    nA = np.abs(A).sum(axis=1).max()
    return res / (nA * np.abs(x).max() + np.abs(b).max())


@pytest.mark.parametrize("case", TC_CASES)
@pytest.mark.parametrize("l", [1, 2])
def test_precond_tc(case, l):
    import torch
    inst = mi.small(**dict(case, l=l))
    p = inst["problem"]
    L = lib()
    n = ops.sizes(p)[1]
    r = mi.random_field(n, 51)
    z_tc = torch.empty(n, dtype=torch.float64, device="cuda")
    z_32 = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row: the second reuses the warmed-up kernel
        L.mfg_apply_precond(L.mfg_plan(dict(p), precision="mixed_tc"), 0, dev(r), z_tc)
    L.mfg_apply_precond(L.mfg_plan(dict(p), precision="mixed"), 0, dev(r), z_32)
    torch.cuda.synchronize()
    zt = host(z_tc)
    assert np.all(np.isfinite(zt))
    P = ops.precond(p)
    assert _backward_error(P, zt, r) <= 5e-5
    # same operator as the FP32 CUDA-core time pass, to within the FP32 round-off
    assert rel(zt, host(z_32)) <= 1e-4


SMALL_TC = [
    dict(seed=47, dim=2, nx=8, ny=12, nt=32, bc=("periodic", "periodic")),
    dict(seed=48, dim=1, nx=40, nt=64, bc=("neumann", "periodic")),
    dict(seed=49, dim=1, nx=20, nt=128, bc=("periodic", "periodic")),
]


@pytest.mark.parametrize("case", SMALL_TC)
def test_cp_iterate_tc(case):
    """25 CP iterations through the graph-captured solve with the tensor-core
    preconditioner, PCG at 1e-12: same bar as the other precisions,
    max(1e-8, 10 kappa u)."""
    import torch
    inst = mi.small(**case)
    p = dict(inst["problem"], max_cp=25, cg_tol=1e-12)
    L = lib()
    plan = L.mfg_plan(p, precision="mixed_tc")
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    torch.cuda.synchronize()
    assert rc == 0 and st[0].status == 0 and st[0].cp_iters == 25
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=25)
    tol = cp_bound(p)
    assert rel(host(y), ref["y"]) <= tol
    assert rel(host(ybar), ref["ybar"]) <= tol
    C = ops.constraint(p)
    assert rel(C.T @ host(z), ref["x"]) <= tol
