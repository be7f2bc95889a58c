"""The allocation-free preconditioner entry point, mfg_apply_precond_noalloc.

It serves callers that may not allocate device memory where they call the
library (graph capture in global mode, pool-managed memory, latency-critical
paths): it takes a bare problem description and keeps its tables and work
buffers in a static device array.  This file checks, through the C ABI, that
two consecutive calls on different problems give the same result as the
plan-based mfg_apply_precond, within the tolerances of the preconditioner
parity tests (normwise backward error against the oracle's assembled P; the
forward difference only loosely, since it carries the condition number of P),
and that repeating a call reproduces it bit for bit.  It is collected last so a
failure here does not hide the other GPU tests.
"""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops

from _gpu_helpers import dev, host, lib, rel

pytestmark = pytest.mark.gpu

PROBLEMS = [
    dict(seed=1, dim=2, nx=19, ny=45, nt=11, bc=("periodic", "periodic"), l=1),
    dict(seed=2, dim=2, nx=17, ny=33, nt=9, bc=("neumann", "neumann"), l=2),
]


def _backward_error(A, x, b):
    res = np.abs(A @ x - b).max()
    nA = np.abs(A).sum(axis=1).max()
    return res / (nA * np.abs(x).max() + np.abs(b).max())


@pytest.mark.parametrize("precision,eta,fwd", [("fp64", 1e-12, 1e-8), ("mixed", 5e-5, 1e-2)])
def test_noalloc_matches_plan_entry_point(precision, eta, fwd):
    import torch
    L = lib()
    outs = []
    for case in PROBLEMS:  # two calls in a row on different problems
        p = dict(mi.small(**case)["problem"], precision=precision)
        n = ops.sizes(p)[1]
        r = dev(mi.random_field(n, 40 + case["seed"]))
        z_na = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        L.mfg_apply_precond_noalloc(p, r, z_na)
        plan = L.mfg_plan(p)
        z_plan = torch.empty(n, dtype=torch.float64, device="cuda")
        L.mfg_apply_precond(plan, 0, r, z_plan)
        torch.cuda.synchronize()
        a, b = host(z_na), host(z_plan)
        assert np.all(np.isfinite(a))
        assert rel(a, b) <= fwd
        P = ops.precond(p)
        assert _backward_error(P, a, host(r)) <= eta
        outs.append((p, r, a))
    # repeating the first call reproduces it exactly (no state carried over)
    p, r, a = outs[0]
    z2 = torch.empty_like(r)
    L.mfg_apply_precond_noalloc(p, r, z2)
    torch.cuda.synchronize()
    assert np.array_equal(host(z2), a)


# at the limits of the static scratch: n = 2^18 with a 256-point axis, N_t = 128,
# and the 1-D geometry; power-of-two axes take the FFT spatial passes, whose
# twiddles live in the static array too
LIMITS = [
    dict(seed=4, dim=2, nx=256, ny=256, nt=4, bc=("periodic", "neumann"), l=1),
    dict(seed=5, dim=2, nx=32, ny=64, nt=128, bc=("neumann", "periodic"), l=1),
    dict(seed=6, dim=1, nx=256, nt=128, bc=("neumann", "periodic"), l=2),
]


@pytest.mark.parametrize("case", LIMITS)
@pytest.mark.parametrize("precision,eta,fwd", [("fp64", 1e-12, 1e-8), ("mixed", 5e-5, 1e-2),
                                               ("mixed_tc", 5e-5, 1e-2)])
def test_noalloc_at_the_limits(case, precision, eta, fwd):
    """Same checks as above at the largest problems the static array takes:
    against the plan entry point and the oracle's assembled P, two calls in a
    row (the second on a different right-hand side)."""
    import torch
    L = lib()
    p = dict(mi.small(**case)["problem"], precision=precision)
    n = ops.sizes(p)[1]
    P = ops.precond(p)
    plan = L.mfg_plan(p)
    for seed in (91, 92):
        r = dev(mi.random_field(n, seed))
        z_na = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        L.mfg_apply_precond_noalloc(p, r, z_na)
        z_plan = torch.empty(n, dtype=torch.float64, device="cuda")
        L.mfg_apply_precond(plan, 0, r, z_plan)
        torch.cuda.synchronize()
        a, b = host(z_na), host(z_plan)
        assert np.all(np.isfinite(a))
        assert rel(a, b) <= fwd
        assert _backward_error(P, a, host(r)) <= eta


def test_noalloc_rejects_oversize():
    """A problem beyond the static scratch (here 2 x 512 x 512 points) is refused
    with MFG_ERR_INVALID_ARG before any kernel runs."""
    import torch
    L = lib()
    p = dict(mi.small(3)["problem"], nt=2, n=(512, 512))
    r = torch.zeros(2 * 512 * 512, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    with pytest.raises(L.MfgError) as e:
        L.mfg_apply_precond_noalloc(p, r, z)
    assert e.value.code == L.MFG_ERR_INVALID_ARG
    assert "static scratch" in L.mfg_last_error()
