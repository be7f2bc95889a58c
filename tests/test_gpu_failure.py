"""Failure detection of the solver, driven from the host so that nothing can
fault or hang the GPU:

  MFG_ERR_NONFINITE      a NaN written into m0 or V on the host; the residual
                         or the CP step norm reports it and the instance stops
                         after the iteration that saw it;
  MFG_ERR_NOT_CONVERGED  max_cg = 1 with an unreachable tolerance;
  MFG_ERR_TIMEOUT        the fault-injection hooks under which the tensor-core
                         time pass issues no MMA and no commit, or the banded
                         substitutions of a viscosity-field plan issue no stage
                         copy, so a bounded mbarrier wait must run out (nothing
                         is ever in flight).

Each case runs in graph and in eager launch mode, checks the status, the
iteration counters and that the call returned, and then checks that the same
plan still solves correctly (the context stays usable)."""
import time

import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle.cp import Solver

from _gpu_helpers import cp_bound, dev, host, lib, rel

pytestmark = pytest.mark.gpu

CASE = dict(seed=61, dim=2, nx=16, ny=32, nt=32, bc=("periodic", "neumann"))
MODES = ["graph", "eager"]


def _run(p, inst, m0=None, V=None, mode="graph", plan=None, precision="mixed"):
    import torch
    L = lib()
    plan = plan or L.mfg_plan(p, precision=precision)
    L.mfg_set_launch_mode(plan, mode)
    m0 = inst["m0"] if m0 is None else m0
    V = inst["V"] if V is None else V
    y = dev(mi.initial_iterate(p, m0))
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    rc, st = L.mfg_solve(plan, dev(m0), dev(V), dev(inst["W"]), y, ybar, z)
    torch.cuda.synchronize()
    return plan, rc, st[0], host(y), time.perf_counter() - t0


def _check_healthy(plan, p, inst, mode):
    """The plan (made for problem p) solves the clean inputs after the failure
    and matches the oracle: the context is still usable."""
    L = lib()
    _, rc, st, y, _ = _run(p, inst, mode=mode, plan=plan)
    assert rc == L.MFG_OK and st.status == L.MFG_OK and st.cp_iters == p["max_cp"]
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="modal").run(inst["y0"], iters=p["max_cp"])
    assert rel(y, ref["y"]) <= cp_bound(p)


def _problem(**kw):
    inst = mi.small(**CASE, eps=0.0)
    p = dict(inst["problem"], max_cp=5, cg_tol=1e-12)
    p.update(kw)
    return p, inst


@pytest.mark.parametrize("mode", MODES)
def test_nonfinite_m0(mode):
    L = lib()
    p, inst = _problem()
    m0 = inst["m0"].copy()
    m0[3, 7] = np.nan
    plan, rc, st, y, _ = _run(p, inst, m0=m0, mode=mode)
    assert rc == L.MFG_ERR_NONFINITE and st.status == L.MFG_ERR_NONFINITE
    assert st.cp_iters == 1, "the instance stops after the iteration that saw the NaN"
    _check_healthy(plan, p, inst, mode)


@pytest.mark.parametrize("mode", MODES)
def test_nonfinite_V(mode):
    """A NaN in the potential reaches only the prox: the cell's root comes out
    NaN (not a clipped zero), the CP step norm is NaN, the instance stops."""
    L = lib()
    p, inst = _problem()
    V = inst["V"].copy()
    V[5, 2] = np.nan
    plan, rc, st, y, _ = _run(p, inst, V=V, mode=mode)
    assert rc == L.MFG_ERR_NONFINITE and st.status == L.MFG_ERR_NONFINITE
    assert st.cp_iters == 1
    s, n, c = ops.sizes(p)
    m = y[:n].reshape(p["nt"], *p["n"])
    assert np.isnan(m[:, 5, 2]).all()
    _check_healthy(plan, p, inst, mode)


def test_prox_entry_point_propagates_nan():
    import torch
    L = lib()
    p, inst = _problem()
    plan = L.mfg_plan(p)
    s, n, c = ops.sizes(p)
    v = mi.random_field((c, p["nt"]) + tuple(p["n"]), 71, -1.0, 1.0)
    v[0] += 1.0
    V = inst["V"].copy()
    V[1, 1] = np.nan
    y = torch.empty(c * n, dtype=torch.float64, device="cuda")
    L.mfg_prox(plan, 0, 0.3, dev(v), dev(V), dev(inst["W"]), y)
    torch.cuda.synchronize()
    out = host(y).reshape(v.shape)
    bad = np.zeros(tuple(p["n"]), dtype=bool)
    bad[1, 1] = True
    assert np.isnan(out[0][:, bad]).all()
    assert np.isfinite(out[:, :, ~bad]).all()


@pytest.mark.parametrize("mode", MODES)
def test_not_converged(mode):
    L = lib()
    p, inst = _problem(max_cg=1, cg_tol=1e-14, max_cp=3)
    plan, rc, st, y, _ = _run(p, inst, mode=mode)
    assert rc == L.MFG_ERR_NOT_CONVERGED and st.status == L.MFG_ERR_NOT_CONVERGED
    assert st.cp_iters == 3 and st.max_cg_in_solve == 1 and st.cg_iters == 3
    assert np.isfinite(y).all()
    ok = dict(p, max_cg=10000, cg_tol=1e-12)
    _check_healthy(L.mfg_plan(ok, precision="mixed"), ok, inst, mode)


@pytest.mark.parametrize("mode", MODES)
def test_tensor_core_wait_times_out(mode):
    """Under MFG_INJECT_TC_NO_COMMIT the tensor-core pass waits on an mbarrier
    that nothing arrives on; the bounded wait gives up, the instance reports
    MFG_ERR_TIMEOUT after its first CP iteration and the call returns."""
    L = lib()
    p, inst = _problem(max_cp=4)
    plan = L.mfg_plan(p, precision="mixed_tc")
    L.mfg_set_fault_injection(plan, "tc_no_commit")
    plan, rc, st, y, secs = _run(p, inst, mode=mode, plan=plan)
    assert rc == L.MFG_ERR_TIMEOUT and st.status == L.MFG_ERR_TIMEOUT
    assert st.cp_iters == 1 and st.cg_iters == 0
    assert secs < 30.0
    L.mfg_set_fault_injection(plan, "none")
    _check_healthy(plan, p, inst, mode)


@pytest.mark.parametrize("mode", MODES)
def test_band_wait_times_out(mode):
    """Under MFG_INJECT_BAND_NO_COPY the banded substitutions of a
    viscosity-field plan wait on a stage that is never copied; the bounded
    wait gives up, the instance reports MFG_ERR_TIMEOUT after its first CP
    iteration and the call returns; the same plan then solves correctly."""
    L = lib()
    inst = mi.small(seed=62, dim=2, nx=12, ny=16, nt=8, bc=("neumann", "periodic"), eps=0.0)
    p = dict(inst["problem"], max_cp=4, cg_tol=1e-12)
    p["nu_field"] = mi.viscosity_field(p, p["nu"], 10.0, 162, "smooth")
    plan = L.mfg_plan(p, precision="mixed_tc")
    L.mfg_set_fault_injection(plan, "band_no_copy")
    plan, rc, st, y, secs = _run(p, inst, mode=mode, plan=plan)
    assert rc == L.MFG_ERR_TIMEOUT and st.status == L.MFG_ERR_TIMEOUT
    assert st.cp_iters == 1 and st.cg_iters == 0
    assert secs < 30.0
    L.mfg_set_fault_injection(plan, "none")
    _, rc, st, y, _ = _run(p, inst, mode=mode, plan=plan)
    assert rc == L.MFG_OK and st.status == L.MFG_OK and st.cp_iters == p["max_cp"]
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=p["max_cp"])
    # the bound of the constant-nu iterates, max(1e-8, 10 kappa u), with
    # kappa = cond(AAt) for K_nu by dense eigenvalues (a 12 x 16 x 8 grid)
    ev = np.linalg.eigvalsh(ops.AAt(p).toarray())
    assert rel(y, ref["y"]) <= max(1e-8, 10.0 * ev[-1] / ev[0] * 2.0 ** -53)


def test_fault_injection_rejects_unknown_codes():
    L = lib()
    p, _ = _problem()
    plan = L.mfg_plan(p, precision="mixed_tc")
    with pytest.raises(L.MfgError) as e:
        L.mfg_set_fault_injection(plan, 7)
    assert e.value.code == L.MFG_ERR_INVALID_ARG
