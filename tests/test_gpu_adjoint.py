"""The adjoint (implicit differentiation) through the C ABI against the
oracle's KKT-based gradient at the same converged point, and the
torch.autograd wrapper against the direct call.  The oracle gradient itself is
pinned by central finite differences (tests/test_oracle_adjoint.py)."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import adjoint as oadj
from oracle import operators as ops

from _gpu_helpers import dev, host, lib, rel

pytestmark = pytest.mark.gpu

CASES = [
    dict(seed=31, dim=2, nx=12, ny=10, nt=6, bc=("periodic", "periodic"), nu=0.2),
    dict(seed=32, dim=2, nx=9, ny=14, nt=5, bc=("neumann", "periodic"), nu=0.05),
    dict(seed=33, dim=1, nx=40, nt=8, bc=("neumann", "periodic"), nu=0.1),
]


def _converged(case, precision, iters=3000):
    import torch
    inst = mi.small(**case, eps=0.0)
    p = dict(inst["problem"], gamma=0.05, max_cp=iters, cg_tol=1e-12, precision=precision)
    rng = np.random.default_rng(case["seed"])
    nx, ny = p["n"]
    m0 = mi._normalise(1.0 + 0.3 * rng.uniform(size=(nx, ny)), p)
    V = 0.3 * rng.normal(size=(nx, ny))
    W = 0.2 * rng.normal(size=(nx, ny))
    mt = mi._normalise(1.0 + 0.3 * rng.uniform(size=(nx, ny)), p)
    L = lib()
    plan = L.mfg_plan(p)
    y = dev(mi.initial_iterate(p, m0))
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(m0), dev(V), dev(W), y, ybar, z)
    assert rc == 0
    return p, plan, m0, V, W, mt, y, z


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_matches_oracle_kkt(case, precision):
    import torch
    p, plan, m0, V, W, mt, y, z = _converged(case, precision)
    yh, zh = host(y).reshape((1 + 2 * p["dim"], p["nt"]) + tuple(p["n"])), host(z)
    _, g = oadj.loss_mT(p, yh, mt)
    ref = oadj.adjoint_gradients(p, yh, zh.reshape(p["nt"], *p["n"]), g)
    S = p["n"][0] * p["n"][1]
    dm0, dV, dW = (torch.empty(S, dtype=torch.float64, device="cuda") for _ in range(3))
    dnu = torch.empty(1, dtype=torch.float64, device="cuda")
    rc, st = lib().mfg_adjoint(plan, 0, y, z, dev(g), dm0, dV, dW, dnu, tol=1e-12)
    assert rc == 0 and st.status == 0 and st.cg_iters > 0
    assert rel(host(dm0), ref["dm0"]) <= 1e-7
    assert rel(host(dV), ref["dV"]) <= 1e-7
    assert rel(host(dW), ref["dW"]) <= 1e-7
    assert abs(host(dnu)[0] - ref["dnu"]) <= 1e-7 * max(1.0, abs(ref["dnu"]))


def test_autograd_function_matches_direct_call():
    import torch
    from paper_2507_01958_gb300.autograd import equilibrium_mT
    case = CASES[0]
    p, plan, m0, V, W, mt, y, z = _converged(case, "fp64")
    m0t = dev(m0).reshape(p["n"]).requires_grad_(True)
    Vt = dev(V).reshape(p["n"]).requires_grad_(True)
    Wt = dev(W).reshape(p["n"]).requires_grad_(True)
    nut = torch.tensor(p["nu"], dtype=torch.float64, device="cuda", requires_grad=True)
    dx, dy = ops.spacing(p)
    mT = equilibrium_mT(m0t, Vt, Wt, nut, p, "fp64", 1e-12)
    loss = ((mT - dev(mt).reshape(p["n"])) ** 2).sum() * dx * dy
    loss.backward()
    yh = host(y).reshape((5, p["nt"]) + tuple(p["n"]))
    _, g = oadj.loss_mT(p, yh, mt)
    ref = oadj.adjoint_gradients(p, yh, host(z).reshape(p["nt"], *p["n"]), g)
    assert rel(host(m0t.grad), ref["dm0"]) <= 1e-7
    assert rel(host(Vt.grad), ref["dV"]) <= 1e-7
    assert abs(float(nut.grad) - ref["dnu"]) <= 1e-7 * max(1.0, abs(ref["dnu"]))
