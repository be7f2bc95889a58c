"""Viscosity fields nu(x) on the device against the oracle (the paper allows a
non-constant viscosity, Sec. 4 before Sec. 4.1, and names LU for the
per-frequency systems of Alg. 1, Sec. 4.1).

  - C, C^T and AAt with K_nu against the oracle's sparse matrices (1e-12);
  - P^{-1} through the banded Cholesky factors against the oracle's Alg. 1
    with one sparse LU per frequency: FP64 forward error, FP32 normwise
    backward error;
  - CP iterates after a fixed count against the oracle's exact solves, in
    every precision, on ragged grids of both boundary conditions and both
    dimensions, with smooth and discontinuous fields;
  - a constant field against the constant-nu path (FFT preconditioner);
  - a 64^2 x 32 Neumann grid with a 10:1 smooth field against the oracle's
    inexact solve, counting PCG iterations;
  - a field instance batched with a constant-nu one (bitwise equal to the solo
    solves), both stop references and the adaptive PCG rule, general q';
  - the adjoint with a field (node derivatives dloss/dnu(x)) against the
    oracle's KKT gradient, directly and through torch.autograd."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import operators as ops
from oracle import solvers
from oracle.cp import Solver

from _gpu_helpers import dev, host, lib, rel

pytestmark = pytest.mark.gpu

# (seed, dim, nx, ny, nt, bc, kind, ratio, l)
CASES = [
    (31, 2, 12, 10, 8, ("neumann", "neumann"), "smooth", 10.0, 1),
    (32, 2, 9, 8, 6, ("periodic", "periodic"), "layers", 20.0, 2),
    (33, 2, 7, 11, 5, ("periodic", "neumann"), "smooth", 5.0, 1),
    (34, 2, 10, 6, 7, ("neumann", "periodic"), "layers", 8.0, 1),
    (35, 1, 24, 1, 16, ("periodic", "periodic"), "smooth", 10.0, 1),
    (36, 1, 19, 1, 9, ("neumann", "neumann"), "layers", 30.0, 2),
]


def _inst(case, **kw):
    seed, dim, nx, ny, nt, bc, kind, ratio, l = case
    inst = mi.small(seed, dim=dim, nx=nx, ny=ny, nt=nt, bc=bc, l=l, **kw)
    p = inst["problem"]
    p["nu_field"] = mi.viscosity_field(p, p["nu"], ratio, seed + 100, kind)
    return inst


def _plan(p, precision="fp64"):
    return lib().mfg_plan(p, precision=precision)


@pytest.mark.parametrize("case", CASES)
def test_field_operators_match_oracle(case):
    import torch
    inst = _inst(case)
    p = inst["problem"]
    L = lib()
    plan = _plan(p)
    s, n, c = ops.sizes(p)
    Cm = ops.constraint(p)
    v = mi.random_field(c * n, 5)
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_C(plan, 0, dev(v), r)
    assert rel(host(r), Cm @ v) <= 1e-12
    q = mi.random_field(n, 6)
    x = torch.empty(c * n, dtype=torch.float64, device="cuda")
    L.mfg_apply_Ct(plan, 0, dev(q), x)
    assert rel(host(x), Cm.T @ q) <= 1e-12
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_AAt(plan, 0, dev(q), out)
    assert rel(host(out), ops.AAt(p, Cm) @ q) <= 1e-12


@pytest.mark.parametrize("case", CASES)
def test_field_precond_fp64_matches_lu(case):
    """Forward error of P^{-1} r in FP64 against Alg. 1 with sparse LU.  Both
    sides are exact solves; their difference is bounded by ~kappa(P) u with
    kappa(P) <= 1e7 on these grids, so 1e-8 leaves a wide margin."""
    import torch
    inst = _inst(case)
    p = inst["problem"]
    L = lib()
    plan = _plan(p, "fp64")
    n = ops.sizes(p)[1]
    r = mi.random_field(n, 7)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_precond(plan, 0, dev(r), z)
    ref = solvers.precond_lu(p, r)
    err = rel(host(z), ref)
    print(f"\nfield P^-1, FP64: rel err {err:.2e}")
    assert err <= 1e-8


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", ["mixed", "mixed_tc"])
def test_field_precond_fp32_backward_error(case, precision):
    """FP32 factors and substitutions: normwise backward error
    ||r - P z|| / (||P||_1 ||z|| + ||r||) against the assembled P.  Banded
    Cholesky with forward and backward substitution is backward stable with
    |dM| <= gamma_{3w+3} |L||L^T| (w the half-bandwidth), and the two FP32
    time transforms add ~N_t u relative perturbations, so the bar is
    (3w + 3 + 2 N_t) u_32."""
    import torch
    inst = _inst(case)
    p = inst["problem"]
    L = lib()
    plan = _plan(p, precision)
    n = ops.sizes(p)[1]
    r = mi.random_field(n, 8)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_precond(plan, 0, dev(r), z)
    P = ops.precond(p)
    zh = host(z)
    eta = np.linalg.norm(r - P @ zh) / (abs(P).sum(axis=0).max() * np.linalg.norm(zh) + np.linalg.norm(r))
    nx, ny = p["n"]
    w = 4 * ny + ny if p["dim"] == 2 else 4
    bar = (3 * w + 3 + 2 * p["nt"]) * 2.0 ** -24
    print(f"\nfield P^-1, {precision}: backward error {eta:.2e} (bar {bar:.1e})")
    assert eta <= bar


# Shapes of the substitutions' block schedule (the block size G follows from
# the half-bandwidth w: the largest power of two <= 32 with 2G <= w whose
# stage fits the kernel's budget): G = 32 with a partial last block (7 x 33 Neumann, w = 66,
# S = 231), G = 32 with three blocks (5 x 17, periodic x, w = 68, S = 85),
# fewer blocks than copies in flight (1-D with two points; 2 x 2 periodic),
# and G = 2 with three blocks (3 x 2 periodic, w = 5).
BAND_SHAPES = [
    (71, 2, 7, 33, 4, ("neumann", "neumann"), "smooth", 10.0, 1),
    (72, 2, 5, 17, 5, ("periodic", "neumann"), "layers", 10.0, 1),
    (73, 1, 2, 1, 4, ("periodic", "periodic"), "smooth", 5.0, 1),
    (74, 2, 2, 2, 3, ("periodic", "periodic"), "smooth", 5.0, 2),
    (75, 2, 3, 2, 6, ("periodic", "periodic"), "layers", 8.0, 1),
]


@pytest.mark.parametrize("case", BAND_SHAPES)
def test_field_precond_band_shapes(case):
    """P^{-1} r on the block-schedule shapes above: FP64 against Alg. 1 with
    sparse LU (forward error, as in the FP64 test), FP32 by its normwise
    backward error (the bar of the FP32 test)."""
    import torch
    inst = _inst(case)
    p = inst["problem"]
    L = lib()
    n = ops.sizes(p)[1]
    r = mi.random_field(n, 9)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mfg_apply_precond(_plan(p, "fp64"), 0, dev(r), z)
    err = rel(host(z), solvers.precond_lu(p, r))
    L.mfg_apply_precond(_plan(p, "mixed_tc"), 0, dev(r), z)
    P = ops.precond(p)
    zh = host(z)
    eta = np.linalg.norm(r - P @ zh) / (abs(P).sum(axis=0).max() * np.linalg.norm(zh) + np.linalg.norm(r))
    nx, ny = p["n"]
    w = 4 * ny + ny if p["dim"] == 2 else 4
    bar = (3 * w + 3 + 2 * p["nt"]) * 2.0 ** -24
    print(f"\nband shape {case[2]}x{case[3]}: FP64 rel err {err:.2e}, FP32 backward error {eta:.2e} (bar {bar:.1e})")
    assert err <= 1e-8
    assert eta <= bar


def _field_cond(p):
    """cond(AAt) by dense eigenvalues (the small grids of this file)."""
    ev = np.linalg.eigvalsh(ops.AAt(p).toarray())
    return ev[-1] / ev[0]


def _run(inst, iters, precision, cg_tol=1e-12):
    import torch
    p = dict(inst["problem"], max_cp=iters, cg_tol=cg_tol)
    L = lib()
    plan = L.mfg_plan(p, precision=precision)
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    return rc, st[0], host(y), host(ybar), host(z)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_tc", "mixed_df"])
def test_field_cp_iterate(case, precision):
    """Bound as for the constant-nu iterates: max(1e-8, 10 kappa u), kappa =
    cond(AAt) with K_nu, u = 2^-53 (an exact AAt solve carries ~kappa u)."""
    inst = _inst(case)
    p = inst["problem"]
    iters = 15
    rc, st, y, ybar, z = _run(inst, iters, precision)
    assert rc == 0 and st.status == 0 and st.cp_iters == iters
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=iters)
    tol = max(1e-8, 10.0 * _field_cond(p) * 2.0 ** -53)
    ey, eb = rel(y, ref["y"]), rel(ybar, ref["ybar"])
    ex = rel(ops.constraint(p).T @ z, ref["x"])
    print(f"\nfield CP, {precision}: y {ey:.1e}, ybar {eb:.1e}, C^T z {ex:.1e} (bar {tol:.1e}); "
          f"{st.cg_iters / iters:.2f} PCG per CP")
    assert ey <= tol and eb <= tol and ex <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed_tc"])
def test_constant_field_matches_constant_nu(precision):
    """A constant field runs the banded path; the constant nu runs the FFT /
    dense-transform path.  Both preconditioners are exact P, so the iterates
    agree to the PCG tolerance."""
    inst = mi.small(40, nx=16, ny=8, nt=16, bc=("neumann", "periodic"), nu=0.05, l=1)
    p = inst["problem"]
    a = _run(inst, 12, precision)
    q = dict(p, nu_field=np.full(p["n"], 0.05))
    b = _run(dict(inst, problem=q), 12, precision)
    assert a[0] == 0 and b[0] == 0
    assert rel(b[2], a[2]) <= 1e-9
    assert abs(a[1].cg_iters - b[1].cg_iters) <= 2


def test_field_neumann_64_against_oracle():
    """2-D Neumann 64^2 x 32 with a smooth 10:1 field around nu = 1e-2, the
    tensor-core precision, 4 CP iterations at PCG 1e-10 against the oracle's
    PCG with the exact Alg. 1 preconditioner (sparse LU per frequency) at
    1e-12; the iterate agrees to ~kappa u and the device needs as few PCG
    iterations as the exact-P oracle (the banded solve is exact P up to FP32)."""
    inst = mi.config_varnu(n=64, nt=32, nu=1e-2, ratio=10.0)
    p = dict(inst["problem"])
    iters = 4
    rc, st, y, _, _ = _run(inst, iters, "mixed_tc", cg_tol=1e-10)
    assert rc == 0 and st.status == 0
    ref = Solver(dict(p, cg_tol=1e-12), inst["m0"], inst["V"], inst["W"], method="pcg",
                 cg_ref="rhs").run(inst["y0"], iters=iters)
    err = rel(y, ref["y"])
    dev_cg = st.cg_iters / iters
    ora_cg = float(np.mean(ref["cg"]))
    print(f"\nfield 64^2 x 32 Neumann: rel err {err:.1e}; {dev_cg:.2f} PCG per CP (oracle at 1e-12: {ora_cg:.2f})")
    assert err <= 1e-8
    assert dev_cg <= ora_cg + 1.0


def _batch_solve(insts, iters, precision):
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
        outs.append((host(y)[lay["primal_off"]:lay["primal_off"] + cn], st[b]))
    return outs


@pytest.mark.parametrize("precision", ["fp64", "mixed_tc"])
def test_field_in_uneven_batch(precision):
    """A field instance and a constant-nu instance in one plan (one CUDA graph):
    each equals its own solo solve bit for bit and the oracle at the CP bound."""
    a = _inst(CASES[0])
    b = mi.small(41, nx=9, ny=14, nt=6, bc=("periodic", "neumann"))
    iters = 10
    batched = _batch_solve([a, b], iters, precision)
    for inst, (yb, st) in zip([a, b], batched):
        assert st.status == 0 and st.cp_iters == iters
        ys, _ = _batch_solve([inst], iters, precision)[0]
        assert np.array_equal(yb, ys)
    ref = Solver(a["problem"], a["m0"], a["V"], a["W"], method="lu").run(a["y0"], iters=iters)
    assert rel(batched[0][0], ref["y"]) <= max(1e-8, 10.0 * _field_cond(a["problem"]) * 2.0 ** -53)


@pytest.mark.parametrize("cg_ref,cg_rule", [("resid", 0), ("rhs", 1), ("resid", 1)])
def test_field_stop_rules_match_oracle(cg_ref, cg_rule):
    """Both stop references and the paper's adaptive rule with a field, FP64:
    the device's PCG counts equal the oracle's (the same P up to rounding)."""
    import torch
    inst = _inst(CASES[2])
    p = dict(inst["problem"], max_cp=8, cg_tol=1e-10, cg_ref=cg_ref, cg_rule=cg_rule)
    L = lib()
    plan = L.mfg_plan(p, precision="fp64")
    y = dev(inst["y0"])
    ybar = y.clone()
    z = torch.zeros(ops.sizes(p)[1], dtype=torch.float64, device="cuda")
    rc, st = L.mfg_solve(plan, dev(inst["m0"]), dev(inst["V"]), dev(inst["W"]), y, ybar, z)
    assert rc == 0 and st[0].status == 0
    ref = Solver(p, inst["m0"], inst["V"], inst["W"], method="pcg", cg_ref=cg_ref).run(inst["y0"], iters=8)
    assert abs(st[0].cg_iters - sum(ref["cg"])) <= 2
    assert rel(host(y), ref["y"]) <= 1e-6


def test_field_general_hamiltonian():
    """q' = 1.5 with a field: the general-q' prox and K_nu in the same kernel
    instantiation, against the oracle's exact solves."""
    inst = _inst(CASES[3])
    inst["problem"]["qprime"] = 1.5
    iters = 10
    rc, st, y, _, _ = _run(inst, iters, "mixed_tc")
    assert rc == 0 and st.status == 0
    ref = Solver(inst["problem"], inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"], iters=iters)
    assert rel(y, ref["y"]) <= max(1e-8, 10.0 * _field_cond(inst["problem"]) * 2.0 ** -53)


def _field_converged(case, precision, iters=3000):
    import torch
    inst = mi.small(**case, eps=0.0)
    p = dict(inst["problem"], gamma=0.05, max_cp=iters, cg_tol=1e-12, precision=precision)
    p["nu_field"] = mi.viscosity_field(p, p["nu"], 4.0, case["seed"] + 3, "smooth")
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


ADJ_CASES = [dict(seed=61, dim=2, nx=12, ny=10, nt=6, bc=("periodic", "periodic"), nu=0.2),
             dict(seed=62, dim=2, nx=9, ny=14, nt=5, bc=("neumann", "periodic"), nu=0.05),
             dict(seed=63, dim=1, nx=40, nt=8, bc=("neumann", "neumann"), nu=0.1)]


@pytest.mark.parametrize("case", ADJ_CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed_tc"])
def test_field_adjoint_matches_oracle_kkt(case, precision):
    """The adjoint with a field (banded P inside the Schur PCG, K_nu in C^T,
    node derivatives dloss/dnu(x)) against the oracle's sparse-LU KKT gradient,
    itself pinned by central differences (tests/test_oracle_varnu.py)."""
    import torch
    from oracle import adjoint as oadj
    p, plan, m0, V, W, mt, y, z = _field_converged(case, precision)
    yh, zh = host(y).reshape((1 + 2 * p["dim"], p["nt"]) + tuple(p["n"])), host(z)
    _, g = oadj.loss_mT(p, yh, mt)
    ref = oadj.adjoint_gradients(p, yh, zh.reshape(p["nt"], *p["n"]), g)
    S = p["n"][0] * p["n"][1]
    dm0, dV, dW, dnu = (torch.empty(S, dtype=torch.float64, device="cuda") for _ in range(4))
    rc, st = lib().mfg_adjoint(plan, 0, y, z, dev(g), dm0, dV, dW, dnu, tol=1e-12)
    assert rc == 0 and st.status == 0 and st.cg_iters > 0
    for got, key in ((dm0, "dm0"), (dV, "dV"), (dW, "dW"), (dnu, "dnu")):
        assert rel(host(got), ref[key]) <= 1e-7, key


def test_field_autograd_gradient():
    """torch.autograd through a field: the (Nx, Ny) nu tensor gets the node
    derivatives of the direct call."""
    import torch
    from oracle import adjoint as oadj
    from paper_2507_01958_gb300.autograd import equilibrium_mT
    case = ADJ_CASES[0]
    p, plan, m0, V, W, mt, y, z = _field_converged(case, "fp64")
    nu = torch.as_tensor(np.asarray(p["nu_field"]), dtype=torch.float64, device="cuda").requires_grad_(True)
    m0t = dev(m0).reshape(p["n"]).requires_grad_(True)
    q = {k: v for k, v in p.items() if k != "nu_field"}
    mT = equilibrium_mT(m0t, dev(V).reshape(p["n"]), dev(W).reshape(p["n"]), nu, q, "fp64", 1e-12)
    dx, dy = ops.spacing(p)
    loss = ((mT - dev(mt).reshape(p["n"])) ** 2).sum() * dx * dy
    loss.backward()
    yh = host(y).reshape((5, p["nt"]) + tuple(p["n"]))
    _, g = oadj.loss_mT(p, yh, mt)
    ref = oadj.adjoint_gradients(p, yh, host(z).reshape(p["nt"], *p["n"]), g)
    assert nu.grad.shape == tuple(p["n"])
    assert rel(host(nu.grad), ref["dnu"]) <= 1e-7
    assert rel(host(m0t.grad), ref["dm0"]) <= 1e-7
