"""Pins of the oracle's viscosity-field operators (a field nu(x) in place of
the constant nu; the paper allows it, Sec. 4 before Sec. 4.1, and leaves the
per-time-step systems of Alg. 1 to LU, incomplete Cholesky or AMG).

The field enters through K_nu = sum over axes of D^1 diag(nu_face) (D^1)^T/dx^2
(Sec. 4.3 blocks, arithmetic face means).  Pins: the energy identity
u.K_nu u = sum_faces nu_f (u_a - u_b)^2/dx^2 summed face by face, the constant
field, mass conservation, the block form of eq. largeA and the rank of
AAt - P (Lemma 1) with K_nu, the LU form of Alg. 1 against a sparse solve of
the assembled P, and the inexact per-frequency variant against its limits."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import mfg_inputs as mi
from oracle import operators as ops
from oracle import solvers
from oracle.cp import Solver

BCS = [("periodic", "periodic"), ("neumann", "neumann"), ("periodic", "neumann"),
       ("neumann", "periodic")]


def _field_inst(seed, dim=2, bc=("neumann", "neumann"), kind="smooth", ratio=8.0, **kw):
    inst = mi.small(seed, dim=dim, bc=bc, **kw)
    p = inst["problem"]
    p["nu_field"] = mi.viscosity_field(p, p["nu"], ratio, seed + 11, kind)
    return inst


def _energy_by_faces(p, u):
    """sum over the faces of each active axis of nu_f (u_a - u_b)^2 / dx^2,
    faces enumerated one by one (periodic axes wrap, Neumann axes have N-1)."""
    nx, ny = p["n"]
    nu = np.asarray(p["nu_field"]).reshape(nx, ny)
    u = u.reshape(nx, ny)
    dx = ops.spacing(p)
    tot = 0.0
    for ax in range(p["dim"]):
        n_ax = (nx, ny)[ax]
        faces = n_ax if p["bc"][ax] == "periodic" else n_ax - 1
        for a in range(nx):
            for b in range(ny):
                idx = (a, b)[ax]
                if idx >= faces:
                    continue
                c = [a, b]
                c[ax] = (idx + 1) % n_ax
                nf = 0.5 * (nu[a, b] + nu[c[0], c[1]])
                tot += nf * (u[a, b] - u[c[0], c[1]]) ** 2 / dx[ax] ** 2
    return tot


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("dim", [1, 2])
def test_Knu_energy_identity(bc, dim):
    inst = _field_inst(3, dim=dim, bc=bc, nx=7, ny=5, nt=3)
    p = inst["problem"]
    Kv = ops.K_nu(p)
    for seed in range(3):
        u = mi.random_field(Kv.shape[0], 40 + seed)
        assert abs(u @ (Kv @ u) - _energy_by_faces(p, u)) <= 1e-12 * abs(u @ (Kv @ u))
    assert abs(Kv - Kv.T).max() == 0.0
    # a constant has no energy: K_nu 1 = 0 and 1^T K_nu = 0 (mass conservation)
    assert np.abs(Kv @ np.ones(Kv.shape[0])).max() <= 1e-12 * abs(Kv).max()


@pytest.mark.parametrize("bc", BCS)
def test_constant_field_is_nu_K(bc):
    inst = mi.small(4, bc=bc, nx=6, ny=9, nt=3, nu=0.37)
    p = inst["problem"]
    _, K = ops.spatial(p)
    q = dict(p, nu_field=np.full(p["n"], 0.37))
    assert abs(ops.K_nu(q) - 0.37 * K).max() <= 1e-13 * abs(K).max()
    assert abs(ops.AAt(q) - ops.AAt(p)).max() <= 1e-12 * abs(ops.AAt(p)).max()
    np.testing.assert_allclose(ops.precond(q).toarray(), ops.precond(p).toarray(), rtol=0,
                               atol=1e-12 * abs(ops.precond(p)).max())


@pytest.mark.parametrize("bc", BCS)
def test_field_AAt_block_form_and_lemma1_rank(bc):
    """eq. largeA with L = K_nu + I/dt, and AAt - P = e_1 e_1^T (x) (H - l L_hat),
    H = (2 K_nu + I/dt)/dt: nonzero in the first diagonal block only (Lemma 1)."""
    inst = _field_inst(5, bc=bc, nx=5, ny=4, nt=4, kind="layers")
    p = inst["problem"]
    A = ops.AAt(p).toarray()
    B, _ = ops.spatial(p)
    Kv = ops.K_nu(p).toarray()
    s = Kv.shape[0]
    h = ops.dt(p)
    L = Kv + np.eye(s) / h
    Cb = L @ L + (B @ B.T).toarray()
    nt = p["nt"]
    assert np.abs(A[:s, :s] - Cb).max() <= 1e-10 * np.abs(A).max()
    assert np.abs(A[s:2*s, s:2*s] - Cb - np.eye(s) / h ** 2).max() <= 1e-10 * np.abs(A).max()
    assert np.abs(A[:s, s:2*s] + L / h).max() <= 1e-10 * np.abs(A).max()
    D = A - ops.precond(p).toarray()
    Hm = (2.0 * Kv + np.eye(s) / h) / h - p["l"] * L / h
    assert np.abs(D[:s, :s] - Hm).max() <= 1e-10 * np.abs(A).max()
    D[:s, :s] = 0.0
    assert np.abs(D).max() <= 1e-10 * np.abs(A).max()
    assert nt * s == A.shape[0]


def test_field_uniform_density_is_feasible():
    inst = _field_inst(6, nx=8, ny=6, nt=5)
    p = inst["problem"]
    nx, ny = p["n"]
    m0 = np.full((nx, ny), 1.0 / (nx * ny * mi.cell_volume(p)))
    y = mi.initial_iterate(p, m0)
    res = ops.constraint(p) @ y.reshape(-1) - ops.rhs_d(p, m0)
    assert np.abs(res).max() < 1e-10 * np.abs(ops.rhs_d(p, m0)).max()


@pytest.mark.parametrize("l", [1, 2])
@pytest.mark.parametrize("nt", [3, 8])
def test_time_basis(l, nt):
    Q, lam = solvers.time_basis(nt, l)
    np.testing.assert_allclose(Q.T @ Q, np.eye(nt), atol=1e-13)
    np.testing.assert_allclose(Q.T @ ops.Dtt(nt, l).toarray() @ Q, np.diag(lam), atol=1e-12)
    k = np.arange(1, nt + 1)
    np.testing.assert_allclose(np.sort(lam), np.sort(2 - 2 * np.cos(np.pi * (k - 1 + l / 2) / (nt + l / 2))),
                               atol=1e-12)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("l", [1, 2])
@pytest.mark.parametrize("dim", [1, 2])
def test_precond_lu_solves_assembled_P(bc, l, dim):
    inst = _field_inst(7, dim=dim, bc=bc, nx=6, ny=5, nt=5, l=l, kind="layers")
    p = inst["problem"]
    P = ops.precond(p).tocsc()
    r = mi.random_field(P.shape[0], 8)
    z = solvers.precond_lu(p, r)
    z_ref = spla.spsolve(P, r)
    assert np.linalg.norm(z - z_ref) <= 1e-10 * np.linalg.norm(z_ref)


def test_precond_lu_constant_field_is_modal():
    inst = mi.small(9, bc=("periodic", "neumann"), nx=8, ny=6, nt=6, nu=0.2, l=1)
    p = inst["problem"]
    q = dict(p, nu_field=np.full(p["n"], 0.2))
    r = mi.random_field(ops.sizes(p)[1], 10)
    z = solvers.precond_lu(q, r)
    z_md = solvers.precond_modal(p, r)
    assert np.linalg.norm(z - z_md) <= 1e-10 * np.linalg.norm(z_md)


def test_precond_inner_limits():
    """s = 1 is exact for a constant field; s = 0 is the constant-coefficient P
    at nu_ref; large s tends to the LU form on a varying field."""
    inst = mi.small(12, bc=("neumann", "neumann"), nx=7, ny=6, nt=4, nu=0.05, l=2)
    p = inst["problem"]
    r = mi.random_field(ops.sizes(p)[1], 13)
    q = dict(p, nu_field=np.full(p["n"], 0.05))
    ex = solvers.precond_lu(q, r)
    assert np.linalg.norm(solvers.precond_inner(q, r, 1) - ex) <= 1e-10 * np.linalg.norm(ex)
    f = _field_inst(12, bc=("neumann", "neumann"), nx=7, ny=6, nt=4, nu=0.05, l=2, ratio=4.0)["problem"]
    z0 = solvers.precond_inner(f, r, 0)
    z_md = solvers.precond_modal(dict(f, nu=solvers.nu_ref(f), nu_field=None), r)
    assert np.linalg.norm(z0 - z_md) <= 1e-10 * np.linalg.norm(z_md)
    ex = solvers.precond_lu(f, r)
    e2 = np.linalg.norm(solvers.precond_inner(f, r, 2) - ex)
    e40 = np.linalg.norm(solvers.precond_inner(f, r, 40) - ex)
    assert e40 <= 1e-8 * np.linalg.norm(ex) and e40 < e2


def test_field_trivial_equilibrium():
    """Uniform m0 with x-independent f and g: m stays m0 and w = 0 for any
    viscosity field (K_nu conserves mass, and by Jensen no flow lowers the cost)."""
    inst = _field_inst(14, nx=6, ny=5, nt=4, f_a=1.0, g_a=0.5, kind="layers")
    p = dict(inst["problem"], max_cp=60)
    nx, ny = p["n"]
    m0 = np.full((nx, ny), 1.0 / (nx * ny * mi.cell_volume(p)))
    V = np.zeros((nx, ny))
    y0 = mi.initial_iterate(p, m0, 1e-2, 3)
    out = Solver(p, m0, V, V, method="lu").run(y0)
    assert np.abs(out["y"][0] - m0[None]).max() <= 1e-6 * m0.max()
    assert np.abs(out["y"][1:]).max() <= 1e-6 * m0.max()


def test_field_pcg_solver_matches_lu():
    inst = _field_inst(15, nx=6, ny=6, nt=5, kind="smooth", max_cp=8)
    p = dict(inst["problem"], cg_tol=1e-12)
    a = Solver(p, inst["m0"], inst["V"], inst["W"], method="lu").run(inst["y0"])
    b = Solver(p, inst["m0"], inst["V"], inst["W"], method="pcg").run(inst["y0"])
    assert np.linalg.norm(a["y"] - b["y"]) <= 1e-9 * np.linalg.norm(a["y"])
    assert max(b["cg"]) <= 30


def _converged_field(seed, bc, kind="smooth"):
    from oracle import adjoint as adj
    inst = mi.small(seed, nx=5, ny=4, nt=4, bc=bc, nu=0.2, eps=0.0)
    p = dict(inst["problem"], gamma=0.05)
    p["nu_field"] = mi.viscosity_field(p, 0.2, 4.0, seed + 3, kind)
    rng = np.random.default_rng(seed)
    nx, ny = p["n"]
    m0 = mi._normalise(1.0 + 0.3 * rng.uniform(size=(nx, ny)), p)
    V = 0.3 * rng.normal(size=(nx, ny))
    W = 0.2 * rng.normal(size=(nx, ny))
    res = Solver(p, m0, V, W).run(mi.initial_iterate(p, m0), iters=1500)
    y, z = adj.kkt_newton(p, res["y"], res["z"], m0, V, W)
    mt = mi._normalise(1.0 + 0.3 * rng.uniform(size=(nx, ny)), p)
    return p, m0, V, W, y, z, mt


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("neumann", "periodic")])
def test_field_adjoint_gradient_matches_finite_differences(bc):
    """dloss/dnu(x) at sample nodes (and dloss/dm0, dV along a random direction)
    against central differences through Newton-refined KKT solutions."""
    from oracle import adjoint as adj
    p, m0, V, W, y, z, mt = _converged_field(8, bc)
    _, g = adj.loss_mT(p, y, mt)
    gr = adj.adjoint_gradients(p, y, z, g)
    assert gr["dnu"].shape == tuple(p["n"])
    h = 1e-6

    def loss(q, m0_=m0, V_=V):
        y2, _ = adj.kkt_newton(q, y, z, m0_, V_, W, iters=12)
        return adj.loss_mT(q, y2, mt)[0]

    nu = np.asarray(p["nu_field"])
    for (i, j) in ((0, 0), (2, 1), (4, 3)):
        up, dn = nu.copy(), nu.copy()
        up[i, j] += h
        dn[i, j] -= h
        fd = (loss(dict(p, nu_field=up)) - loss(dict(p, nu_field=dn))) / (2 * h)
        assert abs(fd - gr["dnu"][i, j]) <= 1e-5 * max(1e-3, abs(fd)), ((i, j), fd, gr["dnu"][i, j])
    d = np.random.default_rng(9).normal(size=m0.shape)
    fd = (loss(p, m0_=m0 + h * d) - loss(p, m0_=m0 - h * d)) / (2 * h)
    assert abs(fd - float((gr["dm0"] * d).sum())) <= 1e-5 * max(1e-3, abs(fd))


def test_constant_field_gradient_sums_to_scalar():
    """For a constant field the node derivatives add up to the scalar dnu
    (each face's term is split half and half between its two nodes)."""
    from oracle import adjoint as adj
    from test_oracle_adjoint import _converged
    p, m0, V, W, y, z, mt = _converged(5, ("neumann", "periodic"))
    _, g = adj.loss_mT(p, y, mt)
    scalar = adj.adjoint_gradients(p, y, z, g)["dnu"]
    field = adj.adjoint_gradients(dict(p, nu_field=np.full(p["n"], p["nu"])), y, z, g)["dnu"]
    assert abs(field.sum() - scalar) <= 1e-10 * max(1.0, abs(scalar))
