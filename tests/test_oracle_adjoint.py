"""Pins of the oracle's implicit-differentiation gradient: central finite
differences of the loss through exact (Newton-refined) KKT solutions."""
import numpy as np
import pytest

import mfg_inputs as mi
from oracle import adjoint as adj
from oracle import operators as ops
from oracle.cp import Solver


def _converged(seed, bc, nu=0.2, dim=2):
    inst = mi.small(seed, dim=dim, nx=5, ny=4, nt=4, bc=bc, nu=nu, eps=0.0)
    p = dict(inst["problem"], gamma=0.05)
    rng = np.random.default_rng(seed)
    nx, ny = p["n"]
    m0 = mi._normalise(1.0 + 0.3 * rng.uniform(size=(nx, ny)), p)
    V = 0.3 * rng.normal(size=(nx, ny))
    W = 0.2 * rng.normal(size=(nx, ny))
    res = Solver(p, m0, V, W).run(mi.initial_iterate(p, m0), iters=1500)
    y, z = adj.kkt_newton(p, res["y"], res["z"], m0, V, W)
    mt = mi._normalise(1.0 + 0.3 * rng.uniform(size=(nx, ny)), p)
    return p, m0, V, W, y, z, mt


def _loss_at(p, m0, V, W, y, z, mt):
    y2, _ = adj.kkt_newton(p, y, z, m0, V, W, iters=12)
    return adj.loss_mT(p, y2, mt)[0]


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("neumann", "periodic")])
def test_kkt_newton_reaches_round_off(bc):
    p, m0, V, W, y, z, mt = _converged(3, bc)
    r1, r2 = adj.kkt_residual(p, y, z, m0, V, W)
    assert np.abs(r1).max() < 1e-10 and np.abs(r2).max() < 1e-10 * np.abs(ops.rhs_d(p, m0)).max()
    # the CP solution and the refined KKT point agree (the CP run had converged)
    assert adj.active_mask(y).sum() > 0


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("neumann", "periodic")])
def test_adjoint_gradient_matches_finite_differences(bc):
    p, m0, V, W, y, z, mt = _converged(5, bc)
    _, g = adj.loss_mT(p, y, mt)
    gr = adj.adjoint_gradients(p, y, z, g)
    rng = np.random.default_rng(7)
    h = 1e-6
    # nu
    lp = _loss_at(dict(p, nu=p["nu"] + h), m0, V, W, y, z, mt)
    lm = _loss_at(dict(p, nu=p["nu"] - h), m0, V, W, y, z, mt)
    fd = (lp - lm) / (2 * h)
    assert abs(fd - gr["dnu"]) <= 1e-5 * max(1e-3, abs(fd))
    # m0, V, W along random directions
    for key, field in (("dm0", "m0"), ("dV", "V"), ("dW", "W")):
        d = rng.normal(size=m0.shape)
        args = {"m0": m0, "V": V, "W": W}
        ap = dict(args); ap[field] = args[field] + h * d
        am = dict(args); am[field] = args[field] - h * d
        lp = _loss_at(p, ap["m0"], ap["V"], ap["W"], y, z, mt)
        lm = _loss_at(p, am["m0"], am["V"], am["W"], y, z, mt)
        fd = (lp - lm) / (2 * h)
        an = float((gr[key] * d).sum())
        assert abs(fd - an) <= 1e-5 * max(1e-3, abs(fd)), (key, fd, an)
