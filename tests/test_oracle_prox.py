"""Pins of the oracle prox: closed forms, the zero branch and brute force."""
import numpy as np
import pytest
from scipy.optimize import minimize

import mfg_inputs as mi
from oracle import operators as ops
from oracle.prox import coupling, h_eq, project_K, prox


def _cell_objective(u, mbar, wbar, tau, a, b, c):
    m, w = u[0], u[1:]
    if m <= 0:
        return np.inf
    F = 0.5 * a * m * m + b * m ** 3 / 3 + c * m
    return (w @ w) / (2 * m) + F + ((m - mbar) ** 2 + (w - wbar) @ (w - wbar)) / (2 * tau)


def _brute(mbar, wbar, tau, a, b, c):
    """Direct minimisation of b_hat + F + |.-v|^2/(2 tau) over m > 0, w in K."""
    ncomp = len(wbar)
    bounds = [(1e-14, None)] + [((0, None) if i % 2 == 0 else (None, 0)) for i in range(ncomp)]
    best = None
    for m_init in (1e-3, 0.1, 1.0, max(mbar, 1e-3) * 2):
        x0 = np.concatenate([[m_init], project_K(wbar) * 0.5])
        r = minimize(_cell_objective, x0, args=(mbar, wbar, tau, a, b, c), method="L-BFGS-B",
                     bounds=bounds, options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
        if best is None or r.fun < best.fun:
            best = r
    return best


def _one_cell_problem(f_a, f_b=0.0, dim=2):
    p = mi.small(1, dim=dim, nx=1, ny=1, nt=2, f_a=f_a, g_a=0.0)["problem"]
    p = dict(p, f_b=f_b, n=(1, 1))
    return p


@pytest.mark.parametrize("seed", range(12))
def test_prox_vs_brute_force(seed):
    rng = np.random.default_rng(seed)
    f_a = rng.uniform(0.1, 3.0)
    f_b = rng.uniform(0.0, 1.0) if seed % 3 == 0 else 0.0
    p = _one_cell_problem(f_a, f_b)
    tau = 10 ** rng.uniform(-2, 0.5)
    V = np.array([[rng.normal()]])
    W = np.zeros((1, 1))
    v = rng.normal(size=(5, 2, 1, 1)) * 2
    v[0] += 1.5
    out = prox(p, tau, v, V, W)
    a, b, c = coupling(p, V, W)
    for k in range(2):
        mbar, wbar = v[0, k, 0, 0], v[1:, k, 0, 0]
        ours = out[:, k, 0, 0]
        val = _cell_objective(ours, mbar, wbar, tau, a[k, 0, 0], b, c[k, 0, 0]) if ours[0] > 0 \
            else 0.5 * (mbar ** 2 + wbar @ wbar) / tau
        bf = _brute(mbar, wbar, tau, a[k, 0, 0], b, c[k, 0, 0])
        zero_val = 0.5 * (mbar ** 2 + wbar @ wbar) / tau
        best = min(bf.fun, zero_val)
        assert val <= best + 1e-9 * max(1.0, abs(best))
        if ours[0] > 1e-6 and bf.fun < zero_val:
            np.testing.assert_allclose(ours, bf.x, atol=2e-5 * max(1, np.abs(bf.x).max()))


def test_prox_closed_form_without_flux():
    """P_K(w_bar) = 0: m = max(0, (m_bar - tau c)/(1 + tau a)), w = 0."""
    p = _one_cell_problem(1.7)
    rng = np.random.default_rng(3)
    for _ in range(50):
        tau = 10 ** rng.uniform(-2, 1)
        mbar = rng.normal() * 2
        c = rng.normal()
        v = np.zeros((5, 2, 1, 1))
        v[0] = mbar
        v[1] = -abs(rng.normal())   # projects to 0 (w1 >= 0)
        v[2] = abs(rng.normal())    # projects to 0 (w2 <= 0)
        out = prox(p, tau, v, np.array([[c]]), np.zeros((1, 1)))
        ref = max(0.0, (mbar - tau * c) / (1 + tau * 1.7))
        assert abs(out[0, 0, 0, 0] - ref) <= 1e-14 * max(1, abs(ref))
        assert np.all(out[1:] == 0)


def test_prox_zero_branch_and_cone():
    inst = mi.small(9, nx=7, ny=5, nt=4)
    p = inst["problem"]
    v = mi.random_field((5, 4, 7, 5), 3, -2, 2)
    tau = 0.3
    out = prox(p, tau, v, inst["V"], inst["W"])
    assert np.all(out[0] >= 0)
    assert np.all(project_K(out[1:]) == out[1:])
    a, b, c = coupling(p, inst["V"], inst["W"])
    P = project_K(v[1:])
    P2 = (P * P).sum(0)
    h0 = h_eq(0.0, v[0], P2, tau, a, b, c)
    assert np.all(out[0][h0 >= 0] == 0)
    assert np.all(out[1:][:, h0 >= 0] == 0)
    pos = h0 < 0
    assert pos.sum() > 10
    res = h_eq(out[0], v[0], P2, tau, a, b, c)
    assert np.abs(res[pos]).max() < 1e-13 * max(1.0, np.abs(v).max()) * 10
    np.testing.assert_allclose(out[1:][:, pos], (out[0] / (out[0] + tau))[pos] * P[:, pos], atol=1e-15)


def test_terminal_plane_carries_g():
    """Sec. 2 calF: only m^{N_t} sees G/dt."""
    inst = mi.small(2, nx=4, ny=3, nt=3, g_a=0.7)
    p = inst["problem"]
    a, b, c = coupling(p, inst["V"], inst["W"])
    h = ops.dt(p)
    np.testing.assert_allclose(a[:-1], p["f_a"])
    np.testing.assert_allclose(a[-1], p["f_a"] + 0.7 / h)
    np.testing.assert_allclose(c[-1], inst["V"] + inst["W"] / h)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("f_b", [0.0, 0.7])
def test_c_bisection_equals_numpy_bisection(dim, f_b):
    """The plain-C copy of the bisection (used for full-size oracle runs) gives
    the NumPy loop's result bit for bit: zero branch, interior roots, tiny and
    large tau, NaN inputs."""
    from oracle.prox import build_c, prox_cells, prox_cells_numpy
    if build_c() is None:
        pytest.skip("no C compiler")
    rng = np.random.default_rng(17 + dim)
    ncomp = 1 + 2 * dim
    for tau in (1e-6, 1e-3, 0.05, 1.0, 7.0, 1e4):
        v = rng.uniform(-3.0, 3.0, size=(ncomp, 3001))
        v[0, :1000] += 2.0
        v[1:, 5] = 0.0
        v[0, 7] = np.nan
        v[2, 9] = np.nan
        a = rng.uniform(0.0, 2.0, size=3001)
        c = rng.normal(size=3001)
        r_np = prox_cells_numpy(tau, v, a, f_b, c)
        r_c = prox_cells(tau, v, a, f_b, c)
        assert np.array_equal(r_np, r_c, equal_nan=True)
        assert (r_c[0] == 0).any() and (r_c[0] > 0).any()


def _cell_objective_q(u, qp, mbar, wbar, tau, a, b, c):
    m, w = u[0], u[1:]
    if m <= 0:
        return np.inf
    q = qp / (qp - 1.0)
    F = 0.5 * a * m * m + b * m ** 3 / 3 + c * m
    return np.linalg.norm(w) ** q / (q * m ** (q - 1)) + F + ((m - mbar) ** 2 + (w - wbar) @ (w - wbar)) / (2 * tau)


@pytest.mark.parametrize("qp", [1.5, 3.0])
def test_general_q_prox_matches_brute_force(qp):
    """The prox for H = |p|^{q'}/q' against direct minimisation of its definition
    (b_hat = |w|^q/(q m^{q-1}) of Sec. 2 plus F, plus the proximal term)."""
    from oracle.prox import prox_cells_q
    rng = np.random.default_rng(int(qp * 10))
    for trial in range(12):
        ncomp = 4 if trial % 2 == 0 else 2
        mbar = rng.uniform(0.2, 2.0)
        wbar = rng.uniform(-1.5, 1.5, size=ncomp)
        tau, a, b, c = rng.uniform(0.1, 1.5), rng.uniform(0.2, 2.0), rng.uniform(0.0, 0.5), rng.normal(0.0, 0.3)
        v = np.concatenate([[mbar], wbar])[:, None]
        got = prox_cells_q(qp, tau, v, np.array([a]), b, np.array([c]))[:, 0]
        bounds = [(1e-12, None)] + [((0, None) if i % 2 == 0 else (None, 0)) for i in range(ncomp)]
        best = None
        for m_init in (1e-2, 0.3, 1.0, 2.0):
            x0 = np.concatenate([[m_init], project_K(wbar) * 0.5])
            r = minimize(_cell_objective_q, x0, args=(qp, mbar, wbar, tau, a, b, c), method="L-BFGS-B",
                         bounds=bounds, options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
            if best is None or r.fun < best.fun:
                best = r
        f_got = _cell_objective_q(got, qp, mbar, wbar, tau, a, b, c) if got[0] > 0 else np.inf
        assert f_got <= best.fun + 1e-9 * max(1.0, abs(best.fun))
        assert np.abs(got - best.x).max() <= 2e-5 * max(1.0, np.abs(best.x).max())


def test_general_q_prox_reduces_to_quadratic():
    """At q' = 2 the nested-bisection solver gives the q' = 2 prox; the zero
    branch and P = 0 (w = 0, m from m - m_bar + tau f(m) = 0) hold for any q'."""
    from oracle.prox import prox_cells_numpy, prox_cells_q
    rng = np.random.default_rng(5)
    v = rng.uniform(-2.0, 2.0, size=(5, 400))
    v[0] += 0.5
    a = rng.uniform(0.0, 2.0, size=400)
    c = rng.normal(size=400)
    ref = prox_cells_numpy(0.7, v, a, 0.3, c)
    got = prox_cells_q(2.0, 0.7, v, a, 0.3, c)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    for qp in (1.5, 3.0):
        w0 = v.copy()
        w0[1::2] = -np.abs(w0[1::2])  # P = 0: every flux outside the cone
        w0[2::2] = np.abs(w0[2::2])
        out = prox_cells_q(qp, 0.7, w0, a, 0.0, c)
        m_lin = np.maximum(0.0, (w0[0] - 0.7 * c) / (1.0 + 0.7 * a))
        assert np.abs(out[0] - m_lin).max() <= 1e-12 and np.all(out[1:] == 0.0)
