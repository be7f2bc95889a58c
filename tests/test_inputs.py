"""CPU checks of the seeded input generators (mfg_inputs): the workloads have
the shapes and parameters their docstrings state, densities are normalised on
the grid (sum m0 dx^d = 1), fields are reproducible from their seeds, and the
uneven batch draws its parameters from the stated sets."""
import numpy as np
import pytest

import mfg_inputs as mi


def _mass(m, prob):
    return float(m.sum() * mi.cell_volume(prob))


def test_config1_shape_and_perturbation():
    a, b = mi.config1(), mi.config1()
    p = a["problem"]
    assert p["dim"] == 1 and p["n"] == (64, 1) and p["nt"] == 32 and p["nu"] == 0.1
    assert p["bc"][0] == mi.PERIODIC and p["f_a"] == 1.0 and p["cg_tol"] == 1e-10
    assert abs(_mass(a["m0"], p) - 1.0) <= 1e-13
    assert np.array_equal(a["y0"], b["y0"])
    clean = mi.initial_iterate(p, a["m0"])
    dev = a["y0"] - clean
    assert 0 < np.abs(dev).max() <= 1e-3
    X, _ = mi.nodes(p)
    assert np.allclose(a["V"], 0.5 * np.sin(2 * np.pi * X))


def test_config2_fields():
    for nu in mi.CONFIG2_NU:
        inst = mi.config2(nu=nu, n=32, nt=8)  # same generators on a smaller grid
        p = inst["problem"]
        assert p["nu"] == nu and p["bc"] == (mi.PERIODIC, mi.PERIODIC)
        assert abs(_mass(inst["m0"], p) - 1.0) <= 1e-13 and inst["m0"].min() > 0
        assert np.array_equal(inst["W"], np.zeros_like(inst["W"]))
    rng = np.random.Generator(np.random.PCG64(1))
    p = mi.config2(n=32, nt=8)["problem"]
    V, info = mi.fourier_potential(p, rng)
    ks = info["k"]
    assert len(ks) == 8 and len(set(ks)) == 8
    assert all(0 < kx * kx + ky * ky <= 16 for kx, ky in ks)
    V2, _ = mi.fourier_potential(p, np.random.Generator(np.random.PCG64(1)))
    assert np.array_equal(V, V2)


def test_config3_structure_on_a_small_grid():
    inst = mi.config3(n=16, nt=4)
    p = inst["problem"]
    assert p["bc"] == (mi.NEUMANN, mi.NEUMANN) and p["nu"] == 1e-2
    dx, dy = mi.spacing(p)
    assert dx == dy == 1.0 / 17  # Neumann: L/(N+1)
    X, Y = mi.nodes(p)
    assert np.allclose(inst["W"], 0.1 * ((X - 0.8) ** 2 + (Y - 0.8) ** 2))
    assert abs(_mass(inst["m0"], p) - 1.0) <= 1e-13
    i, j = np.unravel_index(np.argmax(inst["m0"]), inst["m0"].shape)
    assert abs(X[i, j] - 0.2) <= dx and abs(Y[i, j] - 0.2) <= dy


def test_config5_draws():
    insts = mi.config5(count=12, with_y0=False)
    for inst in insts:
        p = inst["problem"]
        assert p["bc"][0] == p["bc"][1] and p["bc"][0] in (mi.PERIODIC, mi.NEUMANN)
        assert p["n"][0] == p["n"][1] and p["n"][0] in (64, 128, 256)
        assert p["nt"] in (32, 64, 128)
        assert 1e-3 <= p["nu"] <= 1.0
        assert abs(_mass(inst["m0"], p) - 1.0) <= 1e-12
    again = mi.config5(count=12, with_y0=False)
    assert all(np.array_equal(a["V"], b["V"]) and np.array_equal(a["m0"], b["m0"]) for a, b in zip(insts, again))


def test_initial_iterate_layout():
    inst = mi.small(3, dim=2, nx=7, ny=5, nt=4, bc=(mi.PERIODIC, mi.NEUMANN))
    p = inst["problem"]
    y0 = mi.initial_iterate(p, inst["m0"])
    assert y0.shape == (5, 4, 7, 5)
    assert np.array_equal(y0[0], np.broadcast_to(inst["m0"], (4, 7, 5)))
    assert not y0[1:].any()


def test_paper_problems():
    """Problem 1 (Sec. 5.1) and Problem 2 (Sec. 5.2) as the paper states them."""
    p1 = mi.problem1(N=16)
    p = p1["problem"]
    assert p["n"] == (16, 16) and p["nt"] == 128 and p["bc"] == ("periodic", "periodic")
    assert p["f_a"] == 0.0 and p["f_b"] == 0.5 and p["gamma"] == 5e-4 and p["cg_rule"] == 1
    X, Y = mi.nodes(p)
    np.testing.assert_allclose(p1["V"], -0.5 * (np.sin(2 * np.pi * Y) + np.sin(2 * np.pi * X) + np.cos(4 * np.pi * X)))
    assert np.all(p1["m0"] == 1.0) and np.all(p1["W"] == 0.0)
    assert p["cp_tol"] == pytest.approx(1e-4 * 16.0)
    p2 = mi.problem2(N=16)
    q = p2["problem"]
    assert q["bc"] == ("neumann", "neumann") and q["nt"] == 128 and q["gamma"] == 5e-3
    assert q["f_a"] == 0.0 and q["f_b"] == 0.0 and q["g_a"] == pytest.approx(1e3)
    X, Y = mi.nodes(q)
    x, y = X - 0.5, Y - 0.5
    assert x.min() == pytest.approx(-0.5 + 1.0 / 17) and x.max() == pytest.approx(0.5 - 1.0 / 17)
    np.testing.assert_allclose(p2["m0"], 3 * np.exp(-128 * ((x + 0.25) ** 2 + (y - 0.25) ** 2)))
    np.testing.assert_allclose(p2["W"], -1e3 * 3 * np.exp(-128 * ((x - 0.25) ** 2 + (y + 0.25) ** 2)))
    assert np.all(p2["V"] == 0.0)
