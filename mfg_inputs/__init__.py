"""Seeded synthetic inputs for the variational MFG solver.

This module is shared by the CPU oracle and the CUDA path.  It builds problem
descriptors (plain dicts) and input fields (numpy float64 arrays) and holds none
of the method's arithmetic: no operators, no proximal maps, no solves.

Workloads follow the shapes of the paper's experiments (Sec. 5: structured
periodic and Neumann grids, N_t time steps, viscosity nu, quadratic
Hamiltonian) with analytic, seeded fields in place of data; the paper uses no
dataset.  Grid nodes follow Sec. 2: periodic x_i = a + i*dx with dx = L/N,
Neumann interior nodes x_i = a + i*dx, i = 1..N, with dx = L/(N+1).

Problem dict keys (all instances):
  dim (1|2), n (Nx, Ny) with Ny = 1 when dim == 1, len (Lx, Ly),
  bc (per-axis "periodic"|"neumann"), nt, T, nu, qprime, f_a, f_b, g_a, l,
  gamma, tau0, sigma0, max_cp, cp_tol, cg_rule, cg_tol, max_cg.
Fields: m0 (Nx, Ny), V (Nx, Ny), W (Nx, Ny), y0 (c, nt, Nx, Ny) with
c = 1 + 2*dim planes ordered (m, w1, w2[, w3, w4]).
"""
from __future__ import annotations

import numpy as np

PERIODIC = "periodic"
NEUMANN = "neumann"


def _problem(dim, nx, ny, bc, nt, nu, *, T=1.0, lx=1.0, ly=1.0, f_a=1.0, f_b=0.0,
             g_a=0.0, l=1, gamma=1e-3, max_cp=300, cp_tol=0.0, cg_rule=0,
             cg_tol=1e-10, max_cg=10000):
    if dim == 1:
        ny, ly = 1, 1.0
        bc = (bc[0], PERIODIC)
    return {
        "dim": int(dim), "n": (int(nx), int(ny)), "len": (float(lx), float(ly)),
        "bc": (bc[0], bc[1]), "nt": int(nt), "T": float(T), "nu": float(nu),
        "qprime": 2.0, "f_a": float(f_a), "f_b": float(f_b), "g_a": float(g_a),
        "l": int(l), "gamma": float(gamma), "tau0": 1.0, "sigma0": 1.0,
        "max_cp": int(max_cp), "cp_tol": float(cp_tol), "cg_rule": int(cg_rule),
        "cg_tol": float(cg_tol), "max_cg": int(max_cg),
    }


def spacing(prob):
    """Grid spacing per axis (Sec. 2: L/N periodic, L/(N+1) Neumann)."""
    out = []
    for ax in range(2):
        n, length, bc = prob["n"][ax], prob["len"][ax], prob["bc"][ax]
        out.append(length / n if bc == PERIODIC else length / (n + 1))
    return tuple(out)


def nodes(prob):
    """Node coordinates (X, Y), each (Nx, Ny); domain origin at 0."""
    dx, dy = spacing(prob)
    nx, ny = prob["n"]
    off_x = 0 if prob["bc"][0] == PERIODIC else 1
    off_y = 0 if prob["bc"][1] == PERIODIC else 1
    x = (np.arange(nx) + off_x) * dx
    y = (np.arange(ny) + off_y) * dy if prob["dim"] == 2 else np.zeros(1)
    return np.meshgrid(x, y, indexing="ij")


def n_planes(prob):
    return 1 + 2 * prob["dim"]


def cell_volume(prob):
    dx, dy = spacing(prob)
    return dx * (dy if prob["dim"] == 2 else 1.0)


def _normalise(m, prob):
    return m / (m.sum() * cell_volume(prob))


def initial_iterate(prob, m0, eps=0.0, seed=None):
    """CP start: m^k = m0 for every k, w = 0, plus eps*U(-1,1) i.i.d. if eps > 0."""
    nx, ny = prob["n"]
    y0 = np.zeros((n_planes(prob), prob["nt"], nx, ny))
    y0[0] = m0[None]
    if eps > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        y0 += eps * rng.uniform(-1.0, 1.0, size=y0.shape)
    return y0


def gaussian_mixture(prob, rng, k=3, sig_lo=0.05, sig_hi=0.15, images=2):
    """Normalised mixture of k Gaussians; periodic images |p| <= images on periodic axes."""
    X, Y = nodes(prob)
    m = np.zeros_like(X)
    lx, ly = prob["len"]
    for _ in range(k):
        c = rng.uniform(0.0, 1.0, size=2) * np.array([lx, ly])
        s = rng.uniform(sig_lo, sig_hi)
        px = range(-images, images + 1) if prob["bc"][0] == PERIODIC else [0]
        py = range(-images, images + 1) if (prob["bc"][1] == PERIODIC and prob["dim"] == 2) else [0]
        for p in px:
            for q in py:
                dy2 = (Y - c[1] - q * ly) ** 2 if prob["dim"] == 2 else 0.0
                m += np.exp(-((X - c[0] - p * lx) ** 2 + dy2) / (2 * s * s))
    return _normalise(m, prob)


def fourier_potential(prob, rng, modes=8, kmax=4, std=0.5):
    """V(x) = sum a cos(2 pi k.x + phi): distinct nonzero integer k with |k| <= kmax,
    a ~ N(0, std^2), phi ~ U[0, 2 pi)."""
    X, Y = nodes(prob)
    cand = [(a, b) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1)
            if 0 < a * a + b * b <= kmax * kmax]
    if prob["dim"] == 1:
        cand = [(a, 0) for a in range(1, kmax + 1)]
    idx = rng.choice(len(cand), size=min(modes, len(cand)), replace=False)
    amp = rng.normal(0.0, std, size=len(idx))
    ph = rng.uniform(0.0, 2 * np.pi, size=len(idx))
    lx, ly = prob["len"]
    V = np.zeros_like(X)
    for (t, a, p) in zip(idx, amp, ph):
        kx, ky = cand[t]
        V += a * np.cos(2 * np.pi * (kx * X / lx + ky * Y / ly) + p)
    return V, {"k": [cand[t] for t in idx], "amp": amp, "phase": ph}


def cosine_potential(prob, rng, kmax=3, std=0.5):
    """V(x) = sum_{0<=k1,k2<=kmax} a_k cos(pi k1 x) cos(pi k2 y), a_k ~ N(0, std^2)/(1+k1^2+k2^2)."""
    X, Y = nodes(prob)
    lx, ly = prob["len"]
    V = np.zeros_like(X)
    for k1 in range(kmax + 1):
        for k2 in range(kmax + 1 if prob["dim"] == 2 else 1):
            a = rng.normal(0.0, std) / (1 + k1 * k1 + k2 * k2)
            V += a * np.cos(np.pi * k1 * X / lx) * np.cos(np.pi * k2 * Y / ly)
    return V


def _inst(prob, m0, V, W, y0, **extra):
    d = {"problem": prob, "m0": m0, "V": V, "W": W, "y0": y0}
    d.update(extra)
    return d


def config1():
    """1-D periodic torus [0,1), N_x = 64, N_t = 32, T = 1, nu = 0.1,
    f = m + 0.5 sin(2 pi x), g = 0, m0 a normalised periodic Gaussian (centre 0.5,
    sigma 0.1, images |p| <= 4), 300 CP iterations, PCG tol 1e-10, start perturbed by
    1e-3*U(-1,1) (PCG64 seed 0)."""
    prob = _problem(1, 64, 1, (PERIODIC, PERIODIC), 32, 0.1, max_cp=300, cg_tol=1e-10)
    X, _ = nodes(prob)
    m0 = sum(np.exp(-(X - 0.5 - p) ** 2 / (2 * 0.1 ** 2)) for p in range(-4, 5))
    m0 = _normalise(m0, prob)
    V = 0.5 * np.sin(2 * np.pi * X)
    W = np.zeros_like(X)
    return _inst(prob, m0, V, W, initial_iterate(prob, m0, 1e-3, 0))


CONFIG2_NU = (1e-3, 1e-2, 1e-1, 1.0)


def config2(nu=1e-2, n=128, nt=64):
    """2-D periodic torus, 128^2, N_t = 64, f = m + V(x) with V 8 seeded Fourier
    modes (seed 1), g = 0, m0 a 3-Gaussian mixture (seed 2)."""
    prob = _problem(2, n, n, (PERIODIC, PERIODIC), nt, nu, max_cp=300, cg_tol=1e-10)
    V, _ = fourier_potential(prob, np.random.Generator(np.random.PCG64(1)))
    m0 = gaussian_mixture(prob, np.random.Generator(np.random.PCG64(2)))
    W = np.zeros_like(V)
    return _inst(prob, m0, V, W, initial_iterate(prob, m0))


def config3(n=512, nt=128, nu=1e-2):
    """2-D Neumann unit square, 512^2, N_t = 128, nu = 1e-2, V a seeded cosine
    series (seed 3), g(x,m) = 0.1 |x - (0.8,0.8)|^2, m0 a Gaussian at (0.2, 0.2),
    sigma 0.08, normalised on the grid."""
    prob = _problem(2, n, n, (NEUMANN, NEUMANN), nt, nu, max_cp=300, cg_tol=1e-10)
    V = cosine_potential(prob, np.random.Generator(np.random.PCG64(3)))
    X, Y = nodes(prob)
    W = 0.1 * ((X - 0.8) ** 2 + (Y - 0.8) ** 2)
    m0 = _normalise(np.exp(-((X - 0.2) ** 2 + (Y - 0.2) ** 2) / (2 * 0.08 ** 2)), prob)
    return _inst(prob, m0, V, W, initial_iterate(prob, m0))


def config4(n=128, nt=64):
    """Adjoint workload: config2 geometry, nu = 0.05; m0 a 3-Gaussian mixture
    (seed 5), target m_target a 3-Gaussian mixture (seed 4), V as config2."""
    prob = _problem(2, n, n, (PERIODIC, PERIODIC), nt, 0.05, max_cp=300, cg_tol=1e-10)
    V, vinfo = fourier_potential(prob, np.random.Generator(np.random.PCG64(1)))
    m0 = gaussian_mixture(prob, np.random.Generator(np.random.PCG64(5)))
    mt = gaussian_mixture(prob, np.random.Generator(np.random.PCG64(4)))
    W = np.zeros_like(V)
    return _inst(prob, m0, V, W, initial_iterate(prob, m0), m_target=mt, v_modes=vinfo)


def config5_instance(seed, sizes=(64, 128, 256), nts=(32, 64, 128), with_y0=True):
    """One instance of the uneven batch: bc ~ U{periodic, Neumann}, N ~ U(sizes),
    N_t ~ U(nts), nu = 10^U(-3, 0); V, m0 as config2 (cosine series for Neumann)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bc = PERIODIC if rng.uniform() < 0.5 else NEUMANN
    n = int(rng.choice(sizes))
    nt = int(rng.choice(nts))
    nu = float(10.0 ** rng.uniform(-3.0, 0.0))
    prob = _problem(2, n, n, (bc, bc), nt, nu, max_cp=300, cg_tol=1e-10)
    if bc == PERIODIC:
        V, _ = fourier_potential(prob, rng)
    else:
        V = cosine_potential(prob, rng)
    m0 = gaussian_mixture(prob, rng, images=2 if bc == PERIODIC else 0)
    W = np.zeros_like(V)
    return _inst(prob, m0, V, W, initial_iterate(prob, m0) if with_y0 else None)


def config5(count=64, first_seed=100, **kw):
    return [config5_instance(first_seed + i, **kw) for i in range(count)]


def problem1(N=16, nt=None, nu=0.01):
    """Problem 1 of Sec. 5.1 (crowd aversion on the torus [0,1)^2):
    f(x, y, m) = (m^2 - sin 2 pi y - sin 2 pi x - cos 4 pi x)/2, i.e. f_a = 0,
    f_b = 1/2, V = -(sin 2 pi y + sin 2 pi x + cos 4 pi x)/2; m0 = 1, g = 0,
    gamma = 5e-4; N_x = N_y = N, N_t = 8N (Tables 1-2); the stop rule
    CPtol = 1e-4 ||m0|| and the adaptive CG rule of Sec. 5."""
    nt = 8 * N if nt is None else nt
    prob = _problem(2, N, N, (PERIODIC, PERIODIC), nt, nu, f_a=0.0, f_b=0.5, gamma=5e-4, max_cp=5000,
                    cg_rule=1)
    X, Y = nodes(prob)
    V = -0.5 * (np.sin(2 * np.pi * Y) + np.sin(2 * np.pi * X) + np.cos(4 * np.pi * X))
    m0 = np.ones((N, N))
    prob["cp_tol"] = 1e-4 * float(np.linalg.norm(m0))
    W = np.zeros_like(V)
    return _inst(prob, m0, V, W, initial_iterate(prob, m0))


def problem2(N=16, nt=None, nu=0.01, beta=1e-3):
    """Problem 2 of Sec. 5.2 (Gaussian final target on the Neumann square
    [-1/2, 1/2]^2): f = 0, g(x, y, m) = (m - m_bar)/beta with beta = 1e-3 (so
    g_a = 1/beta, W = -m_bar/beta; G enters the last plane divided by dt),
    m0 = 3 exp(-2^7 ((x + 1/4)^2 + (y - 1/4)^2)),
    m_bar = 3 exp(-2^7 ((x - 1/4)^2 + (y + 1/4)^2)) on the interior nodes
    x_i = -1/2 + i dx, dx = 1/(N+1); gamma = 5e-3; N_t = 8N (Table 3); CPtol
    = 1e-4 ||m0|| and the adaptive CG rule of Sec. 5."""
    nt = 8 * N if nt is None else nt
    prob = _problem(2, N, N, (NEUMANN, NEUMANN), nt, nu, f_a=0.0, f_b=0.0, g_a=1.0 / beta, gamma=5e-3,
                    max_cp=5000, cg_rule=1)
    X, Y = nodes(prob)
    X, Y = X - 0.5, Y - 0.5  # the domain starts at -1/2
    m0 = 3.0 * np.exp(-2.0 ** 7 * ((X + 0.25) ** 2 + (Y - 0.25) ** 2))
    mbar = 3.0 * np.exp(-2.0 ** 7 * ((X - 0.25) ** 2 + (Y + 0.25) ** 2))
    prob["cp_tol"] = 1e-4 * float(np.linalg.norm(m0))
    V = np.zeros_like(X)
    W = -mbar / beta
    return _inst(prob, m0, V, W, initial_iterate(prob, m0), m_target=mbar)


def viscosity_field(prob, nu0, ratio, seed, kind="smooth"):
    """Seeded viscosity field nu(x) (shape (Nx, Ny)) with max/min = ratio and
    geometric centre nu0.  kind "smooth": nu0 * ratio**(u/2) with u a random
    cosine series (4 modes per axis, PCG64(seed)) rescaled to [-1, 1];
    kind "layers": nu0 / sqrt(ratio) on one side of a seeded straight interface
    and nu0 * sqrt(ratio) on the other (a discontinuous coefficient)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y = nodes(prob)
    lx, ly = prob["len"]
    if kind == "layers":
        ang = rng.uniform(0.0, np.pi)
        c = rng.uniform(0.35, 0.65)
        side = np.cos(ang) * (X / lx - c) + np.sin(ang) * (Y / ly - c) > 0
        return np.where(side, nu0 * np.sqrt(ratio), nu0 / np.sqrt(ratio))
    u = np.zeros_like(X)
    for _ in range(4):
        kx, ky = rng.integers(0, 4, size=2)
        ph = rng.uniform(0.0, 2.0 * np.pi, size=2)
        u += rng.normal() * np.cos(np.pi * kx * X / lx + ph[0]) * np.cos(np.pi * ky * Y / ly + ph[1])
    span = u.max() - u.min()
    u = 2.0 * (u - u.min()) / span - 1.0 if span > 0 else np.zeros_like(u)
    return nu0 * ratio ** (0.5 * u)


def config_varnu(n=128, nt=64, nu=1e-2, ratio=10.0, kind="smooth"):
    """2-D Neumann unit square with a viscosity field nu(x) (seed 7, max/min =
    ratio around nu), otherwise the Neumann workload's fields: V a seeded cosine
    series (seed 3), g = 0.1 |x - (0.8,0.8)|^2, m0 a Gaussian at (0.2, 0.2),
    sigma 0.08."""
    inst = config3(n=n, nt=nt, nu=nu)
    inst["problem"]["nu_field"] = viscosity_field(inst["problem"], nu, ratio, 7, kind)
    return inst


def small(seed, dim=2, nx=None, ny=None, nt=None, bc=None, nu=None, l=None,
          f_a=None, g_a=None, eps=1e-2, max_cp=20):
    """Small random instance for parity tests: ragged sizes, random fields."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx = nx or int(rng.integers(5, 13))
    ny = ny or int(rng.integers(4, 11))
    nt = nt or int(rng.integers(3, 9))
    if bc is None:
        bc = tuple(PERIODIC if rng.uniform() < 0.5 else NEUMANN for _ in range(2))
    nu = float(10.0 ** rng.uniform(-3, 0)) if nu is None else nu
    l = int(rng.integers(1, 3)) if l is None else l
    f_a = float(rng.uniform(0.2, 2.0)) if f_a is None else f_a
    g_a = float(rng.uniform(0.0, 1.0)) if g_a is None else g_a
    prob = _problem(dim, nx, ny, bc, nt, nu, f_a=f_a, g_a=g_a, l=l, max_cp=max_cp,
                    lx=float(rng.uniform(0.5, 2.0)), ly=float(rng.uniform(0.5, 2.0)),
                    T=float(rng.uniform(0.5, 2.0)))
    shp = prob["n"]
    m0 = _normalise(rng.uniform(0.1, 1.0, size=shp), prob)
    V = rng.normal(0.0, 0.5, size=shp)
    W = rng.normal(0.0, 0.5, size=shp)
    return _inst(prob, m0, V, W, initial_iterate(prob, m0, eps, seed + 1))


def random_field(shape, seed, lo=-1.0, hi=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)
