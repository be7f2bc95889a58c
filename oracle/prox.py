"""Per-cell proximal map of tau*phi, phi_{ij} = b_hat + F (Sec. 3).

The paper takes the formula from its reference [BAKS, Cor. 3.1] without
printing it; the oracle derives it from the first-order conditions for q' = 2:

  phi(m, w) = |w|^2/(2m) + F_eff(m),  m > 0, w in K;  phi(0, 0) = F_eff(0),
  F_eff(m) = F(x, m) [+ G(x, m)/dt on the last time plane, Sec. 2 calF].

For fixed m > 0 the w-part is separable per component and the minimiser is
w = m/(m + tau) * P with P = P_K(w_bar) (Sec. 2 projection onto K).  The
envelope theorem then gives the scalar equation for m,

  h(m) = m - m_bar + tau f_eff(m) - tau |P|^2 / (2 (m + tau)^2) = 0,

with h strictly increasing because f_eff is nondecreasing.  If h(0) >= 0 the
prox is (0, 0); otherwise the root lies in (0, m_hi] with
m_hi = max(0, m_bar - tau f_eff(0)) + |P|^2/(2 tau), where h(m_hi) >= 0.
The oracle brackets the root there and bisects until the bracket cannot shrink
in FP64.  Pins: closed forms for P = 0, the zero branch, and brute-force
minimisation of the definition on random cells (tests).

General power Hamiltonian H = |p|^{q'}/q' (eq. power_hamiltonian), q = q'/(q'-1),
b_hat(m, w) = |w|^q / (q m^{q-1}) (Sec. 2).  For fixed m > 0 the w-part only
depends on |w| and the cone, so the minimiser is w = rho P/|P| with
rho = m t and t >= 0 the root of
  g(t) = m t + tau t^{q-1} - |P| = 0            (d/d rho of the w-part),
and the envelope theorem gives the scalar equation for m,
  h_q(m) = m - m_bar + tau f_eff(m) - (tau/q') t(m)^q = 0,
strictly increasing (t decreases with m).  As m -> 0, t -> t0 = (|P|/tau)^{1/(q-1)}
and rho -> 0: (0, 0) is the prox when h_q(0) = tau f_eff(0) - m_bar
- (tau/q') (|P|/tau)^{q'} >= 0; otherwise the root lies in (0, m_hi] with
m_hi = max(0, m_bar - tau f_eff(0)) + (tau/q') (|P|/tau)^{q'}.  q' = 2 gives the
equation above (t = |P|/(m + tau)).  prox_cells_q solves it by nested
bisection (t for each trial m, then m), both until the bracket cannot shrink.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .operators import dt

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prox_bisect.c")
_SO = os.path.join(_HERE, "_build", "liboracle_prox.so")
_clib = None
_THREADS = os.cpu_count() or 1


def build_c():
    """Compiles prox_bisect.c (the same bisection in plain C, for full-size
    runs) with every operation separately rounded (-ffp-contract=off); returns
    the library path, or None if no C compiler is available."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True)
    except OSError:
        return None
    if r.returncode != 0:
        return None
    os.replace(tmp, _SO)
    return _SO


def _c_library():
    global _clib
    if _clib is None:
        if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            if build_c() is None:
                _clib = False
                return None
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.oracle_prox_cells.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_double, P, P,
                                          ctypes.c_double, P, P, ctypes.c_int, ctypes.c_int]
        lib.oracle_prox_cells.restype = ctypes.c_int
        _clib = lib
    return _clib or None


def project_K(wbar):
    """P_K: components (1, 3) clipped to [0, inf), components (2, 4) to (-inf, 0]."""
    P = np.array(wbar, dtype=np.float64, copy=True)
    P[0::2] = np.maximum(P[0::2], 0.0)
    P[1::2] = np.minimum(P[1::2], 0.0)
    return P


def coupling(prob, V, W):
    """Per-plane coefficients of f_eff(m) = a m + b m^2 + c: (a, b, c) with
    a, c of shape (nt, Nx, Ny); the last plane carries g/dt (Sec. 2, calF)."""
    nt = prob["nt"]
    nx, ny = prob["n"]
    a = np.full((nt, nx, ny), prob["f_a"])
    c = np.broadcast_to(np.asarray(V, dtype=np.float64).reshape(nx, ny), (nt, nx, ny)).copy()
    a[-1] += prob["g_a"] / dt(prob)
    c[-1] += np.asarray(W, dtype=np.float64).reshape(nx, ny) / dt(prob)
    return a, prob["f_b"], c


def h_eq(m, mbar, P2, tau, a, b, c):
    return m - mbar + tau * (a * m + b * m * m + c) - tau * P2 / (2.0 * (m + tau) ** 2)


def prox(prob, tau, v, V, W, max_iter=4000):
    """prox_{tau phi}(v) for v of shape (c, nt, Nx, Ny); returns the same shape.
    prob["qprime"] (default 2) selects the Hamiltonian's exponent q'."""
    v = np.asarray(v, dtype=np.float64)
    a, b, c = coupling(prob, V, W)
    qp = float(prob.get("qprime", 2.0))
    if qp != 2.0:
        return prox_cells_q(qp, tau, v, a, b, c, max_iter)
    return prox_cells(tau, v, a, b, c, max_iter)


def _bisect(fun, lo, hi, max_iter):
    """Vectorised bisection of an increasing function on [lo, hi] (fun(lo) < 0
    <= fun(hi) where active) until the midpoint equals an endpoint; returns
    the endpoint with the smaller |fun|."""
    lo, hi = lo.copy(), hi.copy()
    active = np.ones(lo.shape, dtype=bool)
    for _ in range(max_iter):
        if not active.any():
            break
        mid = lo + 0.5 * (hi - lo)
        active &= ~((mid <= lo) | (mid >= hi))
        fm = fun(mid)
        neg = active & (fm < 0.0)
        pos = active & ~(fm < 0.0)
        lo = np.where(neg, mid, lo)
        hi = np.where(pos, mid, hi)
    return np.where(np.abs(fun(lo)) < np.abs(fun(hi)), lo, hi)


def velocity_q(qprime, tau, m, Pn, max_iter=4000):
    """t >= 0 with m t + tau t^(q-1) = |P| (q = q'/(q'-1)), by bisection on
    [0, min(|P|/m, (|P|/tau)^(1/(q-1)))]; m > 0."""
    q = qprime / (qprime - 1.0)
    m, Pn = np.broadcast_arrays(np.asarray(m, dtype=np.float64), np.asarray(Pn, dtype=np.float64))
    hi = np.minimum(Pn / m, (Pn / tau) ** (1.0 / (q - 1.0)))
    t = _bisect(lambda t: m * t + tau * t ** (q - 1.0) - Pn, np.zeros_like(hi), hi, max_iter)
    return np.where(Pn > 0, t, 0.0)


def prox_cells_q(qprime, tau, v, a, b, c, max_iter=4000):
    """prox_cells for the Hamiltonian |p|^{q'}/q' (header): nested bisection."""
    v = np.asarray(v, dtype=np.float64)
    q = qprime / (qprime - 1.0)
    shp = v.shape[1:]
    mbar = v[0]
    P = project_K(v[1:])
    Pn = np.sqrt((P * P).sum(axis=0))
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), shp)
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), shp)
    f0 = c
    lim = (tau / qprime) * (Pn / tau) ** qprime
    zero = (tau * f0 - mbar - lim) >= 0.0
    hi = np.maximum(0.0, mbar - tau * f0) + lim
    lo = np.zeros_like(hi)
    hi = np.where(zero, 1.0, hi)  # inactive cells: any valid bracket

    def hq(m):
        mm = np.maximum(m, np.finfo(float).tiny)
        t = velocity_q(qprime, tau, mm, Pn, max_iter)
        return m - mbar + tau * (a * m + b * m * m + c) - (tau / qprime) * t ** q

    m = _bisect(hq, lo, hi, max_iter)
    m = np.where(zero, 0.0, m)
    t = velocity_q(qprime, tau, np.maximum(m, np.finfo(float).tiny), Pn, max_iter)
    scale = np.where((Pn > 0) & ~zero, m * t / np.where(Pn > 0, Pn, 1.0), 0.0)
    out = np.empty_like(v)
    out[0] = m
    out[1:] = scale[None] * P
    return out


def prox_cells(tau, v, a, b, c, max_iter=4000, use_c=True):
    """The same map for any set of cells: v of shape (c, ...) with coefficient
    arrays a, c of shape v.shape[1:] and scalar b.  Runs the plain-C copy of
    the bisection (prox_bisect.c, identical results, threads over cells) when
    it can be built, else the NumPy loop below."""
    v = np.asarray(v, dtype=np.float64)
    lib = _c_library() if use_c else None
    if lib is not None and v.shape[0] in (3, 5):
        shp = v.shape
        vc = np.ascontiguousarray(v.reshape(shp[0], -1))
        n = vc.shape[1]
        ac = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shp[1:]).reshape(-1))
        cc = np.ascontiguousarray(np.broadcast_to(np.asarray(c, dtype=np.float64), shp[1:]).reshape(-1))
        out = np.empty_like(vc)
        rc = lib.oracle_prox_cells(shp[0] - 1, n, float(tau), vc.ctypes.data, ac.ctypes.data, float(b),
                                   cc.ctypes.data, out.ctypes.data, int(max_iter), int(_THREADS))
        if rc != 0:
            raise RuntimeError("oracle_prox_cells rejected its arguments")
        return out.reshape(shp)
    return prox_cells_numpy(tau, v, a, b, c, max_iter)


def prox_cells_numpy(tau, v, a, b, c, max_iter=4000):
    """The bisection over all cells at once in NumPy (the reference the C copy
    is checked against)."""
    v = np.asarray(v, dtype=np.float64)
    mbar = v[0]
    P = project_K(v[1:])
    P2 = (P * P).sum(axis=0)
    zero = h_eq(0.0, mbar, P2, tau, a, b, c) >= 0.0
    lo = np.zeros_like(mbar)
    hi = np.maximum(0.0, mbar - tau * c) + P2 / (2.0 * tau)
    active = ~zero
    for _ in range(max_iter):
        if not active.any():
            break
        mid = lo + 0.5 * (hi - lo)
        stuck = (mid <= lo) | (mid >= hi)
        active &= ~stuck
        hm = h_eq(mid, mbar, P2, tau, a, b, c)
        neg = active & (hm < 0.0)
        pos = active & ~(hm < 0.0)
        lo = np.where(neg, mid, lo)
        hi = np.where(pos, mid, hi)
    hlo = np.abs(h_eq(lo, mbar, P2, tau, a, b, c))
    hhi = np.abs(h_eq(hi, mbar, P2, tau, a, b, c))
    m = np.where(hlo < hhi, lo, hi)
    m = np.where(zero, 0.0, m)
    out = np.empty_like(v)
    out[0] = m
    out[1:] = (m / (m + tau))[None] * P
    out[1:, zero] = 0.0
    return out
