"""Shared helpers for the GPU parity tests: the seeded inputs go to the device,
results come back as numpy arrays for comparison with the oracle."""
import numpy as np


def lib():
    import paper_2507_01958_gb300 as pkg
    return pkg.lib()


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).reshape(-1).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def linf_rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def cp_bound(prob):
    """Parity bar of a CP iterate after a fixed count: max(1e-8, 10 kappa u),
    kappa = cond(AAt) from the oracle's exact per-mode spectrum, u = 2^-53.
    Every exact solve with AAt carries a relative error up to ~kappa u (the
    oracle's own LU and spatially diagonalised solves differ by that much on
    the stiffest small grids)."""
    from oracle import solvers
    return max(1e-8, 10.0 * solvers.cond_AAt(prob) * 2.0 ** -53)
