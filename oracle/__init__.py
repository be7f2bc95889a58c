"""Plain FP64 CPU oracle for the variational MFG solver (test infrastructure).

Only the tests, the smoke entry point and the benchmark's CPU-baseline leg may
import this package.  The product path never calls it and shares no code with
it: no kernels, tables, helpers or constant generators.  Both sides only share
the seeded input generators in ``mfg_inputs``.

Contents (paper sections in brackets):
  operators  sparse D1, D2, B, K, L, the reduced constraint C, d, AAt = C C^T and
             the preconditioner P [Sec. 2, Sec. 3 eq. ABC / largeA, Sec. 4 eq. prec]
  solvers    direct LU, plain CG, the exact spatially-diagonalised solver for AAt
             and for P [Sec. 3, Sec. 4.3]
  prox       per-cell prox of tau*phi by bisection [Sec. 3]
  cp         accelerated Chambolle-Pock iteration [Sec. 3, Sec. 5 setup]
  checks     mass, constraint residual, objective, conjugate, duality gap

Every function is pinned by the CPU test-suite against facts fixed by the paper
or by mathematics (identities, closed forms, brute force); see the per-function
docstrings for the pin.

set_threads(k) sets how many host threads the FFTs and the C copy of the prox
bisection use (default: all cores); results do not depend on it.
"""
import os as _os


def set_threads(k=None):
    """Host threads for scipy.fft and the C prox (None: os.cpu_count())."""
    from . import prox, solvers
    k = int(k or _os.cpu_count() or 1)
    solvers._WORKERS = k
    prox._THREADS = k
    return k
