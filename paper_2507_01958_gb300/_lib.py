"""ctypes binding of the C ABI in include/mfg.h: argument marshalling only.

Every computation happens in libmfg_gb300.so (CUDA kernels for sm_103a).  If
the library has not been built this module raises on import; there is no CPU
path.  Tensors are torch tensors (device memory and streams come from
PyTorch); each function has the name of the C entry point it calls.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmfg_gb300.so")

MFG_OK, MFG_ERR_INVALID_ARG, MFG_ERR_UNSUPPORTED, MFG_ERR_CUDA = 0, 1, 2, 3
MFG_ERR_NOT_CONVERGED, MFG_ERR_NONFINITE, MFG_ERR_TIMEOUT = 4, 5, 6
MFG_PERIODIC, MFG_NEUMANN = 0, 1
MFG_FP64, MFG_MIXED, MFG_MIXED_DF, MFG_MIXED_TC = 0, 1, 2, 3
MFG_CG_FIXED, MFG_CG_ADAPTIVE = 0, 1
MFG_LAUNCH_GRAPH, MFG_LAUNCH_EAGER = 0, 1
MFG_CG_REF_RHS, MFG_CG_REF_RESID = 0, 1
MFG_INJECT_NONE, MFG_INJECT_TC_NO_COMMIT, MFG_INJECT_BAND_NO_COPY = 0, 1, 2


class MfgProblem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 2), ("len", C.c_double * 2), ("bc", C.c_int * 2),
                ("nt", C.c_int), ("T", C.c_double), ("nu", C.c_double), ("qprime", C.c_double),
                ("f_a", C.c_double), ("f_b", C.c_double), ("g_a", C.c_double), ("l", C.c_int),
                ("gamma", C.c_double), ("tau0", C.c_double), ("sigma0", C.c_double),
                ("max_cp", C.c_int), ("cp_tol", C.c_double), ("cg_rule", C.c_int),
                ("cg_tol", C.c_double), ("max_cg", C.c_int), ("precision", C.c_int),
                ("cg_ref", C.c_int), ("nu_field", C.POINTER(C.c_double))]


class MfgStats(C.Structure):
    _fields_ = [("status", C.c_int), ("ell", C.c_int), ("cp_iters", C.c_int),
                ("max_cg_in_solve", C.c_int), ("cg_iters", C.c_longlong), ("r_last", C.c_double),
                ("tau", C.c_double), ("sigma", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MfgSchedule(C.Structure):
    _fields_ = [("tuned", C.c_int), ("measured", C.c_int), ("time_pass", C.c_int), ("fft", C.c_int * 2),
                ("aat_blocks", C.c_int), ("vec_blocks", C.c_int), ("precond_us", C.c_double),
                ("aat_us", C.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["fft"] = list(self.fft)
        d["time_pass"] = "tensor_cores" if self.time_pass == 0 else "cuda_cores"
        return d


class MfgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mfg error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2507_01958_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P, I, D, V, SZ = C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_size_t
    sig = {
        "mfg_plan": ([C.POINTER(MfgProblem), I, C.POINTER(C.c_void_p)], I),
        "mfg_destroy": ([P], I),
        "mfg_last_error": ([], C.c_char_p),
        "mfg_layout": ([P, I, C.POINTER(SZ), C.POINTER(SZ), C.POINTER(SZ), C.POINTER(SZ), C.POINTER(I)], I),
        "mfg_sizes": ([P, C.POINTER(SZ), C.POINTER(SZ), C.POINTER(SZ)], I),
        "mfg_solve": ([P, V, V, V, V, V, V, C.POINTER(MfgStats), V], I),
        "mfg_solve_host": ([P, V, V, V, V, V, V, C.POINTER(MfgStats), V], I),
        "mfg_apply_precond": ([P, I, V, V, V], I),
        "mfg_prox": ([P, I, D, V, V, V, V, V], I),
        "mfg_apply_AAt": ([P, I, V, V, V], I),
        "mfg_apply_C": ([P, I, V, V, V], I),
        "mfg_apply_Ct": ([P, I, V, V, V], I),
        "mfg_kernel_launches": ([P], C.c_longlong),
        "mfg_set_launch_mode": ([P, I], I),
        "mfg_adjoint": ([P, I, V, V, V, V, V, V, V, D, I, C.POINTER(MfgStats), V], I),
        "mfg_apply_precond_noalloc": ([C.POINTER(MfgProblem), V, V, V], I),
        "mfg_set_fault_injection": ([P, I], I),
        "mfg_prox_step": ([P, I, D, V, V, V, V, V, V], I),
        "mfg_autotune": ([P, V], I),
        "mfg_get_schedule": ([P, I, C.POINTER(MfgSchedule)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()
EXPORTED = ("mfg_plan", "mfg_destroy", "mfg_last_error", "mfg_layout", "mfg_sizes", "mfg_solve",
            "mfg_solve_host", "mfg_apply_precond", "mfg_prox", "mfg_apply_AAt", "mfg_apply_C",
            "mfg_apply_Ct", "mfg_kernel_launches", "mfg_set_launch_mode", "mfg_adjoint",
            "mfg_apply_precond_noalloc", "mfg_set_fault_injection", "mfg_prox_step", "mfg_autotune",
            "mfg_get_schedule")


# statuses a solve reports as its result rather than raising
_OUTCOMES = (MFG_OK, MFG_ERR_NOT_CONVERGED, MFG_ERR_NONFINITE, MFG_ERR_TIMEOUT)


def mfg_last_error():
    return LIB.mfg_last_error().decode()


def _check(rc):
    if rc != MFG_OK:
        raise MfgError(rc, mfg_last_error())


def problem_struct(d, precision=None):
    """mfg_problem from a problem dict (keys as in mfg_inputs).  precision (the
    argument, else d["precision"], else "fp64"): "fp64" (MFG_FP64), "mixed"
    (FP32 preconditioner, MFG_MIXED), "mixed_tc" (its time transforms on the
    tensor cores, MFG_MIXED_TC), "mixed_df" (double-float AAt, MFG_MIXED_DF),
    or the integer code.  d["cg_ref"] (default "rhs"): "rhs" (MFG_CG_REF_RHS)
    or "resid" (MFG_CG_REF_RESID), or the integer code.  d["nu_field"] (optional,
    (Nx, Ny) array): the viscosity field nu(x) in place of nu."""
    p = MfgProblem()
    p.dim = d["dim"]
    p.n[0], p.n[1] = d["n"]
    p.len[0], p.len[1] = d["len"]
    p.bc[0], p.bc[1] = [MFG_PERIODIC if b == "periodic" else MFG_NEUMANN for b in d["bc"]]
    p.nt, p.T, p.nu, p.qprime = d["nt"], d["T"], d["nu"], d.get("qprime", 2.0)
    p.f_a, p.f_b, p.g_a, p.l = d["f_a"], d["f_b"], d["g_a"], d["l"]
    p.gamma, p.tau0, p.sigma0 = d["gamma"], d["tau0"], d["sigma0"]
    p.max_cp, p.cp_tol, p.cg_rule = d["max_cp"], d["cp_tol"], d["cg_rule"]
    p.cg_tol, p.max_cg = d["cg_tol"], d["max_cg"]
    prec = d.get("precision", "fp64") if precision is None else precision
    p.precision = {"fp64": MFG_FP64, "mixed": MFG_MIXED, "mixed_df": MFG_MIXED_DF,
                   "mixed_tc": MFG_MIXED_TC}.get(prec, prec)
    ref = d.get("cg_ref", "rhs")
    p.cg_ref = {"rhs": MFG_CG_REF_RHS, "resid": MFG_CG_REF_RESID}.get(ref, ref)
    field = d.get("nu_field")
    if field is not None:
        # host copy of the node viscosities, kept alive with the struct (the
        # library reads it only inside the call that takes the struct)
        import numpy as np
        buf = np.ascontiguousarray(np.asarray(field, dtype=np.float64).reshape(-1))
        p._nu_buf = buf
        p.nu_field = buf.ctypes.data_as(C.POINTER(C.c_double))
    return p


class Plan:
    """Owns an mfg_plan_t; freed with mfg_destroy."""

    def __init__(self, handle, batch, nts=(), fields=()):
        self.handle = C.c_void_p(handle)
        self.batch = batch
        self.nts = list(nts)
        self.fields = list(fields) or [False] * batch  # instance b has a viscosity field

    def close(self):
        if self.handle:
            LIB.mfg_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mfg_plan(problems, precision=None):
    if isinstance(problems, dict):
        problems = [problems]
    structs = [problem_struct(d, precision) for d in problems]  # keeps any field buffers alive
    arr = (MfgProblem * len(structs))(*structs)
    h = C.c_void_p()
    _check(LIB.mfg_plan(arr, len(structs), C.byref(h)))
    return Plan(h.value, len(problems), [d["nt"] for d in problems],
                [d.get("nu_field") is not None for d in problems])


def mfg_destroy(plan):
    plan.close()


def mfg_layout(plan, b):
    fo, po, do, n = C.c_size_t(), C.c_size_t(), C.c_size_t(), C.c_size_t()
    c = C.c_int()
    _check(LIB.mfg_layout(plan.handle, b, C.byref(fo), C.byref(po), C.byref(do), C.byref(n), C.byref(c)))
    return {"field_off": fo.value, "primal_off": po.value, "dual_off": do.value, "n": n.value, "c": c.value}


def mfg_sizes(plan):
    f, p, d = C.c_size_t(), C.c_size_t(), C.c_size_t()
    _check(LIB.mfg_sizes(plan.handle, C.byref(f), C.byref(p), C.byref(d)))
    return {"field": f.value, "primal": p.value, "dual": d.value}


def mfg_kernel_launches(plan):
    return int(LIB.mfg_kernel_launches(plan.handle))


def _ptr(t, numel=None, device=True):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    if device and not t.is_cuda:
        raise TypeError("tensor must live on the CUDA device")
    if not device and t.is_cuda:
        raise TypeError("tensor must live in host memory")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"tensor has {t.numel()} elements, need {numel}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _stats(plan, stats):
    if stats is None:
        stats = (MfgStats * plan.batch)()
    return stats


def mfg_solve(plan, m0, V, W, y, ybar, z, stats=None, stream=None):
    """Returns (status, stats array).  Solver outcomes (NOT_CONVERGED,
    NONFINITE, TIMEOUT) are returned, other errors raise."""
    sz = mfg_sizes(plan)
    stats = _stats(plan, stats)
    rc = LIB.mfg_solve(plan.handle, _ptr(m0, sz["field"]), _ptr(V, sz["field"]), _ptr(W, sz["field"]),
                       _ptr(y, sz["primal"]), _ptr(ybar, sz["primal"]), _ptr(z, sz["dual"]), stats,
                       _stream(stream))
    if rc not in _OUTCOMES:
        _check(rc)
    return rc, stats


def mfg_solve_host(plan, m0, V, W, y, ybar, z, stats=None, stream=None):
    sz = mfg_sizes(plan)
    stats = _stats(plan, stats)
    rc = LIB.mfg_solve_host(plan.handle, _ptr(m0, sz["field"], False), _ptr(V, sz["field"], False),
                            _ptr(W, sz["field"], False), _ptr(y, sz["primal"], False),
                            _ptr(ybar, sz["primal"], False), _ptr(z, sz["dual"], False), stats,
                            _stream(stream))
    if rc not in _OUTCOMES:
        _check(rc)
    return rc, stats


def mfg_adjoint(plan, b, y, z, gy, dm0, dV, dW, dnu, tol=1e-10, max_iter=5000, stream=None):
    """Implicit-differentiation gradient at a converged solution (see mfg.h).
    dnu: 1 element, or Nx*Ny (dloss/dnu(x)) for an instance with a viscosity field."""
    lay = mfg_layout(plan, b)
    n, cn = lay["n"], lay["n"] * lay["c"]
    S = n // plan_nt(plan, b)
    st = MfgStats()
    field = plan.fields[b] if b < len(plan.fields) else False
    rc = LIB.mfg_adjoint(plan.handle, b, _ptr(y, cn), _ptr(z, n), _ptr(gy, cn), _ptr(dm0, S), _ptr(dV, S),
                         _ptr(dW, S) if dW is not None else C.c_void_p(), _ptr(dnu, S if field else 1), float(tol),
                         int(max_iter), C.byref(st), _stream(stream))
    if rc not in (MFG_OK, MFG_ERR_NOT_CONVERGED):
        _check(rc)
    return rc, st


def plan_nt(plan, b):
    return plan.nts[b]


def mfg_apply_precond(plan, b, r, z, stream=None):
    n = mfg_layout(plan, b)["n"]
    _check(LIB.mfg_apply_precond(plan.handle, b, _ptr(r, n), _ptr(z, n), _stream(stream)))


def mfg_prox(plan, b, tau, v, V, W, y, stream=None):
    lay = mfg_layout(plan, b)
    cn = lay["n"] * lay["c"]
    _check(LIB.mfg_prox(plan.handle, b, float(tau), _ptr(v, cn), _ptr(V), _ptr(W), _ptr(y, cn),
                        _stream(stream)))


def mfg_prox_step(plan, b, tau, z, y, ybar, V, W, stream=None):
    """One primal CP step in place on y, ybar (see mfg.h)."""
    lay = mfg_layout(plan, b)
    cn = lay["n"] * lay["c"]
    _check(LIB.mfg_prox_step(plan.handle, b, float(tau), _ptr(z, lay["n"]), _ptr(y, cn), _ptr(ybar, cn),
                             _ptr(V), _ptr(W), _stream(stream)))


def mfg_apply_AAt(plan, b, p, q, stream=None):
    n = mfg_layout(plan, b)["n"]
    _check(LIB.mfg_apply_AAt(plan.handle, b, _ptr(p, n), _ptr(q, n), _stream(stream)))


def mfg_apply_C(plan, b, v, r, stream=None):
    lay = mfg_layout(plan, b)
    _check(LIB.mfg_apply_C(plan.handle, b, _ptr(v, lay["n"] * lay["c"]), _ptr(r, lay["n"]), _stream(stream)))


def mfg_apply_Ct(plan, b, p, x, stream=None):
    lay = mfg_layout(plan, b)
    _check(LIB.mfg_apply_Ct(plan.handle, b, _ptr(p, lay["n"]), _ptr(x, lay["n"] * lay["c"]), _stream(stream)))


def mfg_autotune(plan, stream=None):
    """Times the candidate launch choices of every instance and keeps the
    fastest (see mfg.h); synchronises the stream."""
    _check(LIB.mfg_autotune(plan.handle, _stream(stream)))


def mfg_get_schedule(plan, b):
    """The launch schedule instance b uses, as a dict."""
    out = MfgSchedule()
    _check(LIB.mfg_get_schedule(plan.handle, b, C.byref(out)))
    return out.as_dict()


def mfg_set_fault_injection(plan, what):
    """Test hook of the failure-detection paths (see mfg.h): "none" or
    "tc_no_commit", or the integer code."""
    code = {"none": MFG_INJECT_NONE, "tc_no_commit": MFG_INJECT_TC_NO_COMMIT,
            "band_no_copy": MFG_INJECT_BAND_NO_COPY}.get(what, what)
    _check(LIB.mfg_set_fault_injection(plan.handle, code))


def mfg_set_launch_mode(plan, mode):
    _check(LIB.mfg_set_launch_mode(plan.handle, {"graph": MFG_LAUNCH_GRAPH, "eager": MFG_LAUNCH_EAGER}.get(mode, mode)))


def mfg_apply_precond_noalloc(problem, r, z, stream=None, precision=None):
    """z = P^{-1} r for one problem dict without a plan and without allocating
    device memory (static library scratch; see include/mfg.h)."""
    p = problem_struct(problem, precision)
    n = p.nt * p.n[0] * (p.n[1] if p.dim == 2 else 1)
    _check(LIB.mfg_apply_precond_noalloc(C.byref(p), _ptr(r, n), _ptr(z, n), _stream(stream)))
