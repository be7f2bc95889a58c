"""CPU checks of the C ABI: the library loads, exports every entry point that
include/mfg.h declares, and the ctypes structs match the C layout."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mfg.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(mfg_\w+)\s*\(", txt, re.M)))


def _lib():
    import paper_2507_01958_gb300 as pkg
    so = os.path.join(ROOT, "paper_2507_01958_gb300", "libmfg_gb300.so")
    if not os.path.exists(so):
        pkg.build()
    return pkg.lib()


def test_library_exports_every_declared_symbol():
    L = _lib()
    decl = _declared()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L.LIB, name), name
        assert name in L.EXPORTED, name
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mfg_\w+)", out))
    assert set(decl) <= exported


def test_struct_layout_matches_header(tmp_path):
    import ctypes
    L = _lib()
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mfg.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mfg_problem), '
                   'sizeof(mfg_stats), offsetof(mfg_problem, precision), offsetof(mfg_problem, nu), '
                   'offsetof(mfg_stats, cg_iters), offsetof(mfg_stats, sigma), '
                   'offsetof(mfg_problem, nu_field));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(L.MfgProblem), ctypes.sizeof(L.MfgStats),
                    L.MfgProblem.precision.offset, L.MfgProblem.nu.offset,
                    L.MfgStats.cg_iters.offset, L.MfgStats.sigma.offset, L.MfgProblem.nu_field.offset]


def test_plan_rejects_invalid_problems_without_gpu():
    """Validation happens on the host before any device call."""
    import mfg_inputs as mi
    L = _lib()
    base = mi.small(1)["problem"]
    for bad, code in ((dict(base, qprime=1.0), L.MFG_ERR_UNSUPPORTED), (dict(base, qprime=25.0), L.MFG_ERR_UNSUPPORTED),
                      (dict(base, nt=1), L.MFG_ERR_INVALID_ARG),
                      (dict(base, nu=-1.0), L.MFG_ERR_INVALID_ARG), (dict(base, l=3), L.MFG_ERR_INVALID_ARG),
                      (dict(base, f_a=-0.1), L.MFG_ERR_INVALID_ARG), (dict(base, nt=300), L.MFG_ERR_UNSUPPORTED)):
        with pytest.raises(L.MfgError) as e:
            L.mfg_plan(bad)
        assert e.value.code == code
        assert L.mfg_last_error()


def test_plan_rejects_invalid_viscosity_fields_without_gpu():
    """A viscosity field is read and checked on the host: negative or non-finite
    values are invalid, and the exact time solve (l = 0) does not take a field."""
    import numpy as np
    import mfg_inputs as mi
    L = _lib()
    base = mi.small(2, l=1)["problem"]
    good = np.full(base["n"], 0.1)
    neg, nan = good.copy(), good.copy()
    neg[1, 2] = -1e-3
    nan[0, 0] = np.nan
    for bad, code, text in ((dict(base, nu_field=neg), L.MFG_ERR_INVALID_ARG, "viscosity"),
                            (dict(base, nu_field=nan), L.MFG_ERR_INVALID_ARG, "viscosity"),
                            (dict(base, nu_field=good, l=0), L.MFG_ERR_UNSUPPORTED, "l = 1 or 2")):
        with pytest.raises(L.MfgError) as e:
            L.mfg_plan(bad)
        assert e.value.code == code
        assert text in L.mfg_last_error()


def test_fault_injection_codes_match_header():
    """The binding's fault-injection names map to the header's enum values."""
    L = _lib()
    txt = open(HEADER).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"(MFG_INJECT_\w+)\s*=\s*(\d+)", txt))
    assert enum == {"MFG_INJECT_NONE": 0, "MFG_INJECT_TC_NO_COMMIT": 1, "MFG_INJECT_BAND_NO_COPY": 2}
    for key, val in enum.items():
        assert getattr(L, key) == val


def test_precision_codes_match_header():
    """The binding's precision names map to the header's enum values, and an
    unknown code is rejected on the host."""
    import mfg_inputs as mi
    L = _lib()
    txt = open(HEADER).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"(MFG_(?:FP64|MIXED(?:_DF|_TC)?))\s*=\s*(\d+)", txt))
    assert enum == {"MFG_FP64": 0, "MFG_MIXED": 1, "MFG_MIXED_DF": 2, "MFG_MIXED_TC": 3}
    base = mi.small(1)["problem"]
    for name, key in (("fp64", "MFG_FP64"), ("mixed", "MFG_MIXED"), ("mixed_df", "MFG_MIXED_DF"),
                      ("mixed_tc", "MFG_MIXED_TC")):
        assert L.problem_struct(base, name).precision == enum[key] == getattr(L, key)
    with pytest.raises(L.MfgError) as e:
        L.mfg_plan(dict(base), precision=7)
    assert e.value.code == L.MFG_ERR_INVALID_ARG


def test_noalloc_rejects_viscosity_field_without_gpu():
    """The allocation-free apply has no banded factors: a viscosity field is
    refused on the host, before any device call (the pointers are never read)."""
    import ctypes
    import numpy as np
    import mfg_inputs as mi
    L = _lib()
    base = mi.small(3, l=1)["problem"]
    p = L.problem_struct(dict(base, nu_field=np.full(base["n"], 0.2)), "mixed")
    rc = L.LIB.mfg_apply_precond_noalloc(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(512), None)
    assert rc == L.MFG_ERR_UNSUPPORTED
    assert "viscosity field" in L.mfg_last_error()
