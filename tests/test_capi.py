"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every function that
include/ok.h declares, and rejects invalid arguments with OK_EINVAL before touching a device."""
import ctypes
import math

import pytest

import paper_1311_5029_gb300 as ok
from paper_1311_5029_gb300 import build as okbuild


@pytest.fixture(scope="module")
def lib():
    okbuild.build()
    return ok.load()


def test_every_declared_function_is_exported(lib):
    names = ok.header_functions()
    assert len(names) >= 14
    raw = ctypes.CDLL(okbuild.LIB)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert ok.strerror(0) == "success"
    assert ok.strerror(-1) == "invalid argument"
    assert ok.strerror(-4) == "solver did not converge"
    assert ok.strerror(12345) == "unknown status"


def test_null_arguments_are_rejected(lib):
    vp = ctypes.c_void_p
    c = ok.ok_coeffs(*([1.0] * 13))
    lat = ok.ok_lattice((ctypes.c_int * 4)(4, 4, 4, 4), (ctypes.c_int * 4)(1, 1, 1, 1))
    out = vp()
    assert lib.ok_precompute_W(None, None, 0, ctypes.byref(c), 1, None, ctypes.byref(out)) == -1
    assert lib.ok_precompute_W(ctypes.byref(lat), None, 0, None, 1, None, ctypes.byref(out)) == -1
    bad = ok.ok_coeffs(*([float("inf")] + [1.0] * 12))
    assert lib.ok_precompute_W(ctypes.byref(lat), vp(16), 0, ctypes.byref(bad), 1, None, ctypes.byref(out)) == -1
    zero = ok.ok_lattice((ctypes.c_int * 4)(4, 0, 4, 4), (ctypes.c_int * 4)(1, 1, 1, 1))
    assert lib.ok_precompute_W(ctypes.byref(zero), vp(16), 0, ctypes.byref(c), 1, None, ctypes.byref(out)) == -1
    huge = ok.ok_lattice((ctypes.c_int * 4)(1024, 1024, 1024, 4), (ctypes.c_int * 4)(1, 1, 1, 1))
    assert lib.ok_precompute_W(ctypes.byref(huge), vp(16), 0, ctypes.byref(c), 1, None, ctypes.byref(out)) == -1
    assert lib.ok_precompute_W(ctypes.byref(lat), vp(16), 0, ctypes.byref(c), 16, None, ctypes.byref(out)) == -1
    assert lib.ok_apply_M(None, 0, vp(16), vp(32), None) == -1
    prm = lib.ok_default_solve_params(1e-10, 100)
    info = ok.ok_solve_info()
    assert lib.ok_bicgstab_ex(None, vp(16), vp(32), ctypes.byref(prm), ctypes.byref(info), None) == -1
    assert lib.ok_bicgstab(None, vp(16), vp(32), 1e-10, 100, None, None) == -1
    r = ctypes.c_double()
    assert lib.ok_true_residual(None, vp(16), vp(32), ctypes.byref(r), None) == -1
    assert lib.ok_W_expand(None, 0, 0, vp(16), None) == -1
    assert lib.ok_W_info(None, None, None, None) == -1
    assert math.isnan(lib.ok_W_u0(None)) and math.isnan(lib.ok_W_plaquette(None))
    lib.ok_free_W(None)
    assert lib.ok_launch_count() == 0
    assert lib.ok_last_cuda_error() == 0


def test_default_solve_params(lib):
    p = lib.ok_default_solve_params(1e-9, 77)
    assert (p.tol, p.maxiter, p.mode, p.delta, p.max_restarts, p.check_every) == (1e-9, 77, 0, 1e-3, 5, 4)


def test_binding_rejects_host_tensors(lib):
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        ok.precompute_W(torch.zeros((2, 2, 2, 2, 4, 3, 3), dtype=torch.complex128), {})


def test_binding_constants_match_the_header():
    """The binding's precision, copy, solve-mode and reduction constants are the header's values."""
    import re
    text = open(ok.HEADER).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(OK_\w+)\s+(\d+)\b", text)}
    enum = re.search(r"typedef enum \{([^}]*)\} ok_prec;", text).group(1)
    defines.update({m.group(1): int(m.group(2)) for m in re.finditer(r"(OK_\w+)\s*=\s*(\d+)", enum)})
    pairs = {"F64": "OK_F64", "F32": "OK_F32", "F32_W16": "OK_F32_W16", "F16_TC": "OK_F16_TC", "F32_OTF": "OK_F32_OTF",
             "W_F64": "OK_W_F64", "W_F32": "OK_W_F32", "W_DF64": "OK_W_DF64", "W_F16": "OK_W_F16",
             "W_LINKS": "OK_W_LINKS", "W_F16_TC": "OK_W_F16_TC", "W_OTF": "OK_W_OTF",
             "SOLVE_AUTO": "OK_SOLVE_AUTO", "SOLVE_F64": "OK_SOLVE_F64", "SOLVE_MIXED": "OK_SOLVE_MIXED",
             "SOLVE_MIXED16": "OK_SOLVE_MIXED16", "SOLVE_MIXED_TC": "OK_SOLVE_MIXED_TC", "SOLVE_DEFECT": "OK_SOLVE_DEFECT",
             "REDUCE_DOT": "OK_REDUCE_DOT", "REDUCE_TS": "OK_REDUCE_TS"}
    for py, c in pairs.items():
        assert c in defines, c
        assert getattr(ok, py) == defines[c], (py, getattr(ok, py), defines[c])
    # the copy flags are distinct bits; the defect flag is a bit above every solve mode
    flags = [defines[c] for c in pairs.values() if c.startswith("OK_W_")]
    assert all(f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)
    modes = [defines[c] for c in ("OK_SOLVE_AUTO", "OK_SOLVE_F64", "OK_SOLVE_MIXED", "OK_SOLVE_MIXED16", "OK_SOLVE_MIXED_TC")]
    assert all(m & defines["OK_SOLVE_DEFECT"] == 0 for m in modes)
