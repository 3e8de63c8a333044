"""The allocation-free true residual (ok_true_residual_static), for callers that cannot let the
library allocate device memory (programs that keep the whole GPU's memory in their own pool, loops
that cannot take cudaMalloc's synchronisation).

It must give what the allocating entry points give: the same |b - M x| / |b| as ok_true_residual
and the same vector as b - ok_apply_M(x), on two calls in a row (the second call reuses the shared
scratch left by the first).  This file is collected last, so a failure here cannot hide other
failures in a run that stops at the first one."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("dims,bc", [((6, 5, 4, 7), (1, 1, 1, -1)), ((16, 16, 16, 8), (1, 1, 1, 1))])
def test_static_residual_matches_allocating_entry_points(dims, bc):
    lib = ok.load()
    U = synth.random_links(dims, 0.3, 4242)
    W = ok.precompute_W(_dev(U), synth.placeholder_coeffs(0.7), bc, ok.W_F64)
    b = _dev(synth.gaussian_source(dims, 4243))
    x = _dev(synth.gaussian_source(dims, 4244)) * 0.1
    ref_rel = ok.true_residual(W, b, x)
    ref_vec = b - ok.apply_M(W, x)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        r = torch.full_like(b, float("nan"))
        rel = ctypes.c_double(-1.0)
        status = lib.ok_true_residual_static(W.ptr, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(r.data_ptr()), ctypes.byref(rel), stream)
        assert status == 0
        assert abs(rel.value - ref_rel) <= 1e-12 * ref_rel
        err = float(torch.linalg.vector_norm(r - ref_vec) / torch.linalg.vector_norm(ref_vec))
        assert err < 1e-12


def test_static_residual_rejects_bad_arguments():
    lib = ok.load()
    dims = (4, 4, 4, 4)
    W = ok.precompute_W(_dev(synth.random_links(dims, 0.3, 4245)), synth.placeholder_coeffs(1.0), precisions=ok.W_F64)
    b = _dev(synth.gaussian_source(dims, 4246))
    rel = ctypes.c_double()
    # the output may not overlap an input
    assert lib.ok_true_residual_static(W.ptr, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                       ctypes.c_void_p(b.data_ptr()), ctypes.byref(rel), None) == -1
    assert lib.ok_true_residual_static(None, None, None, None, ctypes.byref(rel), None) == -1
