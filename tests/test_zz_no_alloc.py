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


# Driver API (libcuda) attributes of the device's default stream-ordered memory pool, the pool the
# library's allocating entry points draw from: bytes reserved from the device and bytes in use.
_RESERVED_MEM_CURRENT, _USED_MEM_CURRENT = 5, 7


def _memory_snapshot():
    """(free device bytes, default pool reserved bytes, default pool used bytes) of the current device."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    vals = []
    for attr in (_RESERVED_MEM_CURRENT, _USED_MEM_CURRENT):
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        vals.append(v.value)
    free, _ = torch.cuda.mem_get_info()
    return (free, vals[0], vals[1])


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
    outs = [torch.full_like(b, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    snaps = []
    for r in outs:
        rel = ctypes.c_double(-1.0)
        before = _memory_snapshot()
        status = lib.ok_true_residual_static(W.ptr, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(r.data_ptr()), ctypes.byref(rel), stream)
        snaps.append((before, _memory_snapshot()))
        assert status == 0
        assert abs(rel.value - ref_rel) <= 1e-12 * ref_rel
        err = float(torch.linalg.vector_norm(r - ref_vec) / torch.linalg.vector_norm(ref_vec))
        assert err < 1e-12
    # Nothing is allocated: neither call takes memory from the stream-ordered pool (reserved or in
    # use), and the second call leaves the device's free memory unchanged.  (The first call on a
    # device may load the library's module, which holds the fixed scratch array, so its free-memory
    # figure is not compared.)
    for before, after in snaps:
        assert after[1:] == before[1:], f"pool reserved/used bytes changed: {before[1:]} -> {after[1:]}"
    assert snaps[1][1][0] == snaps[1][0][0], f"free device memory changed: {snaps[1][0][0]} -> {snaps[1][1][0]}"


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
