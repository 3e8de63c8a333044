"""Several right-hand sides at once: the multi-RHS apply against the oracle for every right-hand
side and every launch shape, and the graph-captured multi-RHS mixed-precision solve, whose every
system must reach a true FP64 residual below 1e-10 recomputed with the oracle's apply."""
import numpy as np
import pytest

import synth
from oracle import wform
from tests.gpu_common import SMALL_CASES, CASE_IDS, to_dev, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")

FP32_TOL = 1e-5
W16_TOL = 4 * 2.0 ** -11   # FP16 storage of W (see test_gpu_w16)


def _fields(dims, nrhs, seed):
    return np.stack([synth.gaussian_source(dims, seed + k) for k in range(nrhs)]).astype(np.complex64)


def spin_colour_sources(dims, site=0, device="cuda"):
    """The 12 unit sources at one site (spin s, colour c -> source 3 s + c), [12, T, Z, Y, X, 4, 3]."""
    V = int(np.prod(dims))
    b = torch.zeros((12, V, 12), dtype=torch.complex128, device=device)
    for k in range(12):
        b[k, site, k] = 1.0
    return b.reshape((12,) + synth.lattice_shape(dims) + (4, 3))


@pytest.mark.parametrize("case", SMALL_CASES[:5], ids=CASE_IDS[:5])
@pytest.mark.parametrize("nr", [1, 2, 4])
@pytest.mark.parametrize("prec", ["f32", "w16"])
def test_multi_apply_matches_oracle(case, nr, prec):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 8000 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F32 | ok.W_F16)
    p = ok.F32 if prec == "f32" else ok.F32_W16
    ok.set_launch_shape(W, p, nr=nr, blocks_x=0 if nr != 2 else 3)
    psi = _fields(dims, 4, 8100 + sum(dims))
    got = ok.apply_M_multi(W, to_dev(psi), prec=p).cpu().numpy()
    for k in range(4):
        exp = wform.apply(U, c, psi[k].astype(np.complex128), bc)
        assert rel_l2(got[k], exp) < (FP32_TOL if prec == "f32" else W16_TOL), (k, rel_l2(got[k], exp))


def test_multi_apply_equals_single_applies():
    dims, bc = (8, 6, 4, 10), (1, 1, 1, -1)
    U = to_dev(synth.random_links(dims, 0.3, 8201))
    W = ok.precompute_W(U, synth.random_coeffs(8202), bc, ok.W_F32 | ok.W_F16)
    psi = to_dev(_fields(dims, 12, 8203))
    for p in (ok.F32, ok.F32_W16):
        for nr in (1, 2, 4):
            ok.set_launch_shape(W, p, nr=nr)
            multi = ok.apply_M_multi(W, psi, prec=p)
            for k in (0, 5, 11):
                single = ok.apply_M(W, psi[k].contiguous(), prec=p)
                d = float((multi[k] - single).abs().max() / single.abs().max())
                assert d < 2e-6, (p, nr, k, d)


def test_autotune_records_a_shape_and_results_do_not_change():
    dims = (8, 8, 8, 8)
    U = to_dev(synth.random_links(dims, 0.3, 8301))
    W = ok.precompute_W(U, synth.placeholder_coeffs(0.5), (1, 1, 1, 1), ok.W_F32 | ok.W_F16)
    psi = to_dev(_fields(dims, 12, 8302))
    for p in (ok.F32, ok.F32_W16):
        ref1 = ok.apply_M(W, psi[0].contiguous(), prec=p)
        choice, us = ok.autotune(W, p, nrhs=1)
        assert choice in (0, 1) and us > 0
        assert float((ok.apply_M(W, psi[0].contiguous(), prec=p) - ref1).abs().max()) <= 1e-5 * float(ref1.abs().max())
        choice, us = ok.autotune(W, p, nrhs=12)
        assert choice in (1, 2, 4) and us > 0
        multi = ok.apply_M_multi(W, psi, prec=p)
        assert float((multi[0] - ref1).abs().max()) <= 1e-5 * float(ref1.abs().max())
    assert ok.wait_timeouts() == 0


def test_multi_argument_errors():
    dims = (4, 4, 4, 4)
    U = to_dev(synth.random_links(dims, 0.3, 8401))
    W = ok.precompute_W(U, synth.placeholder_coeffs(0.5), (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    psi = to_dev(_fields(dims, 3, 8402))
    with pytest.raises(ok.OKError):           # no FP16 copy
        ok.apply_M_multi(W, psi, prec=ok.F32_W16)
    ok.set_launch_shape(W, ok.F32, nr=4)      # 4 per thread do not divide 3: the default shape is used
    ref = ok.apply_M(W, psi[1].contiguous())
    assert float((ok.apply_M_multi(W, psi)[1] - ref).abs().max()) <= 2e-6 * float(ref.abs().max())
    with pytest.raises(ok.OKError):
        ok.set_launch_shape(W, ok.F32, nr=3)
    with pytest.raises(ValueError):
        ok.apply_M_multi(W, psi.to(torch.complex128))
    ok.set_launch_shape(W, ok.F32, nr=0)
    b = spin_colour_sources(dims)[:3].contiguous()
    with pytest.raises(ok.OKError):           # mixed16 needs the FP16 copy
        ok.bicgstab_multi(W, b, mode=ok.SOLVE_MIXED16)
    with pytest.raises(ok.OKError):           # the multi-RHS solver has no plain FP64 mode
        ok.bicgstab_multi(W, b, mode=ok.SOLVE_F64)


@pytest.mark.parametrize("w64", ["f64", "df64"])
@pytest.mark.parametrize("mode", ["mixed", "mixed16"])
def test_multi_solve_spin_colour_sources_small(mode, w64):
    """Every system to its own true residual, with the residuals on the native FP64 copy or on
    the double-float one."""
    dims, bc = (6, 5, 4, 8), (1, 1, 1, -1)
    U = synth.random_links(dims, 0.3, 8501)
    c = synth.placeholder_coeffs(0.6)
    W = ok.precompute_W(to_dev(U), c, bc, (ok.W_F64 if w64 == "f64" else ok.W_DF64) | ok.W_F32 | ok.W_F16)
    b = spin_colour_sources(dims, site=17)
    m = ok.SOLVE_MIXED if mode == "mixed" else ok.SOLVE_MIXED16
    x, infos = ok.bicgstab_multi(W, b, tol=1e-10, mode=m, delta=1e-2, check_every=4)
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    for k in range(12):
        Mx = wform.apply(U, c, xs[k], bc)
        r = np.linalg.norm(bs[k] - Mx) / np.linalg.norm(bs[k])
        assert infos[k]["true_relres"] < 1e-10 and r < 1e-10, (k, infos[k], r)
        assert abs(infos[k]["true_relres"] - r) < 1e-12
    # the same systems solved one at a time agree
    for k in (0, 7):
        xk, ik = ok.bicgstab(W, b[k].contiguous(), tol=1e-10, mode=ok.SOLVE_F64 if w64 == "f64" else ok.SOLVE_MIXED)
        assert rel_l2(xs[k], xk.cpu().numpy()) < 1e-8


def test_multi_solve_initial_guess_and_zero_source():
    dims = (4, 4, 4, 6)
    U = synth.random_links(dims, 0.3, 8601)
    c = synth.placeholder_coeffs(0.7)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    b = to_dev(np.stack([synth.gaussian_source(dims, 8602 + k) for k in range(4)]))
    b[2] = 0
    x0 = torch.zeros_like(b)
    x0[1] = b[1] * 0.3
    x, infos = ok.bicgstab_multi(W, b, x=x0.clone(), tol=1e-10, mode=ok.SOLVE_MIXED, delta=1e-2)
    assert float(x[2].abs().max()) == 0.0 and infos[2]["iters"] == 0
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    for k in (0, 1, 3):
        r = np.linalg.norm(bs[k] - wform.apply(U, c, xs[k], (1, 1, 1, 1))) / np.linalg.norm(bs[k])
        assert r < 1e-10


@pytest.mark.parametrize("am0", [0.3, 1.0, 2.5])
def test_multi_solve_20cube64_twelve_sources(am0):
    """The 20^3 x 64 workload: 12 spin-colour point sources, FP16 W and FP32 fields with FP64
    reliable updates, one graph-captured multi-RHS solve; every system to a true FP64 residual
    below 1e-10 (the GPU FP64 residual for all twelve, the oracle's apply for two of them)."""
    w = synth.WORKLOADS["20^3x64"]
    dims = w["dims"]
    U = synth.random_links(dims, w["eps"], w["seed"])
    c = synth.placeholder_coeffs(am0)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F16)
    b = spin_colour_sources(dims)
    ok.autotune(W, ok.F32_W16, nrhs=12)
    x, infos = ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-2, check_every=8)
    for k in range(12):
        assert infos[k]["true_relres"] < 1e-10, (k, infos[k])
        assert ok.true_residual(W, b[k].contiguous(), x[k].contiguous()) < 1e-10
    bs = b.cpu().numpy()
    q = wform.quads(U, c)   # the oracle's W, evaluated once for both checks
    for k in (0, 11):
        xk = x[k].cpu().numpy()
        r = np.linalg.norm(bs[k] - wform.apply_quads(q, xk, (1, 1, 1, 1))) / np.linalg.norm(bs[k])
        assert r < 1e-10, (k, r)
