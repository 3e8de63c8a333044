"""GPU parity of the precompute (A0-A2) and the apply (A3) against the oracle, through the C ABI.

Tolerances (the operator's own bar): FP64 1e-12 relative, FP32 1e-5 relative.  W matrices are
compared element by element with every one of the 14 stored forward kinds reconstructed by
ok_W_expand; applies are compared on whole fields at small sizes and on sampled sites at the
16^3 x 32 and 28^3 x 96 sizes."""
import numpy as np
import pytest

import synth
from oracle import wform, direct, gauge
from tests.gpu_common import SMALL_CASES, CASE_IDS, to_dev, rel_l2, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _library():
    ok.load()
    yield


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
def test_plaquette_and_u0(case):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 1000 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64)
    assert abs(W.plaquette - gauge.mean_plaquette(U)) < 1e-13
    u0 = c.u0 if c.u0 > 0 else gauge.tadpole_u0(U)
    assert abs(W.u0 - u0) < 1e-13


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_stored_W_matches_paper_formulas(case, prec):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 2000 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32)
    ref = wform.forward_set(U, c)
    V = int(np.prod(dims))
    tol = FP64_TOL if prec == "f64" else 2e-6
    for kind, name in enumerate(ok.W_KINDS):
        got = ok.W_expand(W, kind, ok.F64 if prec == "f64" else ok.F32).cpu().numpy()
        exp = ref[name].reshape(V, 12, 12)
        assert rel_max(got, exp) < tol, (name, rel_max(got, exp))


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
def test_apply_fp64(case):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 3000 + sum(dims))
    psi = synth.gaussian_source(dims, 3100 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64)
    got = ok.apply_M(W, to_dev(psi)).cpu().numpy()
    exp = wform.apply(U, c, psi, bc)
    assert rel_l2(got, exp) < FP64_TOL
    assert rel_max(got, exp) < 10 * FP64_TOL


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
def test_apply_fp32(case):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 4000 + sum(dims))
    psi = synth.gaussian_source(dims, 4100 + sum(dims)).astype(np.complex64)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F32)
    got = ok.apply_M(W, to_dev(psi)).cpu().numpy()
    exp = wform.apply(U, c, psi.astype(np.complex128), bc)
    assert rel_l2(got, exp) < FP32_TOL
    assert rel_max(got, exp) < FP32_TOL


@pytest.mark.parametrize("case", SMALL_CASES[:5], ids=CASE_IDS[:5])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_w16"])
def test_fused_reduction_applies(case, prec):
    """The launches a BiCGStab iteration runs (v = M p with <rhat, v>; t = M s with <t, s>, <t, t>):
    their output vectors and their fused inner products against the oracle's M psi and numpy's
    inner products of it."""
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 4200 + sum(dims))
    psi = synth.gaussian_source(dims, 4300 + sum(dims))
    y = synth.gaussian_source(dims, 4400 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32 | ok.W_F16)
    if prec == "f64":
        tol, p, dt = FP64_TOL, ok.F64, np.complex128
    else:
        tol, p, dt = (FP32_TOL, ok.F32, np.complex64) if prec == "f32" else (4 * 2.0 ** -11, ok.F32_W16, np.complex64)
        psi, y = psi.astype(dt), y.astype(dt)
    exp = wform.apply(U, c, psi.astype(np.complex128), bc)
    yd, pd = to_dev(y), to_dev(psi)
    out, (dot, _) = ok.apply_M_reduce(W, pd, yd, ok.REDUCE_DOT, prec=p)
    got = out.cpu().numpy()
    assert rel_l2(got, exp) < tol and rel_max(got, exp) < tol
    scale = np.linalg.norm(y) * np.linalg.norm(exp)
    assert abs(dot - np.vdot(y.astype(np.complex128), exp)) < tol * scale
    # <t, s> with s = psi (the unpreconditioned iteration) and, except for the FP64 kernel, a
    # separate y (the right-preconditioned iteration takes <t, s> against s while t = M (P s))
    for second in ([pd] if prec == "f64" else [pd, yd]):
        out, (ts, tt) = ok.apply_M_reduce(W, pd, second, ok.REDUCE_TS, prec=p)
        got = out.cpu().numpy()
        sv = second.cpu().numpy().astype(np.complex128)
        assert rel_l2(got, exp) < tol
        assert abs(ts - np.vdot(exp, sv)) < tol * np.linalg.norm(exp) * np.linalg.norm(sv)
        assert abs(tt - np.vdot(exp, exp).real) < 2 * tol * np.vdot(exp, exp).real


def test_links_in_fp32():
    """complex64 links: the precompute widens them to FP64; the oracle gets the same rounded links."""
    dims, bc = (5, 4, 3, 6), (1, 1, 1, -1)
    U = synth.random_links(dims, 0.4, 5001).astype(np.complex64)
    c = synth.random_coeffs(5002)
    psi = synth.gaussian_source(dims, 5003)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64)
    got = ok.apply_M(W, to_dev(psi)).cpu().numpy()
    exp = wform.apply(U.astype(np.complex128), c, psi, bc)
    assert rel_l2(got, exp) < FP64_TOL


def test_apply_is_linear_and_deterministic():
    dims = (6, 5, 4, 7)
    U = synth.random_links(dims, 0.4, 6001)
    W = ok.precompute_W(to_dev(U), synth.random_coeffs(6002), (1, 1, 1, -1), ok.W_F64 | ok.W_F32)
    a = to_dev(synth.gaussian_source(dims, 6003))
    b = to_dev(synth.gaussian_source(dims, 6004))
    Ma, Mb = ok.apply_M(W, a), ok.apply_M(W, b)
    Mab = ok.apply_M(W, a * (0.3 - 1.1j) + b)
    assert torch.allclose(Mab, Ma * (0.3 - 1.1j) + Mb, rtol=0, atol=1e-12 * float(Mab.abs().max()))
    assert torch.equal(ok.apply_M(W, a), Ma)
    a32 = a.to(torch.complex64)
    assert torch.equal(ok.apply_M(W, a32), ok.apply_M(W, a32))


def _sample_sites(V, n=64, seed=0):
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 31, 32, 127, 128, V // 2, V - 129, V - 33, V - 1]
    return np.unique(np.concatenate([fixed, rng.integers(0, V, n - len(fixed))]))


def test_full_size_16cube32_sampled():
    """The 16^3 x 32 workload in the launch configuration the benchmark uses: FP64 and FP32 applies
    against the oracle evaluated site by site at 64 sampled sites."""
    name = "16^3x32"
    dims, U, c, src = synth.workload_inputs(name)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    V = int(np.prod(dims))
    sites = _sample_sites(V)
    exp = direct.apply_at(U, c, src, sites)
    got64 = ok.apply_M(W, to_dev(src)).cpu().numpy().reshape(V, 4, 3)[sites]
    got32 = ok.apply_M(W, to_dev(src.astype(np.complex64))).cpu().numpy().reshape(V, 4, 3)[sites]
    assert rel_max(got64, exp) < 10 * FP64_TOL
    assert rel_l2(got32, exp) < FP32_TOL
    assert rel_max(got32, exp) < FP32_TOL
    assert abs(W.u0 - gauge.tadpole_u0(U)) < 1e-13
    # the handle holds 43 colour matrices per site in each precision
    assert W.nbytes == ((V + 31) // 32) * 32 * 43 * 9 * (16 + 8)


@pytest.mark.slow
def test_max_size_28cube96_sampled():
    """The largest workload (28^3 x 96, 2.1M sites): FP64 and FP32 W (19.6 GB) fit and the FP32
    apply matches the oracle at sampled sites."""
    name = "28^3x96"
    dims, U, c, src = synth.workload_inputs(name)
    V = int(np.prod(dims))
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    sites = _sample_sites(V, 48, seed=1)
    exp = direct.apply_at(U, c, src, sites)
    psi = to_dev(src)
    got64 = ok.apply_M(W, psi).cpu().numpy().reshape(V, 4, 3)[sites]
    assert rel_max(got64, exp) < 10 * FP64_TOL
    del psi
    got32 = ok.apply_M(W, to_dev(src.astype(np.complex64))).cpu().numpy().reshape(V, 4, 3)[sites]
    assert rel_l2(got32, exp) < FP32_TOL


def test_native_kernels_run():
    """The CUDA library is what runs: its own launch counter moves with every apply."""
    dims = (4, 4, 4, 4)
    W = ok.precompute_W(to_dev(synth.random_links(dims, 0.3, 7001)), synth.placeholder_coeffs(1.0))
    n0 = ok.launch_count()
    ok.apply_M(W, to_dev(synth.gaussian_source(dims, 7002)))
    torch.cuda.synchronize()
    assert ok.launch_count() == n0 + 1


def test_argument_errors():
    dims = (4, 4, 4, 4)
    U = to_dev(synth.random_links(dims, 0.3, 8001))
    W32 = ok.precompute_W(U, synth.placeholder_coeffs(1.0), precisions=ok.W_F32)
    psi64 = to_dev(synth.gaussian_source(dims, 8002))
    with pytest.raises(ok.OKError):          # handle has no FP64 copy
        ok.apply_M(W32, psi64)
    with pytest.raises(ok.OKError):          # FP64 solve needs the FP64 copy
        ok.bicgstab(W32, psi64)
    psi32 = psi64.to(torch.complex64)
    with pytest.raises(ok.OKError):          # out aliases psi
        ok.apply_M(W32, psi32, out=psi32)
    with pytest.raises(ok.OKError):          # bad kind
        ok.W_expand(W32, 14, ok.F32)
    with pytest.raises(ok.OKError):          # bad boundary phase
        ok.precompute_W(U, synth.placeholder_coeffs(1.0), bc=(1, 1, 1, 2))
    with pytest.raises(ok.OKError):          # non-finite coefficient
        ok.precompute_W(U, synth.placeholder_coeffs(1.0).replace(c3=float("nan")))
    with pytest.raises(ValueError):
        ok.apply_M(W32, psi32.reshape(-1)[:10])


# ----------------------------------------------------------------------------- double-float FP64
@pytest.mark.parametrize("case", SMALL_CASES[:5], ids=CASE_IDS[:5])
def test_double_float_copy_matches_oracle(case):
    """A handle holding only the double-float FP64 copy (OK_W_DF64): its stored W and its FP64
    applications must meet the FP64 bar (1e-12) against the oracle."""
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 5100 + sum(dims))
    psi = synth.gaussian_source(dims, 5200 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_DF64)
    ref = wform.forward_set(U, c)
    V = int(np.prod(dims))
    for kind, name in enumerate(ok.W_KINDS):
        got = ok.W_expand(W, kind, ok.F64).cpu().numpy()
        assert rel_max(got, ref[name].reshape(V, 12, 12)) < FP64_TOL, name
    got = ok.apply_M(W, to_dev(psi)).cpu().numpy()
    exp = wform.apply(U, c, psi, bc)
    assert rel_l2(got, exp) < FP64_TOL
    assert rel_max(got, exp) < 10 * FP64_TOL


def test_double_float_true_residual_equals_native():
    dims, bc = (6, 5, 4, 7), (1, 1, 1, -1)
    U = to_dev(synth.random_links(dims, 0.4, 5301))
    c = synth.random_coeffs(5302)
    Wn = ok.precompute_W(U, c, bc, ok.W_F64)
    Wd = ok.precompute_W(U, c, bc, ok.W_DF64)
    b = to_dev(synth.gaussian_source(dims, 5303))
    x = to_dev(synth.gaussian_source(dims, 5304)) * 0.2
    rn, rd = ok.true_residual(Wn, b, x), ok.true_residual(Wd, b, x)
    assert abs(rn - rd) < 1e-12 * rn


def test_handle_with_both_fp64_copies():
    """With OK_W_F64 and OK_W_DF64 on one handle, ok_apply_M in FP64 runs the native kernel and
    the true residual the double-float one (the launch classes recorded by the trace); both meet
    the FP64 bar against the oracle."""
    dims, bc = (5, 4, 6, 4), (1, 1, 1, -1)
    U = synth.random_links(dims, 0.3, 5401)
    c = synth.random_coeffs(5402)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_DF64)
    b = synth.gaussian_source(dims, 5403)
    x = 0.3 * synth.gaussian_source(dims, 5404)
    ok.trace_reset()
    ok.trace_enable(True)
    got = ok.apply_M(W, to_dev(x)).cpu().numpy()
    rel = ok.true_residual(W, to_dev(b), to_dev(x))
    ok.trace_enable(False)
    tr = ok.trace_read()
    assert tr.get("apply_f64", (0, 0))[0] == 1 and tr.get("apply_df64_resid", (0, 0))[0] == 1, tr
    Mx = wform.apply(U, c, x, bc)
    assert rel_l2(got, Mx) < FP64_TOL
    exp = np.linalg.norm(b - Mx) / np.linalg.norm(b)
    assert abs(rel - exp) < FP64_TOL * exp


def test_double_float_16cube32_sampled():
    dims, U, c, src = synth.workload_inputs("16^3x32")
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_DF64 | ok.W_F32)
    V = int(np.prod(dims))
    sites = _sample_sites(V)
    exp = direct.apply_at(U, c, src, sites)
    got = ok.apply_M(W, to_dev(src)).cpu().numpy().reshape(V, 4, 3)[sites]
    assert rel_max(got, exp) < 10 * FP64_TOL


def test_staged_copies_complete():
    """The TMA-staged split kernel (pinned with ok_set_launch_shape): FP32 and FP16-W applies against
    the oracle on lattices with ragged last tiles and with many tiles per resident block; no
    bounded wait may give up."""
    ok.wait_timeouts(reset=True)
    for dims, seed in (((7, 6, 5, 9), 1), ((16, 16, 16, 32), 2), ((3, 5, 4, 3), 3)):
        U = synth.random_links(dims, 0.3, 7100 + seed)
        c = synth.random_coeffs(7200 + seed)
        W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F32 | ok.W_F16)
        ok.set_launch_shape(W, ok.F32, staged=1)
        ok.set_launch_shape(W, ok.F32_W16, staged=1)
        psi = synth.gaussian_source(dims, 7300 + seed).astype(np.complex64)
        a = ok.apply_M(W, to_dev(psi)).cpu().numpy()
        h = ok.apply_M(W, to_dev(psi), prec=ok.F32_W16).cpu().numpy()
        V = int(np.prod(dims))
        if V <= 5000:
            exp = wform.apply(U, c, psi.astype(np.complex128), (1, 1, 1, 1))
            assert rel_l2(a, exp) < FP32_TOL
            assert rel_l2(h, exp) < 4 * 2.0 ** -11
        else:
            sites = _sample_sites(V)
            exp = direct.apply_at(U, c, psi.astype(np.complex128), sites)
            assert rel_l2(a.reshape(V, 4, 3)[sites], exp) < FP32_TOL
    assert ok.wait_timeouts() == 0


def test_staged_mixed_solve():
    dims, U, c, b = synth.workload_inputs("16^3x32")
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    ok.set_launch_shape(W, ok.F32, staged=1)
    x, info = ok.bicgstab(W, to_dev(b), tol=1e-10, mode=ok.SOLVE_MIXED, delta=1e-4)
    assert info["status"] == 0 and info["true_relres"] < 1e-10
    Mx = wform.apply_lean(U, c, x.cpu().numpy(), (1, 1, 1, 1))
    assert np.linalg.norm(b - Mx) / np.linalg.norm(b) < 1e-10


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """Failure detection without a fault: block 0 of a staged launch is made to expect 16 bytes
    that never arrive; its waits give up after about half a second, the launch ends, the timeouts
    are counted, and the next launches on the same context are correct."""
    dims = (8, 8, 8, 8)
    U = synth.random_links(dims, 0.3, 7401)
    c = synth.placeholder_coeffs(0.5)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F32)
    ok.set_launch_shape(W, ok.F32, staged=1)
    psi = to_dev(synth.gaussian_source(dims, 7402).astype(np.complex64))
    ok.wait_timeouts(reset=True)
    try:
        ok.inject_wait_timeout(16)
        ok.apply_M(W, psi)
        torch.cuda.synchronize()
    finally:
        ok.inject_wait_timeout(0)
    assert ok.wait_timeouts(reset=True) >= 1
    got = ok.apply_M(W, psi).cpu().numpy()
    exp = wform.apply(U, c, psi.cpu().numpy().astype(np.complex128), (1, 1, 1, 1))
    assert rel_l2(got, exp) < FP32_TOL
    assert ok.wait_timeouts() == 0
    with pytest.raises(ok.OKError):
        ok.inject_wait_timeout(7)
