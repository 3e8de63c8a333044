"""The tensor-core multi-right-hand-side path (OK_W_F16_TC, OK_F16_TC, OK_SOLVE_MIXED_TC) against the
oracle: the stored blocks element by element (rebuilt into the 14 dense forward matrices), the
apply for every right-hand side, and the lockstep solve, whose every system must reach a true FP64
residual below 1e-10 recomputed with the oracle's apply.

Tolerance of the FP16 tensor-core apply: every stored block entry is rounded once from FP64 and
every field entry once from FP32 (unit roundoff 2^-11 each), products accumulate in FP32, so a
product carries at most about 2 x 2^-11 relative error; summed over the 27 offsets the error of
an application, relative to its norm, stays below 4 x 2^-11 (the bound of the FP16 W copy).
A rebuilt dense matrix entry is half a sum of four rounded block entries: 4 x 2^-11 of the
largest entry of the matrix bounds it."""
import numpy as np
import pytest

import synth
from oracle import wform, direct
from tests.gpu_common import SMALL_CASES, CASE_IDS, to_dev, rel_l2, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")

TC_TOL = 4 * 2.0 ** -11


def _fields(dims, nrhs, seed):
    return np.stack([synth.gaussian_source(dims, seed + k) for k in range(nrhs)]).astype(np.complex64)


def spin_colour_sources(dims, site=0):
    V = int(np.prod(dims))
    b = torch.zeros((12, V, 12), dtype=torch.complex128, device="cuda")
    for k in range(12):
        b[k, site, k] = 1.0
    return b.reshape((12,) + synth.lattice_shape(dims) + (4, 3))


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
@pytest.mark.parametrize("keep64", [True, False])
def test_tc_copy_matches_paper_formulas(case, keep64):
    """The blocks of the tensor-core copy, rebuilt into W = T Q T / 2, against the oracle's
    transcription of Eqs. shifted_W_first .. shifted_W_last (built with and without a kept
    FP64 copy: without one the precompute builds the blocks from a temporary FP64 set)."""
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 9000 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F16_TC | (ok.W_F64 if keep64 else 0))
    ref = wform.forward_set(U, c)
    V = int(np.prod(dims))
    for kind, name in enumerate(ok.W_KINDS):
        got = ok.W_expand(W, kind, ok.F16_TC).cpu().numpy()
        exp = ref[name].reshape(V, 12, 12)
        assert rel_max(got, exp) < TC_TOL, (name, rel_max(got, exp))
    V32 = ((V + 31) // 32) * 32
    assert W.nbytes == V * 3216 + (V32 * 43 * 9 * 16 if keep64 else 0)


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
@pytest.mark.parametrize("nrhs", [1, 5, 12, 16])
def test_tc_apply_matches_oracle(case, nrhs):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 9100 + sum(dims))
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F16_TC)
    psi = _fields(dims, nrhs, 9200 + sum(dims))
    got = ok.apply_M_multi(W, to_dev(psi), prec=ok.F16_TC).cpu().numpy()
    for k in range(nrhs):
        exp = wform.apply(U, c, psi[k].astype(np.complex128), bc)
        assert rel_l2(got[k], exp) < TC_TOL and rel_max(got[k], exp) < TC_TOL, (k, rel_l2(got[k], exp), rel_max(got[k], exp))


def test_tc_apply_agrees_with_fp32_apply_and_is_deterministic():
    dims, bc = (8, 6, 4, 10), (1, 1, 1, -1)
    U = to_dev(synth.random_links(dims, 0.3, 9301))
    W = ok.precompute_W(U, synth.random_coeffs(9302), bc, ok.W_F32 | ok.W_F16_TC)
    psi = to_dev(_fields(dims, 12, 9303))
    tc = ok.apply_M_multi(W, psi, prec=ok.F16_TC)
    f32 = ok.apply_M_multi(W, psi, prec=ok.F32)
    for k in range(12):
        assert float(torch.linalg.vector_norm(tc[k] - f32[k]) / torch.linalg.vector_norm(f32[k])) < TC_TOL
    assert torch.equal(ok.apply_M_multi(W, psi, prec=ok.F16_TC), tc)
    # linearity in the right-hand sides: each row of the product depends on its own field only
    one = ok.apply_M_multi(W, psi[3:4].contiguous(), prec=ok.F16_TC)
    assert torch.equal(one[0], tc[3])


def _sample_sites(V, n, seed):
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 31, 32, V // 2, V - 33, V - 1]
    return np.unique(np.concatenate([fixed, rng.integers(0, V, n - len(fixed))]))


def test_tc_apply_full_size_20cube64_sampled():
    """The 20^3 x 64 workload with 12 right-hand sides, in the launch configuration of the solve:
    three of them against the oracle evaluated site by site at 40 sampled sites."""
    w = synth.WORKLOADS["20^3x64"]
    dims = w["dims"]
    U = synth.random_links(dims, w["eps"], w["seed"])
    c = synth.placeholder_coeffs(1.0)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F16_TC)
    V = int(np.prod(dims))
    g = torch.Generator(device="cuda")
    g.manual_seed(9401)
    psi = torch.view_as_complex(torch.randn((12, V * 12, 2), generator=g, device="cuda", dtype=torch.float32))
    got = ok.apply_M_multi(W, psi, prec=ok.F16_TC).reshape(12, V, 4, 3)
    sites = _sample_sites(V, 40, 9402)
    for k in (0, 6, 11):
        src = psi[k].to(torch.complex128).cpu().numpy().reshape(synth.lattice_shape(dims) + (4, 3))
        exp = direct.apply_at(U, c, src, sites)
        gk = got[k].cpu().numpy()[sites]
        assert rel_l2(gk, exp) < TC_TOL and rel_max(gk, exp) < TC_TOL, (k, rel_l2(gk, exp))


def test_tc_solve_outer_defect_correction():
    """The tensor-core iteration as the inner solve of an outer FP64 defect correction
    (OK_SOLVE_MIXED_TC | OK_SOLVE_DEFECT): every system to a true residual below 1e-10."""
    dims, bc = (6, 5, 4, 8), (1, 1, 1, -1)
    U = synth.random_links(dims, 0.3, 9551)
    c = synth.placeholder_coeffs(0.6)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_DF64 | ok.W_F16_TC)
    b = spin_colour_sources(dims, site=9)
    x, infos = ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED_TC | ok.SOLVE_DEFECT, delta=1e-3, check_every=4)
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    for k in range(12):
        r = np.linalg.norm(bs[k] - wform.apply(U, c, xs[k], bc)) / np.linalg.norm(bs[k])
        assert infos[k]["true_relres"] < 1e-10 and r < 1e-10 and infos[k]["reliable_updates"] >= 2, (k, infos[k], r)


@pytest.mark.parametrize("w64", ["f64", "df64"])
def test_tc_solve_spin_colour_sources_small(w64):
    dims, bc = (6, 5, 4, 8), (1, 1, 1, -1)
    U = synth.random_links(dims, 0.3, 9501)
    c = synth.placeholder_coeffs(0.6)
    W = ok.precompute_W(to_dev(U), c, bc, (ok.W_F64 if w64 == "f64" else ok.W_DF64) | ok.W_F16_TC)
    b = spin_colour_sources(dims, site=17)
    x, infos = ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED_TC, delta=1e-2, check_every=4)
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    for k in range(12):
        r = np.linalg.norm(bs[k] - wform.apply(U, c, xs[k], bc)) / np.linalg.norm(bs[k])
        assert infos[k]["true_relres"] < 1e-10 and r < 1e-10, (k, infos[k], r)
        assert abs(infos[k]["true_relres"] - r) < 1e-12
    # AUTO picks the tensor-core form for this handle; the solve is reproducible bit for bit
    x2, _ = ok.bicgstab_multi(W, b, tol=1e-10, delta=1e-2, check_every=4)
    assert torch.equal(x2, x)


def test_tc_solve_gaussian_sources_guess_and_zero_source():
    dims = (4, 4, 6, 6)
    U = synth.random_links(dims, 0.3, 9601)
    c = synth.placeholder_coeffs(0.7)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F16_TC)
    b = to_dev(np.stack([synth.gaussian_source(dims, 9602 + k) for k in range(5)]))
    b[2] = 0
    x0 = torch.zeros_like(b)
    x0[1] = b[1] * 0.3
    x, infos = ok.bicgstab_multi(W, b, x=x0.clone(), tol=1e-10, mode=ok.SOLVE_MIXED_TC, delta=1e-3)
    assert float(x[2].abs().max()) == 0.0 and infos[2]["iters"] == 0
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    for k in (0, 1, 3, 4):
        r = np.linalg.norm(bs[k] - wform.apply(U, c, xs[k], (1, 1, 1, 1))) / np.linalg.norm(bs[k])
        assert r < 1e-10, (k, r)


def test_tc_argument_errors():
    dims = (4, 4, 4, 4)
    U = to_dev(synth.random_links(dims, 0.3, 9701))
    W = ok.precompute_W(U, synth.placeholder_coeffs(0.5), (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    psi = to_dev(_fields(dims, 3, 9702))
    with pytest.raises(ok.OKError):           # no tensor-core copy
        ok.apply_M_multi(W, psi, prec=ok.F16_TC)
    b = spin_colour_sources(dims)[:3].contiguous()
    with pytest.raises(ok.OKError):
        ok.bicgstab_multi(W, b, mode=ok.SOLVE_MIXED_TC)
    W2 = ok.precompute_W(U, synth.placeholder_coeffs(0.5), (1, 1, 1, 1), ok.W_F64 | ok.W_F16_TC)
    many = to_dev(_fields(dims, 17, 9703))
    with pytest.raises(ok.OKError):           # at most 16 right-hand sides per launch
        ok.apply_M_multi(W2, many, prec=ok.F16_TC)


@pytest.mark.parametrize("am0,defect", [(0.3, False), (1.0, False), (2.5, False), (1.0, True)])
def test_tc_solve_20cube64_twelve_sources(am0, defect):
    """The 20^3 x 64 workload: the 12 spin-colour point sources in one lockstep solve on the tensor
    cores (FP16 operands, FP32 accumulation and vectors, FP64 reliable updates), graph-captured;
    every system to a true FP64 residual below 1e-10 (the GPU residual for all twelve, the
    oracle's apply for two)."""
    w = synth.WORKLOADS["20^3x64"]
    dims = w["dims"]
    U = synth.random_links(dims, w["eps"], w["seed"])
    c = synth.placeholder_coeffs(am0)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F16_TC)
    b = spin_colour_sources(dims)
    mode = ok.SOLVE_MIXED_TC | (ok.SOLVE_DEFECT if defect else 0)
    x, infos = ok.bicgstab_multi(W, b, tol=1e-10, mode=mode, delta=1e-4, check_every=8)
    for k in range(12):
        assert infos[k]["true_relres"] < 1e-10, (k, infos[k])
        assert ok.true_residual(W, b[k].contiguous(), x[k].contiguous()) < 1e-10
    bs = b.cpu().numpy()
    q = wform.quads(U, c)   # the oracle's W, evaluated once for both checks
    for k in (0, 11):
        xk = x[k].cpu().numpy()
        r = np.linalg.norm(bs[k] - wform.apply_quads(q, xk, (1, 1, 1, 1))) / np.linalg.norm(bs[k])
        assert r < 1e-10, (k, r)
