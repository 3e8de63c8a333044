"""Half-precision W copy (OK_W_F16) for the low-precision iteration of the solver.

Tolerances follow from the storage format: every stored colour-matrix element is rounded once to
FP16 (relative error <= 2^-11 for normal numbers), the spin structure combines at most two stored
elements per dense 12x12 entry, so a reconstructed entry is within 2 * 2^-11 of the largest entry;
an application sums 27 such products with FP32 accumulation, and with the on-site term dominating
|M psi| the relative L2 error stays below a few units of 2^-11 (bound used: 4 * 2^-11).  A solve
whose FP32 iteration reads the FP16 copy must still reach a true FP64 residual below 1e-10 checked
with the oracle's apply, because every reliable update recomputes the residual in FP64."""
import numpy as np
import pytest

import synth
from oracle import wform, direct
from tests.gpu_common import SMALL_CASES, CASE_IDS, to_dev, rel_l2, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")

U16 = 2.0 ** -11
EXPAND_TOL = 2 * U16
APPLY_TOL = 4 * U16


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
def test_w16_copy_and_apply(case):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 6000 + sum(dims))
    psi = synth.gaussian_source(dims, 6100 + sum(dims)).astype(np.complex64)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F16)
    ref = wform.forward_set(U, c)
    V = int(np.prod(dims))
    for kind, name in enumerate(ok.W_KINDS):
        got = ok.W_expand(W, kind, ok.F32_W16).cpu().numpy()
        err = rel_max(got, ref[name].reshape(V, 12, 12))
        assert err < EXPAND_TOL, (name, err)
    got = ok.apply_M(W, to_dev(psi), prec=ok.F32_W16).cpu().numpy()
    exp = wform.apply(U, c, psi.astype(np.complex128), bc)
    assert rel_l2(got, exp) < APPLY_TOL


def test_w16_apply_is_not_the_fp32_apply():
    """The FP16 path must really read the FP16 copy: its result differs from the FP32 apply by
    about the FP16 rounding, not by zero, and agrees with it within the FP16 bound."""
    dims, bc = (6, 5, 4, 8), (1, 1, 1, -1)
    U = synth.random_links(dims, 0.4, 6201)
    W = ok.precompute_W(to_dev(U), synth.random_coeffs(6202), bc, ok.W_F32 | ok.W_F16)
    psi = to_dev(synth.gaussian_source(dims, 6203).astype(np.complex64))
    a = ok.apply_M(W, psi).cpu().numpy()
    h = ok.apply_M(W, psi, prec=ok.F32_W16).cpu().numpy()
    d = rel_l2(h, a)
    assert 1e-6 < d < APPLY_TOL, d
    h2 = ok.apply_M(W, psi, prec=ok.F32_W16).cpu().numpy()
    assert np.array_equal(h, h2)


def test_w16_16cube32_sampled():
    dims, U, c, src = synth.workload_inputs("16^3x32")
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F16)
    V = int(np.prod(dims))
    rng = np.random.default_rng(6301)
    sites = np.sort(rng.choice(V, 96, replace=False))
    exp = direct.apply_at(U, c, src, sites)
    got = ok.apply_M(W, to_dev(src.astype(np.complex64)), prec=ok.F32_W16).cpu().numpy().reshape(V, 4, 3)[sites]
    assert rel_l2(got, exp) < APPLY_TOL


@pytest.mark.parametrize("w64", ["f64", "df64"])
def test_mixed16_solve_reaches_fp64_tolerance(w64):
    dims, U, c, b = synth.workload_inputs("16^3x32")
    bc = (1, 1, 1, 1)
    W = ok.precompute_W(to_dev(U), c, bc, (ok.W_F64 if w64 == "f64" else ok.W_DF64) | ok.W_F16)
    x, info = ok.bicgstab(W, to_dev(b), tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-2)
    assert info["status"] == 0 and info["true_relres"] < 1e-10, info
    Mx = wform.apply_lean(U, c, x.cpu().numpy(), bc)
    assert np.linalg.norm(b - Mx) / np.linalg.norm(b) < 1e-10


@pytest.mark.parametrize("dims,bc,seed", [((7, 6, 5, 9), (1, -1, 1, 1), 1), ((3, 3, 3, 4), (1, 1, 1, -1), 2)])
def test_mixed16_small_solves(dims, bc, seed):
    U = synth.random_links(dims, 0.3, 6400 + seed)
    c = synth.placeholder_coeffs(0.6)
    b = synth.gaussian_source(dims, 6500 + seed)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F16)
    x, info = ok.bicgstab(W, to_dev(b), tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-2)
    Mx = wform.apply(U, c, x.cpu().numpy(), bc)
    r = np.linalg.norm(b - Mx) / np.linalg.norm(b)
    assert info["status"] == 0 and r < 1e-10, (info, r)
    assert info["reliable_updates"] >= 1


def test_w16_argument_errors():
    dims = (4, 4, 4, 4)
    U = to_dev(synth.random_links(dims, 0.3, 6601))
    c = synth.placeholder_coeffs(0.5)
    W32 = ok.precompute_W(U, c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    psi = to_dev(synth.gaussian_source(dims, 6602).astype(np.complex64))
    with pytest.raises(ok.OKError):       # no FP16 copy in the handle
        ok.apply_M(W32, psi, prec=ok.F32_W16)
    with pytest.raises(ok.OKError):
        ok.bicgstab(W32, to_dev(synth.gaussian_source(dims, 6603)), mode=ok.SOLVE_MIXED16)
    with pytest.raises(ok.OKError):
        ok.W_expand(W32, 0, ok.F32_W16)
    W16 = ok.precompute_W(U, c, (1, 1, 1, 1), ok.W_F16)
    with pytest.raises(ok.OKError):       # the FP64 residuals need an FP64 copy
        ok.bicgstab(W16, to_dev(synth.gaussian_source(dims, 6604)), mode=ok.SOLVE_MIXED16)
    with pytest.raises(ValueError):
        ok.apply_M(W16, psi.to(torch.complex128), prec=ok.F32_W16)
