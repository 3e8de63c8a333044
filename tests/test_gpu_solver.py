"""GPU BiCGStab (A4, A5) through the C ABI: every solve must reach a true FP64 residual
|b - M x| / |b| < 1e-10 recomputed by the ORACLE's apply, and small solves must agree with the
oracle's own solution."""
import numpy as np
import pytest

import synth
from oracle import wform, bicgstab as obicg
from tests.gpu_common import to_dev, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")

TOL = 1e-10


def oracle_relres(U, c, b, x, bc, lean=False):
    Mx = (wform.apply_lean if lean else wform.apply)(U, c, x, bc)
    return np.linalg.norm(b - Mx) / np.linalg.norm(b)


def test_point_source_4cube8_plain_fp64():
    """The 4^3 x 8 workload: point source, plain FP64 BiCGStab to 1e-10."""
    dims, U, c, b = synth.workload_inputs("4^3x8")
    bc = (1, 1, 1, 1)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64)
    x, info = ok.bicgstab(W, to_dev(b), tol=TOL, mode=ok.SOLVE_F64)
    x = x.cpu().numpy()
    assert info["status"] == 0 and info["true_relres"] < TOL
    assert oracle_relres(U, c, b, x, bc) < TOL
    xo, io = obicg.solve(lambda v: wform.apply(U, c, v, bc), b, tol=1e-12)
    assert io["converged"]
    assert rel_l2(x, xo) < 1e-8


@pytest.mark.parametrize("dims,bc,seed", [((6, 5, 4, 8), (1, 1, 1, -1), 1), ((7, 6, 5, 9), (1, -1, 1, 1), 2),
                                          ((3, 3, 3, 4), (1, 1, 1, 1), 3)])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_small_solves(dims, bc, seed, mode):
    U = synth.random_links(dims, 0.3, 9000 + seed)
    c = synth.placeholder_coeffs(0.6)
    b = synth.gaussian_source(dims, 9100 + seed)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32)
    m = ok.SOLVE_F64 if mode == "f64" else ok.SOLVE_MIXED
    x, info = ok.bicgstab(W, to_dev(b), tol=TOL, mode=m)
    x = x.cpu().numpy()
    r = oracle_relres(U, c, b, x, bc)
    assert info["status"] == 0 and r < TOL, (info, r)
    assert abs(info["true_relres"] - r) < 1e-12
    if mode == "mixed":
        assert info["reliable_updates"] >= 1


def test_16cube32_mixed_and_plain():
    """The 16^3 x 32 workload: FP32 BiCGStab with FP64 reliable updates, and plain FP64, both to
    a true residual below 1e-10 checked with the oracle's apply on the full lattice."""
    dims, U, c, b = synth.workload_inputs("16^3x32")
    bc = (1, 1, 1, 1)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_F64 | ok.W_F32)
    bd = to_dev(b)
    xm, im = ok.bicgstab(W, bd, tol=TOL, mode=ok.SOLVE_MIXED)
    xp, ip = ok.bicgstab(W, bd, tol=TOL, mode=ok.SOLVE_F64)
    assert im["status"] == 0 and ip["status"] == 0
    xm, xp = xm.cpu().numpy(), xp.cpu().numpy()
    assert oracle_relres(U, c, b, xm, bc, lean=True) < TOL
    assert rel_l2(xm, xp) < 1e-8
    assert abs(ok.true_residual(W, bd, to_dev(xp)) - ip["true_relres"]) < 1e-13


def test_initial_guess_and_zero_source():
    dims = (4, 4, 4, 6)
    U = synth.random_links(dims, 0.3, 9201)
    c = synth.placeholder_coeffs(0.7)
    b = synth.gaussian_source(dims, 9202)
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, -1), ok.W_F64 | ok.W_F32)
    bd = to_dev(b)
    x1, i1 = ok.bicgstab(W, bd, tol=1e-4, mode=ok.SOLVE_F64)
    x2, i2 = ok.bicgstab(W, bd, x=x1.clone(), tol=TOL, mode=ok.SOLVE_F64)
    x3, i3 = ok.bicgstab(W, bd, tol=TOL, mode=ok.SOLVE_F64)
    assert i2["status"] == 0 and i2["iters"] < i3["iters"]
    assert oracle_relres(U, c, b, x2.cpu().numpy(), (1, 1, 1, -1)) < TOL
    z, iz = ok.bicgstab(W, torch.zeros_like(bd), x=bd.clone(), tol=TOL)
    assert iz["status"] == 0 and float(z.abs().max()) == 0.0 and iz["iters"] == 0


def test_maxiter_reports_no_convergence():
    dims = (4, 4, 4, 6)
    U = synth.random_links(dims, 0.3, 9301)
    W = ok.precompute_W(to_dev(U), synth.placeholder_coeffs(0.2), (1, 1, 1, 1), ok.W_F64)
    b = to_dev(synth.gaussian_source(dims, 9302))
    x, info = ok.bicgstab(W, b, tol=TOL, maxiter=3, mode=ok.SOLVE_F64, check_every=1,
                          raise_on_noconv=False)
    assert info["status"] == -4 and info["iters"] == 3 and info["true_relres"] > TOL
    with pytest.raises(ok.OKError):
        ok.bicgstab(W, b, tol=TOL, maxiter=3, mode=ok.SOLVE_F64)


def test_solves_are_deterministic():
    dims = (6, 4, 4, 6)
    U = synth.random_links(dims, 0.3, 9401)
    W = ok.precompute_W(to_dev(U), synth.placeholder_coeffs(0.5), (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    b = to_dev(synth.gaussian_source(dims, 9402))
    for mode in (ok.SOLVE_F64, ok.SOLVE_MIXED):
        xa, ia = ok.bicgstab(W, b, tol=TOL, mode=mode)
        xb, ib = ok.bicgstab(W, b, tol=TOL, mode=mode)
        assert torch.equal(xa, xb) and ia["iters"] == ib["iters"]


def test_check_cadence_does_not_change_the_solve():
    """Kernels enqueued after the state halted (the rest of a block, and the iteration enqueued
    behind each state read) do nothing: the solve is bit-identical for any check_every."""
    dims = (6, 4, 4, 6)
    U = synth.random_links(dims, 0.3, 9501)
    W = ok.precompute_W(to_dev(U), synth.placeholder_coeffs(0.5), (1, 1, 1, 1), ok.W_F64 | ok.W_F32)
    b = to_dev(synth.gaussian_source(dims, 9502))
    for mode, delta in ((ok.SOLVE_F64, 1e-2), (ok.SOLVE_MIXED, 1e-2)):
        runs = [ok.bicgstab(W, b, tol=TOL, mode=mode, delta=delta, check_every=ce) for ce in (1, 3, 8)]
        x0, i0 = runs[0]
        assert i0["status"] == 0 and i0["true_relres"] < TOL
        for x, i in runs[1:]:
            assert torch.equal(x, x0)
            assert (i["iters"], i["reliable_updates"], i["restarts"]) == (i0["iters"], i0["reliable_updates"], i0["restarts"])


def test_mixed_solve_with_double_float_residuals():
    """FP32 iteration with reliable updates whose true residuals use the double-float FP64 copy."""
    dims, U, c, b = synth.workload_inputs("16^3x32")
    bc = (1, 1, 1, 1)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_DF64 | ok.W_F32)
    x, info = ok.bicgstab(W, to_dev(b), tol=TOL, mode=ok.SOLVE_MIXED, delta=1e-4)
    assert info["status"] == 0 and info["true_relres"] < TOL
    assert oracle_relres(U, c, b, x.cpu().numpy(), bc, lean=True) < TOL
    with pytest.raises(ok.OKError):   # plain FP64 iteration needs the native copy
        ok.bicgstab(W, to_dev(b), tol=TOL, mode=ok.SOLVE_F64)


@pytest.mark.parametrize("base", ["mixed", "mixed16"])
def test_16cube32_outer_defect_correction(base):
    """The 16^3 x 32 workload with the outer FP64 defect correction (OK_SOLVE_DEFECT): every
    correction restarts the low-precision BiCGStab (FP32 or FP16 W, FP32 fields) on M e = r, and
    the FP64 solution reaches a true residual below 1e-10 checked with the oracle's apply."""
    dims, U, c, b = synth.workload_inputs("16^3x32")
    bc = (1, 1, 1, 1)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_DF64 | ok.W_F32 | ok.W_F16)
    m = (ok.SOLVE_MIXED if base == "mixed" else ok.SOLVE_MIXED16) | ok.SOLVE_DEFECT
    x, info = ok.bicgstab(W, to_dev(b), tol=TOL, mode=m, delta=1e-3)
    r = oracle_relres(U, c, b, x.cpu().numpy(), bc, lean=True)
    assert info["status"] == 0 and r < TOL and info["true_relres"] < TOL, (info, r)
    assert info["reliable_updates"] >= 2
    with pytest.raises(ok.OKError):  # plain FP64 has no low-precision inner solve to correct
        ok.bicgstab(W, to_dev(b), tol=TOL, mode=ok.SOLVE_F64 | ok.SOLVE_DEFECT)
