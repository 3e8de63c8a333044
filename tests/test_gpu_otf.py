"""GPU parity of the on-the-fly apply (OK_F32_OTF): M psi in FP32 with every W matrix of Eqs.
shifted_W_first .. shifted_W_last rebuilt from the FP32 links and clover fields inside the apply,
against the oracle (FP32 bar 1e-5 relative), on whole fields at small sizes and at sampled sites
of the 16^3 x 32 and 28^3 x 96 workloads; and against the stored-W FP32 apply."""
import numpy as np
import pytest

import synth
from oracle import wform, direct
from tests.gpu_common import SMALL_CASES, CASE_IDS, to_dev, rel_l2, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ok = pytest.importorskip("paper_1311_5029_gb300")

FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _library():
    ok.load()
    yield


def _sample_sites(V, n=64, seed=0):
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 31, 32, 127, 128, V // 2, V - 129, V - 33, V - 1]
    return np.unique(np.concatenate([fixed, rng.integers(0, V, n - len(fixed))]))


@pytest.mark.parametrize("case", SMALL_CASES, ids=CASE_IDS)
def test_otf_apply_matches_oracle(case):
    _, dims, bc, eps, c = case
    U = synth.random_links(dims, eps, 8000 + sum(dims))
    psi = synth.gaussian_source(dims, 8100 + sum(dims)).astype(np.complex64)
    W = ok.precompute_W(to_dev(U), c, bc, ok.W_OTF)
    got = ok.apply_M(W, to_dev(psi), prec=ok.F32_OTF).cpu().numpy()
    exp = wform.apply(U, c, psi.astype(np.complex128), bc)
    assert rel_l2(got, exp) < FP32_TOL
    assert rel_max(got, exp) < FP32_TOL


def test_otf_handle_stores_no_W():
    """An OK_W_OTF handle holds only the FP32 links and clover fields (720 B per site, whole 32-site
    blocks), and the stored-W applies refuse it."""
    dims = (4, 4, 4, 8)
    W = ok.precompute_W(to_dev(synth.random_links(dims, 0.3, 8201)), synth.placeholder_coeffs(1.0), (1, 1, 1, 1),
                        ok.W_OTF)
    V = int(np.prod(dims))
    assert W.nbytes == V * (288 + 432)
    psi = to_dev(synth.gaussian_source(dims, 8202).astype(np.complex64))
    with pytest.raises(ok.OKError):
        ok.apply_M(W, psi)


def test_otf_equals_stored_fp32_16cube32():
    """At 16^3 x 32 the rebuilt-W apply and the stored-W apply agree to FP32 rounding, and both match
    the oracle at sampled sites."""
    dims, U, c, src = synth.workload_inputs("16^3x32")
    V = int(np.prod(dims))
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_F32 | ok.W_OTF)
    psi = to_dev(src.astype(np.complex64))
    a = ok.apply_M(W, psi).cpu().numpy()
    b = ok.apply_M(W, psi, prec=ok.F32_OTF).cpu().numpy()
    assert rel_l2(b, a) < FP32_TOL
    sites = _sample_sites(V)
    exp = direct.apply_at(U, c, src, sites)
    assert rel_l2(b.reshape(V, 4, 3)[sites], exp) < FP32_TOL


def test_otf_28cube96_sampled():
    """The largest workload (2.1M sites) with only the 720 B/site inputs on the device."""
    dims, U, c, src = synth.workload_inputs("28^3x96")
    V = int(np.prod(dims))
    W = ok.precompute_W(to_dev(U), c, (1, 1, 1, 1), ok.W_OTF)
    got = ok.apply_M(W, to_dev(src.astype(np.complex64)), prec=ok.F32_OTF).cpu().numpy().reshape(V, 4, 3)
    sites = _sample_sites(V, 48, seed=2)
    exp = direct.apply_at(U, c, src, sites)
    assert rel_l2(got[sites], exp) < FP32_TOL
