"""The oracle's two constructions of M agree: O1 (the action expanded into gauge-link paths) and
O2 (the paper's W formulas, Eqs. shifted_W_first .. shifted_W_last with Eqs. conjugate and
opp_diag_pre_mat), blockwise for every one of the 27 offsets of Eq. minFlopForm; and the shifted
two-step form of Eq. FinalForm gives the same M psi as Eq. minFlopForm."""
import numpy as np
import pytest

import synth
from oracle import direct, wform

EXPECTED_OFFSETS = {(0, 0, 0, 0)}
for _mu in range(4):
    for _s in (1, -1):
        _v = [0, 0, 0, 0]
        _v[_mu] = _s
        EXPECTED_OFFSETS.add(tuple(_v))
for _i in range(3):
    for _s in (2, -2):
        _v = [0, 0, 0, 0]
        _v[_i] = _s
        EXPECTED_OFFSETS.add(tuple(_v))
    for _j in range(_i + 1, 3):
        for _a in (1, -1):
            for _b in (1, -1):
                _v = [0, 0, 0, 0]
                _v[_i], _v[_j] = _a, _b
                EXPECTED_OFFSETS.add(tuple(_v))

DIMS = (5, 5, 5, 4)  # spatial extent 5 keeps offsets -2..2 distinct


@pytest.fixture(scope="module")
def rough_links():
    return synth.random_links(DIMS, 0.5, 3)


def _max_rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_offsets_are_exactly_the_27_of_minflopform(rough_links):
    c = synth.random_coeffs(11)
    b1 = direct.blocks(rough_links, c)
    assert set(b1) == EXPECTED_OFFSETS
    assert len(EXPECTED_OFFSETS) == 27
    # the paper: the full set has 432 colour blocks (27 offsets x 16 blocks of 3x3)
    assert len(b1) * 16 == 432


@pytest.mark.parametrize("cseed,u0", [(11, -1.0), (12, 0.8731), (13, 1.0)])
def test_direct_equals_wform_blockwise(rough_links, cseed, u0):
    c = synth.random_coeffs(cseed, u0=u0)
    b1 = direct.blocks(rough_links, c)
    b2 = wform.blocks(rough_links, c)
    assert set(b2) == EXPECTED_OFFSETS
    for off in EXPECTED_OFFSETS:
        assert _max_rel(b1[off], b2[off]) < 1e-13, off


def test_kappa_parametrisation(rough_links):
    c = synth.random_coeffs(14).replace(kappa=0.093, am0=123.0)  # am0 ignored when kappa > 0
    b1 = direct.blocks(rough_links, c)
    b2 = wform.blocks(rough_links, c)
    for off in EXPECTED_OFFSETS:
        assert _max_rel(b1[off], b2[off]) < 1e-13
    u0 = wform.resolve_u0(rough_links, c)
    diag = np.einsum("...ii->...i", b2[(0, 0, 0, 0)]).real.mean()
    assert abs(diag - u0 / (2 * 0.093)) < 1e-12  # B and E parts are traceless in spin


NAMES = ["zeta", "r_s", "c_B", "c_E", "c_EE", "c1", "c2", "c3", "c4", "c5"]


@pytest.mark.parametrize("name", NAMES)
def test_single_coefficient_isolation(rough_links, name):
    """Each term alone: a mismatch here points at one term of the action or one W formula."""
    base = {k: 0.0 for k in NAMES}
    base[name] = 0.7
    c = synth.OKCoeffs(u0=-1.0, am0=0.3, kappa=-1.0, **base)
    b1 = direct.blocks(rough_links, c)
    b2 = wform.blocks(rough_links, c)
    for off in set(b1) | set(b2):
        z = np.zeros((12, 12))
        assert _max_rel(b1.get(off, z), b2.get(off, z)) < 1e-13 or \
            np.abs(b1.get(off, z) - b2.get(off, z)).max() < 1e-14, (name, off)


@pytest.mark.parametrize("dims,bc", [((5, 5, 5, 4), (1, 1, 1, 1)), ((4, 4, 4, 4), (1, 1, 1, -1)),
                                     ((3, 3, 3, 4), (-1, 1, 1, -1)), ((4, 3, 5, 3), (1, -1, 1, 1))])
def test_final_form_equals_minflop_form(dims, bc):
    U = synth.random_links(dims, 0.4, 21)
    c = synth.random_coeffs(22)
    psi = synth.gaussian_source(dims, 23)
    a = wform.apply(U, c, psi, bc)
    b = wform.apply_final_form(U, c, psi, bc)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


@pytest.mark.parametrize("dims,bc", [((4, 4, 4, 8), (1, 1, 1, 1)), ((3, 3, 3, 4), (1, 1, 1, -1)),
                                     ((2, 3, 4, 3), (-1, -1, 1, 1))])
def test_direct_apply_equals_wform_apply_on_aliased_lattices(dims, bc):
    """On small lattices several offsets land on the same site (4^3: x+2i = x-2i); the applies
    still agree because each offset keeps its own boundary sign and block."""
    U = synth.random_links(dims, 0.4, 31)
    c = synth.random_coeffs(32)
    psi = synth.gaussian_source(dims, 33)
    a = direct.apply(direct.blocks(U, c), psi, bc)
    b = wform.apply(U, c, psi, bc)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


def test_conjugate_relations_hold_for_formula_built_matrices(rough_links):
    """Eq. conjugate: W^{+-}_{ji,x} = -W^{+- dagger}_{ij,x-i+j}, with W^{+-}_{ji} built from its own
    formula (Eq. shifted_W_last with i and j exchanged)."""
    c = synth.random_coeffs(41)
    p = wform.forward_parts(rough_links, c)
    from oracle.lattice import shift_vec, dag
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            v = [0, 0, 0, 0]
            v[i] -= 1
            v[j] += 1
            lhs = wform.blk(*p["W+-ij"][(j, i)])
            rhs = -dag(shift_vec(wform.blk(*p["W+-ij"][(i, j)]), v))
            assert _max_rel(lhs, rhs) < 1e-13
            # W^{++}_{ij} is symmetric in i, j
            assert _max_rel(wform.blk(*p["W++ij"][(i, j)]), wform.blk(*p["W++ij"][(j, i)])) < 1e-13


def test_distinct_colour_blocks_of_the_stored_set(rough_links):
    """Counting the nonzero 3x3 colour blocks of the stored forward matrices that are distinct up
    to a scalar factor (the mass term excluded, as in the paper's footnote): W^0 6, W^+_4 4,
    W^+_i 7 each (D^+_i has no sigma_i component, so two of its four spin blocks coincide up to a
    factor), W^{++}_ii, W^{++}_ij, W^{+-}_ij 1 each: 6 + 4 + 21 + 3 + 3 + 3 = 40. The paper quotes
    50 without giving its counting rule (Sec. 2.2)."""
    c = synth.random_coeffs(42)
    fs = wform.forward_set(rough_links, c)
    fs["W0"] = fs["W0"] - wform.resolve_u0(rough_links, c) * wform.inv_2kappa(c) * np.eye(12)
    site = (1, 2, 3, 2)
    expected = {"W0": 6, "W+x": 7, "W+y": 7, "W+z": 7, "W+t": 4}
    total = 0
    for name, W in fs.items():
        m = W[site]
        reps = []
        for a in range(4):
            for b in range(4):
                blkm = m[3 * a:3 * a + 3, 3 * b:3 * b + 3]
                if np.abs(blkm).max() < 1e-14:
                    continue
                v = blkm.reshape(-1)
                if not any(abs(abs(np.vdot(r, v)) - np.linalg.norm(r) * np.linalg.norm(v))
                           < 1e-10 * np.linalg.norm(r) * np.linalg.norm(v) for r in reps):
                    reps.append(v)
        assert len(reps) == expected.get(name, 1), name
        total += len(reps)
    assert total == 40


@pytest.mark.parametrize("dims,bc", [((4, 4, 4, 8), (1, 1, 1, 1)), ((3, 5, 4, 3), (1, -1, 1, -1))])
def test_lean_and_per_site_evaluations_agree(dims, bc):
    """The memory-lean W-form apply (6x6 blocks) and the per-site evaluation of the action give the
    same M psi as the dense-block applies; these two are what full-size parity tests use."""
    U = synth.random_links(dims, 0.4, 301)
    c = synth.random_coeffs(302)
    psi = synth.gaussian_source(dims, 303)
    ref = wform.apply(U, c, psi, bc)
    assert np.linalg.norm(wform.apply_lean(U, c, psi, bc) - ref) / np.linalg.norm(ref) < 1e-13
    sites = np.array([0, 1, 7, 31, 32, 100, int(np.prod(dims)) - 1])
    at = direct.apply_at(U, c, psi, sites, bc)
    flat = ref.reshape(-1, 4, 3)[sites]
    assert np.abs(at - flat).max() < 1e-13 * np.abs(flat).max()
