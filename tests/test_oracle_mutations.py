"""Planted mistakes in the oracle (on the CPU) must be caught by the pins: each mutation below is a
plausible slip in transcribing the W formulas, and the O1 = O2 comparison or gauge covariance
rejects it."""
import numpy as np
import pytest

import synth
from oracle import direct, wform, gauge
from oracle.lattice import dag

DIMS = (5, 5, 5, 3)


@pytest.fixture(scope="module")
def setup():
    U = synth.random_links(DIMS, 0.5, 201)
    c = synth.random_coeffs(202)
    return U, c, direct.blocks(U, c)


def _mismatch(b1, b2):
    return max(np.abs(b1[o] - b2[o]).max() for o in b1)


def test_unmutated_matches(setup):
    U, c, b1 = setup
    assert _mismatch(b1, wform.blocks(U, c)) < 1e-13


def test_flipped_staple_sign_is_caught(setup, monkeypatch):
    U, c, b1 = setup
    monkeypatch.setattr(wform, "levi_civita", lambda i, j, k: -direct_levi(i, j, k))
    assert _mismatch(b1, wform.blocks(U, c)) > 1e-6


def direct_levi(i, j, k):
    from oracle.spin import levi_civita
    return levi_civita(i, j, k)


def test_wrong_conjugate_relation_sign_is_caught(setup, monkeypatch):
    U, c, b1 = setup
    orig = wform.backward_parts

    def bad(p):
        q = orig(p)
        q["W--ij"] = {k: wform.qmap(v, lambda m: -m) for k, v in q["W--ij"].items()}
        return q
    monkeypatch.setattr(wform, "backward_parts", bad)
    assert _mismatch(b1, wform.blocks(U, c)) > 1e-6


def test_transposed_clover_is_caught(setup, monkeypatch):
    U, c, b1 = setup
    orig = wform.clover_EB

    def bad(Ul):
        E, B = orig(Ul)
        return [np.swapaxes(e, -1, -2) for e in E], B
    monkeypatch.setattr(wform, "clover_EB", bad)
    assert _mismatch(b1, wform.blocks(U, c)) > 1e-6


def test_conjugated_pauli_matrix_is_caught(setup, monkeypatch):
    U, c, b1 = setup
    from oracle import spin
    bad = [spin.PAULI[0], np.conj(spin.PAULI[1]), spin.PAULI[2]]
    monkeypatch.setattr(wform, "PAULI", bad)
    assert _mismatch(b1, wform.blocks(U, c)) > 1e-6


def test_missing_tadpole_power_is_caught(setup, monkeypatch):
    """W^0 with u0^-4 instead of u0^-3 in front of the clover terms."""
    U, c, b1 = setup
    orig = wform.forward_parts

    def bad(Ul, cc):
        p = orig(Ul, cc)
        u0 = p["u0"]
        c0 = u0 * p["inv2kappa"] * np.eye(6)
        A, B, C, D = p["W0"]
        p["W0"] = ((A - c0) / u0 + c0, B / u0, C / u0, (D - c0) / u0 + c0)
        return p
    monkeypatch.setattr(wform, "forward_parts", bad)
    assert _mismatch(b1, wform.blocks(U, c)) > 1e-6


def test_reversed_link_order_breaks_gauge_covariance():
    """A product written in the wrong order (U_j(x+i) U_i(x) instead of U_i(x) U_j(x+i)) is not a
    parallel transporter, and gauge covariance fails."""
    dims = (4, 4, 4, 3)
    U = synth.random_links(dims, 0.5, 211)
    om = synth.random_gauge_transform(dims, 212)
    psi = synth.gaussian_source(dims, 213)
    from oracle.lattice import shift

    def bad_apply(Ul):
        V = Ul[..., 0, :, :]
        W = shift(Ul[..., 1, :, :], 0) @ V            # should be V @ shift(U_y, x)
        nb = np.roll(np.roll(psi_of[0], -1, axis=3), -1, axis=2)
        return np.einsum("...ab,...sb->...sa", W, nb)

    psi_of = [psi]
    lhs_psi = gauge.gauge_transform_spinor(psi, om)
    psi_of[0] = lhs_psi
    lhs = bad_apply(gauge.gauge_transform_links(U, om))
    psi_of[0] = psi
    rhs = gauge.gauge_transform_spinor(bad_apply(U), om)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) > 1e-3
