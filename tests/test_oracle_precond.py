"""Pins of the oracle's learned-preconditioner network (CPU): identity and shift special cases,
the boundary sign, gauge covariance, the adjoint against the forward map, and the loss gradient
against central finite differences."""
import numpy as np
import pytest

import synth
from oracle import precond, gauge, lattice

BC = (1, 1, 1, 1)


def _rand_weights(K, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    A = scale * (rng.standard_normal((K, 9, 4, 4)) + 1j * rng.standard_normal((K, 9, 4, 4)))
    for l in range(K):
        A[l, 0] += np.eye(4)
    return A


def test_identity_weights_give_scaled_identity():
    dims = (3, 2, 4, 3)
    U = synth.random_links(dims, 0.5, 1)
    psi = synth.gaussian_source(dims, 2)
    out = precond.apply(U, precond.identity_weights(4, 0.25), psi)
    assert np.allclose(out, 0.25 * psi, rtol=0, atol=1e-14)


@pytest.mark.parametrize("d,mu,step", [(1, 0, 1), (2, 0, -1), (3, 1, 1), (6, 2, -1), (7, 3, 1), (8, 3, -1)])
def test_single_offset_with_unit_links_is_a_shift(d, mu, step):
    dims = (3, 4, 2, 5)
    U = synth.unit_links(dims)
    psi = synth.gaussian_source(dims, 3)
    A = np.zeros((1, 9, 4, 4), dtype=np.complex128)
    A[0, d] = np.eye(4)
    out = precond.apply(U, A, psi)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}[mu]
    assert np.array_equal(out, np.roll(psi, -step, axis=axis))


def test_antiperiodic_time_boundary_flips_the_sign_of_the_wrapped_hop():
    dims = (2, 2, 2, 4)
    U = synth.unit_links(dims)
    psi = synth.gaussian_source(dims, 4)
    A = np.zeros((1, 9, 4, 4), dtype=np.complex128)
    A[0, 7] = np.eye(4)            # +t
    out = precond.apply(U, A, psi, bc=(1, 1, 1, -1))
    exp = np.roll(psi, -1, axis=0)
    exp[-1] *= -1                  # x + t crosses the boundary from the last time slice
    assert np.array_equal(out, exp)


def test_spin_matrix_acts_on_spin_only():
    dims = (2, 3, 2, 2)
    U = synth.random_links(dims, 0.4, 5)
    psi = synth.gaussian_source(dims, 6)
    A = np.zeros((1, 9, 4, 4), dtype=np.complex128)
    S = np.arange(16).reshape(4, 4) * (1 + 0.5j)
    A[0, 0] = S
    out = precond.apply(U, A, psi)
    assert np.allclose(out, np.einsum("st,...tc->...sc", S, psi), atol=1e-12)


def test_gauge_covariance():
    dims = (3, 3, 2, 4)
    U = synth.random_links(dims, 0.6, 7)
    om = synth.random_gauge_transform(dims, 8)
    psi = synth.gaussian_source(dims, 9)
    A = _rand_weights(3, 10)
    bc = (1, -1, 1, -1)
    lhs = precond.apply(gauge.gauge_transform_links(U, om), A, gauge.gauge_transform_spinor(psi, om), bc)
    rhs = gauge.gauge_transform_spinor(precond.apply(U, A, psi, bc), om)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_adjoint_matches_forward_inner_products():
    dims = (3, 2, 3, 4)
    U = synth.random_links(dims, 0.5, 11)
    A = _rand_weights(1, 12)[0]
    bc = (-1, 1, 1, -1)
    psi = synth.gaussian_source(dims, 13)
    phi = synth.gaussian_source(dims, 14)
    lhs = np.vdot(phi, precond.layer(U, A, psi, bc))
    rhs = np.vdot(precond.layer_adjoint(U, A, phi, bc), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gradient_matches_finite_differences():
    dims = (2, 3, 2, 2)
    U = synth.random_links(dims, 0.5, 15)
    b = synth.gaussian_source(dims, 16)
    x = synth.gaussian_source(dims, 17)
    A = _rand_weights(3, 18, 0.2)
    bc = (1, 1, -1, 1)
    loss, grad = precond.loss_and_grad(U, A, b, x, bc)
    rng = np.random.default_rng(19)
    h = 1e-6
    for _ in range(12):
        l, d, s, t = rng.integers(3), rng.integers(9), rng.integers(4), rng.integers(4)
        for unit, part in ((1.0, "re"), (1j, "im")):
            Ap, Am = A.copy(), A.copy()
            Ap[l, d, s, t] += h * unit
            Am[l, d, s, t] -= h * unit
            fd = (precond.loss_and_grad(U, Ap, b, x, bc)[0] - precond.loss_and_grad(U, Am, b, x, bc)[0]) / (2 * h)
            an = grad[l, d, s, t].real if part == "re" else grad[l, d, s, t].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (l, d, s, t, part, fd, an)
