"""Pins of the oracle to facts outside itself: closed forms, invariants, textbook special cases and
brute force on tiny lattices. Each is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign, a transposed link product, a mis-weighted tadpole factor) fails one of them."""
import numpy as np
import pytest

import synth
from oracle import direct, wform, gauge, bicgstab
from oracle.spin import GAMMA, GAMMA5, SIGMA, ALPHA, I4
from oracle.lattice import dag, shift
from tests.freefield import momenta, M_of_p, plane_wave


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------------------- gamma matrices
def test_gamma_algebra():
    """Euclidean Clifford algebra {gamma_mu, gamma_nu} = 2 delta, Hermitian gammas, gamma5^2 = 1."""
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2 * (mu == nu) * I4)
        assert np.allclose(GAMMA5 @ GAMMA[mu] + GAMMA[mu] @ GAMMA5, 0)
    assert np.allclose(GAMMA5 @ GAMMA5, I4)
    # unitarily equivalent to the Dirac-Pauli set gamma_i = [[0, -i sigma], [i sigma, 0]]
    V = np.diag([1, 1, -1j, -1j])
    for i in range(3):
        dp = np.kron(np.array([[0, -1j], [1j, 0]]), SIGMA[i][:2, :2])
        assert np.allclose(V @ dp @ V.conj().T, GAMMA[i])


# ----------------------------------------------------------------------------- free field
@pytest.mark.parametrize("dims,bc", [((4, 4, 4, 8), (1, 1, 1, 1)), ((3, 3, 3, 4), (1, 1, 1, 1)),
                                     ((4, 4, 4, 6), (1, 1, 1, -1)), ((3, 4, 5, 3), (-1, 1, -1, 1))])
@pytest.mark.parametrize("build", ["direct", "wform"])
def test_free_field_plane_waves(dims, bc, build):
    """Unit links: every plane wave exp(i p.x) chi is mapped to exp(i p.x) M(p) chi."""
    U = synth.unit_links(dims)
    c = synth.random_coeffs(5)
    blocks = direct.blocks(U, c) if build == "direct" else wform.blocks(U, c)
    am0 = direct.am0_effective(c)
    chi = synth.gaussian_source((1, 1, 1, 1), 9).reshape(12)
    rng = np.random.default_rng(0)
    ps = [momenta(L, b) for L, b in zip(dims, bc)]
    for _ in range(12):
        p = [pp[rng.integers(len(pp))] for pp in ps]
        psi = plane_wave(dims, p, chi)
        out = wform.apply_blocks(blocks, psi, bc)
        expect = plane_wave(dims, p, M_of_p(p, c, GAMMA, am0) @ chi)
        assert rel(out, expect) < 1e-13


def test_free_field_u0_is_one_and_clover_vanishes():
    U = synth.unit_links((3, 3, 3, 4))
    assert abs(gauge.tadpole_u0(U) - 1.0) < 1e-15
    E, B = gauge.clover_EB(U)
    assert max(np.abs(f).max() for f in E + B) == 0.0


# ----------------------------------------------------------------------------- u0 and clover
def test_mean_plaquette_closed_form_constant_links():
    """Constant links U_x = A, U_y = B, U_z = U_t = 1: only the xy plaquette A B A^dag B^dag differs
    from 1, so <P> = (5 + Re tr(A B A^dag B^dag) / 3) / 6."""
    A, Bm = synth.random_su3((2,), 1.3, 77)
    U = synth.unit_links((3, 4, 3, 3))
    U[..., 0, :, :] = A
    U[..., 1, :, :] = Bm
    expect = (5 + np.trace(A @ Bm @ A.conj().T @ Bm.conj().T).real / 3) / 6
    assert abs(gauge.mean_plaquette(U) - expect) < 1e-14


def test_u0_pure_gauge_and_gauge_invariance():
    dims = (4, 3, 3, 4)
    om = synth.random_gauge_transform(dims, 5)
    pure = gauge.gauge_transform_links(synth.unit_links(dims), om)
    assert abs(gauge.tadpole_u0(pure) - 1.0) < 1e-14
    U = synth.random_links(dims, 0.4, 6)
    assert abs(gauge.tadpole_u0(U) - gauge.tadpole_u0(gauge.gauge_transform_links(U, om))) < 1e-14
    assert gauge.tadpole_u0(U) < 1.0


def test_clover_constant_abelian_field():
    """U_y(x) = exp(i phi x) (others 1): every xy plaquette away from the x-boundary is exp(i phi), so
    F_xy = (Q - Q^dag)/8 = i sin(phi) and B_z = F_xy; E and B_x, B_y vanish there. This fixes the
    normalisation (1/8) and the orientation (mu then nu) of the clover."""
    X, phi = 8, 0.37
    dims = (X, 3, 3, 3)
    U = synth.unit_links(dims)
    xs = np.arange(X)
    U[..., 1, :, :] = np.exp(1j * phi * xs)[None, None, None, :, None, None] * np.eye(3)
    E, B = gauge.clover_EB(U)
    interior = slice(1, X - 1)
    assert np.allclose(B[2][..., interior, :, :], 1j * np.sin(phi) * np.eye(3), atol=1e-15)
    for f in (B[0], B[1], E[0], E[1], E[2]):
        assert np.abs(f).max() < 1e-15


# ----------------------------------------------------------------------------- invariances
@pytest.mark.parametrize("build", ["direct", "wform"])
def test_gauge_covariance(build):
    """U'_mu(x) = Om(x) U_mu(x) Om(x+mu)^dag, psi' = Om psi  =>  M[U'] psi' = Om M[U] psi
    (u0 is gauge invariant)."""
    dims = (4, 4, 3, 4)
    U = synth.random_links(dims, 0.5, 51)
    om = synth.random_gauge_transform(dims, 52)
    c = synth.random_coeffs(53)
    psi = synth.gaussian_source(dims, 54)
    bc = (1, 1, 1, -1)
    mk = (lambda u: direct.blocks(u, c)) if build == "direct" else (lambda u: wform.blocks(u, c))
    lhs = wform.apply_blocks(mk(gauge.gauge_transform_links(U, om)),
                             gauge.gauge_transform_spinor(psi, om), bc)
    rhs = gauge.gauge_transform_spinor(wform.apply_blocks(mk(U), psi, bc), om)
    assert rel(lhs, rhs) < 1e-13


def test_gamma5_hermiticity_of_direct_action():
    """<phi, g5 M g5 psi> = <M phi, psi>, from O1 (which never uses the conjugate relations)."""
    dims = (4, 3, 4, 4)
    U = synth.random_links(dims, 0.5, 61)
    c = synth.random_coeffs(62)
    blocks = direct.blocks(U, c)
    phi = synth.gaussian_source(dims, 63)
    psi = synth.gaussian_source(dims, 64)
    for bc in [(1, 1, 1, 1), (1, 1, 1, -1)]:
        g5 = lambda f: np.einsum("ab,...bc->...ac", GAMMA5, f)
        lhs = np.vdot(phi, g5(direct.apply(blocks, g5(psi), bc)))
        rhs = np.vdot(direct.apply(blocks, phi, bc), psi)
        assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_W0_is_hermitian():
    U = synth.random_links((3, 3, 3, 4), 0.6, 71)
    W0 = wform.forward_set(U, synth.random_coeffs(72))["W0"]
    assert np.abs(W0 - dag(W0)).max() < 1e-14


# ----------------------------------------------------------------------------- tadpole counting
def test_reduced_path_tadpole_weights_are_what_the_staple_term_needs():
    """The paper's staple term, weighted u0^-2 - u0^-4, appears exactly when each gauge path is
    weighted by its length after cancelling U U^dagger pairs. Weighting by the unreduced length
    disagrees with the W formulas for u0 != 1 and agrees for u0 = 1."""
    dims = (5, 5, 5, 3)
    U = synth.random_links(dims, 0.5, 81)
    for u0, should_match in [(0.83, False), (1.0, True)]:
        c = synth.random_coeffs(82, u0=u0)
        w = wform.blocks(U, c)
        terms = direct.action_terms(c)
        naive = {}
        for s, word, k in terms:
            r = direct.reduce_word(word)
            naive[r] = naive.get(r, 0) + k * u0 ** (1 - len(word)) * s
        out = {}
        for word, s in naive.items():
            if np.abs(s).max() == 0:
                continue
            P, off = direct.path_field(U, word)
            b = np.einsum("ab,...cd->...acbd", s, P).reshape(P.shape[:4] + (12, 12))
            out[off] = out.get(off, 0) + b
        err = max(np.abs(out[o] - w[o]).max() for o in w)
        assert (err < 1e-13) == should_match, (u0, err)


# ----------------------------------------------------------------------------- textbook case
def test_wilson_clover_special_case():
    """zeta = r_s = 1, c_B = c_E = c_SW, all other coefficients 0, u0 = 1: the operator is the
    Wilson-clover (Sheikholeslami-Wohlert) operator
      M psi = (m + 4) psi - 1/2 sum_mu [(1 - gamma_mu) U_mu psi(x+mu) + (1 + gamma_mu) U^dag psi(x-mu)]
              - (c_SW / 2) sum_{mu<nu} sigma_{mu nu} Fh_{mu nu} psi,
    sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], Fh = (Q - Q^dag)/(8i) the Hermitian clover field."""
    dims = (4, 3, 4, 4)
    U = synth.random_links(dims, 0.5, 91)
    m, csw = 0.21, 1.37
    c = synth.OKCoeffs(u0=1.0, am0=m, zeta=1.0, r_s=1.0, c_B=csw, c_E=csw)
    psi = synth.gaussian_source(dims, 92)
    out = (m + 4) * psi
    for mu in range(4):
        Um = U[..., mu, :, :]
        fwd = np.einsum("...ab,...sb->...sa", Um, shift(psi, mu))
        bwd = shift(np.einsum("...ba,...sb->...sa", np.conj(Um), psi), mu, -1)
        out = out - 0.5 * (np.einsum("st,...tc->...sc", I4 - GAMMA[mu], fwd)
                           + np.einsum("st,...tc->...sc", I4 + GAMMA[mu], bwd))
    for mu in range(4):
        for nu in range(mu + 1, 4):
            sig = 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])
            Q = gauge.clover_leaves(U, mu, nu)
            Fh = (Q - dag(Q)) / 8j
            out = out - 0.5 * csw * np.einsum("st,...ab,...tb->...sa", sig, Fh, psi)
    for build in (direct.blocks, wform.blocks):
        assert rel(wform.apply_blocks(build(U, c), psi), out) < 1e-13


# ----------------------------------------------------------------------------- solver
def test_bicgstab_against_dense_lu():
    """3^3 x 4 lattice (dimension 1296): BiCGStab vs a dense LU solve of the full matrix."""
    dims = (3, 3, 3, 4)
    U = synth.random_links(dims, 0.3, 101)
    c = synth.placeholder_coeffs(1.0)
    blocks = direct.blocks(U, c)
    bc = (1, 1, 1, -1)
    Md = direct.dense_matrix(blocks, dims, bc)
    b = synth.gaussian_source(dims, 102)
    x_lu = np.linalg.solve(Md, b.reshape(-1)).reshape(b.shape)
    x, info = bicgstab.solve(lambda v: wform.apply_blocks(blocks, v, bc), b, tol=1e-12)
    assert info["converged"] and info["true_relres"] < 1e-12
    assert rel(x, x_lu) < 1e-10
    assert np.linalg.norm(b.reshape(-1) - Md @ x.reshape(-1)) / np.linalg.norm(b) < 1e-12


def test_bicgstab_free_field_point_source_matches_fourier_solution():
    """x = M^-1 delta_{y,0} chi = V^-1 sum_p exp(i p.y) M(p)^-1 chi on the free field."""
    dims = (4, 4, 4, 8)
    X, Y, Z, T = dims
    c = synth.placeholder_coeffs(0.4).replace(u0=1.0)
    blocks = wform.blocks(synth.unit_links(dims), c)
    b = synth.point_source(dims, 0, 1, 2)
    chi = b.reshape(-1, 12)[0]
    x, info = bicgstab.solve(lambda v: wform.apply_blocks(blocks, v), b, tol=1e-12)
    assert info["converged"]
    expect = np.zeros_like(b)
    am0 = direct.am0_effective(c)
    for px in momenta(X, 1):
        for py in momenta(Y, 1):
            for pz in momenta(Z, 1):
                for pt in momenta(T, 1):
                    p = (px, py, pz, pt)
                    expect += plane_wave(dims, p, np.linalg.solve(M_of_p(p, c, GAMMA, am0), chi))
    expect /= X * Y * Z * T
    assert rel(x, expect) < 1e-10


def test_bicgstab_edge_cases():
    dims = (3, 3, 3, 3)
    U = synth.random_links(dims, 0.3, 111)
    blocks = wform.blocks(U, synth.placeholder_coeffs(1.0))
    A = lambda v: wform.apply_blocks(blocks, v)
    x, info = bicgstab.solve(A, np.zeros((3, 3, 3, 3, 4, 3), complex))
    assert info["converged"] and not np.any(x)
    b = synth.gaussian_source(dims, 112)
    x, info = bicgstab.solve(A, b, maxiter=2, max_restarts=0)
    assert not info["converged"] and info["iters"] == 2 and info["true_relres"] > 1e-10
    # a good initial guess is refined, not discarded
    x1, _ = bicgstab.solve(A, b, tol=1e-6)
    x2, info2 = bicgstab.solve(A, b, x0=x1, tol=1e-11)
    assert info2["converged"] and info2["true_relres"] < 1e-11
