"""O1: the tree-level, tadpole-improved OK operator built directly from the terms of the action
(oracle; test infrastructure).

The paper cites the OK action (Sec. 1) and gives only its rewritten W form (Eqs. minFlopForm,
shifted_W_first .. shifted_W_last). Every entry of those W formulas follows from one operator
expression, which this module expands into gauge-link paths independently of the W formulas:

  K = am0 + gamma_4 Nabla_4 - Delta_4 / 2 + zeta gamma.Nabla - r_s zeta Delta3 / 2
      - (c_B zeta / 2) i Sigma.B - (c_E zeta / 2) alpha.E
      + c1 sum_i gamma_i Nabla_i Delta_i + c2 {gamma.Nabla, Delta3} + c3 {gamma.Nabla, i Sigma.B}
      + c_EE {gamma_4 Nabla_4, alpha.E} + c4 sum_i Delta_i^2 + c5 sum_i sum_{j != i} {i Sigma_i B_i, Delta_j}

with Nabla_mu = (T_+mu - T_-mu) / 2, Delta_mu = T_+mu + T_-mu - 2, (T_+mu psi)_x = U_mu(x) psi_{x+mu},
(T_-mu psi)_x = U_mu(x-mu)^dagger psi_{x-mu}, Delta3 = sum_i Delta_i, Sigma_i = 1 (x) sigma_i,
alpha_i = gamma_4 gamma_i, E_i = F_4i, B_i = eps_ijk F_jk / 2 and F the clover field strength.

Tadpole improvement: M = u0 K evaluated with every gauge path weighted by u0^-(its length after
cancelling adjacent U U^dagger pairs). This reproduces the staple term of D^+_i, whose weight is
u0^-2 - u0^-4 (Eq. shifted_W_first .. shifted_W_last), and the constant u0 / (2 kappa) of W^0 with
1 / (2 kappa) = am0 + 1 + 3 r_s zeta + 18 c4.

The operator is kept as a list of terms (4x4 spin matrix, step word, coefficient); products
concatenate words; words are reduced, grouped, and evaluated as link products over the lattice.
The result is the set of per-site 12x12 blocks, one per lattice offset.
"""
import numpy as np

from .spin import I4, GAMMA, SIGMA, ALPHA
from .lattice import shift_vec, dag, neighbour_spinor
from .gauge import tadpole_u0

# A step is +(mu+1) (forward hop in direction mu) or -(mu+1) (backward hop).


def identity():
    return [(I4, (), 1.0)]


def hop(mu, sgn):
    """T_{+mu} (sgn = +1) or T_{-mu} (sgn = -1)."""
    return [(I4, (sgn * (mu + 1),), 1.0)]


def spin(S):
    return [(np.asarray(S, dtype=np.complex128), (), 1.0)]


def add(*ops):
    out = []
    for op in ops:
        out.extend(op)
    return out


def scale(op, c):
    return [(s, w, c * k) for (s, w, k) in op]


def mul(A, B):
    """Operator product A B (B acts first): spins multiply, words concatenate A then B."""
    return [(sa @ sb, wa + wb, ka * kb) for (sa, wa, ka) in A for (sb, wb, kb) in B]


def anticomm(A, B):
    return add(mul(A, B), mul(B, A))


def nabla(mu):
    return add(scale(hop(mu, +1), 0.5), scale(hop(mu, -1), -0.5))


def lap(mu):
    return add(hop(mu, +1), hop(mu, -1), scale(identity(), -2.0))


def clover_op(mu, nu):
    """F_{mu nu} = (Q - Q^dagger) / 8 as closed paths: the four leaves traversed mu-then-nu and
    their reverses."""
    m, n = mu + 1, nu + 1
    leaves = [(m, n, -m, -n), (n, -m, -n, m), (-m, -n, m, n), (-n, m, n, -m)]
    out = [(I4, w, 1.0 / 8.0) for w in leaves]
    out += [(I4, tuple(-s for s in reversed(w)), -1.0 / 8.0) for w in leaves]
    return out


def B_op(i):
    return clover_op((i + 1) % 3, (i + 2) % 3)


def E_op(i):
    return clover_op(3, i)


def am0_effective(c):
    """The bare mass entering K; derived from kappa when kappa > 0 (1/(2 kappa) = am0 + 1 +
    3 r_s zeta + 18 c4)."""
    if c.kappa > 0:
        return 1.0 / (2.0 * c.kappa) - 1.0 - 3.0 * c.r_s * c.zeta - 18.0 * c.c4
    return c.am0


def action_terms(c):
    """The term list of K for coefficient record c."""
    g_nabla = add(*[mul(spin(GAMMA[i]), nabla(i)) for i in range(3)])
    lap3 = add(*[lap(i) for i in range(3)])
    isb = add(*[mul(spin(1j * SIGMA[k]), B_op(k)) for k in range(3)])
    ae = add(*[mul(spin(ALPHA[k]), E_op(k)) for k in range(3)])
    g4n4 = mul(spin(GAMMA[3]), nabla(3))
    terms = add(
        scale(identity(), am0_effective(c)),
        g4n4,
        scale(lap(3), -0.5),
        scale(g_nabla, c.zeta),
        scale(lap3, -0.5 * c.r_s * c.zeta),
        scale(isb, -0.5 * c.c_B * c.zeta),
        scale(ae, -0.5 * c.c_E * c.zeta),
        scale(add(*[mul(mul(spin(GAMMA[i]), nabla(i)), lap(i)) for i in range(3)]), c.c1),
        scale(anticomm(g_nabla, lap3), c.c2),
        scale(anticomm(g_nabla, isb), c.c3),
        scale(anticomm(g4n4, ae), c.c_EE),
        scale(add(*[mul(lap(i), lap(i)) for i in range(3)]), c.c4),
        scale(add(*[anticomm(mul(spin(1j * SIGMA[i]), B_op(i)), lap(j))
                    for i in range(3) for j in range(3) if j != i]), c.c5),
    )
    return terms


def reduce_word(word):
    """Cancel adjacent opposite steps (U U^dagger = 1)."""
    st = []
    for s in word:
        if st and st[-1] == -s:
            st.pop()
        else:
            st.append(s)
    return tuple(st)


def collect(terms, u0):
    """Group terms by reduced word, with the tadpole weight u0 * u0^-len(reduced word)."""
    out = {}
    for s, w, k in terms:
        if k == 0:
            continue
        r = reduce_word(w)
        wt = k * u0 ** (1 - len(r))
        out[r] = out.get(r, 0) + wt * s
    return {w: s for w, s in out.items() if np.abs(s).max() > 0}


def path_field(U, word):
    """(P, offset): P(x) = product of links along `word` starting at x; offset = end - start."""
    shp = U.shape[:4]
    P = np.broadcast_to(np.eye(3, dtype=np.complex128), shp + (3, 3)).copy()
    pos = [0, 0, 0, 0]
    for s in word:
        mu = abs(s) - 1
        if s > 0:
            P = P @ shift_vec(U[..., mu, :, :], pos)
            pos[mu] += 1
        else:
            pos[mu] -= 1
            P = P @ dag(shift_vec(U[..., mu, :, :], pos))
    return P, tuple(pos)


def resolve_u0(U, c):
    return c.u0 if c.u0 > 0 else tadpole_u0(U)


def blocks(U, c):
    """{offset (dx, dy, dz, dt): 12x12 field} of M = u0 K[U / u0] (with reduced-path weights).

    Offsets are lattice vectors, not reduced modulo the lattice size, so aliased offsets on
    small lattices stay separate.
    """
    u0 = resolve_u0(U, c)
    grouped = collect(action_terms(c), u0)
    shp = U.shape[:4]
    out = {}
    for w, s in grouped.items():
        P, off = path_field(U, w)
        blk = np.einsum("ab,...cd->...acbd", s, P).reshape(shp + (12, 12))
        if off in out:
            out[off] = out[off] + blk
        else:
            out[off] = blk
    return out


def apply(blk, psi, bc=(1, 1, 1, 1)):
    """out_x = sum_offsets block_x psi_{x + offset} (Eq. dslash), psi [T][Z][Y][X][4][3]."""
    shp = psi.shape[:4]
    out = np.zeros(shp + (12,), dtype=np.complex128)
    for off, b in blk.items():
        nb = neighbour_spinor(psi, off, bc).reshape(shp + (12,))
        out += np.einsum("...ij,...j->...i", b, nb)
    return out.reshape(shp + (4, 3))


def dense_matrix(blk, dims, bc=(1, 1, 1, 1)):
    """The full (12 V) x (12 V) matrix M for tiny lattices (site-major, spin, colour)."""
    X, Y, Z, T = dims
    V = X * Y * Z * T
    M = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    for x in range(V):
        e = np.zeros((T, Z, Y, X, 4, 3), dtype=np.complex128)
        for k in range(12):
            e.reshape(V, 12)[x, :] = 0
            e.reshape(V, 12)[x, k] = 1
            M[:, 12 * x + k] = apply(blk, e, bc).reshape(-1)
    return M


def path_at(U, word, coords):
    """(P, offset) for the sites `coords` ((n, 4) integer array of x, y, z, t): the link product
    along `word` starting at each site."""
    T, Z, Y, X = U.shape[:4]
    sizes = np.array([X, Y, Z, T])
    n = coords.shape[0]
    P = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    pos = coords.astype(np.int64).copy()
    off = [0, 0, 0, 0]

    def link(mu):
        w = np.mod(pos, sizes)
        return U[w[:, 3], w[:, 2], w[:, 1], w[:, 0], mu]

    for s in word:
        mu = abs(s) - 1
        if s > 0:
            P = P @ link(mu)
            pos[:, mu] += 1
            off[mu] += 1
        else:
            pos[:, mu] -= 1
            off[mu] -= 1
            P = P @ dag(link(mu))
    return P, tuple(off)


def apply_at(U, c, psi, sites, bc=(1, 1, 1, 1)):
    """(M psi) at the listed site indices only, [n, 4, 3]: every gauge path of the action is
    evaluated site by site, so the cost does not grow with the lattice volume (apart from u0)."""
    T, Z, Y, X = U.shape[:4]
    sizes = np.array([X, Y, Z, T])
    sites = np.asarray(sites, dtype=np.int64)
    coords = np.stack([sites % X, (sites // X) % Y, (sites // (X * Y)) % Z, sites // (X * Y * Z)], axis=1)
    grouped = collect(action_terms(c), resolve_u0(U, c))
    out = np.zeros((len(sites), 12), dtype=np.complex128)
    for w, s in grouped.items():
        P, off = path_at(U, w, coords)
        tgt = coords + np.array(off)
        wraps = np.floor_divide(tgt, sizes)
        sign = np.ones(len(sites))
        for mu in range(4):
            if bc[mu] == -1:
                sign = sign * np.where(wraps[:, mu] % 2 == 0, 1.0, -1.0)
        t = np.mod(tgt, sizes)
        nb = psi[t[:, 3], t[:, 2], t[:, 1], t[:, 0]] * sign[:, None, None]
        out += np.einsum("ab,ncd,nbd->nac", s, P, nb).reshape(len(sites), 12)
    return out.reshape(len(sites), 4, 3)
