"""O2: the precalculation matrices W and the operator in W form (oracle; test infrastructure).

Transcribes Sec. 2.2 of the paper:
* forward matrices W^0_x, W^+_{mu,x}, W^{++}_{ii,x}, W^{++}_{ij,x}, W^{+-}_{ij,x} from
  Eqs. shifted_W_first .. shifted_W_last, in the gamma representation of `spin.py`;
* backward matrices W^-_{mu,x}, W^{--}_{ii,x} from Eq. opp_diag_pre_mat and W^{--}_{ij,x},
  W^{+-}_{ji,x} from Eq. conjugate;
* M psi as the 27-term sum of Eq. minFlopForm, and again in the shifted two-step form of
  Eq. FinalForm (translation operators acting on the whole product, t_{-mu}[W psi]_x = [W psi]_{x-mu}).

Each W is a 12x12 spin-colour matrix per site, made of 2x2 blocks of 6x6 matrices
(2 spins x 3 colours); a colour matrix C inside a block means 1_2 (x) C.
"""
import numpy as np

from .spin import I2, PAULI
from .lattice import shift, shift_vec, dag, neighbour_spinor
from .gauge import link, clover_EB, tadpole_u0
from .spin import levi_civita


def inv_2kappa(c):
    """1 / (2 kappa): given by kappa, or am0 + 1 + 3 r_s zeta + 18 c4 (the diagonal of the
    Wilson-type terms of the action)."""
    if c.kappa > 0:
        return 1.0 / (2.0 * c.kappa)
    return c.am0 + 1.0 + 3.0 * c.r_s * c.zeta + 18.0 * c.c4


def resolve_u0(U, c):
    return c.u0 if c.u0 > 0 else tadpole_u0(U)


def sc(s2, col):
    """(2x2 spin) (x) (3x3 colour field) -> 6x6 field."""
    return np.einsum("ab,...cd->...acbd", s2, col).reshape(col.shape[:-2] + (6, 6))


def one2(col):
    return sc(I2, col)


def blk(A, B, C, D):
    """12x12 field [[A, B], [C, D]] from 6x6 fields (None = 0)."""
    ref = next(m for m in (A, B, C, D) if m is not None)
    z = np.zeros_like(ref)
    A, B, C, D = [z if m is None else m for m in (A, B, C, D)]
    top = np.concatenate([A, B], axis=-1)
    bot = np.concatenate([C, D], axis=-1)
    return np.concatenate([top, bot], axis=-2)


def forward_parts(U, c):
    """The forward matrices (Eqs. shifted_W_first .. shifted_W_last), each kept as its quad of 6x6
    blocks (A, B, C, D) = [[A, B], [C, D]] (None = 0)."""
    u0 = resolve_u0(U, c)
    E, B = clover_EB(U)
    Ul = [link(U, mu) for mu in range(4)]
    ES = sum(sc(PAULI[i], E[i]) for i in range(3))              # E-bar^S = sum_i sigma_i E_i
    BD = 1j * sum(sc(PAULI[i], B[i]) for i in range(3))         # B-bar^D = i sum_i sigma_i B_i
    p = {"u0": u0, "inv2kappa": inv_2kappa(c), "E": E, "B": B}

    # W^0 = u0/(2 kappa) + [[D0, S0], [-S0, D0]]
    D0 = -(c.c_B * c.zeta + 16.0 * c.c5) / (2.0 * u0 ** 3) * BD
    S0 = -(c.c_E * c.zeta) / (2.0 * u0 ** 3) * ES
    D0c = D0 + u0 * p["inv2kappa"] * np.eye(6)
    p["W0"] = (D0c, S0, -S0, D0c)

    # W^+_4 = [[0, S4], [S4, -U4]], S4 = c_EE/(2 u0^4) (U4 ES(x+4) - ES(x) U4)
    U4 = one2(Ul[3])
    S4 = c.c_EE / (2.0 * u0 ** 4) * (U4 @ shift(ES, 3) - ES @ U4)
    p["S+4"] = S4
    p["U4"] = U4
    Wp = [None] * 4
    Wp[3] = (None, S4, S4, -U4)

    # W^+_i = [[D+, S+], [S+, D+]]
    Dp, Sp = [None] * 3, [None] * 3
    for i in range(3):
        Ui = one2(Ul[i])
        si = sc(PAULI[i], np.broadcast_to(np.eye(3), Ul[i].shape))
        S = 0.5 * (c.zeta - 2.0 * c.c1 - 12.0 * c.c2) * sc(PAULI[i], Ul[i])
        S = S + c.c3 / (2.0 * u0 ** 4) * (Ui @ si @ shift(BD, i) - si @ BD @ Ui
                                          + 2j * one2(B[i] @ Ul[i]))
        D = -0.5 * (c.r_s * c.zeta + 8.0 * c.c4) * Ui
        staple = 0
        for j in range(3):
            for k in range(3):
                e = levi_civita(i, j, k)
                if e == 0:
                    continue
                Uk, Uik = Ul[k], Ul[i]
                up = Uk @ shift(Uik, k) @ dag(shift(Uk, i))
                dn = dag(shift(Uk, k, -1)) @ shift(Uik, k, -1) @ shift_vec(Uk, _vec({k: -1, i: 1}))
                staple = staple + e * sc(PAULI[j], up - dn)
        D = D + 1j * (c.c5 / 4.0) * (u0 ** -2 - u0 ** -4) * staple
        D = D + c.c5 / u0 ** 4 * (Ui @ shift(BD, i) + BD @ Ui
                                  - 1j * sc(PAULI[i], Ul[i] @ shift(B[i], i) + B[i] @ Ul[i]))
        Dp[i], Sp[i] = D, S
        Wp[i] = (D, S, S, D)
    p["D+"], p["S+"], p["W+"] = Dp, Sp, Wp

    # W^{++}_ii = [[D++, S++], [S++, D++]]
    Dpp, Spp, Wpp = [None] * 3, [None] * 3, [None] * 3
    for i in range(3):
        UU = Ul[i] @ shift(Ul[i], i)
        Dpp[i] = c.c4 / u0 * one2(UU)
        Spp[i] = (c.c1 + 2.0 * c.c2) / (2.0 * u0) * sc(PAULI[i], UU)
        Wpp[i] = (Dpp[i], Spp[i], Spp[i], Dpp[i])
    p["D++"], p["S++"], p["W++ii"] = Dpp, Spp, Wpp

    # W^{++}_ij, W^{+-}_ij (i != j) = [[0, S], [S, 0]]
    Wppij, Wpmij = {}, {}
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            Ui, Uj = Ul[i], Ul[j]
            Spp_ij = c.c2 / (2.0 * u0) * sc(PAULI[i] + PAULI[j],
                                            Ui @ shift(Uj, i) + Uj @ shift(Ui, j))
            Spm_ij = c.c2 / (2.0 * u0) * sc(PAULI[i] - PAULI[j],
                                            Ui @ dag(shift_vec(Uj, _vec({j: -1, i: 1})))
                                            + dag(shift(Uj, j, -1)) @ shift(Ui, j, -1))
            Wppij[(i, j)] = (None, Spp_ij, Spp_ij, None)
            Wpmij[(i, j)] = (None, Spm_ij, Spm_ij, None)
    p["W++ij"], p["W+-ij"] = Wppij, Wpmij
    return p


def _vec(d):
    v = [0, 0, 0, 0]
    for k, n in d.items():
        v[k] += n
    return v


def qdag(q):
    """Hermitian conjugate (spin and colour) of a quad: [[A, B], [C, D]]^dag = [[A^d, C^d], [B^d, D^d]]."""
    A, B, C, D = q
    d = lambda m: None if m is None else dag(m)
    return (d(A), d(C), d(B), d(D))


def qmap(q, f):
    return tuple(None if m is None else f(m) for m in q)


def backward_parts(p):
    """W^-_mu, W^{--}_ii (Eq. opp_diag_pre_mat) and W^{--}_ij, W^{+-}_ji (Eq. conjugate), as quads."""
    q = {}
    Wm = [None] * 4
    U4m = shift(p["U4"], 3, -1)
    S4m = shift(p["S+4"], 3, -1)
    Wm[3] = (-dag(U4m), -dag(S4m), -dag(S4m), None)
    for i in range(3):
        Dm = dag(shift(p["D+"][i], i, -1))
        Sm = dag(shift(p["S+"][i], i, -1))
        Wm[i] = (Dm, -Sm, -Sm, Dm)
    q["W-"] = Wm
    Wmm = [None] * 3
    for i in range(3):
        Dm = dag(shift(p["D++"][i], i, -2))
        Sm = dag(shift(p["S++"][i], i, -2))
        Wmm[i] = (Dm, -Sm, -Sm, Dm)
    q["W--ii"] = Wmm
    Wmmij, Wmpji = {}, {}
    for i in range(3):
        for j in range(i + 1, 3):
            # W^{--}_{ij,x} = -W^{++ dagger}_{ij, x-i-j}
            Wmmij[(i, j)] = qmap(qdag(p["W++ij"][(i, j)]), lambda m: -shift_vec(m, _vec({i: -1, j: -1})))
            # W^{+-}_{ji,x} = -W^{+- dagger}_{ij, x-i+j}
            Wmpji[(j, i)] = qmap(qdag(p["W+-ij"][(i, j)]), lambda m: -shift_vec(m, _vec({i: -1, j: 1})))
    q["W--ij"], q["W+-ji"] = Wmmij, Wmpji
    return q


def quads(U, c):
    """{offset: quad} for the 27 offsets of Eq. minFlopForm."""
    p = forward_parts(U, c)
    q = backward_parts(p)
    out = {(0, 0, 0, 0): p["W0"]}
    for mu in range(4):
        out[tuple(_vec({mu: 1}))] = p["W+"][mu]
        out[tuple(_vec({mu: -1}))] = q["W-"][mu]
    for i in range(3):
        out[tuple(_vec({i: 2}))] = p["W++ii"][i]
        out[tuple(_vec({i: -2}))] = q["W--ii"][i]
    for i in range(3):
        for j in range(i + 1, 3):
            out[tuple(_vec({i: 1, j: 1}))] = p["W++ij"][(i, j)]
            out[tuple(_vec({i: -1, j: -1}))] = q["W--ij"][(i, j)]
            out[tuple(_vec({i: 1, j: -1}))] = p["W+-ij"][(i, j)]
            out[tuple(_vec({i: -1, j: 1}))] = q["W+-ji"][(j, i)]
    return out


def blocks(U, c):
    """{offset: 12x12 field} of Eq. minFlopForm (27 offsets)."""
    return {off: blk(*q) for off, q in quads(U, c).items()}


def forward_set(U, c):
    """The 14 forward matrices per site, keyed by name, each a 12x12 field:
    'W0', 'W+x', 'W+y', 'W+z', 'W+t', 'W++xx', 'W++yy', 'W++zz', 'W++xy', 'W++xz', 'W++yz',
    'W+-xy', 'W+-xz', 'W+-yz' (the last three multiply psi_{x+i-j})."""
    p = forward_parts(U, c)
    n = "xyzt"
    out = {"W0": blk(*p["W0"])}
    for mu in range(4):
        out["W+" + n[mu]] = blk(*p["W+"][mu])
    for i in range(3):
        out["W++" + n[i] * 2] = blk(*p["W++ii"][i])
    for i in range(3):
        for j in range(i + 1, 3):
            out["W++" + n[i] + n[j]] = blk(*p["W++ij"][(i, j)])
    for i in range(3):
        for j in range(i + 1, 3):
            out["W+-" + n[i] + n[j]] = blk(*p["W+-ij"][(i, j)])
    return out


def _qmv(q, v):
    """[[A, B], [C, D]] applied to the spinor field v [..., 4, 3] without forming 12x12 matrices."""
    shp = v.shape[:4]
    up = v[..., 0:2, :].reshape(shp + (6,))
    lo = v[..., 2:4, :].reshape(shp + (6,))
    A, B, C, D = q
    mv = lambda M, x: np.einsum("...ij,...j->...i", M, x)
    ou = np.zeros(shp + (6,), dtype=np.complex128)
    ol = np.zeros(shp + (6,), dtype=np.complex128)
    if A is not None:
        ou += mv(A, up)
    if B is not None:
        ou += mv(B, lo)
    if C is not None:
        ol += mv(C, up)
    if D is not None:
        ol += mv(D, lo)
    return np.concatenate([ou.reshape(shp + (2, 3)), ol.reshape(shp + (2, 3))], axis=-2)


def apply_quads(quads_, psi, bc=(1, 1, 1, 1)):
    """M psi by Eq. minFlopForm from the 27 precomputed quads (`quads(U, c)`), multiplying the 6x6
    blocks directly (no 12x12 matrices)."""
    out = np.zeros_like(psi, dtype=np.complex128)
    for off, q in quads_.items():
        out += _qmv(q, neighbour_spinor(psi, off, bc))
    return out


def apply_lean(U, c, psi, bc=(1, 1, 1, 1)):
    """M psi by Eq. minFlopForm, multiplying the 6x6 blocks directly (no 12x12 matrices), for
    lattices where the dense blocks would not fit in memory."""
    return apply_quads(quads(U, c), psi, bc)


def _mv(W, v):
    shp = v.shape[:4]
    return np.einsum("...ij,...j->...i", W, v.reshape(shp + (12,))).reshape(shp + (4, 3))


def apply_blocks(blocks_, psi, bc=(1, 1, 1, 1)):
    out = np.zeros_like(psi, dtype=np.complex128)
    for off, W in blocks_.items():
        out += _mv(W, neighbour_spinor(psi, off, bc))
    return out


def apply(U, c, psi, bc=(1, 1, 1, 1)):
    """M psi by Eq. minFlopForm."""
    return apply_blocks(blocks(U, c), psi, bc)


def apply_final_form(U, c, psi, bc=(1, 1, 1, 1)):
    """M psi by the shifted two-step form of Eq. FinalForm.

    The matrices kept at x are W^0_x, W^+_{mu,x}, W^{++}_{ii,x-i}, W^{++}_{ij,x-j}, W^{+-}_{ij,x+j};
    W^-_{mu,x+mu} and W^{--}_{ii,x+i} are formed at x from them (Eq. opp_diag_pre_mat); only
    nearest-neighbour spinors are gathered, and the products are moved by one site.
    """
    p = forward_parts(U, c)

    def t(f, mu, sgn):  # (t_{sgn mu} f)_x = f_{x + sgn mu}
        return neighbour_spinor(f, _vec({mu: sgn}), bc)

    def nb(mu, sgn):
        return neighbour_spinor(psi, _vec({mu: sgn}), bc)

    out = _mv(blk(*p["W0"]), psi)
    for mu in range(4):
        Wp = blk(*p["W+"][mu])
        out += _mv(Wp, nb(mu, +1))
        if mu < 3:
            Dd, Sd = dag(p["D+"][mu]), dag(p["S+"][mu])
            Wm_shift = blk(Dd, -Sd, -Sd, Dd)                       # W^-_{mu, x+mu}
        else:
            Wm_shift = blk(-dag(p["U4"]), -dag(p["S+4"]), -dag(p["S+4"]), None)
        out += t(_mv(Wm_shift, psi), mu, -1)
    for i in range(3):
        A = shift(blk(*p["W++ii"][i]), i, -1)                      # W^{++}_{ii, x-i}
        out += t(_mv(A, nb(i, +1)), i, +1)
        Dd = dag(shift(p["D++"][i], i, -1))
        Sd = dag(shift(p["S++"][i], i, -1))
        Wmm_shift = blk(Dd, -Sd, -Sd, Dd)                          # W^{--}_{ii, x+i}
        out += t(_mv(Wmm_shift, nb(i, -1)), i, -1)
    for i in range(3):
        for j in range(i + 1, 3):
            Bij = shift(blk(*p["W++ij"][(i, j)]), j, -1)           # W^{++}_{ij, x-j}
            Cij = shift(blk(*p["W+-ij"][(i, j)]), j, +1)           # W^{+-}_{ij, x+j}
            out += t(_mv(Bij, nb(i, +1)), j, +1)
            out -= t(_mv(dag(Bij), nb(j, -1)), i, -1)
            out += t(_mv(Cij, nb(i, +1)), j, -1)
            out -= t(_mv(dag(Cij), nb(j, +1)), i, -1)
    return out
