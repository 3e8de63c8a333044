"""Learned right preconditioner: a gauge-covariant linear network (oracle; test infrastructure).

The paper's solver is unpreconditioned BiCGStab (Sec. 2.3); this module is the reference for the
preconditioner P that the library adds to it, written from its definition:

    P = L_K ... L_2 L_1,    (L psi)(x) = sum_d  A_d  (T_d psi)(x)

over the nine offsets d = 0, +x, -x, +y, -y, +z, -z, +t, -t.  T_0 is the identity and T_d for
d = +-mu is the covariant shift with the gauge links, exactly the transport of the hopping terms of
Eq. minFlopForm (W^+_mu multiplies U_mu(x) psi(x + mu), W^-_mu the adjoint link from x - mu):

    (T_{+mu} psi)(x) = U_mu(x) psi(x + mu),   (T_{-mu} psi)(x) = U_mu(x - mu)^dag psi(x - mu),

with the fermion boundary sign of a hop across an antiperiodic boundary.  A_d is a learned 4 x 4
complex spin matrix (the same at every site) acting on the spin index; the colour index is only
transported.  P is linear in psi, so the right-preconditioned system M P y = b has the fixed
operator M P, and it is gauge covariant: P[U^Omega] (Omega psi) = Omega P[U] psi.

Training minimises  loss = |P b - x|^2 / |x|^2  over (source, solution) pairs, and the gradient
with respect to A_{l,d} is, with g_K = (P b - x) / |x|^2, g_{l-1} = L_l^dag g_l and
w_{l,d} = T_d psi_{l-1},

    dloss / dA_{l,d}  =  2 sum_{x, colour} g_l(x) w_{l,d}(x)^dag      (spin s, s' entry),

where the complex derivative is d/dRe + i d/dIm.  Everything is complex128 numpy over whole
lattice arrays, in the order of these definitions.
"""
import numpy as np

from . import lattice as lat

# Offsets in the order of the stored weights: (direction, step); direction -1 is the on-site term.
OFFSETS = [(-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1), (3, 1), (3, -1)]
NOFF = len(OFFSETS)


def _unit(mu):
    v = [0, 0, 0, 0]
    v[mu] = 1
    return tuple(v)


def shift_op(U, psi, d, bc=(1, 1, 1, 1)):
    """T_d psi for offset index d (psi [T, Z, Y, X, 4, 3], U [T, Z, Y, X, 4, 3, 3])."""
    mu, step = OFFSETS[d]
    if mu < 0:
        return psi.copy()
    if step > 0:
        nb = lat.neighbour_spinor(psi, _unit(mu), bc)
        return np.einsum("...ab,...sb->...sa", U[..., mu, :, :], nb)
    back = tuple(-k for k in _unit(mu))
    nb = lat.neighbour_spinor(psi, back, bc)
    Uback = lat.shift_vec(U[..., mu, :, :], back)
    return np.einsum("...ab,...sb->...sa", lat.dag(Uback), nb)


def spin_mul(A, psi):
    """A (4 x 4, spin) times psi on the spin index."""
    return np.einsum("st,...tc->...sc", A, psi)


def layer(U, A, psi, bc=(1, 1, 1, 1)):
    """(L psi)(x) = sum_d A[d] (T_d psi)(x);  A [9, 4, 4]."""
    out = np.zeros_like(psi)
    for d in range(NOFF):
        out = out + spin_mul(A[d], shift_op(U, psi, d, bc))
    return out


def apply(U, A_all, psi, bc=(1, 1, 1, 1)):
    """P psi = L_K ... L_1 psi;  A_all [K, 9, 4, 4]."""
    out = psi
    for A in A_all:
        out = layer(U, A, out, bc)
    return out


def shift_adjoint(U, phi, d, bc=(1, 1, 1, 1)):
    """T_d^dag phi, written from the definition <phi, T_d psi> = <T_d^dag phi, psi>:
    (T_{+mu}^dag phi)(y) = U_mu(y - mu)^dag phi(y - mu) and (T_{-mu}^dag phi)(y) = U_mu(y) phi(y + mu)."""
    mu, step = OFFSETS[d]
    if mu < 0:
        return phi.copy()
    if step > 0:
        back = tuple(-k for k in _unit(mu))
        nb = lat.neighbour_spinor(phi, back, bc)
        Uback = lat.shift_vec(U[..., mu, :, :], back)
        return np.einsum("...ab,...sb->...sa", lat.dag(Uback), nb)
    nb = lat.neighbour_spinor(phi, _unit(mu), bc)
    return np.einsum("...ab,...sb->...sa", U[..., mu, :, :], nb)


def layer_adjoint(U, A, phi, bc=(1, 1, 1, 1)):
    """L^dag phi = sum_d T_d^dag (A[d]^dag phi)."""
    out = np.zeros_like(phi)
    for d in range(NOFF):
        out = out + shift_adjoint(U, spin_mul(np.conj(A[d]).T, phi), d, bc)
    return out


def loss_and_grad(U, A_all, b, x, bc=(1, 1, 1, 1)):
    """loss = |P b - x|^2 / |x|^2 and its complex gradient [K, 9, 4, 4] (d/dRe + i d/dIm)."""
    acts = [b]
    for A in A_all:
        acts.append(layer(U, A, acts[-1], bc))
    n2 = float(np.vdot(x, x).real)
    e = acts[-1] - x
    loss = float(np.vdot(e, e).real) / n2
    g = e / n2
    grad = np.zeros_like(A_all)
    for l in range(len(A_all) - 1, -1, -1):
        for d in range(NOFF):
            w = shift_op(U, acts[l], d, bc)
            grad[l, d] = 2.0 * np.einsum("nsc,ntc->st", g.reshape(-1, 4, 3), np.conj(w).reshape(-1, 4, 3))
        g = layer_adjoint(U, A_all[l], g, bc)
    return loss, grad


def identity_weights(layers: int, scale: float = 1.0):
    """Weights with A_0 = scale^(1/K) 1 and every other offset zero: P = scale * identity."""
    A = np.zeros((layers, NOFF, 4, 4), dtype=np.complex128)
    for l in range(layers):
        A[l, 0] = np.eye(4) * scale ** (1.0 / layers)
    return A
