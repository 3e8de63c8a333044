"""Lattice helpers (oracle; test infrastructure).

Fields carry leading site axes (T, Z, Y, X); direction mu = 0, 1, 2, 3 is x, y, z, t.
"""
import numpy as np

AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def dims_of(field) -> tuple:
    """(X, Y, Z, T) of a field with leading site axes (T, Z, Y, X)."""
    T, Z, Y, X = field.shape[:4]
    return (X, Y, Z, T)


def shift(field, mu: int, n: int = 1):
    """The field at x + n * mu-hat (periodic), as a field over x."""
    return np.roll(field, -n, axis=AXIS[mu])


def shift_vec(field, nvec):
    """The field at x + nvec (periodic), nvec = (nx, ny, nz, nt)."""
    out = field
    for mu, n in enumerate(nvec):
        if n:
            out = np.roll(out, -n, axis=AXIS[mu])
    return out


def dag(m):
    """Hermitian conjugate over the last two axes."""
    return np.conj(np.swapaxes(m, -1, -2))


def bc_sign(dims, nvec, bc):
    """Sign picked up by a fermion hopping from x to x + nvec under boundary phases bc[mu] = +-1.

    Each wrap across the lattice boundary in direction mu multiplies by bc[mu]. Returns an array
    broadcastable over (T, Z, Y, X).
    """
    X, Y, Z, T = dims
    sizes = (X, Y, Z, T)
    sign = np.ones((T, Z, Y, X))
    for mu, n in enumerate(nvec):
        if n == 0 or bc[mu] == 1:
            continue
        L = sizes[mu]
        coord = np.arange(L)
        wraps = np.floor_divide(coord + n, L)
        s = np.where(wraps % 2 == 0, 1.0, -1.0)
        shape = [1, 1, 1, 1]
        shape[AXIS[mu]] = L
        sign = sign * s.reshape(shape)
    return sign


def neighbour_spinor(psi, nvec, bc):
    """psi at x + nvec with boundary signs, as a field over x."""
    dims = dims_of(psi)
    out = shift_vec(psi, nvec)
    if any(b != 1 for b in bc):
        out = out * bc_sign(dims, nvec, bc)[..., None, None]
    return out
