"""Spin matrices (oracle; test infrastructure).

The paper uses the Dirac representation of its Ref. [EKM] without printing it (Sec. 2.2, text before
Eq. shifted_W_first). The block forms of W^+_4 = [[0, S], [S, -U_4]] and W^+_i = [[D, S], [S, D]]
fix it: the forward temporal hop of a Wilson-type action is -(1 - gamma_4) U_4 / 2, whose only
non-zero block is the lower-right one, so gamma_4 = diag(1, 1, -1, -1); the spatial hop
(zeta gamma_i - r_s zeta) U_i / 2 has equal diagonal blocks and equal off-diagonal blocks
proportional to sigma_i, so gamma_i = [[0, sigma_i], [sigma_i, 0]].

Spin index s = 2 * a + b, a = upper/lower 2x2 block, b = index inside the block; spin-colour
index 3 * s + c.
"""
import numpy as np

I2 = np.eye(2, dtype=np.complex128)
I4 = np.eye(4, dtype=np.complex128)
PAULI = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]
TAU1 = PAULI[0]
TAU3 = PAULI[2]

# gamma[mu], mu = 0, 1, 2 spatial (x, y, z) and 3 temporal (the paper's mu = 4).
GAMMA = [np.kron(TAU1, PAULI[i]) for i in range(3)] + [np.kron(TAU3, I2)]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
# Sigma_i = 1 (x) sigma_i (spin rotation generators) and alpha_i = gamma_4 gamma_i.
SIGMA = [np.kron(I2, PAULI[i]) for i in range(3)]
ALPHA = [GAMMA[3] @ GAMMA[i] for i in range(3)]


def levi_civita(i: int, j: int, k: int) -> int:
    """epsilon_ijk for i, j, k in {0, 1, 2}."""
    if len({i, j, k}) < 3:
        return 0
    return 1 if (i, j, k) in ((0, 1, 2), (1, 2, 0), (2, 0, 1)) else -1
