"""Gauge-field quantities (oracle; test infrastructure).

* Mean plaquette and tadpole factor u0. The paper uses the tadpole-improved action (Sec. 1) and
  writes powers of u0 throughout Eqs. shifted_W_first .. shifted_W_last; u0 is the fourth root of
  the mean of (1/3) Re tr of the plaquette over all sites and the six planes.
* Clover field strength F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger) / 8, Q the sum of the four
  plaquette leaves around x with one orientation; no trace is subtracted. E_i = F_{4 i} and
  B_i = (1/2) eps_ijk F_jk, the fields inside E-bar^S and B-bar^D of Eq. shifted_W_first.
"""
import numpy as np

from .lattice import shift, shift_vec, dag


def link(U, mu):
    """U_mu(x) as a field over x, shape (T, Z, Y, X, 3, 3)."""
    return U[..., mu, :, :]


def plaquette(U, mu, nu):
    """U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger."""
    Um, Un = link(U, mu), link(U, nu)
    return Um @ shift(Un, mu) @ dag(shift(Um, nu)) @ dag(Un)


def mean_plaquette(U) -> float:
    """(1/3) Re tr of the plaquette averaged over all sites and the six planes (mu < nu)."""
    acc = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            acc += np.trace(plaquette(U, mu, nu), axis1=-2, axis2=-1).real.mean() / 3.0
    return acc / 6.0


def tadpole_u0(U) -> float:
    """u0 = <(1/3) Re tr U_plaq>^(1/4)."""
    return mean_plaquette(U) ** 0.25


def clover_leaves(U, mu, nu):
    """Q_{mu nu}(x): the four plaquettes in the (mu, nu) plane that start and end at x,
    each traversed mu-then-nu (counter-clockwise)."""
    Um, Un = link(U, mu), link(U, nu)
    e_m = [0, 0, 0, 0]
    e_m[mu] = 1
    e_n = [0, 0, 0, 0]
    e_n[nu] = 1

    def at(f, a, b):  # f at x + a*mu + b*nu
        vec = [a * e_m[k] + b * e_n[k] for k in range(4)]
        return shift_vec(f, vec)

    leaf1 = Um @ at(Un, 1, 0) @ dag(at(Um, 0, 1)) @ dag(Un)
    leaf2 = Un @ dag(at(Um, -1, 1)) @ dag(at(Un, -1, 0)) @ at(Um, -1, 0)
    leaf3 = dag(at(Um, -1, 0)) @ dag(at(Un, -1, -1)) @ at(Um, -1, -1) @ at(Un, 0, -1)
    leaf4 = dag(at(Un, 0, -1)) @ at(Um, 0, -1) @ at(Un, 1, -1) @ dag(Um)
    return leaf1 + leaf2 + leaf3 + leaf4


def clover_F(U, mu, nu):
    """F_{mu nu} = (Q - Q^dagger) / 8 (anti-Hermitian, not traceless-projected)."""
    Q = clover_leaves(U, mu, nu)
    return (Q - dag(Q)) / 8.0


def clover_EB(U):
    """(E, B): lists of three fields, E_i = F_{t i}, B_i = (1/2) eps_ijk F_jk = F_{i+1, i+2}."""
    E = [clover_F(U, 3, i) for i in range(3)]
    B = [clover_F(U, (i + 1) % 3, (i + 2) % 3) for i in range(3)]
    return E, B


def gauge_transform_links(U, omega):
    """U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dagger."""
    out = np.empty_like(U)
    for mu in range(4):
        out[..., mu, :, :] = omega @ U[..., mu, :, :] @ dag(shift(omega, mu))
    return out


def gauge_transform_spinor(psi, omega):
    """psi'(x) = Omega(x) psi(x) on the colour index of a [..., 4, 3] field."""
    return np.einsum("...ab,...sb->...sa", omega, psi)
