"""Free-field closed form of the OK operator in momentum space (a pin for the oracle).

With unit links, u0 = 1 and E = B = 0, a plane wave psi_x = exp(i p.x) chi is an eigenvector of
every shift: T_{+mu} -> exp(i p_mu), T_{-mu} -> exp(-i p_mu), so Nabla_mu -> i sin p_mu and
Delta_mu -> -p_hat_mu^2 with p_hat_mu = 2 sin(p_mu / 2). The action then gives
  M(p) = am0 + p_hat_4^2/2 + (r_s zeta / 2) sum_i p_hat_i^2 + c4 sum_i p_hat_i^4
         + i gamma_4 sin p_4 + i sum_i gamma_i sin p_i [zeta - c1 p_hat_i^2 - 2 c2 sum_j p_hat_j^2].
"""
import numpy as np


def momenta(L, bc):
    n = np.arange(L)
    return 2 * np.pi * n / L if bc == 1 else (2 * n + 1) * np.pi / L


def M_of_p(p, c, gamma, am0):
    """12x12 (spin (x) colour-identity) closed form at momentum p = (px, py, pz, pt)."""
    ph2 = [4 * np.sin(pm / 2) ** 2 for pm in p]
    scal = am0 + 0.5 * ph2[3] + 0.5 * c.r_s * c.zeta * sum(ph2[:3]) + c.c4 * sum(h * h for h in ph2[:3])
    m = scal * np.eye(4, dtype=np.complex128) + 1j * gamma[3] * np.sin(p[3])
    s2 = sum(ph2[:3])
    for i in range(3):
        m = m + 1j * gamma[i] * np.sin(p[i]) * (c.zeta - c.c1 * ph2[i] - 2 * c.c2 * s2)
    return np.kron(m, np.eye(3))


def plane_wave(dims, p, chi):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None] * chi.reshape(4, 3)
