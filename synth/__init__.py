"""Seeded synthetic inputs shared by the CUDA path's tests and benchmarks and by the oracle.

This module generates inputs only: gauge links, gauge transformations, fermion sources and the
coefficient records that parametrise the operator. It holds none of the method's arithmetic
(no plaquette, clover, W matrix, hop or solver step).

Recipe (all deterministic from a 64-bit seed):

* Random numbers: splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014). Output k (k = 0, 1, ...) of the stream seeded with s is
  mix(s + (k+1) * 0x9E3779B97F4A7C15) with the published 64-bit finaliser `mix`, so the stream is
  counter-based and vectorises.  A uniform double in [0, 1) is (output >> 11) * 2^-53.
* Gaussians: Box-Muller on consecutive uniform pairs (u_a, u_b):
  n0 = sqrt(-2 ln(1 - u_a)) cos(2 pi u_b), n1 = sqrt(-2 ln(1 - u_a)) sin(2 pi u_b).
* SU(3) links: for every link, a 3x3 complex A with real and imaginary parts drawn iid N(0, 1),
  H = (A + A^dagger)/2 - tr(.)/3 (traceless Hermitian), U = exp(i eps H) computed through the
  Hermitian eigendecomposition H = Q diag(l) Q^dagger, U = Q diag(exp(i eps l)) Q^dagger.
  eps sets the roughness: eps -> 0 is the free field.
* Layouts: links [T][Z][Y][X][mu=4][3][3] complex with mu = 0,1,2,3 = x,y,z,t; fermion fields
  [T][Z][Y][X][spin=4][colour=3] complex. Site order is lexicographic with x fastest.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict, field
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the splitmix64 stream seeded with `seed` (uint64 array)."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the splitmix64 stream."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m).reshape(m, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    th = 2.0 * np.pi * u[:, 1]
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1).reshape(-1)[:n]


def lattice_shape(dims) -> tuple:
    """dims = (X, Y, Z, T) -> array shape (T, Z, Y, X)."""
    X, Y, Z, T = (int(d) for d in dims)
    return (T, Z, Y, X)


def random_su3(shape, eps: float, seed: int) -> np.ndarray:
    """Array of SU(3) matrices exp(i eps H), H traceless Hermitian with Gaussian entries."""
    shape = tuple(int(s) for s in shape)
    count = int(np.prod(shape)) if shape else 1
    g = gaussian(seed, count * 18).reshape(count, 3, 3, 2)
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    lam, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    u = np.einsum("nab,nb,ncb->nac", q, ph, np.conj(q))
    return u.reshape(shape + (3, 3))


def random_links(dims, eps: float, seed: int) -> np.ndarray:
    """Gauge field [T][Z][Y][X][4][3][3] complex128 of SU(3) links exp(i eps H)."""
    return random_su3(lattice_shape(dims) + (4,), eps, seed)


def device_random_links(dims, eps: float, seed: int, device="cuda"):
    """The distribution of `random_links` drawn on a CUDA device with torch's seeded generator
    (for lattices where the host generator takes minutes): A with iid N(0, 1) real and imaginary
    entries, H = (A + A^dag) / 2 - tr / 3, U = exp(i eps H) (torch's batched matrix exponential;
    the host recipe's eigendecomposition gives the same matrix up to rounding).  Returns a
    [T][Z][Y][X][4][3][3] complex128 tensor on the device; the bits differ from `random_links` for
    the same seed."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    shape = lattice_shape(dims) + (4,)
    n = int(np.prod(shape))
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    chunk = 1 << 18
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    for s0 in range(0, n, chunk):
        m = min(chunk, n - s0)
        a = torch.view_as_complex(torch.randn((m, 3, 3, 2), generator=g, device=device, dtype=torch.float64))
        h = 0.5 * (a + a.conj().transpose(-1, -2))
        tr = torch.diagonal(h, dim1=-2, dim2=-1).sum(-1).real / 3.0
        h = h - tr[:, None, None] * eye
        out[s0:s0 + m] = torch.linalg.matrix_exp((1j * eps) * h)
    return out.reshape(shape + (3, 3))


def unit_links(dims) -> np.ndarray:
    """Free-field gauge configuration: every link is the 3x3 identity."""
    u = np.zeros(lattice_shape(dims) + (4, 3, 3), dtype=np.complex128)
    u[..., :, :] = np.eye(3)
    return u


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """A generic SU(3) matrix per site, [T][Z][Y][X][3][3]."""
    return random_su3(lattice_shape(dims), 2.0, seed)


def point_source(dims, site: int = 0, spin: int = 0, colour: int = 0) -> np.ndarray:
    """Unit source at one (site, spin, colour), [T][Z][Y][X][4][3] complex128."""
    shp = lattice_shape(dims)
    b = np.zeros(shp + (4, 3), dtype=np.complex128)
    b.reshape(-1, 4, 3)[site, spin, colour] = 1.0
    return b


def gaussian_source(dims, seed: int) -> np.ndarray:
    """Complex field with real and imaginary parts iid N(0, 1), [T][Z][Y][X][4][3]."""
    shp = lattice_shape(dims) + (4, 3)
    n = int(np.prod(shp))
    g = gaussian(seed, 2 * n).reshape(n, 2)
    return (g[:, 0] + 1j * g[:, 1]).reshape(shp)


@dataclass
class OKCoeffs:
    """Parameters of the tree-level tadpole-improved OK operator.

    u0 <= 0 means "take the tadpole factor from the mean plaquette of the links";
    kappa <= 0 means "derive the hopping parameter from am0".
    """
    u0: float = -1.0
    am0: float = 0.5
    kappa: float = -1.0
    zeta: float = 1.0
    r_s: float = 1.0
    c_B: float = 1.0
    c_E: float = 1.0
    c_EE: float = 0.0
    c1: float = 0.0
    c2: float = 0.0
    c3: float = 0.0
    c4: float = 0.0
    c5: float = 0.0

    def as_dict(self) -> dict:
        return asdict(self)

    def replace(self, **kw) -> "OKCoeffs":
        d = asdict(self)
        d.update(kw)
        return OKCoeffs(**d)


def placeholder_coeffs(am0: float) -> OKCoeffs:
    """Placeholder coefficient set used for the benchmark workloads.

    The tree-level OK coefficient formulas are given in the works the paper cites, not in the paper
    itself, so these values are placeholders: zeta = r_s = c_B = c_E = 1 (Fermilab tree level at
    small mass) and small positive improvement coefficients, which keeps the free-field real part
    am0 + sum_mu p_hat^2 / 2 + c4 sum_i p_hat_i^4 positive.
    """
    return OKCoeffs(u0=-1.0, am0=am0, kappa=-1.0, zeta=1.0, r_s=1.0, c_B=1.0, c_E=1.0,
                    c_EE=0.03, c1=0.05, c2=0.02, c3=0.04, c4=0.03, c5=0.02)


def random_coeffs(seed: int, u0: float = -1.0) -> OKCoeffs:
    """Coefficients drawn uniformly in [0.1, 1] (every term of the action switched on)."""
    v = 0.1 + 0.9 * uniform(seed, 12)
    return OKCoeffs(u0=u0, am0=0.2 + v[0], kappa=-1.0, zeta=v[1], r_s=v[2], c_B=v[3], c_E=v[4],
                    c_EE=v[5], c1=v[6], c2=v[7], c3=v[8], c4=v[9], c5=v[10])


# Workloads: lattice (X, Y, Z, T), link roughness, link seed, bare mass, source kind.
WORKLOADS = {
    "4^3x8": dict(dims=(4, 4, 4, 8), eps=0.3, seed=13115029, am0=1.0, source="point"),
    "16^3x32": dict(dims=(16, 16, 16, 32), eps=0.2, seed=13115030, am0=0.5, source="gaussian"),
    "20^3x64": dict(dims=(20, 20, 20, 64), eps=0.2, seed=13115031, am0=1.0, source="gaussian"),
    "28^3x96": dict(dims=(28, 28, 28, 96), eps=0.15, seed=13115032, am0=0.8, source="gaussian"),
}


def workload_inputs(name: str, source_seed: int = 7):
    """(dims, links, coeffs, source) for a named workload."""
    w = WORKLOADS[name]
    links = random_links(w["dims"], w["eps"], w["seed"])
    coeffs = placeholder_coeffs(w["am0"])
    if w["source"] == "point":
        src = point_source(w["dims"])
    else:
        src = gaussian_source(w["dims"], source_seed)
    return w["dims"], links, coeffs, src
