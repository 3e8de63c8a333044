"""The table that the double-float apply walks (csrc/ok_dd_table.cuh), built on the host.

The header is compiled for the host and its table printed; the table is then evaluated on random
matrices and spinors (any 43 colour matrices per site, not a physical W) and compared with a
transcription of the templated one-thread-per-site apply of csrc/ok_apply.cu (onsite term, the
hop_spatial, hop_time, hop_two and hop_diag functions), which the GPU parity tests pin to the
oracle.  Random matrices make every entry's matrix, source, accumulator, factor and unit count."""
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1311_5029_gb300", "csrc")

HARNESS = r"""
#include "ok_dd_table.cuh"
#include <cstdio>
int main() {
  const okgb::DDTable t = okgb::ddtab::build_table();
  for (int h = 0; h < okgb::DD_HOPS; ++h) {
    const okgb::DDHop& p = t.hop[h];
    printf("H %d %d %d %d %d %d %d\n", p.d[0], p.d[1], p.d[2], p.d[3], p.kind, p.first, p.count);
  }
  for (int a = 0; a < okgb::DD_ACTS; ++a) {
    const okgb::DDAct& x = t.act[a];
    printf("A %d %d %d %d %d %d\n", x.m, x.flags, x.dst[0], x.dst[1], x.mul[0], x.mul[1]);
  }
  return 0;
}
"""

# matrix indices of the stored forward set (csrc/ok_internal.cuh)
M_Y0P, M_Y0M, M_UT, M_ST, M_WP, M_VII, M_VIJ, M_XIJ = 0, 3, 6, 7, 10, 34, 37, 40
UNITS = [1, 1j, -1, -1j, 1 + 1j, 1 - 1j, -1 - 1j, -1 + 1j]


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("ddtab")
    src = d / "dump.cu"
    src.write_text(HARNESS)
    exe = d / "dump"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True,
                   timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    hops, acts = [], []
    for line in out.splitlines():
        f = line.split()
        (hops if f[0] == "H" else acts).append(list(map(int, f[1:])))
    return hops, acts


class Lattice:
    def __init__(self, L, bcneg, seed):
        self.L, self.bcneg = L, bcneg
        self.V = L[0] * L[1] * L[2] * L[3]
        self.S = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
        rng = np.random.default_rng(seed)
        self.W = rng.standard_normal((self.V, 43, 3, 3)) + 1j * rng.standard_normal((self.V, 43, 3, 3))
        self.psi = rng.standard_normal((self.V, 12)) + 1j * rng.standard_normal((self.V, 12))

    def coords(self, s):
        c = []
        for mu in range(4):
            c.append(s % self.L[mu])
            s //= self.L[mu]
        return c

    def nbr(self, c, d):
        idx, neg = 0, False
        for mu in range(4):
            x, w = c[mu] + d[mu], 0
            while x >= self.L[mu]:
                x, w = x - self.L[mu], w + 1
            while x < 0:
                x, w = x + self.L[mu], w + 1
            if (self.bcneg >> mu) & 1 and w % 2:
                neg = not neg
            idx += x * self.S[mu]
        return idx, neg

    def gather(self, c, d):
        """(neighbour, h+ = u + l, h- = u - l, u, l) with the boundary sign."""
        n, neg = self.nbr(c, d)
        v = -self.psi[n] if neg else self.psi[n]
        u, lo = [v[0:3], v[3:6]], [v[6:9], v[9:12]]
        return n, [u[q] + lo[q] for q in range(2)], [u[q] - lo[q] for q in range(2)], u, lo


def mv(A, v):
    return A @ v


def mdv(A, v):
    return A.conj().T @ v


def add_sigma(acc, k, y, f):
    """acc += f sigma_k y on a 2-spinor of colour vectors (k = 0, 1, 2 for x, y, z)."""
    if k == 0:
        acc[0] = acc[0] + f * y[1]
        acc[1] = acc[1] + f * y[0]
    elif k == 1:
        acc[0] = acc[0] - 1j * f * y[1]
        acc[1] = acc[1] + 1j * f * y[0]
    else:
        acc[0] = acc[0] + f * y[0]
        acc[1] = acc[1] - f * y[1]


def templated_apply(lat, s, c0q, a_ii, b_ii):
    """M psi at site s as the templated kernel computes it, term by term."""
    c = lat.coords(s)
    Wx = lat.W[s]
    x0 = lat.psi[s]
    u, lo = [x0[0:3], x0[3:6]], [x0[6:9], x0[9:12]]
    a = [u[q] - 1j * lo[q] for q in range(2)]
    b = [u[q] + 1j * lo[q] for q in range(2)]
    A = [c0q * a[q] for q in range(2)]
    B = [c0q * b[q] for q in range(2)]
    A[0] += mv(Wx[M_Y0P], a[0]); A[1] -= mv(Wx[M_Y0P], a[1])
    A[0] += mv(Wx[M_Y0P + 1], a[1]); A[1] += mv(Wx[M_Y0P + 2], a[0])
    B[0] += mv(Wx[M_Y0M], b[0]); B[1] -= mv(Wx[M_Y0M], b[1])
    B[0] += mv(Wx[M_Y0M + 1], b[1]); B[1] += mv(Wx[M_Y0M + 2], b[0])
    ap = [(A[q] + B[q]) + 1j * (A[q] - B[q]) for q in range(2)]
    am = [(A[q] + B[q]) - 1j * (A[q] - B[q]) for q in range(2)]

    def block2(Wm, m, h, acc, dag):
        if dag:
            acc[0] += mdv(Wm[m], h[0]); acc[1] += mdv(Wm[m + 1], h[0])
            acc[0] += mdv(Wm[m + 2], h[1]); acc[1] += mdv(Wm[m + 3], h[1])
        else:
            acc[0] += mv(Wm[m], h[0]); acc[0] += mv(Wm[m + 1], h[1])
            acc[1] += mv(Wm[m + 2], h[0]); acc[1] += mv(Wm[m + 3], h[1])

    for I in range(3):
        mp = M_WP + 8 * I
        mm = mp + 4
        e = [int(I == k) for k in range(3)]
        _, hp, hm, _, _ = lat.gather(c, e + [0])
        block2(Wx, mp, hp, ap, False); block2(Wx, mm, hm, am, False)
        n, hp, hm, _, _ = lat.gather(c, [-k for k in e] + [0])
        block2(lat.W[n], mm, hp, ap, True); block2(lat.W[n], mp, hm, am, True)
    # temporal hops
    _, hp, hm, _, low = lat.gather(c, [0, 0, 0, 1])
    w = [mv(Wx[M_UT], low[q]) for q in range(2)]
    for q in range(2):
        ap[q] = ap[q] - w[q]; am[q] = am[q] + w[q]
    s3, n1, n2 = Wx[M_ST], Wx[M_ST + 1], Wx[M_ST + 2]
    ap[0] += mv(s3, hp[0]); ap[1] -= mv(s3, hp[1]); am[0] -= mv(s3, hm[0]); am[1] += mv(s3, hm[1])
    ap[0] += mv(n1, hp[1]); am[0] -= mv(n1, hm[1])
    ap[1] += mv(n2, hp[0]); am[1] -= mv(n2, hm[0])
    n, hp, hm, upp, _ = lat.gather(c, [0, 0, 0, -1])
    Wn = lat.W[n]
    w = [mdv(Wn[M_UT], upp[q]) for q in range(2)]
    for q in range(2):
        ap[q] = ap[q] - w[q]; am[q] = am[q] - w[q]
    s3, n1, n2 = Wn[M_ST], Wn[M_ST + 1], Wn[M_ST + 2]
    ap[0] -= mdv(s3, hp[0]); ap[1] += mdv(s3, hp[1]); am[0] += mdv(s3, hm[0]); am[1] -= mdv(s3, hm[1])
    ap[1] -= mdv(n1, hp[0]); am[1] += mdv(n1, hm[0])
    ap[0] -= mdv(n2, hp[1]); am[0] += mdv(n2, hm[1])
    # straight two hops
    for I in range(3):
        e = [2 * int(I == k) for k in range(3)]
        _, hp, hm, _, _ = lat.gather(c, e + [0])
        Vm = Wx[M_VII + I]
        y = [mv(Vm, hp[q]) for q in range(2)]
        ap[0] += a_ii * y[0]; ap[1] += a_ii * y[1]; add_sigma(ap, I, y, b_ii)
        y = [mv(Vm, hm[q]) for q in range(2)]
        am[0] += a_ii * y[0]; am[1] += a_ii * y[1]; add_sigma(am, I, y, -b_ii)
        n, hp, hm, _, _ = lat.gather(c, [-k for k in e] + [0])
        Vm = lat.W[n][M_VII + I]
        y = [mdv(Vm, hp[q]) for q in range(2)]
        ap[0] += a_ii * y[0]; ap[1] += a_ii * y[1]; add_sigma(ap, I, y, -b_ii)
        y = [mdv(Vm, hm[q]) for q in range(2)]
        am[0] += a_ii * y[0]; am[1] += a_ii * y[1]; add_sigma(am, I, y, b_ii)
    # diagonal pairs
    for P, (I, J) in enumerate([(0, 1), (0, 2), (1, 2)]):
        dA = [int(I == k) + int(J == k) for k in range(3)]
        dB = [int(I == k) - int(J == k) for k in range(3)]
        for d, m, sj in ((dA, M_VIJ + P, 1), (dB, M_XIJ + P, -1)):
            _, hp, hm, _, _ = lat.gather(c, d + [0])
            y = [mv(Wx[m], hp[q]) for q in range(2)]
            add_sigma(ap, I, y, 1); add_sigma(ap, J, y, sj)
            y = [mv(Wx[m], hm[q]) for q in range(2)]
            add_sigma(am, I, y, -1); add_sigma(am, J, y, -sj)
            n, hp, hm, _, _ = lat.gather(c, [-k for k in d] + [0])
            y = [mdv(lat.W[n][m], hp[q]) for q in range(2)]
            add_sigma(ap, I, y, -1); add_sigma(ap, J, y, -sj)
            y = [mdv(lat.W[n][m], hm[q]) for q in range(2)]
            add_sigma(am, I, y, 1); add_sigma(am, J, y, sj)
    return np.concatenate([ap[0] + am[0], ap[1] + am[1], ap[0] - am[0], ap[1] - am[1]])


def table_apply(lat, s, hops, acts, c0q, a_ii, b_ii):
    """M psi at site s by walking the table as the double-float kernel does."""
    c = lat.coords(s)
    scal = [1.0, a_ii, b_ii]
    acc = [np.zeros(3, complex) for _ in range(4)]
    for d0, d1, d2, d3, kind, first, count in hops:
        n, neg = lat.nbr(c, [d0, d1, d2, d3])
        v = -lat.psi[n] if neg else lat.psi[n]
        u, lo = [v[0:3], v[3:6]], [v[6:9], v[9:12]]
        if kind == 0:  # on-site: slots u - i l, u + i l; the c0q part of W^0 initialises acc
            slots = [u[0] - 1j * lo[0], u[1] - 1j * lo[1], u[0] + 1j * lo[0], u[1] + 1j * lo[1], None, None]
            acc = [2 * c0q * (u[0] + lo[0]), 2 * c0q * (u[1] + lo[1]), 2 * c0q * (u[0] - lo[0]), 2 * c0q * (u[1] - lo[1])]
        else:
            t3 = lo if kind == 2 else u
            slots = [u[0] + lo[0], u[1] + lo[1], u[0] - lo[0], u[1] - lo[1], t3[0], t3[1]]
        for m, flags, dst0, dst1, mul0, mul1 in acts[first:first + count]:
            Wm = lat.W[n if flags & 1 else s][m]
            y = mdv(Wm, slots[flags >> 2]) if flags & 2 else mv(Wm, slots[flags >> 2])
            for dst, mul in ((dst0, mul0), (dst1, mul1)):
                if dst >= 0:
                    acc[dst] = acc[dst] + scal[mul & 3] * UNITS[mul >> 2] * y
    return np.concatenate([acc[0] + acc[2], acc[1] + acc[3], acc[0] - acc[2], acc[1] - acc[3]])


def test_table_shape(table):
    hops, acts = table
    assert len(hops) == 27 and len(acts) == 148
    offsets = {tuple(h[:4]) for h in hops}
    expect = {(0, 0, 0, 0)}
    for mu in range(4):
        for st in (1, -1):
            expect.add(tuple(st * int(mu == k) for k in range(4)))
    for i in range(3):
        for st in (2, -2):
            expect.add(tuple(st * int(i == k) for k in range(3)) + (0,))
        for j in range(i + 1, 3):
            for si in (1, -1):
                for sj in (1, -1):
                    expect.add(tuple(si * int(i == k) + sj * int(j == k) for k in range(3)) + (0,))
    assert offsets == expect  # the 27 offsets of Eq. minFlopForm
    assert [h[5] for h in hops] == list(np.cumsum([0] + [h[6] for h in hops[:-1]]))
    # every stored forward matrix is used at x, and only matrices of a neighbour are adjoint
    assert {a[0] for a in acts if not a[1] & 1} == set(range(43))
    assert all(bool(a[1] & 1) == bool(a[1] & 2) for a in acts)


@pytest.mark.parametrize("L,bcneg", [((4, 3, 5, 2), 0b1010), ((2, 1, 3, 4), 0b0001), ((3, 3, 3, 3), 0)])
def test_table_equals_templated_apply(table, L, bcneg):
    hops, acts = table
    lat = Lattice(L, bcneg, seed=sum(L) + bcneg)
    c0q, a_ii, b_ii = 0.23, 0.37, -0.61
    err = 0.0
    for s in range(lat.V):
        r = templated_apply(lat, s, c0q, a_ii, b_ii)
        t = table_apply(lat, s, hops, acts, c0q, a_ii, b_ii)
        err = max(err, np.abs(r - t).max() / np.abs(r).max())
    assert err < 1e-13, err
