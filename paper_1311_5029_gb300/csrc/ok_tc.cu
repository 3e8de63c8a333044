// Tensor-core application of M to several right-hand sides at once (the 12 spin-colour sources of
// a propagator), and the vector kernels of the lockstep multi-right-hand-side BiCGStab in the
// field layout that application reads.
//
// Spin projection.  With psi = (u, l) its upper and lower 2-spin halves, let h_+ = (u + l) / sqrt 2
// and h_- = (u - l) / sqrt 2.  The change of basis T / sqrt 2, T = [[1, 1], [1, -1]] (on u, l
// blocks), is orthogonal, so inner products are the same in both bases.  A hop W of Eq.
// minFlopForm acts on the projections as
//     out_a += sum_b Q_ab h_b(neighbour),   Q = T W T / 2,   a, b in {+, -},
// each Q_ab a 6x6 complex block (2 spins x 3 colours).  The spatial, two-hop and diagonal hops have
// W = [[D, S], [S, D]] and only Q_{++} = D + S and Q_{--} = D - S; the on-site and temporal terms
// have all four blocks.  The backward matrices of Eqs. conjugate and opp_diag_pre_mat,
// W^- = gamma5 W^{+ dagger} gamma5, become
//     Q^-_{++} = (Q^+_{--})^dag,  Q^-_{--} = (Q^+_{++})^dag,  Q^-_{+-} = -(Q^+_{+-})^dag,  Q^-_{-+} = -(Q^+_{-+})^dag
// of the forward blocks stored at the neighbour (gamma5 = [[0, -i], [i, 0]] maps h_+ to i h_- and
// h_- to -i h_+).
//
// The products.  For one site, one hop and one block, the right-hand sides times the block is a
// real-embedded complex GEMM, D (right-hand sides x 6 outputs) += H (right-hand sides x 6 inputs)
// Q^T, done as warp-level mma.sync.m16n8k16 with FP16 operands and FP32 accumulators:
//   M = 16 rows: right-hand side r in row r (up to 16 right-hand sides);
//   K = 16: input pair t = (spin 0, colour t) and pair t + 4 = (spin 1, colour t), re and im
//           interleaved (pairs 3 and 7 are zero);
//   N = 8 per tile: column o = (spin o & 1, colour o >> 1) of the output; the first tile holds the
//           real parts of the outputs, the second the imaginary parts, so that the sign pattern
//           of the real embedding is the same for every lane of a tile.
// A warp handles one site at a time.  A site is 60 block products (120 mma): on-site 4, temporal
// 2 x 4, spatial 6 x 2, two-hop 6 x 2, diagonal 12 x 2.
//
// Field layout (the solve's iteration vectors).  Unit (site, b, r, c) = (h_b spin 0, h_b spin 1) at
// colour c of right-hand side r, at unit index ((site * 2 + b) * nrhs + r) * 3 + c, 16 bytes in
// FP32.  The apply writes these units: they are exactly the accumulators a lane holds after the
// products.  It reads FP16 copies in the tile layout of in16_index below (the A operands as the
// products take them, one 16-byte load per lane and neighbour projection).
//
// Range of the FP16 inputs.  A residual shrinks by many orders of magnitude during a solve, below
// the FP16 range, so each right-hand side's FP16 input carries a power-of-two scale sigma_r (exact
// in binary): the solver's vector kernels write the FP16 copies of p and s as sigma_r x (value) with
// sigma_r |r| < 2^10 from the system's current |r|, and the apply multiplies its FP32 outputs by
// 1 / sigma_r.  The public entry scales each right-hand side by its largest component instead.
//
// W layout (OK_W_F16_TC).  Per site 804 words (FP16 complex, 3216 bytes): 22 blocks of 36 words,
// block word 4 e + k for colour entry e = 3 c + c' and spin entry k = 2 s + s' of
// Q[(s, c)][(s', c')]; then U_t / 2 (9 words).  A lane reads the two entries it needs of a forward
// block with one 8-byte load.
#include "ok_pair.cuh"

#include <cuda_fp16.h>

#include <atomic>

namespace okgb {
namespace tc {

constexpr int REC = 804;        // 32-bit words per site record
constexpr int BLKW = 36;        // words per block
constexpr int UHW = 22 * BLKW;  // U_t / 2, words [3 c + c']
enum : int {
  B_E = 0,     // on-site Q_{++} = Q_{--}
  B_F = 1,     // on-site Q_{+-} (Q_{-+} = -Q_{+-})
  B_TPP = 2,   // temporal forward Q_{++}  (Q_{+-} = Q_{-+} = (U_t / 2) x 1)
  B_TMM = 3,   // temporal forward Q_{--}
  B_SP = 4,    // spatial direction i: Q_{++} at 4 + 2 i, Q_{--} at 5 + 2 i
  B_II = 10,   // two-hop direction i: Q_{++} at 10 + 2 i, Q_{--} at 11 + 2 i
  B_VIJ = 16,  // diagonal pair p, offset +I +J: Q_{++} (Q_{--} = -Q_{++})
  B_XIJ = 19,  // diagonal pair p, offset +I -J: Q_{++} (Q_{--} = -Q_{++})
};
constexpr int TC_THREADS = 128;
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int MAX_RHS = 16;

// ---------------------------------------------------------------------------- W copy
__device__ __forceinline__ unsigned h2bits(cx<double> z) {
  const __half2 h = __halves2half2(__double2half(z.re), __double2half(z.im));
  return *reinterpret_cast<const unsigned*>(&h);
}

// Pauli matrix entries sigma_k[r][c].
__device__ __forceinline__ cx<double> pauli_e(int k, int r, int c) {
  if (k == 0) return mk<double>(r != c ? 1.0 : 0.0, 0.0);
  if (k == 1) return r == c ? mk<double>(0.0, 0.0) : mk<double>(0.0, r == 0 ? -1.0 : 1.0);
  return r != c ? mk<double>(0.0, 0.0) : mk<double>(r == 0 ? 1.0 : -1.0, 0.0);
}

// One thread per site: the blocks Q of every forward hop, from the FP64 stored matrices (the
// stored set keeps the factors 1/2 of the h+- basis of the FP32 kernels: the spatial P+- are
// (D +- S) / 2, the temporal S and U are halves, W^0 = 2 (Y+ + Y-) (+) 2i (Y+ - Y-) ...).
__global__ void tc_build_kernel(const cx<double>* __restrict__ W, Geom g, const WScalars* __restrict__ scp,
                                unsigned* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const WScalars sc = *scp;
  unsigned* o = out + (size_t)s * REC;
  const cx<double> zero = mk<double>(0.0, 0.0);
  // block `blk`, spin entry k: f * m
  auto put = [&](int blk, int k, const M3<double>& m, cx<double> f) {
    for (int e = 0; e < 9; ++e) o[blk * BLKW + 4 * e + k] = h2bits(f * m.e[e]);
  };
  const cx<double> one = mk<double>(1.0, 0.0), two = mk<double>(2.0, 0.0);
  // on-site: Y+- = [[a0 + c0, a1], [a2, c0 - a0]] (2x2 spin blocks of colour matrices);
  // W^0 = [[D', S'], [-S', D']], D' = 2 (Y+ + Y-), S' = -2i (Y+ - Y-); Q_{++} = Q_{--} = D', Q_{+-} = -S'.
  {
    const M3<double> c0 = m_rscale(sc.c0q, m_eye<double>());
    M3<double> yp[4], ym[4];
    const M3<double> a0 = wmat(W, s, M_Y0P), a1 = wmat(W, s, M_Y0P + 1), a2 = wmat(W, s, M_Y0P + 2);
    yp[0] = m_add(a0, c0); yp[1] = a1; yp[2] = a2; yp[3] = m_sub(c0, a0);
    const M3<double> b0 = wmat(W, s, M_Y0M), b1 = wmat(W, s, M_Y0M + 1), b2 = wmat(W, s, M_Y0M + 2);
    ym[0] = m_add(b0, c0); ym[1] = b1; ym[2] = b2; ym[3] = m_sub(c0, b0);
    for (int k = 0; k < 4; ++k) {
      put(B_E, k, m_add(yp[k], ym[k]), two);
      put(B_F, k, m_sub(yp[k], ym[k]), mk<double>(0.0, 2.0));
    }
  }
  // temporal: W^+_4 = [[0, 2S], [2S, -2 U]] (S = [[t0, t1], [t2, -t0]], U = U_t / 2 stored):
  // Q_{++} = 2S - U (x) 1, Q_{--} = -2S - U (x) 1, Q_{+-} = Q_{-+} = U (x) 1.
  {
    const M3<double> Uh = wmat(W, s, M_UT);
    const M3<double> t0 = wmat(W, s, M_ST), t1 = wmat(W, s, M_ST + 1), t2 = wmat(W, s, M_ST + 2);
    const M3<double> S[4] = {t0, t1, t2, m_rscale(-1.0, t0)};
    for (int k = 0; k < 4; ++k) {
      const bool diag = k == 0 || k == 3;
      put(B_TPP, k, diag ? m_sub(m_rscale(2.0, S[k]), Uh) : m_rscale(2.0, S[k]), one);
      put(B_TMM, k, diag ? m_sub(m_rscale(-2.0, S[k]), Uh) : m_rscale(-2.0, S[k]), one);
    }
    for (int e = 0; e < 9; ++e) o[UHW + e] = h2bits(Uh.e[e]);
    for (int e = 9; e < REC - UHW; ++e) o[UHW + e] = 0u;  // padding to a 16-byte record
  }
  // spatial: stored P+- = (D +- S) / 2, so Q_{++} = 2 P+, Q_{--} = 2 P-.
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) {
      put(B_SP + 2 * i, k, wmat(W, s, M_WP + 8 * i + k), two);
      put(B_SP + 2 * i + 1, k, wmat(W, s, M_WP + 8 * i + 4 + k), two);
    }
  // two-hop: Q_{+-+-} = 2 (a +- b sigma_i) (x) V_ii.
  for (int i = 0; i < 3; ++i) {
    const M3<double> V = wmat(W, s, M_VII + i);
    for (int k = 0; k < 4; ++k) {
      const int sr = k >> 1, scc = k & 1;
      const cx<double> a = mk<double>(sr == scc ? 2.0 * sc.a_ii : 0.0, 0.0);
      const cx<double> b = (2.0 * sc.b_ii) * pauli_e(i, sr, scc);
      put(B_II + 2 * i, k, V, a + b);
      put(B_II + 2 * i + 1, k, V, a - b);
    }
  }
  // diagonal pair (I, J): Q_{++} = 2 (sigma_I +- sigma_J) (x) X for the offsets +I +-J.
  for (int p = 0; p < 3; ++p) {
    const int I = p == 2 ? 1 : 0, J = p == 0 ? 1 : 2;
    const M3<double> Vij = wmat(W, s, M_VIJ + p), Xij = wmat(W, s, M_XIJ + p);
    for (int k = 0; k < 4; ++k) {
      const int sr = k >> 1, scc = k & 1;
      put(B_VIJ + p, k, Vij, two * (pauli_e(I, sr, scc) + pauli_e(J, sr, scc)));
      put(B_XIJ + p, k, Xij, two * (pauli_e(I, sr, scc) - pauli_e(J, sr, scc)));
    }
  }
  (void)zero;
}

// The dense forward 12x12 matrix of one kind, rebuilt from the copy: W = T Q T / 2 in (u, l)
// blocks, W_uu = (Q++ + Q+- + Q-+ + Q--) / 2, W_ul = (Q++ - Q+- + Q-+ - Q--) / 2,
// W_lu = (Q++ + Q+- - Q-+ - Q--) / 2, W_ll = (Q++ - Q+- - Q-+ + Q--) / 2.
// kind: 0 W^0; 1..4 W^+_mu; 5..7 W^{++}_ii; 8..10 W^{++}_ij; 11..13 W^{+-}_ij (as ok_W_expand).
__global__ void tc_expand_kernel(const unsigned* __restrict__ Wt, Geom g, int kind, cx<double>* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const unsigned* rec = Wt + (size_t)s * REC;
  // entry (s_r, c_r; s_c, c_c) of block blk times f
  auto q = [&](int blk, int sr, int cr, int scc, int cc) {
    const unsigned w = rec[blk * BLKW + 4 * (3 * cr + cc) + 2 * sr + scc];
    const __half2 h = *reinterpret_cast<const __half2*>(&w);
    return mk<double>((double)__low2float(h), (double)__high2float(h));
  };
  auto uh = [&](int sr, int cr, int scc, int cc) {
    if (sr != scc) return mk<double>(0.0, 0.0);
    const unsigned w = rec[UHW + 3 * cr + cc];
    const __half2 h = *reinterpret_cast<const __half2*>(&w);
    return mk<double>((double)__low2float(h), (double)__high2float(h));
  };
  const cx<double> zero = mk<double>(0.0, 0.0);
  for (int r = 0; r < 12; ++r)
    for (int c = 0; c < 12; ++c) {
      const int tr = r / 6, sr = (r % 6) / 3, cr = r % 3;  // (u or l, spin, colour) of the row
      const int tcb = c / 6, scc = (c % 6) / 3, ccc = c % 3;
      cx<double> pp = zero, pm = zero, mp = zero, mm = zero;
      if (kind == 0) {
        pp = q(B_E, sr, cr, scc, ccc); mm = pp;
        pm = q(B_F, sr, cr, scc, ccc); mp = -pm;
      } else if (kind <= 3) {
        pp = q(B_SP + 2 * (kind - 1), sr, cr, scc, ccc); mm = q(B_SP + 2 * (kind - 1) + 1, sr, cr, scc, ccc);
      } else if (kind == 4) {
        pp = q(B_TPP, sr, cr, scc, ccc); mm = q(B_TMM, sr, cr, scc, ccc);
        pm = uh(sr, cr, scc, ccc); mp = pm;
      } else if (kind <= 7) {
        pp = q(B_II + 2 * (kind - 5), sr, cr, scc, ccc); mm = q(B_II + 2 * (kind - 5) + 1, sr, cr, scc, ccc);
      } else {
        const int p = (kind - 8) % 3;
        pp = q((kind <= 10 ? B_VIJ : B_XIJ) + p, sr, cr, scc, ccc); mm = -pp;
      }
      const double su = tcb == 0 ? 1.0 : -1.0;    // T[., u] = 1, T[., l] = +-1 by the column's half
      const double sl = tr == 0 ? 1.0 : -1.0;     // row half
      // W_{tr,tc} = (1/2) sum_{a,b} T[tr][a] Q_ab T[b][tc]; T[u][a] = 1, T[l][+] = 1, T[l][-] = -1
      const cx<double> w = 0.5 * (pp + su * pm + sl * mp + (sl * su) * mm);
      out[(size_t)s * 144 + r * 12 + c] = w;
    }
}

// ---------------------------------------------------------------------------- the apply
struct AFrag { unsigned r[4]; };   // a0a1 (row g, pair t), a2a3 (row g + 8), a4a5 (pair t + 4), a6a7
struct BFrag { unsigned re0, re1, im0, im1; };

__device__ __forceinline__ unsigned pack_h2(float re, float im) {
  const __half2 h = __floats2half2_rn(re, im);
  return *reinterpret_cast<const unsigned*>(&h);
}
__device__ __forceinline__ unsigned swap_h(unsigned z) { return __byte_perm(z, 0u, 0x1032); }

__device__ __forceinline__ void mma16816(float (&d)[4], const AFrag& a, unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.r[0]), "r"(a.r[1]), "r"(a.r[2]), "r"(a.r[3]), "r"(b0), "r"(b1));
}

// acc[a][0] (real parts) and acc[a][1] (imaginary parts) += H Q^T for one block.
__device__ __forceinline__ void block_mma(float (&re)[4], float (&im)[4], const AFrag& h, const BFrag& q) {
  mma16816(re, h, q.re0, q.re1);
  mma16816(im, h, q.im0, q.im1);
}

// B fragment of a forward block from the two entries z0 = Q[(s, c)][(0, t)], z1 = Q[(s, c)][(1, t)]
// of this lane (real tile: (Re, -Im) per input pair; imaginary tile: (Im, Re)); sm flips the sign.
__device__ __forceinline__ BFrag bf_fwd(unsigned z0, unsigned z1, unsigned sm) {
  BFrag b;
  b.re0 = z0 ^ 0x80000000u ^ sm;
  b.re1 = z1 ^ 0x80000000u ^ sm;
  b.im0 = swap_h(z0) ^ sm;
  b.im1 = swap_h(z1) ^ sm;
  return b;
}
// B fragment of the adjoint of a block from w0 = Q[(0, t)][(s, c)], w1 = Q[(1, t)][(s, c)]:
// conj(w) enters, so the real tile takes (Re w, Im w) and the imaginary tile (-Im w, Re w).
__device__ __forceinline__ BFrag bf_bwd(unsigned w0, unsigned w1, unsigned sm) {
  BFrag b;
  b.re0 = w0 ^ sm;
  b.re1 = w1 ^ sm;
  b.im0 = swap_h(w0) ^ 0x00008000u ^ sm;
  b.im1 = swap_h(w1) ^ 0x00008000u ^ sm;
  return b;
}
__device__ __forceinline__ BFrag neg(BFrag b) {
  b.re0 ^= 0x80008000u; b.re1 ^= 0x80008000u; b.im0 ^= 0x80008000u; b.im1 ^= 0x80008000u;
  return b;
}

// Per-lane constants.
struct Lane {
  int g, t;            // groupID (lane >> 2), thread in group (lane & 3)
  bool wact;           // this lane holds W entries (output column g < 6, input colour t < 3)
  int off_f;           // forward: word offset of (Q[(s,c)][(0,t)], Q[(s,c)][(1,t)]) in a block
  int uh_f, uh_b;      // U_t / 2 entries [c][t] and [t][c]
  int s;               // output spin of this lane's column
  int a_off;           // offset 4 g + t of this lane's A-fragment word in a projection's tile
  int e_b;             // word offset of the adjoint entries' element 3 t + c in a block (4 words)
};

// FP16 input layout (the applied vectors, scaled): per (site, b) a 512-byte tile of 8 pairs x 4
// colour slots x 16 bytes; the word of pair p and colour c < 3 holds right-hand side p in its
// first 8 bytes and p + 8 in its last 8 (each: h_b spin 0, h_b spin 1).  Lane (g, t < 3) reads
// word 4 g + t, both of its rows in one 16-byte load, so a quarter-warp reads 96 bytes of one
// aligned 128-byte line (one L1 wavefront); the slots c = 3 (the zero K pairs) are never read,
// and absent right-hand sides are zero.
constexpr int IN16_TILE_U4 = 32;   // 16-byte words per (site, projection) tile
__host__ __device__ __forceinline__ size_t in16_index(int site, int b, int r, int c) {  // 8-byte units
  return ((((size_t)site * 2 + b) * IN16_TILE_U4) + 4 * (r & 7) + c) * 2 + (r >> 3);
}

// A fragments of the two projections of `site`.
__device__ __forceinline__ void load_h(const uint4* __restrict__ f, int site, const Lane& L, AFrag& hp, AFrag& hm) {
  const uint4* q = f + (size_t)site * (2 * IN16_TILE_U4) + L.a_off;
  uint4 u = make_uint4(0u, 0u, 0u, 0u), v = u;
  if (L.t < 3) {
    u = __ldg(q);
    v = __ldg(q + IN16_TILE_U4);
  }
  hp.r[0] = u.x; hp.r[2] = u.y; hp.r[1] = u.z; hp.r[3] = u.w;
  hm.r[0] = v.x; hm.r[2] = v.y; hm.r[1] = v.z; hm.r[3] = v.w;
}

// Loads of W words that do not allocate in L1: every W byte is used once per application, so L1
// is left to the neighbour tiles that several sites share.
__device__ __forceinline__ uint2 ldw2(const unsigned* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ldw4(const unsigned* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned ldw1(const unsigned* p) {
  unsigned v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Power-of-two scale sigma of a system's FP16 apply inputs: sigma |r| < 2^10 for |r|^2 = rr;
// 1 when rr is zero or not finite.
__device__ __forceinline__ float solve_scale(double rr) {
  if (!(rr > 0.0) || !isfinite(rr)) return 1.f;
  int e;
  frexp(sqrt(rr), &e);  // sqrt(rr) = m 2^e, 1/2 <= m < 1
  const int k = 10 - e;
  return ldexpf(1.f, k < -100 ? -100 : k > 100 ? 100 : k);
}

// FP16 pair of scaled values, clamped to the finite FP16 range.
__device__ __forceinline__ unsigned pack_scaled(float re, float im, float sc) {
  const float a = fminf(fmaxf(re * sc, -65504.f), 65504.f), b = fminf(fmaxf(im * sc, -65504.f), 65504.f);
  return pack_h2(a, b);
}

// The 27 hops of Eq. minFlopForm as a compile-time table.  Hop j has a displacement (mu, dmu)
// [+ (nu, dnu)] (mu < 0: on-site), reads its W at x (forward hops) or at the neighbour (backward
// hops), makes up to three distinct W loads (a block's lane entries, forward or for the adjoint, or
// U_t / 2) and uses them in up to four block products (input projection, output projection, sign).
enum : int { LK_NONE = 0, LK_FWD = 1, LK_BWD = 2, LK_UF = 3, LK_UB = 4 };
struct LoadDesc { int kind, blk; };
struct UseDesc { int load, in, out, neg; };   // load < 0: unused slot
struct HopDesc {
  int mu, dmu, nu, dnu;
  LoadDesc ld[3];
  UseDesc use[4];
};
constexpr int NHOP = 27;
__host__ __device__ constexpr HopDesc hop_desc(int j) {
  constexpr LoadDesc N0{LK_NONE, 0};
  constexpr UseDesc U0{-1, 0, 0, 0};
  if (j == 0)  // on-site: out+ = E h+ + F h-, out- = -F h+ + E h-
    return HopDesc{-1, 0, -1, 0, {{LK_FWD, B_E}, {LK_FWD, B_F}, N0}, {{0, 0, 0, 0}, {1, 1, 0, 0}, {1, 0, 1, 1}, {0, 1, 1, 0}}};
  if (j <= 6) {  // spatial i: forward (+1) Q++, Q-- at x; backward (-1) adjoints of Q--, Q++ at x - i
    const int i = (j - 1) / 2;
    if ((j - 1) % 2 == 0)
      return HopDesc{i, 1, -1, 0, {{LK_FWD, B_SP + 2 * i}, {LK_FWD, B_SP + 2 * i + 1}, N0}, {{0, 0, 0, 0}, {1, 1, 1, 0}, U0, U0}};
    return HopDesc{i, -1, -1, 0, {{LK_BWD, B_SP + 2 * i + 1}, {LK_BWD, B_SP + 2 * i}, N0}, {{0, 0, 0, 0}, {1, 1, 1, 0}, U0, U0}};
  }
  if (j == 7)  // temporal forward: Q++, Q--, Q+- = Q-+ = U_t / 2 (x) 1
    return HopDesc{3, 1, -1, 0, {{LK_FWD, B_TPP}, {LK_FWD, B_TMM}, {LK_UF, 0}}, {{0, 0, 0, 0}, {2, 1, 0, 0}, {2, 0, 1, 0}, {1, 1, 1, 0}}};
  if (j == 8)  // temporal backward: (Q--)^dag, (Q++)^dag, Q+- = Q-+ = -(U_t / 2)^dag x 1
    return HopDesc{3, -1, -1, 0, {{LK_BWD, B_TMM}, {LK_BWD, B_TPP}, {LK_UB, 0}}, {{0, 0, 0, 0}, {2, 1, 0, 1}, {2, 0, 1, 1}, {1, 1, 1, 0}}};
  if (j <= 14) {  // two-hop i
    const int i = (j - 9) / 2;
    if ((j - 9) % 2 == 0)
      return HopDesc{i, 2, -1, 0, {{LK_FWD, B_II + 2 * i}, {LK_FWD, B_II + 2 * i + 1}, N0}, {{0, 0, 0, 0}, {1, 1, 1, 0}, U0, U0}};
    return HopDesc{i, -2, -1, 0, {{LK_BWD, B_II + 2 * i + 1}, {LK_BWD, B_II + 2 * i}, N0}, {{0, 0, 0, 0}, {1, 1, 1, 0}, U0, U0}};
  }
  // diagonal pair p = (I, J): +I+J (V block), -I-J, +I-J (X block), -I+J; Q-- = -Q++, and the
  // backward hops use (Q^-)++ = -(Q++)^dag, (Q^-)-- = (Q++)^dag
  const int p = (j - 15) / 4, q = (j - 15) % 4;
  const int I = p == 2 ? 1 : 0, J = p == 0 ? 1 : 2;
  const int blk = (q < 2 ? B_VIJ : B_XIJ) + p;
  const int sJ = q < 2 ? 1 : -1;
  if (q % 2 == 0)
    return HopDesc{I, 1, J, sJ, {{LK_FWD, blk}, N0, N0}, {{0, 0, 0, 0}, {0, 1, 1, 1}, U0, U0}};
  return HopDesc{I, -1, J, -sJ, {{LK_BWD, blk}, N0, N0}, {{0, 0, 0, 1}, {0, 1, 1, 0}, U0, U0}};
}

// Displacements of the 27 hops packed for a constant-memory table: 4 bits per coordinate (x, y, z,
// t), two's complement.
__host__ __device__ constexpr unsigned hop_disp(int j) {
  const HopDesc d = hop_desc(j);
  int v[4] = {0, 0, 0, 0};
  if (d.mu >= 0) v[d.mu] += d.dmu;
  if (d.nu >= 0) v[d.nu] += d.dnu;
  return (unsigned)(v[0] & 15) | ((unsigned)(v[1] & 15) << 4) | ((unsigned)(v[2] & 15) << 8) | ((unsigned)(v[3] & 15) << 12);
}
struct HopDisp { unsigned d[32]; };
__host__ __device__ constexpr HopDisp make_hop_disp() {
  HopDisp t{};
  for (int j = 0; j < 32; ++j) t.d[j] = j < NHOP ? hop_disp(j) : 0u;
  return t;
}
__constant__ HopDisp k_hop_disp = make_hop_disp();

// Neighbour code of hop `lane` (lanes 0..26, in parallel): (neighbour site << 1) | 1 when the hop
// crosses an antiperiodic boundary an odd number of times.
__device__ __forceinline__ int nbr_code(int lane, int x, const Geom& g) {
  const unsigned w = k_hop_disp.d[lane & 31];
  int r = x, idx = 0, neg = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int L = g.L[mu];
    const int cm = mu < 3 ? r % L : r;
    if (mu < 3) r /= L;
    const int d = ((int)(w << (28 - 4 * mu))) >> 28;   // sign-extended 4-bit field
    int xm = cm + d, wraps = 0;
    if (xm >= L) { xm -= L; ++wraps; if (xm >= L) { xm -= L; ++wraps; } }
    if (xm < 0) { xm += L; ++wraps; if (xm < 0) { xm += L; ++wraps; } }
    neg ^= ((g.bcneg >> mu) & 1) & wraps;
    idx += xm * g.S[mu];
  }
  return (idx << 1) | neg;
}

struct Acc { float v[2][2][4]; };   // [output projection a][real, imaginary tile][c0..c3]

// What one hop has loaded: the neighbour's A fragments, up to three raw W word pairs, the sign.
struct HopRaw {
  AFrag hp, hm;
  unsigned w[3][2];
  unsigned sm;
};

struct Ctx {
  const uint4* __restrict__ in;
  const unsigned* __restrict__ W;
  int x;      // the site
  int code;   // this lane's neighbour code (nbr_code)
  Lane L;
};

// AP: the lattice has an antiperiodic direction (else every boundary sign is +1).
template <int J, bool AP>
__device__ __forceinline__ void hop_load(const Ctx& C, HopRaw& R) {
  constexpr HopDesc d = hop_desc(J);
  int n = C.x;
  R.sm = 0u;
  if constexpr (d.mu >= 0) {
    const int code = __shfl_sync(0xffffffffu, C.code, J);
    n = code >> 1;
    if constexpr (AP) R.sm = (code & 1) ? 0x80008000u : 0u;
  }
  load_h(C.in, n, C.L, R.hp, R.hm);
  constexpr bool at_nbr = d.ld[0].kind == LK_BWD;
  const unsigned* rec = C.W + (size_t)(at_nbr ? n : C.x) * REC;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R.w[k][0] = R.w[k][1] = 0u;
    const int kind = d.ld[k].kind, blk = d.ld[k].blk;
    if (kind == LK_NONE || !C.L.wact) continue;
    if (kind == LK_FWD) {
      const uint2 z = ldw2(rec + blk * BLKW + C.L.off_f);
      R.w[k][0] = z.x;
      R.w[k][1] = z.y;
    } else if (kind == LK_BWD) {
      // the four spin entries of element 3 t + c; this lane takes k = s and k = 2 + s
      const uint4 z = ldw4(rec + blk * BLKW + C.L.e_b);
      R.w[k][0] = C.L.s ? z.y : z.x;
      R.w[k][1] = C.L.s ? z.w : z.z;
    } else {
      const unsigned u = ldw1(rec + UHW + (kind == LK_UF ? C.L.uh_f : C.L.uh_b));
      R.w[k][0] = C.L.s ? 0u : u;   // (U_t / 2) x 1 is diagonal in spin
      R.w[k][1] = C.L.s ? u : 0u;
    }
  }
}

template <int J, bool AP>
__device__ __forceinline__ void hop_compute(const HopRaw& R, Acc& A) {
  constexpr HopDesc d = hop_desc(J);
  const unsigned sm0 = AP ? R.sm : 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const UseDesc u = d.use[k];
    if (u.load < 0) continue;
    const int kind = d.ld[u.load].kind;
    const unsigned sm = sm0 ^ (u.neg ? 0x80008000u : 0u);
    const BFrag q = (kind == LK_FWD || kind == LK_UF) ? bf_fwd(R.w[u.load][0], R.w[u.load][1], sm)
                                                      : bf_bwd(R.w[u.load][0], R.w[u.load][1], sm);
    block_mma(A.v[u.out][0], A.v[u.out][1], u.in ? R.hm : R.hp, q);
  }
}

// Software pipeline over the hop sequence, which runs on from one site of a warp into the next:
// the loads of hop j + 2 are issued before the products of hop j (for j + 2 >= 27, hop j - 25 of the
// warp's next site), so three hops' loads are in flight per warp and a site starts with its first
// hops already loaded.  Three register slots divide the 27 hops, so a hop's slot is a constant.
constexpr int TC_SLOTS = 3;
static_assert(NHOP % TC_SLOTS == 0, "hop slots must divide the hop count");
template <int J, bool AP>
__device__ __forceinline__ void pipe(const Ctx& C, const Ctx& Cn, bool more, HopRaw (&R)[TC_SLOTS], Acc& A) {
  if constexpr (J < NHOP) {
    constexpr int JJ = J + TC_SLOTS - 1;
    if constexpr (JJ < NHOP) hop_load<JJ, AP>(C, R[JJ % TC_SLOTS]);
    else if (more) hop_load<JJ - NHOP, AP>(Cn, R[JJ % TC_SLOTS]);
    hop_compute<J, AP>(R[J % TC_SLOTS], A);
    pipe<J + 1, AP>(C, Cn, more, R, A);
  }
}

// The last block of a launch sums each live right-hand side's partials and finalises its state; the
// right-hand sides are spread over the warps (warp w takes w, w + 4, ...), each summed by its warp's
// lanes in a fixed order and a fixed shuffle tree.
template <int NP>
__device__ __forceinline__ void multi_finish(double (*bsum)[3], const bool* live, int nrhs, const TcEpi& ep) {
  __shared__ int last;
  if (threadIdx.x < nrhs) {
#pragma unroll
    for (int k = 0; k < NP; ++k) ep.part[(size_t)threadIdx.x * ep.pstride + (size_t)blockIdx.x * NP + k] = bsum[threadIdx.x][k];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ep.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const unsigned G = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < nrhs; r += TC_WARPS) {
    if (!live[r]) continue;
    const double* pr = ep.part + (size_t)r * ep.pstride;
    double w[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) w[k] = 0.0;
    for (unsigned b = lane; b < G; b += 32)
#pragma unroll
      for (int k = 0; k < NP; ++k) w[k] += __ldcg(pr + (size_t)b * NP + k);
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
    if (lane == 0) {
      double tot[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < NP; ++k) tot[k] = w[k];
      finalise(ep.st + r, ep.fin, tot);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *ep.ticket = 0u;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Launch bounds: blocks per SM (4: 128 registers, 16 warps); L2 bulk prefetch of the next site's
// record on (1) or off (0).
#ifndef OK_TC_MINB
#define OK_TC_MINB 4
#endif
#ifndef OK_TC_PF
#define OK_TC_PF 1
#endif
// Bulk prefetch of a site's W record (3216 bytes, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_rec(const unsigned* p) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "n"(REC * 4) : "memory");
}

template <int EPI, bool AP>
__global__ void __launch_bounds__(TC_THREADS, OK_TC_MINB) apply_tc_kernel(const unsigned* __restrict__ W, const uint4* __restrict__ in,
                                                                 float4* __restrict__ out, Geom g, int nrhs, TcEpi ep) {
  constexpr bool RED = EPI == EPI_DOT || EPI == EPI_TS;
  __shared__ bool live[MAX_RHS];
  __shared__ double bsum[MAX_RHS][3];
  __shared__ float wsum[TC_WARPS][MAX_RHS][3];
  // the epilogue's operand units of the current site, copied in while its hops run
  __shared__ __align__(16) float4 ybuf[RED ? TC_WARPS : 1][4][32];

  if (RED) {
    if (threadIdx.x < MAX_RHS) live[threadIdx.x] = threadIdx.x < nrhs && ep.st[threadIdx.x].halt == HALT_NONE;
    __syncthreads();
    bool any = false;
    for (int r = 0; r < nrhs; ++r) any = any || live[r];
    if (!any) return;  // every system has halted: nothing to do (uniform over the grid)
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Lane L;
  L.g = lane >> 2;
  L.t = lane & 3;
  L.s = L.g & 1;
  L.wact = L.g < 6 && L.t < 3;
  const int cc = L.g >> 1;
  L.off_f = 4 * (3 * cc + L.t) + 2 * L.s;
  L.uh_f = 3 * cc + L.t;
  L.uh_b = 3 * L.t + cc;
  L.a_off = 4 * L.g + L.t;
  L.e_b = 4 * (3 * L.t + cc);
  // 1 / sigma of the right-hand sides of this lane's rows (g and g + 8)
  float inv[2] = {1.f, 1.f};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = L.g + 8 * h;
    if (r < nrhs) inv[h] = ep.inv_scale ? ep.inv_scale[r] : (ep.st ? 1.f / solve_scale(ep.st[r].rr) : 1.f);
  }
  float red[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // right-hand sides g and g + 8
  // All warps sweep the lattice together, a band of gridDim.x * TC_WARPS consecutive sites at a time,
  // so that a neighbour's tile is read again from L2 before it leaves.  With a grid of whole waves
  // (k blocks on each of S multiprocessors, placed round robin) the k blocks of one multiprocessor
  // take adjacent ranks, so its warps work on consecutive sites and share their x neighbours in L1.
  const int G = gridDim.x, S = g.sms;
  const int rank = (S > 0 && G % S == 0) ? (blockIdx.x % S) * (G / S) + blockIdx.x / S : blockIdx.x;
  const int nw = G * TC_WARPS;
  int x = rank * TC_WARPS + warp;
  if (x < g.V) {
    Ctx C{in, W, x, nbr_code(lane, x, g), L};
    HopRaw R[TC_SLOTS];
    hop_load<0, AP>(C, R[0]);
    hop_load<1, AP>(C, R[1]);
    for (;;) {
      const int xn = x + nw;
      const bool more = xn < g.V;
      const Ctx Cn{in, W, more ? xn : x, more ? nbr_code(lane, xn, g) : C.code, L};
      // the next site's own W record is read from DRAM once, block by block over its hops: have it
      // in L2 before they start
      if (OK_TC_PF && more && lane == 0) prefetch_rec(W + (size_t)xn * REC);
      if constexpr (RED) {
        // copy this site's epilogue operand units (FP32) into shared memory while the hops run
        if (L.t < 3) {
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = L.g + 8 * h;
              if (r < nrhs) {
                const float4* src = ep.y + ((size_t)x * 2 + a) * nrhs * 3 + r * 3 + L.t;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(&ybuf[warp][2 * a + h][lane])),
                             "l"(src)
                             : "memory");
              }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      Acc A;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int k = 0; k < 4; ++k) A.v[a][p][k] = 0.f;
      pipe<0, AP>(C, Cn, more, R, A);
      if constexpr (RED) asm volatile("cp.async.wait_all;" ::: "memory");
      if (L.t < 3) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const size_t row = ((size_t)x * 2 + a) * nrhs * 3;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = L.g + 8 * h;
            if (r >= nrhs) continue;
            const float f = inv[h];
            const float4 o = make_float4(A.v[a][0][2 * h] * f, A.v[a][1][2 * h] * f, A.v[a][0][2 * h + 1] * f,
                                         A.v[a][1][2 * h + 1] * f);
            out[row + r * 3 + L.t] = o;
            if constexpr (RED) {
              const float4 y = ybuf[warp][2 * a + h][lane];
              if (EPI == EPI_DOT) {  // conj(y) o
                red[h][0] += y.x * o.x + y.y * o.y + y.z * o.z + y.w * o.w;
                red[h][1] += y.x * o.y - y.y * o.x + y.z * o.w - y.w * o.z;
              } else {               // conj(o) y, |o|^2
                red[h][0] += o.x * y.x + o.y * y.y + o.z * y.z + o.w * y.w;
                red[h][1] += o.x * y.y - o.y * y.x + o.z * y.w - o.w * y.z;
                red[h][2] += o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
              }
            }
          }
        }
      }
      if (!more) break;
      x = xn;
      C = Cn;
    }
  }
  if constexpr (RED) {
    constexpr int NP = EPI == EPI_DOT ? 2 : 3;
    // lanes of one group (same g) hold the same right-hand sides: sum over t
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float v = red[h][k];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        red[h][k] = v;
      }
    if (L.t == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = L.g + 8 * h;
#pragma unroll
        for (int k = 0; k < NP; ++k) wsum[warp][r][k] = red[h][k];
      }
    }
    __syncthreads();
    if (threadIdx.x < nrhs) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        double v = 0.0;
        for (int w = 0; w < TC_WARPS; ++w) v += (double)wsum[w][threadIdx.x][k];
        bsum[threadIdx.x][k] = v;
      }
    }
    __syncthreads();
    multi_finish<NP>(bsum, live, nrhs, ep);
  }
}

// ---------------------------------------------------------------------------- layout conversions
// canonical complex64 [nrhs][V][4][3] -> the tensor-core layout (projections h_+-, FP16, scaled by a
// power of two per right-hand side that puts its largest |h| below 2^15), and FP32 tensor-core
// layout -> canonical.
constexpr float RSQRT2F = 0.70710678118654752f;

// Largest |re|, |im| of each right-hand side (grid row y = right-hand side), as float bits.
__global__ void tc_amax_kernel(const float4* __restrict__ in, long long n4, unsigned* __restrict__ amax) {
  const float4* p = in + (size_t)blockIdx.y * n4;
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = p[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax + blockIdx.y, __float_as_uint(m));
}

// sigma = 2^(14 - e) for a largest component m 2^e (1/2 <= m < 1): |h| <= sqrt 2 max < 2^15.
__device__ __forceinline__ float max_scale(unsigned bits) {
  const float mx = __uint_as_float(bits);
  if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
  int e;
  frexpf(mx, &e);
  const int k = 14 - e;
  return ldexpf(1.f, k < -100 ? -100 : k > 100 ? 100 : k);
}

__global__ void canon_to_tc16_kernel(const float2* __restrict__ in, uint2* __restrict__ out, int V, int nrhs,
                                     const unsigned* __restrict__ amax, float* __restrict__ inv_scale) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < nrhs) inv_scale[i] = 1.f / max_scale(amax[i]);
  if (i >= 3LL * V * nrhs) return;
  const int c = (int)(i % 3);
  const long long rs = i / 3;
  const int site = (int)(rs % V), r = (int)(rs / V);
  const float sc = max_scale(amax[r]) * RSQRT2F;
  const float2* p = in + ((size_t)r * V + site) * 12;
  const float2 u0 = p[c], u1 = p[3 + c], l0 = p[6 + c], l1 = p[9 + c];
  out[in16_index(site, 0, r, c)] = make_uint2(pack_scaled(u0.x + l0.x, u0.y + l0.y, sc), pack_scaled(u1.x + l1.x, u1.y + l1.y, sc));
  out[in16_index(site, 1, r, c)] = make_uint2(pack_scaled(u0.x - l0.x, u0.y - l0.y, sc), pack_scaled(u1.x - l1.x, u1.y - l1.y, sc));
}

__global__ void tc_to_canon_kernel(const float4* __restrict__ in, float2* __restrict__ out, int V, int nrhs) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 3LL * V * nrhs) return;
  const int c = (int)(i % 3);
  const long long rs = i / 3;
  const int site = (int)(rs % V), r = (int)(rs / V);
  const size_t base = (size_t)site * 2 * nrhs * 3;
  const float4 hp = in[base + (size_t)r * 3 + c], hm = in[base + ((size_t)nrhs + r) * 3 + c];
  float2* p = out + ((size_t)r * V + site) * 12;
  p[c] = make_float2((hp.x + hm.x) * RSQRT2F, (hp.y + hm.y) * RSQRT2F);
  p[3 + c] = make_float2((hp.z + hm.z) * RSQRT2F, (hp.w + hm.w) * RSQRT2F);
  p[6 + c] = make_float2((hp.x - hm.x) * RSQRT2F, (hp.y - hm.y) * RSQRT2F);
  p[9 + c] = make_float2((hp.z - hm.z) * RSQRT2F, (hp.w - hm.w) * RSQRT2F);
}

// ---------------------------------------------------------------------------- solver vectors
// Vector kernels of the lockstep solve on the tensor-core layout.  A block is (3 nrhs) x Y
// threads: threadIdx.x = 3 r + c is one unit of a (site, projection) row, so every thread works on
// one right-hand side r throughout and reads that system's scalars.  Rows are 2 V.
constexpr int VEC_TARGET = 256;
constexpr int TC_RED_CHUNK = 8;

__device__ __forceinline__ void sys_scalars(const SolverState* st, int r, dcx& al, dcx& om, dcx& be, int& halt) {
  al = st[r].alpha;
  om = st[r].omega;
  be = st[r].beta;
  halt = st[r].halt;
}

// s = r - alpha v, and its FP16 copy sigma s for the apply
__global__ void tc_update_s_kernel(const float4* __restrict__ rv, const float4* __restrict__ v, float4* __restrict__ s,
                                   uint2* __restrict__ s16, int rows, int nrhs, const SolverState* __restrict__ st) {
  const int r = threadIdx.x / 3;
  dcx al, om, be;
  int halt;
  sys_scalars(st, r, al, om, be, halt);
  if (halt) return;
  const float ar = (float)al.re, ai = (float)al.im;
  const float sc = solve_scale(st[r].rr);
  const int L = 3 * nrhs;
  for (long long row = blockIdx.x * (long long)blockDim.y + threadIdx.y; row < rows; row += (long long)gridDim.x * blockDim.y) {
    const size_t i = (size_t)row * L + threadIdx.x;
    const float4 a = rv[i], b = v[i];
    const float4 o = make_float4(a.x - (ar * b.x - ai * b.y), a.y - (ar * b.y + ai * b.x), a.z - (ar * b.z - ai * b.w),
                                 a.w - (ar * b.w + ai * b.z));
    s[i] = o;
    s16[in16_index((int)(row >> 1), (int)(row & 1), r, threadIdx.x - 3 * r)] =
        make_uint2(pack_scaled(o.x, o.y, sc), pack_scaled(o.z, o.w, sc));
  }
}

// p = r + beta (p - omega v) and its FP16 copy sigma p; only >= 0: that system alone (the others
// untouched)
__global__ void tc_update_p_kernel(float4* __restrict__ p, uint2* __restrict__ p16, const float4* __restrict__ rv,
                                   const float4* __restrict__ v, int rows, int nrhs, const SolverState* __restrict__ st,
                                   int only) {
  const int r = threadIdx.x / 3;
  dcx al, om, be;
  int halt;
  sys_scalars(st, r, al, om, be, halt);
  if (halt || (only >= 0 && r != only)) return;
  const cx<float> B = mk<float>((float)be.re, (float)be.im), O = mk<float>((float)om.re, (float)om.im);
  const float sc = solve_scale(st[r].rr);
  const int L = 3 * nrhs;
  for (long long row = blockIdx.x * (long long)blockDim.y + threadIdx.y; row < rows; row += (long long)gridDim.x * blockDim.y) {
    const size_t i = (size_t)row * L + threadIdx.x;
    const float4 pp = p[i], rr = rv[i], vv = v[i];
    const cx<float> p0 = mk(pp.x, pp.y) - O * mk(vv.x, vv.y), p1 = mk(pp.z, pp.w) - O * mk(vv.z, vv.w);
    const cx<float> q0 = mk(rr.x, rr.y) + B * p0, q1 = mk(rr.z, rr.w) + B * p1;
    p[i] = make_float4(q0.re, q0.im, q1.re, q1.im);
    p16[in16_index((int)(row >> 1), (int)(row & 1), r, threadIdx.x - 3 * r)] =
        make_uint2(pack_scaled(q0.re, q0.im, sc), pack_scaled(q1.re, q1.im, sc));
  }
}

// FP16 copy sigma p of p for live systems (only >= 0: that system alone), after a restart.
__global__ void tc_half_kernel(const float4* __restrict__ p, uint2* __restrict__ p16, int rows, int nrhs,
                               const SolverState* __restrict__ st, int only) {
  const int r = threadIdx.x / 3;
  if (st[r].halt || (only >= 0 && r != only)) return;
  const float sc = solve_scale(st[r].rr);
  const int L = 3 * nrhs;
  for (long long row = blockIdx.x * (long long)blockDim.y + threadIdx.y; row < rows; row += (long long)gridDim.x * blockDim.y) {
    const size_t i = (size_t)row * L + threadIdx.x;
    const float4 q = p[i];
    p16[in16_index((int)(row >> 1), (int)(row & 1), r, threadIdx.x - 3 * r)] =
        make_uint2(pack_scaled(q.x, q.y, sc), pack_scaled(q.z, q.w, sc));
  }
}

// Per-block sums of each right-hand side (threads of one system: x in [3 r, 3 r + 3), every y).
template <int NP>
__device__ __forceinline__ void vec_block_sums(const double (&red)[NP], double (*bsum)[3], int nrhs) {
  __shared__ double sh[NP][VEC_TARGET + 64];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int k = 0; k < NP; ++k) sh[k][tid] = red[k];
  __syncthreads();
  if (tid < nrhs) {
    const int r = tid;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      double v = 0.0;
      for (int y = 0; y < (int)blockDim.y; ++y)
        for (int u = 0; u < 3; ++u) v += sh[k][y * blockDim.x + 3 * r + u];
      bsum[r][k] = v;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float4 unpack_scaled(uint2 u, float inv) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x * inv, a.y * inv, b.x * inv, b.y * inv);
}

// x += alpha p~ + omega s~;  r = s - omega t;  per system <rhat, r>, <r, r> -> FIN_XR.  p~ and s~ are
// the FP16 copies the applies multiplied (v = M p~, t = M s~), unscaled: so the solution moves by
// exactly the vectors whose images updated the residual, and the iterated residual keeps tracking
// b - M x (up to the rounding of W and of the FP32 accumulation).
__global__ void tc_update_xr_kernel(float4* __restrict__ x, const uint2* __restrict__ p16, const float4* __restrict__ s,
                                    const uint2* __restrict__ s16, const float4* __restrict__ t, float4* __restrict__ rv,
                                    const float4* __restrict__ rhat, int rows, int nrhs, SolverState* __restrict__ st,
                                    TcEpi ep) {
  __shared__ bool live[MAX_RHS];
  __shared__ double bsum[MAX_RHS][3];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid < MAX_RHS) live[tid] = tid < nrhs && st[tid].halt == HALT_NONE;
  __syncthreads();
  bool any = false;
  for (int k = 0; k < nrhs; ++k) any = any || live[k];
  if (!any) return;
  const int r = threadIdx.x / 3;
  double red[3] = {0.0, 0.0, 0.0};
  if (live[r]) {
    const cx<float> al = mk<float>((float)st[r].alpha.re, (float)st[r].alpha.im);
    const cx<float> om = mk<float>((float)st[r].omega.re, (float)st[r].omega.im);
    const float inv = 1.f / solve_scale(st[r].rr);
    const int L = 3 * nrhs;
    // FP32 sums over a chunk of TC_RED_CHUNK rows, added into the FP64 totals once per chunk (FP64
    // arithmetic runs at a small fraction of the FP32 rate)
    const long long gs = (long long)gridDim.x * blockDim.y;
    for (long long row0 = blockIdx.x * (long long)blockDim.y + threadIdx.y; row0 < rows; row0 += gs * TC_RED_CHUNK) {
    float c3[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < TC_RED_CHUNK; ++u) {
      const long long row = row0 + u * gs;
      if (row >= rows) break;
      const size_t i = (size_t)row * L + threadIdx.x;
      const float4 xv = x[i], sv = s[i], tv = t[i], hv = rhat[i];
      const size_t j = in16_index((int)(row >> 1), (int)(row & 1), r, threadIdx.x - 3 * r);
      const float4 pv = unpack_scaled(p16[j], inv), qv = unpack_scaled(s16[j], inv);
      cx<float> x0 = mk(xv.x, xv.y) + al * mk(pv.x, pv.y) + om * mk(qv.x, qv.y);
      cx<float> x1 = mk(xv.z, xv.w) + al * mk(pv.z, pv.w) + om * mk(qv.z, qv.w);
      const cx<float> r0 = mk(sv.x, sv.y) - om * mk(tv.x, tv.y), r1 = mk(sv.z, sv.w) - om * mk(tv.z, tv.w);
      x[i] = make_float4(x0.re, x0.im, x1.re, x1.im);
      rv[i] = make_float4(r0.re, r0.im, r1.re, r1.im);
      cx<float> d = fma_cj(mk(hv.x, hv.y), r0, mk<float>(0.f, 0.f));
      d = fma_cj(mk(hv.z, hv.w), r1, d);
      c3[0] += d.re;
      c3[1] += d.im;
      c3[2] += (r0.re * r0.re + r0.im * r0.im) + (r1.re * r1.re + r1.im * r1.im);
    }
    red[0] += c3[0];
    red[1] += c3[1];
    red[2] += c3[2];
    }
  }
  vec_block_sums<3>(red, bsum, nrhs);
  // the completion logic of the apply, over this block's threads
  __shared__ int last;
  if (tid < nrhs) {
#pragma unroll
    for (int k = 0; k < 3; ++k) ep.part[(size_t)tid * ep.pstride + (size_t)blockIdx.x * 3 + k] = bsum[tid][k];
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(ep.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int T = blockDim.x * blockDim.y;
  __shared__ double sh2[3][VEC_TARGET + 64];
  for (int q = 0; q < nrhs; ++q) {
    if (!live[q]) continue;
    double w[3] = {0.0, 0.0, 0.0};
    const double* pr = ep.part + (size_t)q * ep.pstride;
    for (unsigned b = tid; b < gridDim.x; b += T)
#pragma unroll
      for (int k = 0; k < 3; ++k) w[k] += __ldcg(pr + (size_t)b * 3 + k);
#pragma unroll
    for (int k = 0; k < 3; ++k) sh2[k][tid] = w[k];
    __syncthreads();
    // fixed tree: the first warp sums a strided share each, then a shuffle tree (T >= 32)
    if (tid < 32) {
      double v[3] = {0.0, 0.0, 0.0};
      for (int u = tid; u < T; u += 32)
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] += sh2[k][u];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
      if (tid == 0) {
        double tot[4] = {v[0], v[1], v[2], 0.0};
        finalise(st + q, FIN_XR, tot);
      }
    }
    __syncthreads();
  }
  if (tid == 0) *ep.ticket = 0u;
}

// Mixed precision, system k: r = (h projections of) r64 rounded to FP32; RESTART: rhat = p = r and
// FIN_RESTART on <r, r>; otherwise FIN_CONTINUE on <rhat, r>, <r, r>.  One thread per (site, colour).
template <bool RESTART>
__global__ void __launch_bounds__(256) tc_demote_kernel(const double2* __restrict__ r64, float4* __restrict__ rv,
                                                        float4* __restrict__ rhat, float4* __restrict__ p, int V, int nrhs,
                                                        int k, SolverState* __restrict__ st, RedArgs ra) {
  double red[3] = {0.0, 0.0, 0.0};
  const double s2 = 0.70710678118654752440;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3LL * V; i += (long long)gridDim.x * blockDim.x) {
    const int site = (int)(i / 3), c = (int)(i % 3);
    const double2* q = r64 + (size_t)site * 12;
    const double2 u0 = q[c], u1 = q[3 + c], l0 = q[6 + c], l1 = q[9 + c];
    const size_t base = (size_t)site * 2 * nrhs * 3;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const double sg = b ? -1.0 : 1.0;
      const float4 f = make_float4((float)((u0.x + sg * l0.x) * s2), (float)((u0.y + sg * l0.y) * s2),
                                   (float)((u1.x + sg * l1.x) * s2), (float)((u1.y + sg * l1.y) * s2));
      const size_t j = base + ((size_t)b * nrhs + k) * 3 + c;
      rv[j] = f;
      if (RESTART) {
        rhat[j] = f;
        p[j] = f;
        red[0] += (double)f.x * f.x + (double)f.y * f.y + (double)f.z * f.z + (double)f.w * f.w;
      } else {
        const float4 h = rhat[j];
        red[0] += (double)h.x * f.x + (double)h.y * f.y + (double)h.z * f.z + (double)h.w * f.w;
        red[1] += (double)h.x * f.y - (double)h.y * f.x + (double)h.z * f.w - (double)h.w * f.z;
        red[2] += (double)f.x * f.x + (double)f.y * f.y + (double)f.z * f.z + (double)f.w * f.w;
      }
    }
  }
  if (RESTART) {
    double v1[1] = {red[0]};
    grid_reduce<1, 256>(v1, ra, &st->ticket[4]);
  } else {
    grid_reduce<3, 256>(red, ra, &st->ticket[4]);
  }
}

// Mixed precision, system k: x64 += x (back from the projections), x = 0.
__global__ void __launch_bounds__(256) tc_accum_kernel(double2* __restrict__ x64, float4* __restrict__ x, int V, int nrhs, int k) {
  const double s2 = 0.70710678118654752440;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3LL * V; i += (long long)gridDim.x * blockDim.x) {
    const int site = (int)(i / 3), c = (int)(i % 3);
    const size_t base = (size_t)site * 2 * nrhs * 3;
    const size_t jp = base + (size_t)k * 3 + c, jm = base + ((size_t)nrhs + k) * 3 + c;
    const float4 hp = x[jp], hm = x[jm];
    double2* q = x64 + (size_t)site * 12;
    q[c].x += ((double)hp.x + hm.x) * s2;  q[c].y += ((double)hp.y + hm.y) * s2;
    q[3 + c].x += ((double)hp.z + hm.z) * s2;  q[3 + c].y += ((double)hp.w + hm.w) * s2;
    q[6 + c].x += ((double)hp.x - hm.x) * s2;  q[6 + c].y += ((double)hp.y - hm.y) * s2;
    q[9 + c].x += ((double)hp.z - hm.z) * s2;  q[9 + c].y += ((double)hp.w - hm.w) * s2;
    x[jp] = make_float4(0.f, 0.f, 0.f, 0.f);
    x[jm] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------- host side
int launch_tc_build(const ok_W* W, const cx<double>* W64, const WScalars* dsc, cudaStream_t st) {
  if (!W || !W64 || !W->Wtc) return OK_EINVAL;
  {
    TraceScope ts("tc_build", st);
    tc::tc_build_kernel<<<grid_for(W->g.V, 128), 128, 0, st>>>(W64, W->g, dsc, (unsigned*)W->Wtc);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

size_t tc_record_bytes() { return (size_t)tc::REC * 4; }

int launch_tc_expand(const ok_W* W, int kind, cx<double>* out, cudaStream_t st) {
  if (!W || !W->Wtc || !out || kind < 0 || kind > 13) return OK_EINVAL;
  {
    TraceScope ts("expand", st);
    tc::tc_expand_kernel<<<grid_for(W->g.V, 64), 64, 0, st>>>((const unsigned*)W->Wtc, W->g, kind, out);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int tc_blocks_needed(const ok_W* W) {
  static int resident = 0;
  if (resident == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tc::apply_tc_kernel<EPI_DOT, false>, tc::TC_THREADS, 0) != cudaSuccess ||
        nb < 1)
      nb = 1;
    resident = nb * sm_count();
  }
  const int need = grid_for(W->g.V, tc::TC_WARPS);
  return need < resident ? need : resident;
}

int launch_apply_tc(const ok_W* W, const void* in16, cx<float>* out, int nrhs, int epi, const TcEpi& ep, cudaStream_t st) {
  if (!W || !W->Wtc || !in16 || !out || nrhs < 1 || nrhs > tc::MAX_RHS) return OK_EINVAL;
  if (((uintptr_t)in16 | (uintptr_t)out) & 15) return OK_EINVAL;
  if (epi != EPI_NONE && epi != EPI_DOT && epi != EPI_TS) return OK_EINVAL;
  if (epi != EPI_NONE && (!ep.st || !ep.part || !ep.ticket || !ep.y)) return OK_EINVAL;
  const int grid = tc_blocks_needed(W);
  const unsigned* Wt = (const unsigned*)W->Wtc;
  static const char* names[3] = {"apply_tc", "apply_tc_dot", "apply_tc_ts"};
  {
    TraceScope ts(names[epi], st);
    const uint4* i4 = (const uint4*)in16;
    float4* o4 = (float4*)out;
    Geom gs = W->g;
    gs.sms = sm_count();
    const bool ap = gs.bcneg != 0;
#define OK_TC_LAUNCH(E, AP) tc::apply_tc_kernel<E, AP><<<grid, tc::TC_THREADS, 0, st>>>(Wt, i4, o4, gs, nrhs, ep)
    if (epi == EPI_NONE) { if (ap) OK_TC_LAUNCH(EPI_NONE, true); else OK_TC_LAUNCH(EPI_NONE, false); }
    else if (epi == EPI_DOT) { if (ap) OK_TC_LAUNCH(EPI_DOT, true); else OK_TC_LAUNCH(EPI_DOT, false); }
    else { if (ap) OK_TC_LAUNCH(EPI_TS, true); else OK_TC_LAUNCH(EPI_TS, false); }
#undef OK_TC_LAUNCH
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

size_t tc_in16_bytes(int V) { return (size_t)V * 2 * tc::IN16_TILE_U4 * 16; }

int launch_to_tc16(const cx<float>* in, void* out16, int V, int nrhs, unsigned* amax, float* inv_scale, cudaStream_t st) {
  OK_CUDA_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned) * nrhs, st));
  OK_CUDA_TRY(cudaMemsetAsync(out16, 0, tc_in16_bytes(V), st));  // absent right-hand sides
  const long long n4 = 6LL * V;  // float4 per right-hand side
  const int gx = grid_for(n4, 256) < 1024 ? grid_for(n4, 256) : 1024;
  {
    TraceScope ts("to_tc_layout", st);
    tc::tc_amax_kernel<<<dim3(gx, nrhs), 256, 0, st>>>((const float4*)in, n4, amax);
    tc::canon_to_tc16_kernel<<<grid_for(3LL * V * nrhs, 256), 256, 0, st>>>((const float2*)in, (uint2*)out16, V, nrhs, amax,
                                                                          inv_scale);
  }
  count_launch();
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_from_tc(const cx<float>* in, cx<float>* out, int V, int nrhs, cudaStream_t st) {
  {
    TraceScope ts("from_tc_layout", st);
    tc::tc_to_canon_kernel<<<grid_for(3LL * V * nrhs, 256), 256, 0, st>>>((const float4*)in, (float2*)out, V, nrhs);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

// Block shape and resident grid of the vector kernels for nrhs right-hand sides (occupancy looked
// up once per kernel and nrhs).
enum { VK_S = 0, VK_P = 1, VK_XR = 2 };
static void vec_shape(int nrhs, dim3* block, int* grid, int which) {
  static std::atomic<int> cache[3][tc::MAX_RHS + 1];
  const int X = 3 * nrhs;
  int Y = tc::VEC_TARGET / X;
  if (Y < 1) Y = 1;
  *block = dim3(X, Y);
  int nb = cache[which][nrhs].load(std::memory_order_relaxed);
  if (nb == 0) {
    const void* kern = which == VK_S ? (const void*)tc::tc_update_s_kernel
                       : which == VK_P ? (const void*)tc::tc_update_p_kernel : (const void*)tc::tc_update_xr_kernel;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, X * Y, 0) != cudaSuccess || nb < 1) nb = 1;
    cache[which][nrhs].store(nb, std::memory_order_relaxed);
  }
  *grid = nb * sm_count();
}

int tc_vec_blocks(int nrhs) {
  dim3 b;
  int g = 0;
  vec_shape(nrhs, &b, &g, VK_XR);
  return g;
}

int launch_tc_update_s(const cx<float>* r, const cx<float>* v, cx<float>* s, void* s16, int V, int nrhs, const SolverState* st,
                       cudaStream_t strm) {
  dim3 b;
  int g = 0;
  vec_shape(nrhs, &b, &g, VK_S);
  {
    TraceScope ts("update_s_tc", strm);
    tc::tc_update_s_kernel<<<g, b, 0, strm>>>((const float4*)r, (const float4*)v, (float4*)s, (uint2*)s16, 2 * V, nrhs, st);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_tc_update_p(cx<float>* p, void* p16, const cx<float>* r, const cx<float>* v, int V, int nrhs, const SolverState* st,
                       int only, cudaStream_t strm) {
  dim3 b;
  int g = 0;
  vec_shape(nrhs, &b, &g, VK_P);
  {
    TraceScope ts("update_p_tc", strm);
    tc::tc_update_p_kernel<<<g, b, 0, strm>>>((float4*)p, (uint2*)p16, (const float4*)r, (const float4*)v, 2 * V, nrhs, st,
                                              only);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_tc_half(const cx<float>* p, void* p16, int V, int nrhs, const SolverState* st, int only, cudaStream_t strm) {
  dim3 b;
  int g = 0;
  vec_shape(nrhs, &b, &g, VK_P);
  {
    TraceScope ts("half_tc", strm);
    tc::tc_half_kernel<<<g, b, 0, strm>>>((const float4*)p, (uint2*)p16, 2 * V, nrhs, st, only);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_tc_update_xr(cx<float>* x, const void* p16, const cx<float>* s, const void* s16, const cx<float>* t, cx<float>* r,
                        const cx<float>* rhat, int V, int nrhs, SolverState* st, double* part, long long pstride,
                        unsigned* ticket, cudaStream_t strm) {
  dim3 b;
  int g = 0;
  vec_shape(nrhs, &b, &g, VK_XR);
  if ((long long)g * 3 > pstride) return OK_EINVAL;
  TcEpi ep{nullptr, st, part, pstride, ticket, FIN_XR, nullptr};
  {
    TraceScope ts("update_xr_tc", strm);
    tc::tc_update_xr_kernel<<<g, b, 0, strm>>>((float4*)x, (const uint2*)p16, (const float4*)s, (const uint2*)s16,
                                               (const float4*)t, (float4*)r, (const float4*)rhat, 2 * V, nrhs, st, ep);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_tc_demote(const cx<double>* r64, cx<float>* r, cx<float>* rhat, cx<float>* p, int V, int nrhs, int k, bool restart,
                     SolverState* st, double* part, cudaStream_t strm) {
  const int nb = blas_blocks(3LL * V);
  RedArgs ra{st, part, nullptr, restart ? FIN_RESTART : FIN_CONTINUE};
  {
    TraceScope ts("demote_tc", strm);
    if (restart)
      tc::tc_demote_kernel<true><<<nb, 256, 0, strm>>>((const double2*)r64, (float4*)r, (float4*)rhat, (float4*)p, V, nrhs, k, st, ra);
    else
      tc::tc_demote_kernel<false><<<nb, 256, 0, strm>>>((const double2*)r64, (float4*)r, (float4*)rhat, (float4*)p, V, nrhs, k, st, ra);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_tc_accum(cx<double>* x64, cx<float>* x, int V, int nrhs, int k, cudaStream_t strm) {
  {
    TraceScope ts("accum_x_tc", strm);
    tc::tc_accum_kernel<<<blas_blocks(3LL * V), 256, 0, strm>>>((double2*)x64, (float4*)x, V, nrhs, k);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

}  // namespace okgb
