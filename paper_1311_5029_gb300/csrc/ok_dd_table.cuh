// The table that the double-float apply (ok_apply_dd.cu) walks, built on the host: the 27 offsets
// of Eq. minFlopForm and, for each, its colour matrix-vector products with their accumulators,
// factors and units.  The entries follow the hop functions of ok_apply.cu term by term.
#pragma once
#include "ok_dd.cuh"

namespace okgb {
namespace ddtab {

// Table entries: sources (slot * 2 + spin), accumulators (half * 2 + spin), scalars and units.
constexpr int HP(int q) { return q; }        // slot 0: h+ (on-site: u - i l)
constexpr int HM(int q) { return 2 + q; }    // slot 1: h- (on-site: u + i l)
constexpr int T3(int q) { return 4 + q; }    // slot 2: l or u of the temporal hops
constexpr int AP(int q) { return q; }
constexpr int AM(int q) { return 2 + q; }
enum : int { S1 = 0, SA = 1, SB = 2 };
enum : int { U_P1 = 0, U_PI = 1, U_M1 = 2, U_MI = 3, U_1PI = 4, U_1MI = 5, U_M1MI = 6, U_M1PI = 7 };
constexpr int neg_unit(int u) { return u ^ 2; }

// sigma_k applied to a 2-spinor with only spin q nonzero: the output spin and its unit.
inline void sigma_of(int k, int q, int& qo, int& u) {
  if (k == 0) { qo = 1 - q; u = U_P1; }
  else if (k == 1) { qo = 1 - q; u = q == 1 ? U_MI : U_PI; }
  else { qo = q; u = q == 0 ? U_P1 : U_M1; }
}

struct Builder {
  DDTable t{};
  int nh = 0, na = 0;
  void hop(int d0, int d1, int d2, int d3, int kind) {
    DDHop& h = t.hop[nh++];
    h.d[0] = (signed char)d0; h.d[1] = (signed char)d1; h.d[2] = (signed char)d2; h.d[3] = (signed char)d3;
    h.kind = (unsigned char)kind;
    h.first = (unsigned char)na;
    h.count = 0;
  }
  // y = op(W_m) (source), added to accumulator dst0 (and dst1) with scalar and unit.
  void act(int m, bool at_nbr, bool dag, int src, int dst0, int sc0, int u0, int dst1 = -1, int sc1 = 0, int u1 = 0) {
    DDAct& a = t.act[na++];
    a.m = (unsigned char)m;
    a.flags = (unsigned char)((at_nbr ? 1 : 0) | (dag ? 2 : 0) | (src << 2));
    a.dst[0] = (signed char)dst0;
    a.dst[1] = (signed char)dst1;
    a.mul[0] = (unsigned char)(sc0 | (u0 << 2));
    a.mul[1] = (unsigned char)(sc1 | (u1 << 2));
    t.hop[nh - 1].count++;
  }
};

// The entries follow the hop functions of ok_apply.cu term by term.
inline DDTable build_table() {
  Builder b;
  // on-site: a = u - i l (slot 0), b = u + i l (slot 1); A = Y+ a, B = Y- b enter
  // acc+ = (1 + i) A + (1 - i) B and acc- = (1 - i) A + (1 + i) B (the c0q part is set by the gather)
  b.hop(0, 0, 0, 0, DD_ONSITE);
  b.act(M_Y0P + 0, false, false, HP(0), AP(0), S1, U_1PI, AM(0), S1, U_1MI);
  b.act(M_Y0P + 0, false, false, HP(1), AP(1), S1, U_M1MI, AM(1), S1, U_M1PI);
  b.act(M_Y0P + 1, false, false, HP(1), AP(0), S1, U_1PI, AM(0), S1, U_1MI);
  b.act(M_Y0P + 2, false, false, HP(0), AP(1), S1, U_1PI, AM(1), S1, U_1MI);
  b.act(M_Y0M + 0, false, false, HM(0), AP(0), S1, U_1MI, AM(0), S1, U_1PI);
  b.act(M_Y0M + 0, false, false, HM(1), AP(1), S1, U_M1PI, AM(1), S1, U_M1MI);
  b.act(M_Y0M + 1, false, false, HM(1), AP(0), S1, U_1MI, AM(0), S1, U_1PI);
  b.act(M_Y0M + 2, false, false, HM(0), AP(1), S1, U_1MI, AM(1), S1, U_1PI);
  // spatial nearest neighbours: blocks P+ / 2 at mp .. mp + 3, P- / 2 at mm .. mm + 3
  for (int I = 0; I < 3; ++I) {
    const int mp = M_WP + 8 * I, mm = mp + 4;
    b.hop(I == 0, I == 1, I == 2, 0, DD_PLAIN);
    b.act(mp + 0, false, false, HP(0), AP(0), S1, U_P1);
    b.act(mp + 1, false, false, HP(1), AP(0), S1, U_P1);
    b.act(mp + 2, false, false, HP(0), AP(1), S1, U_P1);
    b.act(mp + 3, false, false, HP(1), AP(1), S1, U_P1);
    b.act(mm + 0, false, false, HM(0), AM(0), S1, U_P1);
    b.act(mm + 1, false, false, HM(1), AM(0), S1, U_P1);
    b.act(mm + 2, false, false, HM(0), AM(1), S1, U_P1);
    b.act(mm + 3, false, false, HM(1), AM(1), S1, U_P1);
    b.hop(-(I == 0), -(I == 1), -(I == 2), 0, DD_PLAIN);
    b.act(mm + 0, true, true, HP(0), AP(0), S1, U_P1);
    b.act(mm + 1, true, true, HP(0), AP(1), S1, U_P1);
    b.act(mm + 2, true, true, HP(1), AP(0), S1, U_P1);
    b.act(mm + 3, true, true, HP(1), AP(1), S1, U_P1);
    b.act(mp + 0, true, true, HM(0), AM(0), S1, U_P1);
    b.act(mp + 1, true, true, HM(0), AM(1), S1, U_P1);
    b.act(mp + 2, true, true, HM(1), AM(0), S1, U_P1);
    b.act(mp + 3, true, true, HM(1), AM(1), S1, U_P1);
  }
  // temporal: forward acc+ += S h+ - U l, acc- += U l - S h-; backward acc+ += -U^dag u - S^dag h+,
  // acc- += -U^dag u + S^dag h-, with S = [[s3, n1], [n2, -s3]]
  b.hop(0, 0, 0, 1, DD_THIRD_L);
  for (int q = 0; q < 2; ++q) b.act(M_UT, false, false, T3(q), AP(q), S1, U_M1, AM(q), S1, U_P1);
  b.act(M_ST + 0, false, false, HP(0), AP(0), S1, U_P1);
  b.act(M_ST + 0, false, false, HP(1), AP(1), S1, U_M1);
  b.act(M_ST + 0, false, false, HM(0), AM(0), S1, U_M1);
  b.act(M_ST + 0, false, false, HM(1), AM(1), S1, U_P1);
  b.act(M_ST + 1, false, false, HP(1), AP(0), S1, U_P1);
  b.act(M_ST + 1, false, false, HM(1), AM(0), S1, U_M1);
  b.act(M_ST + 2, false, false, HP(0), AP(1), S1, U_P1);
  b.act(M_ST + 2, false, false, HM(0), AM(1), S1, U_M1);
  b.hop(0, 0, 0, -1, DD_THIRD_U);
  for (int q = 0; q < 2; ++q) b.act(M_UT, true, true, T3(q), AP(q), S1, U_M1, AM(q), S1, U_M1);
  b.act(M_ST + 0, true, true, HP(0), AP(0), S1, U_M1);
  b.act(M_ST + 0, true, true, HP(1), AP(1), S1, U_P1);
  b.act(M_ST + 0, true, true, HM(0), AM(0), S1, U_P1);
  b.act(M_ST + 0, true, true, HM(1), AM(1), S1, U_M1);
  b.act(M_ST + 1, true, true, HP(0), AP(1), S1, U_M1);
  b.act(M_ST + 1, true, true, HM(0), AM(1), S1, U_P1);
  b.act(M_ST + 2, true, true, HP(1), AP(0), S1, U_M1);
  b.act(M_ST + 2, true, true, HM(1), AM(0), S1, U_P1);
  // straight two hops x +- 2I: (a +- b sigma_I) V h+- forward, (a -+ b sigma_I) V^dag h+- backward
  for (int I = 0; I < 3; ++I) {
    const int V = M_VII + I;
    for (int dir = 0; dir < 2; ++dir) {
      const int st = dir == 0 ? 2 : -2;
      b.hop(st * (I == 0), st * (I == 1), st * (I == 2), 0, DD_PLAIN);
      for (int q = 0; q < 2; ++q) {
        int qo, u;
        sigma_of(I, q, qo, u);
        const int up = dir == 0 ? u : neg_unit(u);  // sign of b on h+
        b.act(V, dir == 1, dir == 1, HP(q), AP(q), SA, U_P1, AP(qo), SB, up);
        b.act(V, dir == 1, dir == 1, HM(q), AM(q), SA, U_P1, AM(qo), SB, neg_unit(up));
      }
    }
  }
  // diagonal pairs (I, J): V at x +- (I + J) with +-(s_I + s_J), X at x +- (I - J) with +-(s_I - s_J)
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int P = 0; P < 3; ++P) {
    const int I = pairs[P][0], J = pairs[P][1];
    for (int form = 0; form < 2; ++form) {      // 0: V (I + J), 1: X (I - J)
      const int sj = form == 0 ? 1 : -1;         // sign of J in the offset and of s_J
      const int m = form == 0 ? M_VIJ + P : M_XIJ + P;
      for (int dir = 0; dir < 2; ++dir) {        // 0: forward (matrix at x), 1: backward (at the neighbour)
        const int st = dir == 0 ? 1 : -1;
        b.hop(st * ((I == 0) + sj * (J == 0)), st * ((I == 1) + sj * (J == 1)), st * ((I == 2) + sj * (J == 2)), 0,
              DD_PLAIN);
        for (int q = 0; q < 2; ++q) {
          int qi, ui, qj, uj;
          sigma_of(I, q, qi, ui);
          sigma_of(J, q, qj, uj);
          // on h+: forward +s_I + sj s_J, backward the negative; on h-: the negative of h+
          int pi = ui, pj = sj > 0 ? uj : neg_unit(uj);
          if (dir == 1) { pi = neg_unit(pi); pj = neg_unit(pj); }
          b.act(m, dir == 1, dir == 1, HP(q), AP(qi), S1, pi, AP(qj), S1, pj);
          b.act(m, dir == 1, dir == 1, HM(q), AM(qi), S1, neg_unit(pi), AM(qj), S1, neg_unit(pj));
        }
      }
    }
  }
  if (b.nh != DD_HOPS || b.na != DD_ACTS) b.t.hop[0].count = 0;  // malformed: launch_apply_dd refuses it
  return b.t;
}

}  // namespace ddtab
}  // namespace okgb
