// FP64-accurate application of M on the FP32 pipes (double-float W and fields), table driven.
#pragma once
#include "ok_launch.cuh"

namespace okgb {

// out = M psi (EPI_NONE) or out = b - M psi with <out, out>, <b, b> reduced (EPI_RESID), in
// double-float arithmetic with the handle's OK_W_DF64 copy: psi double-float [V][12], b and out
// FP64 [V][12].  OK_EINVAL without the copy or for another epilogue.
int launch_apply_dd(const ok_W* W, const cx<dd>* psi_df, cx<double>* out, int epi, const EpiArgs<dd>& ep, cudaStream_t st);

// The stencil as the table the kernel walks: 27 offsets, each with its colour matrix-vector
// products (built by ok_dd_table.cuh, passed to the kernel as a launch parameter).
struct DDHop {
  signed char d[4];       // offset (x, y, z, t)
  unsigned char kind;     // DD_ONSITE, DD_PLAIN, DD_THIRD_L, DD_THIRD_U
  unsigned char first;    // first action
  unsigned char count;    // number of actions
  unsigned char pad;
};
struct DDAct {
  unsigned char m;        // colour matrix of the site record (0 .. 42)
  unsigned char flags;    // bit 0: matrix at the offset's site (else at x); bit 1: adjoint;
                          // bits 2-4: source (slot * 2 + spin)
  signed char dst[2];     // accumulator (half * 2 + spin: acc+ 0, 1; acc- 2, 3), or -1
  unsigned char mul[2];   // bits 0-1: scalar (1, a_ii, b_ii); bits 2-4: unit (1, i, -1, -i, 1+i, 1-i, -1-i, -1+i)
  unsigned char pad[2];
};
constexpr int DD_HOPS = 27;
constexpr int DD_ACTS = 148;
enum : int { DD_ONSITE = 0, DD_PLAIN = 1, DD_THIRD_L = 2, DD_THIRD_U = 3 };
struct DDTable {
  DDHop hop[DD_HOPS];
  DDAct act[DD_ACTS];
};

}  // namespace okgb
