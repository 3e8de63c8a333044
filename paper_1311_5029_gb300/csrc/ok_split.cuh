// Double-float split of an FP64 value, for storing the OK_W_DF64 copy of W.
#pragma once
#include <string.h>

#include "ok_internal.cuh"

namespace okgb {

// Double-float split of d: hi = RN_float(d), lo = RN_float(d - hi), the value dd(d) defines.  The
// remainder is formed from the bits of d and hi with integer operations: GB300's FP64 pipe would
// otherwise convert hi back, subtract and convert again for every stored component.  For
// |d| in [2^-74, 2^127) (where lo is a normal float or zero) the result is bit for bit that of the
// definition; outside that range, and for zero, the definition itself is used.
__host__ __device__ __forceinline__ dd split_df(double d) {
  const float hi = (float)d;
#ifdef __CUDA_ARCH__
  const long long D = __double_as_longlong(d);
  const int H = __float_as_int(hi);
#else
  long long D;
  int H;
  memcpy(&D, &d, sizeof D);
  memcpy(&H, &hi, sizeof H);
#endif
  const int ed = (int)((D >> 52) & 0x7ff);
  if (ed < 1023 - 74 || ed > 1023 + 126) return dd(d);
  // significands in units of 2^(ed - 1075): |d| = md, |hi| = mh (hi is d rounded to 24 bits, so it
  // has d's exponent or, when d rounds up to a power of two, the next one)
  const long long md = (D & ((1LL << 52) - 1)) | (1LL << 52);
  const int eh = ((H >> 23) & 0xff) - 127 + 1023;
  long long mh = (long long)((H & 0x7fffff) | 0x800000) << 29;
  if (eh != ed) mh <<= 1;
  int diff = (int)(md - mh);  // |diff| <= 2^28: half a float ulp
  if (D < 0) diff = -diff;
  // lo = diff * 2^(ed - 1075) (diff signed like d; zero stays +0), the power of two a normal float
  const int scale_bits = (ed - 1075 + 127) << 23;
#ifdef __CUDA_ARCH__
  const float scale = __int_as_float(scale_bits);
  const float lo = __int2float_rn(diff) * scale;
#else
  float scale;
  memcpy(&scale, &scale_bits, sizeof scale);
  const float lo = (float)diff * scale;
#endif
  return dd(hi, lo);
}

}  // namespace okgb
