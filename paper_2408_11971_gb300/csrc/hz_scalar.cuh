// hz_scalar.cuh — Eq. 3 for a scalar operand (scalar addition and
// multiplication, Sec. V-A), exact in 128-bit integers.
#pragma once
#include "hz_common.cuh"

namespace hz {

// ---------------------------------------------------------------- scalar quantization
// Eq. 3 for a scalar operand s (a double), evaluated exactly with 128-bit
// integers: with s = ms 2^es and e = me 2^ee (me, ms integers),
// (s + e) / (2e) = (ms 2^(es-ee) + me) / (2 me), and the floor of that ratio
// is an integer division rounded toward minus infinity. Returns false when
// |rho| would exceed HOSZP_QLIM.
__device__ __forceinline__ bool quantize_scalar(double s, float e, long long& rho) {
  const double de = (double)e;
  if (fabs(s) < de) {
    rho = 0;
    return true;
  }
  if (fabs(s) / de > 2.0 * (double)HOSZP_QLIM + 4.0) return false;
  int es, ee;
  const double fs = frexp(s, &es), fe = frexp(de, &ee);
  const long long ms = (long long)ldexp(fs, 53), me = (long long)ldexp(fe, 53);
  es -= 53;
  ee -= 53;
  const int sh = es - ee;  // |s|/e in [1, 2^32) => sh in [-1, 33]
  __int128 num, den;
  if (sh >= 0) {
    num = (__int128)ms * ((__int128)1 << sh) + me;
    den = (__int128)me * 2;
  } else {
    num = (__int128)ms + (__int128)me * ((__int128)1 << (-sh));
    den = (__int128)me * ((__int128)1 << (1 - sh));
  }
  __int128 qq = num / den;
  if (num % den != 0 && num < 0) qq -= 1;
  if (qq > HOSZP_QLIM || qq < -(__int128)HOSZP_QLIM) return false;
  rho = (long long)qq;
  return true;
}

}  // namespace hz
