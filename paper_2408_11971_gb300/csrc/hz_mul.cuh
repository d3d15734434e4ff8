// hz_mul.cuh — requantization of scalar multiplication (Sec. V-A) and of the
// Hadamard product (Sec. V-C): q' = floor(2e q rho + 1/2) (Eq. 3 applied to
// the product of the dequantized values), exact in integer arithmetic, with
// plans that pick 32-, 64- or 128-bit arithmetic from the header's bound of |q|.
#pragma once
#include "hz_common.cuh"

namespace hz {

// Scalar multiplication requantization: floor(2e * q * rho + 1/2), exact.
// 2e = M 2^E with M the 24-bit significand of the float 2e.
struct MulPlan {
  long long rho;
  long long M;
  int E;
  // fast path: q' = (q * P + 2^(sh-1)) >> sh in 64-bit integers, valid when
  // every |q * P| stays below 2^62 (P = rho * M, sh = -E in [1, 62])
  bool fast;
  long long P;
  int sh;
  // 32-bit path: when sh >= 32 and every |q * rho| < 2^31, t = q * rho fits a
  // 32-bit integer, t * M + 2^(sh-1) is one wide multiply-add, and the result
  // is its high word shifted by sh - 32; |q'| < 2^23 then, so no range check
  bool f32;
  int rho32, M32, sh2;
  long long half;
};

__device__ __forceinline__ MulPlan mul_plan(float e, long long rho, uint32_t qbound) {
  MulPlan p;
  p.rho = rho;
  const uint32_t bits = __float_as_uint(2.0f * e);  // normal: e >= FLT_MIN
  p.M = (long long)((bits & 0x7fffffu) | 0x800000u);
  p.E = (int)((bits >> 23) & 0xffu) - 127 - 23;
  p.P = rho * p.M;  // |rho| <= 2^30, M < 2^24: fits
  p.sh = -p.E;
  const unsigned long long aP = (unsigned long long)(p.P < 0 ? -p.P : p.P);
  // |q| <= qbound < 2^30 ; require qbound * |P| < 2^62
  const unsigned __int128 prod = (unsigned __int128)aP * (unsigned __int128)(qbound + 1ull);
  p.fast = p.sh >= 1 && p.sh <= 62 && prod < ((unsigned __int128)1 << 62);
  const unsigned long long arho = (unsigned long long)(rho < 0 ? -rho : rho);
  p.f32 = p.fast && p.sh >= 32 && arho * (qbound + 1ull) < (1ull << 31);
  p.rho32 = (int)rho;
  p.M32 = (int)p.M;
  p.sh2 = p.sh - 32;
  p.half = p.sh >= 1 ? (1ll << (p.sh - 1)) : 0;
  return p;
}

// Plan for the multiplication by the scalar itself, q' = floor(q s + 1/2):
// s = M 2^E with the trailing zero bits of its 53-bit significand removed (so
// short scalars such as 2.5 reach the 64-bit path), the sign in rho.
__device__ __forceinline__ MulPlan mul_plan_exact(double s, uint32_t qbound) {
  MulPlan p;
  p.rho = 0;
  p.M = 0;
  p.E = 0;
  if (s != 0.0) {
    int ex;
    const double fr = frexp(fabs(s), &ex);
    long long M = (long long)ldexp(fr, 53);
    int E = ex - 53;
    while ((M & 1) == 0) {
      M >>= 1;
      E++;
    }
    p.rho = s < 0.0 ? -1 : 1;
    p.M = M;
    p.E = E;
  }
  p.P = p.rho * p.M;
  p.sh = -p.E;
  const unsigned long long aP = (unsigned long long)(p.P < 0 ? -p.P : p.P);
  const unsigned __int128 prod = (unsigned __int128)aP * (unsigned __int128)(qbound + 1ull);
  p.fast = p.sh >= 1 && p.sh <= 62 && prod < ((unsigned __int128)1 << 62);
  p.f32 = false;
  p.rho32 = (int)p.rho;
  p.M32 = 0;
  p.sh2 = 0;
  p.half = p.sh >= 1 && p.sh <= 62 ? (1ll << (p.sh - 1)) : 0;
  return p;
}

__device__ __forceinline__ int mul_requant_f32(int q, const MulPlan& p) {
  const int t = q * p.rho32;
  const long long v = (long long)t * p.M32 + p.half;  // floor(2e q rho + 1/2) * 2^sh, exact
  return (int)(v >> 32) >> p.sh2;
}

__device__ __forceinline__ int mul_requant_fast(int q, const MulPlan& p, bool& ovf) {
  const long long r = ((long long)q * p.P + (1ll << (p.sh - 1))) >> p.sh;  // floor
  if (r > HOSZP_QLIM || r < -(long long)HOSZP_QLIM) {
    ovf = true;
    return 0;
  }
  return (int)r;
}

// Returns q' and sets ovf when |q'| > HOSZP_QLIM.
__device__ __forceinline__ int mul_requant(int q, const MulPlan& p, bool& ovf) {
  const __int128 km = (__int128)((long long)q * p.rho) * p.M;  // |km| < 2^85
  __int128 r;
  if (p.E >= 0) {
    if (km == 0) return 0;
    if (p.E > 40) {
      ovf = true;
      return 0;
    }
    r = km << p.E;
  } else {
    const int sh = -p.E;
    if (sh >= 120) return 0;  // |2e q rho| < 2^-35
    const __int128 half = (__int128)1 << (sh - 1);
    r = (km + half) >> sh;  // arithmetic shift = floor
  }
  if (r > HOSZP_QLIM || r < -(__int128)HOSZP_QLIM) {
    ovf = true;
    return 0;
  }
  return (int)r;
}

// Hadamard product: q' = floor(2e q_A q_B + 1/2) with the multiplier q_B of the
// value. In 64-bit integers when every |q_A q_B M| < 2^62 (plan.fast set for
// the product of the two header bounds), else the 128-bit path of mul_requant.
__device__ __forceinline__ int mul_requant_pair(int qa, int qb, const MulPlan& p, bool& ovf) {
  if (p.fast) {
    const long long r = ((long long)qa * qb * p.M + p.half) >> p.sh;  // floor
    if (r > HOSZP_QLIM || r < -(long long)HOSZP_QLIM) {
      ovf = true;
      return 0;
    }
    return (int)r;
  }
  MulPlan t = p;
  t.rho = qb;
  return mul_requant(qa, t, ovf);
}

}  // namespace hz
