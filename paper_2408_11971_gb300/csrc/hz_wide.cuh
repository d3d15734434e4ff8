// hz_wide.cuh — exact wide-integer helpers for the reductions (Sec. V-B):
// 128-bit sums, the 256-bit variance numerator, and the FP64 finish.
#pragma once
#include <cstdint>

namespace hz {

struct U128 {
  unsigned long long lo, hi;
};
__device__ __forceinline__ void add_u64(U128& a, unsigned long long v) {
  a.lo += v;
  a.hi += (a.lo < v) ? 1ull : 0ull;
}
__device__ __forceinline__ void add_u128(U128& a, const U128& b) {
  a.lo += b.lo;
  a.hi += b.hi + ((a.lo < b.lo) ? 1ull : 0ull);
}

// exact unsigned 256-bit product helpers for the variance numerator
struct U256 {
  unsigned long long w[4];
};
__device__ __forceinline__ U256 mul_u128_u128(unsigned __int128 a, unsigned __int128 b) {
  unsigned long long a0 = (unsigned long long)a, a1 = (unsigned long long)(a >> 64);
  unsigned long long b0 = (unsigned long long)b, b1 = (unsigned long long)(b >> 64);
  unsigned __int128 p00 = (unsigned __int128)a0 * b0, p01 = (unsigned __int128)a0 * b1;
  unsigned __int128 p10 = (unsigned __int128)a1 * b0, p11 = (unsigned __int128)a1 * b1;
  U256 r;
  r.w[0] = (unsigned long long)p00;
  unsigned __int128 mid = (p00 >> 64) + (unsigned long long)p01 + (unsigned long long)p10;
  r.w[1] = (unsigned long long)mid;
  unsigned __int128 hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (unsigned long long)p11;
  r.w[2] = (unsigned long long)hi;
  r.w[3] = (unsigned long long)(hi >> 64) + (unsigned long long)(p11 >> 64);
  return r;
}
__device__ __forceinline__ U256 sub_u256(const U256& a, const U256& b) {  // a >= b
  U256 r;
  unsigned long long borrow = 0;
  for (int i = 0; i < 4; i++) {
    unsigned long long bi = b.w[i] + borrow;
    unsigned long long nb = (bi < borrow) || (a.w[i] < bi) ? 1ull : 0ull;
    r.w[i] = a.w[i] - bi;
    borrow = nb;
  }
  return r;
}
__device__ __forceinline__ double u256_to_double(const U256& a) {
  const double two64 = 18446744073709551616.0;
  double d = (double)a.w[3];
  d = d * two64 + (double)a.w[2];
  d = d * two64 + (double)a.w[1];
  d = d * two64 + (double)a.w[0];
  return d;
}

// Sum of a signed 128-bit value over the 32 lanes of a warp (lane 0 holds it).
__device__ __forceinline__ __int128 warp_sum_i128(__int128 v) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, o);
    const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, o);
    const unsigned long long nl = lo + l2;
    hi = hi + h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  return (__int128)(((unsigned __int128)hi << 64) | lo);
}
__device__ __forceinline__ U128 warp_sum_u128(U128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    U128 t;
    t.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    t.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    add_u128(v, t);
  }
  return v;
}

// mean = (S1 / n) * 2 eps_q ; variance = (2 eps_q)^2 (n S2 - S1^2) / n^2, the
// numerator exact in 256-bit integers (n S2 >= S1^2 by Cauchy-Schwarz).
__device__ __forceinline__ double moment_finish(__int128 S1, const U128& S2, uint64_t n,
                                                float eps_q, bool var) {
  const double e2 = 2.0 * (double)eps_q;
  if (!var) {
    // sign and magnitude: hi * 2^64 + lo without cancellation
    const unsigned __int128 m = (unsigned __int128)(S1 < 0 ? -S1 : S1);
    const double md =
        (double)(unsigned long long)(m >> 64) * 18446744073709551616.0 + (double)(unsigned long long)m;
    const double s1d = S1 < 0 ? -md : md;
    return (s1d / (double)n) * e2;
  }
  const unsigned __int128 s2u = ((unsigned __int128)S2.hi << 64) | S2.lo;
  const unsigned __int128 a1 = (unsigned __int128)(S1 < 0 ? -S1 : S1);
  const U256 nS2 = mul_u128_u128(s2u, (unsigned __int128)n);
  const U256 S1sq = mul_u128_u128(a1, a1);
  const U256 D = sub_u256(nS2, S1sq);
  const double dn = (double)n;
  return (u256_to_double(D) / (dn * dn)) * (e2 * e2);
}


// Population covariance (Sec. V-D) from exact sums: 2 eps_A 2 eps_B
// (n S_AB - S1_A S1_B) / n^2, the numerator formed exactly in signed 256-bit
// (sign and magnitude), then the same FP64 steps as the variance.
__device__ __forceinline__ bool ge_u256(const U256& a, const U256& b) {
  for (int i = 3; i >= 0; i--)
    if (a.w[i] != b.w[i]) return a.w[i] > b.w[i];
  return true;
}
__device__ __forceinline__ U256 add_u256(const U256& a, const U256& b) {
  U256 r;
  unsigned long long carry = 0;
  for (int i = 0; i < 4; i++) {
    const unsigned long long t = a.w[i] + carry;
    const unsigned long long c1 = (t < carry) ? 1ull : 0ull;
    r.w[i] = t + b.w[i];
    carry = c1 + ((r.w[i] < t) ? 1ull : 0ull);
  }
  return r;
}
__device__ __forceinline__ double cov_finish(__int128 SAB, __int128 S1A, __int128 S1B, uint64_t n,
                                             float eps_a, float eps_b) {
  const bool neg1 = SAB < 0;
  const bool neg2 = (S1A < 0) != (S1B < 0);
  const U256 P1 = mul_u128_u128((unsigned __int128)(neg1 ? -SAB : SAB), (unsigned __int128)n);
  const U256 P2 = mul_u128_u128((unsigned __int128)(S1A < 0 ? -S1A : S1A),
                                (unsigned __int128)(S1B < 0 ? -S1B : S1B));
  // N = (+-P1) - (+-P2)
  U256 mag;
  bool neg;
  if (neg1 != neg2) {
    mag = add_u256(P1, P2);
    neg = neg1;
  } else if (ge_u256(P1, P2)) {
    mag = sub_u256(P1, P2);
    neg = neg1;
  } else {
    mag = sub_u256(P2, P1);
    neg = !neg1;
  }
  const double dn = (double)n;
  const double e2a = 2.0 * (double)eps_a, e2b = 2.0 * (double)eps_b;
  const double v = (u256_to_double(mag) / (dn * dn)) * (e2a * e2b);
  return neg ? -v : v;
}

}  // namespace hz
