// hz_decode.cuh — decoding an octet (lane j's 8 positions of a block) from a
// tile held in shared memory: its 8 deltas (workflow 2) or, with the inverse
// Lorenzo, its 8 quantized integers (workflow 3).
#pragma once
#include "hz_pipe.cuh"

namespace hz {

// Per-octet view of a block of the tile held in an InStage.
struct BlockRef {
  int rate;
  int outlier;
  uint32_t sign_byte;
  const uint64_t* planes;  // shared memory
  int len;                 // valid positions of the block (64, fewer in the tail block)
};

// The planes of a block, transposed: group k (planes 8k..8k+7) becomes 8
// bytes (lo[k], hi[k]) whose byte t holds bits 8k..8k+7 of |delta| at
// position 8j+t. kmax (warp-uniform) >= ceil(rate / 8). KMAX: the most
// groups the calling kernel decodes (4 covers every rate; groups at and above
// KMAX read as zero).
template <int KMAX = 4>
__device__ __forceinline__ void decode_groups(const uint64_t* planes, int r, int kmax,
                                              const OctetSel& S, int j, uint32_t lo[4],
                                              uint32_t hi[4]) {
  uint64_t w[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int p = 8 * k + j;
    w[k] = (k < KMAX && k < kmax && p < r) ? planes[p] : 0ull;
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    lo[k] = (uint32_t)w[k];
    hi[k] = (uint32_t)(w[k] >> 32);
    if (k < KMAX && k < kmax) {
      byte_transpose8(lo[k], hi[k], S);
      tr8x8_d(lo[k], hi[k]);
    }
  }
}

// Magnitudes of the 8 positions from the transposed groups.
template <int KMAX = 4>
__device__ __forceinline__ void mags_from_groups(const uint32_t lo[4], const uint32_t hi[4],
                                                 int kmax, uint32_t m[8]) {
  if (KMAX == 1 || kmax <= 1) {
#pragma unroll
    for (int t = 0; t < 4; t++) {
      m[t] = __byte_perm(lo[0], 0u, 0x4440u + t);
      m[t + 4] = __byte_perm(hi[0], 0u, 0x4440u + t);
    }
  } else if (KMAX == 2 || kmax == 2) {  // two bytes per value: interleave the groups
    uint32_t x;
    x = __byte_perm(lo[0], lo[1], 0x5140u);
    m[0] = x & 0xffffu;
    m[1] = x >> 16;
    x = __byte_perm(lo[0], lo[1], 0x7362u);
    m[2] = x & 0xffffu;
    m[3] = x >> 16;
    x = __byte_perm(hi[0], hi[1], 0x5140u);
    m[4] = x & 0xffffu;
    m[5] = x >> 16;
    x = __byte_perm(hi[0], hi[1], 0x7362u);
    m[6] = x & 0xffffu;
    m[7] = x >> 16;
  } else {
#pragma unroll
    for (int t = 0; t < 4; t++) {
      uint32_t a = 0, b = 0;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        a |= __byte_perm(lo[k], 0u, 0x4440u + t) << (8 * k);
        b |= __byte_perm(hi[k], 0u, 0x4440u + t) << (8 * k);
      }
      m[t] = a;
      m[t + 4] = b;
    }
  }
}

// Signed deltas of lane j's positions; position 0 and positions past the
// block's end are 0. The sign is applied as a multiply by +-1 (FMA pipe).
template <int KMAX = 4>
__device__ __forceinline__ void octet_deltas(const BlockRef& br, int kmax, int j,
                                             const OctetSel& S, int d[8]) {
  uint32_t lo[4], hi[4], m[8];
  decode_groups<KMAX>(br.planes, br.rate, kmax, S, j, lo, hi);
  mags_from_groups<KMAX>(lo, hi, kmax, m);
#pragma unroll
  for (int t = 0; t < 8; t++) {
    const int k = 1 - 2 * (int)((br.sign_byte >> t) & 1u);
    d[t] = (int)m[t] * k;
  }
  if (j == 0) d[0] = 0;
  if (br.len < L) {
#pragma unroll
    for (int t = 0; t < 8; t++)
      if (8 * j + t >= br.len) d[t] = 0;
  }
}

// Inverse Lorenzo: q_i = O + sum_{k <= i} delta_k for lane j's 8 positions.
__device__ __forceinline__ void octet_values(const BlockRef& br, const int d[8], int j, int q[8]) {
  int s[8];
  int acc = 0;
#pragma unroll
  for (int t = 0; t < 8; t++) {
    acc += d[t];
    s[t] = acc;
  }
  const int base = br.outlier + octet_excl_scan(acc, j);
#pragma unroll
  for (int t = 0; t < 8; t++) q[t] = base + s[t];
}

// This lane's share of the block sum S1_b = L_b O + sum_i (L_b - i) delta_i
// (the block's q summed without the inverse Lorenzo).
__device__ __forceinline__ long long octet_sum_q(const BlockRef& br, const int d[8], int j,
                                                 int kmax) {
  long long sd, std_;
  if (kmax <= 2) {  // |delta| < 2^16: 32-bit sums cannot overflow
    int a = 0, b = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) {
      a += d[t];
      b += t * d[t];
    }
    sd = a;
    std_ = b;
  } else {
    sd = 0;
    std_ = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) {
      sd += d[t];
      std_ += (long long)t * d[t];
    }
  }
  long long v = (long long)(br.len - 8 * j) * sd - std_;
  if (j == 0) v += (long long)br.len * br.outlier;
  return v;
}

// Mean fast path (full block, at most 16 planes): this lane's share of the
// block sum S1_b = 64 O + sum_i (64 - i) delta_i, as dot products of the
// transposed magnitudes with signed weights (DP4A on bytes for <= 8 planes,
// DP2A on 16-bit pairs for <= 16). wlo/whi: lane-constant weight bytes
// (64 - 8j - t, 0 at position 0).
__device__ __forceinline__ int dp4a_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_lo_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.lo.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_hi_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.hi.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t sign_weights(uint32_t w, uint32_t nib) {
  // bytes of w negated where the nibble's bit is set (w >= 1 there: no carries)
  const uint32_t s = (nib * 0x00204081u) & 0x01010101u;
  return (w ^ (s * 0xffu)) + s;
}
__device__ __forceinline__ int octet_sum_fast(const BlockRef& br, int kmax, int j,
                                              const OctetSel& S, uint32_t wlo, uint32_t whi) {
  uint32_t lo[4], hi[4];
  decode_groups(br.planes, br.rate, kmax, S, j, lo, hi);
  const uint32_t sb = br.sign_byte & (j == 0 ? 0xfeu : 0xffu);
  const uint32_t clo = sign_weights(wlo, sb & 0xfu), chi = sign_weights(whi, sb >> 4);
  int acc;
  if (kmax <= 1) {
    acc = dp4a_us(hi[0], chi, dp4a_us(lo[0], clo, 0));
  } else {
    acc = dp2a_lo_us(__byte_perm(lo[0], lo[1], 0x5140u), clo, 0);
    acc = dp2a_hi_us(__byte_perm(lo[0], lo[1], 0x7362u), clo, acc);
    acc = dp2a_lo_us(__byte_perm(hi[0], hi[1], 0x5140u), chi, acc);
    acc = dp2a_hi_us(__byte_perm(hi[0], hi[1], 0x7362u), chi, acc);
  }
  return acc;
}

// Checks the pre-scan's totals against the header (a corrupt stream stops here).
__device__ __forceinline__ bool prescan_ok(const Info& h, const unsigned long long* pre,
                                           uint64_t max_tiles) {
  if (!h.ok) return false;
  const uint64_t nt = ntiles_of(h.nb);
  if (nt + 1 > max_tiles) return false;  // the pre-scan refused it (workspace bound)
  return pre[2 * nt] == h.nnc && pre[2 * nt + 1] == h.R;
}

}  // namespace hz
