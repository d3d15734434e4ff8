// hz_moments.cuh — one octet's share of a stream's exact sums S1 = sum q and
// S2 = sum q^2 (Sec. V-B), from a prepared input stage. Shared by the
// single-stream and the batched reduction kernels.
#pragma once
#include "hz_wide.cuh"
#include "hz_ws.cuh"

namespace hz {

// Weight bytes 64 - (8j + t) of the block sum S1_b = 64 O + sum_i (64 - i) delta_i
// for lane j's positions (0 at position 0).
__device__ __forceinline__ void mean_weights(int j, uint32_t& wlo, uint32_t& whi) {
  wlo = 0;
  whi = 0;
#pragma unroll
  for (int t = 0; t < 4; t++) {
    wlo |= (uint32_t)(64 - 8 * j - t) << (8 * t);
    whi |= (uint32_t)(64 - 8 * j - 4 - t) << (8 * t);
  }
  if (j == 0) wlo &= 0xffffff00u;
}

// Adds lane j's share of block g of the stage to s1 (and s2 when VAR).
// release() is called once the stage's shared memory has been read.
template <bool VAR, class Release>
__device__ __forceinline__ void moments_octet(const InStage& sg, const uint64_t* ring, int g,
                                              int j, int w, const OctetSel& S, uint32_t wlo,
                                              uint32_t whi, long long& s1, U128& s2,
                                              Release&& release) {
  const BlockRef br = block_ref_s(sg, ring, g, j);
  const int kmax = sg.kmx[w];
  const bool full_tile = sg.nvalid == TILE && sg.lastlen == L;
  if (!VAR && kmax <= 2 && full_tile) {
    const int v = octet_sum_fast(br, kmax, j, S, wlo, whi);
    release();
    s1 += v;
    if (j == 0) s1 += (long long)L * br.outlier;
    return;
  }
  int d[8];
  octet_deltas(br, kmax, j, S, d);
  release();
  if (!VAR) {
    s1 += octet_sum_q(br, d, j, kmax);
  } else {
    int q[8];
    octet_values(br, d, j, q);
    long long a = 0;
    unsigned long long b = 0;  // 8 squares of |q| <= 2^30 stay below 2^63
#pragma unroll
    for (int t = 0; t < 8; t++) {
      const int qq = (8 * j + t < br.len) ? q[t] : 0;
      a += qq;
      b += (unsigned long long)((long long)qq * qq);
    }
    s1 += a;
    add_u64(s2, b);
  }
}

}  // namespace hz

namespace hz {

// ---------------------------------------------------------------- bit-sliced mean
// The mean needs only S1 = sum_b [L_b O_b + sum_i (L_b - i) delta_{b,i}]
// (Sec. V-B). For a full block (L_b = 64) write each delta through the r-bit
// word u_i = |delta_i| at a non-negative position and 2^r - 1 - |delta_i| at a
// negative one (the plane bits xor the sign bit), so that
//     delta_i = u_i - s_i (2^r - 1)   and
//     sum_i (64 - i) delta_i = sum_i (64 - i) u_i - (2^r - 1) W(s),
// with W(m) = sum_i (64 - i) m_i, a weighted popcount. A lane owns two blocks
// of a tile per visit and adds their u into per-position column sums kept
// bit-sliced, one set per 32-position half: acc[k] holds bit k of every
// position's running sum, and adding a block is a ripple-carry add over its
// plane words, about two logic operations per column per 32 values, with no
// transpose and no per-value arithmetic. The ripple stops at the warp's
// largest rate: the carry word leaving the top column goes straight into the
// exact sum as a weighted popcount, so the columns never overflow and are
// converted once per thread. Planes at or above RF, and the stream's last
// block when it is short, go through popcounts directly (both rare).
__device__ __forceinline__ int wsum32(uint32_t m, int base) {
  // sum over set bits l of m of (base - l)
  const int t = __popc(m & 0xAAAAAAAAu) + 2 * __popc(m & 0xCCCCCCCCu) +
                4 * __popc(m & 0xF0F0F0F0u) + 8 * __popc(m & 0xFF00FF00u) +
                16 * __popc(m & 0xFFFF0000u);
  return base * __popc(m) - t;
}
// both halves of a 64-bit word: sum over set bits i of (64 - i)
__device__ __forceinline__ long long wsum64(uint32_t lo, uint32_t hi) {
  return (long long)wsum32(lo, 64) + wsum32(hi, 32);
}

// RF: planes added through the columns (16 covers every block of a stream
// whose rates stay below 16; a plan that knows its rates stay below 8 may take
// 8, which halves the column registers).
template <int RF_ = 16>
struct MeanAccT {
  static constexpr int RF = RF_;
  uint32_t a0[RF], a1[RF];  // columns of positions 0..31 and 32..63
  __int128 s1;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int k = 0; k < RF; k++) a0[k] = a1[k] = 0u;
    s1 = 0;
  }
  // Moves the column sums into s1: sum_k 2^k W(acc[k]).
  __device__ __forceinline__ void flush() {
    long long t = 0;
#pragma unroll
    for (int k = 0; k < RF; k++) {
      t += wsum64(a0[k], a1[k]) << k;
      a0[k] = a1[k] = 0u;
    }
    s1 += t;
  }
};
using MeanAcc = MeanAccT<16>;

// Ripple-carry add of the first rl (<= R) planes of a block into columns
// 0..R-1; returns the carry words leaving column R-1.
template <int R, class Acc>
__device__ __forceinline__ void mean_cols(Acc& A, const uint2* pl, int rl, uint32_t s0,
                                          uint32_t s1, uint32_t& c0, uint32_t& c1) {
  static_assert(R <= Acc::RF, "columns 0 .. R-1 exist");
#pragma unroll
  for (int k = 0; k < R; k++) {
    uint32_t u0 = 0u, u1 = 0u;
    if (k < rl) {
      const uint2 x = pl[k];
      u0 = (x.x & 0xfffffffeu) ^ s0;  // position 0 holds delta_0 := 0
      u1 = x.y ^ s1;
    }
    const uint32_t a = A.a0[k], b = A.a1[k];
    A.a0[k] = a ^ u0 ^ c0;
    c0 = (a & u0) | (c0 & (a ^ u0));
    A.a1[k] = b ^ u1 ^ c1;
    c1 = (b & u1) | (c1 & (b ^ u1));
  }
}

// Adds one block to A: rate r (<= 31, 0 for a constant block or none), block
// length len (64, fewer for the stream's last block, 0 for no block), outlier
// O, sign word sg and plane words pl[0 .. r-1]. All 32 lanes of the warp call
// this together, each with its own block.
template <class Acc>
__device__ __forceinline__ void mean_block(int r, int len, int O, uint64_t sg, const uint2* pl,
                                           Acc& A) {
  constexpr int RF = Acc::RF;
  const bool full = (len == L);
  const int rl = full ? min(r, RF) : 0;
  const int rw = (int)__reduce_max_sync(0xffffffffu, (unsigned)rl);
  const uint32_t sl = (uint32_t)sg, sh = (uint32_t)(sg >> 32);
  long long e = (long long)len * O;
  if (rw > 0) {
    uint32_t c0 = 0u, c1 = 0u;
    switch (rw) {
#define HZ_MEAN_CASE(R)                                                  \
  case R:                                                                \
    if constexpr (R <= RF) mean_cols<R>(A, pl, rl, sl, sh, c0, c1);      \
    break;
      HZ_MEAN_CASE(1) HZ_MEAN_CASE(2) HZ_MEAN_CASE(3) HZ_MEAN_CASE(4)
      HZ_MEAN_CASE(5) HZ_MEAN_CASE(6) HZ_MEAN_CASE(7) HZ_MEAN_CASE(8)
      HZ_MEAN_CASE(9) HZ_MEAN_CASE(10) HZ_MEAN_CASE(11) HZ_MEAN_CASE(12)
      HZ_MEAN_CASE(13) HZ_MEAN_CASE(14) HZ_MEAN_CASE(15) HZ_MEAN_CASE(16)
#undef HZ_MEAN_CASE
      default:
        break;
    }
    if (c0 | c1) e += wsum64(c0, c1) << rw;  // carry out of the top column: weight 2^rw
  }
  if (r > 0 && full) {
    e -= (long long)((1ull << r) - 1ull) * wsum64(sl, sh);
    for (int p = RF; p < r; p++) {
      const uint2 x = pl[p];
      e += wsum64((x.x & 0xfffffffeu) ^ sl, x.y ^ sh) << p;
    }
  } else if (r > 0 && len > 0) {  // the stream's short last block: weights len - i
    const uint32_t m0 = (len >= 32 ? 0xffffffffu : ((1u << len) - 1u)) & 0xfffffffeu;
    const uint32_t m1 = len >= 64 ? 0xffffffffu : (len <= 32 ? 0u : ((1u << (len - 32)) - 1u));
    for (int p = 0; p < r; p++) {
      const uint2 x = pl[p];
      const uint32_t x0 = x.x & m0, x1 = x.y & m1;
      const long long t = (long long)wsum32(x0, len) + wsum32(x1, len - 32) -
                          2ll * ((long long)wsum32(x0 & sl, len) + wsum32(x1 & sh, len - 32));
      e += t << p;
    }
  }
  A.s1 += e;
}

// Last CTA of a reduction launch, one whole warp: the exact sums of the
// per-CTA partials (lane 0 holds them), read by all lanes at once.
__device__ __forceinline__ void sum_partials_warp(const Partial* P, unsigned int G, __int128& S1,
                                                  U128& S2) {
  const int lane = threadIdx.x & 31;
  __int128 a = 0;
  U128 b = {0, 0};
  for (unsigned int u0 = lane; u0 < G; u0 += 32 * 4) {  // four partials in flight
    Partial p[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const unsigned int u = u0 + 32 * i;
      if (u < G) p[i] = P[u];
      else p[i] = Partial{0, 0, 0ull, 0ull};
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
      a += ((__int128)p[i].s1_hi << 64) | (unsigned long long)p[i].s1_lo;
      const U128 v = {p[i].s2_lo, p[i].s2_hi};
      add_u128(b, v);
    }
  }
  S1 = warp_sum_i128(a);
  S2 = warp_sum_u128(b);
}

}  // namespace hz
