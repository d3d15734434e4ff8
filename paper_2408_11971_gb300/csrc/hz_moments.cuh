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
