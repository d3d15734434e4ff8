// hz_var.cuh — one warp's share of the exact sums S1 = sum q and S2 = sum q^2
// (Sec. V-B) over one 64-block tile of a landed super-tile stage, decoded two
// lanes per block with hz_lanes.cuh. Shared by the single-stream variance and
// the batched reductions.
#pragma once
#include "hz_lanes.cuh"
#include "hz_super.cuh"
#include "hz_wide.cuh"

namespace hz {

// half_sums of hz_lanes.cuh for the warp's widest rate Rw (G = (Rw + 8) / 8
// groups of 8 planes); tails and wide values take the 64-bit sums.
__device__ __forceinline__ lanes::HalfSums half_sums_any(int Rw, bool full, bool narrow,
                                                         const uint32_t t[32], int nval,
                                                         bool zero0, const lanes::Shifts& K) {
  const int G = (Rw + 8) >> 3;
#define HZ_HS(GG)                                                          \
  if (G == GG) {                                                           \
    if (!full) return lanes::half_sums<GG, false, true>(t, nval, zero0, K);   \
    if (narrow) return lanes::half_sums<GG, true, false>(t, nval, zero0, K);  \
    return lanes::half_sums<GG, true, true>(t, nval, zero0, K);               \
  }
  HZ_HS(1)
  HZ_HS(2)
  HZ_HS(3)
#undef HZ_HS
  if (!full) return lanes::half_sums<4, false, true>(t, nval, zero0, K);
  if (narrow) return lanes::half_sums<4, true, false>(t, nval, zero0, K);
  return lanes::half_sums<4, true, true>(t, nval, zero0, K);
}

// Tile `ti` of stage sg (rates in tr, tile index `tile` of a stream of
// `ntiles` tiles whose last block holds `lastlen` values): adds this lane's
// share of S1 and S2. The warp takes 16 blocks per step; lane 2m + hf holds
// half hf of block 16 it + m. qsmall: the stream's header bounds every |q|
// below 2^13.
template <class St>
__device__ __forceinline__ void var_tile(const St& sg, const uint64_t* ring, int ti,
                                         const TileRates& tr, uint64_t tile, uint64_t ntiles,
                                         int lastlen, bool qsmall, const lanes::Shifts& K,
                                         long long& s1, U128& s2) {
  const int lane = threadIdx.x & 31;
  const int hf = lane & 1, m = lane >> 1;
  const uint32_t* sgn = reinterpret_cast<const uint32_t*>(sg.sign + sg.sbase + sg.tnc[ti]);
  const uint32_t* pls = reinterpret_cast<const uint32_t*>(ring + sg.pring + sg.pbase + sg.tr[ti]);
  const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
  for (int it = 0; it < steps; it++) {
    const int b = 16 * it + m;
    uint32_t r, ex;
    tile_block(tr, b, r, ex);
    const int len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
    const int nval = min(max(len - 32 * hf, 0), 32);
    const long long O = len ? sg.outlier[TILE * ti + b] : 0;
    const uint32_t sw = r ? sgn[2 * (ex >> 16) + hf] : 0u;
    const int Rw = (int)__reduce_max_sync(0xffffffffu, r);
    const bool fullblk = __all_sync(0xffffffffu, len == L);
    uint32_t t[32];
    lanes::twos_planes_any(Rw, pls + 2 * (ex & 0xffffu) + hf, (int)r, sw, t);
    // narrow sums of p^2 need every |p_i| < 2^14: |q| < 2^13, or 32 deltas below 2^8
    const bool narrow = fullblk && (qsmall || Rw <= 8);
    const lanes::HalfSums hs = half_sums_any(Rw, fullblk, narrow, t, nval, hf == 0, K);
    const int tot0 = __shfl_xor_sync(0xffffffffu, hs.tot, 1);
    const long long base = O + (hf ? (long long)tot0 : 0ll);
    s1 += (long long)nval * base + hs.sp;
    if (narrow && qsmall) {  // every term below 2^40
      add_u64(s2, (unsigned long long)((long long)nval * base * base + 2ll * base * hs.sp +
                                       (long long)hs.sq));
    } else {
      const __int128 sq = narrow ? (__int128)hs.sq : (((__int128)hs.sqh << 64) | hs.sq);
      const __int128 v = (__int128)(nval * base) * base + (__int128)(2 * base) * hs.sp + sq;
      const U128 vv = {(unsigned long long)v, (unsigned long long)(v >> 64)};
      add_u128(s2, vv);
    }
  }
}

// Block-wise means (Sec. V-B, "Mean", last sentences) of tile `ti`: the warp
// takes 16 blocks per step, lane 2m + hf half hf of block 16 it + m; the
// block's exact sum S1_b = sum of its q is formed from both halves and lane
// 2m writes mean_b = (S1_b / L_b) * e2 (the same two FP64 operations as the
// mean of the whole stream).
template <class St>
__device__ __forceinline__ void block_means_tile(const St& sg, const uint64_t* ring, int ti,
                                                 const TileRates& tr, uint64_t tile,
                                                 uint64_t ntiles, int lastlen, double e2,
                                                 const lanes::Shifts& K, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int hf = lane & 1, m = lane >> 1;
  const uint32_t* sgn = reinterpret_cast<const uint32_t*>(sg.sign + sg.sbase + sg.tnc[ti]);
  const uint32_t* pls = reinterpret_cast<const uint32_t*>(ring + sg.pring + sg.pbase + sg.tr[ti]);
  const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
  for (int it = 0; it < steps; it++) {
    const int b = 16 * it + m;
    uint32_t r, ex;
    tile_block(tr, b, r, ex);
    const int len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
    const int nval = min(max(len - 32 * hf, 0), 32);
    const long long O = len ? sg.outlier[TILE * ti + b] : 0;
    const uint32_t sw = r ? sgn[2 * (ex >> 16) + hf] : 0u;
    const int Rw = (int)__reduce_max_sync(0xffffffffu, r);
    const bool fullblk = __all_sync(0xffffffffu, len == L);
    uint32_t t[32];
    lanes::twos_planes_any(Rw, pls + 2 * (ex & 0xffffu) + hf, (int)r, sw, t);
    const bool narrow = fullblk && Rw <= 20;  // sum_i (32 - i) |delta_i| < 2^31
    lanes::HalfSums hs;
    const int G = (Rw + 8) >> 3;
#define HZ_S1(GG)                                                                      \
  if (G == GG) {                                                                       \
    hs = !fullblk  ? lanes::half_sums<GG, false, true, false>(t, nval, hf == 0, K)   \
         : narrow ? lanes::half_sums<GG, true, false, false>(t, nval, hf == 0, K)    \
                  : lanes::half_sums<GG, true, true, false>(t, nval, hf == 0, K);    \
  }
    HZ_S1(1) else HZ_S1(2) else HZ_S1(3) else HZ_S1(4)
#undef HZ_S1
    const int tot0 = __shfl_xor_sync(0xffffffffu, hs.tot, 1);
    const long long base = O + (hf ? (long long)tot0 : 0ll);
    const long long s1h = (long long)nval * base + hs.sp;
    const long long s1 = s1h + __shfl_xor_sync(0xffffffffu, s1h, 1);
    // a full block divides by 64, exactly a scaling by 2^-6 (no FP64 divide)
    const double mb = (len == L) ? (double)s1 * 0.015625 : (double)s1 / (double)len;
    if (hf == 0 && len > 0) out[tile * TILE + b] = mb * e2;
  }
}

}  // namespace hz
