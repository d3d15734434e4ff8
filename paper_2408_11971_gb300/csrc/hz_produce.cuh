// hz_produce.cuh — the store side of operators that produce a stream from
// values held two lanes per block (hz_lanes.cuh): a half's deltas are turned
// into sign-magnitude bit-planes (Fig. 3), the block's rate is taken from both
// halves, and the sign and plane half-words go to the tile's sign and plane
// slots (the SPLIT rule of hz_ws.cuh) at a running, warp-local prefix.
#pragma once
#include "hz_common.cuh"
#include "hz_lanes.cuh"

namespace hz {

// Encodes a half's deltas d (each below 2^(8G-1) in magnitude) and, once the
// block's rate is known from both halves, stores the half-words of its sign
// word and of its rate planes: sign half-word at *sdst, plane p at dst[2p].
// lim_nc, lim_r: the tile's slot sizes (sign words, plane words); a store
// beyond them is refused with CAPACITY. A nonzero bad on entry (an earlier
// error of the warp) suppresses the stores and the check.
template <int G>
__device__ __forceinline__ int encode_store(const int d[32], const lanes::Shifts& K, bool valid,
                                            uint32_t* sdst_base, uint32_t* pdst_base,
                                            uint32_t lim_nc, uint32_t lim_r, uint32_t& rate_pk,
                                            int& bad) {
  uint32_t z[32];
  lanes::half_planes<G>(d, z, K);
  uint32_t nz;
  const uint32_t sgn = lanes::half_sign_magnitude<G>(z, &nz);
  nz |= __shfl_xor_sync(0xffffffffu, nz, 1);  // the block's planes: both halves
  const int rate = valid ? 32 - __clz(nz) : 0;  // <= 8G - 1 <= 31
  // the tile-local exclusive prefix of (sign words << 16 | plane words),
  // counted once per block (on its first lane)
  const int lane = threadIdx.x & 31;
  const uint32_t pk = ((lane & 1) == 0 && rate > 0) ? ((1u << 16) | (uint32_t)rate) : 0u;
  uint32_t inc = pk;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const uint32_t ex = __shfl_sync(0xffffffffu, inc - pk, lane & ~1);
  const uint32_t step = __shfl_sync(0xffffffffu, inc, 31);
  const uint32_t nc0 = (rate_pk >> 16) + (ex >> 16), r0 = (rate_pk & 0xffffu) + (ex & 0xffffu);
  rate_pk += step;
  if (bad == 0 && rate > 0 && (nc0 >= lim_nc || r0 + (uint32_t)rate > lim_r))
    bad = HOSZP_ERR_CAPACITY;
  if (bad == 0 && rate > 0) {
    sdst_base[2 * nc0 + (lane & 1)] = sgn;
    uint32_t* dst = pdst_base + 2 * r0 + (lane & 1);
#pragma unroll
    for (int p = 0; p < 8 * G - 1; p++)
      if (p < rate) dst[2 * p] = z[p];
  }
  return rate;
}

__device__ __forceinline__ int encode_store_any(int Ge, const int d[32], const lanes::Shifts& K,
                                                bool valid, uint32_t* sdst, uint32_t* pdst,
                                                uint32_t lim_nc, uint32_t lim_r,
                                                uint32_t& rate_pk, int& bad) {
  if (Ge == 1) return encode_store<1>(d, K, valid, sdst, pdst, lim_nc, lim_r, rate_pk, bad);
  if (Ge == 2) return encode_store<2>(d, K, valid, sdst, pdst, lim_nc, lim_r, rate_pk, bad);
  if (Ge == 3) return encode_store<3>(d, K, valid, sdst, pdst, lim_nc, lim_r, rate_pk, bad);
  return encode_store<4>(d, K, valid, sdst, pdst, lim_nc, lim_r, rate_pk, bad);
}

}  // namespace hz
