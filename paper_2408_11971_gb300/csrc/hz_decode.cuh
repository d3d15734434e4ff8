// hz_decode.cuh — the consumer side of a tile: locate each block's sign word
// and planes (rates -> in-tile scan -> look-back over tiles), then decode an
// octet's 8 deltas (workflow 2) or, with the inverse Lorenzo, its 8 quantized
// integers (workflow 3).
#pragma once
#include "hz_common.cuh"

namespace hz {

// Shared state of one input stream inside a CTA.
struct InTile {
  uint8_t rate[TILE];
  TileScan ts;
  unsigned long long pre[2];  // exclusive prefix of the tile: (nc, r)
};

// Loads the tile's rates (threads 0..63), scans them and looks back on chain
// `d` with warp `wid`. Whole CTA. Rates > 31 are reported as a corrupt stream.
__device__ __forceinline__ void in_tile_begin(const uint8_t* __restrict__ c, const Info& h,
                                              uint64_t tile, InTile* s, Desc* d,
                                              unsigned long long epoch, int* st, int wid,
                                              int& bad) {
  const int tid = threadIdx.x;
  if (tid < TILE) {
    const uint64_t b = tile * TILE + tid;
    uint8_t r = (b < h.nb) ? c[HOSZP_HEADER_BYTES + b] : 0;
    if (r > MAX_RATE) {
      bad = HOSZP_ERR_FORMAT;
      r = 0;
    }
    s->rate[tid] = r;
  }
  __syncthreads();
  tile_scan(s->rate, &s->ts);
  tile_prefix(d, (int64_t)tile, epoch, st, s->ts.agg_nc, s->ts.agg_r, wid, s->pre);
}

// Per-octet view of a block after in_tile_begin + __syncthreads.
struct BlockRef {
  int rate;
  int outlier;
  uint32_t sign_byte;
  const uint64_t* planes;
  int len;  // valid positions of the block (64, or fewer in the tail block)
};

__device__ __forceinline__ BlockRef block_ref(const uint8_t* __restrict__ c, const Info& h,
                                              uint64_t tile, const InTile* s, int g, int j,
                                              int& bad) {
  BlockRef br;
  const uint64_t b = tile * TILE + g;
  br.rate = 0;
  br.outlier = 0;
  br.sign_byte = 0;
  br.planes = reinterpret_cast<const uint64_t*>(c + h.o_plane);
  br.len = 0;
  if (b >= h.nb) return br;
  { const uint64_t rem = h.n - b * L; br.len = rem < (uint64_t)L ? (int)rem : L; }
  br.outlier = __ldg(reinterpret_cast<const int*>(c + h.o_out) + b);
  const int r = s->rate[g];
  if (r > 0) {
    const uint64_t si = s->pre[0] + s->ts.nc_excl[g];
    const uint64_t pi = s->pre[1] + s->ts.r_excl[g];
    if (si >= h.nnc || pi + (uint64_t)r > h.R) {
      bad = HOSZP_ERR_FORMAT;
      return br;
    }
    br.rate = r;
    br.sign_byte = __ldg(c + h.o_sign + 8 * si + j);
    br.planes += pi;
  }
  return br;
}

// Signed deltas of lane j's positions 8j..8j+7; position 0 and positions past
// the block's end are 0. kmax: warp-uniform number of 8-plane groups.
__device__ __forceinline__ void octet_deltas(const BlockRef& br, int kmax, int j, int d[8]) {
  uint32_t mag[8];
  decode_mags(br.planes, br.rate, kmax, j, mag);
#pragma unroll
  for (int t = 0; t < 8; t++) {
    const int pos = 8 * j + t;
    int v = ((br.sign_byte >> t) & 1u) ? -(int)mag[t] : (int)mag[t];
    d[t] = (pos == 0 || pos >= br.len) ? 0 : v;
  }
}

// Inverse Lorenzo: q_i = O + sum_{k <= i} delta_k, for lane j's 8 positions.
__device__ __forceinline__ void octet_values(const BlockRef& br, const int d[8], int j, int q[8]) {
  int s[8];
  int acc = 0;
#pragma unroll
  for (int t = 0; t < 8; t++) {
    acc += d[t];
    s[t] = acc;
  }
  const int excl = octet_excl_scan(acc, j);
#pragma unroll
  for (int t = 0; t < 8; t++) q[t] = br.outlier + excl + s[t];
}

}  // namespace hz
