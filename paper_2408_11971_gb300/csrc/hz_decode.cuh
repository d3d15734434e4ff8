// hz_decode.cuh — the consumer side of a tile: a CTA walks its tiles with the
// next tiles' compressed words already in flight into a shared-memory ring
// (bulk copies located by the rate pre-scan), then decodes an octet's 8 deltas
// (workflow 2) or, with the inverse Lorenzo, its 8 quantized integers
// (workflow 3).
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

__device__ __forceinline__ BlockRef block_ref(const InStage& s, const TileScan& ts, const Info& h,
                                              uint64_t tile, int g, int j) {
  BlockRef br;
  const uint64_t b = tile * TILE + g;
  br.rate = s.rate[g];  // sanitized: 0 past the end and for invalid rates
  br.outlier = s.outlier[g];
  br.planes = s.plane + s.pbase + ts.r_excl[g];
  br.sign_byte = br.rate
                     ? reinterpret_cast<const uint8_t*>(s.sign + s.sbase + ts.nc_excl[g])[j]
                     : 0u;
  const uint64_t rem = (b < h.nb) ? h.n - b * L : 0;
  br.len = rem < (uint64_t)L ? (int)rem : L;
  return br;
}

// Magnitudes of lane j's positions 8j..8j+7 from a block's planes in shared
// memory; kmax warp-uniform >= ceil(rate/8).
__device__ __forceinline__ void decode_mags_s(const uint64_t* planes, int r, int kmax, int j,
                                              uint32_t mag[8]) {
  uint64_t w[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int p = 8 * k + j;
    w[k] = (k < kmax && p < r) ? planes[p] : 0ull;
  }
#pragma unroll
  for (int t = 0; t < 8; t++) mag[t] = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k < kmax) {
      uint32_t lo = (uint32_t)w[k], hi = (uint32_t)(w[k] >> 32);
      byte_transpose8(lo, hi, j);
      tr8x8(lo, hi);
      if (k == 0) {
        mag[0] = lo & 0xffu;
        mag[1] = (lo >> 8) & 0xffu;
        mag[2] = (lo >> 16) & 0xffu;
        mag[3] = lo >> 24;
        mag[4] = hi & 0xffu;
        mag[5] = (hi >> 8) & 0xffu;
        mag[6] = (hi >> 16) & 0xffu;
        mag[7] = hi >> 24;
      } else {
        const int sh = 8 * k;
        mag[0] |= (lo & 0xffu) << sh;
        mag[1] |= ((lo >> 8) & 0xffu) << sh;
        mag[2] |= ((lo >> 16) & 0xffu) << sh;
        mag[3] |= (lo >> 24) << sh;
        mag[4] |= (hi & 0xffu) << sh;
        mag[5] |= ((hi >> 8) & 0xffu) << sh;
        mag[6] |= ((hi >> 16) & 0xffu) << sh;
        mag[7] |= (hi >> 24) << sh;
      }
    }
  }
}

// Signed deltas of lane j's positions; position 0 and positions past the
// block's end are 0.
__device__ __forceinline__ void octet_deltas(const BlockRef& br, int kmax, int j, int d[8]) {
  uint32_t mag[8];
  decode_mags_s(br.planes, br.rate, kmax, j, mag);
#pragma unroll
  for (int t = 0; t < 8; t++) {
    const int pos = 8 * j + t;
    const int v = ((br.sign_byte >> t) & 1u) ? -(int)mag[t] : (int)mag[t];
    d[t] = (pos == 0 || pos >= br.len) ? 0 : v;
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
  const int excl = octet_excl_scan(acc, j);
#pragma unroll
  for (int t = 0; t < 8; t++) q[t] = br.outlier + excl + s[t];
}

// Sanitize a freshly landed stage (rates past the end or above 31 become 0)
// and scan its rates. Whole CTA; `bad` collects HOSZP_ERR_FORMAT.
__device__ __forceinline__ void stage_begin(InStage& s, TileScan* ts, const Info& h,
                                            uint64_t tile, int& bad) {
  if (threadIdx.x < TILE) {
    const uint64_t b = tile * TILE + threadIdx.x;
    uint8_t r = s.rate[threadIdx.x];
    if (b >= h.nb) r = 0;
    if (r > MAX_RATE) {
      r = 0;
      bad = HOSZP_ERR_FORMAT;
    }
    s.rate[threadIdx.x] = r;
  }
  __syncthreads();
  tile_scan(s.rate, ts);
}

// Checks the pre-scan's totals against the header (a corrupt stream stops here).
__device__ __forceinline__ bool prescan_ok(const Info& h, const unsigned long long* pre,
                                           uint64_t max_tiles) {
  if (!h.ok) return false;
  const uint64_t nt = ntiles_of(h.nb);
  if (nt + 1 > max_tiles) return false;  // the pre-scan refused it (workspace bound)
  return pre[2 * nt] == h.nnc && pre[2 * nt + 1] == h.R;
}

// Static tile walk of one input stream with an S-stage bulk-copy ring: calls
// body(tile, stage, scan) for tiles blockIdx.x, +gridDim.x, ... Whole CTA.
template <int S, class Body>
__device__ __forceinline__ void consume_tiles(const uint8_t* c, const Info& h, uint64_t ntiles,
                                              const unsigned long long* pre, InStage* stages,
                                              uint64_t* bars, TileScan* ts, int* st, int& bad,
                                              Body&& body) {
  const uint64_t G = gridDim.x, first = blockIdx.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < S - 1; k++) {
      const uint64_t t = first + (uint64_t)k * G;
      if (t < ntiles) issue_in_tile(&stages[k], &bars[k], c, h, t, pre);
    }
  }
  for (uint64_t i = 0;; i++) {
    const uint64_t t = first + i * G;
    if (t >= ntiles) break;
    if (threadIdx.x == 0) {
      const uint64_t tn = first + (i + S - 1) * G;
      const int sn = (int)((i + S - 1) % S);
      if (tn < ntiles) issue_in_tile(&stages[sn], &bars[sn], c, h, tn, pre);
    }
    InStage& sg = stages[i % S];
    mbar_wait(&bars[i % S], (unsigned)((i / S) & 1), st);
    stage_begin(sg, ts, h, t, bad);
    body(t, sg, *ts);
    __syncthreads();
  }
}

template <int S>
__device__ __forceinline__ void init_bars(uint64_t* bars) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < S; k++) mbar_init(&bars[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

}  // namespace hz
