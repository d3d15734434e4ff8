// scan.cu — rate pre-scan of a compressed stream: the exclusive prefix of
// (non-constant blocks, rate sum) at every tile of 64 blocks. With it a tile's
// sign and plane words can be located (and bulk-copied) before anything of the
// tile is decoded; without it, every block's position depends on all rates
// before it (the stream stores no per-block lengths, Sec. VI-B3).
#include "hz_kernels.cuh"

namespace hz {

constexpr int SCAN_THREADS = 256;
constexpr int SUPER_TILES = 64;                    // tiles per CTA step
constexpr int SUPER_BLOCKS = SUPER_TILES * TILE;   // 4096 rate bytes, 16 per thread

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const uint8_t* __restrict__ c,
                                                       uint64_t c_bytes,
                                                       unsigned long long* __restrict__ pre,
                                                       Desc* chain, Ws ws) {
  __shared__ unsigned int s_nc[SUPER_TILES], s_r[SUPER_TILES];
  __shared__ unsigned int s_xnc[SUPER_TILES], s_xr[SUPER_TILES];
  __shared__ unsigned long long s_pre[2];
  __shared__ unsigned int s_tile;
  __shared__ unsigned long long s_epoch;
  const int tid = threadIdx.x;
  const Info h = parse_header(c, c_bytes);
  int bad = h.ok ? 0 : HOSZP_ERR_FORMAT;
  uint64_t ntiles = h.ok ? ntiles_of(h.nb) : 0;
  // pre[] holds 2 (max_tiles) words: a stream claiming more tiles than the
  // caller's sizes allow (a header n larger than the n passed to decompress)
  // is refused before anything is written
  if (ntiles + 1 > ws.max_tiles) {
    bad = HOSZP_ERR_MISMATCH;
    ntiles = 0;
  }
  const uint64_t nsuper = (ntiles + SUPER_TILES - 1) / SUPER_TILES;
  const uint64_t rate_end = align16(h.nb);
  if (tid == 0) s_epoch = launch_epoch(ws);
  if (h.ok && h.nb == 0 && blockIdx.x == 0 && tid == 0) {
    pre[0] = 0;
    pre[1] = 0;
    if (h.nnc != 0 || h.R != 0) bad = HOSZP_ERR_FORMAT;
  }
  __syncthreads();
  const unsigned long long epoch = s_epoch;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&ws.sync->ticket, 1u);
    __syncthreads();
    const uint64_t st = s_tile;
    if (st >= nsuper) break;
    const uint64_t b0 = st * SUPER_BLOCKS + 16 * (uint64_t)tid;
    unsigned int nc = 0, rs = 0;
    if (b0 < rate_end) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(c + HOSZP_HEADER_BYTES + b0));
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 16; k++) {
        unsigned int r = (w[k >> 2] >> (8 * (k & 3))) & 0xffu;
        if (b0 + k >= h.nb) r = 0;
        if (r > MAX_RATE) {
          bad = HOSZP_ERR_FORMAT;
          r = 0;
        }
        nc += r ? 1u : 0u;
        rs += r;
      }
    }
    // 4 threads per tile
    nc += __shfl_xor_sync(0xffffffffu, nc, 1);
    rs += __shfl_xor_sync(0xffffffffu, rs, 1);
    nc += __shfl_xor_sync(0xffffffffu, nc, 2);
    rs += __shfl_xor_sync(0xffffffffu, rs, 2);
    if ((tid & 3) == 0) {
      s_nc[tid >> 2] = nc;
      s_r[tid >> 2] = rs;
    }
    __syncthreads();
    if (tid < 64) {  // exclusive scan over the 64 tiles (two warps, then combine)
      const int lane = tid & 31;
      unsigned int a = s_nc[tid], b = s_r[tid], pa = a, pb = b;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned int ya = __shfl_up_sync(0xffffffffu, pa, o);
        unsigned int yb = __shfl_up_sync(0xffffffffu, pb, o);
        if (lane >= o) { pa += ya; pb += yb; }
      }
      s_xnc[tid] = pa - a;
      s_xr[tid] = pb - b;
    }
    __syncthreads();
    if (tid >= 32 && tid < 64) {
      s_xnc[tid] += s_xnc[31] + s_nc[31];
      s_xr[tid] += s_xr[31] + s_r[31];
    }
    __syncthreads();
    const unsigned int agg_nc = s_xnc[63] + s_nc[63], agg_r = s_xr[63] + s_r[63];
    tile_prefix(chain, (int64_t)st, epoch, ws.status, agg_nc, agg_r, 0, s_pre);
    __syncthreads();
    if (tid < SUPER_TILES) {
      const uint64_t t = st * SUPER_TILES + tid;
      if (t < ntiles) {
        pre[2 * t] = s_pre[0] + s_xnc[tid];
        pre[2 * t + 1] = s_pre[1] + s_xr[tid];
      }
    }
    if (st == nsuper - 1 && tid == 0) {
      const unsigned long long tnc = s_pre[0] + agg_nc, tr = s_pre[1] + agg_r;
      pre[2 * ntiles] = tnc;
      pre[2 * ntiles + 1] = tr;
      if (tnc != h.nnc || tr != h.R) bad = HOSZP_ERR_FORMAT;
    }
    __syncthreads();
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

cudaError_t launch_scan(const Launch& lc, const uint8_t* c, uint64_t c_bytes,
                        unsigned long long* pre, Ws ws) {
  k_scan<<<persistent_grid(k_scan, SCAN_THREADS, lc.grid), SCAN_THREADS, 0, lc.stream>>>(
      c, c_bytes, pre, ws.desc[2], ws);
  return cudaGetLastError();
}

}  // namespace hz

namespace hz {

// ---------------------------------------------------------------- produced-tile scan
// Exclusive prefix over the produced tiles' aggregates (agg[t] = nc << 32 | r,
// written by the producer kernel) into opre[], and the stream totals into
// totals[0] (non-constant blocks) and totals[1] (rate sum).
constexpr int SA_THREADS = 256;
constexpr int SA_PER_THREAD = 16;
constexpr int SA_SUPER = SA_THREADS * SA_PER_THREAD;  // tiles per CTA step

__global__ void __launch_bounds__(SA_THREADS) k_scan_agg(Ws ws, uint64_t ntiles_given) {
  __shared__ unsigned long long s_w[SA_THREADS / 32];
  __shared__ unsigned long long s_pre[2];
  __shared__ unsigned int s_tile;
  __shared__ unsigned long long s_epoch;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // the produced stream's tiles, or (batched producers) the global tile space
  uint64_t ntiles = ntiles_given ? ntiles_given : ntiles_of(nblocks(ws.hdr->n));
  int bad = 0;
  if (ntiles + 1 > ws.max_tiles) {
    bad = HOSZP_ERR_CAPACITY;
    ntiles = 0;
  }
  const uint64_t nsuper = (ntiles + SA_SUPER - 1) / SA_SUPER;
  if (tid == 0) s_epoch = launch_epoch(ws);
  if (ntiles == 0 && blockIdx.x == 0 && tid == 0) {
    ws.opre[0] = 0;
    ws.opre[1] = 0;
    ws.totals[0] = 0;
    ws.totals[1] = 0;
  }
  __syncthreads();
  const unsigned long long epoch = s_epoch;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&ws.sync->ticket, 1u);
    __syncthreads();
    const uint64_t st = s_tile;
    if (st >= nsuper) break;
    const uint64_t t0 = st * SA_SUPER + (uint64_t)SA_PER_THREAD * tid;
    unsigned long long v[SA_PER_THREAD];
    unsigned long long sum = 0;  // packed (nc << 32) | r, both fields stay below 2^32
#pragma unroll
    for (int k = 0; k < SA_PER_THREAD; k++) {
      v[k] = (t0 + k < ntiles) ? ws.agg[t0 + k] : 0ull;
      sum += v[k];
    }
    unsigned long long inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    unsigned long long wbase = 0, total = 0;
    for (int k = 0; k < SA_THREADS / 32; k++) {
      if (k < wid) wbase += s_w[k];
      total += s_w[k];
    }
    tile_prefix(ws.desc[2], (int64_t)st, epoch, ws.status, (unsigned int)(total >> 32),
                (unsigned int)(total & 0xffffffffu), 0, s_pre);
    __syncthreads();
    unsigned long long run = wbase + inc - sum;  // exclusive, within the super-tile
    const unsigned long long pnc = s_pre[0], pr = s_pre[1];
#pragma unroll
    for (int k = 0; k < SA_PER_THREAD; k++) {
      const uint64_t t = t0 + k;
      if (t < ntiles) {
        ws.opre[2 * t] = pnc + (run >> 32);
        ws.opre[2 * t + 1] = pr + (run & 0xffffffffull);
      }
      run += v[k];
    }
    if (st == nsuper - 1 && tid == 0) {
      const unsigned long long tnc = pnc + (total >> 32), tr = pr + (total & 0xffffffffull);
      ws.opre[2 * ntiles] = tnc;
      ws.opre[2 * ntiles + 1] = tr;
      ws.totals[0] = tnc;
      ws.totals[1] = tr;
    }
    __syncthreads();
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

cudaError_t launch_scan_agg(const Launch& lc, Ws ws, uint64_t ntiles_given) {
  k_scan_agg<<<persistent_grid(k_scan_agg, SA_THREADS, lc.grid), SA_THREADS, 0, lc.stream>>>(
      ws, ntiles_given);
  return cudaGetLastError();
}

}  // namespace hz
