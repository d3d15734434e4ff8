// hz_ws.cuh — warp-specialized tile pipeline shared by the codec kernels.
//
// A CTA has NCW = 16 compute warps (512 threads: 8 lanes per block of a
// 64-block tile) and loader warps: an issuer that bulk-copies the next tiles
// into a ring of shared-memory stages (plane words into a plane ring), and a
// preparer that readies each landed tile for the compute warps. The roles meet
// only on mbarriers: full[s] (copy landed), ready[s] (tile prepared) and
// empty[s] (all compute warps done with stage s). Compute warps never wait for
// each other, except once per produced tile (all 64 output rates must be known
// before any block's words can be placed).
#pragma once
#include "hz_decode.cuh"

namespace hz {

constexpr int NCW = 16;                       // compute warps
constexpr int LOADER_WARP = NCW;              // warp index of the first loader warp
constexpr int CONSUMER_THREADS = (NCW + 2) * 32;  // + issuer and preparer warps
constexpr int PRODUCER_THREADS = (NCW + 2) * 32;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// named barrier among the compute warps only
__device__ __forceinline__ void compute_bar() {
  asm volatile("bar.sync 1, %0;" ::"r"(NCW * 32) : "memory");
}

// Warp-redundant in-tile offsets: every compute warp scans the 64 rates of the
// tile itself (no CTA barrier). Returns, for block g of the tile, the number of
// non-constant blocks and the rate sum before it, and the tile totals.
// rates[] are read raw: a block past the stream end counts 0, a rate above 31
// counts 0 and raises `bad`.
struct TileOff {
  unsigned int nc_excl, r_excl, agg_nc, agg_r;
};

// A rate read from a stage: 0 past the stream end; clamped to 31, which keeps
// every index inside the stage arrays (sized for rate 31). A rate above 31 is
// a corrupt stream, which the rate pre-scan reports and which then yields no
// result, so clamping here only has to be memory-safe.
__device__ __forceinline__ unsigned int sane_rate(unsigned int r, uint64_t b, uint64_t nb,
                                                  int& bad) {
  (void)bad;
  return (b < nb) ? min(r, (unsigned int)MAX_RATE) : 0u;
}

__device__ __forceinline__ TileOff warp_tile_offsets(const uint8_t* rates, uint64_t tile,
                                                     uint64_t nb, int g, int& bad) {
  const int lane = threadIdx.x & 31;
  const uint64_t b0 = tile * TILE + 2 * lane;
  const unsigned int r0 = sane_rate(rates[2 * lane], b0, nb, bad);
  const unsigned int r1 = sane_rate(rates[2 * lane + 1], b0 + 1, nb, bad);
  // packed (nc << 16) | r: nc <= 64, r <= 1984 per tile
  const unsigned int v0 = (r0 ? 0x10000u : 0u) | r0;
  const unsigned int v1 = (r1 ? 0x10000u : 0u) | r1;
  const unsigned int pair = v0 + v1;
  unsigned int inc = pair;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const unsigned int excl0 = inc - pair;  // before block 2*lane
  const unsigned int excl1 = excl0 + v0;  // before block 2*lane+1
  const unsigned int total = __shfl_sync(0xffffffffu, inc, 31);
  const unsigned int e0 = __shfl_sync(0xffffffffu, excl0, g >> 1);
  const unsigned int e1 = __shfl_sync(0xffffffffu, excl1, g >> 1);
  const unsigned int e = (g & 1) ? e1 : e0;
  TileOff t;
  t.nc_excl = e >> 16;
  t.r_excl = e & 0xffffu;
  t.agg_nc = total >> 16;
  t.agg_r = total & 0xffffu;
  return t;
}

// Block view for an octet of a prepared stage (see prepare_tile).
__device__ __forceinline__ BlockRef block_ref_s(const InStage& s, const uint64_t* ring, int g,
                                                int j) {
  BlockRef br;
  br.rate = s.rate[g];
  br.outlier = s.outlier[g];
  const uint32_t off = s.off[g];
  br.planes = ring + s.pring + s.pbase + (off & 0xffffu);
  br.sign_byte = br.rate ? reinterpret_cast<const uint8_t*>(s.sign + s.sbase + (off >> 16))[j] : 0u;
  const int nv = (int)s.nvalid;
  br.len = (g < nv - 1) ? L : ((g == nv - 1) ? (int)s.lastlen : 0);
  return br;
}

// Loader warp, after tile t's copy into `s` has landed: sanitize the rates
// (0 past the stream end; clamped to 31, which keeps every index inside the
// stage arrays -- a rate above 31 is a corrupt stream, reported by the rate
// pre-scan, and then no result is produced), write each block's in-tile
// offsets, the plane groups per warp of 4 blocks, and the tile's extent.
// All 32 lanes; lane l handles blocks 2l and 2l+1.
__device__ __forceinline__ void prepare_tile(InStage& s, uint64_t t, const Info& h) {
  const int lane = threadIdx.x & 31;
  const uint64_t first = t * TILE;
  const uint32_t nv = (uint32_t)umin64(TILE, h.nb - first);
  const uint32_t pair = reinterpret_cast<const uint16_t*>(s.rate)[lane];
  uint32_t r0 = pair & 0xffu, r1 = pair >> 8;
  r0 = (2u * lane < nv) ? min(r0, (uint32_t)MAX_RATE) : 0u;
  r1 = (2u * lane + 1 < nv) ? min(r1, (uint32_t)MAX_RATE) : 0u;
  reinterpret_cast<uint16_t*>(s.rate)[lane] = (uint16_t)(r0 | (r1 << 8));
  const uint32_t v0 = (r0 ? 0x10000u : 0u) | r0, v1 = (r1 ? 0x10000u : 0u) | r1;
  const uint32_t pv = v0 + v1;
  uint32_t inc = pv;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  s.off[2 * lane] = inc - pv;
  s.off[2 * lane + 1] = inc - pv + v0;
  uint32_t km = (max(r0, r1) + 7) >> 3;
  km = max(km, __shfl_xor_sync(0xffffffffu, km, 1));
  if ((lane & 1) == 0) s.kmx[lane >> 1] = (uint8_t)km;
  if (lane == 0) {
    s.nvalid = nv;
    s.lastlen = (uint32_t)umin64(L, h.n - (first + nv - 1) * L);
  }
}

// ---------------------------------------------------------------- input ring
struct Ring {
  uint64_t* full;
  uint64_t* empty;
};

template <int S>
__device__ __forceinline__ void ring_init(uint64_t* full, uint64_t* empty) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < S; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Ring of S stages with three barriers per stage: full (bulk copy landed),
// ready (loader warp prepared it), empty (all EMPTY_ARRIVALS compute warps done
// with it).
template <int S, int FULL_ARRIVALS = 1, int EMPTY_ARRIVALS = NCW>
__device__ __forceinline__ void ring_init3(uint64_t* full, uint64_t* ready, uint64_t* empty) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < S; k++) {
      mbar_init(&full[k], FULL_ARRIVALS);
      mbar_init(&ready[k], 1);
      mbar_init(&empty[k], EMPTY_ARRIVALS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Loader warps of a tile pipeline: two warps, so that copying and preparing
// never wait for each other.
//  - issuer (role 0): walks tiles next_tile(0), next_tile(1), ...; before
//    stage use k it waits for the release of use k - S (all compute warps
//    arrived on empty[k % S]; releases are consumed in order, k_rel counts
//    them), then calls issue(s, t, k, k_rel, release_one) with the whole warp
//    (lane 0 issues the copies; a plane ring may wait for further releases
//    through release_one). stage_tile[s] gets the tile id; an id >= ntiles ends
//    the walk (its stage completes without data). With GROUPS compute groups
//    taking stage uses in turn, GROUPS such end stages are made.
//  - preparer (role 1): for each stage use in order, waits for the copy to
//    land, prepares the tile (prepare(s, t), whole warp) and arrives on
//    ready[s], which the compute warps wait for.
template <int S, int FULL_ARRIVALS = 1, int GROUPS = 1, class NextTile, class Issue,
          class Prepare>
__device__ __forceinline__ void loader_warps(int role, unsigned long long* stage_tile,
                                             uint64_t* full, uint64_t* ready, uint64_t* empty,
                                             uint64_t ntiles, int* st, NextTile&& next_tile,
                                             Issue&& issue, Prepare&& prepare) {
  const int lane = threadIdx.x & 31;
  if (role == 0) {
    uint32_t k_rel = 0;  // stage uses released
    auto release_one = [&]() {
      mbar_wait(&empty[k_rel % S], (k_rel / S) & 1, st);
      k_rel++;
    };
    int ends = 0;
    for (uint32_t k = 0; ends < GROUPS; k++) {
      const int sk = (int)(k % S);
      while (k_rel + S <= k) release_one();  // the stage's previous use is done
      const unsigned long long t = next_tile(k);  // same value in every lane
      if (lane == 0) stage_tile[sk] = t;
      __syncwarp();
      if (t < ntiles) {
        issue(sk, t, k, k_rel, release_one);
      } else {
        if (lane == 0)
          for (int a = 0; a < FULL_ARRIVALS; a++) mbar_arrive(&full[sk]);
        ends++;
      }
    }
  } else {
    int ends = 0;
    for (uint32_t k = 0; ends < GROUPS; k++) {
      const int sk = (int)(k % S);
      mbar_wait(&full[sk], (k / S) & 1, st);
      const unsigned long long t = stage_tile[sk];
      if (t < ntiles) prepare(sk, t);
      else ends++;
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[sk]);
    }
  }
}

// Single loader warp for pipelines whose tiles need no preparation: the
// compute warps wait on full[] directly.
template <int S, class NextTile, class Issue>
__device__ __forceinline__ void issuer_warp(unsigned long long* stage_tile, uint64_t* full,
                                            uint64_t* empty, uint64_t ntiles, int* st,
                                            NextTile&& next_tile, Issue&& issue) {
  const int lane = threadIdx.x & 31;
  for (uint32_t k = 0;; k++) {
    const int sk = (int)(k % S);
    if (k >= (uint32_t)S) mbar_wait(&empty[sk], ((k / S) - 1) & 1, st);
    const unsigned long long t = next_tile(k);
    if (lane == 0) stage_tile[sk] = t;
    __syncwarp();
    if (t < ntiles) {
      issue(sk, t);
    } else {
      if (lane == 0) mbar_arrive(&full[sk]);
      return;
    }
  }
}

// Compute-warp side of the ring: stage index and barrier parity.
struct RingPos {
  int s;
  uint32_t par;
  template <int S>
  __device__ __forceinline__ void next() {
    if (++s == S) {
      s = 0;
      par ^= 1u;
    }
  }
};

// ---------------------------------------------------------------- produced tiles
// A produced tile goes to its own slot of the workspace: [sign words | plane
// words] in block order, starting at word slot_off (an upper bound of the
// words of all earlier tiles, known before the tile is computed). Rates and
// outliers go straight to the stream (their positions depend only on the block
// index). The tile's aggregate (non-constant blocks, rate sum) goes to agg[t];
// a scan of the aggregates and the placement kernel then move every slot to
// its final place. No compute warp ever waits for another CTA.
//
// Compute warps: all 16 call this once per tile, in order (kth = k-th tile of
// the CTA); srate is a double-buffered 2 x 64 shared array.
__device__ __forceinline__ void produce_tile(uint8_t (*srate)[TILE], uint64_t kth,
                                             unsigned long long tile, uint64_t nb,
                                             const uint32_t mag[8], uint32_t sb, int rate,
                                             int outlier, bool valid, int g, int j,
                                             uint8_t* __restrict__ out, uint64_t* slots,
                                             uint64_t slot_off, uint64_t slot_words,
                                             unsigned long long* agg, const OctetSel& S,
                                             int& bad) {
  uint8_t* rr = srate[kth & 1];
  const uint64_t b = tile * TILE + g;
  if (j == 0) {
    rr[g] = valid ? (uint8_t)rate : 0;
    if (valid) {
      out[HOSZP_HEADER_BYTES + b] = (uint8_t)rate;
      reinterpret_cast<int*>(out + off_outlier(nb))[b] = outlier;
    }
  }
  compute_bar();
  const TileOff off = warp_tile_offsets(rr, 0, TILE, g, bad);
  const int r = valid ? rate : 0;
  if (slot_off + off.agg_nc + off.agg_r > slot_words) {
    bad = HOSZP_ERR_CAPACITY;
    return;
  }
  uint64_t* slot = slots + slot_off;
  if (r > 0) reinterpret_cast<uint8_t*>(slot + off.nc_excl)[j] = (uint8_t)sb;
  const int kmax = __reduce_max_sync(0xffffffffu, (r + 7) >> 3);
  if (kmax > 0)
    encode_planes(mag, r, kmax, j, slot + off.agg_nc + off.r_excl, S);
  if (threadIdx.x == 0) agg[tile] = ((unsigned long long)off.agg_nc << 32) | off.agg_r;
}

// Word offset of tile t's slot: an upper bound of the words all earlier tiles
// can produce. Rule COMPRESS: 25 words per block (rate <= 24). Rule ADD: the
// inputs' words (a block of A+B needs at most the words of A's and B's block).
// Rule MUL: (1 + e) words per non-constant input block plus the input's plane
// words (a constant block stays constant; a rate grows by at most e bits).
// Rule EXPLICIT: the producer wrote each tile's slot offset into pre0[2t].
// Rule FULL: 32 words per block (a sign word and 31 planes), for products of
// two fields, whose rates the inputs' rates do not bound.
// Rule SPLIT: a tile's sign words and plane words sit in two separate slots,
// whose word offsets the producer wrote into pre0[2t] (signs) and pre0[2t+1]
// (planes); a producer that finds its tile's sign count only at the tile's end
// can then write both kinds as it goes.
enum SlotRule { SLOT_COMPRESS = 0, SLOT_ADD = 1, SLOT_MUL = 2, SLOT_EXPLICIT = 3, SLOT_FULL = 4,
                SLOT_SPLIT = 5 };

__device__ __forceinline__ uint64_t slot_offset(int rule, uint64_t t,
                                                const unsigned long long* pre0,
                                                const unsigned long long* pre1, uint32_t e) {
  if (rule == SLOT_COMPRESS) return (uint64_t)TILE * 25 * t;
  if (rule == SLOT_FULL) return (uint64_t)TILE * 32 * t;
  if (rule == SLOT_ADD) return pre0[2 * t] + pre0[2 * t + 1] + pre1[2 * t] + pre1[2 * t + 1];
  if (rule == SLOT_EXPLICIT) return pre0[2 * t];
  return pre0[2 * t] * (1ull + e) + pre0[2 * t + 1];
}

// ---------------------------------------------------------------- producer header and qbound
__device__ __forceinline__ void write_template(const Info& h, uint32_t qbound_fixed,
                                               const Ws& ws) {
  hoszp_header* H = ws.hdr;
  H->magic = HOSZP_MAGIC;
  H->version = HOSZP_VERSION;
  H->dtype = 0;
  H->ndims = (uint8_t)h.ndims;
  H->dims[0] = h.dims[0];
  H->dims[1] = h.dims[1];
  H->dims[2] = h.dims[2];
  H->eps_q = h.eps_q;
  H->n = h.n;
  H->eps = h.eps;
  H->nnc = 0;
  H->R = 0;
  H->qbound = qbound_fixed;
  H->block = HOSZP_BLOCK;
}

__device__ __forceinline__ void reduce_qmax(uint32_t qmax, const Ws& ws) {
  __shared__ uint32_t s_q[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  if ((threadIdx.x & 31) == 0) s_q[threadIdx.x >> 5] = qmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) qmax = max(qmax, s_q[w]);
    atomicMax(&ws.totals[2], (unsigned long long)qmax);
  }
}

}  // namespace hz
