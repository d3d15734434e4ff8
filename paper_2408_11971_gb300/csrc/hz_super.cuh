// hz_super.cuh — input pipeline over super-tiles: a stage holds STB = 512
// consecutive blocks (8 tiles) of one stream and is filled by one loader warp
// with four bulk copies (rates, outliers, sign words, plane words). Compared
// with one stage per 64-block tile, the loader does an eighth of the work per
// byte: issuing a stage costs the loader several hundred cycles whatever its
// size, so stages must be large for one loader warp to keep HBM busy. The
// consumer warps (one per tile of the stage) find their blocks' sign and plane
// words themselves, from the tile's rates and the tile bases the loader writes
// into the stage.
#pragma once
#include <cstddef>

#include "hz_pipe.cuh"

namespace hz {

constexpr int STILES = 8;              // tiles per super-tile
constexpr int STB = STILES * TILE;     // blocks per super-tile

struct __align__(16) SStage {
  uint64_t sign[STB + 2];  // the super-tile's sign words, from a 16-byte boundary
  int outlier[STB];
  uint8_t rate[STB];       // as copied: read through tile_rates(), which sanitizes
  uint32_t sbase, pbase;   // index of the first sign / plane word in sign[] / its ring span
  uint32_t pring;          // ring word index where the plane copy starts
  uint32_t tnc[STILES];    // non-constant blocks of the super-tile before each tile
  uint32_t tr[STILES];     // plane words of the super-tile before each tile
  uint32_t pad[1];
};
static_assert(sizeof(uint64_t) * (STB + 2) % 16 == 0, "sign[] keeps alignment");
static_assert(sizeof(SStage) % 16 == 0, "stages stay 16-byte aligned");
static_assert(offsetof(SStage, sign) % 16 == 0 && offsetof(SStage, outlier) % 16 == 0 &&
                  offsetof(SStage, rate) % 16 == 0,
              "bulk-copy destinations are 16-byte aligned");

// Largest plane copy of one super-tile, in words (rate 31 everywhere, plus the
// rounding of both ends to 16 bytes).
constexpr uint32_t STILE_PLANE_WORDS_MAX = STB * MAX_RATE + 2;

__device__ __forceinline__ uint64_t nsuper_of(uint64_t ntiles) {
  return (ntiles + STILES - 1) / STILES;
}

// Byte ranges of super-tile s (blocks STB*s ..), from the pre-scan's {nc, r}
// prefixes at its first tile (pv0) and after its last tile (pv1).
struct SSpan {
  uint64_t sa16, pa16;
  unsigned rb, ob, sbytes, pbytes;
  uint32_t sbase, pbase;
  __device__ __forceinline__ uint32_t plane_words() const { return pbytes >> 3; }
};
__device__ __forceinline__ SSpan sspan(const Info& h, uint64_t s, ulonglong2 pv0, ulonglong2 pv1) {
  SSpan sp;
  const uint64_t b0 = (uint64_t)STB * s;
  const uint64_t rate_end = align16(h.nb), out_end = align16(4 * h.nb);
  sp.rb = (unsigned)umin64(STB, rate_end - b0);
  sp.ob = (unsigned)umin64(4 * STB, out_end - 4 * b0);
  const uint64_t sa = h.o_sign + 8 * pv0.x, se = h.o_sign + 8 * pv1.x;
  const uint64_t pa = h.o_plane + 8 * pv0.y, pe = h.o_plane + 8 * pv1.y;
  sp.sa16 = sa & ~15ull;
  sp.pa16 = pa & ~15ull;
  sp.sbytes = (pv1.x > pv0.x) ? (unsigned)(align16(se) - sp.sa16) : 0u;
  sp.pbytes = (pv1.y > pv0.y) ? (unsigned)(align16(pe) - sp.pa16) : 0u;
  // only a corrupt pre-scan (refused before any stage is issued) exceeds these
  if (sp.pbytes > 8u * STILE_PLANE_WORDS_MAX) sp.pbytes = 8u * STILE_PLANE_WORDS_MAX;
  if (sp.sbytes > 8u * (STB + 2)) sp.sbytes = 8u * (STB + 2);
  sp.sbase = (uint32_t)((sa - sp.sa16) >> 3);
  sp.pbase = (uint32_t)((pa - sp.pa16) >> 3);
  return sp;
}

// ---------------------------------------------------------------- in-kernel rate prefix
// The stream stores no per-block lengths (Sec. VI-B3), so finding a block's
// sign and plane words takes the prefix of all rates before it. CTA b takes
// the b-th of G contiguous ranges of super-tiles, sums the rates of its range
// per tile into shared memory and publishes the range total. Its loader then
// adds up the totals of ranges 0..b-1; a total that is not published within a
// few microseconds (its CTA may not be resident yet) is summed by the loader
// itself from the rate bytes, so no CTA ever depends on another being
// scheduled. The CTA then walks its range in order with a running prefix. No
// separate pre-scan launch is made.
constexpr int TS_MAX = 4096;  // tiles of one CTA's range (their sums live in shared memory)

struct SRange {
  uint64_t s0, s1;   // super-tiles [s0, s1) of this CTA
  uint32_t v;        // range index (= blockIdx.x)
};

// Grid for a stream of at most `tiles_bound` tiles: at least `persistent`
// CTAs, and enough that no range exceeds TS_MAX tiles.
__host__ __forceinline__ int range_grid(int persistent, uint64_t tiles_bound) {
  const uint64_t need = (tiles_bound + TS_MAX - 1) / TS_MAX;
  return (int)(need > (uint64_t)persistent ? need : (uint64_t)persistent);
}

// Rate sums of 16 rate bytes starting at block `b0` (a multiple of 16): the
// non-constant blocks and the rate sum, rates above 31 counting as 31 (as
// every decoder reads them) and raising `bad` to FORMAT.
__device__ __forceinline__ void rate_sums16(const uint8_t* c, const Info& h, uint64_t b0,
                                            uint32_t& nc, uint32_t& r, int& bad) {
  nc = 0;
  r = 0;
  if (b0 >= align16(h.nb)) return;
  const uint4 q = __ldg(reinterpret_cast<const uint4*>(c + HOSZP_HEADER_BYTES + b0));
  const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int k = 0; k < 16; k++) {
    uint32_t v = (w4[k >> 2] >> (8 * (k & 3))) & 0xffu;
    if (b0 + k >= h.nb) v = 0;
    if (v > MAX_RATE) {
      bad = HOSZP_ERR_FORMAT;
      v = MAX_RATE;
    }
    nc += v ? 1u : 0u;
    r += v;
  }
}

__device__ __forceinline__ SRange range_of(uint32_t v, uint64_t nst) {
  SRange rg;
  rg.v = v;
  const uint64_t G = gridDim.x;
  rg.s0 = nst * v / G;
  rg.s1 = nst * (v + 1) / G;
  return rg;
}

// All threads of the CTA: its range, the range's per-tile packed sums
// (non-constant blocks << 16 | rate sum) into s_ts, and the published range
// total.
__device__ __forceinline__ SRange range_sums(const uint8_t* c, const Info& h, uint64_t ntiles,
                                             uint64_t nst, uint32_t* s_ts, const Ws& ws,
                                             unsigned long long epoch, int& bad) {
  __shared__ unsigned long long s_tot[2][32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = (int)(blockDim.x >> 5);
  SRange rg = range_of(blockIdx.x, nst);
  const uint64_t t0 = (uint64_t)STILES * rg.s0, t1 = umin64((uint64_t)STILES * rg.s1, ntiles);
  unsigned long long tnc = 0, tr = 0;
  if (t1 > t0 + TS_MAX) {  // the host sizes the grid so that this never happens
    bad = HOSZP_ERR_CAPACITY;
    rg.s1 = rg.s0;
  } else {
    const int nq = (int)(4 * (t1 - t0));  // 16-byte quarters of the range's tiles
    for (int i = tid; i < ((nq + 31) & ~31); i += (int)blockDim.x) {
      uint32_t nc = 0, r = 0;
      if (i < nq) rate_sums16(c, h, TILE * (t0 + (uint64_t)(i >> 2)) + 16 * (uint64_t)(i & 3), nc, r, bad);
      uint32_t pk = (nc << 16) | r;  // a tile: nc <= 64, r <= 1984
      pk += __shfl_xor_sync(0xffffffffu, pk, 1);
      pk += __shfl_xor_sync(0xffffffffu, pk, 2);
      if (i < nq && (i & 3) == 0) {
        s_ts[i >> 2] = pk;
        tnc += pk >> 16;
        tr += pk & 0xffffu;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tnc += __shfl_xor_sync(0xffffffffu, tnc, o);
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
  }
  if (lane == 0) {
    s_tot[0][wid] = tnc;
    s_tot[1][wid] = tr;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long a = 0, b = 0;
    for (int k = 0; k < nw; k++) {
      a += s_tot[0][k];
      b += s_tot[1][k];
    }
    CtaAgg* g = ws.cta_agg + rg.v;
    g->nc = a;
    g->r = b;
    __threadfence();
    st_release(&g->flag, (epoch << 1) | 1ull);
  }
  return rg;
}

// Loader warp: the exclusive prefix (nc, r) of range v, summed from the
// published totals of ranges 0..v-1. A total still missing after about
// RANGE_POLL_NS is computed here from the rate bytes instead (whole warp).
constexpr unsigned long long RANGE_POLL_NS = 4000;
__device__ __forceinline__ void range_base(const uint8_t* c, const Info& h, uint64_t ntiles,
                                           uint64_t nst, const Ws& ws, uint32_t v,
                                           unsigned long long epoch, unsigned long long& bnc,
                                           unsigned long long& br, int& bad) {
  const int lane = threadIdx.x & 31;
  const unsigned long long want = (epoch << 1) | 1ull;
  unsigned long long a = 0, b = 0;
  const unsigned long long t0 = globaltimer_ns();
  for (uint32_t base = 0; base < v; base += 32) {
    const uint32_t u = base + lane;
    bool have = u >= v;
    if (!have) {
      const CtaAgg* g = ws.cta_agg + u;
      for (;;) {
        if (ld_acquire(&g->flag) == want) {
          a += *reinterpret_cast<const volatile unsigned long long*>(&g->nc);
          b += *reinterpret_cast<const volatile unsigned long long*>(&g->r);
          have = true;
          break;
        }
        if (globaltimer_ns() - t0 > RANGE_POLL_NS) break;
        __nanosleep(128);
      }
    }
    // ranges still missing: the whole warp sums them from the rate bytes
    unsigned int miss = __ballot_sync(0xffffffffu, !have);
    while (miss) {
      const int src = __ffs(miss) - 1;
      miss &= miss - 1;
      const SRange ru = range_of(base + src, nst);
      const uint64_t q0 = 4 * (uint64_t)STILES * ru.s0;
      const uint64_t q1 = 4 * umin64((uint64_t)STILES * ru.s1, ntiles);
      unsigned long long sa = 0, sb = 0;
      for (uint64_t q = q0 + lane; q < q1; q += 32) {
        uint32_t nc, r;
        rate_sums16(c, h, 16 * q, nc, r, bad);
        sa += nc;
        sb += r;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
      }
      if (lane == src) {
        a += sa;
        b += sb;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  bnc = a;
  br = b;
}

// Loader warp of a super-tile pipeline over the CTA's range [rg.s0, rg.s1):
// for stage use k = 0, 1, ... it waits for the release of use k - S
// (empty[k % S], released in order), then bulk-copies super-tile rg.s0 + k
// into stages[k % S] and its plane words into the ring; the copy completes on
// full[k % S]. stage_st[] gets the super-tile id, ~0 once the walk ends (one
// such end stage per consumer group, each completing without data). Offsets
// come from the range base and the tile sums in s_ts; a range whose words
// would run past the header's totals stops with FORMAT.
template <int S, uint32_t RW, int GROUPS>
__device__ __forceinline__ void super_loader(SStage* stages, uint64_t* ring, uint32_t* s_beg,
                                             uint64_t* full, uint64_t* empty,
                                             unsigned long long* stage_st, const uint8_t* c,
                                             const Info& h, const SRange& rg,
                                             const uint32_t* s_ts, const Ws& ws,
                                             unsigned long long epoch) {
  static_assert(RW >= STILE_PLANE_WORDS_MAX + 2, "the ring holds the largest super-tile");
  const int lane = threadIdx.x & 31;
  PlaneRing<S, RW> pr;
  pr.init(ring, s_beg);
  uint32_t k_rel = 0;
  auto release_one = [&]() {
    mbar_wait(&empty[k_rel % S], (k_rel / S) & 1, ws.status);
    k_rel++;
  };
  unsigned long long nc = 0, r = 0;
  int bad = 0;
  if (rg.s1 > rg.s0) range_base(c, h, ntiles_of(h.nb), nsuper_of(ntiles_of(h.nb)), ws, rg.v, epoch, nc, r, bad);
  if (bad && lane == 0) set_status(ws.status, bad);
  bool stop = false;
  int ends = 0;
  for (uint32_t k = 0; ends < GROUPS; k++) {
    const int sk = (int)(k % S);
    while (k_rel + S <= k) release_one();
    const uint64_t s = rg.s0 + k;
    // this super-tile's tile sums: lanes 0..STILES-1 hold one tile each
    uint32_t pk = 0;
    if (!stop && s < rg.s1 && lane < STILES && (uint64_t)STILES * s + lane < ntiles_of(h.nb))
      pk = s_ts[STILES * k + lane];  // tiles past the stream's end have no sums
    uint32_t inc = pk;
#pragma unroll
    for (int o = 1; o < STILES; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - pk;
    const uint32_t tot = __shfl_sync(0xffffffffu, inc, STILES - 1);
    const unsigned long long nc1 = nc + (tot >> 16), r1 = r + (tot & 0xffffu);
    if (!stop && s < rg.s1 && (nc1 > h.nnc || r1 > h.R)) {
      if (lane == 0) set_status(ws.status, HOSZP_ERR_FORMAT);
      stop = true;
    }
    if (stop || s >= rg.s1) {
      if (lane == 0) {
        stage_st[sk] = ~0ull;
        mbar_arrive(&full[sk]);
      }
      ends++;
      __syncwarp();
      continue;
    }
    const SSpan sp = sspan(h, s, make_ulonglong2(nc, r), make_ulonglong2(nc1, r1));
    const uint32_t p0 = pr.reserve(k, sp.plane_words(), k_rel, release_one);
    const uint32_t at = pr.commit(k, p0, sp.plane_words());
    SStage* sg = &stages[sk];
    if (lane < STILES) {
      sg->tnc[lane] = excl >> 16;
      sg->tr[lane] = excl & 0xffffu;
    }
    __syncwarp();  // the tile bases are ordered before lane 0's arrival on full[]
    if (lane == 0) {
      stage_st[sk] = s;
      sg->sbase = sp.sbase;
      sg->pbase = sp.pbase;
      sg->pring = at;
      fence_proxy_async();
      mbar_expect_tx(&full[sk], sp.rb + sp.ob + sp.sbytes + sp.pbytes);
      const uint64_t b0 = (uint64_t)STB * s;
      bulk_g2s(sg->rate, c + HOSZP_HEADER_BYTES + b0, sp.rb, &full[sk]);
      bulk_g2s(sg->outlier, c + h.o_out + 4 * b0, sp.ob, &full[sk]);
      if (sp.sbytes) bulk_g2s(sg->sign, c + sp.sa16, sp.sbytes, &full[sk]);
      if (sp.pbytes) bulk_g2s(ring + at, c + sp.pa16, sp.pbytes, &full[sk]);
    }
    __syncwarp();
    nc = nc1;
    r = r1;
  }
}

// Last CTA of a launch, one whole warp: the published range totals must add
// up to the header's (nnc, R); a stream whose rates disagree with its header
// is FORMAT. Every lane gets the answer.
__device__ __forceinline__ bool range_totals_ok(const Ws& ws, const Info& h) {
  const int lane = threadIdx.x & 31;
  unsigned long long a = 0, b = 0;
  for (unsigned int u = lane; u < gridDim.x; u += 32) {
    a += ws.cta_agg[u].nc;
    b += ws.cta_agg[u].r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  return a == h.nnc && b == h.R;
}

// A consumer warp's view of tile `ti` of a landed super-tile stage: lane l
// holds the sanitized rates of blocks 2l and 2l+1 (0 past the stream end,
// clamped to 31) and their exclusive in-tile prefixes of (non-constant
// blocks << 16 | plane words).
struct TileRates {
  uint32_t r0, r1;    // this lane's two rates
  uint32_t e0, e1;    // exclusive prefixes before blocks 2l and 2l+1
  int nvt;            // blocks of the tile inside the stream (0 .. 64)
};
__device__ __forceinline__ TileRates tile_rates(const SStage& sg, int ti, uint64_t tile,
                                                uint64_t nb) {
  const int lane = threadIdx.x & 31;
  TileRates tr;
  const uint64_t first = tile * TILE;
  tr.nvt = first < nb ? (int)umin64(TILE, nb - first) : 0;
  const uint32_t pair = reinterpret_cast<const uint16_t*>(sg.rate + TILE * ti)[lane];
  tr.r0 = (2 * lane < tr.nvt) ? min(pair & 0xffu, (uint32_t)MAX_RATE) : 0u;
  tr.r1 = (2 * lane + 1 < tr.nvt) ? min(pair >> 8, (uint32_t)MAX_RATE) : 0u;
  const uint32_t v0 = (tr.r0 ? 0x10000u : 0u) | tr.r0, v1 = (tr.r1 ? 0x10000u : 0u) | tr.r1;
  const uint32_t pv = v0 + v1;
  uint32_t inc = pv;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  tr.e0 = inc - pv;
  tr.e1 = tr.e0 + v0;
  return tr;
}
// Rate and exclusive prefix of block b (0..63) of the tile, from the lane
// holding it (every lane of the warp calls this with its own b).
__device__ __forceinline__ void tile_block(const TileRates& tr, int b, uint32_t& r,
                                           uint32_t& excl) {
  const int src = b >> 1;
  const uint32_t ra = __shfl_sync(0xffffffffu, tr.r0, src), rb = __shfl_sync(0xffffffffu, tr.r1, src);
  const uint32_t ea = __shfl_sync(0xffffffffu, tr.e0, src), eb = __shfl_sync(0xffffffffu, tr.e1, src);
  r = (b & 1) ? rb : ra;
  excl = (b & 1) ? eb : ea;
}

}  // namespace hz
