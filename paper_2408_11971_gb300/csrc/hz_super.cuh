// hz_super.cuh — input pipeline over super-tiles: a stage holds NT
// consecutive tiles (64 NT blocks) of one stream -- or of two streams with
// the same block count, for the bivariate operators -- and is filled by one
// loader warp with four bulk copies per stream (rates, outliers, sign words,
// plane words). Compared with one stage per 64-block tile, the loader does
// 1/NT of the work per byte: issuing a stage costs the loader several hundred
// cycles whatever its size, so stages must be large for one loader warp to
// keep HBM busy. The consumer warps find their blocks' sign and plane words
// themselves, from the tile's rates and the tile bases the loader writes into
// the stage.
#pragma once
#include <cstddef>

#include "hz_ws.cuh"

namespace hz {

template <int NT>
struct __align__(16) SStageT {
  uint64_t sign[NT * TILE + 2];  // the super-tile's sign words, from a 16-byte boundary
  int outlier[NT * TILE];
  uint8_t rate[NT * TILE];       // as copied: read through tile_rates(), which sanitizes
  uint32_t sbase, pbase;         // index of the first sign / plane word in sign[] / its ring span
  uint32_t pring;                // ring word index where the plane copy starts
  uint32_t tnc[NT];              // non-constant blocks of the super-tile before each tile
  uint32_t tr[NT];               // plane words of the super-tile before each tile
  unsigned long long bnc, br;    // the stream's prefix (non-constant blocks, words) at the stage
};

constexpr int STILES = 8;            // tiles per super-tile of the univariate kernels
constexpr int STB = STILES * TILE;   // blocks per super-tile
using SStage = SStageT<STILES>;

template <int NT>
struct SuperChecks {
  static_assert(sizeof(uint64_t) * (NT * TILE + 2) % 16 == 0, "sign[] keeps alignment");
  static_assert(sizeof(SStageT<NT>) % 16 == 0, "stages stay 16-byte aligned");
  static_assert(offsetof(SStageT<NT>, sign) % 16 == 0 && offsetof(SStageT<NT>, outlier) % 16 == 0 &&
                    offsetof(SStageT<NT>, rate) % 16 == 0,
                "bulk-copy destinations are 16-byte aligned");
  // Largest plane copy of one super-tile, in words (rate 31 everywhere, plus
  // the rounding of both ends to 16 bytes).
  static constexpr uint32_t kPlaneWordsMax = NT * TILE * MAX_RATE + 2;
};
constexpr uint32_t STILE_PLANE_WORDS_MAX = SuperChecks<STILES>::kPlaneWordsMax;

template <int NT = STILES>
__device__ __forceinline__ uint64_t nsuper_of(uint64_t ntiles) {
  return (ntiles + NT - 1) / NT;
}

// Byte ranges of super-tile s (blocks 64 NT s ..), from the {nc, r} prefixes
// of the stream at its first tile (pv0) and after its last tile (pv1).
struct SSpan {
  uint64_t sa16, pa16;
  unsigned rb, ob, sbytes, pbytes;
  uint32_t sbase, pbase;
  __device__ __forceinline__ uint32_t plane_words() const { return pbytes >> 3; }
};
template <int NT>
__device__ __forceinline__ SSpan sspan(const Info& h, uint64_t s, ulonglong2 pv0, ulonglong2 pv1) {
  constexpr int NB = NT * TILE;
  SSpan sp;
  const uint64_t b0 = (uint64_t)NB * s;
  const uint64_t rate_end = align16(h.nb), out_end = align16(4 * h.nb);
  sp.rb = (unsigned)umin64(NB, rate_end - b0);
  sp.ob = (unsigned)umin64(4 * NB, out_end - 4 * b0);
  const uint64_t sa = h.o_sign + 8 * pv0.x, se = h.o_sign + 8 * pv1.x;
  const uint64_t pa = h.o_plane + 8 * pv0.y, pe = h.o_plane + 8 * pv1.y;
  sp.sa16 = sa & ~15ull;
  sp.pa16 = pa & ~15ull;
  sp.sbytes = (pv1.x > pv0.x) ? (unsigned)(align16(se) - sp.sa16) : 0u;
  sp.pbytes = (pv1.y > pv0.y) ? (unsigned)(align16(pe) - sp.pa16) : 0u;
  // only a range that runs past the header's totals exceeds these, and the
  // loader refuses such a range before any copy
  if (sp.pbytes > 8u * SuperChecks<NT>::kPlaneWordsMax) sp.pbytes = 8u * SuperChecks<NT>::kPlaneWordsMax;
  if (sp.sbytes > 8u * (NB + 2)) sp.sbytes = 8u * (NB + 2);
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
// separate pre-scan launch is made. With NS streams (same block count), the
// totals of stream k of range v live at cta_agg[NS v + k].
// The sums of a range's first TS_MAX tiles are kept in shared memory; a range
// longer than that (a stream of billions of values) has the sums of its later
// tiles recomputed by the loader from the rate bytes, stage by stage.
constexpr int TS_MAX = 4096;

struct SRange {
  uint64_t s0, s1;   // super-tiles [s0, s1) of this CTA
  uint32_t v;        // range index (= blockIdx.x)
};

// Rate sums of 16 rate bytes starting at block `b0` (a multiple of 16): the
// non-constant blocks and the rate sum, rates above 31 counting as 31 (as
// every decoder reads them) and raising `bad` to FORMAT. rate_load16 fetches
// the bytes (zero past the rate section), rate_sum16 sums fetched bytes, so a
// caller can have several fetches in flight before summing.
__device__ __forceinline__ uint4 rate_load16(const uint8_t* c, const Info& h, uint64_t b0) {
  if (b0 >= align16(h.nb)) return make_uint4(0u, 0u, 0u, 0u);
  return __ldg(reinterpret_cast<const uint4*>(c + HOSZP_HEADER_BYTES + b0));
}
__device__ __forceinline__ void rate_sum16(uint4 q, const Info& h, uint64_t b0, uint32_t& nc,
                                           uint32_t& r, int& bad) {
  nc = 0;
  r = 0;
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
// (non-constant blocks << 16 | rate sum) of each of the NS streams into
// s_ts[k * ts_max ..], and the published range totals.
template <int NT, int NS>
__device__ __forceinline__ SRange range_sums_n(const uint8_t* const* c, const Info* h,
                                               uint64_t ntiles, uint64_t nst, uint32_t* s_ts,
                                               int ts_max, const Ws& ws, unsigned long long epoch,
                                               int& bad) {
  __shared__ unsigned long long s_tot[2 * NS][32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = (int)(blockDim.x >> 5);
  SRange rg = range_of(blockIdx.x, nst);
  const uint64_t t0 = (uint64_t)NT * rg.s0, t1 = umin64((uint64_t)NT * rg.s1, ntiles);
  unsigned long long tnc[NS], tr[NS];
#pragma unroll
  for (int k = 0; k < NS; k++) tnc[k] = tr[k] = 0;
  if constexpr (NS == 1) {
    // 16-byte quarters of the range's tiles; a single stream keeps two fetches
    // per thread in flight (one round trip for a 512^3 field's ranges)
    constexpr int INF = 2;
    const uint64_t nq = 4 * (t1 - t0);
    const uint64_t nq32 = (nq + 31) & ~31ull;
    const uint64_t bd = blockDim.x;
    for (uint64_t i0 = tid; i0 < nq32; i0 += INF * bd) {
      uint4 qv[INF][NS];
#pragma unroll
      for (int u = 0; u < INF; u++) {
        const uint64_t i = i0 + u * bd;
#pragma unroll
        for (int k = 0; k < NS; k++)
          qv[u][k] = (i < nq) ? rate_load16(c[k], h[k], TILE * (t0 + (i >> 2)) + 16 * (i & 3))
                              : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < INF; u++) {
        const uint64_t i = i0 + u * bd;
        if (i - lane >= nq32) break;  // warp-uniform: the warp's quarters are all past the end
#pragma unroll
        for (int k = 0; k < NS; k++) {
          uint32_t nc = 0, r = 0;
          if (i < nq) rate_sum16(qv[u][k], h[k], TILE * (t0 + (i >> 2)) + 16 * (i & 3), nc, r, bad);
          uint32_t pk = (nc << 16) | r;  // a tile: nc <= 64, r <= 1984
          pk += __shfl_xor_sync(0xffffffffu, pk, 1);
          pk += __shfl_xor_sync(0xffffffffu, pk, 2);
          if (i < nq && (i & 3) == 0) {
            if ((i >> 2) < (uint64_t)ts_max) s_ts[k * ts_max + (i >> 2)] = pk;
            tnc[k] += pk >> 16;
            tr[k] += pk & 0xffffu;
          }
        }
      }
    }
  } else {
    const uint64_t nq = 4 * (t1 - t0);  // 16-byte quarters of the range's tiles
    for (uint64_t i = tid; i < ((nq + 31) & ~31ull); i += blockDim.x) {
#pragma unroll
      for (int k = 0; k < NS; k++) {
        uint32_t nc = 0, r = 0;
        if (i < nq) rate_sums16(c[k], h[k], TILE * (t0 + (i >> 2)) + 16 * (i & 3), nc, r, bad);
        uint32_t pk = (nc << 16) | r;  // a tile: nc <= 64, r <= 1984
        pk += __shfl_xor_sync(0xffffffffu, pk, 1);
        pk += __shfl_xor_sync(0xffffffffu, pk, 2);
        if (i < nq && (i & 3) == 0) {
          if ((i >> 2) < (uint64_t)ts_max) s_ts[k * ts_max + (i >> 2)] = pk;
          tnc[k] += pk >> 16;
          tr[k] += pk & 0xffffu;
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NS; k++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tnc[k] += __shfl_xor_sync(0xffffffffu, tnc[k], o);
      tr[k] += __shfl_xor_sync(0xffffffffu, tr[k], o);
    }
    if (lane == 0) {
      s_tot[2 * k][wid] = tnc[k];
      s_tot[2 * k + 1][wid] = tr[k];
    }
  }
  __syncthreads();
  if (wid < NS) {  // warp k adds up stream k's per-warp totals
    unsigned long long a = (lane < nw) ? s_tot[2 * wid][lane] : 0ull;
    unsigned long long b = (lane < nw) ? s_tot[2 * wid + 1][lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      CtaAgg* g = ws.cta_agg + (uint64_t)NS * rg.v + wid;
      g->nc = a;
      g->r = b;
      __threadfence();
      st_release(&g->flag, (epoch << 1) | 1ull);
    }
  }
  return rg;
}

// Single-stream form (mean, variance, decompression).
__device__ __forceinline__ SRange range_sums(const uint8_t* c, const Info& h, uint64_t ntiles,
                                             uint64_t nst, uint32_t* s_ts, const Ws& ws,
                                             unsigned long long epoch, int& bad) {
  return range_sums_n<STILES, 1>(&c, &h, ntiles, nst, s_ts, TS_MAX, ws, epoch, bad);
}

// Loader warp: the exclusive prefix (nc, r) of stream k (of NS) at range v,
// summed from the published totals of ranges 0..v-1. A total still missing
// after about RANGE_POLL_NS is computed here from the rate bytes instead
// (whole warp).
constexpr unsigned long long RANGE_POLL_NS = 4000;
template <int NT, int NS>
__device__ __forceinline__ void range_base(const uint8_t* c, const Info& h, uint64_t ntiles,
                                           uint64_t nst, const Ws& ws, uint32_t v, int k,
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
      const CtaAgg* g = ws.cta_agg + (uint64_t)NS * u + k;
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
      const uint64_t q0 = 4 * (uint64_t)NT * ru.s0;
      const uint64_t q1 = 4 * umin64((uint64_t)NT * ru.s1, ntiles);
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

// Loader warp of a super-tile pipeline over the CTA's range [rg.s0, rg.s1) of
// NS streams with the same block count (c[k], h[k], tile sums at
// s_ts[k ts_max ..]). For stage use k = 0, 1, ... it waits for the release of
// use k - S (empty[k % S], released in order), then bulk-copies super-tile
// rg.s0 + k of stream q into stages[q S + k % S] and the plane words of all
// streams into one span of the ring (stream order); the copies complete on
// full[k % S]. stage_st[] gets the super-tile id, ~0 once the walk ends (one
// such end stage per consumer group, each completing without data). A range
// whose words would run past a header's totals stops with FORMAT.
template <int NT, int NS, int S, uint32_t RW, int GROUPS>
__device__ __forceinline__ void super_loader_n(SStageT<NT>* stages, uint64_t* ring,
                                               uint32_t* s_beg, uint64_t* full, uint64_t* empty,
                                               unsigned long long* stage_st,
                                               const uint8_t* const* c, const Info* h,
                                               const SRange& rg, const uint32_t* s_ts, int ts_max,
                                               const Ws& ws, unsigned long long epoch) {
  static_assert(RW >= NS * SuperChecks<NT>::kPlaneWordsMax + 2,
                "the ring holds the largest super-tile of every stream");
  static_assert(NT <= 16 && NS <= 2, "tile sums are spread over the warp's lanes");
  const int lane = threadIdx.x & 31;
  PlaneRing<S, RW> pr;
  pr.init(ring, s_beg);
  uint32_t k_rel = 0;
  bool dead = false;  // a wait gave up: issue nothing more, wait for nothing more
  auto release_one = [&]() {
    if (!dead && !mbar_wait_warp(&empty[k_rel % S], (k_rel / S) & 1, ws.status)) dead = true;
    k_rel++;
  };
  const uint64_t ntiles = ntiles_of(h[0].nb);
  const uint64_t nst = nsuper_of<NT>(ntiles);
  unsigned long long nc[NS], r[NS];
  int bad = 0;
#pragma unroll
  for (int k = 0; k < NS; k++) {
    nc[k] = r[k] = 0;
    if (rg.s1 > rg.s0)
      range_base<NT, NS>(c[k], h[k], ntiles, nst, ws, rg.v, k, epoch, nc[k], r[k], bad);
  }
  if (bad && lane == 0) set_status(ws.status, bad);
  bool stop = false;
  int ends = 0;
  uint32_t k_end = 0;  // stage uses issued so far
  // lanes 16q .. 16q + NT - 1 hold the tile sums of stream q
  const int ks = lane >> 4, ti = lane & 15;
  for (uint32_t k = 0; ends < GROUPS; k++) {
    const int sk = (int)(k % S);
    while (k_rel + S <= k) release_one();
    if (dead) break;  // no end markers either: a stage may still be in flight
    const uint64_t s = rg.s0 + k;
    uint32_t pk = 0;
    if (!stop && s < rg.s1 && ks < NS && ti < NT && (uint64_t)NT * s + ti < ntiles) {
      if (NT * k + ti < (uint32_t)ts_max) {
        pk = s_ts[ks * ts_max + NT * k + ti];  // tiles past the stream's end have no sums
      } else {  // beyond the sums kept: this tile's 64 rate bytes, read again
        for (int qq = 0; qq < 4; qq++) {
          uint32_t a, b;
          rate_sums16(c[ks], h[ks], TILE * ((uint64_t)NT * s + ti) + 16 * qq, a, b, bad);
          pk += (a << 16) | b;
        }
      }
    }
    uint32_t inc = pk;
#pragma unroll
    for (int o = 1; o < NT; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o, 16);
      if (ti >= o) inc += y;
    }
    const uint32_t excl = inc - pk;
    bool over = false;
    unsigned long long nc1[NS], r1[NS];
#pragma unroll
    for (int q = 0; q < NS; q++) {
      const uint32_t tot = __shfl_sync(0xffffffffu, inc, 16 * q + NT - 1);
      nc1[q] = nc[q] + (tot >> 16);
      r1[q] = r[q] + (tot & 0xffffu);
      over = over || nc1[q] > h[q].nnc || r1[q] > h[q].R;
    }
    if (!stop && s < rg.s1 && over) {
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
    SSpan sp[NS];
    uint32_t words[NS], all = 0;
#pragma unroll
    for (int q = 0; q < NS; q++) {
      sp[q] = sspan<NT>(h[q], s, make_ulonglong2(nc[q], r[q]), make_ulonglong2(nc1[q], r1[q]));
      words[q] = sp[q].plane_words();
      all += words[q];
    }
    const uint32_t p0 = pr.reserve(k, all, k_rel, release_one);
    if (dead) break;
    const uint32_t at = pr.commit(k, p0, all);
    if (ks < NS && ti < NT) {
      SStageT<NT>* sg = &stages[ks * S + sk];
      sg->tnc[ti] = excl >> 16;
      sg->tr[ti] = excl & 0xffffu;
    }
    __syncwarp();  // the tile bases are ordered before lane 0's arrival on full[]
    if (lane == 0) {
      stage_st[sk] = s;
      uint32_t tx = 0, a = at;
#pragma unroll
      for (int q = 0; q < NS; q++) {
        SStageT<NT>* sg = &stages[q * S + sk];
        sg->sbase = sp[q].sbase;
        sg->pbase = sp[q].pbase;
        sg->pring = a;
        sg->bnc = nc[q];
        sg->br = r[q];
        a += words[q];
        tx += sp[q].rb + sp[q].ob + sp[q].sbytes + sp[q].pbytes;
      }
      fence_proxy_async();
      mbar_expect_tx(&full[sk], tx);
      const uint64_t b0 = (uint64_t)NT * TILE * s;
      a = at;
#pragma unroll
      for (int q = 0; q < NS; q++) {
        SStageT<NT>* sg = &stages[q * S + sk];
        bulk_g2s(sg->rate, c[q] + HOSZP_HEADER_BYTES + b0, sp[q].rb, &full[sk]);
        bulk_g2s(sg->outlier, c[q] + h[q].o_out + 4 * b0, sp[q].ob, &full[sk]);
        if (sp[q].sbytes) bulk_g2s(sg->sign, c[q] + sp[q].sa16, sp[q].sbytes, &full[sk]);
        if (sp[q].pbytes) bulk_g2s(ring + a, c[q] + sp[q].pa16, sp[q].pbytes, &full[sk]);
        a += words[q];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NS; q++) {
      nc[q] = nc1[q];
      r[q] = r1[q];
    }
    k_end = k + 1;
  }
  // After a wait gave up, consumers may have left: the copies already issued
  // must land before the CTA exits (bounded waits; a use not yet released is
  // the last use of its stage, so its parity is unambiguous).
  if (dead)
    for (uint32_t u = k_rel; u < k_end; u++) mbar_wait(&full[u % S], (u / S) & 1, ws.status);
  if (bad) set_status(ws.status, bad);
}

// Single-stream form (mean, variance, decompression).
template <int S, uint32_t RW, int GROUPS>
__device__ __forceinline__ void super_loader(SStage* stages, uint64_t* ring, uint32_t* s_beg,
                                             uint64_t* full, uint64_t* empty,
                                             unsigned long long* stage_st, const uint8_t* c,
                                             const Info& h, const SRange& rg,
                                             const uint32_t* s_ts, const Ws& ws,
                                             unsigned long long epoch) {
  super_loader_n<STILES, 1, S, RW, GROUPS>(stages, ring, s_beg, full, empty, stage_st, &c, &h, rg,
                                           s_ts, TS_MAX, ws, epoch);
}

// Last CTA of a launch, one whole warp: the published range totals of stream
// k (of ns) must add up to its header's (nnc, R); a stream whose rates
// disagree with its header is FORMAT. Every lane gets the answer.
__device__ __forceinline__ bool range_totals_ok(const Ws& ws, const Info& h, int k = 0,
                                                int ns = 1) {
  const int lane = threadIdx.x & 31;
  unsigned long long a = 0, b = 0;
  for (unsigned int u0 = lane; u0 < gridDim.x; u0 += 32 * 4) {  // four records in flight
    unsigned long long x[4], y[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const unsigned int u = u0 + 32 * i;
      x[i] = (u < gridDim.x) ? ws.cta_agg[(uint64_t)ns * u + k].nc : 0ull;
      y[i] = (u < gridDim.x) ? ws.cta_agg[(uint64_t)ns * u + k].r : 0ull;
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
      a += x[i];
      b += y[i];
    }
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
template <class St>
__device__ __forceinline__ TileRates tile_rates(const St& sg, int ti, uint64_t tile, uint64_t nb) {
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
