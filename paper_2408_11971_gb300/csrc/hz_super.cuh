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

// Loader warp of a super-tile pipeline: walks super-tiles next(k) for stage
// uses k = 0, 1, ...; before use k it waits for the release of use k - S
// (empty[k % S], released in order), then bulk-copies the super-tile into
// stages[k % S] and its plane words into the ring; the copy completes on
// full[k % S]. stage_st[] gets the super-tile id, ~0 once the walk ends (one
// such end stage per consumer group, each completing without data).
// The pre-scan prefixes of the loader's next 32 super-tiles are fetched with
// one warp-wide load into `win` (STILES + 1 tile boundaries each).
template <int S, uint32_t RW, int GROUPS, class Next>
__device__ __forceinline__ void super_loader(SStage* stages, uint64_t* ring, uint32_t* s_beg,
                                             ulonglong2 (*win)[STILES + 1], uint64_t* full,
                                             uint64_t* empty, unsigned long long* stage_st,
                                             const uint8_t* c, const Info& h,
                                             const unsigned long long* pre, uint64_t ntiles,
                                             uint64_t nst, int* st, Next&& next) {
  static_assert(RW >= STILE_PLANE_WORDS_MAX + 2, "the ring holds the largest super-tile");
  const int lane = threadIdx.x & 31;
  PlaneRing<S, RW> pr;
  pr.init(ring, s_beg);
  uint32_t k_rel = 0;
  auto release_one = [&]() {
    mbar_wait(&empty[k_rel % S], (k_rel / S) & 1, st);
    k_rel++;
  };
  uint64_t k0 = ~0ull;
  int ends = 0;
  for (uint32_t k = 0; ends < GROUPS; k++) {
    const int sk = (int)(k % S);
    while (k_rel + S <= k) release_one();
    const uint64_t s = next(k);
    if (s >= nst) {
      if (lane == 0) {
        stage_st[sk] = ~0ull;
        mbar_arrive(&full[sk]);
      }
      ends++;
      continue;
    }
    if (k0 == ~0ull || k >= k0 + 32) {  // refill the prefix window
      k0 = k;
      const uint64_t sl = next(k0 + lane);
      __syncwarp();
      if (sl < nst) {
#pragma unroll
        for (int i = 0; i <= STILES; i++) {
          const uint64_t t = umin64((uint64_t)STILES * sl + i, ntiles);
          win[lane][i] = __ldg(reinterpret_cast<const ulonglong2*>(pre + 2 * t));
        }
      }
      __syncwarp();
    }
    const ulonglong2* pv = win[k - k0];
    const SSpan sp = sspan(h, s, pv[0], pv[STILES]);
    const uint32_t p0 = pr.reserve(k, sp.plane_words(), k_rel, release_one);
    const uint32_t at = pr.commit(k, p0, sp.plane_words());
    if (lane == 0) {
      SStage* sg = &stages[sk];
      stage_st[sk] = s;
      sg->sbase = sp.sbase;
      sg->pbase = sp.pbase;
      sg->pring = at;
#pragma unroll
      for (int i = 0; i < STILES; i++) {
        sg->tnc[i] = (uint32_t)(pv[i].x - pv[0].x);
        sg->tr[i] = (uint32_t)(pv[i].y - pv[0].y);
      }
      fence_proxy_async();
      mbar_expect_tx(&full[sk], sp.rb + sp.ob + sp.sbytes + sp.pbytes);
      const uint64_t b0 = (uint64_t)STB * s;
      bulk_g2s(sg->rate, c + HOSZP_HEADER_BYTES + b0, sp.rb, &full[sk]);
      bulk_g2s(sg->outlier, c + h.o_out + 4 * b0, sp.ob, &full[sk]);
      if (sp.sbytes) bulk_g2s(sg->sign, c + sp.sa16, sp.sbytes, &full[sk]);
      if (sp.pbytes) bulk_g2s(ring + at, c + sp.pa16, sp.pbytes, &full[sk]);
    }
    __syncwarp();
  }
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
