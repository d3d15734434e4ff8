// hz_pipe.cuh — tile pipelines: 1-D TMA bulk copies (cp.async.bulk) of a
// compressed tile into a shared-memory ring completed on mbarriers, and the
// shared-memory output stage of a produced tile.
#pragma once
#include <cstddef>

#include "hz_common.cuh"

namespace hz {

// ---------------------------------------------------------------- mbarrier / bulk copy
constexpr unsigned long long MBAR_TIMEOUT_NS = 1000000000ull;  // a wait gives up after 1 s
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: after about a second the status word gets TIMEOUT and the wait
// gives up (the data in the stage is then not used for a valid result). The
// clock is read once per 256 polls.
// Returns false when the wait gave up (status TIMEOUT set): callers then stop
// their loops, so a stalled pipeline costs about a second, not a second per
// remaining stage.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* st,
                                          unsigned long long timeout_ns = MBAR_TIMEOUT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned spins = 1;; spins++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spins & 255u) == 0 && globaltimer_ns() - t0 > timeout_ns) {
      set_status(st, HOSZP_ERR_TIMEOUT);
      return false;
    }
  }
}
// The same for a whole warp, with one answer for all its lanes (each lane
// times out on its own clock).
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, unsigned parity, int* st) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, st));
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// global -> shared bulk copy of `bytes` (multiple of 16, both ends 16-aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------- input stage
// One tile of an input stream in shared memory: its rates, outliers and sign
// words in a fixed-size stage, its plane words (anywhere from 0 to 64 x 31
// words) in a per-CTA plane ring (PlaneRing) where each tile takes only the
// words it has. Sign and plane words are copied from the 16-byte-aligned
// addresses around the tile's words; sbase and pbase give the index of the
// tile's first word inside sign[] and inside its ring span starting at pring.
struct __align__(16) InStage {
  uint64_t sign[TILE + 2];
  int outlier[TILE];
  uint8_t rate[TILE];  // bulk-copied; then sanitized by the loader warp
  uint32_t sbase, pbase;
  uint32_t pring;  // ring word index where the tile's plane copy starts
  // written by the loader warp once the copy has landed (see prepare_tile):
  uint32_t off[TILE];              // (non-constant blocks before << 16) | rate sum before
  uint8_t kmx[TILE / 4];           // plane groups (ceil(rate/8)) to decode, per warp of 4 blocks
  uint32_t nvalid;                 // blocks of the tile inside the stream
  uint32_t lastlen;                // values in block nvalid-1
};
static_assert(sizeof(uint64_t) * (TILE + 2) % 16 == 0, "sign[] keeps alignment");
static_assert(sizeof(InStage) % 16 == 0, "ring stages must stay 16-byte aligned (bulk copies)");
static_assert(TILE == 64, "prepare_tile scans 64 blocks with one warp (2 per lane)");
static_assert(offsetof(InStage, sign) % 16 == 0 && offsetof(InStage, outlier) % 16 == 0 &&
                  offsetof(InStage, rate) % 16 == 0,
              "bulk-copy destinations are 16-byte aligned");

// Largest plane copy of one tile, in words: 64 blocks of rate 31, plus the
// rounding of both ends to 16 bytes.
constexpr uint32_t TILE_PLANE_WORDS_MAX = TILE * MAX_RATE + 2;

// Byte ranges of tile t of a stream (pv = {nc, r} exclusive prefixes of tile t
// and of tile t+1, from the rate pre-scan), rounded out to 16 bytes.
struct TileSpan {
  uint64_t sa16, pa16;
  unsigned rb, ob, sbytes, pbytes;
  uint32_t sbase, pbase;
  __device__ __forceinline__ uint32_t plane_words() const { return pbytes >> 3; }
};
__device__ __forceinline__ TileSpan tile_span(const Info& h, uint64_t t,
                                              const unsigned long long pv[4]) {
  const unsigned long long NC0 = pv[0], R0 = pv[1];
  const unsigned long long NC1 = pv[2], R1 = pv[3];
  TileSpan sp;
  const uint64_t rate_end = align16(h.nb), out_end = align16(4 * h.nb);
  sp.rb = (unsigned)umin64(TILE, rate_end - TILE * t);
  sp.ob = (unsigned)umin64(4 * TILE, out_end - 4 * TILE * t);
  const uint64_t sa = h.o_sign + 8 * NC0, se = h.o_sign + 8 * NC1;
  sp.sa16 = sa & ~15ull;
  const uint64_t se16 = align16(se);
  const uint64_t pa = h.o_plane + 8 * R0, pe = h.o_plane + 8 * R1;
  sp.pa16 = pa & ~15ull;
  const uint64_t pe16 = align16(pe);
  sp.sbytes = (NC1 > NC0) ? (unsigned)(se16 - sp.sa16) : 0u;
  sp.pbytes = (R1 > R0) ? (unsigned)(pe16 - sp.pa16) : 0u;
  // a corrupt pre-scan (refused before any tile is issued) aside, pbytes <= 8 * TILE_PLANE_WORDS_MAX
  if (sp.pbytes > 8u * TILE_PLANE_WORDS_MAX) sp.pbytes = 8u * TILE_PLANE_WORDS_MAX;
  if (sp.sbytes > 8u * (TILE + 2)) sp.sbytes = 8u * (TILE + 2);
  sp.sbase = (uint32_t)((sa - sp.sa16) >> 3);
  sp.pbase = (uint32_t)((pa - sp.pa16) >> 3);
  return sp;
}

// Issued by one thread: bulk-copy tile `t` of stream `c` into stage `s` and
// its planes into ring words [at, at + sp.plane_words()), completing on `bar`.
__device__ __forceinline__ void issue_in_tile(InStage* s, uint64_t* bar, const uint8_t* c,
                                              const Info& h, uint64_t t, const TileSpan& sp,
                                              uint64_t* ring, uint32_t at) {
  s->sbase = sp.sbase;
  s->pbase = sp.pbase;
  s->pring = at;
  fence_proxy_async();
  mbar_expect_tx(bar, sp.rb + sp.ob + sp.sbytes + sp.pbytes);
  bulk_g2s(s->rate, c + HOSZP_HEADER_BYTES + TILE * t, sp.rb, bar);
  bulk_g2s(s->outlier, c + h.o_out + 4 * TILE * t, sp.ob, bar);
  if (sp.sbytes) bulk_g2s(s->sign, c + sp.sa16, sp.sbytes, bar);
  if (sp.pbytes) bulk_g2s(ring + at, c + sp.pa16, sp.pbytes, bar);
}

// ---------------------------------------------------------------- plane ring
// A circular buffer of RW words in shared memory holding the plane words of
// the tiles in flight, each tile's copy contiguous (a copy that would cross
// the end starts over at word 0). Positions are word counts that only grow;
// beg[k % S] is where stage use k's copy starts. The issuer warp keeps the
// state (identical in every lane).
template <int S, uint32_t RW>
struct PlaneRing {
  static_assert(RW % 2 == 0 && RW >= TILE_PLANE_WORDS_MAX + 2, "ring size");
  // word index of a position (positions only grow and stay below 2^32 per launch)
  static __device__ __forceinline__ uint32_t wrap(uint32_t p) {
    if constexpr ((RW & (RW - 1)) == 0) return p & (RW - 1);
    else return p % RW;
  }
  uint64_t* ring;  // shared, RW words, 16-byte aligned
  uint32_t* beg;   // shared, S entries
  uint32_t head;   // next free position (even)
  __device__ __forceinline__ void init(uint64_t* r, uint32_t* b) {
    ring = r;
    beg = b;
    head = 0;
  }
  // Finds room for `words` (even) for stage use k, waiting for releases of
  // older stage uses (consumed in order: k_rel = uses released so far,
  // release_one() waits for use k_rel and advances it). Every older use has
  // been issued, so each wait ends. Whole issuer warp.
  template <class ReleaseOne>
  __device__ __forceinline__ uint32_t reserve(uint32_t k, uint32_t words, const uint32_t& k_rel,
                                              ReleaseOne&& release_one) const {
    uint32_t p0 = head;
    if (wrap(p0) + words > RW) p0 += RW - wrap(p0);
    for (;;) {
      const uint32_t tail = (k_rel < k) ? beg[k_rel % S] : p0;
      if (p0 + words - tail <= RW) return p0;
      release_one();
    }
  }
  __device__ __forceinline__ uint32_t commit(uint32_t k, uint32_t p0, uint32_t words) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) beg[k % S] = p0;
    __syncwarp();
    head = p0 + words;
    return wrap(p0);
  }
};

// Loader-warp window over the pre-scan's prefixes: the prefixes of the
// loader's tiles k0 .. k0+31 (tile bid + k * G) are fetched in one warp-wide
// load per 32 tiles into a shared-memory window, so issuing a tile needs no
// dependent global load. All 32 lanes call get() with the same, increasing k;
// `out` is meaningful in lane 0.
struct PreWindow {
  ulonglong2 (*win)[2];  // shared: [32][2] = {nc, r} of tile k and of tile k + 1
  uint64_t k0;
  __device__ __forceinline__ void init(ulonglong2 (*w)[2]) {
    win = w;
    k0 = ~0ull;
  }
  __device__ __forceinline__ void get(const unsigned long long* pre, uint64_t k, uint64_t bid,
                                      uint64_t G, uint64_t ntiles, unsigned long long out[4]) {
    const int lane = threadIdx.x & 31;
    if (k0 == ~0ull || k >= k0 + 32) {
      k0 = k;
      const uint64_t t = bid + (k0 + lane) * G;
      __syncwarp();
      if (t < ntiles) {
        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(pre + 2 * t);
        win[lane][0] = __ldg(p);
        win[lane][1] = __ldg(p + 1);
      }
      __syncwarp();
    }
    const ulonglong2 a = win[k - k0][0], b = win[k - k0][1];
    out[0] = a.x;
    out[1] = a.y;
    out[2] = b.x;
    out[3] = b.y;
  }
};

}  // namespace hz
