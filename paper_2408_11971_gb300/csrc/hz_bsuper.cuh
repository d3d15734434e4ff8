// hz_bsuper.cuh — the batched super-tile input pipeline: one loader warp
// walks its CTA's contiguous range of a batch plan's global tile space and
// bulk-copies stages of up to NT consecutive tiles of one field (rates,
// outliers, sign words, plane words) into a ring of shared-memory stages, as
// the single-stream super-tile pipeline does for one stream. Used by the
// batched reductions and decompression (batch.cu) and the batched scalar
// multiplication (bproduce.cu).
#pragma once
#include "hz_super.cuh"
#include "batch_plan.cuh"

namespace hz {

// The current field of a walker (one per loader warp), advanced as tiles grow.
struct Walk {
  uint32_t f;
  uint64_t tile0, ntiles, pre0;
  const uint8_t* c;
  Info h;
  __device__ __forceinline__ void load(const BField* F, uint32_t fi) {
    f = fi;
    const BField& b = F[fi];
    tile0 = b.tile0;
    ntiles = b.ntiles;
    pre0 = b.pre0;
    c = b.c;
    h = b.h;
  }
  __device__ __forceinline__ void to_tile(const BField* F, uint32_t nf, uint64_t t) {
    if (f == ~0u || t < tile0) load(F, field_of_tile(F, nf, t));
    while (t >= tile0 + ntiles && f + 1 < nf) load(F, f + 1);
  }
};

struct BStageMeta {
  uint32_t f, nt;   // field, tiles in the stage (0: end of the walk)
  uint64_t t0;      // first tile of the stage, local to the field
};

// Byte ranges of local tiles [t0, t0 + nt) of a stream, from its prefixes at
// t0 (pv0) and at t0 + nt (pv1).
template <int NT>
__device__ __forceinline__ SSpan tile_range_span(const Info& h, uint64_t t0, uint32_t nt,
                                                 ulonglong2 pv0, ulonglong2 pv1) {
  SSpan sp;
  const uint64_t b0 = (uint64_t)TILE * t0;
  const uint64_t rate_end = align16(h.nb), out_end = align16(4 * h.nb);
  sp.rb = (unsigned)umin64((uint64_t)TILE * nt, rate_end - b0);
  sp.ob = (unsigned)umin64(4ull * TILE * nt, out_end - 4 * b0);
  const uint64_t sa = h.o_sign + 8 * pv0.x, se = h.o_sign + 8 * pv1.x;
  const uint64_t pa = h.o_plane + 8 * pv0.y, pe = h.o_plane + 8 * pv1.y;
  sp.sa16 = sa & ~15ull;
  sp.pa16 = pa & ~15ull;
  sp.sbytes = (pv1.x > pv0.x) ? (unsigned)(align16(se) - sp.sa16) : 0u;
  sp.pbytes = (pv1.y > pv0.y) ? (unsigned)(align16(pe) - sp.pa16) : 0u;
  if (sp.pbytes > 8u * SuperChecks<NT>::kPlaneWordsMax) sp.pbytes = 8u * SuperChecks<NT>::kPlaneWordsMax;
  if (sp.sbytes > 8u * (NT * TILE + 2)) sp.sbytes = 8u * (NT * TILE + 2);
  sp.sbase = (uint32_t)((sa - sp.sa16) >> 3);
  sp.pbase = (uint32_t)((pa - sp.pa16) >> 3);
  return sp;
}

// The loader warp. A stage use k waits for the release of use k - STAGES
// (empty[], in order), copies the next up to NT tiles of the current field
// into stages[k % STAGES] and their planes into the ring, records the field,
// tile count and first tile in s_meta[], the in-stage tile bases in tnc[] /
// tr[] and the field's prefix at the stage in bnc / br, and completes the
// copies on full[k % STAGES]. After the range it hands each of the GROUPS
// consumer groups an end stage (nt = 0). Every wait is bounded; after one gave
// up, the copies already issued land before it returns.
template <int NT, int STAGES, uint32_t RING, int GROUPS>
__device__ __forceinline__ void bsuper_loader(SStageT<NT>* stages, uint64_t* ring, uint32_t* s_beg,
                                              uint64_t* full, uint64_t* empty,
                                              BStageMeta* s_meta, const BField* F, uint32_t nf,
                                              const unsigned long long* pre, uint64_t t_begin,
                                              uint64_t t_end, int* status) {
  const int lane = threadIdx.x & 31;
  PlaneRing<STAGES, RING> pr;
  pr.init(ring, s_beg);
  uint32_t k_rel = 0;
  bool dead = false;  // a wait gave up: issue nothing more, wait for nothing more
  auto release_one = [&]() {
    if (!dead && !mbar_wait_warp(&empty[k_rel % STAGES], (k_rel / STAGES) & 1, status))
      dead = true;
    k_rel++;
  };
  uint32_t k_end = 0;  // stage uses issued so far
  Walk wk;
  wk.f = ~0u;
  uint64_t t = t_begin;
  int ends = 0;
  for (uint32_t k = 0; ends < GROUPS; k++) {
    const int sk = (int)(k % STAGES);
    while (k_rel + STAGES <= k) release_one();
    if (dead) break;  // no end markers either: a stage may still be in flight
    if (t >= t_end) {
      if (lane == 0) {
        s_meta[sk].nt = 0;
        mbar_arrive(&full[sk]);
      }
      ends++;
      __syncwarp();
      continue;
    }
    wk.to_tile(F, nf, t);
    const uint64_t lt = t - wk.tile0;
    const uint32_t nt = (uint32_t)umin64(umin64(NT, wk.ntiles - lt), t_end - t);
    // the stream's prefixes at the stage's tile boundaries (lanes 0 .. nt)
    ulonglong2 pv = make_ulonglong2(0, 0);
    if (lane <= (int)nt)
      pv = __ldg(reinterpret_cast<const ulonglong2*>(pre + wk.pre0 + 2 * (lt + lane)));
    const ulonglong2 pv0 = make_ulonglong2(__shfl_sync(0xffffffffu, pv.x, 0),
                                           __shfl_sync(0xffffffffu, pv.y, 0));
    const ulonglong2 pv1 = make_ulonglong2(__shfl_sync(0xffffffffu, pv.x, nt),
                                           __shfl_sync(0xffffffffu, pv.y, nt));
    const SSpan sp = tile_range_span<NT>(wk.h, lt, nt, pv0, pv1);
    const uint32_t p0 = pr.reserve(k, sp.plane_words(), k_rel, release_one);
    if (dead) break;
    const uint32_t at = pr.commit(k, p0, sp.plane_words());
    SStageT<NT>* sg = &stages[sk];
    if (lane < (int)nt) {
      sg->tnc[lane] = (uint32_t)(pv.x - pv0.x);
      sg->tr[lane] = (uint32_t)(pv.y - pv0.y);
    }
    __syncwarp();  // the tile bases are ordered before lane 0's arrival on full[]
    if (lane == 0) {
      s_meta[sk].f = wk.f;
      s_meta[sk].nt = nt;
      s_meta[sk].t0 = lt;
      sg->sbase = sp.sbase;
      sg->pbase = sp.pbase;
      sg->pring = at;
      sg->bnc = pv0.x;  // the field's prefix at the stage's first tile
      sg->br = pv0.y;
      fence_proxy_async();
      mbar_expect_tx(&full[sk], sp.rb + sp.ob + sp.sbytes + sp.pbytes);
      const uint64_t b0 = (uint64_t)TILE * lt;
      bulk_g2s(sg->rate, wk.c + HOSZP_HEADER_BYTES + b0, sp.rb, &full[sk]);
      bulk_g2s(sg->outlier, wk.c + wk.h.o_out + 4 * b0, sp.ob, &full[sk]);
      if (sp.sbytes) bulk_g2s(sg->sign, wk.c + sp.sa16, sp.sbytes, &full[sk]);
      if (sp.pbytes) bulk_g2s(ring + at, wk.c + sp.pa16, sp.pbytes, &full[sk]);
    }
    __syncwarp();
    t += nt;
    k_end = k + 1;
  }
  // after a wait gave up, the copies already issued land before the CTA exits
  if (dead)
    for (uint32_t u = k_rel; u < k_end; u++)
      mbar_wait(&full[u % STAGES], (u / STAGES) & 1, status);
}

}  // namespace hz
