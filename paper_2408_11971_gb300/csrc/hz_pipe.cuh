// hz_pipe.cuh — tile pipelines: 1-D TMA bulk copies (cp.async.bulk) of a
// compressed tile into a shared-memory ring completed on mbarriers, and the
// shared-memory output stage of a produced tile.
#pragma once
#include <cstddef>

#include "hz_common.cuh"

namespace hz {

// ---------------------------------------------------------------- mbarrier / bulk copy
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
// Bounded wait: after ~a second of polling the status word gets TIMEOUT and the
// wait gives up (the data in the stage is then not used for a valid result).
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* st) {
  long long spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > (1ll << 24)) {
      set_status(st, HOSZP_ERR_TIMEOUT);
      return;
    }
  }
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
// One tile of an input stream in shared memory. Sign and plane words are
// copied from the 16-byte-aligned addresses around the tile's words; sbase and
// pbase give the index of the tile's first word inside sign[] and plane[].
struct __align__(16) InStage {
  uint64_t plane[TILE * MAX_RATE + 2];
  uint64_t sign[TILE + 2];
  int outlier[TILE];
  uint8_t rate[TILE];  // bulk-copied; then sanitized by the loader warp
  uint32_t sbase, pbase;
  // written by the loader warp once the copy has landed (see prepare_tile):
  uint32_t off[TILE];              // (non-constant blocks before << 16) | rate sum before
  uint8_t kmx[TILE / 4];           // plane groups (ceil(rate/8)) to decode, per warp of 4 blocks
  uint32_t nvalid;                 // blocks of the tile inside the stream
  uint32_t lastlen;                // values in block nvalid-1
};
static_assert(sizeof(uint64_t) * (TILE * MAX_RATE + 2) % 16 == 0, "plane[] keeps alignment");
static_assert(sizeof(uint64_t) * (TILE + 2) % 16 == 0, "sign[] keeps alignment");
static_assert(sizeof(InStage) % 16 == 0, "ring stages must stay 16-byte aligned (bulk copies)");
static_assert(TILE == 64, "prepare_tile scans 64 blocks with one warp (2 per lane)");
static_assert(offsetof(InStage, sign) % 16 == 0 && offsetof(InStage, outlier) % 16 == 0 &&
                  offsetof(InStage, rate) % 16 == 0,
              "bulk-copy destinations are 16-byte aligned");

// Issued by one thread: bulk-copy tile `t` of stream `c` into `s`, completing
// on `bar`. pv = {nc, r} exclusive prefixes (non-constant blocks, rate sum) of
// tile t and of tile t+1, from the rate pre-scan.
__device__ __forceinline__ void issue_in_tile(InStage* s, uint64_t* bar, const uint8_t* c,
                                              const Info& h, uint64_t t,
                                              const unsigned long long pv[4]) {
  const unsigned long long NC0 = pv[0], R0 = pv[1];
  const unsigned long long NC1 = pv[2], R1 = pv[3];
  const uint64_t rate_end = align16(h.nb), out_end = align16(4 * h.nb);
  const unsigned rb = (unsigned)umin64(TILE, rate_end - TILE * t);
  const unsigned ob = (unsigned)umin64(4 * TILE, out_end - 4 * TILE * t);
  const uint64_t sa = h.o_sign + 8 * NC0, se = h.o_sign + 8 * NC1;
  const uint64_t sa16 = sa & ~15ull, se16 = align16(se);
  const uint64_t pa = h.o_plane + 8 * R0, pe = h.o_plane + 8 * R1;
  const uint64_t pa16 = pa & ~15ull, pe16 = align16(pe);
  const unsigned sbytes = (NC1 > NC0) ? (unsigned)(se16 - sa16) : 0u;
  const unsigned pbytes = (R1 > R0) ? (unsigned)(pe16 - pa16) : 0u;
  s->sbase = (uint32_t)((sa - sa16) >> 3);
  s->pbase = (uint32_t)((pa - pa16) >> 3);
  fence_proxy_async();
  mbar_expect_tx(bar, rb + ob + sbytes + pbytes);
  bulk_g2s(s->rate, c + HOSZP_HEADER_BYTES + TILE * t, rb, bar);
  bulk_g2s(s->outlier, c + h.o_out + 4 * TILE * t, ob, bar);
  if (sbytes) bulk_g2s(s->sign, c + sa16, sbytes, bar);
  if (pbytes) bulk_g2s(s->plane, c + pa16, pbytes, bar);
}

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
