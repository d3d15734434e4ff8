// hz_common.cuh — device building blocks shared by the libhoszp kernels.
//
// Thread layout used by every codec kernel ("octet" layout): a CTA of
// HZ_CTA = 512 threads covers one tile of HZ_TILE = 64 blocks; thread tid owns
// block g = tid / 8 of the tile and, inside it, the 8 consecutive positions
// 8j..8j+7 with j = tid % 8. Eight lanes of a warp therefore hold one 64-value
// block; a warp holds 4 blocks. A block's bit planes (Sec. IV-A step 3) are
// 64-bit words whose byte j covers exactly lane j's positions, so planes move
// between memory and registers as whole words and are redistributed with an
// 8x8 byte transpose across the 8 lanes (3 shuffles) and an 8x8 bit transpose
// inside each lane (3 delta swaps).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hoszp.h"

#define HZ_HD __host__ __device__ __forceinline__

namespace hz {

constexpr int L = 64;        // values per block (Table 6)
constexpr int TILE = 64;     // blocks per tile
constexpr int CTA = 512;     // threads per CTA (8 per block)
constexpr int TILE_VALUES = TILE * L;
constexpr int MAX_RATE = 31;
constexpr int NCHAIN = 3;    // look-back chains per launch (add uses 2 inputs + 1 output)

// ---------------------------------------------------------------- stream layout (Fig. 3)
HZ_HD uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
HZ_HD uint64_t align16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }
HZ_HD uint64_t nblocks(uint64_t n) { return (n + L - 1) / L; }
HZ_HD uint64_t off_outlier(uint64_t nb) { return HOSZP_HEADER_BYTES + align16(nb); }
HZ_HD uint64_t off_sign(uint64_t nb) { return off_outlier(nb) + align16(4 * nb); }
HZ_HD uint64_t off_plane(uint64_t nb, uint64_t nnc) { return off_sign(nb) + 8 * nnc; }
HZ_HD uint64_t stream_bytes(uint64_t nb, uint64_t nnc, uint64_t R) {
  return align16(off_plane(nb, nnc) + 8 * R);  // zero padding to 16 bytes
}
HZ_HD uint64_t ntiles_of(uint64_t nb) { return (nb + TILE - 1) / TILE; }

// Parsed header plus derived section offsets.
struct Info {
  uint64_t n, nb, nnc, R, o_out, o_sign, o_plane, size;
  float eps_q;
  uint32_t qbound;
  double eps;
  uint32_t ndims, dims[3];
  int ok;
};

// Reads and checks the 64-byte header (every field that bounds a later read).
__device__ __forceinline__ Info parse_header(const uint8_t* c, uint64_t c_bytes) {
  Info h;
  h.ok = 0;
  h.n = h.nb = h.nnc = h.R = 0;
  if (c_bytes < HOSZP_HEADER_BYTES) return h;
  const hoszp_header* H = reinterpret_cast<const hoszp_header*>(c);
  hoszp_header v = *H;
  h.n = v.n;
  h.nnc = v.nnc;
  h.R = v.R;
  h.eps_q = v.eps_q;
  h.qbound = v.qbound;
  h.eps = v.eps;
  h.ndims = v.ndims;
  h.dims[0] = v.dims[0];
  h.dims[1] = v.dims[1];
  h.dims[2] = v.dims[2];
  h.nb = nblocks(v.n);
  bool ok = v.magic == HOSZP_MAGIC && v.version == HOSZP_VERSION && v.dtype == 0 &&
            v.block == HOSZP_BLOCK && v.eps_q >= 1.17549435e-38f && v.eps_q <= 1.70141173e38f &&
            v.qbound <= (uint32_t)HOSZP_QLIM && v.n <= (1ull << 56) && v.nnc <= h.nb &&
            v.R <= 31ull * v.nnc;
  if (!ok) { h.nb = 0; return h; }
  h.o_out = off_outlier(h.nb);
  h.o_sign = off_sign(h.nb);
  h.o_plane = off_plane(h.nb, h.nnc);
  h.size = stream_bytes(h.nb, h.nnc, h.R);
  if (h.size > c_bytes) { h.nb = 0; return h; }
  h.ok = 1;
  return h;
}

// ---------------------------------------------------------------- errors
__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// ---------------------------------------------------------------- memory ordering
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------- workspace
// Per-tile look-back descriptor: flag = (epoch << 2) | state, state 1 = the
// tile's own aggregate is published, 2 = its inclusive prefix is published.
struct Desc {
  unsigned long long flag;
  unsigned long long agg;  // (nc << 32) | r of the tile
  unsigned long long inc_nc, inc_r;
};

struct Sync {
  unsigned int ticket;  // next tile to hand out in this launch
  unsigned int done;    // CTAs finished in this launch
  unsigned long long epoch;
};

// Per-CTA record of the in-kernel rate prefix: the CTA's (non-constant
// blocks, rate sum) over its range of the stream, published under `flag` =
// (epoch << 1) | 1 of the launch.
struct CtaAgg {
  unsigned long long flag, nc, r, pad;
};

struct Partial {  // per-CTA exact sums for the reductions
  long long s1_lo, s1_hi;
  unsigned long long s2_lo, s2_hi;
};

// Device workspace seen by the kernels (pointers into one allocation).
struct Ws {
  Sync* sync;
  int* status;
  unsigned long long* totals;  // [0] nnc, [1] R of the output, [2] qmax, [3] ticket base
  float* eps_q;                // bound computed on the device (relative mode)
  double* eps;
  Desc* desc[NCHAIN];
  uint64_t max_tiles;
  Partial* partials;
  CtaAgg* cta_agg;     // max_grid records (in-kernel rate prefix)
  float* range_part;  // per-CTA min, max (2 floats) + nonfinite flag as float
  uint64_t max_grid;
  uint64_t* staging;  // plane words of a produced stream before placement
  uint64_t staging_words;
  hoszp_header* hdr;  // header of the stream being produced (filled in by the producer)
  unsigned long long* pre[2];  // per-tile (nc, r) prefixes of up to two input streams
  unsigned long long* agg;     // per-tile (nc << 32 | r) of a produced stream
  unsigned long long* opre;    // per-tile (nc, r) prefixes of the produced stream
};

// Tile hand-out and launch bookkeeping. Every CTA calls begin() once, next()
// per tile and end() once; the CTA that finishes last resets the counters and
// advances the epoch, so stale descriptors of earlier launches never match.
struct LaunchState {
  unsigned long long epoch;
};

__device__ __forceinline__ unsigned long long launch_epoch(const Ws& ws) {
  return *reinterpret_cast<volatile unsigned long long*>(&ws.sync->epoch);
}

// Returns true in exactly one CTA: the last to finish this launch.
__device__ __forceinline__ bool launch_end_is_last(const Ws& ws) {
  __shared__ unsigned int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(&ws.sync->done, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
    if (s_last) __threadfence();
  }
  __syncthreads();
  return s_last != 0;
}

__device__ __forceinline__ void launch_reset(const Ws& ws) {
  // called by one thread of the last CTA after its final work
  ws.sync->ticket = 0;
  ws.sync->done = 0;
  ws.sync->epoch = ws.sync->epoch + 1;
  __threadfence();
}

// ---------------------------------------------------------------- decoupled look-back
constexpr long long SPIN_LIMIT = 1ll << 22;  // x ~256 ns sleeps: about a second

__device__ __forceinline__ void publish(Desc* d, int64_t tile, unsigned long long epoch,
                                        int state, unsigned long long agg,
                                        unsigned long long inc_nc, unsigned long long inc_r) {
  if (state == 1) {
    d[tile].agg = agg;
  } else {
    d[tile].agg = agg;
    d[tile].inc_nc = inc_nc;
    d[tile].inc_r = inc_r;
  }
  __threadfence();
  st_release(&d[tile].flag, (epoch << 2) | (unsigned long long)state);
}

// Warp-wide look-back: returns the exclusive prefix (nc, r) of `tile` over the
// chain. All 32 lanes of the calling warp must take part. Spins are bounded;
// on timeout the status word gets HOSZP_ERR_TIMEOUT and a zero prefix is used.
__device__ __forceinline__ void lookback(Desc* d, int64_t tile, unsigned long long epoch, int* st,
                                         unsigned long long& pnc, unsigned long long& pr,
                                         long long spin_limit = SPIN_LIMIT) {
  const int lane = threadIdx.x & 31;
  unsigned long long acc_nc = 0, acc_r = 0;
  int64_t base = tile - 1;
  while (base >= 0) {
    int64_t j = base - lane;
    int state = 2;
    unsigned long long a = 0, inc_nc = 0, inc_r = 0;
    if (j >= 0) {
      long long spins = 0;
      for (;;) {
        unsigned long long f = ld_acquire(&d[j].flag);
        state = ((f >> 2) == epoch) ? (int)(f & 3) : 0;
        if (state != 0) break;
        if (++spins > spin_limit) {
          set_status(st, HOSZP_ERR_TIMEOUT);
          state = 2;
          break;
        }
        __nanosleep(256);
      }
      if (state != 0) {
        a = *reinterpret_cast<volatile unsigned long long*>(&d[j].agg);
        if (state == 2) {
          inc_nc = *reinterpret_cast<volatile unsigned long long*>(&d[j].inc_nc);
          inc_r = *reinterpret_cast<volatile unsigned long long*>(&d[j].inc_r);
        }
      }
    }
    unsigned int incmask = __ballot_sync(0xffffffffu, state == 2);
    int stop = incmask ? (__ffs(incmask) - 1) : 32;  // nearest tile with an inclusive prefix
    unsigned long long vnc = 0, vr = 0;
    if (lane < stop) {
      vnc = a >> 32;
      vr = a & 0xffffffffull;
    } else if (lane == stop) {
      vnc = inc_nc;
      vr = inc_r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vnc += __shfl_xor_sync(0xffffffffu, vnc, o);
      vr += __shfl_xor_sync(0xffffffffu, vr, o);
    }
    acc_nc += vnc;
    acc_r += vr;
    if (incmask) break;
    base -= 32;
  }
  pnc = acc_nc;
  pr = acc_r;
}

// Tile-level prefix for one chain, called by the whole CTA: publishes the
// tile's aggregate, looks back (warp `wid`), publishes the inclusive prefix and
// returns the exclusive prefix through shared memory.
__device__ __forceinline__ void tile_prefix(Desc* d, int64_t tile, unsigned long long epoch,
                                            int* st, unsigned int agg_nc, unsigned int agg_r,
                                            int wid, unsigned long long* s_out /*[2]*/) {
  if ((int)(threadIdx.x >> 5) == wid) {
    unsigned long long agg = ((unsigned long long)agg_nc << 32) | agg_r;
    unsigned long long pnc = 0, pr = 0;
    if (tile == 0) {
      if ((threadIdx.x & 31) == 0) publish(d, tile, epoch, 2, agg, agg_nc, agg_r);
    } else {
      if ((threadIdx.x & 31) == 0) publish(d, tile, epoch, 1, agg, 0, 0);
      __syncwarp();
      lookback(d, tile, epoch, st, pnc, pr);
      if ((threadIdx.x & 31) == 0) publish(d, tile, epoch, 2, agg, pnc + agg_nc, pr + agg_r);
    }
    if ((threadIdx.x & 31) == 0) {
      s_out[0] = pnc;
      s_out[1] = pr;
    }
  }
}

// ---------------------------------------------------------------- bit manipulation
// 8x8 bit transpose of the matrix held in (lo, hi): byte i = row i, bit j of a
// byte = column j. Afterwards byte i holds column i. Three delta swaps.
HZ_HD void tr8x8(uint32_t& lo, uint32_t& hi) {
  uint32_t t;
  t = (lo ^ (lo >> 7)) & 0x00AA00AAu;
  lo = lo ^ t ^ (t << 7);
  t = (hi ^ (hi >> 7)) & 0x00AA00AAu;
  hi = hi ^ t ^ (t << 7);
  t = (lo ^ (lo >> 14)) & 0x0000CCCCu;
  lo = lo ^ t ^ (t << 14);
  t = (hi ^ (hi >> 14)) & 0x0000CCCCu;
  hi = hi ^ t ^ (t << 14);
  t = (lo ^ (hi << 4)) & 0xF0F0F0F0u;
  lo = lo ^ t;
  hi = hi ^ (t >> 4);
}

#ifdef __CUDACC__
// Lane constants for byte_transpose8 (PRMT selectors; j = lane % 8).
struct OctetSel {
  uint32_t a0, a1, b0, b1, b2, c0, c1, c2;
};
__device__ __forceinline__ OctetSel octet_sel(int j) {
  OctetSel S;
  const bool x4 = (j & 4) != 0, x2 = (j & 2) != 0, x1 = (j & 1) != 0;
  S.a0 = x4 ? 0x3210u : 0x7654u;
  S.a1 = S.a0 ^ 0x4444u;
  S.b0 = x2 ? 0x5410u : 0x7632u;
  S.b1 = x2 ? 0x3254u : 0x5410u;
  S.b2 = x2 ? 0x3276u : 0x7610u;
  S.c0 = x1 ? 0x6420u : 0x7531u;
  S.c1 = x1 ? 0x3514u : 0x5240u;
  S.c2 = x1 ? 0x3716u : 0x7260u;
  return S;
}

// 8x8 byte transpose across the 8 lanes of an octet: lane j holds row j
// (bytes 0..3 in lo, 4..7 in hi); afterwards lane j holds column j. All lanes
// of the warp must call it (full-mask shuffles; partners differ in bits 0..2).
// Three exchange steps (distance 4, 2, 1), each one shuffle and three byte
// permutes with lane-constant selectors.
__device__ __forceinline__ void byte_transpose8(uint32_t& lo, uint32_t& hi, const OctetSel& S) {
  uint32_t send = __byte_perm(lo, hi, S.a0);
  uint32_t recv = __shfl_xor_sync(0xffffffffu, send, 4);
  lo = __byte_perm(lo, recv, S.a1);
  hi = __byte_perm(hi, recv, S.a0);
  send = __byte_perm(lo, hi, S.b0);
  recv = __shfl_xor_sync(0xffffffffu, send, 2);
  lo = __byte_perm(lo, recv, S.b1);
  hi = __byte_perm(hi, recv, S.b2);
  send = __byte_perm(lo, hi, S.c0);
  recv = __shfl_xor_sync(0xffffffffu, send, 1);
  lo = __byte_perm(lo, recv, S.c1);
  hi = __byte_perm(hi, recv, S.c2);
}
__device__ __forceinline__ void byte_transpose8(uint32_t& lo, uint32_t& hi, int j) {
  byte_transpose8(lo, hi, octet_sel(j));
}

// tr8x8 with the shifts written as integer multiplies (high part for right
// shifts), so they issue on the FMA pipe and the logic pipe only sees the
// LOP3 operations. Same result as tr8x8.
__device__ __forceinline__ void tr8x8_d(uint32_t& lo, uint32_t& hi) {
  uint32_t t;
  t = (lo ^ __umulhi(lo, 1u << 25)) & 0x00AA00AAu;  // >> 7
  lo = lo ^ t ^ (t * 128u);
  t = (hi ^ __umulhi(hi, 1u << 25)) & 0x00AA00AAu;
  hi = hi ^ t ^ (t * 128u);
  t = (lo ^ __umulhi(lo, 1u << 18)) & 0x0000CCCCu;  // >> 14
  lo = lo ^ t ^ (t * 16384u);
  t = (hi ^ __umulhi(hi, 1u << 18)) & 0x0000CCCCu;
  hi = hi ^ t ^ (t * 16384u);
  t = (lo ^ (hi * 16u)) & 0xF0F0F0F0u;
  lo = lo ^ t;
  hi = hi ^ __umulhi(t, 1u << 28);  // >> 4
}

// ---------------------------------------------------------------- quantization (Eq. 3)
// Exact q = floor((x + e) / (2e)) for float x, e = eps_q (normal float), using
// only FP32 FMA arithmetic: an estimate k rounds x * r (r ~ 1/(2e)) to an
// integer, d = x - k*2e is formed with one rounding by an FMA, and d against
// +-e decides q in {k-1, k, k+1}. d is exact-or-monotonically-rounded, so only
// d == +-e is ambiguous; that case is settled exactly with an error-free
// product (two FMAs) and Sterbenz subtractions.
struct Quant {
  float e, e2, r;  // eps_q, 2 eps_q, fl(1 / (2 eps_q))
};

__device__ __forceinline__ int quant_fix(float x, float kf, int k, const Quant& Q) {
  float d = __fmaf_rn(-kf, Q.e2, x);
  if (d < -Q.e) return k - 1;
  if (d > Q.e) return k + 1;
  if (d == -Q.e || d == Q.e) {
    float p = __fmul_rn(kf, Q.e2);
    float perr = __fmaf_rn(kf, Q.e2, -p);  // kf*e2 = p + perr exactly
    float d1 = __fsub_rn(x, p);            // exact here
    if (d == -Q.e) return (__fadd_rn(d1, Q.e) < perr) ? k - 1 : k;
    return (__fsub_rn(d1, Q.e) >= perr) ? k + 1 : k;
  }
  return k;
}

// Returns q; sets *bad to HOSZP_ERR_NONFINITE or HOSZP_ERR_RANGE when needed.
__device__ __forceinline__ int quantize(float x, const Quant& Q, int& bad) {
  const float MAGIC = 12582912.0f;  // 1.5 * 2^23
  float t = __fmul_rn(x, Q.r);
  if (fabsf(t) < 4194300.0f) {  // |x r| < 2^22: integer rounding by the magic add
    float y = __fmaf_rn(x, Q.r, MAGIC);
    int k = __float_as_int(y) - 0x4B400000;
    float kf = __fsub_rn(y, MAGIC);
    return quant_fix(x, kf, k, Q);
  }
  if (!(fabsf(x) <= 3.40282347e38f)) {
    bad = HOSZP_ERR_NONFINITE;
    return 0;
  }
  if (!(fabsf(t) <= 8388612.0f)) {  // |q| >= 2^23 + 3 > HOSZP_QMAX_COMPRESS
    bad = HOSZP_ERR_RANGE;
    return 0;
  }
  int k = __float2int_rn(t);
  int q = quant_fix(x, (float)k, k, Q);
  if (q > HOSZP_QMAX_COMPRESS || q < -HOSZP_QMAX_COMPRESS) bad = HOSZP_ERR_RANGE;
  return q;
}

// Eq. 3 for 8 values. Fast path, taken when it holds for all 8: y = x r +
// 1.5 2^23 (one rounding) lies in [2^23, 2^24), so k = y - 1.5 2^23 is an
// integer read off y's bits, and d = x - 2e k (one rounding) has |d| < e.
// Rounding is monotone and e is a float, so then the exact |x - 2e k| < e as
// well: k is the one integer with (x + e) / 2e in (k, k + 1), which is Eq. 3's
// q. Otherwise (a value on or near a cell edge, a large or non-finite x)
// quantize() settles all 8 exactly. Either way q is the exact Eq. 3 value.
__device__ __forceinline__ void quantize8(const float v[8], const Quant& Q, int q[8], int& bad) {
  const float MAGIC = 12582912.0f;  // 1.5 * 2^23
  uint32_t span = 0;
  bool inside = true;
#pragma unroll
  for (int t = 0; t < 8; t++) {
    const float y = __fmaf_rn(v[t], Q.r, MAGIC);
    const uint32_t yb = __float_as_uint(y);
    span |= yb ^ 0x4B000000u;  // < 2^23 iff y in [2^23, 2^24)
    const float kf = __fsub_rn(y, MAGIC);
    const float d = __fmaf_rn(-kf, Q.e2, v[t]);
    inside = inside && (fabsf(d) < Q.e);
    q[t] = (int)yb - 0x4B400000;
  }
  if (span >= 0x800000u || !inside) {
#pragma unroll
    for (int t = 0; t < 8; t++) q[t] = quantize(v[t], Q, bad);
  }
}

// x' = 2e * q rounded once to float32 (reverse quantization, proof of
// Theorem 1). For |q| < 2^22 the conversion of q is exact (magic-number trick
// on the FP32 pipe) and the one float multiply is the only rounding.
__device__ __forceinline__ float dequant_small(int q, float e2) {
  float qf = __fsub_rn(__int_as_float(q + 0x4B400000), 12582912.0f);
  return __fmul_rn(qf, e2);
}
// Any |q| < 2^31 (operator outputs reach 2^30 - 1, where float(q) would
// already round). With 2e = M 2^E (M its integer significand, < 2^24), the
// product P = q M is exact in 64 bits (< 2^55), the int64 -> float conversion
// rounds it once to nearest-even, and the scaling by 2^E is exact: for q != 0
// and a normal 2e, |P| >= 2^23 and E >= -149 keep the result normal; for a
// subnormal 2e (E = -149) a P below 2^24 converts exactly and its multiple of
// 2^-149 is representable. A product beyond FLT_MAX becomes infinity.
__device__ __forceinline__ float dequant_any(int q, float e2) {
  const uint32_t b = __float_as_uint(e2);
  const int ex = (int)((b >> 23) & 0xffu);
  const long long M = (long long)(ex ? ((b & 0x7fffffu) | 0x800000u) : (b & 0x7fffffu));
  const int E = ex ? ex - 150 : -149;  // in [-149, 104]
  const float p2 = E >= -126 ? __int_as_float((E + 127) << 23) : __int_as_float(1 << (E + 149));
  return __fmul_rn(__ll2float_rn((long long)q * M), p2);
}

// ---------------------------------------------------------------- octet codec
// Encode: lane j holds magnitudes of its 8 positions; writes plane words
// 8k+j (< r) of the block to planes_out. kmax warp-uniform >= ceil(r/8).
template <int K>
__device__ __forceinline__ void encode_groups(const uint32_t mag[8], int r, int j,
                                              uint64_t* planes_out, const OctetSel& S) {
#pragma unroll
  for (int k = 0; k < K; k++) {
    // byte k of each magnitude, gathered with byte permutes: (m0.k, m1.k) then
    // the two pairs side by side
    const uint32_t sel = (uint32_t)k | ((4u + (uint32_t)k) << 4);
    uint32_t lo = __byte_perm(__byte_perm(mag[0], mag[1], sel), __byte_perm(mag[2], mag[3], sel),
                              0x5410u);
    uint32_t hi = __byte_perm(__byte_perm(mag[4], mag[5], sel), __byte_perm(mag[6], mag[7], sel),
                              0x5410u);
    tr8x8_d(lo, hi);             // byte p' = bit 8k+p' of the 8 magnitudes
    byte_transpose8(lo, hi, S);  // lane j: plane word 8k+j
    const int p = 8 * k + j;
    if (p < r) planes_out[p] = ((uint64_t)hi << 32) | lo;
  }
}
__device__ __forceinline__ void encode_planes(const uint32_t mag[8], int r, int kmax, int j,
                                              uint64_t* planes_out, const OctetSel& S) {
  switch (kmax) {
    case 1: encode_groups<1>(mag, r, j, planes_out, S); break;
    case 2: encode_groups<2>(mag, r, j, planes_out, S); break;
    case 3: encode_groups<3>(mag, r, j, planes_out, S); break;
    default: encode_groups<4>(mag, r, j, planes_out, S); break;
  }
}

// Rate of a block from lane magnitudes: bit length of the octet-wide maximum.
__device__ __forceinline__ int octet_rate(const uint32_t mag[8]) {
  uint32_t m = 0;
#pragma unroll
  for (int t = 0; t < 8; t++) m = max(m, mag[t]);
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 4));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
  return 32 - __clz(m);
}

// Exclusive scan of a per-octet value across the 8 lanes of the octet.
__device__ __forceinline__ int octet_excl_scan(int v, int j) {
  int x = v;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o, 8);
    if (j >= o) x += y;
  }
  return x - v;
}
#endif  // __CUDACC__

}  // namespace hz
