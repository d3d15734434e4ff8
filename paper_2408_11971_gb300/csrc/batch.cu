// batch.cu — batched persistent execution over many resident streams.
//
// A snapshot holds thousands of fields of very different sizes; one launch per
// field per operator would spend more time launching than working on the small
// ones. A batch plan fixes a set of resident streams and lays their tiles end
// to end in one global tile space (field f owns tiles [tile0_f, tile0_f +
// ntiles_f)); each operator is then one persistent launch in which CTA b takes
// the contiguous tile range [T b / G, T (b+1) / G) and walks the field table
// as its range crosses field boundaries. Per-field results are finished inside
// the same launch by whichever warp contributes a field's last tiles.
//
// Plan creation parses every header and runs each stream's rate pre-scan once
// (the prefixes stay valid for negation and scalar addition, which change no
// rate). The operators launch no allocation and no synchronization, so a
// sequence of them can be captured in a CUDA graph. A small autotuner picks,
// per reduction, the pipeline depth and the CTAs per SM from timed runs on the
// plan's own data.
#include <algorithm>
#include <vector>

#include "hz_moments.cuh"
#include "hz_scalar.cuh"
#include "hz_super.cuh"
#include "hz_var.cuh"
#include "hz_kernels.cuh"
#include "batch_plan.cuh"
#include "hz_bsuper.cuh"

namespace hz {
int ctx_prepare(hoszp_ctx* ctx, uint64_t tiles, Ws* ws, int* device, int* num_sms);  // api.cu
int* ctx_status_word(hoszp_ctx* ctx);                                                   // api.cu
}  // namespace hz

namespace hz {
namespace {

// ---------------------------------------------------------------- plan parsing
__global__ void k_bparse(const uint8_t* const* ptrs, const uint64_t* bytes, uint32_t nf,
                         BField* F, int* status) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  BField b{};
  b.c = ptrs[f];
  b.cw = const_cast<uint8_t*>(ptrs[f]);
  b.h = parse_header(ptrs[f], bytes[f]);
  if (!b.h.ok) set_status(status, HOSZP_ERR_FORMAT);
  else if (b.h.n == 0) set_status(status, HOSZP_ERR_ARG);
  b.ntiles = b.h.ok ? ntiles_of(b.h.nb) : 0;
  if (b.h.ok) {
    b.nch[0] = (align16(b.h.o_plane) - b.h.o_out) / 16;
    b.nch[1] = (b.h.o_sign - b.h.o_out) / 16;
  }
  F[f] = b;
}

// ---------------------------------------------------------------- field walk
__device__ __forceinline__ uint32_t field_of_chunk(const BField* F, uint32_t nf, int op,
                                                   uint64_t ch) {
  uint32_t lo = 0, hi = nf;
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (F[mid].ch0[op] <= ch) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void atomic_add_u128(unsigned long long* p, unsigned long long lo,
                                                unsigned long long hi) {
  const unsigned long long old = atomicAdd(p, lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(p + 1, hi + carry);
}

// ---------------------------------------------------------------- batched mean / variance
// Per field: acc[4f .. 4f+3] = S1 (128-bit two's complement), S2 (128-bit);
// done[f] counts warp-tiles (16 per tile); both are zero between launches.
template <bool VAR, int STAGES>
__global__ void __launch_bounds__(CONSUMER_THREADS, 2) k_bmoments(
    const BField* __restrict__ F, uint32_t nf, uint64_t total_tiles,
    const unsigned long long* __restrict__ pre, unsigned long long* acc, unsigned int* done,
    double* results, int* status) {
  constexpr uint32_t RING = 8192;
  extern __shared__ __align__(16) uint8_t dyn[];
  InStage* stages = reinterpret_cast<InStage*>(dyn);
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + STAGES);
  __shared__ uint64_t full[STAGES], ready[STAGES], empty[STAGES];
  __shared__ unsigned long long stage_tile[STAGES];
  __shared__ uint32_t stage_field[STAGES];
  const int tid = threadIdx.x, w = tid >> 5, g = tid >> 3, j = tid & 7, lane = tid & 31;
  const uint64_t G = gridDim.x;
  const uint64_t t_begin = total_tiles * blockIdx.x / G;
  const uint64_t t_end = total_tiles * (blockIdx.x + 1) / G;
  ring_init3<STAGES>(full, ready, empty);
  if (w >= LOADER_WARP) {
    __shared__ uint32_t s_beg[STAGES];
    __shared__ unsigned long long s_win[32][4];
    PlaneRing<STAGES, RING> pr;
    pr.init(ring, s_beg);
    Walk wk;
    wk.f = ~0u;
    uint64_t win_f = ~0ull, win0 = 0;  // prefixes of local tiles win0 .. win0+31 of field win_f
    loader_warps<STAGES>(
        w - LOADER_WARP, stage_tile, full, ready, empty, total_tiles, status,
        [&](uint32_t k) {
          const uint64_t t = t_begin + k;
          return (unsigned long long)(t < t_end ? t : total_tiles);
        },
        [&](int sk, unsigned long long t, uint32_t k, const uint32_t& k_rel,
            auto&& release_one) {
          wk.to_tile(F, nf, t);
          const uint64_t lt = t - wk.tile0;
          if (win_f != wk.f || lt >= win0 + 32) {  // refill the prefix window
            win_f = wk.f;
            win0 = lt;
            __syncwarp();
            if (lt + lane < wk.ntiles) {
              const ulonglong2* p =
                  reinterpret_cast<const ulonglong2*>(pre + wk.pre0 + 2 * (lt + lane));
              const ulonglong2 a = __ldg(p), b = __ldg(p + 1);
              s_win[lane][0] = a.x;
              s_win[lane][1] = a.y;
              s_win[lane][2] = b.x;
              s_win[lane][3] = b.y;
            }
            __syncwarp();
          }
          unsigned long long pv[4];
#pragma unroll
          for (int i = 0; i < 4; i++) pv[i] = s_win[lt - win0][i];
          const TileSpan sp = tile_span(wk.h, lt, pv);
          const uint32_t p0 = pr.reserve(k, sp.plane_words(), k_rel, release_one);
          const uint32_t at = pr.commit(k, p0, sp.plane_words());
          if (lane == 0) {
            stage_field[sk] = wk.f;
            issue_in_tile(&stages[sk], &full[sk], wk.c, wk.h, lt, sp, ring, at);
          }
        },
        [&](int sk, unsigned long long t) {
          wk.to_tile(F, nf, t);
          prepare_tile(stages[sk], t - wk.tile0, wk.h);
        });
  } else {
    const OctetSel S = octet_sel(j);
    uint32_t wlo, whi;
    mean_weights(j, wlo, whi);
    long long s1 = 0;
    U128 s2 = {0, 0};
    uint32_t cur = ~0u, cnt = 0;  // field being accumulated, warp-tiles of it
    auto flush = [&]() {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        if (VAR) {
          U128 t;
          t.lo = __shfl_xor_sync(0xffffffffu, s2.lo, o);
          t.hi = __shfl_xor_sync(0xffffffffu, s2.hi, o);
          add_u128(s2, t);
        }
      }
      if (lane == 0) {
        unsigned long long* a = acc + 4 * (uint64_t)cur;
        atomic_add_u128(a, (unsigned long long)s1, s1 < 0 ? ~0ull : 0ull);
        if (VAR) atomic_add_u128(a + 2, s2.lo, s2.hi);
        __threadfence();
        const unsigned int need = (unsigned int)(F[cur].ntiles * NCW);
        const unsigned int prev = atomicAdd(&done[cur], cnt);
        if (prev + cnt == need) {  // this warp completes the field
          __threadfence();
          const volatile unsigned long long* va = a;
          const __int128 S1 = (__int128)(((unsigned __int128)va[1] << 64) | va[0]);
          U128 S2 = {va[2], va[3]};
          const Info& h = F[cur].h;
          results[cur] = moment_finish(S1, S2, h.n, h.eps_q, VAR);
          a[0] = a[1] = a[2] = a[3] = 0;
          done[cur] = 0;
        }
      }
      s1 = 0;
      s2 = {0, 0};
      cnt = 0;
    };
    RingPos rp{0, 0u};
    for (;;) {
      const int st = rp.s;
      mbar_wait(&ready[st], rp.par, status);
      const unsigned long long t = stage_tile[st];
      if (t >= total_tiles) break;
      const uint32_t f = stage_field[st];
      if (f != cur) {
        if (cur != ~0u) flush();
        cur = f;
      }
      moments_octet<VAR>(stages[st], ring, g, j, w, S, wlo, whi, s1, s2, [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
      });
      cnt++;
      rp.next<STAGES>();
    }
    if (cur != ~0u) flush();
  }
}

// ---------------------------------------------------------------- batched reductions on super-tiles
// The same per-field accumulators as k_bmoments, fed by the super-tile
// pipeline of the single-stream reductions: a stage holds up to STILES
// consecutive tiles of one field (a stage never spans two fields), copied
// with four bulk copies and located by the plan's per-field prefixes; the
// consumer warps run the single-stream mean (bit-sliced column sums) or
// variance (octet decode) on their tile and flush a field's sums when their
// next stage belongs to another field.
// Launch shapes: NT tiles per stage = warps per block group (a warp takes a
// tile), GROUPS groups taking the stages in turn, STAGES stages in the ring,
// GMAX plane groups decoded (4: any rate; 2: rates below 16; 1: below 8).
template <int NT, int GROUPS>
__host__ __device__ constexpr int bs_threads() { return (NT * GROUPS + 1) * 32; }
// The decompression stages each compute warp's 4 KB of output in a shared box.
template <int MODE, int NT, int GROUPS>
__host__ __device__ constexpr size_t bs_box_bytes() { return MODE == 2 ? (size_t)NT * GROUPS * 4096 : 0; }
// Plane-ring words: 176 KB, less the decompression's boxes.
template <int MODE, int NT, int GROUPS, int STAGES>
__host__ __device__ constexpr uint32_t bs_ring() {
  return MODE == 2 ? (uint32_t)(((232448 - 3072 - 128 - bs_box_bytes<MODE, NT, GROUPS>() -
                                  STAGES * sizeof(SStageT<NT>)) / 8) & ~(size_t)1)
                   : 22528u;
}

// Adds a warp's sums of field f to the field's accumulators; the warp whose
// tiles complete the field finishes it (lane 0 holds s1 / s2 after the warp
// reduction inside).
template <bool VAR>
__device__ __forceinline__ void bflush(const BField* F, uint32_t f, __int128 s1, U128 s2,
                                       unsigned int cnt, unsigned long long* acc,
                                       unsigned int* done, double* results) {
  s1 = warp_sum_i128(s1);
  if (VAR) s2 = warp_sum_u128(s2);
  if ((threadIdx.x & 31) == 0 && cnt) {
    unsigned long long* a = acc + 4 * (uint64_t)f;
    atomic_add_u128(a, (unsigned long long)s1, (unsigned long long)((unsigned __int128)s1 >> 64));
    if (VAR) atomic_add_u128(a + 2, s2.lo, s2.hi);
    __threadfence();
    const unsigned int need = (unsigned int)F[f].ntiles;
    const unsigned int prev = atomicAdd(&done[f], cnt);
    if (prev + cnt == need) {  // this warp completes the field
      __threadfence();
      const volatile unsigned long long* va = a;
      const __int128 S1 = (__int128)(((unsigned __int128)va[1] << 64) | va[0]);
      U128 S2 = {va[2], va[3]};
      const Info& h = F[f].h;
      results[f] = moment_finish(S1, S2, h.n, h.eps_q, VAR);
      a[0] = a[1] = a[2] = a[3] = 0;
      done[f] = 0;
    }
  }
}

// MODE 0: mean, 1: variance (per-field exact sums, finished by the warp that
// completes a field), 2: decompression into each field's output outs[f].
template <int MODE, int NT, int GROUPS, int STAGES, int GMAX>
__global__ void __launch_bounds__(bs_threads<NT, GROUPS>(), 1) k_bsuper(
    const BField* __restrict__ F, uint32_t nf, uint64_t total_tiles,
    const unsigned long long* __restrict__ pre, unsigned long long* acc, unsigned int* done,
    double* results, int* status, float* const* __restrict__ outs) {
  constexpr int BS_STAGES = STAGES, BS_GW = NT, BS_GROUPS = GROUPS, BS_NCW = NT * GROUPS;
  constexpr uint32_t BS_RING = bs_ring<MODE, NT, GROUPS, STAGES>();
  using St = SStageT<NT>;
  extern __shared__ __align__(16) uint8_t dyn[];
  // decompression: one 4 KB output box per compute warp first (128-byte aligned;
  // its launch adds the 128 bytes of slack); the reductions start at dyn
  uint8_t* const dbase =
      MODE == 2 ? reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 127) &
                                             ~(uintptr_t)127)
                : dyn;
  int4* const box = reinterpret_cast<int4*>(dbase) + 256 * (threadIdx.x >> 5);
  St* stages = reinterpret_cast<St*>(dbase + bs_box_bytes<MODE, NT, GROUPS>());
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + BS_STAGES);
  __shared__ uint64_t full[BS_STAGES], empty[BS_STAGES];
  __shared__ BStageMeta s_meta[BS_STAGES];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const uint64_t G = gridDim.x;
  const uint64_t t_begin = total_tiles * blockIdx.x / G;
  const uint64_t t_end = total_tiles * (blockIdx.x + 1) / G;
  if (tid == 0) {
    for (int k = 0; k < BS_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], BS_GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (w == BS_NCW) {
    __shared__ uint32_t s_beg[BS_STAGES];
    bsuper_loader<NT, BS_STAGES, BS_RING, BS_GROUPS>(stages, ring, s_beg, full, empty, s_meta, F,
                                                     nf, pre, t_begin, t_end, status);
  } else if (w < BS_NCW) {
    const int grp = w / BS_GW, ti = w % BS_GW;
    const lanes::Shifts K = lanes::make_shifts(nf != 0 ? 1u : 0u);
    MeanAccT<(GMAX <= 1 ? 8 : 16)> A;
    A.init();
    long long v1 = 0;
    U128 v2 = {0, 0};
    uint32_t cur = ~0u;
    unsigned int cnt = 0;
    auto flush = [&]() {
      if (MODE == 1) {
        bflush<true>(F, cur, (__int128)v1, v2, cnt, acc, done, results);
        v1 = 0;
        v2 = {0, 0};
      } else if (MODE == 0) {
        A.flush();
        bflush<false>(F, cur, A.s1, U128{0, 0}, cnt, acc, done, results);
        A.s1 = 0;
      }
      cnt = 0;
    };
    for (uint64_t k = 0;; k++) {
      const uint64_t u = k * BS_GROUPS + grp;  // stage use taken by this group
      const int sk = (int)(u % BS_STAGES);
      if (!mbar_wait_warp(&full[sk], (uint32_t)((u / BS_STAGES) & 1), status)) break;
      const BStageMeta meta = s_meta[sk];
      if (meta.nt == 0) break;
      if (meta.f != cur) {
        if (cur != ~0u) flush();
        cur = meta.f;
      }
      if (ti < (int)meta.nt) {  // warp-uniform
        const St& sg = stages[sk];
        const Info& h = F[cur].h;
        const uint64_t tile = meta.t0 + ti;
        const uint64_t ntiles = F[cur].ntiles;
        const int lastlen = (int)(h.n - (h.nb - 1) * L);
        const TileRates tr = tile_rates(sg, ti, tile, h.nb);
        const uint64_t* sgn = sg.sign + sg.sbase + sg.tnc[ti];
        const uint64_t* pls = ring + sg.pring + sg.pbase + sg.tr[ti];
        if (MODE == 2) {  // two lanes per block, as the single-stream decompression
          float* __restrict__ x = outs[cur];
          const int hf = lane & 1, m = lane >> 1;
          const float e2 = 2.0f * h.eps_q;
          const bool small = h.qbound < (1u << 22);
          const uint32_t* sgn32 = reinterpret_cast<const uint32_t*>(sgn);
          const uint32_t* pls32 = reinterpret_cast<const uint32_t*>(pls);
          const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
          for (int it = 0; it < steps; it++) {
            const int b = 16 * it + m;
            uint32_t r, ex;
            tile_block(tr, b, r, ex);
            const int len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
            const int nval = min(max(len - 32 * hf, 0), 32);
            const int O = len ? sg.outlier[TILE * ti + b] : 0;
            const uint32_t sw = r ? sgn32[2 * (ex >> 16) + hf] : 0u;
            const int Rw = min((int)__reduce_max_sync(0xffffffffu, r), 8 * GMAX - 1);
            int v[32];
            {
              uint32_t t[32];
              lanes::twos_planes_any<8 * GMAX - 1>(Rw, pls32 + 2 * (ex & 0xffffu) + hf, (int)r,
                                                   sw, t);
              half_prefix_any<GMAX>(Rw, t, hf == 0, K, v);
            }
            const int tot0 = __shfl_xor_sync(0xffffffffu, v[31], 1);
            const int qb = O + (hf ? tot0 : 0);
            if (small) {  // uniform over the stream: no per-value select
#pragma unroll
              for (int i = 0; i < 32; i++) v[i] = __float_as_int(dequant_small(v[i] + qb, e2));
            } else {
#pragma unroll
              for (int i = 0; i < 32; i++) v[i] = __float_as_int(dequant_any(v[i] + qb, e2));
            }
            const uint64_t s0 = (tile * TILE + 16 * (uint64_t)it) * L;  // the step's first value
            if (s0 + 16 * L <= h.n) {
              // the lane's row into the warp's box (chunk j of row r at chunk j ^ (r % 8)),
              // then the step's 4 KB stored as 8 coalesced 512-byte warp stores
#pragma unroll
              for (int j = 0; j < 8; j++)
                box[8 * lane + (j ^ (lane & 7))] =
                    make_int4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
              __syncwarp();
              int4* dst = reinterpret_cast<int4*>(x + s0);
#pragma unroll
              for (int j = 0; j < 8; j++) {
                const int row = 4 * j + (lane >> 3), c = lane & 7;
                __stcs(dst + 32 * j + lane, box[8 * row + (c ^ (row & 7))]);
              }
              __syncwarp();  // the box is read before the next step writes it
            } else {
              const uint64_t i0 = (tile * TILE + b) * L + 32 * hf;
#pragma unroll
              for (int i = 0; i < 32; i++)
                if (i < nval) x[i0 + i] = __int_as_float(v[i]);
            }
          }
        } else if (MODE == 0) {
#pragma unroll 1
          for (int jj = 0; jj < 2; jj++) {  // blocks 2 lane and 2 lane + 1
            const int b = 2 * lane + jj;
            const uint32_t r = jj ? tr.r1 : tr.r0, ex = jj ? tr.e1 : tr.e0;
            const int len = (b < tr.nvt - 1) ? L
                            : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
            const int O = sg.outlier[TILE * ti + b];
            const uint64_t sw = r ? sgn[ex >> 16] : 0ull;
            mean_block((int)r, len, O, sw, reinterpret_cast<const uint2*>(pls + (ex & 0xffffu)), A);
          }
        } else {
          var_tile<GMAX>(sg, ring, ti, tr, tile, ntiles, lastlen, h.qbound < (1u << 13), K, v1, v2);
        }
        cnt++;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sk]);
    }
    if (cur != ~0u) flush();
  }
}

template <int MODE, int NT, int GROUPS, int STAGES, int GMAX>
cudaError_t launch_bsuper_shape(int num_sms, cudaStream_t s, const BField* F, uint32_t nf,
                                uint64_t total_tiles, const unsigned long long* pre,
                                unsigned long long* acc, unsigned int* done, double* results,
                                int* status, float* const* outs) {
  constexpr int threads = bs_threads<NT, GROUPS>();
  auto kern = k_bsuper<MODE, NT, GROUPS, STAGES, GMAX>;
  const size_t smem = (MODE == 2 ? 128 + bs_box_bytes<MODE, NT, GROUPS>() : 0) +
                      STAGES * sizeof(SStageT<NT>) +
                      bs_ring<MODE, NT, GROUPS, STAGES>() * sizeof(uint64_t);
  smem_attr<k_bsuper<MODE, NT, GROUPS, STAGES, GMAX>>(smem);
  kern<<<persistent_grid(kern, threads, num_sms, smem), threads, smem, s>>>(
      F, nf, total_tiles, pre, acc, done, results, status, outs);
  return cudaGetLastError();
}

// The super-tile launch of one shape: wpg warps per block group (8: two
// groups of 8 over 4 stages of 8 tiles; 4: four groups of 4 over 8 stages of
// 4 tiles) and gmax plane groups (4, 2 or 1).
template <int MODE>
cudaError_t launch_bsuper(int num_sms, cudaStream_t s, const BField* F, uint32_t nf,
                          uint64_t total_tiles, const unsigned long long* pre,
                          unsigned long long* acc, unsigned int* done, double* results,
                          int* status, float* const* outs = nullptr, int wpg = 8,
                          int gmax = 4) {
#define HZ_BS(W, GR, ST, GM)                                                                  \
  if (wpg == W && gmax == GM)                                                                 \
    return launch_bsuper_shape<MODE, W, GR, ST, GM>(num_sms, s, F, nf, total_tiles, pre, acc, \
                                                    done, results, status, outs);
  HZ_BS(8, 2, 4, 4) HZ_BS(8, 2, 4, 2) HZ_BS(8, 2, 4, 1)
  HZ_BS(4, 4, 8, 4) HZ_BS(4, 4, 8, 2) HZ_BS(4, 4, 8, 1)
#undef HZ_BS
  return cudaErrorInvalidValue;
}

template <bool VAR, int STAGES>
cudaError_t launch_bmoments(int grid, cudaStream_t s, const BField* F, uint32_t nf,
                            uint64_t total_tiles, const unsigned long long* pre,
                            unsigned long long* acc, unsigned int* done, double* results,
                            int* status) {
  const size_t smem = STAGES * sizeof(InStage) + 8192 * sizeof(uint64_t);
  smem_attr<k_bmoments<VAR, STAGES>>(smem);
  k_bmoments<VAR, STAGES><<<grid, CONSUMER_THREADS, smem, s>>>(F, nf, total_tiles, pre, acc,
                                                               done, results, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched negate / add_scalar
// In place over the fields' metadata regions laid end to end as 16-byte
// chunks (negation: outliers and sign words; scalar addition: outliers).
__global__ void k_brho(BField* F, uint32_t nf, double s, int* status) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  BField& b = F[f];
  long long rho = 0;
  if (!quantize_scalar(s, b.h.eps_q, rho)) {
    set_status(status, HOSZP_ERR_RANGE);
    b.rho = 0;
    return;
  }
  const long long arho = rho < 0 ? -rho : rho;
  if ((long long)b.h.qbound + arho > HOSZP_QLIM) {
    set_status(status, HOSZP_ERR_OVERFLOW);
    b.rho = 0;
    return;
  }
  b.rho = rho;
  if (rho != 0) {  // the header's bound grows by |rho| (Sec. V-A)
    b.h.qbound = (uint32_t)((long long)b.h.qbound + arho);
    reinterpret_cast<hoszp_header*>(b.cw)->qbound = b.h.qbound;
  }
}

template <bool NEG>
__global__ void __launch_bounds__(512) k_bmeta(const BField* __restrict__ F, uint32_t nf,
                                               uint64_t total_ch) {
  constexpr int OP = NEG ? 0 : 1;
  const uint64_t G = gridDim.x;
  const uint64_t c_begin = total_ch * blockIdx.x / G, c_end = total_ch * (blockIdx.x + 1) / G;
  if (c_begin >= c_end) return;
  __shared__ uint32_t s_f;
  if (threadIdx.x == 0) s_f = field_of_chunk(F, nf, OP, c_begin);
  __syncthreads();
  for (uint32_t f = s_f; f < nf; f++) {
    const BField& b = F[f];
    const uint64_t f0 = b.ch0[OP], f1 = f0 + b.nch[OP];
    if (f0 >= c_end) break;
    const uint64_t lo = max(f0, c_begin), hi = min(f1, c_end);
    if (lo >= hi) continue;
    const int r32 = (int)b.rho;
    if (!NEG && r32 == 0) continue;
    const Info& h = b.h;
    uint4* base = reinterpret_cast<uint4*>(b.cw + h.o_out);  // chunk i of the region
    constexpr int U = 4;
    const uint64_t n = hi - lo, off = lo - f0;
    for (uint64_t i0 = threadIdx.x; i0 < n; i0 += U * blockDim.x) {
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; u++)
        if (i0 + u * blockDim.x < n) v[u] = base[off + i0 + u * blockDim.x];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint64_t i = i0 + u * blockDim.x;
        if (i >= n) break;
        const uint64_t bpos = h.o_out + 16 * (off + i);
        if (bpos < h.o_sign) {  // 4 outliers (padding past nb unchanged)
          const uint64_t k0 = (bpos - h.o_out) >> 2;
          uint32_t* wv = reinterpret_cast<uint32_t*>(&v[u]);
#pragma unroll
          for (int k = 0; k < 4; k++)
            if (k0 + k < h.nb)
              wv[k] = NEG ? (uint32_t)(-(int)wv[k]) : (uint32_t)((int)wv[k] + r32);
        } else if (NEG) {  // sign words (the second may be a plane word)
          v[u].x = ~v[u].x;
          v[u].y = ~v[u].y;
          if (bpos + 8 < h.o_plane) {
            v[u].z = ~v[u].z;
            v[u].w = ~v[u].w;
          }
        }
        base[off + i] = v[u];
      }
    }
  }
}

}  // namespace
}  // namespace hz

using namespace hz;

namespace {

int run_moments(hoszp_batch* b, bool var, const BatchCfg& c, double* d_results,
                cudaStream_t s) {
  const int grid = b->num_sms * c.cps;
  cudaError_t e;
  if (c.variant == 2)
    e = var ? launch_bsuper<1>(b->num_sms, s, b->d_fields, b->nf, b->total_tiles, b->d_pre,
                               b->d_acc, b->d_done, d_results, b->status, nullptr, c.wpg, c.gmax)
            : launch_bsuper<0>(b->num_sms, s, b->d_fields, b->nf, b->total_tiles, b->d_pre,
                               b->d_acc, b->d_done, d_results, b->status, nullptr, c.wpg, c.gmax);
  else if (var)
    e = c.variant == 0 ? launch_bmoments<true, 8>(grid, s, b->d_fields, b->nf, b->total_tiles,
                                                   b->d_pre, b->d_acc, b->d_done, d_results,
                                                   b->status)
                       : launch_bmoments<true, 4>(grid, s, b->d_fields, b->nf, b->total_tiles,
                                                   b->d_pre, b->d_acc, b->d_done, d_results,
                                                   b->status);
  else
    e = c.variant == 0 ? launch_bmoments<false, 8>(grid, s, b->d_fields, b->nf, b->total_tiles,
                                                    b->d_pre, b->d_acc, b->d_done, d_results,
                                                    b->status)
                       : launch_bmoments<false, 4>(grid, s, b->d_fields, b->nf, b->total_tiles,
                                                    b->d_pre, b->d_acc, b->d_done, d_results,
                                                    b->status);
  return rc_of(e);
}

int run_decompress(hoszp_batch* b, const BatchCfg& c, float* const* d_outs, cudaStream_t s) {
  return rc_of(launch_bsuper<2>(b->num_sms, s, b->d_fields, b->nf, b->total_tiles, b->d_pre,
                                b->d_acc, b->d_done, nullptr, b->status, d_outs, c.wpg, c.gmax));
}

// The autotuner's candidates for op (0 mean, 1 variance, 2 decompression):
// pipeline depth x CTAs per SM of the tile pipeline (reductions only), and
// warps per block group x plane groups of the super-tile pipeline. The
// rate-specialised shapes decode fewer plane groups and are offered only
// where they are exact for every field of the plan: the variance needs
// ceil((rmax + 1) / 8) groups (the rates' planes and the sign), as does the
// decompression; the mean is exact with any column count
// (planes above the columns go through popcounts), so its 8-column shape is
// always offered.
int candidates(const hoszp_batch* b, int op, BatchCfg out[12]) {
  int n = 0;
  if (op < 2)
    for (int v = 0; v < 2; v++)
      for (int cps = 1; cps <= 2; cps++) out[n++] = BatchCfg{v, cps, 8, 4};
  int gm[2] = {4, 0}, ng = 1;
  const int need = op == 0 ? 1 : (b->rmax + 8) >> 3;  // the rates' planes and the sign
  if (need == 1 || need == 2) gm[ng++] = need;
  for (int w : {8, 4})
    for (int i = 0; i < ng; i++) out[n++] = BatchCfg{2, 1, w, gm[i]};
  return n;
}

}  // namespace

extern "C" {

int hoszp_batch_create(hoszp_ctx* ctx, uint32_t nfields, const void* const* d_streams,
                       const size_t* stream_bytes, hoszp_batch** out) {
  if (!ctx || !out || nfields == 0 || !d_streams || !stream_bytes) return HOSZP_ERR_ARG;
  *out = nullptr;
  for (uint32_t f = 0; f < nfields; f++) {
    if (!d_streams[f] || ((uintptr_t)d_streams[f] & 15u) || stream_bytes[f] < HOSZP_HEADER_BYTES)
      return HOSZP_ERR_ARG;
  }
  Ws ws;
  int device = 0, sms = 0;
  int rc = ctx_prepare(ctx, 1, &ws, &device, &sms);
  if (rc) return rc;
  DeviceGuard guard(device);
  // parse every header on the device
  std::vector<BField> F(nfields);
  void* tmp = nullptr;
  const size_t tbytes = nfields * (sizeof(void*) + sizeof(uint64_t)) + nfields * sizeof(BField);
  if (cudaMalloc(&tmp, tbytes) != cudaSuccess) return rc_of(cudaErrorMemoryAllocation);
  const uint8_t** d_ptrs = (const uint8_t**)tmp;
  uint64_t* d_bytes = (uint64_t*)(d_ptrs + nfields);
  BField* d_tmpF = (BField*)(d_bytes + nfields);
  std::vector<uint64_t> hb(stream_bytes, stream_bytes + nfields);
  cudaMemcpy(d_ptrs, d_streams, nfields * sizeof(void*), cudaMemcpyHostToDevice);
  cudaMemcpy(d_bytes, hb.data(), nfields * sizeof(uint64_t), cudaMemcpyHostToDevice);
  k_bparse<<<(nfields + 127) / 128, 128>>>(d_ptrs, d_bytes, nfields, d_tmpF, ws.status);
  int st = 0;
  if (cudaMemcpy(F.data(), d_tmpF, nfields * sizeof(BField), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      cudaMemcpy(&st, ws.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaFree(tmp);
    return rc_of(cudaErrorUnknown);
  }
  cudaFree(tmp);
  if (st) {
    cudaMemset(ws.status, 0, sizeof(int));
    return st;
  }
  // global tile space, prefix offsets, metadata chunk spaces
  uint64_t tiles = 0, pre_words = 0, ch[2] = {0, 0}, max_tiles = 0;
  for (uint32_t f = 0; f < nfields; f++) {
    F[f].tile0 = tiles;
    F[f].pre0 = pre_words;
    for (int o = 0; o < 2; o++) {
      F[f].ch0[o] = ch[o];
      ch[o] += F[f].nch[o];
    }
    tiles += F[f].ntiles;
    pre_words += 2 * (F[f].ntiles + 1);
    max_tiles = std::max<uint64_t>(max_tiles, F[f].ntiles);
  }
  hoszp_batch* b = new hoszp_batch();
  b->ctx = ctx;
  b->device = device;
  b->num_sms = sms;
  b->nf = nfields;
  b->total_tiles = tiles;
  b->total_ch[0] = ch[0];
  b->total_ch[1] = ch[1];
  b->cfg[0] = b->cfg[1] = b->cfg[2] = BatchCfg{2, 1, 8, 4};
  b->rmax = 0;
  for (uint32_t f = 0; f < nfields; f++) {  // |delta| <= 2 max|q|: its bit length bounds the rate
    const uint64_t d = 2ull * F[f].h.qbound;
    const int bits = d ? 64 - __builtin_clzll(d) : 0;
    b->rmax = std::max(b->rmax, std::min(bits, (int)MAX_RATE));
  }
  const size_t fbytes = (nfields * sizeof(BField) + 255) / 256 * 256;
  const size_t pbytes = (pre_words * 8 + 255) / 256 * 256;
  const size_t abytes = (nfields * 32 + 255) / 256 * 256;
  const size_t dbytes = (nfields * 4 + 255) / 256 * 256;
  const size_t xbytes = ((nfields + 1) * 16 + 255) / 256 * 256;  // fpre
  const size_t obytes = (nfields * sizeof(BOut) + 255) / 256 * 256;
  if (cudaMalloc(&b->mem, fbytes + pbytes + abytes + dbytes + 256 + xbytes + obytes) !=
      cudaSuccess) {
    delete b;
    return rc_of(cudaErrorMemoryAllocation);
  }
  uint8_t* m = (uint8_t*)b->mem;
  b->d_fields = (BField*)m;
  b->d_pre = (unsigned long long*)(m + fbytes);
  b->d_acc = (unsigned long long*)(m + fbytes + pbytes);
  b->d_done = (unsigned int*)(m + fbytes + pbytes + abytes);
  b->status = (int*)(m + fbytes + pbytes + abytes + dbytes);
  b->d_fpre = (unsigned long long*)(m + fbytes + pbytes + abytes + dbytes + 256);
  b->d_out = (BOut*)(m + fbytes + pbytes + abytes + dbytes + 256 + xbytes);
  cudaMemcpy(b->d_fields, F.data(), nfields * sizeof(BField), cudaMemcpyHostToDevice);
  {
    std::vector<unsigned long long> fp(2 * (nfields + 1), 0ull);
    for (uint32_t f = 0; f < nfields; f++) {
      fp[2 * (f + 1)] = fp[2 * f] + F[f].h.nnc;
      fp[2 * (f + 1) + 1] = fp[2 * f + 1] + F[f].h.R;
    }
    cudaMemcpy(b->d_fpre, fp.data(), fp.size() * 8, cudaMemcpyHostToDevice);
    b->total_nnc = fp[2 * nfields];
    b->total_R = fp[2 * nfields + 1];
    cudaMemset(b->d_out, 0, obytes);
  }
  cudaMemset(b->d_acc, 0, abytes + dbytes + 256);
  // each stream's rate pre-scan, once
  rc = ctx_prepare(ctx, max_tiles + 1, &ws, &device, &sms);
  if (rc) {
    hoszp_batch_destroy(b);
    return rc;
  }
  Launch lc;
  lc.grid = sms;
  lc.stream = 0;
  for (uint32_t f = 0; f < nfields; f++) {
    const cudaError_t e = launch_scan(lc, F[f].c, F[f].h.size, b->d_pre + F[f].pre0, ws);
    if (e != cudaSuccess) {
      hoszp_batch_destroy(b);
      return rc_of(e);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&st, ws.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    hoszp_batch_destroy(b);
    return rc_of(cudaErrorUnknown);
  }
  if (st) {
    cudaMemset(ws.status, 0, sizeof(int));
    hoszp_batch_destroy(b);
    return st;
  }
  *out = b;
  return HOSZP_OK;
}

void hoszp_batch_destroy(hoszp_batch* b) {
  if (!b) return;
  DeviceGuard guard(b->device);
  if (b->mem) cudaFree(b->mem);
  delete b;
}

int hoszp_batch_get_status(hoszp_batch* b, int* status) {
  if (!b || !status) return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  int v = 0, vc = 0;
  // the plan's own word, then the context's (the word scan of the producing
  // operators reports there)
  int* cst = ctx_status_word(b->ctx);
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&v, b->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(b->status, 0, sizeof(int)) != cudaSuccess ||
      (cst && (cudaMemcpy(&vc, cst, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
               cudaMemset(cst, 0, sizeof(int)) != cudaSuccess))) {
    cudaGetLastError();
    *status = HOSZP_ERR_CUDA;
    return HOSZP_ERR_CUDA;
  }
  *status = v ? v : vc;
  return HOSZP_OK;
}

int hoszp_batch_info(const hoszp_batch* b, uint32_t* nfields, uint64_t* total_tiles) {
  if (!b) return HOSZP_ERR_ARG;
  if (nfields) *nfields = b->nf;
  if (total_tiles) *total_tiles = b->total_tiles;
  return HOSZP_OK;
}

int hoszp_batch_mean(hoszp_batch* b, double* d_results, hoszp_stream_t stream) {
  if (!b || !d_results || ((uintptr_t)d_results & 7u)) return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  return run_moments(b, false, b->cfg[0], d_results, (cudaStream_t)stream);
}

int hoszp_batch_var(hoszp_batch* b, double* d_results, hoszp_stream_t stream) {
  if (!b || !d_results || ((uintptr_t)d_results & 7u)) return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  return run_moments(b, true, b->cfg[1], d_results, (cudaStream_t)stream);
}

int hoszp_batch_decompress(hoszp_batch* b, float* const* d_outs, hoszp_stream_t stream) {
  if (!b || !d_outs || ((uintptr_t)d_outs & 7u)) return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  return run_decompress(b, b->cfg[2], d_outs, (cudaStream_t)stream);
}

int hoszp_batch_negate(hoszp_batch* b, hoszp_stream_t stream) {
  if (!b) return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  if (b->total_ch[0] == 0) return HOSZP_OK;
  k_bmeta<true><<<b->num_sms * 4, 512, 0, (cudaStream_t)stream>>>(b->d_fields, b->nf,
                                                                  b->total_ch[0]);
  return rc_of(cudaGetLastError());
}

int hoszp_batch_add_scalar(hoszp_batch* b, double s, hoszp_stream_t stream) {
  if (!b || !(s == s) || s - s != 0.0) return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  const cudaStream_t cs = (cudaStream_t)stream;
  k_brho<<<(b->nf + 127) / 128, 128, 0, cs>>>(b->d_fields, b->nf, s, b->status);
  if (b->total_ch[1] == 0) return rc_of(cudaGetLastError());
  k_bmeta<false><<<b->num_sms * 4, 512, 0, cs>>>(b->d_fields, b->nf, b->total_ch[1]);
  return rc_of(cudaGetLastError());
}

int hoszp_batch_tune(hoszp_batch* b, double* d_results, float* const* d_outs,
                     hoszp_stream_t stream) {
  if (!b || !d_results || ((uintptr_t)d_results & 7u) || ((uintptr_t)d_outs & 7u))
    return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  const cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return rc_of(cudaErrorUnknown);
  int rc = HOSZP_OK;
  for (int op = 0; op < 3 && !rc; op++) {
    if (op == 2 && !d_outs) break;  // decompression is tuned when outputs are given
    BatchCfg cands[12];
    const int nc = candidates(b, op, cands);
    float best = 1e30f;
    BatchCfg pick = b->cfg[op];
    for (int i = 0; i < nc && !rc; i++) {
      const BatchCfg& c = cands[i];
      auto run = [&]() {
        return op == 2 ? run_decompress(b, c, d_outs, s) : run_moments(b, op == 1, c, d_results, s);
      };
      if ((rc = run())) break;  // warm-up
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3 && !rc; r++) rc = run();
      cudaEventRecord(e1, s);
      if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = rc ? rc : HOSZP_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    b->cfg[op] = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int hoszp_batch_shapes(const hoszp_batch* b, int op) {
  if (!b || op < 0 || op > 2) return HOSZP_ERR_ARG;
  BatchCfg c[12];
  return candidates(b, op, c);
}

int hoszp_batch_set_shape(hoszp_batch* b, int op, int index) {
  if (!b || op < 0 || op > 2) return HOSZP_ERR_ARG;
  BatchCfg c[12];
  const int n = candidates(b, op, c);
  if (index < 0 || index >= n) return HOSZP_ERR_ARG;
  b->cfg[op] = c[index];
  return HOSZP_OK;
}

int hoszp_batch_config(const hoszp_batch* b, int op, int* stages, int* ctas_per_sm,
                       int* warps_per_group, int* plane_groups) {
  if (!b || op < 0 || op > 2) return HOSZP_ERR_ARG;
  const BatchCfg& c = b->cfg[op];
  if (stages) *stages = c.variant == 0 ? 8 : c.variant == 1 ? 4 : (c.wpg == 8 ? 4 : 8);
  if (ctas_per_sm) *ctas_per_sm = c.cps;
  // the tile pipeline's 16 compute warps each take a quarter of a tile's blocks
  if (warps_per_group) *warps_per_group = c.variant == 2 ? c.wpg : 16;
  if (plane_groups) *plane_groups = c.variant == 2 ? c.gmax : 4;
  return HOSZP_OK;
}

}  // extern "C"
