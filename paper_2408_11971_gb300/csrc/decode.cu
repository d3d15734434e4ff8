// decode.cu — full decompression (inverse of every pipeline step, Fig. 2) and
// the univariate reductions mean and variance (Sec. V-B, workflow 3), which
// sum the quantized integers exactly and finish in FP64.
#include <cfloat>

#include "hz_moments.cuh"
#include "hz_var.cuh"
#include "hz_super.cuh"
#include "hz_kernels.cuh"

namespace hz {

// ---------------------------------------------------------------- mean / variance
// Mean alone: the bit-sliced column sums of hz_moments.cuh over the
// super-tile pipeline of hz_super.cuh. MEAN_GROUPS groups of STILES compute
// warps take the stages in turn; warp i of a group takes tile i of the stage,
// and lane l blocks 2l and 2l+1 of that tile.
constexpr int MEAN_GW = STILES;  // warps per group: one per tile of a stage
constexpr int MEAN_GROUPS = 2;   // groups per CTA
constexpr int MEAN_NCW = MEAN_GW * MEAN_GROUPS;
constexpr int MEAN_THREADS = (MEAN_NCW + 1) * 32;  // + loader warp
constexpr int MEAN_STAGES = 4;
constexpr uint32_t MEAN_RING = 22528;  // plane-ring words (176 KB)
constexpr int MEAN_MIN_CTAS = 1;       // resident CTAs per SM (shared memory)

__device__ __forceinline__ void cta_sum_i128_partial(__int128 v, Partial* out, __int128* s_w) {
  const int tid = threadIdx.x;
  v = warp_sum_i128(v);
  if ((tid & 31) == 0) s_w[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    __int128 t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
    Partial p;
    p.s1_lo = (long long)(unsigned long long)t;
    p.s1_hi = (long long)(t >> 64);
    p.s2_lo = 0;
    p.s2_hi = 0;
    *out = p;
  }
}

__global__ void __launch_bounds__(MEAN_THREADS, MEAN_MIN_CTAS) k_mean(
    const uint8_t* __restrict__ c, uint64_t c_bytes, double* result, Ws ws) {
  extern __shared__ __align__(16) uint8_t dyn[];
  SStage* stages = reinterpret_cast<SStage*>(dyn);
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + MEAN_STAGES);
  __shared__ uint64_t full[MEAN_STAGES], empty[MEAN_STAGES];
  __shared__ unsigned long long stage_st[MEAN_STAGES];
  __shared__ uint32_t s_ts[TS_MAX];
  __shared__ __int128 s_w[MEAN_THREADS / 32];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const Info h = parse_header(c, c_bytes);
  const unsigned long long epoch = launch_epoch(ws);
  int bad = h.ok ? 0 : HOSZP_ERR_FORMAT;
  const uint64_t ntiles = h.ok ? ntiles_of(h.nb) : 0;
  const uint64_t nst = nsuper_of(ntiles);
  // full: the loader's arrival; empty: the MEAN_GW warps of the group that took the stage
  if (tid == 0) {
    for (int k = 0; k < MEAN_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], MEAN_GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const SRange rg = range_sums(c, h, ntiles, nst, s_ts, ws, epoch, bad);
  __syncthreads();
  MeanAcc A;
  A.init();
  if (w == MEAN_NCW) {
    __shared__ uint32_t s_beg[MEAN_STAGES];
    super_loader<MEAN_STAGES, MEAN_RING, MEAN_GROUPS>(stages, ring, s_beg, full, empty, stage_st,
                                                       c, h, rg, s_ts, ws, epoch);
  } else if (w < MEAN_NCW) {
    const int grp = w / MEAN_GW, ti = w % MEAN_GW;
    const int lastlen = (int)(h.n - (h.nb - 1) * L);
    for (uint64_t k = 0;; k++) {
      const uint64_t u = k * MEAN_GROUPS + grp;  // stage use taken by this group
      const int sk = (int)(u % MEAN_STAGES);
      if (!mbar_wait_warp(&full[sk], (uint32_t)((u / MEAN_STAGES) & 1), ws.status)) break;
      const unsigned long long s = stage_st[sk];
      if (s == ~0ull) break;
      const SStage& sg = stages[sk];
      const uint64_t tile = (uint64_t)STILES * s + ti;
      const TileRates tr = tile_rates(sg, ti, tile, h.nb);
      const uint64_t* sgn = sg.sign + sg.sbase + sg.tnc[ti];
      const uint64_t* pls = ring + sg.pring + sg.pbase + sg.tr[ti];
#pragma unroll 1
      for (int j = 0; j < 2; j++) {  // blocks 2 lane and 2 lane + 1
        const int b = 2 * lane + j;
        const uint32_t r = j ? tr.r1 : tr.r0, ex = j ? tr.e1 : tr.e0;
        const int len = (b < tr.nvt - 1) ? L
                        : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
        const int O = sg.outlier[TILE * ti + b];
        const uint64_t sw = r ? sgn[ex >> 16] : 0ull;
        mean_block((int)r, len, O, sw, reinterpret_cast<const uint2*>(pls + (ex & 0xffffu)), A);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sk]);
    }
    A.flush();
  }
  cta_sum_i128_partial(A.s1, &ws.partials[blockIdx.x], s_w);
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && w == 0) {
    __int128 S1;
    U128 S2;
    sum_partials_warp(ws.partials, gridDim.x, S1, S2);
    const bool tot_ok = range_totals_ok(ws, h);
    if (tid == 0) {
      double res = 0.0;
      if (h.ok && !tot_ok) {
        set_status(ws.status, HOSZP_ERR_FORMAT);
      } else if (h.ok && h.n == 0) {
        set_status(ws.status, HOSZP_ERR_ARG);
      } else if (h.ok) {
        res = moment_finish(S1, S2, h.n, h.eps_q, false);
      }
      *result = res;
      launch_reset(ws);
    }
  }
}

// Variance over the same super-tile pipeline: warp i of a group takes tile i
// of the stage and decodes it 16 blocks at a time, two lanes per block (one
// per 32-position half, hz_lanes.cuh), summing q and q^2 exactly.
__global__ void __launch_bounds__(MEAN_THREADS, MEAN_MIN_CTAS) k_var(
    const uint8_t* __restrict__ c, uint64_t c_bytes, double* result, unsigned long long* sums,
    int take_sqrt, Ws ws) {
  extern __shared__ __align__(16) uint8_t dyn[];
  SStage* stages = reinterpret_cast<SStage*>(dyn);
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + MEAN_STAGES);
  __shared__ uint64_t full[MEAN_STAGES], empty[MEAN_STAGES];
  __shared__ unsigned long long stage_st[MEAN_STAGES];
  __shared__ uint32_t s_ts[TS_MAX];
  __shared__ long long s_s1[MEAN_THREADS / 32];
  __shared__ U128 s_s2[MEAN_THREADS / 32];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const Info h = parse_header(c, c_bytes);
  const unsigned long long epoch = launch_epoch(ws);
  int bad = h.ok ? 0 : HOSZP_ERR_FORMAT;
  const uint64_t ntiles = h.ok ? ntiles_of(h.nb) : 0;
  const uint64_t nst = nsuper_of(ntiles);
  if (tid == 0) {
    for (int k = 0; k < MEAN_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], MEAN_GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const SRange rg = range_sums(c, h, ntiles, nst, s_ts, ws, epoch, bad);
  __syncthreads();
  long long s1 = 0;  // per thread: |q| <= 2^30, far fewer than 2^32 values per thread
  U128 s2 = {0, 0};
  if (w == MEAN_NCW) {
    __shared__ uint32_t s_beg[MEAN_STAGES];
    super_loader<MEAN_STAGES, MEAN_RING, MEAN_GROUPS>(stages, ring, s_beg, full, empty, stage_st,
                                                       c, h, rg, s_ts, ws, epoch);
  } else if (w < MEAN_NCW) {
    const int grp = w / MEAN_GW, ti = w % MEAN_GW;
    const int lastlen = (int)(h.n - (h.nb - 1) * L);
    const bool qsmall = h.qbound < (1u << 13);  // the header bounds every |q|
    const lanes::Shifts K = lanes::make_shifts(c_bytes != 0 ? 1u : 0u);
    for (uint64_t k = 0;; k++) {
      const uint64_t u = k * MEAN_GROUPS + grp;  // stage use taken by this group
      const int sk = (int)(u % MEAN_STAGES);
      if (!mbar_wait_warp(&full[sk], (uint32_t)((u / MEAN_STAGES) & 1), ws.status)) break;
      const unsigned long long s = stage_st[sk];
      if (s == ~0ull) break;
      const SStage& sg = stages[sk];
      const uint64_t tile = (uint64_t)STILES * s + ti;
      const TileRates tr = tile_rates(sg, ti, tile, h.nb);
      var_tile(sg, ring, ti, tr, tile, ntiles, lastlen, qsmall, K, s1, s2);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sk]);
    }
  }
  // CTA reduction -> per-CTA partial
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    U128 t;
    t.lo = __shfl_xor_sync(0xffffffffu, s2.lo, o);
    t.hi = __shfl_xor_sync(0xffffffffu, s2.hi, o);
    add_u128(s2, t);
  }
  if (lane == 0) {
    s_s1[w] = s1;
    s_s2[w] = s2;
  }
  __syncthreads();
  if (tid == 0) {
    __int128 t1 = 0;
    U128 t2 = {0, 0};
    for (int k = 0; k < MEAN_THREADS / 32; k++) {
      t1 += s_s1[k];
      add_u128(t2, s_s2[k]);
    }
    Partial p;
    p.s1_lo = (long long)(unsigned long long)t1;
    p.s1_hi = (long long)(t1 >> 64);
    p.s2_lo = t2.lo;
    p.s2_hi = t2.hi;
    ws.partials[blockIdx.x] = p;
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && w == 0) {
    __int128 S1;
    U128 S2;
    sum_partials_warp(ws.partials, gridDim.x, S1, S2);
    const bool tot_ok = range_totals_ok(ws, h);
    if (tid == 0) {
      double res = 0.0;
      if (h.ok && !tot_ok) {
        set_status(ws.status, HOSZP_ERR_FORMAT);
      } else if (h.ok && h.n == 0) {
        set_status(ws.status, HOSZP_ERR_ARG);
      } else if (h.ok) {
        res = moment_finish(S1, S2, h.n, h.eps_q, true);
        if (take_sqrt) res = sqrt(res);  // standard deviation (Sec. V-B), correctly rounded
      }
      if (result) *result = res;
      if (sums) {  // the exact sums themselves (for combining shards)
        sums[0] = (unsigned long long)S1;
        sums[1] = (unsigned long long)((unsigned __int128)S1 >> 64);
        sums[2] = S2.lo;
        sums[3] = S2.hi;
        sums[4] = h.ok ? h.n : 0ull;
      }
      launch_reset(ws);
    }
  }
}

// ---------------------------------------------------------------- decompression
// Full decompression (inverse of every pipeline step, Fig. 2) over the
// super-tile pipeline: warp i of a group decodes tile i of the stage 16
// blocks at a time, two lanes per block (hz_lanes.cuh), to q, dequantizes
// x' = float(q) * 2 eps_q and stores each half's 32 floats (a warp writes
// 4 KB contiguous per step). MODE 1 writes the block-wise means instead
// (Sec. V-B): out is a double per block and n_expect the block count. MODE 2
// writes the quantized integers q themselves (int32, one per value), the
// other operand of the Hadamard product.
template <int MODE>
__global__ void __launch_bounds__(MEAN_THREADS, MEAN_MIN_CTAS) k_decompress(
    const uint8_t* __restrict__ c, uint64_t c_bytes, void* __restrict__ out, uint64_t n_expect,
    Ws ws) {
  extern __shared__ __align__(16) uint8_t dyn[];
  SStage* stages = reinterpret_cast<SStage*>(dyn);
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + MEAN_STAGES);
  __shared__ uint64_t full[MEAN_STAGES], empty[MEAN_STAGES];
  __shared__ unsigned long long stage_st[MEAN_STAGES];
  __shared__ uint32_t s_ts[TS_MAX];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const Info h = parse_header(c, c_bytes);
  const unsigned long long epoch = launch_epoch(ws);
  int bad = 0;
  bool ok = h.ok;
  if (!h.ok) bad = HOSZP_ERR_FORMAT;
  else if ((MODE == 1 ? h.nb : h.n) != n_expect) {
    bad = HOSZP_ERR_MISMATCH;
    ok = false;
  }
  const uint64_t ntiles = ok ? ntiles_of(h.nb) : 0;
  const uint64_t nst = nsuper_of(ntiles);
  if (tid == 0) {
    for (int k = 0; k < MEAN_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], MEAN_GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const SRange rg = range_sums(c, h, ntiles, nst, s_ts, ws, epoch, bad);
  __syncthreads();
  if (w == MEAN_NCW) {
    __shared__ uint32_t s_beg[MEAN_STAGES];
    super_loader<MEAN_STAGES, MEAN_RING, MEAN_GROUPS>(stages, ring, s_beg, full, empty, stage_st,
                                                       c, h, rg, s_ts, ws, epoch);
  } else if (w < MEAN_NCW) {
    const int grp = w / MEAN_GW, ti = w % MEAN_GW;
    const int lastlen = (int)(h.n - (h.nb - 1) * L);
    if (MODE == 1) {
      const lanes::Shifts K = lanes::make_shifts(c_bytes != 0 ? 1u : 0u);
      const double e2d = 2.0 * (double)h.eps_q;
      for (uint64_t k = 0;; k++) {
        const uint64_t u = k * MEAN_GROUPS + grp;  // stage use taken by this group
        const int sk = (int)(u % MEAN_STAGES);
        if (!mbar_wait_warp(&full[sk], (uint32_t)((u / MEAN_STAGES) & 1), ws.status)) break;
        const unsigned long long s = stage_st[sk];
        if (s == ~0ull) break;
        const SStage& sg = stages[sk];
        const uint64_t tile = (uint64_t)STILES * s + ti;
        const TileRates tr = tile_rates(sg, ti, tile, h.nb);
        block_means_tile(sg, ring, ti, tr, tile, ntiles, lastlen, e2d, K, static_cast<double*>(out));
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sk]);
      }
    } else {
      float* __restrict__ x = static_cast<float*>(out);
      const int j = lane & 7, gq = lane >> 3;
      const OctetSel S = octet_sel(j);
      const float e2 = 2.0f * h.eps_q;
      const bool small = h.qbound < (1u << 22);
      for (uint64_t k = 0;; k++) {
        const uint64_t u = k * MEAN_GROUPS + grp;  // stage use taken by this group
        const int sk = (int)(u % MEAN_STAGES);
        if (!mbar_wait_warp(&full[sk], (uint32_t)((u / MEAN_STAGES) & 1), ws.status)) break;
        const unsigned long long s = stage_st[sk];
        if (s == ~0ull) break;
        const SStage& sg = stages[sk];
        const uint64_t tile = (uint64_t)STILES * s + ti;
        const TileRates tr = tile_rates(sg, ti, tile, h.nb);
        const uint64_t* sgn = sg.sign + sg.sbase + sg.tnc[ti];
        const uint64_t* pls = ring + sg.pring + sg.pbase + sg.tr[ti];
        const int steps = (tr.nvt + 3) >> 2;  // warp-uniform
        for (int it = 0; it < steps; it++) {
          const int b = 4 * it + gq;
          uint32_t r, ex;
          tile_block(tr, b, r, ex);
          BlockRef br;
          br.rate = (int)r;
          br.outlier = sg.outlier[TILE * ti + b];
          br.len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
          br.planes = pls + (ex & 0xffffu);
          br.sign_byte = r ? reinterpret_cast<const uint8_t*>(sgn + (ex >> 16))[j] : 0u;
          const int kmax = (int)__reduce_max_sync(0xffffffffu, (r + 7) >> 3);
          int d[8], q[8];
          octet_deltas(br, kmax, j, S, d);
          octet_values(br, d, j, q);
          const uint64_t i0 = (tile * TILE + b) * L + 8 * j;
          if (MODE == 2) {  // the integers themselves
            int* qo = static_cast<int*>(out);
            if (br.len == L) {
              int4* o = reinterpret_cast<int4*>(qo + i0);
              __stcs(o, make_int4(q[0], q[1], q[2], q[3]));
              __stcs(o + 1, make_int4(q[4], q[5], q[6], q[7]));
            } else {
#pragma unroll
              for (int t = 0; t < 8; t++)
                if (8 * j + t < br.len) qo[i0 + t] = q[t];
            }
            continue;
          }
          float v[8];
          if (small) {  // uniform over the stream: no per-value select
#pragma unroll
            for (int t = 0; t < 8; t++) v[t] = dequant_small(q[t], e2);
          } else {
#pragma unroll
            for (int t = 0; t < 8; t++) v[t] = dequant_any(q[t], e2);
          }
          if (br.len == L) {
            float4* o = reinterpret_cast<float4*>(x + i0);
            __stcs(o, make_float4(v[0], v[1], v[2], v[3]));
            __stcs(o + 1, make_float4(v[4], v[5], v[6], v[7]));
          } else {
#pragma unroll
            for (int t = 0; t < 8; t++)
              if (8 * j + t < br.len) x[i0 + t] = v[t];
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sk]);
      }
    }
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && w == 0) {
    const bool tot_ok = range_totals_ok(ws, h);
    if (tid == 0) {
      if (ok && !tot_ok) set_status(ws.status, HOSZP_ERR_FORMAT);
      launch_reset(ws);
    }
  }
}

// ---------------------------------------------------------------- decompression, two lanes
// Full decompression (Fig. 2) with two lanes per block: lane 2m + h decodes
// half h of block m of its warp's 16-block step in registers (two's-complement
// planes, transposes and the local prefix of hz_lanes.cuh), adds the half's
// base (O, or O plus the first half's delta total) and dequantizes its 32
// values. Those 32 floats are one 128-byte row of the step's 1024 contiguous
// output floats: the warp writes its rows to a shared-memory box (the 128-byte
// swizzle: chunk j of row r at chunk j ^ (r % 8), conflict-free for the lanes)
// and one 2-D tensor copy stores the 4 KB box, so the global writes leave the
// SM as whole lines. A step that is not whole (the field's last) is stored
// value by value. The input comes through the super-tile pipeline with the
// in-kernel rate prefix, as for the reductions; a smaller tile-sum table
// leaves room for the 16 output boxes.
constexpr int DL_TS = 1024;  // tile sums kept per CTA (a longer range re-sums its rate bytes)
constexpr int DL_STAGES = MEAN_STAGES;
constexpr size_t DL_BOX_BYTES = ROW_STEP_FLOATS * 4;
constexpr size_t DL_OUT_BYTES = (size_t)MEAN_NCW * DL_BOX_BYTES;
constexpr size_t DL_STATIC = 6144;  // upper bound of the kernel's static shared memory
constexpr uint32_t DL_RING = (uint32_t)(((232448 - DL_STATIC - 1024 - DL_OUT_BYTES -
                                          DL_STAGES * sizeof(SStage)) / 8) & ~(size_t)1);
static_assert(DL_RING >= STILE_PLANE_WORDS_MAX + 2, "the ring holds the largest super-tile");
constexpr size_t DL_SMEM = 1024 + DL_OUT_BYTES + DL_STAGES * sizeof(SStage) + DL_RING * 8;

__device__ __forceinline__ void tma_store_rows(const CUtensorMap* map, int row, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   map),
               "r"(0), "r"(row), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the issuing thread's earlier box stores have finished reading shared memory
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// the issuing thread's earlier box stores are complete
__device__ __forceinline__ void tma_store_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__global__ void __launch_bounds__(MEAN_THREADS, MEAN_MIN_CTAS) k_decompress_lanes(
    const __grid_constant__ CUtensorMap rows, int use_rows, const uint8_t* __restrict__ c,
    uint64_t c_bytes, float* __restrict__ x, uint64_t n_expect, Ws ws) {
  extern __shared__ uint8_t dl_dyn[];
  uint8_t* const base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(dl_dyn) + 1023) & ~(uintptr_t)1023);
  SStage* stages = reinterpret_cast<SStage*>(base + DL_OUT_BYTES);
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + DL_STAGES);
  __shared__ uint64_t full[DL_STAGES], empty[DL_STAGES];
  __shared__ unsigned long long stage_st[DL_STAGES];
  __shared__ uint32_t s_ts[DL_TS];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const Info h = parse_header(c, c_bytes);
  const unsigned long long epoch = launch_epoch(ws);
  int bad = 0;
  bool ok = h.ok;
  if (!h.ok) bad = HOSZP_ERR_FORMAT;
  else if (h.n != n_expect) {
    bad = HOSZP_ERR_MISMATCH;
    ok = false;
  }
  const uint64_t ntiles = ok ? ntiles_of(h.nb) : 0;
  const uint64_t nst = nsuper_of(ntiles);
  if (tid == 0) {
    for (int k = 0; k < DL_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], MEAN_GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint8_t* const cs = c;
  const SRange rg = range_sums_n<STILES, 1>(&cs, &h, ntiles, nst, s_ts, DL_TS, ws, epoch, bad);
  __syncthreads();
  if (w == MEAN_NCW) {
    __shared__ uint32_t s_beg[DL_STAGES];
    super_loader_n<STILES, 1, DL_STAGES, DL_RING, MEAN_GROUPS>(stages, ring, s_beg, full, empty,
                                                              stage_st, &cs, &h, rg, s_ts, DL_TS,
                                                              ws, epoch);
  } else if (w < MEAN_NCW) {
    const int grp = w / MEAN_GW, ti = w % MEAN_GW;
    const int hf = lane & 1, m = lane >> 1;
    const int lastlen = (int)(h.n - (h.nb - 1) * L);
    const lanes::Shifts K = lanes::make_shifts(c_bytes != 0 ? 1u : 0u);
    const float e2 = 2.0f * h.eps_q;
    const bool small = h.qbound < (1u << 22);
    float4* const box = reinterpret_cast<float4*>(base + (size_t)w * DL_BOX_BYTES);
    bool stored = false;  // lane 0 has a box store outstanding
    for (uint64_t k = 0;; k++) {
      const uint64_t u = k * MEAN_GROUPS + grp;  // stage use taken by this group
      const int sk = (int)(u % DL_STAGES);
      if (!mbar_wait_warp(&full[sk], (uint32_t)((u / DL_STAGES) & 1), ws.status)) break;
      const unsigned long long s = stage_st[sk];
      if (s == ~0ull) break;
      const SStage& sg = stages[sk];
      const uint64_t tile = (uint64_t)STILES * s + ti;
      const TileRates tr = tile_rates(sg, ti, tile, h.nb);
      const uint32_t* sgn = reinterpret_cast<const uint32_t*>(sg.sign + sg.sbase + sg.tnc[ti]);
      const uint32_t* pls =
          reinterpret_cast<const uint32_t*>(ring + sg.pring + sg.pbase + sg.tr[ti]);
      const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
      for (int it = 0; it < steps; it++) {
        const int b = 16 * it + m;
        uint32_t r, ex;
        tile_block(tr, b, r, ex);
        const int len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
        const int nval = min(max(len - 32 * hf, 0), 32);
        const int O = len ? sg.outlier[TILE * ti + b] : 0;
        const uint32_t sw = r ? sgn[2 * (ex >> 16) + hf] : 0u;
        const int Rw = (int)__reduce_max_sync(0xffffffffu, r);
        int v[32];
        {
          uint32_t t[32];
          lanes::twos_planes_any(Rw, pls + 2 * (ex & 0xffffu) + hf, (int)r, sw, t);
          half_prefix_any(Rw, t, hf == 0, K, v);
        }
        // the second half's base: O plus the first half's delta total (every
        // lane takes part in the exchange, then selects)
        const int tot0 = __shfl_xor_sync(0xffffffffu, v[31], 1);
        const int qb = O + (hf ? tot0 : 0);
        // dequantized in place: v[i] holds the float's bits from here on
        if (small) {  // uniform over the stream: no per-value select
#pragma unroll
          for (int i = 0; i < 32; i++) v[i] = __float_as_int(dequant_small(v[i] + qb, e2));
        } else {
#pragma unroll
          for (int i = 0; i < 32; i++) v[i] = __float_as_int(dequant_any(v[i] + qb, e2));
        }
        const uint64_t s0 = (tile * TILE + 16 * (uint64_t)it) * L;  // the step's first value
        if (use_rows && s0 + ROW_STEP_FLOATS <= h.n) {
          if (lane == 0 && stored) tma_store_wait_read();  // the box is free again
          __syncwarp();
          int4* const b4 = reinterpret_cast<int4*>(box);
#pragma unroll
          for (int j = 0; j < 8; j++)
            b4[8 * lane + (j ^ (lane & 7))] = make_int4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          fence_proxy_async();  // this lane's box writes before the tensor copy reads them
          __syncwarp();
          if (lane == 0) tma_store_rows(&rows, (int)(s0 / 32), box);
          stored = true;
        } else {
          const uint64_t i0 = (tile * TILE + b) * L + 32 * hf;
#pragma unroll
          for (int i = 0; i < 32; i++)
            if (i < nval) x[i0 + i] = __int_as_float(v[i]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sk]);
    }
    if (lane == 0 && stored) tma_store_wait_all();
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && w == 0) {
    const bool tot_ok = range_totals_ok(ws, h);
    if (tid == 0) {
      if (ok && !tot_ok) set_status(ws.status, HOSZP_ERR_FORMAT);
      launch_reset(ws);
    }
  }
}

cudaError_t launch_decompress(const Launch& lc, const uint8_t* c, uint64_t c_bytes, float* x,
                              uint64_t n, Ws ws) {
  // the kernel finds the rate prefix itself (range_sums): no pre-scan
  CUtensorMap rows;
  const int use_rows = encode_rows(x, n, &rows) ? 1 : 0;
  smem_attr<k_decompress_lanes>(DL_SMEM);
  const int grid = persistent_grid(k_decompress_lanes, MEAN_THREADS, lc.grid, DL_SMEM);
  k_decompress_lanes<<<grid, MEAN_THREADS, DL_SMEM, lc.stream>>>(rows, use_rows, c, c_bytes, x, n,
                                                                 ws);
  return cudaGetLastError();
}

cudaError_t launch_decode_q(const Launch& lc, const uint8_t* c, uint64_t c_bytes, int* q,
                           uint64_t n, Ws ws) {
  const size_t smem = MEAN_STAGES * sizeof(SStage) + MEAN_RING * sizeof(uint64_t);
  smem_attr<k_decompress<2>>(smem);
  const int grid = persistent_grid(k_decompress<2>, MEAN_THREADS, lc.grid, smem);
  k_decompress<2><<<grid, MEAN_THREADS, smem, lc.stream>>>(c, c_bytes, q, n, ws);
  return cudaGetLastError();
}

cudaError_t launch_block_means(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double* out,
                               uint64_t nb, Ws ws) {
  const size_t smem = MEAN_STAGES * sizeof(SStage) + MEAN_RING * sizeof(uint64_t);
  smem_attr<k_decompress<1>>(smem);
  const int grid = persistent_grid(k_decompress<1>, MEAN_THREADS, lc.grid, smem);
  k_decompress<1><<<grid, MEAN_THREADS, smem, lc.stream>>>(c, c_bytes, out, nb, ws);
  return cudaGetLastError();
}

cudaError_t launch_moments(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double* result,
                           bool variance, Ws ws, unsigned long long* sums, bool take_sqrt) {
  // both kernels find the rate prefix themselves (range_sums): no pre-scan
  const size_t smem = MEAN_STAGES * sizeof(SStage) + MEAN_RING * sizeof(uint64_t);
  smem_attr<k_mean>(smem);
  smem_attr<k_var>(smem);
  const int grid = (variance || sums) ? persistent_grid(k_var, MEAN_THREADS, lc.grid, smem)
                                      : persistent_grid(k_mean, MEAN_THREADS, lc.grid, smem);
  if (variance || sums)
    k_var<<<grid, MEAN_THREADS, smem, lc.stream>>>(c, c_bytes, variance ? result : nullptr, sums,
                                                   take_sqrt ? 1 : 0, ws);
  else
    k_mean<<<grid, MEAN_THREADS, smem, lc.stream>>>(c, c_bytes, result, ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- finish of combined sums
// Mean and variance of a field from exact sums added over its shards (five
// words as hoszp_sums writes them: S1 low/high, S2 low/high, n), with the same
// FP64 steps as the single-stream kernels, so a sharded field gives the same
// doubles as the whole field on one device.
__global__ void k_finish_sums(const unsigned long long* sums, float eps_q, double* mean,
                              double* var, Ws ws) {
  const __int128 S1 = (__int128)(((unsigned __int128)sums[1] << 64) | sums[0]);
  const U128 S2 = {sums[2], sums[3]};
  const uint64_t n = sums[4];
  if (n == 0 || !(eps_q >= FLT_MIN) || !(eps_q <= FLT_MAX)) {
    set_status(ws.status, HOSZP_ERR_ARG);
    if (mean) *mean = 0.0;
    if (var) *var = 0.0;
    return;
  }
  if (mean) *mean = moment_finish(S1, S2, n, eps_q, false);
  if (var) *var = moment_finish(S1, S2, n, eps_q, true);
}

cudaError_t launch_finish_sums(const Launch& lc, const unsigned long long* sums, float eps_q,
                               double* mean, double* var, Ws ws) {
  k_finish_sums<<<1, 1, 0, lc.stream>>>(sums, eps_q, mean, var, ws);
  return cudaGetLastError();
}

}  // namespace hz
