// compress.cu — relative-bound range pass and the compression kernel
// (Sec. IV-A: Eq. 3 quantization, Eq. 4 in-block Lorenzo, sign separation,
// blockwise fixed-length bit-plane encoding, stream layout of Fig. 3).
#include <cfloat>
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "hz_produce.cuh"
#include "hz_ws.cuh"
#include "hz_kernels.cuh"

namespace hz {

// ---------------------------------------------------------------- range pass
// eps = rel * (max - min) over the field (NaN/Inf -> HOSZP_ERR_NONFINITE), then
// eps_q = largest float32 <= eps; written to the workspace for the compressor.
__global__ void __launch_bounds__(512) k_range(const float* __restrict__ x, uint64_t n, double rel,
                                                Ws ws) {
  float mn = FLT_MAX, mx = -FLT_MAX;
  int nonfinite = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n4 = n / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  // from the end of the field down, so that the compression pass, which starts
  // at the field's beginning, finds the last part read here still in L2
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n4; j += stride) {
    float4 v = __ldg(x4 + (n4 - 1 - j));
    float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int t = 0; t < 4; t++) {
      if (!(fabsf(a[t]) <= FLT_MAX)) nonfinite = 1;
      mn = fminf(mn, a[t]);
      mx = fmaxf(mx, a[t]);
    }
  }
  for (uint64_t i = n4 * 4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float a = __ldg(x + i);
    if (!(fabsf(a) <= FLT_MAX)) nonfinite = 1;
    mn = fminf(mn, a);
    mx = fmaxf(mx, a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
  }
  __shared__ float s_mn[16], s_mx[16];
  __shared__ int s_nf[16];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_mn[w] = mn;
    s_mx[w] = mx;
    s_nf[w] = nonfinite;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
      mn = fminf(mn, s_mn[k]);
      mx = fmaxf(mx, s_mx[k]);
      nonfinite |= s_nf[k];
    }
    ws.range_part[3 * blockIdx.x + 0] = mn;
    ws.range_part[3 * blockIdx.x + 1] = mx;
    ws.range_part[3 * blockIdx.x + 2] = (float)nonfinite;
  }
  if (launch_end_is_last(ws) && threadIdx.x < 32) {  // one warp reads all partials at once
    float gmn = FLT_MAX, gmx = -FLT_MAX;
    int nf = 0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += 32) {
      gmn = fminf(gmn, ws.range_part[3 * b + 0]);
      gmx = fmaxf(gmx, ws.range_part[3 * b + 1]);
      nf |= ws.range_part[3 * b + 2] != 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gmn = fminf(gmn, __shfl_xor_sync(0xffffffffu, gmn, o));
      gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, o));
      nf |= __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if (threadIdx.x != 0) return;
    float eq = 0.0f;
    double eps = 0.0;
    if (nf) {
      set_status(ws.status, HOSZP_ERR_NONFINITE);
    } else {
      double range = (n > 0) ? (double)gmx - (double)gmn : 0.0;
      if (range == 0.0) range = (n > 0 && gmx != 0.0f) ? fabs((double)gmx) : 1.0;
      eps = rel * range;
      float f = __double2float_rn(eps);
      if ((double)f > eps) f = nextafterf(f, 0.0f);
      if (!(f >= FLT_MIN && f <= FLT_MAX / 2)) {
        set_status(ws.status, HOSZP_ERR_RANGE);
        f = 0.0f;
      }
      eq = f;
    }
    *ws.eps_q = eq;
    *ws.eps = eps;
    launch_reset(ws);
  }
}

cudaError_t launch_range(const Launch& lc, const float* x, uint64_t n, double rel, Ws ws) {
  k_range<<<persistent_grid(k_range, 512, lc.grid), 512, 0, lc.stream>>>(x, n, rel, ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- compression
// Two lanes per block (hz_lanes.cuh, hz_produce.cuh): lane 2m + h of a warp
// holds positions 32h .. 32h + 31 of block m of the warp's 16-block step, all
// in registers, from the float loads to the stored bit-planes:
//   32 floats -> q (Eq. 3, exact) -> delta (Eq. 4; the second half's first
//   delta takes the first half's last q) -> two's-complement planes ->
//   sign word half and magnitude planes (Fig. 3).
// A warp takes whole 64-block tiles from a launch-wide ticket and walks each in
// four steps, keeping the tile's running count of sign and plane words, so it
// writes every block's words at once: signs to the tile's sign slot (64 words
// per tile), planes to its plane slot (64 x 24 words per tile: |q| <= 2^23 - 2
// keeps every rate at or below 24). Rates and outliers go straight to the
// stream; the placement kernel (which scans the tiles' word counts) finishes it.
//
// Input: a step's 1024 floats are contiguous, one 128-byte row per lane. Each
// warp streams its steps through CMP_NBUF shared-memory buffers with 2-D
// tensor copies (the field viewed as rows of 32 floats, a 32 x 32 box per
// step), issued CMP_NBUF - 1 steps ahead across its current and next tile,
// so the loads of a step land while the warp computes the steps before it.
// The copies use the 128-byte swizzle: chunk j of row r lands at chunk
// j ^ (r % 8), so the eight 16-byte reads of a row by its lane hit eight
// different bank groups within each quarter warp. Steps that are not whole
// (the field's last, and any field too short or too long for the tensor view)
// are read directly from global memory.
constexpr int CMP_WARPS = 16;
constexpr int CMP_THREADS = CMP_WARPS * 32;
constexpr uint32_t CMP_PLANE_SLOT = TILE * 24;  // plane words per tile slot
constexpr int CMP_NBUF = 3;                     // per-warp step buffers
constexpr uint32_t CMP_STEP_FLOATS = ROW_STEP_FLOATS;  // one warp step: 16 blocks
constexpr size_t CMP_SMEM = (size_t)CMP_WARPS * CMP_NBUF * CMP_STEP_FLOATS * 4 + 1024;

__device__ __forceinline__ void tma_load_rows(void* dst, const CUtensorMap* map, int row,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(0), "r"(row), "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(CMP_THREADS, 1) k_compress(
    const __grid_constant__ CUtensorMap rows, int use_rows, const float* __restrict__ x,
    uint64_t n, const uint32_t dims0, const uint32_t dims1, const uint32_t dims2,
    const uint32_t ndims, float eps_q_abs, double eps_abs, int rel, uint8_t* __restrict__ out,
    uint64_t cap, Ws ws) {
  extern __shared__ uint8_t cmp_dyn[];
  __shared__ unsigned int s_qmax[CMP_WARPS];
  __shared__ uint64_t s_bar[CMP_WARPS][CMP_NBUF];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int hf = lane & 1, m = lane >> 1;
  const float e = rel ? *ws.eps_q : eps_q_abs;
  const uint64_t nb = nblocks(n);
  uint64_t ntiles = (e >= FLT_MIN) ? ntiles_of(nb) : 0;  // range pass failed: no work
  int bad = 0;
  // slots: 64 sign words per tile, then 64 x 24 plane words per tile
  if (ntiles + 1 > ws.max_tiles ||
      (uint64_t)(TILE + CMP_PLANE_SLOT) * ntiles > ws.staging_words) {
    bad = HOSZP_ERR_CAPACITY;
    ntiles = 0;
  }
  Quant Q;
  Q.e = e;
  Q.e2 = 2.0f * e;
  Q.r = (e >= FLT_MIN) ? __double2float_rn(1.0 / (double)Q.e2) : 0.0f;
  if (tid == 0 && blockIdx.x == 0) {  // header template for the placement kernel
    hoszp_header* H = ws.hdr;
    H->magic = HOSZP_MAGIC;
    H->version = HOSZP_VERSION;
    H->dtype = 0;
    H->ndims = (uint8_t)ndims;
    H->dims[0] = dims0;
    H->dims[1] = dims1;
    H->dims[2] = dims2;
    H->eps_q = e;
    H->n = n;
    H->eps = rel ? *ws.eps : eps_abs;
    H->nnc = 0;
    H->R = 0;
    H->qbound = 0;
    H->block = HOSZP_BLOCK;
  }
  // this warp's step buffers (1024-byte aligned for the swizzle pattern)
  float* const wbuf = reinterpret_cast<float*>(
      ((reinterpret_cast<uintptr_t>(cmp_dyn) + 1023) & ~(uintptr_t)1023) +
      (size_t)w * CMP_NBUF * CMP_STEP_FLOATS * 4);
  uint64_t* const bar = s_bar[w];
  if (lane == 0) {
    for (int k = 0; k < CMP_NBUF; k++) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const lanes::Shifts K = lanes::make_shifts(n != 0 ? 1u : 0u);
  int qhi = 0, qlo = 0;  // extremes of q (zeros included: max |q| is unchanged)
  uint64_t* const pslots = ws.staging + (uint64_t)TILE * ntiles;
  auto fetch_tile = [&]() -> uint64_t {
    unsigned int t32 = 0;
    if (lane == 0) t32 = atomicAdd(&ws.sync->ticket, 1u);
    return __shfl_sync(0xffffffffu, t32, 0);
  };
  auto nsteps = [&](uint64_t t) -> int {
    return t < ntiles ? (int)((umin64(TILE, nb - t * TILE) + 15) >> 4) : 0;
  };
  // a step goes through the tensor copies when all its 1024 values exist
  auto whole = [&](uint64_t t, int it) -> bool {
    return use_rows && t < ntiles && (t * TILE + 16 * (uint64_t)it) * L + CMP_STEP_FLOATS <= n;
  };
  uint32_t phase = 0;    // bit k: parity of the next completion of bar[k]
  uint32_t pending = 0;  // bit k: a copy into buffer k is in flight
  bool dead = false;     // a wait gave up: issue nothing more
  auto issue = [&](uint64_t t, int it, uint32_t u) {
    if (dead || !whole(t, it)) return;
    const int k = (int)(u % CMP_NBUF);
    if (lane == 0) {
      fence_proxy_async();  // the warp's reads of the buffer come before the copy's writes
      mbar_expect_tx(&bar[k], CMP_STEP_FLOATS * 4);
      tma_load_rows(wbuf + (size_t)k * CMP_STEP_FLOATS, &rows,
                    (int)((t * TILE + 16 * (uint64_t)it) * (L / 32)), &bar[k]);
    }
    pending |= 1u << k;
  };
  // a unit is step `it` of the current tile (it < steps) or of the next one
  auto issue_rel = [&](uint64_t t, uint64_t tn, int steps, int j, uint32_t u) {
    if (j < steps) issue(t, j, u);
    else if (j - steps < nsteps(tn)) issue(tn, j - steps, u);
  };
  uint64_t tile = fetch_tile();
  uint64_t nxt = tile < ntiles ? fetch_tile() : ntiles;
  uint32_t u0 = 0;  // unit number of the tile's first step
  for (int j = 0; j < CMP_NBUF - 1; j++) issue_rel(tile, nxt, nsteps(tile), j, (uint32_t)j);
  while (tile < ntiles && !dead) {
    const int nvt = (int)umin64(TILE, nb - tile * TILE);
    const uint64_t so = (uint64_t)TILE * tile, po = (uint64_t)CMP_PLANE_SLOT * tile;
    uint32_t* sdst = reinterpret_cast<uint32_t*>(ws.staging + so);
    uint32_t* pdst = reinterpret_cast<uint32_t*>(pslots + po);
    uint32_t run = 0;  // (sign words << 16 | plane words) of the tile so far
    int tbad = 0;
    const int steps = (nvt + 15) >> 4;
    for (int it = 0; it < steps; it++) {
      const uint32_t u = u0 + (uint32_t)it;
      const int kb = (int)(u % CMP_NBUF);
      const int b = 16 * it + m;
      const bool valid = b < nvt;
      const uint64_t bi = tile * TILE + b;
      const uint64_t i0 = bi * L + 32 * hf;  // the half's first value
      const int nval = (valid && i0 < n) ? (int)umin64(32, n - i0) : 0;
      const bool fullblk = __all_sync(0xffffffffu, nval == 32);
      int q[32];
      {
        float f[32];
        if ((pending >> kb) & 1u) {  // the step's rows, landed in buffer kb
          if (!mbar_wait_warp(&bar[kb], (phase >> kb) & 1u, ws.status)) {
            dead = true;
            break;
          }
          phase ^= 1u << kb;
          pending &= ~(1u << kb);
          const float4* r4 = reinterpret_cast<const float4*>(wbuf + (size_t)kb * CMP_STEP_FLOATS) +
                             8 * lane;
#pragma unroll
          for (int k = 0; k < 8; k++) {
            const float4 a = r4[k ^ (lane & 7)];
            f[4 * k] = a.x;
            f[4 * k + 1] = a.y;
            f[4 * k + 2] = a.z;
            f[4 * k + 3] = a.w;
          }
        } else if (fullblk) {
          const float4* x4 = reinterpret_cast<const float4*>(x + i0);
#pragma unroll
          for (int k = 0; k < 8; k++) {
            const float4 a = __ldcs(x4 + k);  // read once: streaming
            f[4 * k] = a.x;
            f[4 * k + 1] = a.y;
            f[4 * k + 2] = a.z;
            f[4 * k + 3] = a.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; i++) f[i] = (i < nval) ? __ldg(x + i0 + i) : 0.0f;
        }
        __syncwarp();  // every lane has read buffer kb: the copy two steps ahead may reuse it
        issue_rel(tile, nxt, steps, it + CMP_NBUF - 1, u + CMP_NBUF - 1);
#pragma unroll
        for (int k = 0; k < 4; k++) quantize8(f + 8 * k, Q, q + 8 * k, bad);
      }
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        qhi = __vimax3_s32(qhi, q[i], q[i + 1]);
        qlo = __vimin3_s32(qlo, q[i], q[i + 1]);
      }
      // Eq. 4 inside the block: delta_i = q_i - q_(i-1), delta_0 := 0 (outlier)
      const int last0 = __shfl_xor_sync(0xffffffffu, q[31], 1);
      const int o_new = q[0];
#pragma unroll
      for (int i = 31; i > 0; i--) q[i] -= q[i - 1];
      q[0] = hf ? q[0] - last0 : 0;
      if (!fullblk) {
#pragma unroll
        for (int i = 0; i < 32; i++)
          if (i >= nval) q[i] = 0;
      }
      // plane groups for the warp's widest delta (its sign takes one more bit)
      int dhi = 0, dlo = 0;
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        dhi = __vimax3_s32(dhi, q[i], q[i + 1]);
        dlo = __vimin3_s32(dlo, q[i], q[i + 1]);
      }
      const uint32_t dm = __reduce_or_sync(0xffffffffu, (uint32_t)max(dhi, -dlo));
      const int Ge = min(4, (40 - __clz(dm)) >> 3);  // (bit length + 8) / 8
      // a quantizer error anywhere in the warp: its values are not stored
      int sbad = __any_sync(0xffffffffu, bad != 0) ? HOSZP_ERR_RANGE : tbad;
      const int rate = encode_store_any(Ge, q, K, valid, sdst, pdst, TILE, CMP_PLANE_SLOT, run,
                                        sbad);
      if (sbad == HOSZP_ERR_CAPACITY) tbad = sbad;
      if (valid && hf == 0) {
        out[HOSZP_HEADER_BYTES + bi] = (uint8_t)rate;
        reinterpret_cast<int*>(out + off_outlier(nb))[bi] = o_new;
      }
    }
    if (dead) break;
    if (tbad) bad = tbad;
    if (lane == 0) {
      ws.agg[tile] = ((unsigned long long)(run >> 16) << 32) | (run & 0xffffu);
      ws.pre[0][2 * tile] = so;
      ws.pre[0][2 * tile + 1] = (uint64_t)TILE * ntiles + po;
    }
    u0 += (uint32_t)steps;
    tile = nxt;
    nxt = tile < ntiles ? fetch_tile() : ntiles;
  }
  // after a wait gave up, the copies still in flight land before the CTA exits
  // (bounded waits; each pending buffer has exactly one copy outstanding)
  if (dead)
    for (int k = 0; k < CMP_NBUF; k++)
      if ((pending >> k) & 1u) mbar_wait(&bar[k], (phase >> k) & 1u, ws.status);
  // epilogue: max |q| for the header's qbound, first error, launch bookkeeping
  uint32_t qmax = max((uint32_t)qhi, (uint32_t)(-(long long)qlo));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  if (lane == 0) s_qmax[w] = qmax;
  __syncthreads();
  if (tid == 0) {
    for (int k = 1; k < CMP_WARPS; k++) qmax = max(qmax, s_qmax[k]);
    atomicMax(&ws.totals[2], (unsigned long long)qmax);
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

// The field as a 2-D tensor of rows of 32 floats (128 bytes), copied in boxes
// of 32 rows with the 128-byte swizzle. False when the tensor view does not
// apply (fewer than one step of values, more rows than a copy coordinate
// reaches, an unaligned base) or the driver cannot encode it; the kernels then
// read or write every step directly.
bool encode_rows(const float* x, uint64_t n, CUtensorMap* map) {
  std::memset(map, 0, sizeof(*map));
  const uint64_t nrows = n / 32;
  if (n < ROW_STEP_FLOATS || nrows > 0x7fffffffull || ((uintptr_t)x & 15u)) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dim[2] = {32, nrows};
  const cuuint64_t stride[1] = {128};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estride[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dim, stride, box,
                estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

cudaError_t launch_compress(const Launch& lc, const float* x, uint64_t n, const uint32_t dims[3],
                            uint32_t ndims, float eps_q_abs, double eps_abs, bool rel, uint8_t* out,
                            uint64_t cap, Ws ws) {
  CUtensorMap rows;
  const int use_rows = encode_rows(x, n, &rows) ? 1 : 0;
  smem_attr<k_compress>(CMP_SMEM);
  const int grid = persistent_grid(k_compress, CMP_THREADS, lc.grid, CMP_SMEM);
  k_compress<<<grid, CMP_THREADS, CMP_SMEM, lc.stream>>>(rows, use_rows, x, n, dims[0], dims[1],
                                                         dims[2], ndims, eps_q_abs, eps_abs,
                                                         rel ? 1 : 0, out, cap, ws);
  return cudaGetLastError();
}

}  // namespace hz
