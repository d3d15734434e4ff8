// compress.cu — relative-bound range pass and the compression kernel
// (Sec. IV-A: Eq. 3 quantization, Eq. 4 in-block Lorenzo, sign separation,
// blockwise fixed-length bit-plane encoding, stream layout of Fig. 3).
#include <cfloat>

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
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 v = __ldg(x4 + i);
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
// Pipeline per CTA: the next tiles' 16 KB of input are bulk-copied into a
// shared-memory ring while the current tile is quantized and encoded into an
// output stage; a tile's place in the stream (look-back over the tiles before
// it) is resolved one tile later, so the look-back latency overlaps compute.
constexpr int CMP_STAGES = 4;
constexpr int CMP_THREADS = (NCW + 1) * 32;  // compute warps + one issuer warp

struct InX {
  float v[TILE_VALUES];
};

__device__ __forceinline__ void issue_x(InX* s, uint64_t* bar, const float* x, uint64_t n,
                                        uint64_t t) {
  const uint64_t first = (uint64_t)TILE_VALUES * t;
  const uint64_t cnt = umin64(TILE_VALUES, n - first);
  const unsigned bytes = (unsigned)((cnt * 4) & ~15ull);
  fence_proxy_async();
  mbar_expect_tx(bar, bytes);
  if (bytes) bulk_g2s(s->v, x + first, bytes, bar);
}

__global__ void __launch_bounds__(CMP_THREADS, 2) k_compress(
    const float* __restrict__ x, uint64_t n, const uint32_t dims0, const uint32_t dims1,
    const uint32_t dims2, const uint32_t ndims, float eps_q_abs, double eps_abs, int rel,
    uint8_t* __restrict__ out, uint64_t cap, Ws ws) {
  extern __shared__ __align__(16) uint8_t dyn[];
  InX* ins = reinterpret_cast<InX*>(dyn);
  __shared__ uint64_t full[CMP_STAGES], empty[CMP_STAGES];
  __shared__ unsigned long long stage_tile[CMP_STAGES];
  __shared__ uint8_t srate[2][TILE];
  __shared__ unsigned int s_qmax[CMP_THREADS / 32];
  const int tid = threadIdx.x, w = tid >> 5, g = tid >> 3, j = tid & 7;

  const float e = rel ? *ws.eps_q : eps_q_abs;
  const uint64_t nb = nblocks(n);
  const uint64_t ntiles = (e >= FLT_MIN) ? ntiles_of(nb) : 0;  // range pass failed: no work
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
  ring_init<CMP_STAGES>(full, empty);
  const OctetSel S = octet_sel(j);
  uint32_t qmax = 0;
  int bad = 0;
  if (w == LOADER_WARP) {
    const uint64_t G = gridDim.x;
    issuer_warp<CMP_STAGES>(
        stage_tile, full, empty, ntiles, ws.status,
        [&](uint32_t k) { return (unsigned long long)(blockIdx.x + (uint64_t)k * G); },
        [&](int sk, unsigned long long t) {
          if ((tid & 31) == 0) issue_x(&ins[sk], &full[sk], x, n, t);
        });
  } else {
    RingPos rp{0, 0u};
    for (uint64_t k = 0;; k++) {
      const int s = rp.s;
      mbar_wait(&full[s], rp.par, ws.status);
      const unsigned long long tile = stage_tile[s];
      if (tile >= ntiles) break;
      const InX& in = ins[s];
      const uint64_t b = tile * TILE + g;
      const uint64_t first = (uint64_t)TILE_VALUES * tile;
      const uint64_t copied = umin64(TILE_VALUES, n - first) & ~3ull;
      const int o0 = 64 * g + 8 * j;  // offset in the tile
      const uint64_t i0 = first + o0;
      float v[8];
      if ((uint64_t)o0 + 8 <= copied) {
        const float4 a = *reinterpret_cast<const float4*>(&in.v[o0]);
        const float4 c = *reinterpret_cast<const float4*>(&in.v[o0 + 4]);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
      } else {
#pragma unroll
        for (int t = 0; t < 8; t++) {
          const uint64_t o = (uint64_t)o0 + t;
          v[t] = (o < copied) ? in.v[o] : ((i0 + t < n) ? __ldg(x + i0 + t) : 0.0f);
        }
      }
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[s]);
      rp.next<CMP_STAGES>();
      int q[8];
      quantize8(v, Q, q, bad);
      const bool past_end = i0 + 8 > n;  // only in the stream's last block
      if (past_end) {
#pragma unroll
        for (int t = 0; t < 8; t++)
          if (i0 + t >= n) q[t] = 0;
      }
#pragma unroll
      for (int t = 0; t < 8; t++) qmax = max(qmax, (uint32_t)abs(q[t]));
      // Eq. 4 inside the block: delta_i = q_i - q_{i-1}, delta_0 := 0 (outlier)
      const int prev = __shfl_up_sync(0xffffffffu, q[7], 1, 8);
      int d[8];
#pragma unroll
      for (int t = 0; t < 8; t++) d[t] = (t == 0) ? ((j == 0) ? 0 : q[0] - prev) : q[t] - q[t - 1];
      if (past_end) {
#pragma unroll
        for (int t = 0; t < 8; t++)
          if (i0 + t >= n) d[t] = 0;
      }
      uint32_t mag[8];
      uint32_t sb = 0;
#pragma unroll
      for (int t = 0; t < 8; t++) {
        mag[t] = (uint32_t)abs(d[t]);
        sb |= (d[t] < 0 ? 1u : 0u) << t;
      }
      const int rate = octet_rate(mag);
      produce_tile(srate, k, tile, nb, mag, sb, rate, q[0], b < nb, g, j, out, ws.staging,
                   slot_offset(SLOT_COMPRESS, tile, nullptr, nullptr, 0), ws.staging_words,
                   ws.agg, S, bad);
    }
  }
  // epilogue: max |q| for the header's qbound, first error, launch bookkeeping
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  if ((tid & 31) == 0) s_qmax[tid >> 5] = qmax;
  __syncthreads();
  if (tid == 0) {
    for (int k = 1; k < CMP_THREADS / 32; k++) qmax = max(qmax, s_qmax[k]);
    atomicMax(&ws.totals[2], (unsigned long long)qmax);
  }
  if (bad) set_status(ws.status, bad);
}

cudaError_t launch_compress(const Launch& lc, const float* x, uint64_t n, const uint32_t dims[3],
                            uint32_t ndims, float eps_q_abs, double eps_abs, bool rel, uint8_t* out,
                            uint64_t cap, Ws ws) {
  const size_t smem = CMP_STAGES * sizeof(InX);
  smem_attr<k_compress>(smem);
  k_compress<<<persistent_grid(k_compress, CMP_THREADS, lc.grid, smem), CMP_THREADS, smem,
               lc.stream>>>(x, n, dims[0], dims[1], dims[2], ndims, eps_q_abs, eps_abs,
                                  rel ? 1 : 0, out, cap, ws);
  return cudaGetLastError();
}

}  // namespace hz
