// compress.cu — relative-bound range pass and the compression kernel
// (Sec. IV-A: Eq. 3 quantization, Eq. 4 in-block Lorenzo, sign separation,
// blockwise fixed-length bit-plane encoding, stream layout of Fig. 3).
#include <cfloat>

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
  if (launch_end_is_last(ws) && threadIdx.x == 0) {
    float gmn = FLT_MAX, gmx = -FLT_MAX;
    int nf = 0;
    for (unsigned int b = 0; b < gridDim.x; b++) {
      gmn = fminf(gmn, ws.range_part[3 * b + 0]);
      gmx = fmaxf(gmx, ws.range_part[3 * b + 1]);
      nf |= ws.range_part[3 * b + 2] != 0.0f;
    }
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
__global__ void __launch_bounds__(CTA) k_compress(const float* __restrict__ x, uint64_t n,
                                                  const uint32_t dims0, const uint32_t dims1,
                                                  const uint32_t dims2, const uint32_t ndims,
                                                  float eps_q_abs, double eps_abs, int rel,
                                                  uint8_t* __restrict__ out, uint64_t cap, Ws ws) {
  __shared__ uint8_t s_rate[TILE];
  __shared__ TileScan ts;
  __shared__ unsigned long long s_pre[2];
  __shared__ unsigned int s_tile;
  __shared__ unsigned long long s_epoch;
  __shared__ unsigned int s_qmax[CTA / 32];
  const int tid = threadIdx.x, g = tid >> 3, j = tid & 7;

  const float e = rel ? *ws.eps_q : eps_q_abs;
  const uint64_t nb = nblocks(n);
  const uint64_t ntiles = (e >= FLT_MIN) ? ntiles_of(nb) : 0;  // range pass failed: no work
  Quant Q;
  Q.e = e;
  Q.e2 = 2.0f * e;
  Q.r = (e >= FLT_MIN) ? __double2float_rn(1.0 / (double)Q.e2) : 0.0f;
  const uint64_t o_out = off_outlier(nb), o_sign = off_sign(nb);
  int* const outlier = reinterpret_cast<int*>(out + o_out);

  if (tid == 0) {
    s_epoch = launch_epoch(ws);
    if (blockIdx.x == 0) {  // header template for the placement kernel
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
  }
  __syncthreads();
  const unsigned long long epoch = s_epoch;
  uint32_t qmax = 0;
  int bad = 0;

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&ws.sync->ticket, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint64_t b = tile * TILE + g;
    const uint64_t i0 = b * L + 8 * j;
    float v[8];
    if (i0 + 8 <= n) {
      float4 a = __ldg(reinterpret_cast<const float4*>(x + i0));
      float4 c = __ldg(reinterpret_cast<const float4*>(x + i0 + 4));
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
    } else {
#pragma unroll
      for (int t = 0; t < 8; t++) v[t] = (i0 + t < n) ? __ldg(x + i0 + t) : 0.0f;
    }
    int q[8];
#pragma unroll
    for (int t = 0; t < 8; t++) {
      q[t] = quantize(v[t], Q, bad);
      if (i0 + t >= n) q[t] = 0;
      uint32_t a = (uint32_t)abs(q[t]);
      qmax = max(qmax, a);
    }
    // Eq. 4 inside the block: delta_i = q_i - q_{i-1}, delta_0 := 0 (outlier)
    const int prev = __shfl_up_sync(0xffffffffu, q[7], 1, 8);
    uint32_t mag[8];
    uint32_t sb = 0;
#pragma unroll
    for (int t = 0; t < 8; t++) {
      int d = (t == 0) ? ((j == 0) ? 0 : q[0] - prev) : q[t] - q[t - 1];
      if (i0 + t >= n) d = 0;
      mag[t] = (uint32_t)abs(d);
      sb |= (d < 0 ? 1u : 0u) << t;
    }
    const int rate = octet_rate(mag);
    if (j == 0) s_rate[g] = (b < nb) ? (uint8_t)rate : 0;
    __syncthreads();
    tile_scan(s_rate, &ts);
    tile_prefix(ws.desc[0], (int64_t)tile, epoch, ws.status, ts.agg_nc, ts.agg_r, 0, s_pre);
    __syncthreads();
    const uint64_t NC = s_pre[0], RR = s_pre[1];
    const int r = (b < nb) ? rate : 0;
    if (b < nb && j == 0) {
      out[HOSZP_HEADER_BYTES + b] = (uint8_t)rate;
      outlier[b] = q[0];
    }
    const uint64_t si = NC + ts.nc_excl[g];
    const uint64_t pi = RR + ts.r_excl[g];
    if (r > 0) {
      const uint64_t pos = o_sign + 8 * si + j;
      if (pos < cap) out[pos] = (uint8_t)sb;
      else bad = HOSZP_ERR_CAPACITY;
    }
    const int kmax = __reduce_max_sync(0xffffffffu, (r + 7) >> 3);
    const uint64_t lim = (pi < ws.staging_words) ? ws.staging_words - pi : 0;
    if (kmax > 0) encode_planes(mag, r, kmax, j, ws.staging + pi, lim);
    if (r > 0 && pi + r > ws.staging_words) bad = HOSZP_ERR_CAPACITY;
    if (tile == ntiles - 1 && tid == 0) {
      ws.totals[0] = NC + ts.agg_nc;
      ws.totals[1] = RR + ts.agg_r;
    }
    __syncthreads();
  }
  // epilogue: max |q| for the header's qbound, first error, launch bookkeeping
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
  if ((tid & 31) == 0) s_qmax[tid >> 5] = qmax;
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < CTA / 32; w++) qmax = max(qmax, s_qmax[w]);
    atomicMax(&ws.totals[2], (unsigned long long)qmax);
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

cudaError_t launch_compress(const Launch& lc, const float* x, uint64_t n, const uint32_t dims[3],
                            uint32_t ndims, float eps_q_abs, double eps_abs, bool rel, uint8_t* out,
                            uint64_t cap, Ws ws) {
  k_compress<<<persistent_grid(k_compress, CTA, lc.grid), CTA, 0, lc.stream>>>(x, n, dims[0], dims[1], dims[2], ndims, eps_q_abs,
                                             eps_abs, rel ? 1 : 0, out, cap, ws);
  return cudaGetLastError();
}

}  // namespace hz
