// baseline.cu — float32 operators of the traditional workflow (Sec. IV-B,
// Fig. 4a): used between a full decompression and a full recompression to
// time the "decompress -> op -> recompress" comparator on the same GPU.
#include "hoszp_baseline.h"
#include "hz_kernels.cuh"

namespace hz {

__global__ void __launch_bounds__(512) k_axpb(const float4* __restrict__ x, float4* y, uint64_t n4,
                                              const float* xs, float* ys, uint64_t n, float a,
                                              float b) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 v = x[i];
    v.x = __fmaf_rn(a, v.x, b);
    v.y = __fmaf_rn(a, v.y, b);
    v.z = __fmaf_rn(a, v.z, b);
    v.w = __fmaf_rn(a, v.w, b);
    y[i] = v;
  }
  for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    ys[i] = __fmaf_rn(a, xs[i], b);
}

__global__ void __launch_bounds__(512) k_add2(const float4* __restrict__ x,
                                              const float4* __restrict__ y, float4* z, uint64_t n4,
                                              const float* xs, const float* yss, float* zs,
                                              uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 u = x[i], v = y[i];
    z[i] = make_float4(u.x + v.x, u.y + v.y, u.z + v.z, u.w + v.w);
  }
  for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    zs[i] = xs[i] + yss[i];
}

__global__ void __launch_bounds__(512) k_fmoments(const float4* __restrict__ x, uint64_t n4,
                                                  const float* xs, uint64_t n, int variance,
                                                  double* result, Ws ws) {
  float s = 0.f, s2 = 0.f;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 v = x[i];
    s += (v.x + v.y) + (v.z + v.w);
    s2 = __fmaf_rn(v.x, v.x, s2);
    s2 = __fmaf_rn(v.y, v.y, s2);
    s2 = __fmaf_rn(v.z, v.z, s2);
    s2 = __fmaf_rn(v.w, v.w, s2);
  }
  for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    s += xs[i];
    s2 = __fmaf_rn(xs[i], xs[i], s2);
  }
  double ds = s, ds2 = s2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ds += __shfl_xor_sync(0xffffffffu, ds, o);
    ds2 += __shfl_xor_sync(0xffffffffu, ds2, o);
  }
  __shared__ double sh[2][16];
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = ds;
    sh[1][threadIdx.x >> 5] = ds2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      ds += sh[0][w];
      ds2 += sh[1][w];
    }
    double* p = reinterpret_cast<double*>(ws.partials) + 2 * blockIdx.x;
    p[0] = ds;
    p[1] = ds2;
  }
  if (launch_end_is_last(ws) && threadIdx.x == 0) {
    double t = 0, t2 = 0;
    const double* p = reinterpret_cast<const double*>(ws.partials);
    for (unsigned int b = 0; b < gridDim.x; b++) {
      t += p[2 * b];
      t2 += p[2 * b + 1];
    }
    const double m = t / (double)n;
    *result = variance ? (t2 / (double)n - m * m) : m;
    launch_reset(ws);
  }
}

}  // namespace hz

using namespace hz;

namespace {
inline bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
int grid_of(const void* k) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 4;
}
}  // namespace

extern "C" int hoszp_fop_axpb(const float* d_x, float* d_y, uint64_t n, float a, float b,
                              hoszp_stream_t stream) {
  if ((n > 0 && (!d_x || !d_y)) || !al16(d_x) || !al16(d_y)) return HOSZP_ERR_ARG;
  if (n == 0) return HOSZP_OK;
  k_axpb<<<grid_of((const void*)k_axpb), 512, 0, (cudaStream_t)stream>>>(
      (const float4*)d_x, (float4*)d_y, n / 4, d_x, d_y, n, a, b);
  return cudaGetLastError() == cudaSuccess ? HOSZP_OK : HOSZP_ERR_CUDA;
}

extern "C" int hoszp_fop_add(const float* d_x, const float* d_y, float* d_z, uint64_t n,
                             hoszp_stream_t stream) {
  if ((n > 0 && (!d_x || !d_y || !d_z)) || !al16(d_x) || !al16(d_y) || !al16(d_z))
    return HOSZP_ERR_ARG;
  if (n == 0) return HOSZP_OK;
  k_add2<<<grid_of((const void*)k_add2), 512, 0, (cudaStream_t)stream>>>(
      (const float4*)d_x, (const float4*)d_y, (float4*)d_z, n / 4, d_x, d_y, d_z, n);
  return cudaGetLastError() == cudaSuccess ? HOSZP_OK : HOSZP_ERR_CUDA;
}

// defined in api.cu: the context's workspace (partials + launch bookkeeping)
namespace hz {
Ws ctx_workspace(hoszp_ctx* ctx);
}

extern "C" int hoszp_fop_moments(hoszp_ctx* ctx, const float* d_x, uint64_t n, int variance,
                                 double* d_result, hoszp_stream_t stream) {
  if (!ctx || !d_x || !d_result || n == 0 || !al16(d_x)) return HOSZP_ERR_ARG;
  Ws ws = ctx_workspace(ctx);
  if (!ws.partials) return HOSZP_ERR_CUDA;
  k_fmoments<<<grid_of((const void*)k_fmoments), 512, 0, (cudaStream_t)stream>>>(
      (const float4*)d_x, n / 4, d_x, n, variance, d_result, ws);
  return cudaGetLastError() == cudaSuccess ? HOSZP_OK : HOSZP_ERR_CUDA;
}
