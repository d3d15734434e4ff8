// place.cu — completes a produced stream (compress, scalar multiplication,
// element-wise addition). The producer has written rates, outliers and sign
// words at their final offsets and the plane words, in order, into the
// workspace; only once the total number of non-constant blocks is known does
// the plane section's start (right after the sign section, Fig. 3) exist, so
// the planes are copied there here, and the header is written last.
#include "hz_kernels.cuh"

namespace hz {

__global__ void __launch_bounds__(512) k_place(uint8_t* __restrict__ out, uint64_t cap,
                                               uint64_t* out_bytes, Ws ws) {
  const hoszp_header tmpl = *ws.hdr;
  const uint64_t nb = nblocks(tmpl.n);
  const uint64_t nnc = ws.totals[0], R = ws.totals[1];
  const uint64_t size = stream_bytes(nb, nnc, R);
  const bool fits = size <= cap && R <= ws.staging_words;
  if (fits) {
    const uint64_t* __restrict__ src = ws.staging;
    uint64_t* __restrict__ dst = reinterpret_cast<uint64_t*>(out + off_plane(nb, nnc));
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += stride)
      dst[i] = src[i];
    if (blockIdx.x == 0) {
      // zero the end padding and the padding after the rate and outlier sections
      const uint64_t end = off_plane(nb, nnc) + 8 * R;
      if (threadIdx.x == 32 && (end & 15)) *reinterpret_cast<uint64_t*>(out + end) = 0;
      const uint64_t pr = HOSZP_HEADER_BYTES + nb, pr_end = off_outlier(nb);
      const uint64_t po = off_outlier(nb) + 4 * nb, po_end = off_sign(nb);
      if (threadIdx.x < 16 && pr + threadIdx.x < pr_end) out[pr + threadIdx.x] = 0;
      if (threadIdx.x >= 16 && threadIdx.x < 32 && po + threadIdx.x - 16 < po_end)
        out[po + threadIdx.x - 16] = 0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (fits) {
      hoszp_header h = tmpl;
      h.nnc = nnc;
      h.R = R;
      h.qbound = (uint32_t)ws.totals[2];
      *reinterpret_cast<hoszp_header*>(out) = h;
      *out_bytes = size;
    } else {
      set_status(ws.status, HOSZP_ERR_CAPACITY);
      *out_bytes = 0;
    }
  }
  if (launch_end_is_last(ws) && threadIdx.x == 0) {
    ws.totals[0] = 0;
    ws.totals[1] = 0;
    ws.totals[2] = 0;
    launch_reset(ws);
  }
}

cudaError_t launch_place(const Launch& lc, uint8_t* out, uint64_t cap, uint64_t* out_bytes,
                         Ws ws) {
  k_place<<<persistent_grid(k_place, 512, lc.grid), 512, 0, lc.stream>>>(out, cap, out_bytes, ws);
  return cudaGetLastError();
}

}  // namespace hz
