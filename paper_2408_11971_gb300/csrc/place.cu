// place.cu — completes a produced stream (compress, scalar multiplication,
// element-wise addition). The producer wrote rates and outliers at their
// final offsets and each tile's sign and plane words into the tile's
// workspace slot; the produced-tile scan gave every tile's place. Only with
// the total number of non-constant blocks does the plane section's start
// (right after the sign section, Fig. 3) exist, so the words are moved here,
// and the header is written last.
#include "hz_ws.cuh"
#include "hz_kernels.cuh"

namespace hz {

__global__ void __launch_bounds__(512) k_place(uint8_t* __restrict__ out, uint64_t cap,
                                               uint64_t* out_bytes, int rule, uint32_t e_bits,
                                               Ws ws) {
  const hoszp_header tmpl = *ws.hdr;
  const uint64_t nb = nblocks(tmpl.n);
  const uint64_t ntiles = ntiles_of(nb);
  const uint64_t nnc = ws.totals[0], R = ws.totals[1];
  const uint64_t size = stream_bytes(nb, nnc, R);
  const bool fits = size <= cap && ntiles + 1 <= ws.max_tiles;
  int bad = 0;
  if (fits) {
    uint64_t* sdst = reinterpret_cast<uint64_t*>(out + off_sign(nb));
    uint64_t* pdst = reinterpret_cast<uint64_t*>(out + off_plane(nb, nnc));
    // one warp per tile; each lane moves up to 8 words per step with all its
    // loads issued before its stores
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles;
         t += nwarps) {
      const unsigned long long a = ws.agg[t];
      const uint64_t nc = a >> 32, r = a & 0xffffffffull;
      uint64_t so, po;  // word offsets of the tile's sign words and plane words
      if (rule == SLOT_SPLIT) {
        so = ws.pre[0][2 * t];
        po = ws.pre[0][2 * t + 1];
      } else {
        so = slot_offset(rule, t, ws.pre[0], ws.pre[1], e_bits);
        po = so + nc;
      }
      const uint64_t NC = ws.opre[2 * t], RR = ws.opre[2 * t + 1];
      if (so + nc > ws.staging_words || po + r > ws.staging_words || NC + nc > nnc ||
          RR + r > R) {
        bad = HOSZP_ERR_CAPACITY;
        continue;
      }
      const uint64_t* ssrc = ws.staging + so;
      const uint64_t* psrc = ws.staging + po - nc;  // word i >= nc of the tile at psrc[i]
      const uint64_t words = nc + r;
      constexpr int U = 8;
      for (uint64_t i0 = lane; i0 < words; i0 += 32 * U) {
        uint64_t v[U];
#pragma unroll
        for (int u = 0; u < U; u++)
          if (i0 + 32 * u < words)
            v[u] = __ldcs((i0 + 32 * u < nc ? ssrc : psrc) + i0 + 32 * u);
#pragma unroll
        for (int u = 0; u < U; u++) {
          const uint64_t i = i0 + 32 * u;
          if (i < nc) sdst[NC + i] = v[u];
          else if (i < words) pdst[RR + i - nc] = v[u];
        }
      }
    }
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
  if (bad) set_status(ws.status, bad);
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
                         int rule, uint32_t e_bits, Ws ws) {
  cudaError_t e = launch_scan_agg(lc, ws);
  if (e != cudaSuccess) return e;
  k_place<<<persistent_grid(k_place, 512, lc.grid), 512, 0, lc.stream>>>(out, cap, out_bytes,
                                                                         rule, e_bits, ws);
  return cudaGetLastError();
}

}  // namespace hz
