// place.cu — completes a produced stream (compress, scalar multiplication,
// element-wise addition). The producer wrote rates and outliers at their
// final offsets, each tile's sign and plane words into the tile's workspace
// slot and each tile's word counts into agg[]; the exclusive prefix of those
// counts gives every tile's place. Only with
// the total number of non-constant blocks does the plane section's start
// (right after the sign section, Fig. 3) exist, so the words are moved here,
// and the header is written last.
#include "hz_ws.cuh"
#include "hz_kernels.cuh"

namespace hz {

// The tile-aggregate scan is folded in: CTA g of G takes the g-th of G
// contiguous chunks of the produced tiles, sums the chunk's aggregates and
// publishes the sum (under the launch's epoch, like the in-kernel rate prefix
// of the reductions). One warp then adds up every chunk's sum: those before g
// give the chunk's base, all of them the stream's totals (nnc, R), which place
// the plane section. A chunk sum that is not published within PLACE_POLL_NS
// (its CTA may not be resident yet) is summed by the waiting warp itself from
// the aggregates, so no CTA depends on another being scheduled. The chunk is
// then walked in rounds of PL_THREADS tiles: a CTA scan gives each tile's
// offsets, and one warp per tile moves its words.
constexpr int PL_THREADS = 512;
constexpr int PL_WARPS = PL_THREADS / 32;
constexpr unsigned long long PLACE_POLL_NS = 4000;

__device__ __forceinline__ unsigned long long place_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Whole warp: the (nc, r) sums of the produced tiles [t0, t1); every lane gets them.
__device__ __forceinline__ void agg_range_sum(const unsigned long long* agg, uint64_t t0,
                                              uint64_t t1, unsigned long long& nc,
                                              unsigned long long& r) {
  const int lane = threadIdx.x & 31;
  nc = 0;
  r = 0;
  for (uint64_t t = t0 + lane; t < t1; t += 32) {
    const unsigned long long a = agg[t];
    nc += a >> 32;
    r += a & 0xffffffffull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nc += __shfl_xor_sync(0xffffffffu, nc, o);
    r += __shfl_xor_sync(0xffffffffu, r, o);
  }
}

__global__ void __launch_bounds__(PL_THREADS, 2) k_place(uint8_t* __restrict__ out, uint64_t cap,
                                                      uint64_t* out_bytes, int rule,
                                                      uint32_t e_bits, Ws ws) {
  __shared__ unsigned long long s_red[2][PL_WARPS];
  __shared__ unsigned long long s_base[4];  // chunk base (nc, r), stream totals (nnc, R)
  __shared__ unsigned long long s_off[PL_THREADS], s_agg[PL_THREADS];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const hoszp_header tmpl = *ws.hdr;
  const uint64_t nb = nblocks(tmpl.n);
  const bool tiles_fit = ntiles_of(nb) + 1 <= ws.max_tiles && gridDim.x <= ws.max_grid;
  const uint64_t ntiles = tiles_fit ? ntiles_of(nb) : 0;
  const unsigned long long epoch = launch_epoch(ws);
  const unsigned long long want = (epoch << 1) | 1ull;
  const uint64_t G = gridDim.x, g = blockIdx.x;
  const uint64_t t0 = ntiles * g / G, t1 = ntiles * (g + 1) / G;

  // the chunk's sum, published for the other CTAs
  {
    unsigned long long nc = 0, r = 0;
    for (uint64_t t = t0 + tid; t < t1; t += PL_THREADS) {
      const unsigned long long a = ws.agg[t];
      nc += a >> 32;
      r += a & 0xffffffffull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nc += __shfl_xor_sync(0xffffffffu, nc, o);
      r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if (lane == 0) {
      s_red[0][w] = nc;
      s_red[1][w] = r;
    }
    __syncthreads();
    if (tid == 0) {
      unsigned long long a = 0, b = 0;
      for (int k = 0; k < PL_WARPS; k++) {
        a += s_red[0][k];
        b += s_red[1][k];
      }
      if (tiles_fit) {
        CtaAgg* c = ws.cta_agg + g;
        c->nc = a;
        c->r = b;
        __threadfence();
        st_release(&c->flag, want);
      }
    }
  }
  // every chunk's sum: the base of this chunk and the stream's totals
  if (w == 0) {
    unsigned long long bnc = 0, br = 0, tnc = 0, tr = 0;
    const unsigned long long ts = place_timer_ns();
    for (uint64_t base = 0; tiles_fit && base < G; base += 32) {
      const uint64_t u = base + lane;
      unsigned long long a = 0, b = 0;
      bool have = u >= G;
      if (!have) {
        const CtaAgg* c = ws.cta_agg + u;
        for (;;) {
          if (ld_acquire(&c->flag) == want) {
            a = *reinterpret_cast<const volatile unsigned long long*>(&c->nc);
            b = *reinterpret_cast<const volatile unsigned long long*>(&c->r);
            have = true;
            break;
          }
          if (place_timer_ns() - ts > PLACE_POLL_NS) break;
          __nanosleep(128);
        }
      }
      unsigned int miss = __ballot_sync(0xffffffffu, !have);
      while (miss) {  // late chunks: the whole warp sums them from the aggregates
        const int src = __ffs(miss) - 1;
        miss &= miss - 1;
        const uint64_t v = base + src;
        unsigned long long sa, sb;
        agg_range_sum(ws.agg, ntiles * v / G, ntiles * (v + 1) / G, sa, sb);
        if (lane == src) {
          a = sa;
          b = sb;
        }
      }
      if (u < G) {
        tnc += a;
        tr += b;
        if (u < g) {
          bnc += a;
          br += b;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bnc += __shfl_xor_sync(0xffffffffu, bnc, o);
      br += __shfl_xor_sync(0xffffffffu, br, o);
      tnc += __shfl_xor_sync(0xffffffffu, tnc, o);
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    if (lane == 0) {
      s_base[0] = bnc;
      s_base[1] = br;
      s_base[2] = tnc;
      s_base[3] = tr;
    }
  }
  __syncthreads();
  const uint64_t nnc = s_base[2], R = s_base[3];
  const uint64_t size = stream_bytes(nb, nnc, R);
  const bool fits = tiles_fit && size <= cap;
  int bad = 0;
  if (fits) {
    uint64_t* sdst = reinterpret_cast<uint64_t*>(out + off_sign(nb));
    uint64_t* pdst = reinterpret_cast<uint64_t*>(out + off_plane(nb, nnc));
    unsigned long long run_nc = s_base[0], run_r = s_base[1];
    for (uint64_t r0 = t0; r0 < t1; r0 += PL_THREADS) {
      // offsets of the round's tiles: a CTA scan of (nc << 32 | r), which
      // cannot carry between the halves within PL_THREADS tiles
      const uint64_t t = r0 + tid;
      const unsigned long long a = (t < t1) ? ws.agg[t] : 0ull;
      unsigned long long inc = a;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) s_red[0][w] = inc;
      __syncthreads();
      unsigned long long wb = 0, tot = 0;
#pragma unroll
      for (int k = 0; k < PL_WARPS; k++) {
        const unsigned long long v = s_red[0][k];
        wb += (k < w) ? v : 0ull;
        tot += v;
      }
      s_off[tid] = wb + inc - a;
      s_agg[tid] = a;
      __syncthreads();
      const int nt = (int)umin64(PL_THREADS, t1 - r0);
      for (int k = w; k < nt; k += PL_WARPS) {
        const uint64_t tt = r0 + k;
        const unsigned long long ag = s_agg[k], ex = s_off[k];
        const uint64_t nc = ag >> 32, r = ag & 0xffffffffull;
        const uint64_t NC = run_nc + (ex >> 32), RR = run_r + (ex & 0xffffffffull);
        uint64_t so, po;  // word offsets of the tile's sign words and plane words
        if (rule == SLOT_SPLIT) {
          so = ws.pre[0][2 * tt];
          po = ws.pre[0][2 * tt + 1];
        } else {
          so = slot_offset(rule, tt, ws.pre[0], ws.pre[1], e_bits);
          po = so + nc;
        }
        if (so + nc > ws.staging_words || po + r > ws.staging_words || NC + nc > nnc ||
            RR + r > R) {
          bad = HOSZP_ERR_CAPACITY;
          continue;
        }
        const uint64_t* ssrc = ws.staging + so;
        const uint64_t* psrc = ws.staging + po;
        uint64_t* sd = sdst + NC;
        uint64_t* pd = pdst + RR;
        const uint32_t nc32 = (uint32_t)nc, words = nc32 + (uint32_t)r;  // <= 64 + 1984
        // each lane moves up to 8 words per step, all its loads before its stores
        constexpr int U = 8;
        for (uint32_t i0 = lane; i0 < words; i0 += 32 * U) {
          uint64_t v[U];
#pragma unroll
          for (int u = 0; u < U; u++) {
            const uint32_t i = i0 + 32 * u;
            if (i < words) v[u] = __ldcs(i < nc32 ? ssrc + i : psrc + (i - nc32));
          }
#pragma unroll
          for (int u = 0; u < U; u++) {
            const uint32_t i = i0 + 32 * u;
            if (i < nc32) sd[i] = v[u];
            else if (i < words) pd[i - nc32] = v[u];
          }
        }
      }
      run_nc += tot >> 32;
      run_r += tot & 0xffffffffull;
      __syncthreads();  // s_red, s_off and s_agg are rewritten by the next round
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
  k_place<<<persistent_grid(k_place, PL_THREADS, lc.grid), PL_THREADS, 0, lc.stream>>>(
      out, cap, out_bytes, rule, e_bits, ws);
  return cudaGetLastError();
}

}  // namespace hz
