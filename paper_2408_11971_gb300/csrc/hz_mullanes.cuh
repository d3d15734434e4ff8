// hz_mullanes.cuh — one 64-block tile of scalar multiplication (Sec. V-A,
// workflow 3) held two lanes per block: decode to q, requantize
// q' = floor(2e q rho + 1/2), Lorenzo, encode and store the sign and plane
// half-words into the tile's slots. Shared by the single-stream kernel (input
// tiles in shared-memory stages) and the batched kernel (input tiles read from
// each field's stream in global memory).
#pragma once
#include "hz_lanes.cuh"
#include "hz_mul.cuh"
#include "hz_produce.cuh"
#include "hz_super.cuh"

namespace hz {

// Local prefixes of a half for the warp's widest input rate Rw.
__device__ __forceinline__ void half_prefix_any(int Rw, const uint32_t t[32], bool zero0,
                                                const lanes::Shifts& K, int p[32]) {
  const int G = (Rw + 8) >> 3;
  if (G == 1) lanes::half_prefix<1>(t, zero0, K, p);
  else if (G == 2) lanes::half_prefix<2>(t, zero0, K, p);
  else if (G == 3) lanes::half_prefix<3>(t, zero0, K, p);
  else lanes::half_prefix<4>(t, zero0, K, p);
}

// Orders the work on v[0 .. 7] before the work on v[8 .. 15]: an empty asm
// that takes the first eight as inputs and gives the next eight as outputs,
// so the compiler cannot start the next chunk's 64- or 128-bit products early
// (which would keep wide temporaries of all 32 values live at once).
__device__ __forceinline__ void chunk_fence(int* v) {
  asm volatile(""
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]));
}

// Bits of the largest |delta'| a warp can produce from input deltas below
// 2^Rw: |q'_i - q'_(i-1)| < |k| |delta| + 1, so |delta'| <= ceil(|k| (2^Rw - 1))
// (k = 2e rho, or s for the exact variant; kabs carries a relative margin).
__device__ __forceinline__ int delta_bits(double kabs, int Rw) {
  const double b = ceil(kabs * (double)((1u << Rw) - 1u));
  if (!(b < 2147483648.0)) return 31;
  const uint32_t v = (uint32_t)b;
  return 32 - __clz(v);
}

// The tile: its rates and in-tile prefixes tr, the half-words of its sign
// words (sgn) and plane words (pls), its 64 outliers (outl), the length of its
// last block (lastlen). The plan vp and the plane-group table s_ge (by the
// warp's widest input rate) sit in shared memory. Writes every block's rate and
// new outlier to out_rate[b], out_outl[b] and the words to the slots sdst /
// pdst (at most lim_nc sign and lim_r plane words); returns the tile's output
// (sign words << 16 | plane words). vmax / vmin gather the extremes of q'; ovf
// and tbad collect overflow and slot errors.
__device__ __forceinline__ uint32_t mul_lanes_tile(
    const TileRates& tr, const uint32_t* sgn, const uint32_t* pls, const int* outl, int lastlen,
    const volatile MulPlan* vp, const uint8_t* s_ge, const lanes::Shifts& K, uint32_t* sdst,
    uint32_t* pdst, uint32_t lim_nc, uint32_t lim_r, uint8_t* out_rate, int* out_outl, int& vmax,
    int& vmin, bool& ovf, int& tbad) {
  const int lane = threadIdx.x & 31;
  const int hf = lane & 1, m = lane >> 1;
        uint32_t run = 0;  // output (sign words << 16 | plane words) of the tile so far
        const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
        for (int it = 0; it < steps; it++) {
          const int b = 16 * it + m;
          uint32_t r, ex;
          tile_block(tr, b, r, ex);
          const int len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? lastlen : 0;
          const int nval = min(max(len - 32 * hf, 0), 32);
          const int O = len ? outl[b] : 0;
          const uint32_t sw = r ? sgn[2 * (ex >> 16) + hf] : 0u;
          const int Rw = (int)__reduce_max_sync(0xffffffffu, r);
          const bool fullblk = __all_sync(0xffffffffu, len == L);
          int v[32];
          {
            uint32_t t[32];
            lanes::twos_planes_any(Rw, pls + 2 * (ex & 0xffffu) + hf, (int)r, sw, t);
            half_prefix_any(Rw, t, hf == 0, K, v);
          }
          // the second half's base: O plus the first half's delta total (every
          // lane takes part in the exchange, then selects)
          const int tot0 = __shfl_xor_sync(0xffffffffu, v[31], 1);
          const int base = O + (hf ? tot0 : 0);
          if (fullblk) {
  #pragma unroll
            for (int i = 0; i < 32; i++) v[i] += base;
          } else {
  #pragma unroll
            for (int i = 0; i < 32; i++) v[i] = (i < nval) ? v[i] + base : 0;
          }
          // requantization (the plan is uniform over the launch)
          if (vp->f32) {
            MulPlan mp;
            mp.rho32 = vp->rho32;
            mp.M32 = vp->M32;
            mp.sh2 = vp->sh2;
            mp.half = vp->half;
  #pragma unroll
            for (int c8 = 0; c8 < 32; c8 += 8) {
  #pragma unroll
              for (int i = c8; i < c8 + 8; i++) v[i] = mul_requant_f32(v[i], mp);
              if (c8 < 24) chunk_fence(v + c8);
            }
          } else if (vp->fast) {
            MulPlan mp;
            mp.P = vp->P;
            mp.sh = vp->sh;
  #pragma unroll
            for (int c8 = 0; c8 < 32; c8 += 8) {
  #pragma unroll
              for (int i = c8; i < c8 + 8; i++) v[i] = mul_requant_fast(v[i], mp, ovf);
              if (c8 < 24) chunk_fence(v + c8);
            }
          } else {  // 128-bit products (rare): one value at a time, rotating the half
            MulPlan mp;
            mp.rho = vp->rho;
            mp.M = vp->M;
            mp.E = vp->E;
  #pragma unroll 1
            for (int i = 0; i < 32; i++) {
              const int x = mul_requant(v[0], mp, ovf);
  #pragma unroll
              for (int j = 0; j < 31; j++) v[j] = v[j + 1];
              v[31] = x;
            }
          }
  #pragma unroll
          for (int i = 0; i < 32; i += 2) {
            vmax = __vimax3_s32(vmax, v[i], v[i + 1]);
            vmin = __vimin3_s32(vmin, v[i], v[i + 1]);
          }
          // Lorenzo on q' (Eq. 4): the second half's first delta takes the first
          // half's last value
          const int last0 = __shfl_xor_sync(0xffffffffu, v[31], 1);
          const int o_new = v[0];
  #pragma unroll
          for (int i = 31; i > 0; i--) v[i] -= v[i - 1];
          v[0] = hf ? v[0] - last0 : 0;
          if (!fullblk) {
  #pragma unroll
            for (int i = 0; i < 32; i++)
              if (i >= nval) v[i] = 0;
          }
          const bool valid = b < tr.nvt;
          const int Ge = s_ge[Rw];
          const int rate = encode_store_any(Ge, v, K, valid, sdst, pdst, lim_nc, lim_r, run, tbad);
          if (valid && hf == 0) {
        out_rate[b] = (uint8_t)rate;
        out_outl[b] = o_new;
      }
        }
  return run;
}

}  // namespace hz
