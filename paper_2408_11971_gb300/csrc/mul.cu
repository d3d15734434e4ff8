// mul.cu — scalar multiplication (Sec. V-A, workflow 3) and multiplication by
// the scalar itself, two lanes per block on the super-tile pipeline.
//
// Each value goes through the quantized integers: q from the stored deltas
// (inverse Lorenzo), q' = floor(2e q rho + 1/2) (Eq. 3 applied to the product
// of the dequantized values), then Lorenzo, sign, rate and bit-planes again
// (Eq. 4, Fig. 3). A lane holds one 32-position half of a block in registers
// the whole way (hz_lanes.cuh):
//   planes -> two's-complement planes -> per-position prefixes  (decode)
//   -> q, q', delta'                                           (per value)
//   -> two's-complement planes of delta' -> sign and magnitude  (encode)
// so no value crosses lanes except the one base and one last value that the
// two halves of a block exchange.
//
// Input: the single-stream super-tile pipeline (one loader warp, in-kernel
// rate prefix, no pre-scan launch). Warp i of a group takes tile i of a stage
// and walks it 16 blocks at a time, keeping a running count of the tile's
// output sign and plane words, so it can write every block's words as soon as
// they exist: sign words to the tile's sign slot, plane words to its plane
// slot (the SPLIT rule of hz_ws.cuh). Both slots start at upper bounds known
// from the input's prefix before the tile: a constant input block stays
// constant, and a block's rate grows by at most e bits. The produced-tile scan
// and the placement kernel then move the words to their final places.
#include <climits>

#include "hz_lanes.cuh"
#include "hz_mul.cuh"
#include "hz_produce.cuh"
#include "hz_scalar.cuh"
#include "hz_super.cuh"
#include "hz_kernels.cuh"

namespace hz {

// Five tiles per stage, one per compute warp of a group, three groups: 16
// warps, so that a thread may hold 128 registers (a lane keeps 32 values and
// up to 32 plane words of its half at once).
constexpr int ML_NT = 5;
constexpr int ML_GW = ML_NT;  // warps per group: one per tile of a stage
constexpr int ML_GROUPS = 3;
constexpr int ML_NCW = ML_GW * ML_GROUPS;
constexpr int ML_THREADS = (ML_NCW + 1) * 32;  // + loader warp
constexpr int ML_STAGES = 6;
constexpr uint32_t ML_RING = 22528;  // plane-ring words (176 KB)

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

template <int MODE>
__global__ void __launch_bounds__(ML_THREADS, 1) k_mul_lanes(
    const uint8_t* __restrict__ c, uint64_t c_bytes, double s, uint8_t* __restrict__ out,
    uint64_t cap, uint32_t e_bits, Ws ws) {
  extern __shared__ __align__(16) uint8_t dyn[];
  using St = SStageT<ML_NT>;
  St* stages = reinterpret_cast<St*>(dyn);
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + ML_STAGES);
  __shared__ uint64_t full[ML_STAGES], empty[ML_STAGES];
  __shared__ unsigned long long stage_st[ML_STAGES];
  __shared__ uint32_t s_ts[TS_MAX];
  __shared__ MulPlan s_mp;  // read back (volatile) where used: no registers held across steps
  __shared__ uint8_t s_ge[32];  // plane groups of the output deltas, by the warp's widest input rate
  __shared__ int s_ok;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const Info h = parse_header(c, c_bytes);
  const unsigned long long epoch = launch_epoch(ws);
  int bad = 0;
  if (tid == 0) {
    int ok = h.ok;
    long long rho = 0;
    if (!h.ok) {
      bad = HOSZP_ERR_FORMAT;
    } else if (MODE == 0 && !quantize_scalar(s, h.eps_q, rho)) {
      ok = 0;
      bad = HOSZP_ERR_RANGE;
    } else if (cap < off_sign(h.nb) || ntiles_of(h.nb) + 1 > ws.max_tiles) {
      ok = 0;
      bad = HOSZP_ERR_CAPACITY;
    }
    s_ok = ok;
    s_mp = MODE == 1 ? mul_plan_exact(s, h.ok ? h.qbound : 0u)
                     : mul_plan(h.ok ? h.eps_q : 1.0f, rho, h.ok ? h.qbound : 0u);
    // |k| for the bound of the output deltas, with a relative margin
    const double kabs =
        (MODE == 1 ? fabs(s) : fabs(2.0 * (double)h.eps_q * (double)rho)) * (1.0 + 0x1p-40);
    for (int R = 0; R < 32; R++) s_ge[R] = (uint8_t)min(4, (delta_bits(kabs, R) + 8) >> 3);
    if (blockIdx.x == 0) write_template(h, 0, ws);
    for (int k = 0; k < ML_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], ML_GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  const uint64_t ntiles = ok ? ntiles_of(h.nb) : 0;
  const uint64_t nst = nsuper_of<ML_NT>(ntiles);
  const uint8_t* const cs = c;
  const SRange rg = range_sums_n<ML_NT, 1>(&cs, &h, ntiles, nst, s_ts, TS_MAX, ws, epoch, bad);
  __syncthreads();
  int vmax = 0, vmin = 0;  // extremes of q' (zeros included: max |q'| is unchanged)
  bool ovf = false;
  if (w == ML_NCW) {
    __shared__ uint32_t s_beg[ML_STAGES];
    super_loader_n<ML_NT, 1, ML_STAGES, ML_RING, ML_GROUPS>(stages, ring, s_beg, full, empty,
                                                             stage_st, &cs, &h, rg, s_ts, TS_MAX,
                                                             ws, epoch);
  } else if (w < ML_NCW) {
    const volatile MulPlan* vp = &s_mp;
    const int grp = w / ML_GW, ti = w % ML_GW;
    const int hf = lane & 1, m = lane >> 1;
    const int lastlen = (int)(h.n - (h.nb - 1) * L);
    const lanes::Shifts K = lanes::make_shifts(c_bytes != 0 ? 1u : 0u);
    // sign slots first ([0, nnc) words), plane slots after them
    const uint64_t sign_cap = umin64(h.nnc, ws.staging_words);
    for (uint64_t k = 0;; k++) {
      const uint64_t u = k * ML_GROUPS + grp;  // stage use taken by this group
      const int sk = (int)(u % ML_STAGES);
      if (!mbar_wait_warp(&full[sk], (uint32_t)((u / ML_STAGES) & 1), ws.status)) break;
      const unsigned long long st = stage_st[sk];
      if (st == ~0ull) break;
      const St& sg = stages[sk];
      const uint64_t tile = (uint64_t)ML_NT * st + ti;
      const TileRates tr = tile_rates(sg, ti, tile, h.nb);
      const uint32_t* sgn = reinterpret_cast<const uint32_t*>(sg.sign + sg.sbase + sg.tnc[ti]);
      const uint32_t* pls =
          reinterpret_cast<const uint32_t*>(ring + sg.pring + sg.pbase + sg.tr[ti]);
      // upper bounds of the output words before this tile
      const uint64_t pnc = sg.bnc + sg.tnc[ti], pr = sg.br + sg.tr[ti];
      const uint64_t so = pnc, po = sign_cap + pnc * e_bits + pr;
      // the tile's input words bound its output words: check once per tile
      const uint32_t tin = (tr.nvt > 0) ? __shfl_sync(0xffffffffu, tr.e1 + (tr.r1 ? 0x10000u : 0u) + tr.r1, 31) : 0u;
      const uint64_t tin_nc = tin >> 16, tin_r = tin & 0xffffu;
      const uint32_t lim_nc = (uint32_t)tin_nc, lim_r = (uint32_t)(tin_nc * e_bits + tin_r);
      int tbad = 0;
      if (so + lim_nc > sign_cap || po + lim_r > ws.staging_words) tbad = HOSZP_ERR_CAPACITY;
      uint32_t* sdst = reinterpret_cast<uint32_t*>(ws.staging + so);
      uint32_t* pdst = reinterpret_cast<uint32_t*>(ws.staging + po);
      uint32_t run = 0;  // output (sign words << 16 | plane words) of the tile so far
      const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
      for (int it = 0; it < steps; it++) {
        const int b = 16 * it + m;
        uint32_t r, ex;
        tile_block(tr, b, r, ex);
        const int len =
            (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
        const int nval = min(max(len - 32 * hf, 0), 32);
        const int O = len ? sg.outlier[TILE * ti + b] : 0;
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
          const uint64_t bi = tile * TILE + b;
          out[HOSZP_HEADER_BYTES + bi] = (uint8_t)rate;
          reinterpret_cast<int*>(out + off_outlier(h.nb))[bi] = o_new;
        }
      }
      if (tbad) bad = tbad;
      if (lane == 0 && tile < ntiles) {
        ws.agg[tile] = ((unsigned long long)(run >> 16) << 32) | (run & 0xffffu);
        ws.pre[0][2 * tile] = so;
        ws.pre[0][2 * tile + 1] = po;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sk]);
    }
  }
  if (ovf) bad = HOSZP_ERR_OVERFLOW;
  reduce_qmax(max((uint32_t)vmax, (uint32_t)(-(long long)vmin)), ws);
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && w == 0) {
    const bool tot_ok = range_totals_ok(ws, h);
    if (tid == 0) {
      if (ok && !tot_ok) set_status(ws.status, HOSZP_ERR_FORMAT);
      launch_reset(ws);
    }
  }
}

template <int MODE>
static cudaError_t launch_mul_lanes(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                                    uint32_t e_bits, uint8_t* out, uint64_t cap, Ws ws) {
  const size_t smem = ML_STAGES * sizeof(SStageT<ML_NT>) + ML_RING * sizeof(uint64_t);
  smem_attr<k_mul_lanes<MODE>>(smem);
  const int grid = persistent_grid(k_mul_lanes<MODE>, ML_THREADS, lc.grid, smem);
  if ((uint64_t)grid > ws.max_grid) return cudaErrorInvalidConfiguration;
  k_mul_lanes<MODE><<<grid, ML_THREADS, smem, lc.stream>>>(c, c_bytes, s, out, cap, e_bits, ws);
  return cudaGetLastError();
}

cudaError_t launch_mul_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              bool exact, uint32_t e_bits, uint8_t* out, uint64_t cap, Ws ws) {
  return exact ? launch_mul_lanes<1>(lc, c, c_bytes, s, e_bits, out, cap, ws)
               : launch_mul_lanes<0>(lc, c, c_bytes, s, e_bits, out, cap, ws);
}

}  // namespace hz
