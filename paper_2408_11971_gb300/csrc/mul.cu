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
// constant, and a block's rate grows by at most e bits. The placement kernel
// then scans the tiles' word counts and moves the words to their final places.
#include <climits>

#include "hz_mullanes.cuh"
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
    super_loader_n<ML_NT, 1, ML_STAGES, ML_RING, ML_GROUPS>(
        stages, ring, s_beg, full, empty, stage_st, &cs, &h, rg, s_ts, TS_MAX, ws, epoch);
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
      const int lastlen_t = (tile + 1 == ntiles) ? lastlen : L;
      const uint32_t run =
          mul_lanes_tile(tr, sgn, pls, &sg.outlier[TILE * ti], lastlen_t, vp, s_ge, K, sdst, pdst,
                         lim_nc, lim_r, out + HOSZP_HEADER_BYTES + tile * TILE,
                         reinterpret_cast<int*>(out + off_outlier(h.nb)) + tile * TILE, vmax, vmin,
                         ovf, tbad);
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
