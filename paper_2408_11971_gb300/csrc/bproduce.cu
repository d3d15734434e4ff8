// bproduce.cu — batched producing operators: scalar multiplication and
// element-wise addition / subtraction of every field of a batch plan (Sec. V,
// applied field by field), and compression of many float fields, each as one
// persistent launch over the fields' global tile space.
//
// Addition and compression: a warp takes whole 64-block tiles of the global
// tile space from a ticket, finds the tile's field (binary search of the field
// table), and runs the single-stream kernels' per-tile work with the field's
// own bound and plan. Scalar multiplication reads its input through the
// batched super-tile pipeline instead (stages of one field's tiles in shared
// memory). Either way:
// rates and outliers go straight to the field's output buffer, sign and plane
// words to the tile's slots in the context's staging (slot bases per field,
// the SPLIT rule of hz_ws.cuh). One scan over all tiles' word counts and one
// placement launch then complete every field's stream: each field's words go
// to its plane section (whose start needs the field's own count of
// non-constant blocks), its header gets the field's totals and largest |q|,
// and its size goes to the caller's per-field size array. No per-field launch
// and no host synchronization: a sequence of these calls can be captured in a
// CUDA graph once the context's workspace has grown to the batch's needs.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "hz_mullanes.cuh"
#include "hz_scalar.cuh"
#include "hz_kernels.cuh"
#include "batch_plan.cuh"
#include "hz_bsuper.cuh"

namespace hz {
float eps_q_host(double eps);  // api.cu
int ctx_prepare_staging(hoszp_ctx* ctx, uint64_t tiles, uint64_t staging_words, Ws* ws,
                        int* device, int* num_sms);  // api.cu
}  // namespace hz

namespace hz {
namespace {

constexpr int BP_WARPS = 16;
constexpr int BP_THREADS = BP_WARPS * 32;

// Warp-uniform ticket over the global tile space.
__device__ __forceinline__ uint64_t bp_ticket(const Ws& ws) {
  unsigned int t = 0;
  if ((threadIdx.x & 31) == 0) t = atomicAdd(&ws.sync->ticket, 1u);
  return __shfl_sync(0xffffffffu, t, 0);
}

// Index of the output field holding global tile t.
__device__ __forceinline__ uint32_t out_of_tile(const BOut* O, uint32_t nf, uint64_t t) {
  uint32_t lo = 0, hi = nf;
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (O[mid].tile0 <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// A tile's rates from global memory (only the tile's nvt blocks are read) and
// their in-tile prefixes, as tile_rates() gives them from a stage.
__device__ __forceinline__ TileRates tile_rates_g(const uint8_t* rate, int nvt) {
  const int lane = threadIdx.x & 31;
  TileRates tr;
  tr.nvt = nvt;
  tr.r0 = (2 * lane < nvt) ? min((uint32_t)rate[2 * lane], (uint32_t)MAX_RATE) : 0u;
  tr.r1 = (2 * lane + 1 < nvt) ? min((uint32_t)rate[2 * lane + 1], (uint32_t)MAX_RATE) : 0u;
  const uint32_t v0 = (tr.r0 ? 0x10000u : 0u) | tr.r0, v1 = (tr.r1 ? 0x10000u : 0u) | tr.r1;
  const uint32_t pv = v0 + v1;
  uint32_t inc = pv;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  tr.e0 = inc - pv;
  tr.e1 = tr.e0 + v0;
  return tr;
}

__device__ __forceinline__ hoszp_header header_of(const Info& h) {
  hoszp_header H;
  H.magic = HOSZP_MAGIC;
  H.version = HOSZP_VERSION;
  H.dtype = 0;
  H.ndims = (uint8_t)h.ndims;
  H.dims[0] = h.dims[0];
  H.dims[1] = h.dims[1];
  H.dims[2] = h.dims[2];
  H.eps_q = h.eps_q;
  H.n = h.n;
  H.eps = h.eps;
  H.nnc = 0;
  H.R = 0;
  H.qbound = 0;
  H.block = HOSZP_BLOCK;
  return H;
}

// ---------------------------------------------------------------- output tables
// Scalar multiplication: field f's sign slots start at the input non-constant
// blocks before it, its plane slots (after all sign slots) at e bits more per
// input non-constant block plus the input plane words before it.
__global__ void k_bout_mul(const BField* F, uint32_t nf, const unsigned long long* fpre,
                           uint32_t e_bits, uint8_t* const* outs, const uint64_t* caps, BOut* O,
                           int* status) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const BField& b = F[f];
  BOut o;
  o.out = outs[f];
  o.cap = caps[f];
  o.tile0 = b.tile0;
  o.ntiles = b.ntiles;
  o.nb = b.h.nb;
  o.sbase = fpre[2 * f];
  o.pbase = fpre[2 * nf] + fpre[2 * f] * e_bits + fpre[2 * f + 1];
  o.hdr = header_of(b.h);
  o.qmax = 0;
  o.ok = 1;
  if (!o.out || ((uintptr_t)o.out & 15u) || o.cap < off_sign(o.nb)) {
    set_status(status, HOSZP_ERR_CAPACITY);
    o.ok = 0;
  }
  O[f] = o;
}

// ---------------------------------------------------------------- scalar multiplication
// Every field times s (Sec. V-A): q' = floor(2e_f q rho_f + 1/2) with the
// field's own bound e_f and scalar bin rho_f (Eq. 3 of s at e_f), on the
// batched super-tile pipeline (hz_bsuper.cuh): a loader warp streams stages of
// up to BM_NT tiles of one field into shared memory, warp i of a group takes
// tile i of a stage, as the single-stream kernel does; a warp rebuilds its
// multiplication plan when its stage's field differs from its last one.
constexpr int BM_NT = 5;
constexpr int BM_GROUPS = 3;
constexpr int BM_NCW = BM_NT * BM_GROUPS;
constexpr int BM_THREADS = (BM_NCW + 1) * 32;
constexpr int BM_STAGES = 6;
constexpr uint32_t BM_RING = 22528;  // plane-ring words (176 KB)

__global__ void __launch_bounds__(BM_THREADS, 1) k_bmul_super(
    const BField* __restrict__ F, uint32_t nf, uint64_t T,
    const unsigned long long* __restrict__ pre, BOut* O, double s, uint32_t e_bits, Ws ws,
    int* status) {
  using St = SStageT<BM_NT>;
  extern __shared__ __align__(16) uint8_t dyn[];
  St* stages = reinterpret_cast<St*>(dyn);
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + BM_STAGES);
  __shared__ uint64_t full[BM_STAGES], empty[BM_STAGES];
  __shared__ BStageMeta s_meta[BM_STAGES];
  __shared__ MulPlan s_mp[BM_NCW];
  __shared__ uint8_t s_ge[BM_NCW][32];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const uint64_t G = gridDim.x;
  const uint64_t t_begin = T * blockIdx.x / G, t_end = T * (blockIdx.x + 1) / G;
  if (tid == 0) {
    for (int k = 0; k < BM_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], BM_NT);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int bad = 0;
  bool ovf = false;
  if (w == BM_NCW) {
    __shared__ uint32_t s_beg[BM_STAGES];
    bsuper_loader<BM_NT, BM_STAGES, BM_RING, BM_GROUPS>(stages, ring, s_beg, full, empty, s_meta,
                                                         F, nf, pre, t_begin, t_end, status);
  } else {
    const int grp = w / BM_NT, ti = w % BM_NT;
    const lanes::Shifts K = lanes::make_shifts(nf != 0 ? 1u : 0u);
    uint32_t cur = ~0u;  // the field of this warp's plan
    bool cur_ok = false;
    for (uint64_t k = 0;; k++) {
      const uint64_t u = k * BM_GROUPS + grp;  // stage use taken by this group
      const int sk = (int)(u % BM_STAGES);
      if (!mbar_wait_warp(&full[sk], (uint32_t)((u / BM_STAGES) & 1), status)) break;
      const BStageMeta meta = s_meta[sk];
      if (meta.nt == 0) break;
      const uint32_t f = meta.f;
      if (f != cur) {  // the field's scalar bin and plan, for this warp
        cur = f;
        int pbad = 0;
        if (lane == 0) {
          const Info& h = F[f].h;
          long long rho = 0;
          if (!quantize_scalar(s, h.eps_q, rho)) pbad = HOSZP_ERR_RANGE;
          s_mp[w] = mul_plan(h.eps_q, rho, h.qbound);
          const double kabs = fabs(2.0 * (double)h.eps_q * (double)rho) * (1.0 + 0x1p-40);
          for (int R = 0; R < 32; R++) s_ge[w][R] = (uint8_t)min(4, (delta_bits(kabs, R) + 8) >> 3);
        }
        __syncwarp();
        pbad = __shfl_sync(0xffffffffu, pbad, 0);
        if (pbad) {  // the scalar's bin is out of range for this field
          bad = HOSZP_ERR_RANGE;
          if (lane == 0) O[f].ok = 0;
        }
        cur_ok = !pbad;
      }
      if (ti < (int)meta.nt) {  // warp-uniform
        const uint64_t lt = meta.t0 + ti;
        const uint64_t t = F[f].tile0 + lt;
        if (!cur_ok || !*reinterpret_cast<const volatile int*>(&O[f].ok)) {
          if (lane == 0) ws.agg[t] = 0;  // the tile adds nothing to the word scan
        } else {
          const St& sg = stages[sk];
          const uint64_t fnb = F[f].h.nb, fn = F[f].h.n;
          const TileRates tr = tile_rates(sg, ti, lt, fnb);
          const uint32_t* sgn = reinterpret_cast<const uint32_t*>(sg.sign + sg.sbase + sg.tnc[ti]);
          const uint32_t* pls =
              reinterpret_cast<const uint32_t*>(ring + sg.pring + sg.pbase + sg.tr[ti]);
          // slots of the tile: upper bounds of the field's output words before it
          const uint64_t pnc = sg.bnc + sg.tnc[ti], pr = sg.br + sg.tr[ti];
          const uint64_t so = O[f].sbase + pnc, po = O[f].pbase + pnc * e_bits + pr;
          const uint32_t tin =
              (tr.nvt > 0) ? __shfl_sync(0xffffffffu, tr.e1 + (tr.r1 ? 0x10000u : 0u) + tr.r1, 31) : 0u;
          const uint32_t lim_nc = tin >> 16, lim_r = (tin >> 16) * e_bits + (tin & 0xffffu);
          int tbad = 0;
          if (so + lim_nc > ws.staging_words || po + lim_r > ws.staging_words)
            tbad = HOSZP_ERR_CAPACITY;
          uint8_t* const out = O[f].out;
          int vmax = 0, vmin = 0;
          const int lastlen = (lt + 1 == F[f].ntiles) ? (int)(fn - (fnb - 1) * L) : L;
          const uint32_t run = mul_lanes_tile(
              tr, sgn, pls, &sg.outlier[TILE * ti], lastlen, &s_mp[w], s_ge[w], K,
              reinterpret_cast<uint32_t*>(ws.staging + so),
              reinterpret_cast<uint32_t*>(ws.staging + po), lim_nc, lim_r,
              out + HOSZP_HEADER_BYTES + lt * TILE,
              reinterpret_cast<int*>(out + off_outlier(fnb)) + lt * TILE, vmax, vmin, ovf, tbad);
          if (tbad) bad = tbad;
          uint32_t qm = max((uint32_t)vmax, (uint32_t)(-(long long)vmin));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) qm = max(qm, __shfl_xor_sync(0xffffffffu, qm, o));
          if (lane == 0) {
            atomicMax(&O[f].qmax, qm);
            ws.agg[t] = ((unsigned long long)(run >> 16) << 32) | (run & 0xffffu);
            ws.pre[0][2 * t] = so;
            ws.pre[0][2 * t + 1] = po;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sk]);
    }
  }
  if (ovf) bad = HOSZP_ERR_OVERFLOW;
  if (bad) set_status(status, bad);
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

// ---------------------------------------------------------------- element-wise addition
// Field f's output is A_f + B_f (or A_f - B_f): the bit-sliced addition of the
// single-stream kernel (two's-complement planes of both inputs, a full adder
// per plane, back to sign and magnitude; Sec. V-C), one 32-position half of a
// block per lane. Slots: a block of the sum has a sign word only where A or B
// has one, and at most max(rate_A, rate_B) + 1 planes.
__global__ void k_bout_add(const BField* FA, const BField* FB, uint32_t nf,
                           const unsigned long long* fpa, const unsigned long long* fpb,
                           uint8_t* const* outs, const uint64_t* caps, BOut* O, int* status) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const BField& a = FA[f];
  const BField& b = FB[f];
  BOut o;
  o.out = outs[f];
  o.cap = caps[f];
  o.tile0 = a.tile0;
  o.ntiles = a.ntiles;
  o.nb = a.h.nb;
  const uint64_t SC = fpa[2 * nf] + fpb[2 * nf];
  o.sbase = fpa[2 * f] + fpb[2 * f];
  o.pbase = SC + fpa[2 * f] + fpb[2 * f] + fpa[2 * f + 1] + fpb[2 * f + 1];
  o.hdr = header_of(a.h);
  o.qmax = a.h.qbound + b.h.qbound;  // the sum's bound: the inputs' bounds added
  o.ok = 1;
  int bad = 0;
  if (a.h.n != b.h.n || a.tile0 != b.tile0 ||
      __float_as_uint(a.h.eps_q) != __float_as_uint(b.h.eps_q))
    bad = HOSZP_ERR_MISMATCH;
  else if ((long long)a.h.qbound + (long long)b.h.qbound > HOSZP_QLIM)
    bad = HOSZP_ERR_OVERFLOW;
  else if (!o.out || ((uintptr_t)o.out & 15u) || o.cap < off_sign(o.nb))
    bad = HOSZP_ERR_CAPACITY;
  if (bad) {
    set_status(status, bad);
    o.ok = 0;
  }
  O[f] = o;
}

template <bool SUB>
__global__ void __launch_bounds__(BP_THREADS, 1) k_badd(
    const BField* __restrict__ FA, const BField* __restrict__ FB, uint32_t nf, uint64_t T,
    const unsigned long long* __restrict__ prea, const unsigned long long* __restrict__ preb,
    BOut* O, Ws ws, int* status) {
  const int lane = threadIdx.x & 31, hf = lane & 1, m = lane >> 1;
  int bad = 0;
  for (;;) {
    const uint64_t t = bp_ticket(ws);
    if (t >= T) break;
    const uint32_t f = out_of_tile(O, nf, t);
    if (!O[f].ok) {
      if (lane == 0) ws.agg[t] = 0;
      continue;
    }
    const BField* fa = &FA[f];
    const BField* fb = &FB[f];
    const Info ha = fa->h, hb = fb->h;
    const uint64_t lt = t - fa->tile0;
    const int nvt = (int)umin64(TILE, ha.nb - lt * TILE);
    const uint8_t* ca = fa->c;
    const uint8_t* cb = fb->c;
    const TileRates tra = tile_rates_g(ca + HOSZP_HEADER_BYTES + lt * TILE, nvt);
    const TileRates trb = tile_rates_g(cb + HOSZP_HEADER_BYTES + lt * TILE, nvt);
    const unsigned long long ancA = prea[fa->pre0 + 2 * lt], arA = prea[fa->pre0 + 2 * lt + 1];
    const unsigned long long ancB = preb[fb->pre0 + 2 * lt], arB = preb[fb->pre0 + 2 * lt + 1];
    const uint32_t* sgA = reinterpret_cast<const uint32_t*>(ca + ha.o_sign + 8 * ancA);
    const uint32_t* plA = reinterpret_cast<const uint32_t*>(ca + ha.o_plane + 8 * arA);
    const uint32_t* sgB = reinterpret_cast<const uint32_t*>(cb + hb.o_sign + 8 * ancB);
    const uint32_t* plB = reinterpret_cast<const uint32_t*>(cb + hb.o_plane + 8 * arB);
    const int* oA = reinterpret_cast<const int*>(ca + ha.o_out) + lt * TILE;
    const int* oB = reinterpret_cast<const int*>(cb + hb.o_out) + lt * TILE;
    uint8_t* const out = O[f].out;
    const uint64_t so = O[f].sbase + ancA + ancB, po = O[f].pbase + ancA + ancB + arA + arB;
    const uint32_t tA = __shfl_sync(0xffffffffu, tra.e1 + (tra.r1 ? 0x10000u : 0u) + tra.r1, 31);
    const uint32_t tB = __shfl_sync(0xffffffffu, trb.e1 + (trb.r1 ? 0x10000u : 0u) + trb.r1, 31);
    const uint32_t lim_nc = (tA >> 16) + (tB >> 16);
    const uint32_t lim_r = lim_nc + (tA & 0xffffu) + (tB & 0xffffu);
    int tbad = 0;
    if (so + lim_nc > ws.staging_words || po + lim_r > ws.staging_words) tbad = HOSZP_ERR_CAPACITY;
    uint32_t* sdst = reinterpret_cast<uint32_t*>(ws.staging + so);
    uint32_t* pdst = reinterpret_cast<uint32_t*>(ws.staging + po);
    uint32_t run = 0;
    const int steps = (nvt + 15) >> 4;
    for (int it = 0; it < steps; it++) {
      const int b = 16 * it + m;
      uint32_t ra, exa, rb, exb;
      tile_block(tra, b, ra, exa);
      tile_block(trb, b, rb, exb);
      const bool valid = b < nvt;
      const uint32_t* pa = plA + 2 * (exa & 0xffffu) + hf;
      const uint32_t* pb = plB + 2 * (exb & 0xffffu) + hf;
      const uint32_t siga = ra ? sgA[2 * (exa >> 16) + hf] : 0u;
      uint32_t sigb = rb ? sgB[2 * (exb >> 16) + hf] : 0u;
      if (SUB) sigb = ~sigb;  // negation flips every sign bit (a zero stays zero)
      const int mr = max((int)ra, (int)rb);
      // planes 0 .. P of the two's-complement sum, P = the warp's largest m + 1
      const int P = (int)__reduce_max_sync(0xffffffffu, (unsigned)(mr > 0 ? mr + 1 : 0));
      uint32_t z[MAX_RATE + 2];
      uint32_t sgn = 0u, nzp = 0u;
      if (P > 0) {
        uint32_t cA = siga, cB = sigb, cz = 0u;
#pragma unroll
        for (int p = 0; p <= MAX_RATE + 1; p++) {
          if (p > P) break;
          const uint32_t xa = (p < (int)ra ? pa[2 * p] : 0u) ^ siga;
          const uint32_t xb = (p < (int)rb ? pb[2 * p] : 0u) ^ sigb;
          const uint32_t x = xa ^ cA, y = xb ^ cB;
          cA &= xa;
          cB &= xb;
          z[p] = x ^ y ^ cz;
          cz = (x & y) | (cz & (x ^ y));
          sgn = z[p];  // the last plane computed, P, is the sign
        }
        uint32_t cu = sgn;  // back to sign and magnitude over planes 0 .. P-1
#pragma unroll
        for (int p = 0; p <= MAX_RATE; p++) {
          if (p >= P) break;
          const uint32_t tt = z[p] ^ sgn;
          const uint32_t mg = tt ^ cu;
          cu &= tt;
          z[p] = mg;
          nzp |= (mg != 0u ? 1u : 0u) << p;
        }
      }
      nzp |= __shfl_xor_sync(0xffffffffu, nzp, 1);
      int rate = valid ? 32 - __clz(nzp) : 0;
      if (rate > MAX_RATE) {  // only a header whose qbound understates its values gets here
        tbad = HOSZP_ERR_OVERFLOW;
        rate = MAX_RATE;
      }
      // the tile-local exclusive prefix (sign words << 16 | plane words)
      const uint32_t pk = (hf == 0 && rate > 0) ? ((1u << 16) | (uint32_t)rate) : 0u;
      uint32_t inc = pk;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const uint32_t ex = __shfl_sync(0xffffffffu, inc - pk, lane & ~1);
      const uint32_t step = __shfl_sync(0xffffffffu, inc, 31);
      const uint32_t nc0 = (run >> 16) + (ex >> 16), r0 = (run & 0xffffu) + (ex & 0xffffu);
      run += step;
      if (tbad == 0 && rate > 0 && (nc0 >= lim_nc || r0 + (uint32_t)rate > lim_r))
        tbad = HOSZP_ERR_CAPACITY;
      if (tbad == 0 && rate > 0) {
        sdst[2 * nc0 + hf] = sgn;
        uint32_t* dst = pdst + 2 * r0 + hf;
#pragma unroll
        for (int p = 0; p <= MAX_RATE; p++) {
          if (p >= P) break;
          if (p < rate) dst[2 * p] = z[p];
        }
      }
      if (valid && hf == 0) {
        out[HOSZP_HEADER_BYTES + lt * TILE + b] = (uint8_t)rate;
        reinterpret_cast<int*>(out + off_outlier(ha.nb))[lt * TILE + b] = SUB ? oA[b] - oB[b]
                                                                             : oA[b] + oB[b];
      }
    }
    if (tbad) bad = tbad;
    if (lane == 0) {
      ws.agg[t] = ((unsigned long long)(run >> 16) << 32) | (run & 0xffffu);
      ws.pre[0][2 * t] = so;
      ws.pre[0][2 * t + 1] = po;
    }
  }
  if (bad) set_status(status, bad);
  if (launch_end_is_last(ws) && threadIdx.x == 0) launch_reset(ws);
}

// ---------------------------------------------------------------- compression
// Many float fields, each with its own bound, compressed in one launch: the
// two-lanes compression of the single-stream kernel (exact Eq. 3, Lorenzo,
// register encode) with the tile's field looked up per tile. With relative
// bounds a range pass over all fields' values (chunks of 2^16 values from a
// ticket, per-field extremes kept as order-preserving integers) and a finish
// per field give each field's eps and eps_q exactly as the single-stream range
// pass does. A field's tiles get fixed slots (64 sign words and 64 x 24 plane
// words per tile: the compressor keeps every rate at or below 24).
struct CField {
  const float* x;
  uint8_t* out;
  uint64_t cap;
  uint64_t n;
  uint64_t tile0, chunk0;
  double eb;        // the requested bound (absolute) or the relative factor
  float eps_q;      // the quantizer's bound (set on the host, or by the range finish)
  double eps;       // the header's bound
  unsigned int mn, mx, nonfinite;  // range pass: extremes as ordered integers
};
constexpr uint64_t BC_CHUNK = 1u << 16;

__device__ __forceinline__ unsigned int float_order(float v) {
  const unsigned int u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float order_float(unsigned int o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ uint32_t cfield_of(const CField* C, uint32_t nf, uint64_t key,
                                              bool by_chunk) {
  uint32_t lo = 0, hi = nf;
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if ((by_chunk ? C[mid].chunk0 : C[mid].tile0) <= key) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(512) k_bcmp_range(CField* C, uint32_t nf, uint64_t nchunks,
                                                    Ws ws) {
  __shared__ unsigned int s_k;
  __shared__ unsigned int s_mn[16], s_mx[16], s_nf[16];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (;;) {
    if (tid == 0) s_k = atomicAdd(&ws.sync->ticket, 1u);
    __syncthreads();
    const uint64_t k = s_k;
    __syncthreads();
    if (k >= nchunks) break;
    const uint32_t f = cfield_of(C, nf, k, true);
    const float* x = C[f].x;
    const uint64_t n = C[f].n;
    const uint64_t i0 = (k - C[f].chunk0) * BC_CHUNK, i1 = umin64(n, i0 + BC_CHUNK);
    unsigned int mn = 0xffffffffu, mx = 0u, bad = 0u;
    for (uint64_t i = i0 + tid; i < i1; i += blockDim.x) {
      const float v = __ldg(x + i);
      if (!(fabsf(v) <= FLT_MAX)) bad = 1u;
      const unsigned int o = float_order(v);
      mn = min(mn, o);
      mx = max(mx, o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
      s_mn[w] = mn;
      s_mx[w] = mx;
      s_nf[w] = bad;
    }
    __syncthreads();
    if (tid == 0) {
      for (int j = 1; j < (int)(blockDim.x >> 5); j++) {
        mn = min(mn, s_mn[j]);
        mx = max(mx, s_mx[j]);
        bad |= s_nf[j];
      }
      atomicMin(&C[f].mn, mn);
      atomicMax(&C[f].mx, mx);
      if (bad) atomicOr(&C[f].nonfinite, 1u);
    }
  }
  if (launch_end_is_last(ws) && tid == 0) launch_reset(ws);
}

// eps = rel (max - min) in double (a constant field uses |max|, an empty or
// zero one 1), eps_q = the largest float not above eps; NaN or Inf in the
// field is NONFINITE, an eps_q outside the normal range RANGE.
__global__ void k_bcmp_finish(CField* C, uint32_t nf, int* status) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  CField& c = C[f];
  if (c.nonfinite) {
    set_status(status, HOSZP_ERR_NONFINITE);
    c.eps_q = 0.0f;
    return;
  }
  const float gmn = order_float(c.mn), gmx = order_float(c.mx);
  double range = (c.n > 0) ? (double)gmx - (double)gmn : 0.0;
  if (range == 0.0) range = (c.n > 0 && gmx != 0.0f) ? fabs((double)gmx) : 1.0;
  const double eps = c.eb * range;
  float q = __double2float_rn(eps);
  if ((double)q > eps) q = nextafterf(q, 0.0f);
  if (!(q >= FLT_MIN && q <= FLT_MAX / 2)) {
    set_status(status, HOSZP_ERR_RANGE);
    q = 0.0f;
  }
  c.eps_q = q;
  c.eps = eps;
}

__global__ void k_bout_cmp(const CField* C, uint32_t nf, uint64_t T, BOut* O, int* status) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const CField& c = C[f];
  BOut o;
  o.out = c.out;
  o.cap = c.cap;
  o.tile0 = c.tile0;
  o.nb = nblocks(c.n);
  o.ntiles = ntiles_of(o.nb);
  o.sbase = (uint64_t)TILE * c.tile0;
  o.pbase = (uint64_t)TILE * T + (uint64_t)TILE * 24 * c.tile0;
  Info h{};
  h.ndims = 1;
  h.dims[0] = (uint32_t)c.n;
  h.eps_q = c.eps_q;
  h.n = c.n;
  h.eps = c.eps;
  o.hdr = header_of(h);
  o.qmax = 0;
  o.ok = c.eps_q >= FLT_MIN ? 1 : 0;  // a failed range pass has set its error
  if (o.ok && (!o.out || ((uintptr_t)o.out & 15u) || o.cap < off_sign(o.nb))) {
    set_status(status, HOSZP_ERR_CAPACITY);
    o.ok = 0;
  }
  O[f] = o;
}

__global__ void __launch_bounds__(BP_THREADS, 1) k_bcompress(const CField* __restrict__ C,
                                                           uint32_t nf, uint64_t T, BOut* O,
                                                           Ws ws, int* status) {
  const int lane = threadIdx.x & 31, hf = lane & 1, m = lane >> 1;
  const lanes::Shifts K = lanes::make_shifts(nf != 0 ? 1u : 0u);
  int bad = 0;
  for (;;) {
    const uint64_t t = bp_ticket(ws);
    if (t >= T) break;
    const uint32_t f = cfield_of(C, nf, t, false);
    if (!O[f].ok) {
      if (lane == 0) ws.agg[t] = 0;
      continue;
    }
    const float* x = C[f].x;
    const uint64_t n = C[f].n, nb = nblocks(n);
    const uint64_t lt = t - C[f].tile0;
    Quant Q;
    Q.e = C[f].eps_q;
    Q.e2 = 2.0f * Q.e;
    Q.r = __double2float_rn(1.0 / (double)Q.e2);
    const int nvt = (int)umin64(TILE, nb - lt * TILE);
    uint8_t* const out = O[f].out;
    const uint64_t so = (uint64_t)TILE * t, po = (uint64_t)TILE * T + (uint64_t)TILE * 24 * t;
    uint32_t* sdst = reinterpret_cast<uint32_t*>(ws.staging + so);
    uint32_t* pdst = reinterpret_cast<uint32_t*>(ws.staging + po);
    uint32_t run = 0;
    int tbad = 0, qhi = 0, qlo = 0, qbad = 0;
    const int steps = (nvt + 15) >> 4;
    for (int it = 0; it < steps; it++) {
      const int b = 16 * it + m;
      const bool valid = b < nvt;
      const uint64_t bi = lt * TILE + b;
      const uint64_t i0 = bi * L + 32 * hf;
      const int nval = (valid && i0 < n) ? (int)umin64(32, n - i0) : 0;
      const bool fullblk = __all_sync(0xffffffffu, nval == 32);
      int q[32];
      {
        float fv[32];
        if (fullblk && ((uintptr_t)x & 15u) == 0) {
          const float4* x4 = reinterpret_cast<const float4*>(x + i0);
#pragma unroll
          for (int k = 0; k < 8; k++) {
            const float4 a = __ldg(x4 + k);
            fv[4 * k] = a.x;
            fv[4 * k + 1] = a.y;
            fv[4 * k + 2] = a.z;
            fv[4 * k + 3] = a.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; i++) fv[i] = (i < nval) ? __ldg(x + i0 + i) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) quantize8(fv + 8 * k, Q, q + 8 * k, qbad);
      }
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        qhi = __vimax3_s32(qhi, q[i], q[i + 1]);
        qlo = __vimin3_s32(qlo, q[i], q[i + 1]);
      }
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
      int dhi = 0, dlo = 0;
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        dhi = __vimax3_s32(dhi, q[i], q[i + 1]);
        dlo = __vimin3_s32(dlo, q[i], q[i + 1]);
      }
      const uint32_t dm = __reduce_or_sync(0xffffffffu, (uint32_t)max(dhi, -dlo));
      const int Ge = min(4, (40 - __clz(dm)) >> 3);
      int sbad = __any_sync(0xffffffffu, qbad != 0) ? HOSZP_ERR_RANGE : tbad;
      const int rate = encode_store_any(Ge, q, K, valid, sdst, pdst, TILE, TILE * 24, run, sbad);
      if (sbad == HOSZP_ERR_CAPACITY) tbad = sbad;
      if (valid && hf == 0) {
        out[HOSZP_HEADER_BYTES + bi] = (uint8_t)rate;
        reinterpret_cast<int*>(out + off_outlier(nb))[bi] = o_new;
      }
    }
    if (qbad) bad = qbad;
    if (tbad) bad = tbad;
    uint32_t qm = max((uint32_t)qhi, (uint32_t)(-(long long)qlo));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qm = max(qm, __shfl_xor_sync(0xffffffffu, qm, o));
    if (lane == 0) {
      atomicMax(&O[f].qmax, qm);
      ws.agg[t] = ((unsigned long long)(run >> 16) << 32) | (run & 0xffffu);
      ws.pre[0][2 * t] = so;
      ws.pre[0][2 * t + 1] = po;
    }
  }
  if (bad) set_status(status, bad);
  if (launch_end_is_last(ws) && threadIdx.x == 0) launch_reset(ws);
}

// ---------------------------------------------------------------- placement
// One warp per global tile moves the tile's sign and plane words from its
// slots to its field's stream; one thread per field then writes the field's
// header (its totals from the tile scan, its largest |q'|), the padding and
// its size (0 for a field that failed).
__global__ void __launch_bounds__(512) k_bplace(BOut* O, uint32_t nf, uint64_t T, Ws ws,
                                                uint64_t* out_bytes, int* status) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  int bad = 0;
  for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < T;
       t += nwarps) {
    const uint32_t f = out_of_tile(O, nf, t);
    const BOut& o = O[f];
    if (!o.ok) continue;
    const uint64_t f0 = o.tile0, f1 = o.tile0 + o.ntiles;
    const uint64_t nnc = ws.opre[2 * f1] - ws.opre[2 * f0], R = ws.opre[2 * f1 + 1] - ws.opre[2 * f0 + 1];
    if (stream_bytes(o.nb, nnc, R) > o.cap) continue;  // the field's thread reports it
    const unsigned long long a = ws.agg[t];
    const uint64_t nc = a >> 32, r = a & 0xffffffffull;
    const uint64_t NC = ws.opre[2 * t] - ws.opre[2 * f0], RR = ws.opre[2 * t + 1] - ws.opre[2 * f0 + 1];
    const uint64_t so = ws.pre[0][2 * t], po = ws.pre[0][2 * t + 1];
    if (so + nc > ws.staging_words || po + r > ws.staging_words || NC + nc > nnc || RR + r > R) {
      bad = HOSZP_ERR_CAPACITY;
      continue;
    }
    uint64_t* sdst = reinterpret_cast<uint64_t*>(o.out + off_sign(o.nb)) + NC;
    uint64_t* pdst = reinterpret_cast<uint64_t*>(o.out + off_plane(o.nb, nnc)) + RR;
    for (uint64_t i = lane; i < nc; i += 32) sdst[i] = __ldcs(ws.staging + so + i);
    for (uint64_t i = lane; i < r; i += 32) pdst[i] = __ldcs(ws.staging + po + i);
  }
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf;
       f += (uint64_t)gridDim.x * blockDim.x) {
    BOut& o = O[f];
    const uint64_t f0 = o.tile0, f1 = o.tile0 + o.ntiles;
    const uint64_t nnc = ws.opre[2 * f1] - ws.opre[2 * f0], R = ws.opre[2 * f1 + 1] - ws.opre[2 * f0 + 1];
    const uint64_t size = stream_bytes(o.nb, nnc, R);
    if (!o.ok || size > o.cap) {
      if (o.ok) bad = HOSZP_ERR_CAPACITY;
      out_bytes[f] = 0;
      o.qmax = 0;
      continue;
    }
    hoszp_header H = o.hdr;
    H.nnc = nnc;
    H.R = R;
    H.qbound = o.qmax;
    o.qmax = 0;
    uint8_t* out = o.out;
    *reinterpret_cast<hoszp_header*>(out) = H;
    for (uint64_t b = HOSZP_HEADER_BYTES + o.nb; b < off_outlier(o.nb); b++) out[b] = 0;
    for (uint64_t b = off_outlier(o.nb) + 4 * o.nb; b < off_sign(o.nb); b++) out[b] = 0;
    for (uint64_t b = off_plane(o.nb, nnc) + 8 * R; b < size; b++) out[b] = 0;
    out_bytes[f] = size;
  }
  if (bad) set_status(status, bad);
  if (launch_end_is_last(ws) && threadIdx.x == 0) {
    ws.totals[0] = 0;
    ws.totals[1] = 0;
    ws.totals[2] = 0;
    launch_reset(ws);
  }
}

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" int hoszp_batch_mul_scalar(hoszp_batch* b, double s, void* const* d_outs,
                                      const uint64_t* d_caps, uint64_t* d_out_bytes,
                                      hoszp_stream_t stream) {
  if (!b || !d_outs || !d_caps || !d_out_bytes || !(s == s) || s - s != 0.0) return HOSZP_ERR_ARG;
  if (((uintptr_t)d_outs & 7u) || ((uintptr_t)d_caps & 7u) || ((uintptr_t)d_out_bytes & 7u))
    return HOSZP_ERR_ARG;
  DeviceGuard guard(b->device);
  // e bounds the growth of a block's rate (as for one stream): |2e rho| <= 2|s|
  const uint32_t e_bits =
      std::min(31u, (uint32_t)std::ceil(std::log2(2.0 * std::fabs(s) + 1.0)) + 1u);
  const uint64_t T = b->total_tiles;
  const uint64_t words = b->total_nnc * (1ull + e_bits) + b->total_R + 64;
  Ws ws;
  int device = 0, sms = 0;
  int rc = ctx_prepare_staging(b->ctx, T + 1, words, &ws, &device, &sms);
  if (rc) return rc;
  const cudaStream_t cs = (cudaStream_t)stream;
  k_bout_mul<<<(b->nf + 127) / 128, 128, 0, cs>>>(b->d_fields, b->nf, b->d_fpre, e_bits,
                                                  (uint8_t* const*)d_outs, d_caps, b->d_out,
                                                  b->status);
  {
    const size_t smem = BM_STAGES * sizeof(SStageT<BM_NT>) + BM_RING * sizeof(uint64_t);
    smem_attr<k_bmul_super>(smem);
    k_bmul_super<<<persistent_grid(k_bmul_super, BM_THREADS, sms, smem), BM_THREADS, smem, cs>>>(
        b->d_fields, b->nf, T, b->d_pre, b->d_out, s, e_bits, ws, b->status);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rc_of(e);
  Launch lc;
  lc.grid = sms;
  lc.stream = cs;
  e = launch_scan_agg(lc, ws, T);
  if (e != cudaSuccess) return rc_of(e);
  k_bplace<<<sms * 2, 512, 0, cs>>>(b->d_out, b->nf, T, ws, d_out_bytes, b->status);
  return rc_of(cudaGetLastError());
}

extern "C" int hoszp_batch_add(hoszp_batch* a, hoszp_batch* b, int subtract, void* const* d_outs,
                               const uint64_t* d_caps, uint64_t* d_out_bytes,
                               hoszp_stream_t stream) {
  if (!a || !b || !d_outs || !d_caps || !d_out_bytes) return HOSZP_ERR_ARG;
  if (((uintptr_t)d_outs & 7u) || ((uintptr_t)d_caps & 7u) || ((uintptr_t)d_out_bytes & 7u))
    return HOSZP_ERR_ARG;
  // the plans' shapes must agree field by field (checked again on the device)
  if (a->nf != b->nf || a->total_tiles != b->total_tiles || a->device != b->device)
    return HOSZP_ERR_MISMATCH;
  DeviceGuard guard(a->device);
  const uint64_t T = a->total_tiles;
  const uint64_t SC = a->total_nnc + b->total_nnc;
  const uint64_t words = SC + SC + a->total_R + b->total_R + 64;
  Ws ws;
  int device = 0, sms = 0;
  int rc = ctx_prepare_staging(a->ctx, T + 1, words, &ws, &device, &sms);
  if (rc) return rc;
  const cudaStream_t cs = (cudaStream_t)stream;
  k_bout_add<<<(a->nf + 127) / 128, 128, 0, cs>>>(a->d_fields, b->d_fields, a->nf, a->d_fpre,
                                                  b->d_fpre, (uint8_t* const*)d_outs, d_caps,
                                                  a->d_out, a->status);
  if (subtract)
    k_badd<true><<<sms, BP_THREADS, 0, cs>>>(a->d_fields, b->d_fields, a->nf, T, a->d_pre,
                                             b->d_pre, a->d_out, ws, a->status);
  else
    k_badd<false><<<sms, BP_THREADS, 0, cs>>>(a->d_fields, b->d_fields, a->nf, T, a->d_pre,
                                              b->d_pre, a->d_out, ws, a->status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rc_of(e);
  Launch lc;
  lc.grid = sms;
  lc.stream = cs;
  e = launch_scan_agg(lc, ws, T);
  if (e != cudaSuccess) return rc_of(e);
  k_bplace<<<sms * 2, 512, 0, cs>>>(a->d_out, a->nf, T, ws, d_out_bytes, a->status);
  return rc_of(cudaGetLastError());
}

extern "C" int hoszp_batch_compress(hoszp_ctx* ctx, uint32_t nfields, const float* const* d_x,
                                    const uint64_t* n, const double* eb, int eb_mode,
                                    void* const* d_outs, const size_t* caps,
                                    uint64_t* d_out_bytes, hoszp_stream_t stream) {
  if (!ctx || nfields == 0 || !d_x || !n || !eb || !d_outs || !caps || !d_out_bytes)
    return HOSZP_ERR_ARG;
  if ((eb_mode != HOSZP_EB_ABS && eb_mode != HOSZP_EB_REL) || ((uintptr_t)d_out_bytes & 7u))
    return HOSZP_ERR_ARG;
  std::vector<CField> C(nfields);
  uint64_t T = 0, chunks = 0;
  for (uint32_t f = 0; f < nfields; f++) {
    if (!d_x[f] || ((uintptr_t)d_x[f] & 3u) || n[f] == 0 || n[f] > (1ull << 40) || !d_outs[f] ||
        ((uintptr_t)d_outs[f] & 15u) || !(eb[f] > 0) || !std::isfinite(eb[f]) ||
        n[f] > 0xffffffffull)
      return HOSZP_ERR_ARG;
    CField c{};
    c.x = d_x[f];
    c.out = (uint8_t*)d_outs[f];
    c.cap = caps[f];
    c.n = n[f];
    c.tile0 = T;
    c.chunk0 = chunks;
    c.eb = eb[f];
    c.mn = 0xffffffffu;
    c.mx = 0u;
    if (eb_mode == HOSZP_EB_ABS) {
      c.eps_q = eps_q_host(eb[f]);
      c.eps = eb[f];
      if (c.eps_q == 0.0f) return HOSZP_ERR_ARG;
    }
    C[f] = c;
    T += ntiles_of(nblocks(n[f]));
    chunks += (n[f] + BC_CHUNK - 1) / BC_CHUNK;
  }
  // workspace: slots (64 + 64 x 24 words per tile), then the field and output tables
  const uint64_t slot_words = (uint64_t)TILE * 25 * T;
  const uint64_t cwords = (nfields * sizeof(CField) + 255) / 256 * 32;
  const uint64_t owords = (nfields * sizeof(BOut) + 255) / 256 * 32;
  Ws ws;
  int device = 0, sms = 0;
  int rc = ctx_prepare_staging(ctx, T + 1, slot_words + cwords + owords + 32, &ws, &device, &sms);
  if (rc) return rc;
  DeviceGuard guard2(device);
  const uint64_t ctab = (slot_words + 31) / 32 * 32;  // 256-byte aligned
  CField* d_C = reinterpret_cast<CField*>(ws.staging + ctab);
  BOut* d_O = reinterpret_cast<BOut*>(ws.staging + ctab + cwords);
  const cudaStream_t cs = (cudaStream_t)stream;
  // pageable source: the call returns once the table is staged for the copy
  cudaError_t e = cudaMemcpyAsync(d_C, C.data(), nfields * sizeof(CField), cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return rc_of(e);
  if (eb_mode == HOSZP_EB_REL) {
    k_bcmp_range<<<sms * 2, 512, 0, cs>>>(d_C, nfields, chunks, ws);
    k_bcmp_finish<<<(nfields + 127) / 128, 128, 0, cs>>>(d_C, nfields, ws.status);
  }
  k_bout_cmp<<<(nfields + 127) / 128, 128, 0, cs>>>(d_C, nfields, T, d_O, ws.status);
  k_bcompress<<<sms, BP_THREADS, 0, cs>>>(d_C, nfields, T, d_O, ws, ws.status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rc_of(e);
  Launch lc;
  lc.grid = sms;
  lc.stream = cs;
  e = launch_scan_agg(lc, ws, T);
  if (e != cudaSuccess) return rc_of(e);
  k_bplace<<<sms * 2, 512, 0, cs>>>(d_O, nfields, T, ws, d_out_bytes, ws.status);
  return rc_of(cudaGetLastError());
}
