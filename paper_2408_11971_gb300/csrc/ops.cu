// ops.cu — homomorphic operators on compressed streams (Sec. V, Table 2):
//   negation and scalar addition in fully compressed space (workflow 1),
//   scalar multiplication through the quantized integers (workflow 3),
//   element-wise addition through the decoded deltas (workflow 2).
#include "hz_mul.cuh"
#include "hz_scalar.cuh"
#include "hz_super.cuh"
#include "hz_var.cuh"
#include "hz_ws.cuh"
#include "hz_kernels.cuh"

namespace hz {

// ---------------------------------------------------------------- workflow 1
// Stream copy (out of place) with every outlier transformed (negated or
// shifted by rho) and, for negation, every sign word inverted.
template <bool NEG>
__global__ void __launch_bounds__(512) k_meta(const uint8_t* c, uint64_t c_bytes, double s,
                                              int sub, uint8_t* out, uint64_t cap,
                                              uint64_t* out_bytes, Ws ws) {
  const Info h = parse_header(c, c_bytes);
  __shared__ int s_ok;
  __shared__ long long s_rho;
  if (threadIdx.x == 0) {
    int ok = h.ok;
    long long rho = 0;
    if (!h.ok) {
      if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_FORMAT);
    } else if (h.size > cap) {
      ok = 0;
      if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_CAPACITY);
    } else if (!NEG) {
      if (!quantize_scalar(s, h.eps_q, rho)) {
        ok = 0;
        if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_RANGE);
      } else {
        if (sub) rho = -rho;  // scalar subtraction: O' = O - rho_s
        if ((long long)h.qbound + (rho < 0 ? -rho : rho) > HOSZP_QLIM) {
          ok = 0;
          if (blockIdx.x == 0) set_status(ws.status, HOSZP_ERR_OVERFLOW);
        }
      }
    }
    s_ok = ok;
    s_rho = rho;
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  const long long rho = s_rho;
  if (ok) {
    // The stream after the header as 16-byte chunks (every section starts on
    // a 16-byte boundary except the plane section, which starts on 8): each
    // thread loads 4 chunks before it transforms and stores them, so enough
    // bytes are in flight to keep HBM busy. In place, only the outlier and
    // (negation) sign chunks are touched.
    const bool inplace = (out == c);
    const uint64_t b_lo = inplace ? h.o_out : HOSZP_HEADER_BYTES;
    const uint64_t b_hi = inplace ? (NEG ? align16(h.o_plane) : h.o_sign) : h.size;
    const uint64_t nch = (b_hi - b_lo) / 16;
    const uint4* src = reinterpret_cast<const uint4*>(c + b_lo);
    uint4* dst = reinterpret_cast<uint4*>(out + b_lo);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int r32 = (int)rho;  // |outlier| + |rho| <= HOSZP_QLIM: 32-bit arithmetic is exact
    constexpr int U = 4;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nch;
         i0 += U * stride) {
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; u++)
        if (i0 + u * stride < nch) v[u] = __ldcs(src + i0 + u * stride);
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint64_t i = i0 + u * stride;
        if (i >= nch) break;
        const uint64_t b = b_lo + 16 * i;
        if (b >= h.o_out && b < h.o_sign) {  // 4 outliers (padding past nb unchanged)
          const uint64_t k0 = (b - h.o_out) >> 2;
          uint32_t* w = reinterpret_cast<uint32_t*>(&v[u]);
#pragma unroll
          for (int k = 0; k < 4; k++)
            if (k0 + k < h.nb) w[k] = NEG ? (uint32_t)(-(int)w[k]) : (uint32_t)((int)w[k] + r32);
        } else if (NEG && b >= h.o_sign && b < h.o_plane) {  // sign words (the 2nd may be a plane)
          v[u].x = ~v[u].x;
          v[u].y = ~v[u].y;
          if (b + 8 < h.o_plane) {
            v[u].z = ~v[u].z;
            v[u].w = ~v[u].w;
          }
        }
        __stcs(dst + i, v[u]);
      }
    }
  }
  // the header is written by the CTA that finishes last: in place, every other
  // CTA has parsed the input header by then
  if (launch_end_is_last(ws) && threadIdx.x == 0) {
    if (ok) {
      hoszp_header H = *reinterpret_cast<const hoszp_header*>(c);
      if (!NEG) H.qbound = (uint32_t)((long long)H.qbound + (rho < 0 ? -rho : rho));
      *reinterpret_cast<hoszp_header*>(out) = H;
      *out_bytes = h.size;
    } else {
      *out_bytes = 0;
    }
    launch_reset(ws);
  }
}

cudaError_t launch_negate(const Launch& lc, const uint8_t* c, uint64_t c_bytes, uint8_t* out,
                          uint64_t cap, uint64_t* out_bytes, Ws ws) {
  k_meta<true><<<persistent_grid(k_meta<true>, 512, lc.grid), 512, 0, lc.stream>>>(c, c_bytes, 0.0, 0, out, cap, out_bytes, ws);
  return cudaGetLastError();
}

cudaError_t launch_add_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws) {
  k_meta<false><<<persistent_grid(k_meta<false>, 512, lc.grid), 512, 0, lc.stream>>>(c, c_bytes, s, 0, out, cap, out_bytes, ws);
  return cudaGetLastError();
}

// Scalar subtraction (Sec. V-A "Scalar Subtraction"): the same pass with the
// scalar's bin deducted, O' = O - rho_s.
cudaError_t launch_sub_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws) {
  k_meta<false><<<persistent_grid(k_meta<false>, 512, lc.grid), 512, 0, lc.stream>>>(c, c_bytes, s, 1, out, cap, out_bytes, ws);
  return cudaGetLastError();
}

// magnitudes and sign byte of an octet of deltas
__device__ __forceinline__ void octet_mag_sign(const int d[8], uint32_t mag[8], uint32_t& sb) {
  sb = 0;
#pragma unroll
  for (int t = 0; t < 8; t++) {
    mag[t] = (uint32_t)abs(d[t]);
    sb |= (d[t] < 0 ? 1u : 0u) << t;
  }
}

// ---------------------------------------------------------------- Hadamard product
// The octet tile pipeline of the product by per-value multipliers: a loader
// warp bulk-copies input tiles (located by the rate pre-scan); compute warps
// decode them to q (workflow 3), requantize, and Lorenzo + BF re-encode each
// tile into its workspace slot (see produce_tile). Scalar multiplication runs
// on the two-lanes kernel of mul.cu; modes 0 and 1 of this template remain
// its octet form.
constexpr int MUL_STAGES = 8;
constexpr uint32_t MUL_RING = 8192;  // plane-ring words (64 KB)

// MODE 0: the paper's operator (multiplier rho_s); 1: the scalar itself;
// 2: the Hadamard product, with the multiplier of each value read from qb (the
// second stream b decoded to its integers).
template <int MODE>
__global__ void __launch_bounds__(PRODUCER_THREADS, 2) k_mul_scalar(
    const uint8_t* __restrict__ c, uint64_t c_bytes, double s, const uint8_t* __restrict__ b,
    uint64_t b_bytes, const int* __restrict__ qb, uint8_t* __restrict__ out, uint64_t cap,
    uint32_t e_bits, const unsigned long long* __restrict__ pre, Ws ws) {
  extern __shared__ __align__(16) uint8_t dyn[];
  InStage* ins = reinterpret_cast<InStage*>(dyn);
  uint64_t* ring = reinterpret_cast<uint64_t*>(ins + MUL_STAGES);
  __shared__ uint64_t full[MUL_STAGES], ready[MUL_STAGES], empty[MUL_STAGES];
  __shared__ unsigned long long stage_tile[MUL_STAGES];
  __shared__ uint8_t srate[2][TILE];
  __shared__ long long s_rho;
  __shared__ int s_ok;
  const int tid = threadIdx.x, w = tid >> 5, g = tid >> 3, j = tid & 7;
  const Info h = parse_header(c, c_bytes);
  int bad = 0;
  if (tid == 0) {
    int ok = h.ok;
    long long rho = 0;
    if (!h.ok) bad = HOSZP_ERR_FORMAT;
    else if (MODE == 0 && !quantize_scalar(s, h.eps_q, rho)) {
      ok = 0;
      bad = HOSZP_ERR_RANGE;
    } else if (cap < off_sign(h.nb)) {
      ok = 0;
      bad = HOSZP_ERR_CAPACITY;
    } else if (MODE == 2) {  // the multipliers' stream: same n and eps_q
      const Info hb = parse_header(b, b_bytes);
      if (!hb.ok) {
        ok = 0;
        bad = HOSZP_ERR_FORMAT;
      } else if (hb.n != h.n || __float_as_uint(hb.eps_q) != __float_as_uint(h.eps_q)) {
        ok = 0;
        bad = HOSZP_ERR_MISMATCH;
      } else {
        rho = hb.qbound;  // the largest multiplier, for the plan
      }
    }
    s_ok = ok;
    s_rho = rho;
    if (blockIdx.x == 0) write_template(h, 0, ws);
  }
  ring_init3<MUL_STAGES>(full, ready, empty);
  const uint64_t ntiles = (s_ok && prescan_ok(h, pre, ws.max_tiles)) ? ntiles_of(h.nb) : 0;
  MulPlan mp;
  if (MODE == 1) {
    mp = mul_plan_exact(s, h.ok ? h.qbound : 0u);
  } else if (MODE == 2) {
    // plan for the largest multiplier: its 64-bit path bounds every product
    mp = mul_plan(h.ok ? h.eps_q : 1.0f, s_rho, h.ok ? h.qbound : 0u);
    mp.f32 = false;
  } else {
    mp = mul_plan(h.ok ? h.eps_q : 1.0f, s_rho, h.ok ? h.qbound : 0u);
  }
  const OctetSel S = octet_sel(j);
  uint32_t qmax = 0;
  bool ovf = false;
  if (w >= LOADER_WARP) {
    const uint64_t G = gridDim.x;
    __shared__ ulonglong2 s_win[32][2];
    PreWindow pw;
    pw.init(s_win);
    __shared__ uint32_t s_beg[MUL_STAGES];
    PlaneRing<MUL_STAGES, MUL_RING> pr;
    pr.init(ring, s_beg);
    loader_warps<MUL_STAGES>(
        w - LOADER_WARP, stage_tile, full, ready, empty, ntiles, ws.status,
        [&](uint32_t k) { return (unsigned long long)(blockIdx.x + (uint64_t)k * G); },
        [&](int sk, unsigned long long t, uint32_t k, const uint32_t& k_rel,
            auto&& release_one) {
          unsigned long long pv[4];
          pw.get(pre, k, blockIdx.x, G, ntiles, pv);
          const TileSpan sp = tile_span(h, t, pv);
          const uint32_t p0 = pr.reserve(k, sp.plane_words(), k_rel, release_one);
          const uint32_t at = pr.commit(k, p0, sp.plane_words());
          if ((tid & 31) == 0) issue_in_tile(&ins[sk], &full[sk], c, h, t, sp, ring, at);
        },
        [&](int sk, unsigned long long t) { prepare_tile(ins[sk], t, h); });
  } else {
    RingPos rp{0, 0u};
    for (uint64_t k = 0;; k++) {
      const int st = rp.s;
      mbar_wait(&ready[st], rp.par, ws.status);
      const unsigned long long tile = stage_tile[st];
      if (tile >= ntiles) break;
      const InStage& sg = ins[st];
      const BlockRef br = block_ref_s(sg, ring, g, j);
      const int kmax = sg.kmx[w];
      int d[8], q[8];
      octet_deltas(br, kmax, j, S, d);
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[st]);
      rp.next<MUL_STAGES>();
      octet_values(br, d, j, q);
      if (br.len < L) {  // positions past the stream end hold no value
#pragma unroll
        for (int t = 0; t < 8; t++)
          if (8 * j + t >= br.len) q[t] = 0;
      }
      if (MODE == 2) {  // Hadamard product: this octet's multipliers
        const uint64_t i0 = (tile * TILE + g) * L + 8 * j;
        int m8[8];
        if (br.len == L) {
          const int4 u0 = __ldcs(reinterpret_cast<const int4*>(qb + i0));
          const int4 u1 = __ldcs(reinterpret_cast<const int4*>(qb + i0) + 1);
          m8[0] = u0.x; m8[1] = u0.y; m8[2] = u0.z; m8[3] = u0.w;
          m8[4] = u1.x; m8[5] = u1.y; m8[6] = u1.z; m8[7] = u1.w;
        } else {
#pragma unroll
          for (int t = 0; t < 8; t++) m8[t] = (8 * j + t < br.len) ? qb[i0 + t] : 0;
        }
#pragma unroll
        for (int t = 0; t < 8; t++) q[t] = mul_requant_pair(q[t], m8[t], mp, ovf);
      } else if (mp.f32) {
#pragma unroll
        for (int t = 0; t < 8; t++) q[t] = mul_requant_f32(q[t], mp);
      } else if (mp.fast) {
#pragma unroll
        for (int t = 0; t < 8; t++) q[t] = mul_requant_fast(q[t], mp, ovf);
      } else {
#pragma unroll
        for (int t = 0; t < 8; t++) q[t] = mul_requant(q[t], mp, ovf);
      }
      if (br.len < L) {
#pragma unroll
        for (int t = 0; t < 8; t++)
          if (8 * j + t >= br.len) q[t] = 0;
      }
#pragma unroll
      for (int t = 0; t < 8; t++) qmax = max(qmax, (uint32_t)abs(q[t]));
      // Lorenzo on the new integers
      const int prev = __shfl_up_sync(0xffffffffu, q[7], 1, 8);
      const int outlier = __shfl_sync(0xffffffffu, q[0], (tid & 31) & ~7);
      int nd[8];
#pragma unroll
      for (int t = 0; t < 8; t++) nd[t] = (t == 0) ? ((j == 0) ? 0 : q[0] - prev) : q[t] - q[t - 1];
      if (br.len < L) {
#pragma unroll
        for (int t = 0; t < 8; t++)
          if (8 * j + t >= br.len) nd[t] = 0;
      }
      uint32_t mag[8], sb;
      octet_mag_sign(nd, mag, sb);
      const int rate = octet_rate(mag);
      produce_tile(srate, k, tile, h.nb, mag, sb, rate, outlier, tile * TILE + g < h.nb, g, j,
                   out, ws.staging,
                   slot_offset(MODE == 2 ? SLOT_FULL : SLOT_MUL, tile, pre, nullptr, e_bits),
                   ws.staging_words, ws.agg, S, bad);
    }
  }
  if (ovf) bad = HOSZP_ERR_OVERFLOW;
  reduce_qmax(qmax, ws);
  if (bad) set_status(ws.status, bad);
}

template <int MODE>
static cudaError_t launch_mul_mode(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                                   const uint8_t* b, uint64_t b_bytes, const int* qb,
                                   uint32_t e_bits, uint8_t* out, uint64_t cap, Ws ws) {
  cudaError_t e = launch_scan(lc, c, c_bytes, ws.pre[0], ws);
  if (e != cudaSuccess) return e;
  const size_t smem = MUL_STAGES * sizeof(InStage) + MUL_RING * sizeof(uint64_t);
  smem_attr<k_mul_scalar<MODE>>(smem);
  k_mul_scalar<MODE><<<persistent_grid(k_mul_scalar<MODE>, PRODUCER_THREADS, lc.grid, smem),
                       PRODUCER_THREADS, smem, lc.stream>>>(c, c_bytes, s, b, b_bytes, qb, out,
                                                            cap, e_bits, ws.pre[0], ws);
  return cudaGetLastError();
}

// Hadamard product (Sec. V-C): b's integers already decoded into qb.
cudaError_t launch_hadamard(const Launch& lc, const uint8_t* a, uint64_t a_bytes,
                            const uint8_t* b, uint64_t b_bytes, const int* qb, uint8_t* out,
                            uint64_t cap, Ws ws) {
  return launch_mul_mode<2>(lc, a, a_bytes, 0.0, b, b_bytes, qb, 0u, out, cap, ws);
}

// ---------------------------------------------------------------- element-wise addition
// Workflow 2 on the bit-planes themselves. A block's deltas are stored
// bit-sliced (plane p holds bit p of |delta_i| at bit i; the sign word holds
// the signs), so the 64 additions delta_A,i + delta_B,i of a block are done
// plane by plane with 32 positions per 32-bit word:
//   two's complement of each input:  x = (m XOR s) + s   (carry chain, carry-in s)
//   sum:                             z = x + y           (full adder per plane)
//   back to sign and magnitude:      s' = top plane of z; m' = (z XOR s') + s'
// over W = max(rate_A, rate_B) + 2 planes (|delta_A + delta_B| < 2^(max+1)).
// The result's rate is the highest nonzero plane of m'. Element-wise
// subtraction is the same with the second input's signs inverted (negation
// flips every sign bit; a zero magnitude stays zero whatever its sign).
//
// Inputs come through the two-stream super-tile pipeline of hz_super.cuh
// (4 tiles of A and of B per stage, one loader warp, in-kernel rate prefixes of
// both streams, no pre-scan launch). Four groups of 4 compute warps take the
// stages in turn; warp i of a group takes tile i of its stage and walks it 16
// blocks at a time (lane 2m + h: half h of block m), keeping a running count
// of the tile's output sign and plane words, so it writes every block's words
// at once -- no barrier inside the loop. Sign words go to the tile's sign slot
// and plane words to its plane slot (the SPLIT rule), at upper bounds known from
// the inputs' prefixes: a block of the sum has a sign word only where A or B
// has one, and at most max(rate_A, rate_B) + 1 planes.
constexpr int ADD_NT = 4;        // tiles per stage
constexpr int ADD_STAGES = 8;
constexpr uint32_t ADD_RING = 18432;  // plane-ring words (144 KB), A's and B's words of stages
constexpr int ADD_TS = 2048;     // tile sums kept per stream
constexpr int ADD_GW = ADD_NT;   // warps per group (one per tile)
constexpr int ADD_GROUPS = 4;
constexpr int ADD_NCW = ADD_GROUPS * ADD_GW;
constexpr int ADD_THREADS = (ADD_NCW + 1) * 32;  // + loader warp

template <bool SUB>
__global__ void __launch_bounds__(ADD_THREADS, 1) k_add(
    const uint8_t* __restrict__ a, uint64_t a_bytes, const uint8_t* __restrict__ b,
    uint64_t b_bytes, uint8_t* __restrict__ out, uint64_t cap, Ws ws) {
  using St = SStageT<ADD_NT>;
  extern __shared__ __align__(16) uint8_t dyn[];
  St* stages = reinterpret_cast<St*>(dyn);  // [2][ADD_STAGES]: A's, then B's
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + 2 * ADD_STAGES);
  __shared__ uint64_t full[ADD_STAGES], empty[ADD_STAGES];
  __shared__ unsigned long long stage_st[ADD_STAGES];
  __shared__ uint32_t s_ts[2 * ADD_TS];
  __shared__ int s_ok;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const Info ha = parse_header(a, a_bytes);
  const Info hb = parse_header(b, b_bytes);
  const unsigned long long epoch = launch_epoch(ws);
  int bad = 0;
  if (tid == 0) {
    int ok = 0;
    if (!ha.ok || !hb.ok) bad = HOSZP_ERR_FORMAT;
    else if (ha.n != hb.n || __float_as_uint(ha.eps_q) != __float_as_uint(hb.eps_q))
      bad = HOSZP_ERR_MISMATCH;
    else if ((long long)ha.qbound + (long long)hb.qbound > HOSZP_QLIM)
      bad = HOSZP_ERR_OVERFLOW;
    else if (cap < off_sign(ha.nb) || ntiles_of(ha.nb) + 1 > ws.max_tiles)
      bad = HOSZP_ERR_CAPACITY;
    else
      ok = 1;
    s_ok = ok;
    if (blockIdx.x == 0) {
      write_template(ha, ok ? ha.qbound + hb.qbound : 0, ws);
      if (ok) atomicMax(&ws.totals[2], (unsigned long long)(ha.qbound + hb.qbound));
    }
    for (int k = 0; k < ADD_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], ADD_GW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  const uint64_t ntiles = ok ? ntiles_of(ha.nb) : 0;
  const uint64_t nst = nsuper_of<ADD_NT>(ntiles);
  const uint8_t* cs[2] = {a, b};
  const Info hs[2] = {ha, hb};
  const SRange rg = range_sums_n<ADD_NT, 2>(cs, hs, ntiles, nst, s_ts, ADD_TS, ws, epoch, bad);
  __syncthreads();
  if (w == ADD_NCW) {
    __shared__ uint32_t s_beg[ADD_STAGES];
    super_loader_n<ADD_NT, 2, ADD_STAGES, ADD_RING, ADD_GROUPS>(
        stages, ring, s_beg, full, empty, stage_st, cs, hs, rg, s_ts, ADD_TS, ws, epoch);
  } else if (w < ADD_NCW) {
    const int grp = w / ADD_GW, ti = w % ADD_GW;
    const int hf = lane & 1, m = lane >> 1;
    // the header values the loop needs, in registers (the stream tables above
    // are passed by address and may live in local memory)
    const uint64_t nb = ha.nb;
    // sign slots first (at most A's plus B's sign words), plane slots after
    const uint64_t sign_cap = umin64(ha.nnc + hb.nnc, ws.staging_words);
    for (uint64_t k = 0;; k++) {
      const uint64_t u = k * ADD_GROUPS + grp;  // stage use taken by this group
      const int st = (int)(u % ADD_STAGES);
      if (!mbar_wait_warp(&full[st], (uint32_t)((u / ADD_STAGES) & 1), ws.status)) break;
      const unsigned long long s = stage_st[st];
      if (s == ~0ull) break;
      const St& sa = stages[st];
      const St& sb = stages[ADD_STAGES + st];
      const uint64_t tile = (uint64_t)ADD_NT * s + ti;
      const TileRates tra = tile_rates(sa, ti, tile, nb);
      const TileRates trb = tile_rates(sb, ti, tile, nb);
      const int nvt = tra.nvt;
      const uint32_t* sgA = reinterpret_cast<const uint32_t*>(sa.sign + sa.sbase + sa.tnc[ti]);
      const uint32_t* plA =
          reinterpret_cast<const uint32_t*>(ring + sa.pring + sa.pbase + sa.tr[ti]);
      const uint32_t* sgB = reinterpret_cast<const uint32_t*>(sb.sign + sb.sbase + sb.tnc[ti]);
      const uint32_t* plB =
          reinterpret_cast<const uint32_t*>(ring + sb.pring + sb.pbase + sb.tr[ti]);
      // slots of the tile: upper bounds of the sum's words before it
      const uint64_t ancA = sa.bnc + sa.tnc[ti], arA = sa.br + sa.tr[ti];
      const uint64_t ancB = sb.bnc + sb.tnc[ti], arB = sb.br + sb.tr[ti];
      const uint64_t so = ancA + ancB, po = sign_cap + ancA + ancB + arA + arB;
      const uint32_t tA = __shfl_sync(0xffffffffu, tra.e1 + (tra.r1 ? 0x10000u : 0u) + tra.r1, 31);
      const uint32_t tB = __shfl_sync(0xffffffffu, trb.e1 + (trb.r1 ? 0x10000u : 0u) + trb.r1, 31);
      const uint32_t lim_nc = (tA >> 16) + (tB >> 16);
      const uint32_t lim_r = lim_nc + (tA & 0xffffu) + (tB & 0xffffu);
      int tbad = 0;
      if (so + lim_nc > sign_cap || po + lim_r > ws.staging_words) tbad = HOSZP_ERR_CAPACITY;
      uint32_t* sdst = reinterpret_cast<uint32_t*>(ws.staging + so);
      uint32_t* pdst = reinterpret_cast<uint32_t*>(ws.staging + po);
      uint32_t run = 0;  // output (sign words << 16 | plane words) of the tile so far
      const int steps = (nvt + 15) >> 4;  // warp-uniform
      for (int it = 0; it < steps; it++) {
        const int bk = 16 * it + m;
        uint32_t ra, exa, rb, exb;
        tile_block(tra, bk, ra, exa);
        tile_block(trb, bk, rb, exb);
        const bool valid = bk < nvt;
        const uint32_t* pa = plA + 2 * (exa & 0xffffu) + hf;
        const uint32_t* pb = plB + 2 * (exb & 0xffffu) + hf;
        const uint32_t siga = ra ? sgA[2 * (exa >> 16) + hf] : 0u;
        uint32_t sigb = rb ? sgB[2 * (exb >> 16) + hf] : 0u;
        if (SUB) sigb = ~sigb;  // negation flips every sign bit (a zero stays zero)
        const int mr = max((int)ra, (int)rb);
        // planes 0 .. P of the two's-complement sum, P = the warp's largest m + 1
        // (|delta_A + delta_B| < 2^(m+1), so plane m+1 and above are the sign; a
        // lane whose own m is smaller just sign-extends further). Unrolled over P
        // so the planes live in registers and every load of the block is issued
        // at once.
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
          const uint64_t bi = tile * TILE + bk;
          const int oa = sa.outlier[TILE * ti + bk], ob = sb.outlier[TILE * ti + bk];
          out[HOSZP_HEADER_BYTES + bi] = (uint8_t)rate;
          reinterpret_cast<int*>(out + off_outlier(nb))[bi] = SUB ? oa - ob : oa + ob;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (tbad) bad = tbad;
      if (lane == 0 && tile < ntiles) {
        ws.agg[tile] = ((unsigned long long)(run >> 16) << 32) | (run & 0xffffu);
        ws.pre[0][2 * tile] = so;
        ws.pre[0][2 * tile + 1] = po;
      }
    }
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && w == 0) {
    const bool ok_a = range_totals_ok(ws, ha, 0, 2), ok_b = range_totals_ok(ws, hb, 1, 2);
    if (tid == 0) {
      if (ok && !(ok_a && ok_b)) set_status(ws.status, HOSZP_ERR_FORMAT);
      launch_reset(ws);
    }
  }
}

cudaError_t launch_add(const Launch& lc, const uint8_t* a, uint64_t a_bytes, const uint8_t* b,
                       uint64_t b_bytes, uint8_t* out, uint64_t cap, bool subtract, Ws ws) {
  const size_t smem = 2 * ADD_STAGES * sizeof(SStageT<ADD_NT>) + ADD_RING * sizeof(uint64_t);
  smem_attr<k_add<false>>(smem);
  smem_attr<k_add<true>>(smem);
  const int grid = subtract ? persistent_grid(k_add<true>, ADD_THREADS, lc.grid, smem)
                            : persistent_grid(k_add<false>, ADD_THREADS, lc.grid, smem);
  if (subtract)
    k_add<true><<<grid, ADD_THREADS, smem, lc.stream>>>(a, a_bytes, b, b_bytes, out, cap, ws);
  else
    k_add<false><<<grid, ADD_THREADS, smem, lc.stream>>>(a, a_bytes, b, b_bytes, out, cap, ws);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- covariance
// Population covariance of two streams of one length (Sec. V-D, done like the
// variance of Sec. V-B over two fields) in one pass: exact sums
// S_AB = sum q_A q_B, S1_A and S1_B, finished in FP64 by the last CTA. Each
// side scales by its own 2 eps, so the error bounds may differ. The inputs come
// through the addition's two-stream super-tile pipeline, with three tiles per
// stage: 12 jobs (3 tiles x 4 quarters of 16 blocks), one per compute warp,
// two lanes per block of both streams (cov_quarter, hz_var.cuh). Twelve
// compute warps and the loader leave 128 registers per thread (a lane keeps its
// half's 32 prefixes of A while it decodes B). No named barrier in the stage
// loop, so a warp whose bounded wait gave up leaves it. Per-CTA partials:
// [bid] holds S1_A and S1_B, [G + bid] S_AB.
constexpr int COV_NT = 3;
constexpr int COV_NCW = 12;
constexpr int COV_JOBS = COV_NT * 4;  // quarters of a stage
constexpr int COV_THREADS = (COV_NCW + 1) * 32;
static_assert(COV_JOBS % COV_NCW == 0, "every compute warp takes as many jobs");

__global__ void __launch_bounds__(COV_THREADS, 1) k_cov(
    const uint8_t* __restrict__ a, uint64_t a_bytes, const uint8_t* __restrict__ b,
    uint64_t b_bytes, double* result, Ws ws) {
  using St = SStageT<COV_NT>;
  extern __shared__ __align__(16) uint8_t dyn[];
  St* stages = reinterpret_cast<St*>(dyn);  // [2][ADD_STAGES]: A's, then B's
  uint64_t* ring = reinterpret_cast<uint64_t*>(stages + 2 * ADD_STAGES);
  __shared__ uint64_t full[ADD_STAGES], empty[ADD_STAGES];
  __shared__ unsigned long long stage_st[ADD_STAGES];
  __shared__ uint32_t s_ts[2 * ADD_TS];
  __shared__ __int128 s_w[3][COV_THREADS / 32];
  __shared__ int s_ok;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const Info ha = parse_header(a, a_bytes);
  const Info hb = parse_header(b, b_bytes);
  const unsigned long long epoch = launch_epoch(ws);
  int bad = 0;
  if (tid == 0) {
    int ok = 0;
    if (!ha.ok || !hb.ok) bad = HOSZP_ERR_FORMAT;
    else if (ha.n != hb.n) bad = HOSZP_ERR_MISMATCH;
    else ok = 1;
    s_ok = ok;
    for (int k = 0; k < ADD_STAGES; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], COV_NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  const uint64_t ntiles = ok ? ntiles_of(ha.nb) : 0;
  const uint64_t nst = nsuper_of<COV_NT>(ntiles);
  const uint8_t* cs[2] = {a, b};
  const Info hs[2] = {ha, hb};
  const SRange rg = range_sums_n<COV_NT, 2>(cs, hs, ntiles, nst, s_ts, ADD_TS, ws, epoch, bad);
  __syncthreads();
  __int128 sab = 0;
  long long s1a = 0, s1b = 0;
  if (w == COV_NCW) {
    __shared__ uint32_t s_beg[ADD_STAGES];
    super_loader_n<COV_NT, 2, ADD_STAGES, ADD_RING, 1>(stages, ring, s_beg, full, empty, stage_st,
                                                        cs, hs, rg, s_ts, ADD_TS, ws, epoch);
  } else if (w < COV_NCW) {
    const int lastlen = ok ? (int)(ha.n - (ha.nb - 1) * L) : 0;
    const bool qsmall = ha.qbound < (1u << 13) && hb.qbound < (1u << 13);
    const lanes::Shifts K = lanes::make_shifts(a_bytes != 0 ? 1u : 0u);
    for (uint64_t k = 0;; k++) {
      const int st = (int)(k % ADD_STAGES);
      if (!mbar_wait_warp(&full[st], (uint32_t)((k / ADD_STAGES) & 1), ws.status)) break;
      const unsigned long long s = stage_st[st];
      if (s == ~0ull) break;
      const St& sa = stages[st];
      const St& sb = stages[ADD_STAGES + st];
#pragma unroll 1
      for (int jb = w; jb < COV_JOBS; jb += COV_NCW) {
        const int grp = jb >> 2, quarter = jb & 3;
        const uint64_t tile = (uint64_t)COV_NT * s + grp;
        const TileRates tra = tile_rates(sa, grp, tile, ha.nb);
        const TileRates trb = tile_rates(sb, grp, tile, hb.nb);
        cov_quarter(sa, sb, ring, grp, tra, trb, tile, ntiles, lastlen, quarter, qsmall, K, sab,
                    s1a, s1b);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  // CTA reduction -> two partials per CTA
  sab = warp_sum_i128(sab);
  const __int128 t1a = warp_sum_i128((__int128)s1a), t1b = warp_sum_i128((__int128)s1b);
  if (lane == 0) {
    s_w[0][w] = sab;
    s_w[1][w] = t1a;
    s_w[2][w] = t1b;
  }
  __syncthreads();
  if (tid == 0) {
    __int128 x = 0, y = 0, z = 0;
    for (int k = 0; k < COV_THREADS / 32; k++) {
      x += s_w[0][k];
      y += s_w[1][k];
      z += s_w[2][k];
    }
    Partial p1, p2;  // signed 128-bit values as two's-complement words
    p1.s1_lo = (long long)(unsigned long long)y;
    p1.s1_hi = (long long)(y >> 64);
    p1.s2_lo = (unsigned long long)z;
    p1.s2_hi = (unsigned long long)(z >> 64);
    p2.s1_lo = (long long)(unsigned long long)x;
    p2.s1_hi = (long long)(x >> 64);
    p2.s2_lo = 0;
    p2.s2_hi = 0;
    ws.partials[blockIdx.x] = p1;
    ws.partials[gridDim.x + blockIdx.x] = p2;
  }
  if (bad) set_status(ws.status, bad);
  if (launch_end_is_last(ws) && w == 0) {
    __int128 ya = 0, zb = 0, xab = 0;
    for (unsigned int u = lane; u < gridDim.x; u += 32) {
      const Partial p1 = ws.partials[u], p2 = ws.partials[gridDim.x + u];
      ya += (__int128)(((unsigned __int128)(unsigned long long)p1.s1_hi << 64) |
                       (unsigned long long)p1.s1_lo);
      zb += (__int128)(((unsigned __int128)p1.s2_hi << 64) | p1.s2_lo);
      xab += (__int128)(((unsigned __int128)(unsigned long long)p2.s1_hi << 64) |
                        (unsigned long long)p2.s1_lo);
    }
    ya = warp_sum_i128(ya);
    zb = warp_sum_i128(zb);
    xab = warp_sum_i128(xab);
    const bool ok_a = range_totals_ok(ws, ha, 0, 2), ok_b = range_totals_ok(ws, hb, 1, 2);
    if (tid == 0) {
      double res = 0.0;
      if (ok && !(ok_a && ok_b)) set_status(ws.status, HOSZP_ERR_FORMAT);
      else if (ok && ha.n == 0) set_status(ws.status, HOSZP_ERR_ARG);
      else if (ok) res = cov_finish(xab, ya, zb, ha.n, ha.eps_q, hb.eps_q);
      *result = res;
      launch_reset(ws);
    }
  }
}

cudaError_t launch_cov(const Launch& lc, const uint8_t* a, uint64_t a_bytes, const uint8_t* b,
                       uint64_t b_bytes, double* result, Ws ws) {
  const size_t smem = 2 * ADD_STAGES * sizeof(SStageT<COV_NT>) + ADD_RING * sizeof(uint64_t);
  smem_attr<k_cov>(smem);
  const int grid = persistent_grid(k_cov, COV_THREADS, lc.grid, smem);
  if ((uint64_t)2 * grid > ws.max_grid) return cudaErrorInvalidConfiguration;  // two partials per CTA
  k_cov<<<grid, COV_THREADS, smem, lc.stream>>>(a, a_bytes, b, b_bytes, result, ws);
  return cudaGetLastError();
}

}  // namespace hz
