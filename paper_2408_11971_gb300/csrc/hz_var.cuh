// hz_var.cuh — one warp's share of the exact sums S1 = sum q and S2 = sum q^2
// (Sec. V-B) over one 64-block tile of a landed super-tile stage, decoded two
// lanes per block with hz_lanes.cuh. Shared by the single-stream variance and
// the batched reductions; the block-wise means and the covariance sums of two
// streams (Sec. V-D) use the same decode.
#pragma once
#include "hz_lanes.cuh"
#include "hz_super.cuh"
#include "hz_wide.cuh"

namespace hz {

// half_sums of hz_lanes.cuh for the warp's widest rate Rw (G = (Rw + 8) / 8
// groups of 8 planes); tails and wide values take the 64-bit sums.
// The two's-complement planes of a half span G = (Rw + 8) / 8 groups of 8
// (the rate's planes and the sign). GMAX: the most groups the calling kernel
// was built for (4 covers every rate; a plan whose rates stay below 8 GMAX
// may take fewer, which drops the wider cases and their registers).
template <int GMAX = 4>
__device__ __forceinline__ lanes::HalfSums half_sums_any(int Rw, bool full, bool narrow,
                                                         const uint32_t t[32], int nval,
                                                         bool zero0, const lanes::Shifts& K) {
  const int G = min((Rw + 8) >> 3, GMAX);
#define HZ_HS(GG)                                                          \
  if (GG == GMAX || G == GG) {                                             \
    if (!full) return lanes::half_sums<GG, false, true>(t, nval, zero0, K);   \
    if (narrow) return lanes::half_sums<GG, true, false>(t, nval, zero0, K);  \
    return lanes::half_sums<GG, true, true>(t, nval, zero0, K);               \
  }
  HZ_HS(1)
  if constexpr (GMAX >= 2) HZ_HS(2)
  if constexpr (GMAX >= 3) HZ_HS(3)
#undef HZ_HS
  if (!full) return lanes::half_sums<4, false, true>(t, nval, zero0, K);
  if (narrow) return lanes::half_sums<4, true, false>(t, nval, zero0, K);
  return lanes::half_sums<4, true, true>(t, nval, zero0, K);
}

// Tile `ti` of stage sg (rates in tr, tile index `tile` of a stream of
// `ntiles` tiles whose last block holds `lastlen` values): adds this lane's
// share of S1 and S2. The warp takes 16 blocks per step; lane 2m + hf holds
// half hf of block 16 it + m. qsmall: the stream's header bounds every |q|
// below 2^13. GMAX: as half_sums_any (rates below 8 GMAX decode exactly).
template <int GMAX = 4, class St>
__device__ __forceinline__ void var_tile(const St& sg, const uint64_t* ring, int ti,
                                         const TileRates& tr, uint64_t tile, uint64_t ntiles,
                                         int lastlen, bool qsmall, const lanes::Shifts& K,
                                         long long& s1, U128& s2) {
  const int lane = threadIdx.x & 31;
  const int hf = lane & 1, m = lane >> 1;
  const uint32_t* sgn = reinterpret_cast<const uint32_t*>(sg.sign + sg.sbase + sg.tnc[ti]);
  const uint32_t* pls = reinterpret_cast<const uint32_t*>(ring + sg.pring + sg.pbase + sg.tr[ti]);
  const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
  for (int it = 0; it < steps; it++) {
    const int b = 16 * it + m;
    uint32_t r, ex;
    tile_block(tr, b, r, ex);
    const int len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
    const int nval = min(max(len - 32 * hf, 0), 32);
    const long long O = len ? sg.outlier[TILE * ti + b] : 0;
    const uint32_t sw = r ? sgn[2 * (ex >> 16) + hf] : 0u;
    const int Rw = (int)__reduce_max_sync(0xffffffffu, r);
    const bool fullblk = __all_sync(0xffffffffu, len == L);
    uint32_t t[32];
    lanes::twos_planes_any<8 * GMAX - 1>(Rw, pls + 2 * (ex & 0xffffu) + hf, (int)r, sw, t);
    // narrow sums of p^2 need every |p_i| < 2^14: |q| < 2^13, or 32 deltas below 2^8
    const bool narrow = fullblk && (qsmall || Rw <= 8);
    const lanes::HalfSums hs = half_sums_any<GMAX>(Rw, fullblk, narrow, t, nval, hf == 0, K);
    const int tot0 = __shfl_xor_sync(0xffffffffu, hs.tot, 1);
    const long long base = O + (hf ? (long long)tot0 : 0ll);
    s1 += (long long)nval * base + hs.sp;
    if (narrow && qsmall) {  // every term below 2^40
      add_u64(s2, (unsigned long long)((long long)nval * base * base + 2ll * base * hs.sp +
                                       (long long)hs.sq));
    } else {
      const __int128 sq = narrow ? (__int128)hs.sq : (((__int128)hs.sqh << 64) | hs.sq);
      const __int128 v = (__int128)(nval * base) * base + (__int128)(2 * base) * hs.sp + sq;
      const U128 vv = {(unsigned long long)v, (unsigned long long)(v >> 64)};
      add_u128(s2, vv);
    }
  }
}

// Block-wise means (Sec. V-B, "Mean", last sentences) of tile `ti`: the warp
// takes 16 blocks per step, lane 2m + hf half hf of block 16 it + m; the
// block's exact sum S1_b = sum of its q is formed from both halves and lane
// 2m writes mean_b = (S1_b / L_b) * e2 (the same two FP64 operations as the
// mean of the whole stream).
template <class St>
__device__ __forceinline__ void block_means_tile(const St& sg, const uint64_t* ring, int ti,
                                                 const TileRates& tr, uint64_t tile,
                                                 uint64_t ntiles, int lastlen, double e2,
                                                 const lanes::Shifts& K, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int hf = lane & 1, m = lane >> 1;
  const uint32_t* sgn = reinterpret_cast<const uint32_t*>(sg.sign + sg.sbase + sg.tnc[ti]);
  const uint32_t* pls = reinterpret_cast<const uint32_t*>(ring + sg.pring + sg.pbase + sg.tr[ti]);
  const int steps = (tr.nvt + 15) >> 4;  // warp-uniform
  for (int it = 0; it < steps; it++) {
    const int b = 16 * it + m;
    uint32_t r, ex;
    tile_block(tr, b, r, ex);
    const int len = (b < tr.nvt - 1) ? L : (b == tr.nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
    const int nval = min(max(len - 32 * hf, 0), 32);
    const long long O = len ? sg.outlier[TILE * ti + b] : 0;
    const uint32_t sw = r ? sgn[2 * (ex >> 16) + hf] : 0u;
    const int Rw = (int)__reduce_max_sync(0xffffffffu, r);
    const bool fullblk = __all_sync(0xffffffffu, len == L);
    uint32_t t[32];
    lanes::twos_planes_any(Rw, pls + 2 * (ex & 0xffffu) + hf, (int)r, sw, t);
    const bool narrow = fullblk && Rw <= 20;  // sum_i (32 - i) |delta_i| < 2^31
    lanes::HalfSums hs;
    const int G = (Rw + 8) >> 3;
#define HZ_S1(GG)                                                                      \
  if (G == GG) {                                                                       \
    hs = !fullblk  ? lanes::half_sums<GG, false, true, false>(t, nval, hf == 0, K)   \
         : narrow ? lanes::half_sums<GG, true, false, false>(t, nval, hf == 0, K)    \
                  : lanes::half_sums<GG, true, true, false>(t, nval, hf == 0, K);    \
  }
    HZ_S1(1) else HZ_S1(2) else HZ_S1(3) else HZ_S1(4)
#undef HZ_S1
    const int tot0 = __shfl_xor_sync(0xffffffffu, hs.tot, 1);
    const long long base = O + (hf ? (long long)tot0 : 0ll);
    const long long s1h = (long long)nval * base + hs.sp;
    const long long s1 = s1h + __shfl_xor_sync(0xffffffffu, s1h, 1);
    // a full block divides by 64, exactly a scaling by 2^-6 (no FP64 divide)
    const double mb = (len == L) ? (double)s1 * 0.015625 : (double)s1 / (double)len;
    if (hf == 0 && len > 0) out[tile * TILE + b] = mb * e2;
  }
}

// half_visit / half_prefix of hz_lanes.cuh for the warp's widest rate Rw.
template <class F>
__device__ __forceinline__ void half_visit_any(int Rw, const uint32_t t[32], bool zero0,
                                               const lanes::Shifts& K, F&& f) {
  switch ((Rw + 8) >> 3) {
    case 1: lanes::half_visit<1>(t, zero0, K, f); break;
    case 2: lanes::half_visit<2>(t, zero0, K, f); break;
    case 3: lanes::half_visit<3>(t, zero0, K, f); break;
    default: lanes::half_visit<4>(t, zero0, K, f); break;
  }
}
template <int GMAX = 4>
__device__ __forceinline__ void half_prefix_any(int Rw, const uint32_t t[32], bool zero0,
                                                const lanes::Shifts& K, int p[32]) {
  const int G = min((Rw + 8) >> 3, GMAX);
  if (GMAX == 1 || G == 1) lanes::half_prefix<1>(t, zero0, K, p);
  else if constexpr (GMAX >= 2) {
    if (GMAX == 2 || G == 2) lanes::half_prefix<2>(t, zero0, K, p);
    else if constexpr (GMAX >= 3) {
      if (GMAX == 3 || G == 3) lanes::half_prefix<3>(t, zero0, K, p);
      else lanes::half_prefix<4>(t, zero0, K, p);
    }
  }
}

// Covariance sums (Sec. V-D) over 16 blocks of tile `ti` of two landed stages
// of streams of one length: blocks 16 quarter .. 16 quarter + 15, lane 2m + hf
// holding half hf of block 16 quarter + m of both streams. With q = b + p on
// each side (b the half's base, p its local prefix), a half adds
//   sum q_A q_B = n b_A b_B + b_A sum p_B + b_B sum p_A + sum p_A p_B
// to sab and its sums of q_A and q_B to s1a and s1b. qsmall: both headers
// bound every |q| below 2^13. Every warp collective here runs on all 32 lanes
// (the half bases are exchanged unconditionally, then selected).
template <class St>
__device__ __forceinline__ void cov_quarter(const St& sa, const St& sb, const uint64_t* ring,
                                            int ti, const TileRates& tra, const TileRates& trb,
                                            uint64_t tile, uint64_t ntiles, int lastlen,
                                            int quarter, bool qsmall, const lanes::Shifts& K,
                                            __int128& sab, long long& s1a, long long& s1b) {
  const int lane = threadIdx.x & 31;
  const int hf = lane & 1, m = lane >> 1;
  const int nvt = tra.nvt;
  if (16 * quarter >= nvt) return;  // warp-uniform: the whole quarter lies past the stream's end
  const int b = 16 * quarter + m;
  uint32_t ra, exa, rb, exb;
  tile_block(tra, b, ra, exa);
  tile_block(trb, b, rb, exb);
  const int len = (b < nvt - 1) ? L : (b == nvt - 1) ? ((tile + 1 == ntiles) ? lastlen : L) : 0;
  const int nval = min(max(len - 32 * hf, 0), 32);
  const long long OA = len ? sa.outlier[TILE * ti + b] : 0;
  const long long OB = len ? sb.outlier[TILE * ti + b] : 0;
  const uint32_t* sga = reinterpret_cast<const uint32_t*>(sa.sign + sa.sbase + sa.tnc[ti]);
  const uint32_t* sgb = reinterpret_cast<const uint32_t*>(sb.sign + sb.sbase + sb.tnc[ti]);
  const uint32_t* pla = reinterpret_cast<const uint32_t*>(ring + sa.pring + sa.pbase + sa.tr[ti]);
  const uint32_t* plb = reinterpret_cast<const uint32_t*>(ring + sb.pring + sb.pbase + sb.tr[ti]);
  const uint32_t swa = ra ? sga[2 * (exa >> 16) + hf] : 0u;
  const uint32_t swb = rb ? sgb[2 * (exb >> 16) + hf] : 0u;
  const int RwA = (int)__reduce_max_sync(0xffffffffu, ra);
  const int RwB = (int)__reduce_max_sync(0xffffffffu, rb);
  const bool fullblk = __all_sync(0xffffffffu, len == L);
  int pA[32];
  {
    uint32_t t[32];
    lanes::twos_planes_any(RwA, pla + 2 * (exa & 0xffffu) + hf, (int)ra, swa, t);
    half_prefix_any(RwA, t, hf == 0, K, pA);
  }
  // narrow: every |p| < 2^14, so eight products p_A p_B add up inside 32 bits
  const bool narrow = fullblk && (qsmall || (RwA <= 8 && RwB <= 8));
  long long spa = 0, spb = 0;
  __int128 pab = 0;
  int lastB = 0;
  {
    uint32_t t[32];
    lanes::twos_planes_any(RwB, plb + 2 * (exb & 0xffffu) + hf, (int)rb, swb, t);
    if (narrow) {
      int x = 0, y = 0, acc = 0;
      long long s8 = 0;
      half_visit_any(RwB, t, hf == 0, K, [&](int i, int pb) {
        x += pA[i];
        y += pb;
        acc = (int)lanes::mad((uint32_t)pA[i], (uint32_t)pb, (uint32_t)acc);
        if ((i & 7) == 7) {
          s8 += acc;
          acc = 0;
        }
        if (i == 31) lastB = pb;
      });
      spa = x;
      spb = y;
      pab = s8;
    } else {
      half_visit_any(RwB, t, hf == 0, K, [&](int i, int pb) {
        const long long xa = (i < nval) ? pA[i] : 0, yb = (i < nval) ? pb : 0;
        spa += xa;
        spb += yb;
        pab += (__int128)(xa * yb);
        if (i == 31) lastB = pb;
      });
    }
  }
  // the first half's totals, exchanged by every lane; the second half adds them
  const int totA = __shfl_xor_sync(0xffffffffu, pA[31], 1);
  const int totB = __shfl_xor_sync(0xffffffffu, lastB, 1);
  const long long bA = OA + (hf ? (long long)totA : 0ll);
  const long long bB = OB + (hf ? (long long)totB : 0ll);
  sab += (__int128)(nval * bA) * bB + (__int128)bA * spb + (__int128)bB * spa + pab;
  s1a += (long long)nval * bA + spa;
  s1b += (long long)nval * bB + spb;
}

}  // namespace hz
