// hz_lanes.cuh — decoding a block with two lanes, one per 32-position half,
// all in registers: the quantized integers q_i of Sec. V-B's variance without
// the cross-lane byte transposes of the octet decode.
//
// A lane holds, for its half, the sign half-word s and the plane half-words
// m_0 .. m_{r-1} (bit i of m_p = bit p of |delta| at position i, Fig. 3).
//  1. Two's-complement planes, bit-sliced: delta = (|delta| xor -s) + s is a
//     ripple carry over the planes (two logic operations per plane for 32
//     positions). Planes at and above the warp's widest rate all equal one
//     sign-fill word.
//  2. Transpose: for each group of 8 planes, two 4x4 byte transposes give,
//     per octet of positions, the 8 plane bytes; an 8x8 bit transpose turns
//     them into one byte of each of the 8 deltas.
//  3. Each delta is gathered from its group bytes by one byte permute that
//     also sign-extends (PRMT's sign-replicate selectors), then summed into
//     the local prefix p_i = sum of the half's deltas up to i.
// A half returns n_h, sum p_i and sum p_i^2 over its valid positions; with the
// base b (O for the first half, O plus the first half's delta total for the
// second) the half's exact sums are
//     S1_h = n_h b + sum p,      S2_h = n_h b^2 + 2 b sum p + sum p^2
// (q_i = b + p_i). The block's position 0 carries delta_0 := 0 (Eq. 4).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define HZL_HD __host__ __device__ __forceinline__
#else
#define HZL_HD inline
#endif

namespace hz {
namespace lanes {

// prmt.b32 in its default mode: result byte k = byte (sel_k & 7) of {a, b}
// (a holds bytes 0..3), or, when bit 3 of sel_k is set, that byte's sign bit
// replicated over all 8 bits.
HZL_HD uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
#ifdef __CUDA_ARCH__
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
#else
  const uint64_t x = ((uint64_t)b << 32) | a;
  uint32_t d = 0;
  for (int k = 0; k < 4; k++) {
    const uint32_t s = (sel >> (4 * k)) & 0xfu;
    uint32_t byte = (uint32_t)(x >> (8 * (s & 7u))) & 0xffu;
    if (s & 8u) byte = (byte & 0x80u) ? 0xffu : 0u;
    d |= byte << (8 * k);
  }
  return d;
#endif
}
// high word of a 32x32 product (a right shift issued on the FMA pipe)
HZL_HD uint32_t mulhi(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// a * b + c as an integer multiply-add (FMA pipe). With b a run-time 1 the
// compiler cannot turn it into an add on the logic pipe.
HZL_HD uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
#ifdef __CUDA_ARCH__
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
#else
  return a * b + c;
#endif
}

// Multipliers of the shifts in tr8x8, passed in at run time (built from a
// kernel argument) so that the compiler keeps them as integer multiplies on
// the multiply-add pipe instead of turning them back into shifts on the logic
// pipe, which the byte permutes and logic operations of the decode keep busy.
struct Shifts {
  uint32_t r7, r14, r4;  // 2^25, 2^18, 2^28: high words give >> 7, >> 14, >> 4
  uint32_t l7, l14, l4;  // 2^7, 2^14, 2^4: low words give << 7, << 14, << 4
};
HZL_HD Shifts make_shifts(uint32_t one) {
  Shifts k;
  k.r7 = one << 25;
  k.r14 = one << 18;
  k.r4 = one << 28;
  k.l7 = one << 7;
  k.l14 = one << 14;
  k.l4 = one << 4;
  return k;
}
HZL_HD uint32_t mullo(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  uint32_t d;
  asm("mul.lo.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
#else
  return a * b;
#endif
}

// 8x8 bit transpose of the matrix whose row k is byte k of (lo, hi) (bytes
// 0..3 of lo, then of hi) and whose column t is bit t: afterwards byte t holds
// what was bit t of every row (three delta swaps).
HZL_HD void tr8x8(uint32_t& lo, uint32_t& hi, const Shifts& K) {
  uint32_t t;
  t = (lo ^ mulhi(lo, K.r7)) & 0x00AA00AAu;
  lo = lo ^ t ^ mullo(t, K.l7);
  t = (hi ^ mulhi(hi, K.r7)) & 0x00AA00AAu;
  hi = hi ^ t ^ mullo(t, K.l7);
  t = (lo ^ mulhi(lo, K.r14)) & 0x0000CCCCu;
  lo = lo ^ t ^ mullo(t, K.l14);
  t = (hi ^ mulhi(hi, K.r14)) & 0x0000CCCCu;
  hi = hi ^ t ^ mullo(t, K.l14);
  t = (lo ^ mullo(hi, K.l4)) & 0xF0F0F0F0u;
  lo = lo ^ t;
  hi = hi ^ mulhi(t, K.r4);
}

// 4x4 byte transpose: x[k] byte p <- a[p] byte k.
HZL_HD void bt4x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t x[4]) {
  const uint32_t l01 = prmt(a0, a1, 0x5140u), h01 = prmt(a0, a1, 0x7362u);
  const uint32_t l23 = prmt(a2, a3, 0x5140u), h23 = prmt(a2, a3, 0x7362u);
  x[0] = prmt(l01, l23, 0x5410u);
  x[1] = prmt(l01, l23, 0x7632u);
  x[2] = prmt(h01, h23, 0x5410u);
  x[3] = prmt(h01, h23, 0x7632u);
}

// Step 1 for a warp whose widest rate is R: t[0 .. 8G-1] are the two's-
// complement planes of this half (G = (R + 8) / 8 groups of 8). pl points at
// this half's word of the block's plane 0 (plane p at pl[2p]); r <= R is the
// block's rate, s its sign half-word (0 for a constant block).
template <int R>
HZL_HD void twos_planes(const uint32_t* pl, int r, uint32_t s, uint32_t t[32]) {
  constexpr int W = 8 * ((R + 8) / 8);
  uint32_t c = s;
#pragma unroll
  for (int p = 0; p < R; p++) {
    const uint32_t m = (p < r) ? pl[2 * p] : 0u;
    const uint32_t x = m ^ s;
    t[p] = x ^ c;
    c = x & c;
  }
  const uint32_t f = s ^ c;
#pragma unroll
  for (int p = R; p < W; p++) t[p] = f;
}

// Dispatch of twos_planes on the warp-uniform R (0 .. MAXR). A kernel built
// for streams whose rates stay at or below MAXR instantiates only those cases;
// a larger R (a header that understates its values) decodes as MAXR.
template <int MAXR = 31>
HZL_HD void twos_planes_any(int R, const uint32_t* pl, int r, uint32_t s, uint32_t t[32]) {
  switch (R) {
#define HZL_CASE(K)                              \
  case K:                                        \
    if constexpr (K <= MAXR) twos_planes<K>(pl, r, s, t); \
    else twos_planes<MAXR>(pl, r, s, t);         \
    break;
    HZL_CASE(0) HZL_CASE(1) HZL_CASE(2) HZL_CASE(3) HZL_CASE(4) HZL_CASE(5) HZL_CASE(6)
    HZL_CASE(7) HZL_CASE(8) HZL_CASE(9) HZL_CASE(10) HZL_CASE(11) HZL_CASE(12) HZL_CASE(13)
    HZL_CASE(14) HZL_CASE(15) HZL_CASE(16) HZL_CASE(17) HZL_CASE(18) HZL_CASE(19) HZL_CASE(20)
    HZL_CASE(21) HZL_CASE(22) HZL_CASE(23) HZL_CASE(24) HZL_CASE(25) HZL_CASE(26) HZL_CASE(27)
    HZL_CASE(28) HZL_CASE(29) HZL_CASE(30)
    default:
      twos_planes<MAXR>(pl, r, s, t);
      break;
#undef HZL_CASE
  }
}

// The delta at position 4u + v (v = 0..3) of an octet from its G group bytes:
// word g holds group g's bytes of positions 4u .. 4u + 3.
template <int G>
HZL_HD int gather_delta(const uint32_t* w, int v) {
  const uint32_t b = (uint32_t)v;
  if (G == 1) return (int)prmt(w[0], 0u, b | ((8u | b) * 0x1110u));
  if (G == 2) return (int)prmt(w[0], w[1], b | ((4u + b) << 4) | ((12u + b) * 0x1100u));
  const uint32_t lo = prmt(w[0], w[1], b | ((4u + b) << 4));
  if (G == 3) return (int)prmt(lo, w[2], 0x10u | ((4u + b) << 8) | ((12u + b) << 12));
  const uint32_t hi = prmt(w[2], w[3], (b << 8) | ((4u + b) << 12));
  return (int)prmt(lo, hi, 0x7610u);
}

// Sums of one half (steps 2 and 3). nval: valid positions of the half (32 for
// a full one). zero0: this is the block's first half (position 0 is 0).
// WIDE: sum p^2 in 64-bit words (else in 32-bit words flushed every 16
// positions, valid while every |p_i| < 2^14; the narrow path needs FULL).
// K: the shift multipliers of tr8x8. Squares and position-weighted sums go
// through integer multiply-adds, in two independent chains each. SQ = false
// skips the squares (sums of q only); its narrow path then needs only
// |delta| < 2^21 (sum_i (32 - i) |delta_i| < 2^31).
struct HalfSums {
  int tot;                 // sum of the half's deltas (the next half's base offset)
  long long sp;            // sum of p_i
  unsigned long long sq;   // sum of p_i^2 (narrow path)
  unsigned long long sqh;  // high word of sum p_i^2 (wide path)
};
template <int G, bool FULL, bool WIDE, bool SQ = true>
HZL_HD HalfSums half_sums(const uint32_t t[32], int nval, bool zero0, const Shifts& K) {
  uint32_t X[4][4], Y[4][4];  // [group][octet]: planes 8g..8g+3 / 8g+4..8g+7
#pragma unroll
  for (int g = 0; g < G; g++) {
    bt4x4(t[8 * g], t[8 * g + 1], t[8 * g + 2], t[8 * g + 3], X[g]);
    bt4x4(t[8 * g + 4], t[8 * g + 5], t[8 * g + 6], t[8 * g + 7], Y[g]);
#pragma unroll
    for (int k = 0; k < 4; k++) tr8x8(X[g][k], Y[g][k], K);
  }
  HalfSums hs;
  uint32_t acc = 0;
  int sp[2] = {0, 0};
  long long sp64 = 0;
  uint32_t sq32[2] = {0, 0};  // octets 0, 2 / 1, 3: 16 squares each
  unsigned long long sq = 0, sqh = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
#pragma unroll
    for (int u = 0; u < 2; u++) {
      uint32_t w[4];
#pragma unroll
      for (int g = 0; g < G; g++) w[g] = u ? Y[g][k] : X[g][k];
#pragma unroll
      for (int v = 0; v < 4; v++) {
        const int i = 8 * k + 4 * u + v;  // position within the half
        int d = gather_delta<G>(w, v);
        if (i == 0 && zero0) d = 0;
        if (!FULL && i >= nval) d = 0;
        acc += (uint32_t)d;
        const int a = (!FULL && i >= nval) ? 0 : (int)acc;
        if (WIDE) {
          sp64 += a;
          if (SQ) {
            const unsigned long long p2 = (unsigned long long)((long long)a * a);
            sq += p2;
            sqh += (sq < p2) ? 1ull : 0ull;
          }
        } else {
          sp[k & 1] += d * (32 - i);  // sum_i p_i = sum_i (32 - i) d_i over a full half
          if (SQ) sq32[k & 1] = mad((uint32_t)a, (uint32_t)a, sq32[k & 1]);
        }
      }
    }
  }
  if (!WIDE && SQ) sq = (unsigned long long)sq32[0] + sq32[1];
  hs.tot = (int)acc;
  hs.sp = WIDE ? sp64 : (long long)sp[0] + sp[1];
  hs.sq = sq;
  hs.sqh = sqh;
  return hs;
}

// The local prefixes p_i (i = 0 .. 31) of one half (steps 2 and 3), handed to
// f(i, p_i) in position order (once unrolled, i is a compile-time constant in
// each call). Positions past the block's end are not masked.
template <int G, class F>
HZL_HD void half_visit(const uint32_t t[32], bool zero0, const Shifts& K, F&& f) {
  uint32_t X[4][4], Y[4][4];
#pragma unroll
  for (int g = 0; g < G; g++) {
    bt4x4(t[8 * g], t[8 * g + 1], t[8 * g + 2], t[8 * g + 3], X[g]);
    bt4x4(t[8 * g + 4], t[8 * g + 5], t[8 * g + 6], t[8 * g + 7], Y[g]);
#pragma unroll
    for (int k = 0; k < 4; k++) tr8x8(X[g][k], Y[g][k], K);
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
#pragma unroll
    for (int u = 0; u < 2; u++) {
      uint32_t w[4];
#pragma unroll
      for (int g = 0; g < G; g++) w[g] = u ? Y[g][k] : X[g][k];
#pragma unroll
      for (int v = 0; v < 4; v++) {
        const int i = 8 * k + 4 * u + v;
        int d = gather_delta<G>(w, v);
        if (i == 0 && zero0) d = 0;
        acc += (uint32_t)d;
        f(i, (int)acc);
      }
    }
  }
}

// The local prefixes of one half into p[0 .. 31].
template <int G>
HZL_HD void half_prefix(const uint32_t t[32], bool zero0, const Shifts& K, int p[32]) {
  half_visit<G>(t, zero0, K, [&](int i, int v) { p[i] = v; });
}

// ---------------------------------------------------------------- encode
// The inverse transposes, for operators that produce a stream from values
// held two lanes per block: the two's-complement planes z[0 .. 8G-1] of the
// half's 32 deltas d[0 .. 31] (bit i of z[p] = bit p of d_i). Per group g of
// 8 planes: byte g of each delta, four to a word (byte permutes); an 8x8 bit
// transpose per octet of positions turns its 8 bytes into the octet's byte of
// each of the 8 planes; two 4x4 byte transposes assemble each plane's word
// from the four octets.
template <int G>
HZL_HD void half_planes(const int d[32], uint32_t z[32], const Shifts& K) {
#pragma unroll
  for (int g = 0; g < G; g++) {
    const uint32_t sel = (uint32_t)g | ((4u + (uint32_t)g) << 4);  // byte g of a, of b
    uint32_t lo[4], hi[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int* o = d + 8 * u;
      lo[u] = prmt(prmt((uint32_t)o[0], (uint32_t)o[1], sel), prmt((uint32_t)o[2], (uint32_t)o[3], sel),
                   0x5410u);
      hi[u] = prmt(prmt((uint32_t)o[4], (uint32_t)o[5], sel), prmt((uint32_t)o[6], (uint32_t)o[7], sel),
                   0x5410u);
      tr8x8(lo[u], hi[u], K);  // byte t: bit 8g + t of the octet's 8 deltas
    }
    bt4x4(lo[0], lo[1], lo[2], lo[3], z + 8 * g);
    bt4x4(hi[0], hi[1], hi[2], hi[3], z + 8 * g + 4);
  }
}

// Two's-complement planes z[0 .. 8G-1] (values below 2^(8G-1) in magnitude,
// so plane 8G-1 is the sign) to the stream's sign-magnitude form: returns the
// sign half-word; z[p] becomes magnitude plane p for p < 8G - 1, with
// |d| = (d xor -s) + s as a bit-sliced carry chain. *nz gets bit p set when
// magnitude plane p is not zero.
template <int G>
HZL_HD uint32_t half_sign_magnitude(uint32_t z[32], uint32_t* nz) {
  constexpr int W = 8 * G - 1;
  const uint32_t s = z[W];
  uint32_t c = s, m = 0;
#pragma unroll
  for (int p = 0; p < W; p++) {
    const uint32_t t = z[p] ^ s;
    z[p] = t ^ c;
    c &= t;
    m |= (z[p] != 0u ? 1u : 0u) << p;
  }
  *nz = m;
  return s;
}

}  // namespace lanes
}  // namespace hz
