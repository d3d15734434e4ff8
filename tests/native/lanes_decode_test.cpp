// Host check of the two-lanes-per-block decode (hz_lanes.cuh) against brute
// force: random blocks of every rate 0..31 (Delta_0 := 0, signs on zero
// magnitudes, bits at position 0 that must be ignored, short last blocks, the
// narrow and wide accumulations), each decoded as two 32-position halves and
// recombined into the block's exact sums S1 = sum q and S2 = sum q^2.
// Then pairs of such blocks through the position-order prefixes (half_prefix
// for one block, half_visit for the other) into the covariance sums
// sum q_A q_B, sum q_A and sum q_B, narrow (8 products per 32-bit word) and
// wide. The device intrinsics (byte permute, high multiply) run as the
// header's host definitions.
#include <cstdint>
#include <cstdio>

#include "hz_lanes.cuh"

using namespace hz::lanes;

static uint64_t g_state = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() {
  g_state ^= g_state << 13;
  g_state ^= g_state >> 7;
  g_state ^= g_state << 17;
  return g_state;
}

template <int G, bool FULL, bool WIDE>
static HalfSums run(const uint32_t t[32], int nval, bool z0) {
  return half_sums<G, FULL, WIDE>(t, nval, z0, make_shifts(1u));
}
static HalfSums run_any(int G, bool full, bool wide, const uint32_t t[32], int nval, bool z0) {
  if (!full) wide = true;
  switch (G) {
    case 1: return !full ? run<1, false, true>(t, nval, z0) : wide ? run<1, true, true>(t, nval, z0) : run<1, true, false>(t, nval, z0);
    case 2: return !full ? run<2, false, true>(t, nval, z0) : wide ? run<2, true, true>(t, nval, z0) : run<2, true, false>(t, nval, z0);
    case 3: return !full ? run<3, false, true>(t, nval, z0) : wide ? run<3, true, true>(t, nval, z0) : run<3, true, false>(t, nval, z0);
    default: return !full ? run<4, false, true>(t, nval, z0) : wide ? run<4, true, true>(t, nval, z0) : run<4, true, false>(t, nval, z0);
  }
}

// A random block of rate r (widest rate of its warp Rw) and its values q.
struct Blk {
  long long O;
  uint64_t sign;
  uint32_t words[64];  // plane p's halves at 2p, 2p + 1
  long long q[64];
  int r;
};
static void gen_block(Blk& b, int Rw, bool qsmall) {
  int r = Rw ? (int)(rnd() % (Rw + 1)) : 0;
  if (rnd() % 4 == 0) r = Rw;
  const long long lim = qsmall ? (1ll << 13) - 1 : (1ll << 30) - 1;
  b.O = (long long)(rnd() % (2 * lim + 1)) - lim;
  uint64_t mag[64], planes[32] = {0};
  b.sign = 0;
  long long q = b.O;
  for (int i = 0; i < 64; i++) {
    long long m = r ? (long long)(rnd() & ((1ull << r) - 1)) : 0;
    long long d = (rnd() & 1) ? -m : m;
    if (i == 0) d = 0;
    if (q + d > lim || q + d < -lim) d = -d;
    if (q + d > lim) d = lim - q;
    if (q + d < -lim) d = -lim - q;
    q += d;
    b.q[i] = q;
    mag[i] = (uint64_t)(d < 0 ? -d : d);
    if (d < 0) b.sign |= 1ull << i;
    else if (r && d == 0 && rnd() % 7 == 0) b.sign |= 1ull << i;  // a sign on a zero magnitude
  }
  if (r && (rnd() % 2)) mag[0] = rnd() & ((1ull << r) - 1);  // ignored: Delta_0 := 0
  for (int p = 0; p < r; p++)
    for (int i = 0; i < 64; i++) planes[p] |= ((mag[i] >> p) & 1ull) << i;
  for (int p = 0; p < 32; p++) {
    b.words[2 * p] = (uint32_t)planes[p];
    b.words[2 * p + 1] = (uint32_t)(planes[p] >> 32);
  }
  b.r = r;
}

static void prefix_any(int G, const uint32_t t[32], bool z0, int p[32]) {
  const Shifts K = make_shifts(1u);
  switch (G) {
    case 1: half_prefix<1>(t, z0, K, p); break;
    case 2: half_prefix<2>(t, z0, K, p); break;
    case 3: half_prefix<3>(t, z0, K, p); break;
    default: half_prefix<4>(t, z0, K, p); break;
  }
}
template <class F>
static void visit_any(int G, const uint32_t t[32], bool z0, F&& f) {
  const Shifts K = make_shifts(1u);
  switch (G) {
    case 1: half_visit<1>(t, z0, K, f); break;
    case 2: half_visit<2>(t, z0, K, f); break;
    case 3: half_visit<3>(t, z0, K, f); break;
    default: half_visit<4>(t, z0, K, f); break;
  }
}

// Covariance sums of block pairs against brute force; returns the failures.
static long cov_pairs() {
  long fails = 0;
  for (int it = 0; it < 50000; it++) {
    const int RwA = (int)(rnd() % 32), RwB = (int)(rnd() % 32);
    const bool qsmall = (rnd() % 2) == 0;
    int len = 64;
    if (rnd() % 5 == 0) len = 1 + (int)(rnd() % 64);
    Blk A, B;
    gen_block(A, RwA, qsmall);
    gen_block(B, RwB, qsmall);
    __int128 SAB = 0, S1A = 0, S1B = 0;
    for (int i = 0; i < len; i++) {
      SAB += (__int128)A.q[i] * B.q[i];
      S1A += A.q[i];
      S1B += B.q[i];
    }
    const bool narrow = len == 64 && (qsmall || (RwA <= 8 && RwB <= 8));
    __int128 TAB = 0, T1A = 0, T1B = 0;
    int totA = 0, totB = 0;  // the first half's totals
    for (int h = 0; h < 2; h++) {
      const int nval = len - 32 * h < 0 ? 0 : (len - 32 * h > 32 ? 32 : len - 32 * h);
      uint32_t ta[32], tb[32];
      twos_planes_any(RwA, A.words + h, A.r, A.r ? (uint32_t)(A.sign >> (32 * h)) : 0u, ta);
      twos_planes_any(RwB, B.words + h, B.r, B.r ? (uint32_t)(B.sign >> (32 * h)) : 0u, tb);
      int pA[32];
      prefix_any((RwA + 8) >> 3, ta, h == 0, pA);
      long long spa = 0, spb = 0;
      __int128 pab = 0;
      int lastB = 0;
      if (narrow) {
        int x = 0, y = 0, acc = 0;
        long long s8 = 0;
        visit_any((RwB + 8) >> 3, tb, h == 0, [&](int i, int pb) {
          x += pA[i];
          y += pb;
          acc = (int)mad((uint32_t)pA[i], (uint32_t)pb, (uint32_t)acc);
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
        visit_any((RwB + 8) >> 3, tb, h == 0, [&](int i, int pb) {
          const long long xa = (i < nval) ? pA[i] : 0, yb = (i < nval) ? pb : 0;
          spa += xa;
          spb += yb;
          pab += (__int128)(xa * yb);
          if (i == 31) lastB = pb;
        });
      }
      const long long bA = A.O + (h ? totA : 0), bB = B.O + (h ? totB : 0);
      TAB += (__int128)nval * bA * bB + (__int128)bA * spb + (__int128)bB * spa + pab;
      T1A += (__int128)nval * bA + spa;
      T1B += (__int128)nval * bB + spb;
      totA = pA[31];
      totB = lastB;
    }
    if (TAB != SAB || T1A != S1A || T1B != S1B) {
      if (fails < 5) printf("cov differs: RwA %d RwB %d len %d narrow %d\n", RwA, RwB, len, (int)narrow);
      fails++;
    }
  }
  return fails;
}


// Encode of one half (half_planes + half_sign_magnitude) against brute force:
// magnitude planes and sign bits of 32 random deltas below 2^B in magnitude.
template <int G>
static bool encode_ok(const int d[32], int B) {
  uint32_t z[32] = {0};
  half_planes<G>(d, z, make_shifts(1u));
  uint32_t nz = 0;
  const uint32_t s = half_sign_magnitude<G>(z, &nz);
  uint32_t want_nz = 0;
  for (int i = 0; i < 32; i++) {
    if (((s >> i) & 1u) != (d[i] < 0 ? 1u : 0u)) return false;
  }
  for (int p = 0; p < 8 * G - 1; p++) {
    uint32_t w = 0;
    for (int i = 0; i < 32; i++) {
      const uint32_t a = (uint32_t)(d[i] < 0 ? -(long long)d[i] : d[i]);
      w |= ((a >> p) & 1u) << i;
    }
    if (w != z[p]) return false;
    if (w) want_nz |= 1u << p;
  }
  (void)B;
  return nz == want_nz;
}
static bool encode_any(int G, const int d[32], int B) {
  switch (G) {
    case 1: return encode_ok<1>(d, B);
    case 2: return encode_ok<2>(d, B);
    case 3: return encode_ok<3>(d, B);
    default: return encode_ok<4>(d, B);
  }
}

int main() {
  // the 8x8 bit transpose is a transpose
  for (int it = 0; it < 2000; it++) {
    const uint32_t lo = (uint32_t)rnd(), hi = (uint32_t)rnd();
    uint32_t a = lo, b = hi;
    tr8x8(a, b, make_shifts(1u));
    for (int t = 0; t < 8; t++)
      for (int k = 0; k < 8; k++) {
        const uint32_t in = (k < 4 ? lo >> (8 * k) : hi >> (8 * (k - 4))) & 0xffu;
        const uint32_t out = (t < 4 ? a >> (8 * t) : b >> (8 * (t - 4))) & 0xffu;
        if (((out >> k) & 1u) != ((in >> t) & 1u)) {
          printf("tr8x8 differs\n");
          return 1;
        }
      }
  }
  // encode of a half: every magnitude width 0..31, with the group count the
  // kernels use (8 G >= B + 1: the top plane is the sign)
  for (int it = 0; it < 20000; it++) {
    const int B = (int)(rnd() % 32);
    const int G = (B + 8) / 8;
    int d[32];
    for (int i = 0; i < 32; i++) {
      long long m = B ? (long long)(rnd() & ((1ull << B) - 1)) : 0;
      if (rnd() % 7 == 0) m = B ? (long long)((1ull << B) - 1) : 0;
      d[i] = (int)((rnd() & 1) ? -m : m);
    }
    if (!encode_any(G, d, B)) {
      printf("encode differs at B=%d\n", B);
      return 1;
    }
  }
  const long long QL = (1ll << 30) - 1;
  long fails = 0;
  for (int it = 0; it < 100000; it++) {
    const int Rw = (int)(rnd() % 32);
    int r = Rw ? (int)(rnd() % (Rw + 1)) : 0;
    if (rnd() % 4 == 0) r = Rw;
    int len = 64;
    if (rnd() % 5 == 0) len = 1 + (int)(rnd() % 64);
    const bool qsmall = (rnd() % 2) == 0;
    const long long lim = qsmall ? (1ll << 13) - 1 : QL;
    long long O = (long long)(rnd() % (2 * lim + 1)) - lim;
    uint64_t mag[64], sign = 0, planes[32] = {0};
    long long q = O;
    for (int i = 0; i < 64; i++) {
      long long m = r ? (long long)(rnd() & ((1ull << r) - 1)) : 0;
      long long d = (rnd() & 1) ? -m : m;
      if (i == 0) d = 0;
      if (q + d > lim || q + d < -lim) d = -d;
      if (q + d > lim) d = lim - q;
      if (q + d < -lim) d = -lim - q;
      q += d;
      mag[i] = (uint64_t)(d < 0 ? -d : d);
      if (d < 0) sign |= 1ull << i;
      else if (r && rnd() % 7 == 0) sign |= 1ull << i;  // a sign on a zero magnitude
      if (d > 0) sign &= ~(1ull << i);
    }
    if (r && (rnd() % 2)) mag[0] = rnd() & ((1ull << r) - 1);  // ignored: Delta_0 := 0
    for (int p = 0; p < r; p++)
      for (int i = 0; i < 64; i++) planes[p] |= ((mag[i] >> p) & 1ull) << i;
    __int128 S1 = 0, S2 = 0;
    long long v = O;
    for (int i = 0; i < len; i++) {
      const long long d = (i == 0) ? 0 : (((sign >> i) & 1) ? -(long long)mag[i] : (long long)mag[i]);
      v += d;
      S1 += v;
      S2 += (__int128)v * v;
    }
    uint32_t half_words[64];
    for (int p = 0; p < 32; p++) {
      half_words[2 * p] = (uint32_t)planes[p];
      half_words[2 * p + 1] = (uint32_t)(planes[p] >> 32);
    }
    const int G = (Rw + 8) >> 3;
    const bool wide = !(Rw <= 8 || qsmall) || (rnd() % 2);
    HalfSums hs[2];
    int nv[2];
    for (int h = 0; h < 2; h++) {
      uint32_t t[32];
      twos_planes_any(Rw, half_words + h, r, r ? (uint32_t)(sign >> (32 * h)) : 0u, t);
      nv[h] = len - 32 * h < 0 ? 0 : (len - 32 * h > 32 ? 32 : len - 32 * h);
      hs[h] = run_any(G, len == 64, wide, t, nv[h], h == 0);
    }
    __int128 T1 = 0, T2 = 0;
    for (int h = 0; h < 2; h++) {
      const long long base = O + (h ? hs[0].tot : 0);
      const __int128 sq = (wide || len != 64) ? (((__int128)hs[h].sqh << 64) | hs[h].sq)
                                             : (__int128)hs[h].sq;
      T1 += (__int128)nv[h] * base + hs[h].sp;
      T2 += (__int128)nv[h] * base * base + (__int128)2 * base * hs[h].sp + sq;
    }
    if (T1 != S1 || T2 != S2) {
      if (fails < 5) printf("differs: Rw %d r %d len %d\n", Rw, r, len);
      fails++;
    }
  }
  if (fails) {
    printf("%ld blocks differ\n", fails);
    return 1;
  }
  const long cfails = cov_pairs();
  if (cfails) {
    printf("%ld block pairs differ\n", cfails);
    return 1;
  }
  printf("ok\n");
  return 0;
}
