/*
 * hoszp_oracle.c — plain, slow, single-threaded CPU reference of the HoSZp codec
 * and its homomorphic operators (Agarwal et al., "HoSZp", arXiv 2408.11971).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library calls this file: it is
 * compiled and loaded by the tests, by the smoke check and by the CPU-baseline
 * leg of the benchmark, to say what the GPU path must produce. It shares no
 * code, header, table or helper with the CUDA path; it does not include the
 * public header, and restates the stream layout and error codes itself.
 *
 * Every operator below is written the slow, obvious way: the stream is decoded
 * to the quantized integers q, the integer definition is applied element by
 * element, and the result is encoded again block by block, bit by bit. Only
 * negation and scalar addition are (also) written as the paper's metadata-only
 * operations, because that is their definition (Sec. V-A).
 *
 * Readings of the paper taken here (listed with reasons in the design notes):
 *  - Eq. 3 is evaluated exactly (no rounding) on float32 x and on eps_q, the
 *    largest float32 not above the requested bound eps.
 *  - Blocks are L = 64 consecutive values of the flattened array (Table 6),
 *    the last block may be short; delta_0 := 0 and the first value is the
 *    outlier (Eq. 4 and the example of Sec. IV-A).
 *  - Bit-plane packing: plane p of a block is a 64-bit word whose bit i is bit
 *    p of |delta_i|; the sign word has bit i set iff delta_i < 0.
 *  - Section order of Fig. 3: rates, outliers, sign words, compressed bits.
 *  - Negation flips all 64 bits of every sign word and negates every outlier.
 *  - Scalars are quantized with Eq. 3 (rho_s); scalar multiplication applies
 *    Eq. 3 to the product of the dequantized values: q' = floor(2e*q*rho + 1/2).
 *  - Integer range: every stream keeps |q| <= 2^30-1; the compressor keeps
 *    |q| <= 2^23-2, the range in which its quantizer is exact on the GPU.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

/* error codes (same numbering as the library's ABI) */
enum {
  ORC_OK = 0,
  ORC_ERR_ARG = -1,
  ORC_ERR_CAPACITY = -2,
  ORC_ERR_FORMAT = -3,
  ORC_ERR_MISMATCH = -4,
  ORC_ERR_RANGE = -5,
  ORC_ERR_OVERFLOW = -6,
  ORC_ERR_NONFINITE = -7
};

#define ORC_L 64
#define ORC_MAGIC 0x505A5348u
#define ORC_VERSION 1
#define ORC_HDR 64
#define ORC_QMAX_COMPRESS 8388606LL /* 2^23 - 2 */
#define ORC_QLIM 1073741823LL       /* 2^30 - 1 */

/* ------------------------------------------------------------------ */
/* little-endian byte access (the stream is a byte array)               */
/* ------------------------------------------------------------------ */
static uint64_t rd_le(const uint8_t* p, int nbytes) {
  uint64_t v = 0;
  for (int i = nbytes - 1; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}
static void wr_le(uint8_t* p, uint64_t v, int nbytes) {
  for (int i = 0; i < nbytes; i++) { p[i] = (uint8_t)(v & 0xff); v >>= 8; }
}
static float bits_to_float(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t float_to_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }
static double bits_to_double(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t double_to_bits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }

static uint64_t align16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

/* ------------------------------------------------------------------ */
/* stream layout (Fig. 3)                                               */
/* ------------------------------------------------------------------ */
typedef struct {
  uint32_t ndims;
  uint32_t dims[3];
  float eps_q;
  uint64_t n;
  double eps;
  uint64_t nnc, R;
  uint32_t qbound;
} orc_hdr;

static uint64_t nblocks(uint64_t n) { return (n + ORC_L - 1) / ORC_L; }
static uint64_t off_rate(void) { return ORC_HDR; }
static uint64_t off_outlier(uint64_t nb) { return ORC_HDR + align16(nb); }
static uint64_t off_sign(uint64_t nb) { return off_outlier(nb) + align16(4 * nb); }
static uint64_t off_plane(uint64_t nb, uint64_t nnc) { return off_sign(nb) + 8 * nnc; }
/* the stream ends on a 16-byte boundary (8 zero bytes after the last plane
 * word when needed), so every section can be moved in 16-byte units */
static uint64_t stream_size(uint64_t nb, uint64_t nnc, uint64_t R) {
  return align16(off_plane(nb, nnc) + 8 * R);
}

size_t orc_bound(uint64_t n) {
  uint64_t nb = nblocks(n);
  return (size_t)(off_sign(nb) + 8 * nb * 32);
}

static void write_header(uint8_t* out, const orc_hdr* h) {
  memset(out, 0, ORC_HDR);
  wr_le(out + 0, ORC_MAGIC, 4);
  wr_le(out + 4, ORC_VERSION, 2);
  out[6] = 0; /* float32 */
  out[7] = (uint8_t)h->ndims;
  for (int d = 0; d < 3; d++) wr_le(out + 8 + 4 * d, h->dims[d], 4);
  wr_le(out + 20, float_to_bits(h->eps_q), 4);
  wr_le(out + 24, h->n, 8);
  wr_le(out + 32, double_to_bits(h->eps), 8);
  wr_le(out + 40, h->nnc, 8);
  wr_le(out + 48, h->R, 8);
  wr_le(out + 56, h->qbound, 4);
  wr_le(out + 60, ORC_L, 4);
}

/* Parse and validate a stream: header fields, section sizes against the byte
 * count, every rate <= 31, and the header's nnc and R against the rates. */
static int read_header(const uint8_t* c, size_t bytes, orc_hdr* h) {
  if (c == NULL || bytes < ORC_HDR) return ORC_ERR_FORMAT;
  if (rd_le(c, 4) != ORC_MAGIC || rd_le(c + 4, 2) != ORC_VERSION || c[6] != 0 ||
      rd_le(c + 60, 4) != ORC_L)
    return ORC_ERR_FORMAT;
  h->ndims = c[7];
  for (int d = 0; d < 3; d++) h->dims[d] = (uint32_t)rd_le(c + 8 + 4 * d, 4);
  h->eps_q = bits_to_float((uint32_t)rd_le(c + 20, 4));
  h->n = rd_le(c + 24, 8);
  h->eps = bits_to_double(rd_le(c + 32, 8));
  h->nnc = rd_le(c + 40, 8);
  h->R = rd_le(c + 48, 8);
  h->qbound = (uint32_t)rd_le(c + 56, 4);
  if (!(h->eps_q >= FLT_MIN && h->eps_q <= FLT_MAX / 2)) return ORC_ERR_FORMAT;
  if (h->qbound > ORC_QLIM) return ORC_ERR_FORMAT;
  uint64_t nb = nblocks(h->n);
  if (h->n > ((uint64_t)1 << 56) || h->nnc > nb || h->R > 31 * h->nnc) return ORC_ERR_FORMAT;
  if (stream_size(nb, h->nnc, h->R) > bytes) return ORC_ERR_FORMAT;
  uint64_t cnt = 0, sum = 0;
  for (uint64_t b = 0; b < nb; b++) {
    uint8_t r = c[off_rate() + b];
    if (r > 31) return ORC_ERR_FORMAT;
    if (r > 0) cnt++;
    sum += r;
  }
  if (cnt != h->nnc || sum != h->R) return ORC_ERR_FORMAT;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* error bound, quantization (Eq. 3) and dequantization                 */
/* ------------------------------------------------------------------ */

/* eps_q: the largest float32 that does not exceed eps (so |x - x'| stays within
 * the requested bound). Must be a normal float with 2*eps_q finite. */
int orc_eps_q(double eps, float* out) {
  if (!(eps > 0) || !isfinite(eps)) return ORC_ERR_ARG;
  float f = (float)eps; /* round to nearest */
  if ((double)f > eps) f = nextafterf(f, 0.0f);
  if (!(f >= FLT_MIN && f <= FLT_MAX / 2)) return ORC_ERR_ARG;
  *out = f;
  return ORC_OK;
}

/* Split a finite nonzero double into an odd-or-even integer mantissa m and an
 * exponent e with v = m * 2^e exactly (|m| < 2^53). */
static void split_double(double v, int64_t* m, int* e) {
  int ex;
  double fr = frexp(v, &ex); /* v = fr * 2^ex, 0.5 <= |fr| < 1 */
  *m = (int64_t)ldexp(fr, 53);
  *e = ex - 53;
}

/* Eq. 3, evaluated exactly: q = floor((v + e) / (2e)) for a real v given as a
 * double (a float32 value converts exactly) and e = eps_q > 0.
 * Write v = mv 2^ev, e = me 2^ee. Then (v + e)/(2e) = (mv 2^(ev-ee) + me)/(2 me),
 * and the floor of a ratio of integers is taken with integer division. */
static int quantize_exact(double v, float eps_q, int64_t limit, int64_t* q) {
  if (!isfinite(v)) return ORC_ERR_NONFINITE;
  double e = (double)eps_q;
  if (fabs(v) < e) { /* (v + e)/(2e) lies in (0, 1) */
    *q = 0;
    return ORC_OK;
  }
  /* |v| >= e here, and |v|/e must stay below 2 (limit + 1) for q to be in range */
  if (fabs(v) / e > 2.0 * (double)limit + 4.0) return ORC_ERR_RANGE;
  int64_t mv, me;
  int ev, ee;
  split_double(v, &mv, &ev);
  split_double(e, &me, &ee);
  int s = ev - ee; /* v/e = (mv/me) 2^s, with |v/e| < 2^32 so s < 32 + 54 */
  i128 num, den;
  if (s >= 0) {
    num = (i128)mv * ((i128)1 << s) + (i128)me;
    den = 2 * (i128)me;
  } else { /* multiply numerator and denominator by 2^-s */
    if (-s > 70) { *q = 0; return ORC_OK; } /* unreachable for |v| >= e */
    num = (i128)mv + (i128)me * ((i128)1 << (-s));
    den = 2 * (i128)me * ((i128)1 << (-s));
  }
  i128 qq = num / den; /* C division truncates toward zero */
  if ((num % den != 0) && (num < 0)) qq -= 1; /* floor for negative ratios */
  if (qq > limit || qq < -limit) return ORC_ERR_RANGE;
  *q = (int64_t)qq;
  return ORC_OK;
}

int orc_quantize(float x, float eps_q, int64_t* q) {
  return quantize_exact((double)x, eps_q, ORC_QMAX_COMPRESS, q);
}

/* Eq. 3 applied to a scalar operand s (Sec. V-A: "the quantized bin index of
 * the scalar"), allowed up to the stream range 2^30-1. */
int orc_quantize_scalar(double s, float eps_q, int64_t* q) {
  if (!isfinite(s)) return ORC_ERR_ARG;
  int rc = quantize_exact(s, eps_q, ORC_QLIM, q);
  return rc == ORC_ERR_NONFINITE ? ORC_ERR_ARG : rc;
}

/* Reverse quantization (proof of Theorem 1, step 2): x' = 2 eps_q * q, the real
 * product rounded ONCE to the nearest float32 (ties to even). Streams made by
 * the operators hold |q| up to 2^30-1, where float(q) itself would already
 * round; so the product is formed exactly as an integer P = q * M (2 eps_q =
 * M 2^E, M < 2^53) and P is rounded to 24 significant bits by integer shifts.
 * The scaling by 2^E is then exact: 2 eps_q >= 2^-148, so with M odd E >= -148
 * and every P 2^E is a multiple of 2^-148, which float32 holds while P has at
 * most 24 significant bits (the subnormal clamp below is kept for clarity and
 * never shortens the grid); a product beyond FLT_MAX rounds to infinity. */
float orc_dequantize(int64_t q, float eps_q) {
  if (q == 0) return 0.0f;
  int64_t M;
  int E;
  split_double(2.0 * (double)eps_q, &M, &E); /* 2 eps_q = M 2^E exactly */
  while ((M & 1) == 0) { /* odd M: fewer bits to carry */
    M >>= 1;
    E += 1;
  }
  const int neg = q < 0;
  u128 P = (u128)(neg ? -(i128)q : (i128)q) * (u128)M; /* exact, < 2^54 */
  int bits = 0;
  for (u128 t = P; t; t >>= 1) bits++;
  /* the float32 grid at the product's binade: 24 significant bits, but never
   * finer than 2^-149 (subnormals) */
  int keep_lsb = bits - 24;                           /* exponent of the grid step in P units */
  if (E + keep_lsb < -149) keep_lsb = -149 - E;       /* subnormal grid */
  if (keep_lsb > 0) {
    u128 rem = P & (((u128)1 << keep_lsb) - 1);
    u128 half = (u128)1 << (keep_lsb - 1);
    P >>= keep_lsb;
    if (rem > half || (rem == half && (P & 1))) P += 1; /* nearest, ties to even */
    E += keep_lsb;
  }
  /* P <= 2^24 now (2^24 after a carry), so (double)P is exact and so is the
   * scaling; the final conversion to float is exact unless the value lies
   * beyond FLT_MAX, where it gives infinity */
  double v = ldexp((double)P, E);
  float f = (float)v;
  return neg ? -f : f;
}

/* Scalar multiplication requantization (Sec. V-A example): q' = floor(2e*q*rho + 1/2),
 * evaluated exactly. With 2e = M 2^E (M integer): 2e*K = K*M*2^E for K = q*rho. */
static int mul_requant(int64_t q, int64_t rho, float eps_q, int64_t* out) {
  i128 K = (i128)q * (i128)rho; /* |K| < 2^61 */
  int64_t M;
  int E;
  split_double(2.0 * (double)eps_q, &M, &E);
  i128 KM = K * (i128)M; /* |KM| < 2^114 */
  i128 r;
  if (E >= 0) {
    if (KM != 0 && (E > 40 || (KM > 0 ? KM : -KM) > ((i128)ORC_QLIM >> E))) return ORC_ERR_OVERFLOW;
    r = KM * ((i128)1 << E);
  } else if (-E >= 120) {
    r = 0; /* |K M 2^E| < 2^-6 so floor(. + 1/2) = 0 */
  } else {
    int sh = -E;
    i128 num = 2 * KM + ((i128)1 << sh); /* 2^(sh+1) * (K M 2^E + 1/2) */
    i128 den = (i128)1 << (sh + 1);
    r = num / den;
    if ((num % den != 0) && (num < 0)) r -= 1;
  }
  if (r > ORC_QLIM || r < -ORC_QLIM) return ORC_ERR_OVERFLOW;
  *out = (int64_t)r;
  return ORC_OK;
}

int orc_mul_requant(int64_t q, int64_t rho, float eps_q, int64_t* out) {
  return mul_requant(q, rho, eps_q, out);
}

/* ------------------------------------------------------------------ */
/* blockwise encoding: Lorenzo (Eq. 4), signs, fixed length (BF)        */
/* ------------------------------------------------------------------ */

/* Encode integer values q[0..n) into a stream. `h` supplies the header fields
 * other than nnc and R, which are computed here. */
static int encode_q(const int64_t* q, const orc_hdr* h_in, uint8_t* out, size_t cap,
                    uint64_t* out_bytes) {
  orc_hdr h = *h_in;
  uint64_t n = h.n, nb = nblocks(n);
  uint8_t* rate = (uint8_t*)calloc(nb ? nb : 1, 1);
  if (!rate) return ORC_ERR_ARG;
  /* pass 1: rates (bit length of the largest |delta| in the block, Sec. IV-A step 3) */
  h.nnc = 0;
  h.R = 0;
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t start = b * ORC_L, len = (n - start < ORC_L) ? n - start : ORC_L;
    uint64_t maxabs = 0;
    for (uint64_t i = 1; i < len; i++) {
      int64_t d = q[start + i] - q[start + i - 1];
      uint64_t a = (uint64_t)(d < 0 ? -d : d);
      if (a > maxabs) maxabs = a;
    }
    int r = 0;
    while (r < 64 && (maxabs >> r) != 0) r++;
    if (r > 31) { free(rate); return ORC_ERR_OVERFLOW; }
    rate[b] = (uint8_t)r;
    if (r > 0) h.nnc++;
    h.R += (uint64_t)r;
  }
  uint64_t size = stream_size(nb, h.nnc, h.R);
  if (size > cap) { free(rate); return ORC_ERR_CAPACITY; }
  memset(out, 0, size);
  write_header(out, &h);
  uint64_t si = 0, pi = 0; /* running sign-word and plane-word indices */
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t start = b * ORC_L, len = (n - start < ORC_L) ? n - start : ORC_L;
    out[off_rate() + b] = rate[b];
    wr_le(out + off_outlier(nb) + 4 * b, (uint64_t)(uint32_t)(int32_t)q[start], 4);
    if (rate[b] == 0) continue; /* constant block: no sign word, no planes */
    uint64_t sign = 0;
    for (uint64_t i = 1; i < len; i++)
      if (q[start + i] - q[start + i - 1] < 0) sign |= (uint64_t)1 << i;
    wr_le(out + off_sign(nb) + 8 * si, sign, 8);
    si++;
    for (int p = 0; p < rate[b]; p++) {
      uint64_t plane = 0;
      for (uint64_t i = 1; i < len; i++) {
        int64_t d = q[start + i] - q[start + i - 1];
        uint64_t a = (uint64_t)(d < 0 ? -d : d);
        if ((a >> p) & 1) plane |= (uint64_t)1 << i;
      }
      wr_le(out + off_plane(nb, h.nnc) + 8 * pi, plane, 8);
      pi++;
    }
  }
  free(rate);
  *out_bytes = size;
  return ORC_OK;
}

/* Decode a stream to its integers: bit planes -> |delta|, sign -> delta, then
 * the inverse Lorenzo q_i = q_{i-1} + delta_i from the outlier (Sec. IV-B). */
static int decode_q(const uint8_t* c, size_t bytes, const orc_hdr* h, int64_t* q) {
  (void)bytes;
  uint64_t n = h->n, nb = nblocks(n);
  uint64_t si = 0, pi = 0;
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t start = b * ORC_L, len = (n - start < ORC_L) ? n - start : ORC_L;
    int rate = c[off_rate() + b];
    int64_t outlier = (int32_t)(uint32_t)rd_le(c + off_outlier(nb) + 4 * b, 4);
    q[start] = outlier;
    if (rate == 0) {
      for (uint64_t i = 1; i < len; i++) q[start + i] = outlier;
      continue;
    }
    uint64_t sign = rd_le(c + off_sign(nb) + 8 * si, 8);
    si++;
    uint64_t mag[ORC_L];
    memset(mag, 0, sizeof(mag));
    for (int p = 0; p < rate; p++) {
      uint64_t plane = rd_le(c + off_plane(nb, h->nnc) + 8 * pi, 8);
      pi++;
      for (int i = 0; i < ORC_L; i++)
        if ((plane >> i) & 1) mag[i] |= (uint64_t)1 << p;
    }
    for (uint64_t i = 1; i < len; i++) {
      int64_t d = (int64_t)mag[i];
      if ((sign >> i) & 1) d = -d;
      q[start + i] = q[start + i - 1] + d;
    }
  }
  return ORC_OK;
}

int orc_decode_q(const uint8_t* c, size_t bytes, int64_t* q, uint64_t n) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  if (h.n != n) return ORC_ERR_MISMATCH;
  return decode_q(c, bytes, &h, q);
}

/* ------------------------------------------------------------------ */
/* compression and decompression (Sec. IV-A, Fig. 2)                    */
/* ------------------------------------------------------------------ */
int orc_compress(const float* x, uint64_t n, const uint32_t* dims, int ndims, double eb,
                 int eb_mode, uint8_t* out, size_t cap, uint64_t* out_bytes) {
  if (out == NULL || out_bytes == NULL || (n > 0 && x == NULL)) return ORC_ERR_ARG;
  if (ndims < 1 || ndims > 3 || dims == NULL) return ORC_ERR_ARG;
  uint64_t prod = 1;
  for (int d = 0; d < ndims; d++) prod *= dims[d];
  if (prod != n) return ORC_ERR_ARG;
  if (!(eb > 0) || !isfinite(eb) || (eb_mode != 0 && eb_mode != 1)) return ORC_ERR_ARG;
  orc_hdr h;
  memset(&h, 0, sizeof(h));
  h.ndims = (uint32_t)ndims;
  for (int d = 0; d < ndims; d++) h.dims[d] = dims[d];
  h.n = n;
  double eps = eb;
  if (eb_mode == 1) {
    /* value-range-relative bound: eps = eb * (max - min) over the field */
    double mx = 0, mn = 0;
    for (uint64_t i = 0; i < n; i++) {
      if (!isfinite(x[i])) return ORC_ERR_NONFINITE;
      double v = (double)x[i];
      if (i == 0 || v > mx) mx = v;
      if (i == 0 || v < mn) mn = v;
    }
    double range = mx - mn;
    if (range == 0) range = (fabs(mx) > 0) ? fabs(mx) : 1.0; /* constant or empty field */
    eps = eb * range;
    if (orc_eps_q(eps, &h.eps_q) != ORC_OK) return ORC_ERR_RANGE;
  } else {
    if (orc_eps_q(eps, &h.eps_q) != ORC_OK) return ORC_ERR_ARG;
  }
  h.eps = eps;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!q) return ORC_ERR_ARG;
  int64_t qmax = 0;
  for (uint64_t i = 0; i < n; i++) {
    int rc = orc_quantize(x[i], h.eps_q, &q[i]);
    if (rc) { free(q); return rc; }
    int64_t a = q[i] < 0 ? -q[i] : q[i];
    if (a > qmax) qmax = a;
  }
  h.qbound = (uint32_t)qmax;
  int rc = encode_q(q, &h, out, cap, out_bytes);
  free(q);
  return rc;
}

int orc_decompress(const uint8_t* c, size_t bytes, float* x, uint64_t n) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  if (h.n != n) return ORC_ERR_MISMATCH;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!q) return ORC_ERR_ARG;
  decode_q(c, bytes, &h, q);
  for (uint64_t i = 0; i < n; i++) x[i] = orc_dequantize(q[i], h.eps_q);
  free(q);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* workflow 1: negation and scalar addition on the metadata (Sec. V-A)  */
/* ------------------------------------------------------------------ */
int orc_negate(const uint8_t* c, size_t bytes, uint8_t* out, size_t cap, uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  uint64_t nb = nblocks(h.n), size = stream_size(nb, h.nnc, h.R);
  if (size > cap) return ORC_ERR_CAPACITY;
  memmove(out, c, size);
  for (uint64_t b = 0; b < nb; b++) { /* outliers carry the first value's sign */
    int64_t o = (int32_t)(uint32_t)rd_le(out + off_outlier(nb) + 4 * b, 4);
    wr_le(out + off_outlier(nb) + 4 * b, (uint64_t)(uint32_t)(int32_t)(-o), 4);
  }
  for (uint64_t s = 0; s < h.nnc; s++) { /* logical NOT of every sign bit */
    uint64_t w = rd_le(out + off_sign(nb) + 8 * s, 8);
    wr_le(out + off_sign(nb) + 8 * s, ~w, 8);
  }
  *out_bytes = size;
  return ORC_OK;
}

int orc_add_scalar(const uint8_t* c, size_t bytes, double s, uint8_t* out, size_t cap,
                   uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  int64_t rho;
  rc = orc_quantize_scalar(s, h.eps_q, &rho);
  if (rc) return rc == ORC_ERR_ARG ? ORC_ERR_ARG : ORC_ERR_RANGE;
  int64_t arho = rho < 0 ? -rho : rho;
  if ((int64_t)h.qbound + arho > ORC_QLIM) return ORC_ERR_OVERFLOW;
  uint64_t nb = nblocks(h.n), size = stream_size(nb, h.nnc, h.R);
  if (size > cap) return ORC_ERR_CAPACITY;
  memmove(out, c, size);
  for (uint64_t b = 0; b < nb; b++) { /* O' = O + rho_s for every block */
    int64_t o = (int32_t)(uint32_t)rd_le(out + off_outlier(nb) + 4 * b, 4);
    wr_le(out + off_outlier(nb) + 4 * b, (uint64_t)(uint32_t)(int32_t)(o + rho), 4);
  }
  wr_le(out + 56, (uint64_t)(h.qbound + arho), 4);
  *out_bytes = size;
  return ORC_OK;
}

/* Scalar subtraction (Sec. V-A "Scalar Subtraction"): the scalar's bin
 * rho_s (Eq. 3 applied to s) is deducted from every block's outlier,
 * O' = O - rho_s; the rest of the stream is copied. The result bound is
 * qbound + |rho_s|. */
int orc_sub_scalar(const uint8_t* c, size_t bytes, double s, uint8_t* out, size_t cap,
                   uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  int64_t rho;
  rc = orc_quantize_scalar(s, h.eps_q, &rho);
  if (rc) return rc == ORC_ERR_ARG ? ORC_ERR_ARG : ORC_ERR_RANGE;
  int64_t arho = rho < 0 ? -rho : rho;
  if ((int64_t)h.qbound + arho > ORC_QLIM) return ORC_ERR_OVERFLOW;
  uint64_t nb = nblocks(h.n), size = stream_size(nb, h.nnc, h.R);
  if (size > cap) return ORC_ERR_CAPACITY;
  memmove(out, c, size);
  for (uint64_t b = 0; b < nb; b++) {
    int64_t o = (int32_t)(uint32_t)rd_le(out + off_outlier(nb) + 4 * b, 4);
    wr_le(out + off_outlier(nb) + 4 * b, (uint64_t)(uint32_t)(int32_t)(o - rho), 4);
  }
  wr_le(out + 56, (uint64_t)(h.qbound + arho), 4);
  *out_bytes = size;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* workflows 2 and 3, written as decode -> integer op -> encode          */
/* ------------------------------------------------------------------ */

/* Scalar multiplication (Sec. V-A): q' = floor(2e q rho_s + 1/2), re-encoded. */
int orc_mul_scalar(const uint8_t* c, size_t bytes, double s, uint8_t* out, size_t cap,
                   uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  int64_t rho;
  rc = orc_quantize_scalar(s, h.eps_q, &rho);
  if (rc) return rc == ORC_ERR_ARG ? ORC_ERR_ARG : ORC_ERR_RANGE;
  uint64_t n = h.n;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!q) return ORC_ERR_ARG;
  decode_q(c, bytes, &h, q);
  int64_t qmax = 0;
  for (uint64_t i = 0; i < n; i++) {
    int64_t r;
    rc = mul_requant(q[i], rho, h.eps_q, &r);
    if (rc) { free(q); return rc; }
    q[i] = r;
    if ((r < 0 ? -r : r) > qmax) qmax = r < 0 ? -r : r;
  }
  h.qbound = (uint32_t)qmax;
  rc = encode_q(q, &h, out, cap, out_bytes);
  free(q);
  return rc;
}

/* Scalar multiplication by the scalar itself (the variant that avoids the
 * scalar's quantization; Sec. V-A multiplies by the bin rho_s instead):
 * q' = floor(q s + 1/2), evaluated exactly (s = M 2^E with a 53-bit M). Unlike
 * the paper's form, a scalar below eps does not collapse the field to zero. */
static int mul_requant_s(int64_t q, double s, int64_t* out) {
  if (q == 0 || s == 0.0) { *out = 0; return ORC_OK; }
  int64_t M;
  int E;
  split_double(s, &M, &E);     /* s = M 2^E, |M| < 2^53 */
  i128 KM = (i128)q * (i128)M; /* |KM| < 2^84 */
  i128 r;
  if (E >= 0) {
    if (E > 40 || (KM > 0 ? KM : -KM) > ((i128)ORC_QLIM >> E)) return ORC_ERR_OVERFLOW;
    r = KM * ((i128)1 << E);
  } else if (-E >= 120) {
    r = 0; /* |q s| < 2^-36 */
  } else {
    int sh = -E;
    i128 num = 2 * KM + ((i128)1 << sh); /* 2^(sh+1) (q s + 1/2) */
    i128 den = (i128)1 << (sh + 1);
    r = num / den;
    if ((num % den != 0) && (num < 0)) r -= 1;
  }
  if (r > ORC_QLIM || r < -ORC_QLIM) return ORC_ERR_OVERFLOW;
  *out = (int64_t)r;
  return ORC_OK;
}

int orc_mul_scalar_exact(const uint8_t* c, size_t bytes, double s, uint8_t* out, size_t cap,
                         uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  if (!isfinite(s)) return ORC_ERR_ARG;
  uint64_t n = h.n;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!q) return ORC_ERR_ARG;
  decode_q(c, bytes, &h, q);
  int64_t qmax = 0;
  for (uint64_t i = 0; i < n; i++) {
    int64_t r;
    rc = mul_requant_s(q[i], s, &r);
    if (rc) { free(q); return rc; }
    q[i] = r;
    if ((r < 0 ? -r : r) > qmax) qmax = r < 0 ? -r : r;
  }
  h.qbound = (uint32_t)qmax;
  rc = encode_q(q, &h, out, cap, out_bytes);
  free(q);
  return rc;
}

/* Element-wise addition (Sec. V-C): O' = O_A + O_B and delta' = delta_A + delta_B,
 * i.e. q' = q_A + q_B, re-encoded. The result bound is qbound_A + qbound_B. */
int orc_add(const uint8_t* a, size_t a_bytes, const uint8_t* b, size_t b_bytes, uint8_t* out,
            size_t cap, uint64_t* out_bytes) {
  orc_hdr ha, hb;
  int rc = read_header(a, a_bytes, &ha);
  if (rc) return rc;
  rc = read_header(b, b_bytes, &hb);
  if (rc) return rc;
  if (ha.n != hb.n || float_to_bits(ha.eps_q) != float_to_bits(hb.eps_q)) return ORC_ERR_MISMATCH;
  if ((int64_t)ha.qbound + (int64_t)hb.qbound > ORC_QLIM) return ORC_ERR_OVERFLOW;
  uint64_t n = ha.n;
  int64_t* qa = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  int64_t* qb = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!qa || !qb) { free(qa); free(qb); return ORC_ERR_ARG; }
  decode_q(a, a_bytes, &ha, qa);
  decode_q(b, b_bytes, &hb, qb);
  for (uint64_t i = 0; i < n; i++) qa[i] += qb[i];
  orc_hdr h = ha;
  h.qbound = ha.qbound + hb.qbound;
  rc = encode_q(qa, &h, out, cap, out_bytes);
  free(qa);
  free(qb);
  return rc;
}

/* Hadamard product (Sec. V-C "Hadamard Product": like the scalar
 * multiplication, with the other field's quantized values in place of the
 * scalar's bin): q' = floor(2e q_A q_B + 1/2), Eq. 3 applied to the product of
 * the dequantized values, re-encoded. The streams must agree in n and eps_q. */
int orc_hadamard(const uint8_t* a, size_t a_bytes, const uint8_t* b, size_t b_bytes,
                 uint8_t* out, size_t cap, uint64_t* out_bytes) {
  orc_hdr ha, hb;
  int rc = read_header(a, a_bytes, &ha);
  if (rc) return rc;
  rc = read_header(b, b_bytes, &hb);
  if (rc) return rc;
  if (ha.n != hb.n || float_to_bits(ha.eps_q) != float_to_bits(hb.eps_q)) return ORC_ERR_MISMATCH;
  uint64_t n = ha.n;
  int64_t* qa = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  int64_t* qb = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!qa || !qb) { free(qa); free(qb); return ORC_ERR_ARG; }
  decode_q(a, a_bytes, &ha, qa);
  decode_q(b, b_bytes, &hb, qb);
  int64_t qmax = 0;
  for (uint64_t i = 0; i < n; i++) {
    int64_t r;
    rc = mul_requant(qa[i], qb[i], ha.eps_q, &r);
    if (rc) { free(qa); free(qb); return rc; }
    qa[i] = r;
    if ((r < 0 ? -r : r) > qmax) qmax = r < 0 ? -r : r;
  }
  orc_hdr h = ha;
  h.qbound = (uint32_t)qmax;
  rc = encode_q(qa, &h, out, cap, out_bytes);
  free(qa);
  free(qb);
  return rc;
}

/* Element-wise subtraction (Sec. V-C, "Element-wise Subtraction"): as the
 * addition with B's quantized values negated, q' = q_A - q_B, re-encoded. The
 * result bound is qbound_A + qbound_B. */
int orc_sub(const uint8_t* a, size_t a_bytes, const uint8_t* b, size_t b_bytes, uint8_t* out,
            size_t cap, uint64_t* out_bytes) {
  orc_hdr ha, hb;
  int rc = read_header(a, a_bytes, &ha);
  if (rc) return rc;
  rc = read_header(b, b_bytes, &hb);
  if (rc) return rc;
  if (ha.n != hb.n || float_to_bits(ha.eps_q) != float_to_bits(hb.eps_q)) return ORC_ERR_MISMATCH;
  if ((int64_t)ha.qbound + (int64_t)hb.qbound > ORC_QLIM) return ORC_ERR_OVERFLOW;
  uint64_t n = ha.n;
  int64_t* qa = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  int64_t* qb = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!qa || !qb) { free(qa); free(qb); return ORC_ERR_ARG; }
  decode_q(a, a_bytes, &ha, qa);
  decode_q(b, b_bytes, &hb, qb);
  for (uint64_t i = 0; i < n; i++) qa[i] -= qb[i];
  orc_hdr h = ha;
  h.qbound = ha.qbound + hb.qbound;
  rc = encode_q(qa, &h, out, cap, out_bytes);
  free(qa);
  free(qb);
  return rc;
}

/* ------------------------------------------------------------------ */
/* reductions (Sec. V-B): exact integer sums; the caller finishes them  */
/* ------------------------------------------------------------------ */

/* S1 = sum q (signed 128-bit, returned as hi:lo words) and S2 = sum q^2
 * (unsigned 128-bit). Also returns n and eps_q so mean and variance can be
 * formed from exact rationals. */
int orc_sums(const uint8_t* c, size_t bytes, int64_t* s1_hi, uint64_t* s1_lo, uint64_t* s2_hi,
             uint64_t* s2_lo, uint64_t* n_out, float* eps_q_out) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  uint64_t n = h.n;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!q) return ORC_ERR_ARG;
  decode_q(c, bytes, &h, q);
  i128 s1 = 0;
  u128 s2 = 0;
  for (uint64_t i = 0; i < n; i++) {
    s1 += q[i];
    s2 += (u128)((i128)q[i] * q[i]);
  }
  free(q);
  *s1_hi = (int64_t)(s1 >> 64);
  *s1_lo = (uint64_t)s1;
  *s2_hi = (uint64_t)(s2 >> 64);
  *s2_lo = (uint64_t)s2;
  *n_out = n;
  *eps_q_out = h.eps_q;
  return ORC_OK;
}

/* Block-wise means (Sec. V-B "Mean", last sentences): the quantized values
 * of each block are summed and the sum is divided by the number of values in
 * the block, then scaled by 2 eps_q: mean_b = (S1_b / L_b) * 2 eps_q in FP64
 * (S1_b exact, |S1_b| < 2^37; the same two rounded operations as the mean of
 * the whole stream). out has nb = ceil(n / 64) doubles. */
int orc_block_means(const uint8_t* c, size_t bytes, double* out, uint64_t nb_out) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  uint64_t n = h.n, nb = nblocks(n);
  if (nb_out != nb) return ORC_ERR_ARG;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!q) return ORC_ERR_ARG;
  decode_q(c, bytes, &h, q);
  const double e2 = 2.0 * (double)h.eps_q;
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t i0 = b * ORC_L, i1 = i0 + ORC_L < n ? i0 + ORC_L : n;
    int64_t s1 = 0;
    for (uint64_t i = i0; i < i1; i++) s1 += q[i];
    out[b] = ((double)s1 / (double)(i1 - i0)) * e2;
  }
  free(q);
  return ORC_OK;
}

/* The exact sums behind the covariance of two streams of the same length
 * (Sec. V-D "Covariance", done like the variance of Sec. V-B over two
 * fields): S_AB = sum q_A q_B (signed 128-bit), S1_A = sum q_A, S1_B = sum q_B.
 * The population covariance is 2 eps_A 2 eps_B (n S_AB - S1_A S1_B) / n^2.
 * The two streams may have different error bounds; their lengths must agree. */
int orc_cov_sums(const uint8_t* a, size_t a_bytes, const uint8_t* b, size_t b_bytes,
                 int64_t* sab_hi, uint64_t* sab_lo, int64_t* s1a_hi, uint64_t* s1a_lo,
                 int64_t* s1b_hi, uint64_t* s1b_lo, uint64_t* n_out) {
  orc_hdr ha, hb;
  int rc = read_header(a, a_bytes, &ha);
  if (rc) return rc;
  rc = read_header(b, b_bytes, &hb);
  if (rc) return rc;
  if (ha.n != hb.n) return ORC_ERR_MISMATCH;
  uint64_t n = ha.n;
  int64_t* qa = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  int64_t* qb = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!qa || !qb) { free(qa); free(qb); return ORC_ERR_ARG; }
  decode_q(a, a_bytes, &ha, qa);
  decode_q(b, b_bytes, &hb, qb);
  i128 sab = 0, sa = 0, sb = 0;
  for (uint64_t i = 0; i < n; i++) {
    sab += (i128)qa[i] * qb[i];
    sa += qa[i];
    sb += qb[i];
  }
  free(qa);
  free(qb);
  *sab_hi = (int64_t)(sab >> 64);
  *sab_lo = (uint64_t)sab;
  *s1a_hi = (int64_t)(sa >> 64);
  *s1a_lo = (uint64_t)sa;
  *s1b_hi = (int64_t)(sb >> 64);
  *s1b_lo = (uint64_t)sb;
  *n_out = n;
  return ORC_OK;
}

/* Header fields, for tests. */
/* Streams of consecutive shards of one field joined into the field's stream
 * (Sec. VI-B5: the nodes' compressed data gathered at a root). The plain
 * definition: decode every shard to its integers, join them in order, and
 * encode the whole field. Shards must share eps_q and eps bits (MISMATCH),
 * and every shard but the last must hold whole blocks (MISMATCH); dims give
 * the field's shape (their product must be the total n, else ARG). The header's
 * qbound is the largest of the shards'. */
int orc_concat(uint32_t k, const uint8_t* const* streams, const size_t* bytes,
               const uint32_t* dims, int ndims, uint8_t* out, size_t cap, uint64_t* out_bytes) {
  if (k == 0 || ndims < 1 || ndims > 3) return ORC_ERR_ARG;
  orc_hdr h0, hk;
  uint64_t n = 0;
  uint32_t qb = 0;
  for (uint32_t s = 0; s < k; s++) {
    int rc = read_header(streams[s], bytes[s], &hk);
    if (rc) return rc;
    if (s == 0) h0 = hk;
    if (float_to_bits(hk.eps_q) != float_to_bits(h0.eps_q) ||
        double_to_bits(hk.eps) != double_to_bits(h0.eps))
      return ORC_ERR_MISMATCH;
    if (s + 1 < k && hk.n % ORC_L != 0) return ORC_ERR_MISMATCH;
    n += hk.n;
    if (hk.qbound > qb) qb = hk.qbound;
  }
  uint64_t prod = 1;
  for (int d = 0; d < ndims; d++) prod *= dims[d];
  if (prod != n) return ORC_ERR_ARG;
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!q) return ORC_ERR_ARG;
  uint64_t at = 0;
  for (uint32_t s = 0; s < k; s++) {
    read_header(streams[s], bytes[s], &hk);
    decode_q(streams[s], bytes[s], &hk, q + at);
    at += hk.n;
  }
  orc_hdr h = h0;
  h.n = n;
  h.ndims = (uint32_t)ndims;
  for (int d = 0; d < 3; d++) h.dims[d] = d < ndims ? dims[d] : 0;
  h.qbound = qb;
  int rc = encode_q(q, &h, out, cap, out_bytes);
  free(q);
  return rc;
}

int orc_header(const uint8_t* c, size_t bytes, uint64_t* n, uint64_t* nnc, uint64_t* R,
               uint32_t* qbound, float* eps_q, uint64_t* size) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  *n = h.n;
  *nnc = h.nnc;
  *R = h.R;
  *qbound = h.qbound;
  *eps_q = h.eps_q;
  *size = stream_size(nblocks(h.n), h.nnc, h.R);
  return ORC_OK;
}
