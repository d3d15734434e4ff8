/*
 * hoszp_omp.c — CPU throughput baseline: the oracle's codec and operators with
 * an OpenMP parallel loop over blocks, the organisation of the paper's own
 * CPU design (Sec. VI-A: SZp and HoSZp parallelised over blocks on a
 * multi-core node).
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the oracle it includes: its
 * arithmetic (exact Eq. 3, exact requantization, single-rounded
 * dequantization, exact sums) is the oracle's own functions; only the loops
 * over blocks run in parallel, and variable-length output is placed by a
 * prefix sum of the blocks' word counts (the stream stores no per-block
 * lengths, Sec. VI-B3). The benchmark times it on every host core beside the
 * single-threaded oracle; the tests check it byte for byte against the oracle.
 */
#include "hoszp_oracle.c"

#include <omp.h>

/* ------------------------------------------------------------------ */
/* block-parallel encode and decode                                    */
/* ------------------------------------------------------------------ */
static int blk_rate(const int64_t* q, uint64_t len) {
  uint64_t maxabs = 0;
  for (uint64_t i = 1; i < len; i++) {
    int64_t d = q[i] - q[i - 1];
    uint64_t a = (uint64_t)(d < 0 ? -d : d);
    if (a > maxabs) maxabs = a;
  }
  int r = 0;
  while (r < 64 && (maxabs >> r) != 0) r++;
  return r;
}

/* Encode q[0..n) (header fields from h_in except nnc, R). */
static int omp_encode_q(const int64_t* q, const orc_hdr* h_in, uint8_t* out, size_t cap,
                        uint64_t* out_bytes) {
  orc_hdr h = *h_in;
  const uint64_t n = h.n, nb = nblocks(n);
  uint8_t* rate = (uint8_t*)malloc(nb ? nb : 1);
  uint64_t* ncp = (uint64_t*)malloc(sizeof(uint64_t) * (nb + 1));
  uint64_t* rp = (uint64_t*)malloc(sizeof(uint64_t) * (nb + 1));
  if (!rate || !ncp || !rp) { free(rate); free(ncp); free(rp); return ORC_ERR_ARG; }
  int over = 0;
#pragma omp parallel for schedule(static) reduction(| : over)
  for (int64_t b = 0; b < (int64_t)nb; b++) {
    const uint64_t start = (uint64_t)b * ORC_L, len = (n - start < ORC_L) ? n - start : ORC_L;
    const int r = blk_rate(q + start, len);
    if (r > 31) over = 1;
    rate[b] = (uint8_t)(r > 31 ? 31 : r);
  }
  if (over) { free(rate); free(ncp); free(rp); return ORC_ERR_OVERFLOW; }
  ncp[0] = rp[0] = 0;
  for (uint64_t b = 0; b < nb; b++) { /* the placement prefix */
    ncp[b + 1] = ncp[b] + (rate[b] ? 1 : 0);
    rp[b + 1] = rp[b] + rate[b];
  }
  h.nnc = ncp[nb];
  h.R = rp[nb];
  const uint64_t size = stream_size(nb, h.nnc, h.R);
  if (size > cap) { free(rate); free(ncp); free(rp); return ORC_ERR_CAPACITY; }
  write_header(out, &h);
  memset(out + off_rate() + nb, 0, off_outlier(nb) - (off_rate() + nb));
  memset(out + off_outlier(nb) + 4 * nb, 0, off_sign(nb) - (off_outlier(nb) + 4 * nb));
  memset(out + off_plane(nb, h.nnc) + 8 * h.R, 0, size - (off_plane(nb, h.nnc) + 8 * h.R));
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < (int64_t)nb; b++) {
    const uint64_t start = (uint64_t)b * ORC_L, len = (n - start < ORC_L) ? n - start : ORC_L;
    const int64_t* qb = q + start;
    out[off_rate() + b] = rate[b];
    wr_le(out + off_outlier(nb) + 4 * b, (uint64_t)(uint32_t)(int32_t)qb[0], 4);
    if (rate[b] == 0) continue;
    uint64_t sign = 0, plane[31];
    memset(plane, 0, sizeof(plane));
    for (uint64_t i = 1; i < len; i++) {
      const int64_t d = qb[i] - qb[i - 1];
      const uint64_t a = (uint64_t)(d < 0 ? -d : d);
      if (d < 0) sign |= (uint64_t)1 << i;
      for (int p = 0; p < rate[b]; p++)
        if ((a >> p) & 1) plane[p] |= (uint64_t)1 << i;
    }
    wr_le(out + off_sign(nb) + 8 * ncp[b], sign, 8);
    for (int p = 0; p < rate[b]; p++) wr_le(out + off_plane(nb, h.nnc) + 8 * (rp[b] + p), plane[p], 8);
  }
  free(rate);
  free(ncp);
  free(rp);
  *out_bytes = size;
  return ORC_OK;
}

/* Decode to q[0..n) (header already read and checked). */
static int omp_decode_q(const uint8_t* c, const orc_hdr* h, int64_t* q) {
  const uint64_t n = h->n, nb = nblocks(n);
  uint64_t* ncp = (uint64_t*)malloc(sizeof(uint64_t) * (nb + 1));
  uint64_t* rp = (uint64_t*)malloc(sizeof(uint64_t) * (nb + 1));
  if (!ncp || !rp) { free(ncp); free(rp); return ORC_ERR_ARG; }
  ncp[0] = rp[0] = 0;
  for (uint64_t b = 0; b < nb; b++) {
    const uint8_t r = c[off_rate() + b];
    ncp[b + 1] = ncp[b] + (r ? 1 : 0);
    rp[b + 1] = rp[b] + r;
  }
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < (int64_t)nb; b++) {
    const uint64_t start = (uint64_t)b * ORC_L, len = (n - start < ORC_L) ? n - start : ORC_L;
    const int rate = c[off_rate() + b];
    const int64_t outlier = (int32_t)(uint32_t)rd_le(c + off_outlier(nb) + 4 * b, 4);
    q[start] = outlier;
    if (rate == 0) {
      for (uint64_t i = 1; i < len; i++) q[start + i] = outlier;
      continue;
    }
    const uint64_t sign = rd_le(c + off_sign(nb) + 8 * ncp[b], 8);
    uint64_t mag[ORC_L];
    memset(mag, 0, sizeof(mag));
    for (int p = 0; p < rate; p++) {
      const uint64_t plane = rd_le(c + off_plane(nb, h->nnc) + 8 * (rp[b] + p), 8);
      for (int i = 0; i < ORC_L; i++)
        if ((plane >> i) & 1) mag[i] |= (uint64_t)1 << p;
    }
    for (uint64_t i = 1; i < len; i++) {
      int64_t d = (int64_t)mag[i];
      if ((sign >> i) & 1) d = -d;
      q[start + i] = q[start + i - 1] + d;
    }
  }
  free(ncp);
  free(rp);
  return ORC_OK;
}

static int64_t* alloc_q(uint64_t n) { return (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1)); }

/* ------------------------------------------------------------------ */
/* codec                                                                */
/* ------------------------------------------------------------------ */
int omp_compress(const float* x, uint64_t n, const uint32_t* dims, int ndims, double eb,
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
    double mx = -INFINITY, mn = INFINITY;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(max : mx) reduction(min : mn) reduction(| : bad)
    for (int64_t i = 0; i < (int64_t)n; i++) {
      if (!isfinite(x[i])) bad = 1;
      const double v = (double)x[i];
      if (v > mx) mx = v;
      if (v < mn) mn = v;
    }
    if (bad) return ORC_ERR_NONFINITE;
    if (n == 0) mx = mn = 0;
    double range = mx - mn;
    if (range == 0) range = (fabs(mx) > 0) ? fabs(mx) : 1.0;
    eps = eb * range;
    if (orc_eps_q(eps, &h.eps_q) != ORC_OK) return ORC_ERR_RANGE;
  } else {
    if (orc_eps_q(eps, &h.eps_q) != ORC_OK) return ORC_ERR_ARG;
  }
  h.eps = eps;
  int64_t* q = alloc_q(n);
  if (!q) return ORC_ERR_ARG;
  int64_t qmax = 0;
  int err = 0;
#pragma omp parallel for schedule(static) reduction(max : qmax) reduction(min : err)
  for (int64_t i = 0; i < (int64_t)n; i++) {
    const int rc = orc_quantize(x[i], h.eps_q, &q[i]);
    if (rc) err = rc < err ? rc : err;
    const int64_t a = q[i] < 0 ? -q[i] : q[i];
    if (a > qmax) qmax = a;
  }
  if (err) { free(q); return err; }
  h.qbound = (uint32_t)qmax;
  const int rc = omp_encode_q(q, &h, out, cap, out_bytes);
  free(q);
  return rc;
}

int omp_decompress(const uint8_t* c, size_t bytes, float* x, uint64_t n) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  if (h.n != n) return ORC_ERR_MISMATCH;
  int64_t* q = alloc_q(n);
  if (!q) return ORC_ERR_ARG;
  rc = omp_decode_q(c, &h, q);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; i++) x[i] = orc_dequantize(q[i], h.eps_q);
  free(q);
  return rc;
}

/* ------------------------------------------------------------------ */
/* operators                                                            */
/* ------------------------------------------------------------------ */
static void par_copy(uint8_t* out, const uint8_t* c, uint64_t size) {
  const uint64_t chunk = 1 << 20;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)((size + chunk - 1) / chunk); k++) {
    const uint64_t a = (uint64_t)k * chunk, e = a + chunk < size ? a + chunk : size;
    memcpy(out + a, c + a, e - a);
  }
}

int omp_negate(const uint8_t* c, size_t bytes, uint8_t* out, size_t cap, uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  const uint64_t nb = nblocks(h.n), size = stream_size(nb, h.nnc, h.R);
  if (size > cap) return ORC_ERR_CAPACITY;
  par_copy(out, c, size);
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < (int64_t)nb; b++) {
    const int64_t o = (int32_t)(uint32_t)rd_le(out + off_outlier(nb) + 4 * b, 4);
    wr_le(out + off_outlier(nb) + 4 * b, (uint64_t)(uint32_t)(int32_t)(-o), 4);
  }
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < (int64_t)h.nnc; s++) {
    const uint64_t w = rd_le(out + off_sign(nb) + 8 * s, 8);
    wr_le(out + off_sign(nb) + 8 * s, ~w, 8);
  }
  *out_bytes = size;
  return ORC_OK;
}

int omp_add_scalar(const uint8_t* c, size_t bytes, double s, uint8_t* out, size_t cap,
                   uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  int64_t rho;
  rc = orc_quantize_scalar(s, h.eps_q, &rho);
  if (rc) return rc == ORC_ERR_ARG ? ORC_ERR_ARG : ORC_ERR_RANGE;
  const int64_t arho = rho < 0 ? -rho : rho;
  if ((int64_t)h.qbound + arho > ORC_QLIM) return ORC_ERR_OVERFLOW;
  const uint64_t nb = nblocks(h.n), size = stream_size(nb, h.nnc, h.R);
  if (size > cap) return ORC_ERR_CAPACITY;
  par_copy(out, c, size);
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < (int64_t)nb; b++) {
    const int64_t o = (int32_t)(uint32_t)rd_le(out + off_outlier(nb) + 4 * b, 4);
    wr_le(out + off_outlier(nb) + 4 * b, (uint64_t)(uint32_t)(int32_t)(o + rho), 4);
  }
  wr_le(out + 56, (uint64_t)(h.qbound + arho), 4);
  *out_bytes = size;
  return ORC_OK;
}

int omp_mul_scalar(const uint8_t* c, size_t bytes, double s, uint8_t* out, size_t cap,
                   uint64_t* out_bytes) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  int64_t rho;
  rc = orc_quantize_scalar(s, h.eps_q, &rho);
  if (rc) return rc == ORC_ERR_ARG ? ORC_ERR_ARG : ORC_ERR_RANGE;
  const uint64_t n = h.n;
  int64_t* q = alloc_q(n);
  if (!q) return ORC_ERR_ARG;
  omp_decode_q(c, &h, q);
  int64_t qmax = 0;
  int err = 0;
#pragma omp parallel for schedule(static) reduction(max : qmax) reduction(min : err)
  for (int64_t i = 0; i < (int64_t)n; i++) {
    int64_t r = 0;
    const int e = mul_requant(q[i], rho, h.eps_q, &r);
    if (e) err = e < err ? e : err;
    q[i] = r;
    const int64_t a = r < 0 ? -r : r;
    if (a > qmax) qmax = a;
  }
  if (err) { free(q); return err; }
  h.qbound = (uint32_t)qmax;
  rc = omp_encode_q(q, &h, out, cap, out_bytes);
  free(q);
  return rc;
}

int omp_add(const uint8_t* a, size_t a_bytes, const uint8_t* b, size_t b_bytes, uint8_t* out,
            size_t cap, uint64_t* out_bytes) {
  orc_hdr ha, hb;
  int rc = read_header(a, a_bytes, &ha);
  if (rc) return rc;
  rc = read_header(b, b_bytes, &hb);
  if (rc) return rc;
  if (ha.n != hb.n || float_to_bits(ha.eps_q) != float_to_bits(hb.eps_q)) return ORC_ERR_MISMATCH;
  if ((int64_t)ha.qbound + (int64_t)hb.qbound > ORC_QLIM) return ORC_ERR_OVERFLOW;
  const uint64_t n = ha.n;
  int64_t* qa = alloc_q(n);
  int64_t* qb = alloc_q(n);
  if (!qa || !qb) { free(qa); free(qb); return ORC_ERR_ARG; }
  omp_decode_q(a, &ha, qa);
  omp_decode_q(b, &hb, qb);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; i++) qa[i] += qb[i];
  orc_hdr h = ha;
  h.qbound = ha.qbound + hb.qbound;
  rc = omp_encode_q(qa, &h, out, cap, out_bytes);
  free(qa);
  free(qb);
  return rc;
}

/* Exact sums S1 = sum q and S2 = sum q^2 (Sec. V-B), per thread then added. */
int omp_sums(const uint8_t* c, size_t bytes, int64_t* s1_hi, uint64_t* s1_lo, uint64_t* s2_hi,
             uint64_t* s2_lo, uint64_t* n_out, float* eps_q_out) {
  orc_hdr h;
  int rc = read_header(c, bytes, &h);
  if (rc) return rc;
  const uint64_t n = h.n;
  int64_t* q = alloc_q(n);
  if (!q) return ORC_ERR_ARG;
  omp_decode_q(c, &h, q);
  i128 s1 = 0;
  u128 s2 = 0;
#pragma omp parallel
  {
    i128 t1 = 0;
    u128 t2 = 0;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; i++) {
      t1 += q[i];
      t2 += (u128)((i128)q[i] * q[i]);
    }
#pragma omp critical
    {
      s1 += t1;
      s2 += t2;
    }
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

int omp_threads(void) { return omp_get_max_threads(); }
