// api.cu — the C ABI of libhoszp (declared in include/hoszp.h): argument
// checks, the context's device workspace, and kernel launches.
#include <cfloat>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "hz_kernels.cuh"
#include "hz_ws.cuh"

using namespace hz;

struct hoszp_ctx {
  int device;
  int num_sms;
  void* ws_mem;
  size_t ws_bytes;
  uint64_t ws_tiles, ws_staging_words, ws_grid;
  Ws ws;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// Largest float32 <= eps, or 0 when eps is not a usable bound.
float eps_q_of(double eps) {
  if (!(eps > 0) || !std::isfinite(eps)) return 0.0f;
  float f = (float)eps;
  if ((double)f > eps) f = std::nextafter(f, 0.0f);
  if (!(f >= FLT_MIN && f <= FLT_MAX / 2)) return 0.0f;
  return f;
}

// Size the workspace for `tiles` tiles and `staging_words` plane words; grows
// (never shrinks) by freeing and reallocating, which synchronizes the device.
int ensure_ws(hoszp_ctx* c, uint64_t tiles, uint64_t staging_words) {
  const uint64_t grid = (uint64_t)c->num_sms * 8;  // upper bound of any persistent grid
  tiles = tiles < 1 ? 1 : tiles;
  if (c->ws_mem && tiles <= c->ws_tiles && staging_words <= c->ws_staging_words &&
      grid <= c->ws_grid)
    return HOSZP_OK;
  tiles = tiles > c->ws_tiles ? tiles : c->ws_tiles;
  staging_words = staging_words > c->ws_staging_words ? staging_words : c->ws_staging_words;
  staging_words = staging_words < 16 ? 16 : staging_words;
  // layout: sync | status | totals | eps_q, eps | hdr | desc x3 | pre x3 | agg | cta_agg |
  // partials | range | staging
  uint64_t off = 0;
  const uint64_t o_sync = off;
  off += 256;
  const uint64_t o_status = off;
  off += 256;
  const uint64_t o_totals = off;
  off += 256;
  const uint64_t o_eps = off;
  off += 256;
  const uint64_t o_hdr = off;
  off += 256;
  uint64_t o_desc[NCHAIN];
  for (int k = 0; k < NCHAIN; k++) {
    o_desc[k] = off;
    off = round_up(off + tiles * sizeof(Desc), 256);
  }
  uint64_t o_pre[3];
  for (int k = 0; k < 3; k++) {
    o_pre[k] = off;
    off = round_up(off + (tiles + 1) * 16, 256);
  }
  const uint64_t o_agg = off;
  off = round_up(off + (tiles + 1) * 8, 256);
  const uint64_t o_cagg = off;
  off = round_up(off + 2 * grid * sizeof(CtaAgg), 256);  // two streams per CTA (addition)
  const uint64_t o_part = off;
  off = round_up(off + grid * sizeof(Partial), 256);
  const uint64_t o_range = off;
  off = round_up(off + grid * 3 * sizeof(float), 256);
  const uint64_t o_stage = off;
  off = round_up(off + staging_words * 8, 256);

  // keep the epoch across reallocations so stale descriptors never match
  unsigned long long epoch = 1;
  if (c->ws_mem) {
    Sync s;
    if (cudaMemcpy(&s, c->ws.sync, sizeof(Sync), cudaMemcpyDeviceToHost) == cudaSuccess)
      epoch = s.epoch + 1;
    cudaFree(c->ws_mem);
    c->ws_mem = nullptr;
  }
  void* mem = nullptr;
  if (cudaMalloc(&mem, off) != cudaSuccess) {
    cudaGetLastError();
    c->ws_bytes = 0;
    c->ws_tiles = c->ws_staging_words = c->ws_grid = 0;
    return HOSZP_ERR_CUDA;
  }
  // zero the bookkeeping and the descriptors (flags 0 never match an epoch >= 1)
  if (cudaMemset(mem, 0, o_part) != cudaSuccess) return HOSZP_ERR_CUDA;
  uint8_t* base = (uint8_t*)mem;
  c->ws_mem = mem;
  c->ws_bytes = off;
  c->ws_tiles = tiles;
  c->ws_staging_words = staging_words;
  c->ws_grid = grid;
  Ws& w = c->ws;
  w.sync = (Sync*)(base + o_sync);
  w.status = (int*)(base + o_status);
  w.totals = (unsigned long long*)(base + o_totals);
  w.eps_q = (float*)(base + o_eps);
  w.eps = (double*)(base + o_eps + 8);
  w.hdr = (hoszp_header*)(base + o_hdr);
  for (int k = 0; k < NCHAIN; k++) w.desc[k] = (Desc*)(base + o_desc[k]);
  w.max_tiles = tiles;
  for (int k = 0; k < 2; k++) w.pre[k] = (unsigned long long*)(base + o_pre[k]);
  w.opre = (unsigned long long*)(base + o_pre[2]);
  w.agg = (unsigned long long*)(base + o_agg);
  w.partials = (Partial*)(base + o_part);
  w.cta_agg = (CtaAgg*)(base + o_cagg);
  w.range_part = (float*)(base + o_range);
  w.max_grid = grid;
  w.staging = (uint64_t*)(base + o_stage);
  w.staging_words = staging_words;
  Sync s0 = {0u, 0u, epoch};
  if (cudaMemcpy(w.sync, &s0, sizeof(Sync), cudaMemcpyHostToDevice) != cudaSuccess)
    return HOSZP_ERR_CUDA;
  return HOSZP_OK;
}

// Tiles of a stream whose block count is unknown on the host: each block
// stores at least its rate byte and its 4-byte outlier.
uint64_t tiles_from_bytes(uint64_t bytes) {
  const uint64_t nb = bytes > HOSZP_HEADER_BYTES ? (bytes - HOSZP_HEADER_BYTES) / 5 + 1 : 1;
  return ntiles_of(nb) + 1;
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
inline bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

inline int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return HOSZP_OK;
  cudaGetLastError();
  return HOSZP_ERR_CUDA;
}

Launch lc_of(hoszp_ctx* c, hoszp_stream_t s) {
  Launch l;
  l.grid = c->num_sms;
  l.stream = (cudaStream_t)s;
  return l;
}

}  // namespace

extern "C" {

int hoszp_ctx_create(hoszp_ctx** ctx, int device) {
  if (!ctx) return HOSZP_ERR_ARG;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HOSZP_ERR_ARG;
  }
  DeviceGuard g(device);
  hoszp_ctx* c = new (std::nothrow) hoszp_ctx();
  if (!c) return HOSZP_ERR_CUDA;
  c->device = device;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return HOSZP_ERR_CUDA;
  }
  int rc = ensure_ws(c, 1, 16);
  if (rc != HOSZP_OK) {
    delete c;
    return rc;
  }
  *ctx = c;
  return HOSZP_OK;
}

void hoszp_ctx_destroy(hoszp_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws_mem) cudaFree(ctx->ws_mem);
  delete ctx;
}

int hoszp_ctx_reserve(hoszp_ctx* ctx, uint64_t n) {
  if (!ctx) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  const uint64_t nb = nblocks(n);
  return ensure_ws(ctx, ntiles_of(nb) + 1, 31 * nb + 16);
}

int hoszp_get_status(hoszp_ctx* ctx, int* status) {
  if (!ctx || !status) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    *status = HOSZP_ERR_CUDA;
    return HOSZP_ERR_CUDA;
  }
  int v = 0;
  if (cudaMemcpy(&v, ctx->ws.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(ctx->ws.status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    *status = HOSZP_ERR_CUDA;
    return HOSZP_ERR_CUDA;
  }
  *status = v;
  return HOSZP_OK;
}

size_t hoszp_compress_bound(uint64_t n) {
  const uint64_t nb = nblocks(n);
  return (size_t)(off_sign(nb) + 8ull * nb * 32ull);
}

int hoszp_compress(hoszp_ctx* ctx, const float* d_x, uint64_t n, const uint32_t dims[3],
                   int ndims, double eb, int eb_mode, void* d_out, size_t cap,
                   uint64_t* d_out_bytes, hoszp_stream_t stream) {
  if (!ctx || !d_out || !d_out_bytes || !dims || (n > 0 && !d_x)) return HOSZP_ERR_ARG;
  if (ndims < 1 || ndims > 3) return HOSZP_ERR_ARG;
  uint64_t prod = 1;
  for (int d = 0; d < ndims; d++) prod *= dims[d];
  if (prod != n || n > (1ull << 40)) return HOSZP_ERR_ARG;
  if (!(eb > 0) || !std::isfinite(eb) || (eb_mode != HOSZP_EB_ABS && eb_mode != HOSZP_EB_REL))
    return HOSZP_ERR_ARG;
  if ((n > 0 && !aligned16(d_x)) || !aligned16(d_out) || !aligned8(d_out_bytes))
    return HOSZP_ERR_ARG;
  const uint64_t nb = nblocks(n);
  if (cap < off_sign(nb)) return HOSZP_ERR_CAPACITY;
  float eq = 0.0f;
  if (eb_mode == HOSZP_EB_ABS) {
    eq = eps_q_of(eb);
    if (eq == 0.0f) return HOSZP_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, ntiles_of(nb) + 1, 25ull * TILE * ntiles_of(nb) + 16);
  if (rc) return rc;
  Launch lc = lc_of(ctx, stream);
  uint32_t d3[3] = {0, 0, 0};
  for (int d = 0; d < ndims; d++) d3[d] = dims[d];
  if (eb_mode == HOSZP_EB_REL) {
    rc = cuda_rc(launch_range(lc, d_x, n, eb, ctx->ws));
    if (rc) return rc;
  }
  rc = cuda_rc(launch_compress(lc, d_x, n, d3, (uint32_t)ndims, eq, eb,
                               eb_mode == HOSZP_EB_REL, (uint8_t*)d_out, cap, ctx->ws));
  if (rc) return rc;
  return cuda_rc(launch_place(lc, (uint8_t*)d_out, cap, d_out_bytes, SLOT_SPLIT, 0, ctx->ws));
}

int hoszp_decompress(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, float* d_x, uint64_t n,
                     hoszp_stream_t stream) {
  if (!ctx || !d_c || (n > 0 && !d_x) || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || (n > 0 && !aligned16(d_x))) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, ntiles_of(nblocks(n)) + 1, 16);
  if (rc) return rc;
  return cuda_rc(launch_decompress(lc_of(ctx, stream), (const uint8_t*)d_c, c_bytes, d_x, n,
                                   ctx->ws));
}

int hoszp_negate(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, void* d_out, size_t cap,
                 uint64_t* d_out_bytes, hoszp_stream_t stream) {
  if (!ctx || !d_c || !d_out || !d_out_bytes || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || !aligned16(d_out) || !aligned8(d_out_bytes)) return HOSZP_ERR_ARG;
  const uint8_t* a = (const uint8_t*)d_c;
  uint8_t* o = (uint8_t*)d_out;
  if (o != a && o < a + c_bytes && a < o + cap) return HOSZP_ERR_ARG;  // partial overlap
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, 1, 16);
  if (rc) return rc;
  return cuda_rc(launch_negate(lc_of(ctx, stream), a, c_bytes, o, cap, d_out_bytes, ctx->ws));
}

int hoszp_add_scalar(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s, void* d_out,
                     size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream) {
  if (!ctx || !d_c || !d_out || !d_out_bytes || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!std::isfinite(s)) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || !aligned16(d_out) || !aligned8(d_out_bytes)) return HOSZP_ERR_ARG;
  const uint8_t* a = (const uint8_t*)d_c;
  uint8_t* o = (uint8_t*)d_out;
  if (o != a && o < a + c_bytes && a < o + cap) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, 1, 16);
  if (rc) return rc;
  return cuda_rc(launch_add_scalar(lc_of(ctx, stream), a, c_bytes, s, o, cap, d_out_bytes,
                                   ctx->ws));
}

int hoszp_sub_scalar(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s, void* d_out,
                     size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream) {
  if (!ctx || !d_c || !d_out || !d_out_bytes || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!std::isfinite(s)) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || !aligned16(d_out) || !aligned8(d_out_bytes)) return HOSZP_ERR_ARG;
  const uint8_t* a = (const uint8_t*)d_c;
  uint8_t* o = (uint8_t*)d_out;
  if (o != a && o < a + c_bytes && a < o + cap) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, 1, 16);
  if (rc) return rc;
  return cuda_rc(launch_sub_scalar(lc_of(ctx, stream), a, c_bytes, s, o, cap, d_out_bytes,
                                   ctx->ws));
}

static int mul_scalar_any(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s, void* d_out,
                          size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream, bool exact) {
  if (!ctx || !d_c || !d_out || !d_out_bytes || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!std::isfinite(s)) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || !aligned16(d_out) || !aligned8(d_out_bytes)) return HOSZP_ERR_ARG;
  const uint8_t* a = (const uint8_t*)d_c;
  uint8_t* o = (uint8_t*)d_out;
  if (o < a + c_bytes && a < o + cap) return HOSZP_ERR_ARG;  // no aliasing
  DeviceGuard g(ctx->device);
  const uint64_t tiles = tiles_from_bytes(c_bytes);
  // slot words: one sign word per non-constant input block (sign slots), then
  // e + the input's rate words per non-constant input block (plane slots),
  // where e bounds the growth of a block's rate: |2e rho| <= 2|s| when rho != 0
  // (|q' - q'_prev| <= |s| |delta| + 1 for the exact variant too); no rate exceeds 31
  const uint32_t e_bits =
      std::min(31u, (uint32_t)std::ceil(std::log2(2.0 * std::fabs(s) + 1.0)) + 1u);
  const uint64_t nnc_bound = c_bytes / 21 + 1;  // a non-constant block takes >= 21 bytes
  int rc = ensure_ws(ctx, tiles, nnc_bound * (1ull + e_bits) + c_bytes / 8 + 64);
  if (rc) return rc;
  Launch lc = lc_of(ctx, stream);
  rc = cuda_rc(launch_mul_scalar(lc, a, c_bytes, s, exact, e_bits, o, cap, ctx->ws));
  if (rc) return rc;
  return cuda_rc(launch_place(lc, o, cap, d_out_bytes, SLOT_SPLIT, e_bits, ctx->ws));
}

int hoszp_mul_scalar(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s, void* d_out,
                     size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream) {
  return mul_scalar_any(ctx, d_c, c_bytes, s, d_out, cap, d_out_bytes, stream, false);
}

int hoszp_mul_scalar_exact(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s,
                           void* d_out, size_t cap, uint64_t* d_out_bytes,
                           hoszp_stream_t stream) {
  return mul_scalar_any(ctx, d_c, c_bytes, s, d_out, cap, d_out_bytes, stream, true);
}

int hoszp_hadamard(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b,
                   size_t b_bytes, int32_t* d_scratch, uint64_t n, void* d_out, size_t cap,
                   uint64_t* d_out_bytes, hoszp_stream_t stream) {
  if (!ctx || !d_a || !d_b || !d_out || !d_out_bytes || a_bytes < HOSZP_HEADER_BYTES ||
      b_bytes < HOSZP_HEADER_BYTES || (n > 0 && !d_scratch))
    return HOSZP_ERR_ARG;
  if (!aligned16(d_a) || !aligned16(d_b) || !aligned16(d_out) || !aligned8(d_out_bytes) ||
      (n > 0 && !aligned16(d_scratch)))
    return HOSZP_ERR_ARG;
  const uint8_t* a = (const uint8_t*)d_a;
  const uint8_t* b = (const uint8_t*)d_b;
  uint8_t* o = (uint8_t*)d_out;
  if ((o < a + a_bytes && a < o + cap) || (o < b + b_bytes && b < o + cap)) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  const uint64_t nt = ntiles_of(nblocks(n));
  const uint64_t ta = tiles_from_bytes(a_bytes);
  // full slots: a sign word and 31 planes per block
  int rc = ensure_ws(ctx, (ta > nt + 1 ? ta : nt + 1), 32ull * TILE * (nt + 1) + 64);
  if (rc) return rc;
  Launch lc = lc_of(ctx, stream);
  rc = cuda_rc(launch_decode_q(lc, b, b_bytes, (int*)d_scratch, n, ctx->ws));
  if (rc) return rc;
  rc = cuda_rc(launch_hadamard(lc, a, a_bytes, b, b_bytes, (const int*)d_scratch, o, cap,
                               ctx->ws));
  if (rc) return rc;
  return cuda_rc(launch_place(lc, o, cap, d_out_bytes, SLOT_FULL, 0, ctx->ws));
}

static int add_sub(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b,
                   size_t b_bytes, void* d_out, size_t cap, uint64_t* d_out_bytes,
                   hoszp_stream_t stream, bool subtract) {
  if (!ctx || !d_a || !d_b || !d_out || !d_out_bytes || a_bytes < HOSZP_HEADER_BYTES ||
      b_bytes < HOSZP_HEADER_BYTES)
    return HOSZP_ERR_ARG;
  if (!aligned16(d_a) || !aligned16(d_b) || !aligned16(d_out) || !aligned8(d_out_bytes))
    return HOSZP_ERR_ARG;
  const uint8_t* a = (const uint8_t*)d_a;
  const uint8_t* b = (const uint8_t*)d_b;
  uint8_t* o = (uint8_t*)d_out;
  if ((o < a + a_bytes && a < o + cap) || (o < b + b_bytes && b < o + cap)) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  const uint64_t ta = tiles_from_bytes(a_bytes), tb = tiles_from_bytes(b_bytes);
  // slot words: sign slots for A's plus B's sign words, then plane slots for
  // their sign and plane words (a non-constant block takes >= 21 stream bytes)
  const uint64_t nnc_bound = a_bytes / 21 + b_bytes / 21 + 2;
  int rc = ensure_ws(ctx, ta > tb ? ta : tb, 2 * nnc_bound + (a_bytes + b_bytes) / 8 + 64);
  if (rc) return rc;
  Launch lc = lc_of(ctx, stream);
  rc = cuda_rc(launch_add(lc, a, a_bytes, b, b_bytes, o, cap, subtract, ctx->ws));
  if (rc) return rc;
  return cuda_rc(launch_place(lc, o, cap, d_out_bytes, SLOT_SPLIT, 0, ctx->ws));
}

int hoszp_add(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b, size_t b_bytes,
              void* d_out, size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream) {
  return add_sub(ctx, d_a, a_bytes, d_b, b_bytes, d_out, cap, d_out_bytes, stream, false);
}

int hoszp_sub(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b, size_t b_bytes,
              void* d_out, size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream) {
  return add_sub(ctx, d_a, a_bytes, d_b, b_bytes, d_out, cap, d_out_bytes, stream, true);
}

// Covariance in one pass over both streams (k_cov).
int hoszp_cov(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b, size_t b_bytes,
              double* d_result, hoszp_stream_t stream) {
  if (!ctx || !d_a || !d_b || !d_result || a_bytes < HOSZP_HEADER_BYTES ||
      b_bytes < HOSZP_HEADER_BYTES)
    return HOSZP_ERR_ARG;
  if (!aligned16(d_a) || !aligned16(d_b) || !aligned8(d_result)) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  const uint64_t ta = tiles_from_bytes(a_bytes), tb = tiles_from_bytes(b_bytes);
  int rc = ensure_ws(ctx, ta > tb ? ta : tb, 16);
  if (rc) return rc;
  return cuda_rc(launch_cov(lc_of(ctx, stream), (const uint8_t*)d_a, a_bytes, (const uint8_t*)d_b,
                            b_bytes, d_result, ctx->ws));
}

static int moments(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_result,
                   hoszp_stream_t stream, bool var, bool take_sqrt = false) {
  if (!ctx || !d_c || !d_result || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || !aligned8(d_result)) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, tiles_from_bytes(c_bytes), 16);
  if (rc) return rc;
  return cuda_rc(launch_moments(lc_of(ctx, stream), (const uint8_t*)d_c, c_bytes, d_result, var,
                                ctx->ws, nullptr, take_sqrt));
}

int hoszp_std(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_result,
              hoszp_stream_t stream) {
  return moments(ctx, d_c, c_bytes, d_result, stream, true, true);
}

int hoszp_block_means(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_out, uint64_t nb,
                      hoszp_stream_t stream) {
  if (!ctx || !d_c || (nb > 0 && !d_out) || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || (nb > 0 && !aligned8(d_out))) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, ntiles_of(nb) + 1, 16);
  if (rc) return rc;
  return cuda_rc(launch_block_means(lc_of(ctx, stream), (const uint8_t*)d_c, c_bytes, d_out, nb,
                                    ctx->ws));
}

int hoszp_sums(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, uint64_t* d_sums,
               hoszp_stream_t stream) {
  if (!ctx || !d_c || !d_sums || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (!aligned16(d_c) || !aligned8(d_sums)) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, tiles_from_bytes(c_bytes), 16);
  if (rc) return rc;
  return cuda_rc(launch_moments(lc_of(ctx, stream), (const uint8_t*)d_c, c_bytes, nullptr, false,
                                ctx->ws, reinterpret_cast<unsigned long long*>(d_sums)));
}

int hoszp_finish_sums(hoszp_ctx* ctx, const uint64_t* d_sums, float eps_q, double* d_mean,
                      double* d_var, hoszp_stream_t stream) {
  if (!ctx || !d_sums || (!d_mean && !d_var)) return HOSZP_ERR_ARG;
  if (!aligned8(d_sums) || (d_mean && !aligned8(d_mean)) || (d_var && !aligned8(d_var)))
    return HOSZP_ERR_ARG;
  if (!(eps_q > 0.0f) || !std::isfinite(eps_q)) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, 1, 16);
  if (rc) return rc;
  return cuda_rc(launch_finish_sums(lc_of(ctx, stream),
                                    reinterpret_cast<const unsigned long long*>(d_sums), eps_q,
                                    d_mean, d_var, ctx->ws));
}

int hoszp_concat(hoszp_ctx* ctx, uint32_t nstreams, const void* const* d_streams,
                 const size_t* stream_bytes, const uint32_t dims[3], int ndims, void* d_out,
                 size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream) {
  if (!ctx || nstreams == 0 || !d_streams || !stream_bytes || !dims || !d_out || !d_out_bytes)
    return HOSZP_ERR_ARG;
  if (ndims < 1 || ndims > 3 || !aligned16(d_out) || !aligned8(d_out_bytes)) return HOSZP_ERR_ARG;
  for (uint32_t s = 0; s < nstreams; s++) {
    if (!d_streams[s] || !aligned16(d_streams[s]) || stream_bytes[s] < HOSZP_HEADER_BYTES)
      return HOSZP_ERR_ARG;
    const uint8_t* c = (const uint8_t*)d_streams[s];
    const uint8_t* o = (const uint8_t*)d_out;
    if (o < c + stream_bytes[s] && c < o + cap) return HOSZP_ERR_ARG;  // no aliasing
  }
  uint32_t d3[3] = {0, 0, 0};
  for (int d = 0; d < ndims; d++) d3[d] = dims[d];
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, 1, concat_table_words(nstreams) + 16);
  if (rc) return rc;
  return cuda_rc(launch_concat(lc_of(ctx, stream), nstreams, d_streams, stream_bytes, d3,
                               (uint32_t)ndims, (uint8_t*)d_out, cap, d_out_bytes, ctx->ws));
}

int hoszp_selftest_wait(hoszp_ctx* ctx, int which, uint64_t limit, hoszp_stream_t stream) {
  if (!ctx || (which != 0 && which != 1) || limit == 0) return HOSZP_ERR_ARG;
  // at most about a second either way: 2^22 polls of ~256 ns, or 10^9 ns
  if ((which == 0 && limit > (1ull << 22)) || (which == 1 && limit > 1000000000ull))
    return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  int rc = ensure_ws(ctx, 2, 16);
  if (rc) return rc;
  return cuda_rc(launch_wait_selftest(lc_of(ctx, stream), which, (long long)limit, ctx->ws));
}

int hoszp_mean(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_result,
               hoszp_stream_t stream) {
  return moments(ctx, d_c, c_bytes, d_result, stream, false);
}

int hoszp_var(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_result,
              hoszp_stream_t stream) {
  return moments(ctx, d_c, c_bytes, d_result, stream, true);
}

}  // extern "C"

namespace hz {
// Context access for batch plans (batch.cu): grows the workspace to `tiles`
// tiles and returns it with the context's device and SM count.
int ctx_prepare(hoszp_ctx* ctx, uint64_t tiles, Ws* ws, int* device, int* num_sms) {
  if (!ctx) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  const int rc = ensure_ws(ctx, tiles, 16);
  if (rc) return rc;
  *ws = ctx->ws;
  *device = ctx->device;
  *num_sms = ctx->num_sms;
  return HOSZP_OK;
}

// The compressor's bound for an absolute eps (batched compression, bproduce.cu).
float eps_q_host(double eps) { return eps_q_of(eps); }

// Batched producing operators (bproduce.cu): the workspace grown to a tile
// count and a number of staging words.
int ctx_prepare_staging(hoszp_ctx* ctx, uint64_t tiles, uint64_t staging_words, Ws* ws,
                        int* device, int* num_sms) {
  if (!ctx) return HOSZP_ERR_ARG;
  DeviceGuard g(ctx->device);
  const int rc = ensure_ws(ctx, tiles, staging_words);
  if (rc) return rc;
  *ws = ctx->ws;
  *device = ctx->device;
  *num_sms = ctx->num_sms;
  return HOSZP_OK;
}

// Serving (serve.cu): the context's device status word, its workspace size,
// and a cap on the SMs its persistent grids spread over (0 restores all).
int* ctx_status_word(hoszp_ctx* ctx) { return ctx ? ctx->ws.status : nullptr; }
size_t ctx_workspace_bytes(const hoszp_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }
void ctx_limit_sms(hoszp_ctx* ctx, int sms) {
  if (!ctx) return;
  int all = 0;
  if (cudaDeviceGetAttribute(&all, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  ctx->num_sms = (sms > 0 && sms < all) ? sms : all;
}

// Workspace access for the traditional-workflow helpers (baseline.cu); the
// grid they use (SMs x 4) stays within the partials the workspace holds.
Ws ctx_workspace(hoszp_ctx* ctx) {
  if (ensure_ws(ctx, 1, 16) != HOSZP_OK) {
    Ws w{};
    return w;
  }
  return ctx->ws;
}
}  // namespace hz
