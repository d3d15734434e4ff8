/*
 * hoszp.h — C ABI of libhoszp, a GB300 (sm_103a) implementation of the HoSZp
 * homomorphic error-bounded lossy compressor (Agarwal et al., arXiv 2408.11971).
 *
 * The library compresses float32 fields into a blockwise stream (quantization,
 * in-block 1-D Lorenzo, blockwise fixed-length bit-plane encoding; Sec. IV-A,
 * Fig. 2) and runs the paper's homomorphic operators directly on that stream
 * (Sec. IV-B workflows 1-3, Sec. V, Table 2): negation, scalar addition, scalar
 * multiplication, element-wise addition of two streams, mean and variance.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every data pointer named d_* is DEVICE memory owned by the caller (for example a
 *    torch tensor's data_ptr()). The library never frees caller memory.
 *  - Calls are asynchronous on `stream`. Argument errors the host can see
 *    (null pointers, zero capacity, bad modes, sizes) are returned immediately
 *    as a negative hoszp_status and nothing is launched.
 *  - Errors only the device can see (non-finite input, quantization range,
 *    overflow, corrupt or mismatched streams, output capacity, spin-wait
 *    timeouts) are recorded in the context's device status word; the output
 *    is then undefined. hoszp_get_status() synchronizes and returns/clears it.
 *  - Output sizes of stream-producing calls are written to the device word
 *    *d_out_bytes (uint64), so no call needs a host round trip.
 *  - One context serves one stream at a time: its workspace is reused by every
 *    call, so two calls on one context must not overlap on the device.
 *
 * Stream format ("R-FMT", little-endian; section order of Fig. 3):
 *   [header 64 B][rate u8 x nb][pad16][outlier i32 x nb][pad16]
 *   [sign u64 x nnc][plane u64 x R][pad16]
 *   nb  = ceil(n/64) blocks of L = 64 consecutive values (last block short),
 *   rate_b = bit length of max |delta| in block b (0 = constant block, which
 *            stores no sign word and no planes; Sec. IV-A step 3),
 *   outlier_b = quantized value of the first element of block b (Sec. IV-A step 2),
 *   sign word: bit i = 1 iff delta_i < 0 (Sec. IV-A, sign array),
 *   plane p (p < rate_b): bit i = bit p of |delta_i|, i = 0..63, delta_0 := 0.
 *   nnc = number of non-constant blocks, R = sum of rates. Every section starts
 *   on a 16-byte boundary except the plane section (8-byte aligned), and the
 *   stream length is a multiple of 16 bytes (zero padding), so sections can be
 *   moved with 16-byte bulk copies.
 */
#ifndef HOSZP_H
#define HOSZP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* hoszp_stream_t; /* same object as cudaStream_t */

typedef enum {
  HOSZP_OK = 0,
  HOSZP_ERR_ARG = -1,       /* bad argument (host check) */
  HOSZP_ERR_CAPACITY = -2,  /* output buffer too small */
  HOSZP_ERR_FORMAT = -3,    /* stream header/size corrupt */
  HOSZP_ERR_MISMATCH = -4,  /* two streams differ in n, block length or eps */
  HOSZP_ERR_RANGE = -5,     /* |q| beyond the quantizer's exact range */
  HOSZP_ERR_OVERFLOW = -6,  /* an operator's result leaves the integer range */
  HOSZP_ERR_NONFINITE = -7, /* NaN or Inf in the input field */
  HOSZP_ERR_TIMEOUT = -8,   /* a bounded device spin-wait gave up */
  HOSZP_ERR_CUDA = -9       /* a CUDA runtime call failed */
} hoszp_status;

enum { HOSZP_EB_ABS = 0, HOSZP_EB_REL = 1 };

/* Format constants. */
#define HOSZP_MAGIC 0x505A5348u       /* bytes 'H','S','Z','P' */
#define HOSZP_VERSION 1u
#define HOSZP_BLOCK 64u               /* L: values per block (Table 6 gives 64) */
#define HOSZP_HEADER_BYTES 64u
#define HOSZP_QMAX_COMPRESS 8388606   /* 2^23-2: exact range of the quantizer */
#define HOSZP_QLIM 1073741823         /* 2^30-1: integer range of every stream */

/* Header, 64 bytes at offset 0 of every stream. */
typedef struct hoszp_header {
  uint32_t magic;     /* HOSZP_MAGIC */
  uint16_t version;   /* HOSZP_VERSION */
  uint8_t dtype;      /* 0 = float32 */
  uint8_t ndims;      /* 1..3 */
  uint32_t dims[3];   /* informational shape, row-major, product == n */
  float eps_q;        /* bound used by the quantizer: largest float <= eps */
  uint64_t n;         /* number of values */
  double eps;         /* absolute error bound the caller asked for */
  uint64_t nnc;       /* non-constant blocks */
  uint64_t R;         /* sum of block rates = number of plane words */
  uint32_t qbound;    /* upper bound on |q| over the stream (<= HOSZP_QLIM) */
  uint32_t block;     /* HOSZP_BLOCK */
} hoszp_header;

typedef struct hoszp_ctx hoszp_ctx;

/* Create a context on CUDA device `device`: a device status word and a workspace
 * that grows on demand (the only memory the library allocates). Returns
 * HOSZP_OK and *ctx, or HOSZP_ERR_ARG / HOSZP_ERR_CUDA. */
int hoszp_ctx_create(hoszp_ctx** ctx, int device);
/* Free the context and its workspace. Synchronizes the device. NULL is a no-op. */
void hoszp_ctx_destroy(hoszp_ctx* ctx);
/* Pre-size the workspace for fields of up to n values, so that later calls on
 * that size allocate nothing. HOSZP_ERR_CUDA if the allocation fails. */
int hoszp_ctx_reserve(hoszp_ctx* ctx, uint64_t n);
/* Synchronize the device, return the first device-side error recorded since
 * the last call (HOSZP_OK if none) in *status, and clear it. */
int hoszp_get_status(hoszp_ctx* ctx, int* status);

/* Worst-case stream size for n values: header + rates + outliers + one sign
 * word and 31 planes per block (section sizes of Fig. 3 at maximum rate). */
size_t hoszp_compress_bound(uint64_t n);

/* Compression, Sec. IV-A (Eq. 3 quantization, Eq. 4 Lorenzo, BF encoding).
 * d_x: n float32 values (device). dims/ndims: informational shape (1..3 dims,
 * product == n). eb: error bound; eb_mode HOSZP_EB_ABS uses it as eps,
 * HOSZP_EB_REL uses eps = eb * (max - min) of the field (a range pass on the
 * device). Quantizer: q = floor((x + e) / (2e)) evaluated exactly, e = eps_q.
 * Every reconstructed value then satisfies |x - x'| <= eps + ulp(x')/2.
 * Output: stream at d_out (capacity cap bytes), its size in *d_out_bytes.
 * Device errors: NONFINITE, RANGE (|q| > HOSZP_QMAX_COMPRESS), CAPACITY. */
int hoszp_compress(hoszp_ctx* ctx, const float* d_x, uint64_t n, const uint32_t dims[3],
                   int ndims, double eb, int eb_mode, void* d_out, size_t cap,
                   uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Full decompression (inverse of every step, Fig. 2 caption): decode the bit
 * planes, invert the Lorenzo prediction, x' = float(q) * (2 eps_q).
 * d_c: stream of c_bytes bytes; d_x: room for n floats (n must equal the header's). */
int hoszp_decompress(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, float* d_x, uint64_t n,
                     hoszp_stream_t stream);

/* Negation, Sec. V-A "Negation", workflow 1: every sign word is bit-inverted
 * (all 64 bits) and every outlier negated; rates and planes are copied.
 * d_out may equal d_c (in place; then only outliers and signs are touched). */
int hoszp_negate(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, void* d_out, size_t cap,
                 uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Scalar addition, Sec. V-A "Scalar Addition", workflow 1: rho_s = Eq. 3
 * quantization of s; every outlier becomes O + rho_s. In place allowed.
 * Errors: RANGE if |rho_s| > HOSZP_QLIM (host), OVERFLOW if qbound + |rho_s|
 * exceeds HOSZP_QLIM (device). */
int hoszp_add_scalar(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s, void* d_out,
                     size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Scalar subtraction, Sec. V-A "Scalar Subtraction", workflow 1: rho_s = Eq. 3
 * quantization of s is deducted from every outlier, O' = O - rho_s; rates,
 * signs and planes are copied. In place allowed. Same arguments and errors as
 * hoszp_add_scalar; the header bound becomes qbound + |rho_s|. At a tie of
 * Eq. 3 (s an odd multiple of eps_q) this differs from adding -s, whose bin is
 * not -rho_s. */
int hoszp_sub_scalar(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s, void* d_out,
                     size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Scalar multiplication, Sec. V-A "Scalar Multiplication", workflow 3: decode
 * to q, q' = floor(2 eps_q * q * rho_s + 1/2) (Eq. 3 applied to the product of
 * the dequantized values), then Lorenzo + BF re-encode. Output stream is
 * canonical. Errors: RANGE (rho_s), OVERFLOW (|q'| > HOSZP_QLIM), CAPACITY. */
int hoszp_mul_scalar(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s, void* d_out,
                     size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Multiplication by the scalar itself: q' = floor(q s + 1/2) evaluated exactly
 * (s = M 2^E, 53-bit M), i.e. Eq. 3 applied to the dequantized value times s
 * without first quantizing s to its bin rho_s as Sec. V-A does. The paper's
 * form turns every scalar with |s| < eps into 0 (rho_s = 0); this variant does
 * not. Same arguments and errors as hoszp_mul_scalar, except that no scalar is
 * out of range: a product beyond HOSZP_QLIM is OVERFLOW on the device. */
int hoszp_mul_scalar_exact(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double s,
                           void* d_out, size_t cap, uint64_t* d_out_bytes,
                           hoszp_stream_t stream);

/* Element-wise addition, Sec. V-C, workflow 2: outliers add, signed deltas add,
 * blockwise fixed-length re-encode (no Lorenzo inverse). Streams must agree in
 * n, block length and eps_q (MISMATCH otherwise). OVERFLOW if the sum of the
 * two qbounds exceeds HOSZP_QLIM. Output stream is canonical. */
int hoszp_add(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b, size_t b_bytes,
              void* d_out, size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Hadamard product A o B, Sec. V-C "Hadamard Product" (the scalar
 * multiplication with the other field's quantized values in place of the
 * scalar's bin): q' = floor(2 eps_q q_A q_B + 1/2), Eq. 3 applied to the product
 * of the dequantized values, evaluated exactly, then Lorenzo + BF re-encode.
 * The streams must agree in n and eps_q (MISMATCH otherwise; n is the streams'
 * value count). d_scratch: caller-owned device buffer of n int32 values
 * (16-byte aligned) that receives B's quantized integers. Output stream is
 * canonical. Errors: OVERFLOW (|q'| > HOSZP_QLIM), CAPACITY, MISMATCH. */
int hoszp_hadamard(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b,
                   size_t b_bytes, int32_t* d_scratch, uint64_t n, void* d_out, size_t cap,
                   uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Element-wise subtraction A - B, Sec. V-C "Element-wise Subtraction": as
 * hoszp_add with B's signed deltas and outliers negated (O' = O_A - O_B,
 * delta' = delta_A - delta_B). Same arguments, checks and errors as
 * hoszp_add; the qbound of the result is qbound_A + qbound_B. */
int hoszp_sub(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b, size_t b_bytes,
              void* d_out, size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Mean, Sec. V-B: S1 = sum of q (exact integer), mean = (S1 / n) * 2 eps_q in
 * FP64, written to the device double *d_result. n == 0 -> HOSZP_ERR_ARG. */
int hoszp_mean(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_result,
               hoszp_stream_t stream);

/* Population variance, Sec. V-B: (2 eps_q)^2 * (n*S2 - S1^2) / n^2 with S1, S2
 * exact integer sums of q and q^2, finished in FP64 into *d_result. */
int hoszp_var(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_result,
              hoszp_stream_t stream);

/* Standard deviation, Sec. V-B "Standard Deviation": the square root of the
 * population variance above, taken in FP64 (correctly rounded) after the
 * same finish, into the device double *d_result. Same errors as hoszp_var. */
int hoszp_std(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_result,
              hoszp_stream_t stream);

/* Block-wise means, Sec. V-B "Mean" (its last sentences: the same kernel sums
 * each block's quantized values and divides by the block's length): d_out
 * (device, nb doubles, 8-byte aligned) gets mean_b = (S1_b / L_b) * 2 eps_q in
 * FP64 for every block b, with S1_b the exact sum of the block's q and L_b its
 * length (64; the last block may be shorter). nb must be the stream's block
 * count ceil(n / 64) (device status MISMATCH otherwise); nb = 0 writes
 * nothing. */
int hoszp_block_means(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, double* d_out, uint64_t nb,
                      hoszp_stream_t stream);

/* Population covariance of two streams, Sec. V-D "Covariance" (done like the
 * variance of Sec. V-B, over two fields): 2 eps_A 2 eps_B (n S_AB - S1_A S1_B) / n^2
 * with S_AB = sum q_A q_B, S1_A = sum q_A, S1_B = sum q_B exact integers from
 * one pass over both streams, finished in FP64 into the device double
 * *d_result. The streams must hold the same number of values n (device status
 * MISMATCH otherwise); their error bounds may differ, since each side is scaled
 * by its own 2 eps_q. n = 0 -> ARG. Needs no memory beyond the context's
 * workspace. */
int hoszp_cov(hoszp_ctx* ctx, const void* d_a, size_t a_bytes, const void* d_b, size_t b_bytes,
              double* d_result, hoszp_stream_t stream);

/* The exact integer sums behind mean and variance (Sec. V-B), for combining
 * shards of one field held by several devices or processes: d_sums (device,
 * 5 words) gets S1 = sum of q as a 128-bit two's complement integer (words 0
 * low, 1 high), S2 = sum of q^2 as a 128-bit unsigned integer (words 2, 3) and
 * n (word 4). Shards of one field (whole blocks each, the same eps_q) combine
 * by adding the sums; mean = (S1 / n) 2 eps_q and the population variance
 * (2 eps_q)^2 (n S2 - S1^2) / n^2 then follow exactly as for one stream. */
int hoszp_sums(hoszp_ctx* ctx, const void* d_c, size_t c_bytes, uint64_t* d_sums,
               hoszp_stream_t stream);

/* Mean and population variance of a field from exact sums combined over its
 * shards (Sec. V-B: mean = (S1 / n) 2 eps_q, variance = (2 eps_q)^2
 * (n S2 - S1^2) / n^2 over the integers): d_sums (device, 5 words, the layout
 * hoszp_sums writes) holds the word-wise 128-bit sums of the shards' S1 and S2
 * and the total n; eps_q is the shards' common bound (the header's eps_q
 * bits). Writes *d_mean and/or *d_var (device doubles; either may be NULL, not
 * both) with the same FP64 steps as hoszp_mean and hoszp_var, so the result
 * equals those of the whole field on one device bit for bit. n == 0 sets the
 * context's status to HOSZP_ERR_ARG (results 0). Asynchronous on stream. */
int hoszp_finish_sums(hoszp_ctx* ctx, const uint64_t* d_sums, float eps_q, double* d_mean,
                      double* d_var, hoszp_stream_t stream);

/* The streams of consecutive shards of one field joined into the field's
 * stream (Sec. VI-B5: the nodes' compressed data gathered at a root). Blocks
 * are independent (Sec. IV-A), so the result is the stream the compressor
 * gives for the whole field: the shards' rate, outlier, sign and plane
 * sections laid end to end (Fig. 3) under one header with the total n, the
 * given shape (ndims 1..3, dims[0..ndims-1], product == total n), the shards'
 * summed nnc and R and the largest qbound. Nothing is decoded.
 * d_streams, stream_bytes: host arrays of nstreams >= 1 device pointers
 * (16-byte aligned, not overlapping d_out) and sizes, in the field's order.
 * Every shard must carry the same eps_q and eps bits, and every shard but the
 * last a whole number of blocks (n a multiple of 64). Device-side errors go to
 * the context's status: FORMAT (a bad header), MISMATCH (bounds differ, or a
 * ragged shard before the last), ARG (the shape's product is not the total n),
 * CAPACITY (cap too small); *d_out_bytes is then 0. Uses the context's
 * workspace for the shard table; asynchronous on stream (the host arrays may
 * be released when the call returns). */
int hoszp_concat(hoszp_ctx* ctx, uint32_t nstreams, const void* const* d_streams,
                 const size_t* stream_bytes, const uint32_t dims[3], int ndims, void* d_out,
                 size_t cap, uint64_t* d_out_bytes, hoszp_stream_t stream);

/* Failure-detection self-test (the paper has no counterpart): runs one of the
 * library's bounded device waits on a flag that nothing sets, so the caller
 * can check that the wait gives up. which = 0: the decoupled look-back's poll
 * loop, waiting for a predecessor tile that never publishes, limited to
 * `limit` polls of about 256 ns (1 .. 2^22); which = 1: the copy rings'
 * mbarrier wait on a stage that never lands, limited to `limit` ns
 * (1 .. 10^9). The kernel sets HOSZP_ERR_TIMEOUT in the context's status word
 * (read and cleared by hoszp_get_status) and returns; the context stays
 * usable. Nothing faults, traps or spins without a limit. Asynchronous on
 * stream; ARG for another `which` or a limit outside its range. */
int hoszp_selftest_wait(hoszp_ctx* ctx, int which, uint64_t limit, hoszp_stream_t stream);

/* Mean of a stream without allocating: for callers that may not allocate
 * device memory when they call -- e.g. code whose device memory is owned by a
 * host framework's pool that forbids driver allocations while it runs, or a
 * latency-critical loop that cannot afford the device synchronization a
 * cudaMalloc implies -- and that therefore cannot create a hoszp_ctx. The
 * paper has no counterpart; the result is the same as hoszp_mean's.
 * Scratch: one file-scope device array of about 256 KB per device (per-CTA
 * records only), kept for as long as the library is loaded. Streams of more
 * than 2^28 values are refused (a policy limit of this entry point, not of the
 * kernel): status HOSZP_ERR_CAPACITY, and *d_result is set to NaN. The array's
 * device address is looked up with the caller's device current on every call
 * (so it stays right after a cudaDeviceReset and in a non-primary context); the
 * first call on a device also loads the library's kernels there, so make it
 * before capturing any stream. Every call shares the array, so calls that
 * overlap on the GPU (e.g. on two streams at once) race and must not.
 * d_c: stream (16-byte aligned), d_result: device double, d_status: device int
 * that receives the call's device-side status (HOSZP_OK or an error code).
 * Host-checkable argument errors are returned immediately; a device with more
 * than 512 SMs (more CTAs than the array holds records for) gets
 * HOSZP_ERR_CAPACITY. */
int hoszp_mean_noalloc(const void* d_c, size_t c_bytes, double* d_result, int* d_status,
                       hoszp_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched execution over many resident streams (one snapshot's fields).
 *
 * A plan fixes a set of resident compressed streams (the paper's operators
 * applied field by field, Sec. V) and lays their 64-block tiles end to end in
 * one global tile space. Each batched operator is one persistent launch over
 * that space, with every CTA walking the per-field table as its contiguous tile
 * range crosses field boundaries. The paper has no batched form; the results
 * are exactly those of the single-stream operators applied to each field.
 *
 * hoszp_batch_create: d_streams[f] (host array of device pointers, 16-byte
 * aligned) and stream_bytes[f] describe nfields >= 1 streams, each with n >= 1.
 * Synchronous: parses every header (FORMAT on a bad one, ARG on n == 0) and
 * runs each stream's rate pre-scan once. The plan owns a small device table
 * and the prefixes; it does not own the streams, which must stay resident and
 * keep their rates (only the batched negate / add_scalar below may modify them
 * in place). The plan keeps a pointer to ctx, which must outlive it.
 * Batched operators allocate nothing and never synchronize, so a sequence of
 * them can be captured in a CUDA graph. Device errors go to the plan's own
 * status word (hoszp_batch_get_status). Calls on one plan must not overlap. */
typedef struct hoszp_batch hoszp_batch;
int hoszp_batch_create(hoszp_ctx* ctx, uint32_t nfields, const void* const* d_streams,
                       const size_t* stream_bytes, hoszp_batch** out);
void hoszp_batch_destroy(hoszp_batch* b);
int hoszp_batch_info(const hoszp_batch* b, uint32_t* nfields, uint64_t* total_tiles);
/* Batched producing operators: every field of a plan gets its own output
 * stream, from one persistent launch over the plan's global tile space (a
 * warp per 64-block tile, the field found per tile), one scan of all tiles'
 * word counts and one placement launch -- no launch per field. Each field's
 * result is byte for byte what the single-stream operator gives for it.
 * d_outs: device array of nfields device pointers (16-byte aligned), d_caps:
 * device array of their capacities in bytes, d_out_bytes: device array that
 * receives each field's stream size (0 for a field that failed). Errors go to
 * the plan's status (hoszp_batch_get_status). The first call may grow the
 * plan's context workspace (a device allocation) to the batch's slots; later
 * calls with the same or a smaller need allocate nothing, synchronize nothing
 * and can be captured in a CUDA graph. Calls on one plan must not overlap.
 * hoszp_batch_mul_scalar: every field times s (Sec. V-A), each with its own
 *   bound's bin of s; RANGE when a field's bin of s is out of range.
 * hoszp_batch_add: field by field A_f + B_f, or A_f - B_f when subtract != 0
 *   (Sec. V-C); plan b must hold the same number of fields with the same n
 *   and eps_q bits field by field (MISMATCH), the sums' bounds must stay
 *   within 2^30 - 1 (OVERFLOW); errors go to plan a's status. */
int hoszp_batch_mul_scalar(hoszp_batch* b, double s, void* const* d_outs, const uint64_t* d_caps,
                           uint64_t* d_out_bytes, hoszp_stream_t stream);
int hoszp_batch_add(hoszp_batch* a, hoszp_batch* b, int subtract, void* const* d_outs,
                    const uint64_t* d_caps, uint64_t* d_out_bytes, hoszp_stream_t stream);
/* Compression of many float fields in one launch over all their tiles (Sec.
 * IV-A per field), with a range pass over every field's values first for
 * relative bounds (eb_mode HOSZP_EB_REL: eps_f = eb[f] (max - min) of field f).
 * d_x, d_outs: host arrays of nfields device pointers (fields 4-byte aligned,
 * outputs 16-byte aligned); n, eb, caps: host arrays (n[f] in 1 .. 2^32 - 1);
 * d_out_bytes: device array of nfields sizes. Each field is compressed as a
 * 1-D field of n[f] values, byte for byte the stream hoszp_compress gives with
 * dims = {n[f]}. Device errors go to the context's status. Uses the context's
 * workspace for slots and tables (grown on the first call); asynchronous on
 * stream, the host arrays may be released when the call returns. */
int hoszp_batch_compress(hoszp_ctx* ctx, uint32_t nfields, const float* const* d_x,
                         const uint64_t* n, const double* eb, int eb_mode, void* const* d_outs,
                         const size_t* caps, uint64_t* d_out_bytes, hoszp_stream_t stream);
/* Synchronizes the plan's device, returns its status word and clears it. */
int hoszp_batch_get_status(hoszp_batch* b, int* status);

/* Per-field mean / population variance (Sec. V-B) into d_results[f] (device
 * doubles, nfields of them); each equals hoszp_mean / hoszp_var of field f. */
int hoszp_batch_mean(hoszp_batch* b, double* d_results, hoszp_stream_t stream);
int hoszp_batch_var(hoszp_batch* b, double* d_results, hoszp_stream_t stream);

/* Decompression of every field (Fig. 2) in one persistent launch: field f's n_f
 * floats go to d_outs[f]. d_outs: device array of nfields device pointers, each
 * 16-byte aligned with room for its field's n_f floats (caller-owned). Each
 * output equals hoszp_decompress of field f, bit for bit. */
int hoszp_batch_decompress(hoszp_batch* b, float* const* d_outs, hoszp_stream_t stream);

/* In place on every field: negation (Sec. V-A), and scalar addition with the
 * same s for all fields, each field quantizing s with its own eps (Eq. 3).
 * A field whose rho_s or bound would leave the integer range is left
 * unchanged and the plan's status gets RANGE or OVERFLOW. */
int hoszp_batch_negate(hoszp_batch* b, hoszp_stream_t stream);
int hoszp_batch_add_scalar(hoszp_batch* b, double s, hoszp_stream_t stream);

/* Autotuner: times the batched mean (op 0), variance (op 1) and, when d_outs
 * is given, decompression (op 2) under each candidate launch shape on the
 * plan's own data, and keeps the fastest for later calls. The candidates:
 *   - the tile pipeline (reductions only): 8 or 4 stages x 1 or 2 CTAs per SM,
 *     16 warps per 64-block group;
 *   - the super-tile pipeline: 8 or 4 warps per block group (a warp takes one
 *     64-block tile of a stage; two groups over 4 stages, or four over 8), each
 *     with the generic decode (4 plane groups, any rate) and, where it is
 *     exact for every field, a rate-specialised one that decodes fewer plane
 *     groups. The plan bounds every field's rates by the bit length of twice
 *     its header's bound on |q|; the variance then needs ceil((rmax + 1) / 8)
 *     groups and the decompression ceil(rmax / 8); the mean is exact with 8 or
 *     16 bit-sliced columns for any rate, so both are offered.
 * d_results (nfields doubles) and the outputs d_outs[f] (as
 * hoszp_batch_decompress) receive the results of the timed runs.
 * Synchronizes the stream. hoszp_batch_config reports the pick: the stages,
 * CTAs per SM, warps per block group and plane groups of op's shape.
 * hoszp_batch_shapes returns how many candidates op has (or a negative
 * status) and hoszp_batch_set_shape(b, op, i) selects candidate i without
 * timing, which lets a test run every shape. */
int hoszp_batch_tune(hoszp_batch* b, double* d_results, float* const* d_outs,
                     hoszp_stream_t stream);
int hoszp_batch_config(const hoszp_batch* b, int op, int* stages, int* ctas_per_sm,
                       int* warps_per_group, int* plane_groups);
int hoszp_batch_shapes(const hoszp_batch* b, int op);
int hoszp_batch_set_shape(hoszp_batch* b, int op, int index);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of operator requests over resident streams.
 *
 * Analysis queries arrive as a stream of mixed operators over compressed fields
 * that stay resident on the device. A server owns `slots` execution slots (each
 * a context and a CUDA stream of its own, so the work of different requests
 * overlaps on the device) and an arena of device memory for the requests'
 * outputs. A scheduling thread of the library admits requests in arrival order
 * as soon as a slot is free and the arena can hold the request's output
 * (reductions need none and may pass a request that waits for memory), launches
 * them, and reports each completion with its latency. Every result is exactly
 * the one the same call gives alone (the operators are deterministic). The
 * paper has no serving form; the operators are those of Sec. V.
 *
 * Memory: hbm_budget_bytes bounds everything the server allocates -- the slot
 * workspaces (sized for streams of up to max_n values) and the output arena,
 * which gets the rest; creation fails with HOSZP_ERR_CAPACITY if nothing is
 * left for outputs. Output bounds used for admission: negate / add_scalar: the
 * input's size; mul_scalar: the input's size plus 8 bytes per block and bit of
 * rate growth; add / sub: the two inputs' sizes; decompress: 4 n. After a
 * request completes, the unused tail of its block returns to the arena.
 * Outputs are server memory: the caller reads them, then hands them back with
 * hoszp_server_release(). Requests on one server must name registered streams;
 * registered streams must stay resident and unmodified while requests use them.
 * Times are microseconds on the server's clock (hoszp_server_now_us).
 * --------------------------------------------------------------------------- */
typedef enum {
  HOSZP_OP_MEAN = 0,
  HOSZP_OP_VAR = 1,
  HOSZP_OP_NEGATE = 2,
  HOSZP_OP_ADD_SCALAR = 3,
  HOSZP_OP_MUL_SCALAR = 4,
  HOSZP_OP_ADD = 5,
  HOSZP_OP_SUB = 6,
  HOSZP_OP_DECOMPRESS = 7
} hoszp_op;

typedef struct hoszp_request {
  uint64_t tag;        /* the caller's id, returned with the completion */
  int32_t op;          /* hoszp_op */
  uint32_t a, b;       /* registered stream ids (b: ADD and SUB only) */
  double scalar;       /* ADD_SCALAR, MUL_SCALAR */
  uint64_t arrival_us; /* when the request arrives (0: at submission) */
} hoszp_request;

typedef struct hoszp_completion {
  uint64_t tag;
  int32_t op;
  int32_t status;      /* HOSZP_OK, or the request's host or device error */
  double value;        /* MEAN, VAR */
  void* d_out;         /* output stream or floats (NULL for reductions and errors) */
  uint64_t out_bytes;  /* bytes of d_out */
  uint64_t arrival_us, start_us, done_us; /* arrival, launch, completion seen by the server */
} hoszp_completion;

typedef struct hoszp_server_stats {
  uint64_t submitted, completed, pending, in_flight;
  uint64_t arena_bytes, arena_in_use, arena_peak;  /* output arena (bytes) */
  uint64_t workspace_bytes;                        /* slot workspaces and scratch */
  uint64_t max_in_flight;                          /* most requests on the device at once */
} hoszp_server_stats;

typedef struct hoszp_server hoszp_server;

/* Create a server on `device` with `slots` (1..64) execution slots, an HBM
 * budget in bytes and the largest stream (in values) any request will name.
 * sms_per_request limits the SMs one request's kernels spread over (0: all),
 * so that requests in different slots can run side by side. Starts the
 * scheduling thread. Errors: ARG, CAPACITY (budget too small), CUDA. */
int hoszp_server_create(int device, uint32_t slots, uint64_t hbm_budget_bytes, uint64_t max_n,
                        uint32_t sms_per_request, hoszp_server** out);
/* Stop admitting, wait for requests on the device, free everything (outputs
 * not yet released included). NULL is a no-op. */
void hoszp_server_destroy(hoszp_server* s);
/* Register a resident stream (device pointer, 16-byte aligned, and its size);
 * reads its header once (synchronous). *id names it in requests. Errors: ARG,
 * FORMAT (bad header), CAPACITY (more values than max_n). */
int hoszp_server_register(hoszp_server* s, const void* d_stream, size_t bytes, uint32_t* id);
/* Queue a request; thread-safe, never waits for the device. Requests are
 * considered in submission order, so arrival_us must not decrease. ARG on an
 * unknown op or stream id (nothing queued). */
int hoszp_server_submit(hoszp_server* s, const hoszp_request* r);
/* Move up to `max` completions (in completion order) into out[]; *count gets
 * how many. Waits up to wait_us microseconds for the first one. */
int hoszp_server_poll(hoszp_server* s, hoszp_completion* out, uint32_t max, uint32_t* count,
                      uint64_t wait_us);
/* Hand an output (a completion's d_out) back to the arena. ARG if unknown. */
int hoszp_server_release(hoszp_server* s, void* d_out);
/* Current time on the server's clock, microseconds since creation. */
uint64_t hoszp_server_now_us(const hoszp_server* s);
int hoszp_server_get_stats(hoszp_server* s, hoszp_server_stats* st);

#ifdef __cplusplus
}
#endif
#endif /* HOSZP_H */
