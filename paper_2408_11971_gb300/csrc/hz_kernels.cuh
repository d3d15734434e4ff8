// hz_kernels.cuh — host-side launch wrappers implemented by the .cu files and
// called by the C ABI (api.cu).
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "hz_common.cuh"

namespace hz {

struct Launch {
  int grid;  // number of SMs; each kernel multiplies by its resident CTAs per SM
  cudaStream_t stream;
};

// compress.cu
// One warp step of the two-lanes kernels: 16 blocks, 1024 contiguous floats,
// 32 rows of 32 (one row per lane).
constexpr uint32_t ROW_STEP_FLOATS = 16 * L;
// The float array x[0 .. n) as a 2-D tensor of 128-byte rows, copied in 32 x 32
// boxes with the 128-byte swizzle; false when that view does not apply.
bool encode_rows(const float* x, uint64_t n, CUtensorMap* map);
cudaError_t launch_range(const Launch& lc, const float* x, uint64_t n, double rel, Ws ws);
cudaError_t launch_compress(const Launch& lc, const float* x, uint64_t n, const uint32_t dims[3],
                            uint32_t ndims, float eps_q_abs, double eps_abs, bool rel, uint8_t* out,
                            uint64_t cap, Ws ws);
// place.cu: move staged planes behind the sign section and write the header
// Completes a produced stream: scans the per-tile word counts the producer
// left in agg[] (totals nnc, R; qbound from totals[2]), checks the capacity,
// copies the staged sign and plane words to their places and writes the
// header and the size word. One launch.
cudaError_t launch_place(const Launch& lc, uint8_t* out, uint64_t cap, uint64_t* out_bytes,
                         int rule, uint32_t e_bits, Ws ws);
// scan.cu: per-tile (nc, r) exclusive prefixes of a stream's rates into pre[]
cudaError_t launch_scan(const Launch& lc, const uint8_t* c, uint64_t c_bytes,
                        unsigned long long* pre, Ws ws);
// scan.cu: prefixes of the produced tiles' aggregates (batched producers)
cudaError_t launch_scan_agg(const Launch& lc, Ws ws, uint64_t ntiles_given = 0);
// decode.cu
cudaError_t launch_decompress(const Launch& lc, const uint8_t* c, uint64_t c_bytes, float* x,
                              uint64_t n, Ws ws);
// sums (optional, 5 words): S1 (two's complement, lo, hi), S2 (lo, hi), n
cudaError_t launch_moments(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double* result,
                           bool variance, Ws ws, unsigned long long* sums = nullptr,
                           bool take_sqrt = false);
cudaError_t launch_decode_q(const Launch& lc, const uint8_t* c, uint64_t c_bytes, int* q,
                           uint64_t n, Ws ws);
cudaError_t launch_block_means(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double* out,
                               uint64_t nb, Ws ws);
// ops.cu
cudaError_t launch_negate(const Launch& lc, const uint8_t* c, uint64_t c_bytes, uint8_t* out,
                          uint64_t cap, uint64_t* out_bytes, Ws ws);
cudaError_t launch_add_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws);
cudaError_t launch_sub_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws);
cudaError_t launch_mul_scalar(const Launch& lc, const uint8_t* c, uint64_t c_bytes, double s,
                              bool exact, uint32_t e_bits, uint8_t* out, uint64_t cap, Ws ws);
cudaError_t launch_hadamard(const Launch& lc, const uint8_t* a, uint64_t a_bytes,
                            const uint8_t* b, uint64_t b_bytes, const int* qb, uint8_t* out,
                            uint64_t cap, Ws ws);
cudaError_t launch_add(const Launch& lc, const uint8_t* a, uint64_t a_bytes, const uint8_t* b,
                       uint64_t b_bytes, uint8_t* out, uint64_t cap, bool subtract, Ws ws);
cudaError_t launch_cov(const Launch& lc, const uint8_t* a, uint64_t a_bytes, const uint8_t* b,
                       uint64_t b_bytes, double* result, Ws ws);

cudaError_t launch_finish_sums(const Launch& lc, const unsigned long long* sums, float eps_q,
                               double* mean, double* var, Ws ws);

uint64_t concat_table_words(uint32_t k);
cudaError_t launch_concat(const Launch& lc, uint32_t k, const void* const* streams,
                          const size_t* bytes, const uint32_t dims[3], uint32_t ndims,
                          uint8_t* out, uint64_t cap, uint64_t* out_bytes, Ws ws);

cudaError_t launch_wait_selftest(const Launch& lc, int which, long long limit, Ws ws);

// Persistent grid: SMs x resident CTAs per SM of `kernel` (capped at 8).
template <typename K>
inline int persistent_grid(K kernel, int threads, int num_sms, size_t smem = 0) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    per = 1;
  }
  per = per < 1 ? 1 : (per > 8 ? 8 : per);
  return num_sms * per;
}

// Raises kernel Kern's dynamic shared-memory limit to smem on the current
// device, once per device: function attributes belong to a device's context,
// so a process that launches on several devices sets it on each. Thread-safe
// (a race sets the same value twice). Devices 64 and above set it every time.
template <auto Kern>
inline void smem_attr(size_t smem) {
  static std::atomic<unsigned long long> done{0};  // bit d: set on device d
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 64;
  }
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  if (cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
      cudaSuccess) {
    if (bit) done.fetch_or(bit, std::memory_order_release);
  } else {
    cudaGetLastError();  // the launch then reports the error
  }
}

}  // namespace hz
