// noalloc.cu — hoszp_mean_noalloc: the mean of a compressed stream for callers
// that may not allocate device memory at call time (no context, no workspace).
//
// Who needs it: code whose device memory is owned by a host framework that
// hands out every buffer from its own pool and forbids driver allocations
// while it runs, and latency-critical loops that cannot afford the implicit
// device synchronization of a cudaMalloc. Such callers cannot create a
// hoszp_ctx (its workspace is a device allocation), so this entry point keeps
// its scratch -- launch counters, the status word, the per-CTA rate totals of
// the in-kernel rate prefix and the per-CTA partial sums -- in one file-scope
// array that exists for as long as the library is loaded on a device. It runs
// the same reduction kernel as hoszp_mean, which needs no rate pre-scan.
#include "hz_kernels.cuh"

namespace hz {
namespace {

// Policy limit of this entry point: streams of at most 2^28 values (1 GiB of
// float32). The scratch below holds per-CTA records only, so its size does not
// grow with the stream.
constexpr uint64_t NA_MAX_VALUES = 1ull << 28;
constexpr uint64_t NA_MAX_GRID = 4096;  // CTAs of one launch

constexpr uint64_t NA_OFF_SYNC = 0;
constexpr uint64_t NA_OFF_STATUS = 64;
constexpr uint64_t NA_OFF_CAGG = 256;
constexpr uint64_t NA_OFF_PART = NA_OFF_CAGG + NA_MAX_GRID * sizeof(CtaAgg);
constexpr uint64_t NA_BYTES = NA_OFF_PART + NA_MAX_GRID * sizeof(Partial);  // 256 KB + 256 B
static_assert(sizeof(Sync) <= NA_OFF_STATUS && NA_OFF_CAGG % 16 == 0 && NA_OFF_PART % 16 == 0,
              "scratch regions overlap or are misaligned");

// The scratch: zero at load (rate-total flags 0 never match a published state;
// the launch epoch counts up from 0 and is never reset).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// The scratch's device address on the current device. Looked up on every call
// rather than cached: an address cached per device ordinal would be stale after
// a cudaDeviceReset, or wrong when the caller runs in a context other than the
// device's primary one. The lookup allocates nothing.
int scratch_base(unsigned char** base) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return HOSZP_ERR_CUDA;
  }
  *base = static_cast<unsigned char*>(p);
  return HOSZP_OK;
}

// Streams of more than NA_MAX_VALUES values are refused.
__global__ void k_na_check(const uint8_t* c, uint64_t c_bytes, int* status) {
  const Info h = parse_header(c, c_bytes);
  if (h.ok && h.n > NA_MAX_VALUES) set_status(status, HOSZP_ERR_CAPACITY);
}

// Copies the call's status out; a refused stream's result becomes NaN.
__global__ void k_na_status(const int* status, int* d_status, double* d_result) {
  const int st = *status;
  *d_status = st;
  if (st == HOSZP_ERR_CAPACITY) *d_result = __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" int hoszp_mean_noalloc(const void* d_c, size_t c_bytes, double* d_result,
                                  int* d_status, hoszp_stream_t stream) {
  if (!d_c || !d_result || !d_status || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (((uintptr_t)d_c & 15u) || ((uintptr_t)d_result & 7u) || ((uintptr_t)d_status & 3u))
    return HOSZP_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return HOSZP_ERR_CUDA;
  }
  if ((uint64_t)sms * 8 > NA_MAX_GRID) return HOSZP_ERR_CAPACITY;  // persistent grids cap at 8/SM
  unsigned char* base = nullptr;
  const int rc = scratch_base(&base);
  if (rc) return rc;
  Ws w{};
  w.sync = reinterpret_cast<Sync*>(base + NA_OFF_SYNC);
  w.status = reinterpret_cast<int*>(base + NA_OFF_STATUS);
  w.partials = reinterpret_cast<Partial*>(base + NA_OFF_PART);
  w.cta_agg = reinterpret_cast<CtaAgg*>(base + NA_OFF_CAGG);
  w.max_grid = NA_MAX_GRID;
  // no rate pre-scan, descriptor chains or totals: the mean kernel finds the
  // rate prefix itself
  const cudaStream_t s = (cudaStream_t)stream;
  // the status word starts at zero for every call
  if (cudaMemsetAsync(w.status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return HOSZP_ERR_CUDA;
  }
  const uint8_t* c = static_cast<const uint8_t*>(d_c);
  k_na_check<<<1, 1, 0, s>>>(c, c_bytes, w.status);
  Launch lc;
  lc.grid = sms;
  lc.stream = s;
  if (cudaGetLastError() != cudaSuccess) return HOSZP_ERR_CUDA;
  if (launch_moments(lc, c, c_bytes, d_result, false, w) != cudaSuccess) {
    cudaGetLastError();
    return HOSZP_ERR_CUDA;
  }
  k_na_status<<<1, 1, 0, s>>>(w.status, d_status, d_result);
  return cudaGetLastError() == cudaSuccess ? HOSZP_OK : HOSZP_ERR_CUDA;
}
