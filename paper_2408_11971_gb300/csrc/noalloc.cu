// noalloc.cu — hoszp_mean_noalloc: the mean of a compressed stream for callers
// that may not allocate device memory at call time (no context, no workspace).
//
// Who needs it: code whose device memory is owned by a host framework that
// hands out every buffer from its own pool and forbids driver allocations
// while it runs, and latency-critical loops that cannot afford the implicit
// device synchronization of a cudaMalloc. Such callers cannot create a
// hoszp_ctx (its workspace is a device allocation), so this entry point keeps
// its scratch -- launch counters, status word, the per-CTA rate aggregates,
// the per-CTA partial sums and room for a rate pre-scan -- in one
// file-scope array that exists for as long as the library is loaded on a
// device. It runs the same rate pre-scan and reduction kernels as hoszp_mean.
#include <mutex>

#include "hz_kernels.cuh"

namespace hz {
namespace {

constexpr uint64_t NA_MAX_VALUES = 1ull << 28;                      // 1 GiB of float32
constexpr uint64_t NA_MAX_TILES = NA_MAX_VALUES / TILE_VALUES + 2;  // pre[] entries (+ totals)
constexpr uint64_t NA_MAX_SUPER = NA_MAX_TILES / 64 + 2;            // pre-scan look-back steps
constexpr uint64_t NA_MAX_GRID = 4096;                              // CTAs of one launch

constexpr uint64_t NA_OFF_SYNC = 0;
constexpr uint64_t NA_OFF_STATUS = 64;
constexpr uint64_t NA_OFF_TOTALS = 128;
constexpr uint64_t NA_OFF_DESC = 256;
constexpr uint64_t NA_OFF_PRE = NA_OFF_DESC + NA_MAX_SUPER * sizeof(Desc);
constexpr uint64_t NA_OFF_CAGG = NA_OFF_PRE + 2 * (NA_MAX_TILES + 1) * 8;
constexpr uint64_t NA_OFF_PART = NA_OFF_CAGG + NA_MAX_GRID * sizeof(CtaAgg);
constexpr uint64_t NA_BYTES = NA_OFF_PART + NA_MAX_GRID * sizeof(Partial);

// The scratch: zero at load (look-back flags 0 never match a published state;
// the launch epoch counts up from 0 and is never reset).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mutex;
unsigned char* g_base[NA_MAX_DEVICES];  // device address of the scratch, per device
int g_sms[NA_MAX_DEVICES];

// Once per device, with that device current: the address of the scratch.
int setup(int dev, unsigned char** base, int* sms) {
  if (dev < 0 || dev >= NA_MAX_DEVICES) return HOSZP_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return HOSZP_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return HOSZP_ERR_CUDA;
    }
    g_sms[dev] = n;
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  *base = g_base[dev];
  *sms = g_sms[dev];
  return HOSZP_OK;
}

// Streams of more than NA_MAX_VALUES values do not fit the scratch.
__global__ void k_na_check(const uint8_t* c, uint64_t c_bytes, int* status) {
  const Info h = parse_header(c, c_bytes);
  if (h.ok && h.n > NA_MAX_VALUES) set_status(status, HOSZP_ERR_CAPACITY);
}

__global__ void k_na_status(const int* status, int* d_status) { *d_status = *status; }

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" int hoszp_mean_noalloc(const void* d_c, size_t c_bytes, double* d_result,
                                  int* d_status, hoszp_stream_t stream) {
  if (!d_c || !d_result || !d_status || c_bytes < HOSZP_HEADER_BYTES) return HOSZP_ERR_ARG;
  if (((uintptr_t)d_c & 15u) || ((uintptr_t)d_result & 7u) || ((uintptr_t)d_status & 3u))
    return HOSZP_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HOSZP_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  int sms = 0;
  int rc = setup(dev, &base, &sms);
  if (rc) return rc;
  if ((uint64_t)sms * 8 > NA_MAX_GRID) return HOSZP_ERR_CAPACITY;  // persistent grids cap at 8/SM
  Ws w{};
  w.sync = reinterpret_cast<Sync*>(base + NA_OFF_SYNC);
  w.status = reinterpret_cast<int*>(base + NA_OFF_STATUS);
  w.totals = reinterpret_cast<unsigned long long*>(base + NA_OFF_TOTALS);
  for (int k = 0; k < NCHAIN; k++) w.desc[k] = reinterpret_cast<Desc*>(base + NA_OFF_DESC);
  w.max_tiles = NA_MAX_TILES;
  w.partials = reinterpret_cast<Partial*>(base + NA_OFF_PART);
  w.cta_agg = reinterpret_cast<CtaAgg*>(base + NA_OFF_CAGG);
  w.max_grid = NA_MAX_GRID;
  w.pre[0] = w.pre[1] = reinterpret_cast<unsigned long long*>(base + NA_OFF_PRE);
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
  k_na_status<<<1, 1, 0, s>>>(w.status, d_status);
  return cudaGetLastError() == cudaSuccess ? HOSZP_OK : HOSZP_ERR_CUDA;
}
