// batch_plan.cuh — the batch plan shared by the batched kernels: the device
// table of fields over one global tile space, and the per-field output table
// of the batched producing operators.
#pragma once
#include "hz_common.cuh"

namespace hz {

// One field of a plan (device table).
struct BField {
  const uint8_t* c;
  uint8_t* cw;       // same stream, writable (in-place operators)
  Info h;
  uint64_t tile0;    // first tile in the global tile space
  uint64_t ntiles;
  uint64_t pre0;     // first word of the field's (nc, r) prefixes in pre[]
  uint64_t ch0[2];   // first 16-byte chunk of the field's metadata region: [0] negate, [1] add
  uint64_t nch[2];
  long long rho;     // scalar addition: this field's quantized scalar (0: field skipped)
};

// Index of the field holding global tile t (fields have >= 1 tile; tile0 grows).
__device__ __forceinline__ uint32_t field_of_tile(const BField* F, uint32_t nf, uint64_t t) {
  uint32_t lo = 0, hi = nf;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (F[mid].tile0 <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}
// One field of a batched producing operator's output: its caller-owned
// buffer, its tiles in the global tile space, its slot bases in the context's
// staging (sign words from sbase, plane words from pbase) and the header it
// gets (nnc, R and qbound filled in at placement; qmax is the largest |q| the
// producer met, reset by the placement kernel).
struct BOut {
  uint8_t* out;
  uint64_t cap;
  uint64_t tile0, ntiles, nb;
  uint64_t sbase, pbase;
  hoszp_header hdr;
  uint32_t qmax;
  int ok;  // 0: the field is skipped (an error was set for it)
};

}  // namespace hz

// Autotuned launch shape of one batched operator.
struct BatchCfg {
  int variant;  // 0: tile pipeline, 8 stages; 1: tile pipeline, 4 stages; 2: super-tile pipeline
  int cps;      // CTAs per SM (the tile pipeline: 1 or 2; the super-tile pipeline takes one)
  int wpg;      // super-tile pipeline: warps per block group (8 or 4)
  int gmax;     // super-tile pipeline: plane groups decoded (4: any rate; 2 or 1: rate-specialised)
};

struct hoszp_batch {
  hoszp_ctx* ctx;
  int device, num_sms;
  uint32_t nf;
  uint64_t total_tiles, total_ch[2];
  void* mem;
  hz::BField* d_fields;
  unsigned long long* d_pre;
  unsigned long long* d_acc;
  unsigned int* d_done;
  int* status;  // the plan's own status word (first device error of its operators)
  BatchCfg cfg[3];  // mean, variance, decompression
  int rmax;         // bound on every field's rates, from the headers' bounds on |q|
  // producing operators (bproduce.cu): per-field input word prefixes
  // (fpre[2f] = non-constant blocks, fpre[2f + 1] = plane words of the fields
  // before f) and the per-field output table
  unsigned long long* d_fpre;
  hz::BOut* d_out;
  uint64_t total_nnc, total_R;  // the fields' non-constant blocks and plane words
};

namespace hz {
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

inline int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return HOSZP_OK;
  cudaGetLastError();
  return HOSZP_ERR_CUDA;
}
}  // namespace hz


