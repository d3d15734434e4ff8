// selftest.cu — runs one of the library's bounded device waits on a flag that
// nothing sets, so that a test can watch the wait give up: the kernel must set
// HOSZP_ERR_TIMEOUT in the context's status word and return, and the context
// must stay usable. The waits are the ones every pipeline uses: the
// decoupled look-back's poll loop (a predecessor that never publishes) and the
// mbarrier wait of the copy rings (a stage that never lands).
#include "hz_pipe.cuh"
#include "hz_kernels.cuh"

namespace hz {

__global__ void k_wait_selftest(int which, long long limit, Ws ws) {
  if (which == 0) {
    // tile 1's look-back finds tile 0 unpublished under an epoch no launch uses
    const unsigned long long never = launch_epoch(ws) + (1ull << 40);
    unsigned long long pnc = 0, pr = 0;
    lookback(ws.desc[0], 1, never, ws.status, pnc, pr, limit);
  } else {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);  // one arrival expected; none comes
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, ws.status, (unsigned long long)limit);
  }
}

cudaError_t launch_wait_selftest(const Launch& lc, int which, long long limit, Ws ws) {
  k_wait_selftest<<<1, 32, 0, lc.stream>>>(which, limit, ws);
  return cudaGetLastError();
}

}  // namespace hz
