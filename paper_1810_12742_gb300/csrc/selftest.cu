// Check of the bounded device wait (hines_check_bounded_wait).
//
// Staging of contiguous blocks waits on a shared-memory barrier with a
// bounded number of polls; a wait that runs out raises HINES_ERR_TIMEOUT in
// the plan's status word and the kernel goes on instead of hanging.  This
// entry point makes such a wait run out on purpose, without any fault: one
// CTA initialises a barrier that expects one arrival and, unless asked to
// make that arrival itself, polls it a given number of times with nothing
// in flight (no copy is ever issued), then records the status it would raise
// and the time the polls took, and returns.  The context stays usable.
#include <cuda_runtime.h>

#include "../../include/hines.h"
#include "device_common.cuh"

namespace hines {
namespace {

__global__ void k_bounded_wait(int polls, int arrive, int32_t* status, unsigned long long* ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) dev::mbar_init(&bar);
  __syncthreads();
  if (arrive && threadIdx.x == 0) dev::mbar_expect_tx(&bar, 0);  // the one arrival, no bytes: the phase completes
  unsigned long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  const bool done = dev::mbar_wait(&bar, 0u, polls);
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  if (threadIdx.x == 0) {
    if (!done) atomicCAS(status, 0, (int32_t)HINES_ERR_TIMEOUT);
    *ns = t1 - t0;
  }
}

}  // namespace
}  // namespace hines

extern "C" hines_status hines_check_bounded_wait(int32_t polls, int32_t arrive, int32_t* status_out,
                                                 int64_t* elapsed_ns) {
  if (polls < 1 || polls > (1 << 16) || !status_out) return HINES_ERR_INVALID_ARG;
  struct Out {
    int32_t status;
    int32_t pad;
    unsigned long long ns;
  };
  Out* d = nullptr;
  if (cudaMalloc(&d, sizeof(Out)) != cudaSuccess) {
    cudaGetLastError();
    return HINES_ERR_OOM;
  }
  Out h{0, 0, 0};
  cudaError_t e = cudaMemset(d, 0, sizeof(Out));
  if (e == cudaSuccess) {
    hines::k_bounded_wait<<<1, 32>>>(polls, arrive ? 1 : 0, &d->status, &d->ns);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(Out), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HINES_ERR_CUDA;
  }
  *status_out = h.status;
  if (elapsed_ns) *elapsed_ns = (int64_t)h.ns;
  return HINES_OK;
}
