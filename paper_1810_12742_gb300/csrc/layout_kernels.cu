// Permutations between the natural layout and the solver layout (Section 5:
// the data of a chunk interleaved so that a warp reads one row of it as one
// contiguous run).  Internal to libhines.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace hines {
namespace {

// packed[p] = natural[perm[p]]; padding slots (perm -1) are set to zero.
template <typename W>
__global__ void k_pack(const int64_t* __restrict__ perm, int64_t n_packed, const W* __restrict__ nat,
                       W* __restrict__ pk) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_packed; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[p];
    pk[p] = i >= 0 ? nat[i] : W(0);
  }
}

// natural[perm[p]] = packed[p] for every non-padding slot.
template <typename W>
__global__ void k_unpack(const int64_t* __restrict__ perm, int64_t n_packed, const W* __restrict__ pk,
                         W* __restrict__ nat) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_packed; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = perm[p];
    if (i >= 0) nat[i] = pk[p];
  }
}

int blocks_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_pack(const DevPlan& P, int elem_bytes, const void* natural, void* packed, cudaStream_t s,
                        bool coupling) {
  if (P.n_packed == 0) return cudaSuccess;
  const int64_t* perm = coupling ? P.pk_edge : P.pk_perm;
  if (elem_bytes == 8)
    k_pack<uint64_t><<<blocks_for(P.n_packed), 256, 0, s>>>(perm, P.n_packed, (const uint64_t*)natural,
                                                             (uint64_t*)packed);
  else
    k_pack<uint32_t><<<blocks_for(P.n_packed), 256, 0, s>>>(perm, P.n_packed, (const uint32_t*)natural,
                                                             (uint32_t*)packed);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const DevPlan& P, int elem_bytes, const void* packed, void* natural, cudaStream_t s) {
  if (P.n_packed == 0) return cudaSuccess;
  if (elem_bytes == 8)
    k_unpack<uint64_t><<<blocks_for(P.n_packed), 256, 0, s>>>(P.pk_perm, P.n_packed, (const uint64_t*)packed,
                                                               (uint64_t*)natural);
  else
    k_unpack<uint32_t><<<blocks_for(P.n_packed), 256, 0, s>>>(P.pk_perm, P.n_packed, (const uint32_t*)packed,
                                                               (uint32_t*)natural);
  return cudaGetLastError();
}

}  // namespace hines
