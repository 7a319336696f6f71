// Permutations between the natural layout and the solver layout (Section 5:
// the data of a chunk interleaved so that a warp reads one row of it as one
// contiguous run).  Internal to libhines.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "unit_kernels.cuh"

namespace hines {
namespace {

// Unpacking chunk by chunk with the solve's task driver: every chunk's block
// is staged with one bulk copy (contiguous in the solver layout) and written
// out piece by piece, each piece's run contiguous in the natural layout, as
// the solves write x.  The elimination visit does nothing; every chunk is
// visited once in the substitution visit.  Plans whose pieces follow the
// caller's numbering only (re-rooted plans) use the slot-by-slot kernel below.
template <typename W, int P>
struct UnpackMode {
  using G = Geo<P>;
  static constexpr bool kPacked = false;  // pieces located by their natural first compartment
  static constexpr bool kNeedsBlk = true;
  static constexpr int kPer = P;
  struct Args {
    const W* pk;
    W* nat;
  };
  static constexpr int kTab = G::kSlots * 8;
  static constexpr int kStageBytes = kTab + 80;
  static constexpr int kStages = 1;
  static constexpr int kCacheBytes = 16;
  static constexpr int kWarpBytes = kStageBytes + kCacheBytes;
  static constexpr int kMinBlocks = 8;
  static constexpr bool kBulk = true;
  static_assert(kStageBytes % 16 == 0, "16-byte aligned staging");
  using Bulk = BulkStage<kStageBytes>;
  __device__ static void init_warp(unsigned char* wbase, int lane) { Bulk::init(wbase, lane); }

  __device__ static void stage(const DevPlan& Pl, const Args& A, int visit, Meta<P>& m, int, int lane,
                               unsigned char* buf, const Prev&) {
    if (visit == 0) return;
    int* tab = reinterpret_cast<int*>(buf + kTab);
    build_row_table<P>(m.L, lane, tab);
    // whole 16-byte words: the block's padding completes the last
    constexpr int kPerWord = 16 / (int)sizeof(W);
    const int e = (tab[kL] + kPerWord - 1) / kPerWord * kPerWord;
    Bulk::template issue<1>(buf, lane, (unsigned)(e * (int)sizeof(W)), buf, A.pk + m.blk);
  }
  __device__ static void compute(const DevPlan& Pl, const Args&, int visit, int, int, int lane, const Meta<P>&,
                                 unsigned char* buf, const Prev&, unsigned char*, int) {
    if (visit == 1) Bulk::wait(Pl, buf, lane);
  }
  __device__ static void copy_out(const DevPlan&, const Args& A, int visit, const Meta<P>& m, int n, int lane,
                                  unsigned char* buf) {
    if (visit == 0) return;
    const W* sw = reinterpret_cast<const W*>(buf);
    const int* tab = reinterpret_cast<const int*>(buf + kTab);
    for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) { A.nat[g] = sw[tab[row] + i]; });
  }
};

template <typename W, int P>
cudaError_t unpack_by_chunks(const DevPlan& Pd, const W* pk, W* nat, cudaStream_t s) {
  using M = UnpackMode<W, P>;
  int grid = 0;
  cudaError_t e = grid_of<M>(Pd, &grid);
  if (e != cudaSuccess) return e;
  return launch_phases<M>(Pd, typename M::Args{pk, nat}, grid, s);
}

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
  if (P.pk_edge == P.pk_perm && P.n_wtasks > 0) {  // pieces in the caller's numbering: chunk by chunk
    if (elem_bytes == 8)
      return P.per_lane == 2 ? unpack_by_chunks<uint64_t, 2>(P, (const uint64_t*)packed, (uint64_t*)natural, s)
                             : unpack_by_chunks<uint64_t, 1>(P, (const uint64_t*)packed, (uint64_t*)natural, s);
    return P.per_lane == 2 ? unpack_by_chunks<uint32_t, 2>(P, (const uint32_t*)packed, (uint32_t*)natural, s)
                           : unpack_by_chunks<uint32_t, 1>(P, (const uint32_t*)packed, (uint32_t*)natural, s);
  }
  if (elem_bytes == 8)
    k_unpack<uint64_t><<<blocks_for(P.n_packed), 256, 0, s>>>(P.pk_perm, P.n_packed, (const uint64_t*)packed,
                                                               (uint64_t*)natural);
  else
    k_unpack<uint32_t><<<blocks_for(P.n_packed), 256, 0, s>>>(P.pk_perm, P.n_packed, (const uint32_t*)packed,
                                                               (uint32_t*)natural);
  return cudaGetLastError();
}

}  // namespace hines
