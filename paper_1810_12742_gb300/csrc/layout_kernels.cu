// Permutations between the natural layout and the solver layout (Section 5:
// the data of a chunk interleaved so that a warp reads one row of it as one
// contiguous run).  Internal to libhines.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "unit_kernels.cuh"

namespace hines {
namespace {

// Unpacking chunk by chunk with the solve's task driver.  A chunk's block is
// contiguous in the solver layout (row r: the r-th compartment from the
// distal end of every piece longer than r), and each of its pieces is one
// contiguous run in the plan's numbering.  The block arrives in shared
// memory in block order (R) by one bulk copy; each lane moves the slots of
// its own pieces, row by row (consecutive words of R), into piece order (C:
// one row of kPitch words per piece, kPitch odd); half-warps then write each
// piece's run to the natural layout (consecutive words of C).  Neither side
// conflicts on shared-memory banks, and every global write is a contiguous
// run, as the solves write x.  Only the substitution visit does anything, so
// every chunk is handled once.  kMapped: the plan's numbering is not the
// caller's (re-rooted plans), so the caller's index of every slot comes from
// the plan's slot map.
//
// (Packing stays slot by slot: a chunk-wise gather measured slower than the
// plain kernel below, 1.02 against 0.66 ms per FP32 array of the full
// uneven population, which reads scattered but writes contiguously.)
template <typename W, int P, bool kMapped>
struct UnpackMode {
  using G = Geo<P>;
  static constexpr bool kPacked = false;  // pieces located by their first compartment in the plan's numbering
  static constexpr bool kNeedsBlk = true;
  static constexpr int kPer = P;
  struct Args {
    const W* src;
    W* dst;
    const int64_t* map;  // kMapped: the caller's index of every slot (-1: padding)
  };
  static constexpr int kPitch = kL + 1;
  static constexpr int kRowBytes = G::kSlots * 8;              // R (holds a padded block)
  static constexpr int kColBytes = G::kChunk * kPitch * 8;     // C
  static constexpr int kTab = kRowBytes + kColBytes;           // the block's row offsets
  static constexpr int kStageBytes = kTab + 80;
  static constexpr int kStages = 1;
  static constexpr int kCacheBytes = 16;
  static constexpr int kWarpBytes = kStageBytes + kCacheBytes;
  static constexpr int kMinBlocks = 8;
  static_assert(kRowBytes % 16 == 0 && kColBytes % 16 == 0 && kStageBytes % 16 == 0, "16-byte aligned regions");
  using Bulk = BulkStage<kStageBytes>;
  __device__ static void init_warp(unsigned char* wbase, int lane) { Bulk::init(wbase, lane); }

  // the block with its padding: blocks start on multiples of 4 slots, so
  // this is the distance to the next block (whole 16-byte words)
  __device__ static int padded(const int* tab) { return (tab[kL] + 3) & ~3; }
  __device__ static W* rows_of(unsigned char* buf) { return reinterpret_cast<W*>(buf); }
  __device__ static W* cols_of(unsigned char* buf) { return reinterpret_cast<W*>(buf + kRowBytes); }

  // every slot of the lane's pieces, row by row: f(slot in R, word in C)
  template <typename F>
  __device__ static void for_lane_slots(const Meta<P>& m, int lane, const int* tab, F&& f) {
    const int L = m.L;
    for (int r = 0; r < L; ++r) {
      const int t = L - 1 - r;  // distance from the proximal end (pieces of a pair aligned there)
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const int i = P * lane + h;
        if (t < m.p[h].len) f(tab[r] + i, i * kPitch + t);
      }
    }
  }

  __device__ static void stage(const DevPlan&, const Args& A, int visit, Meta<P>& m, int n, int lane,
                               unsigned char* buf, const Prev&) {
    if (visit == 0) return;
    int* tab = reinterpret_cast<int*>(buf + kTab);
    build_row_table<P>(m.L, lane, tab);
    Bulk::template issue<1>(buf, lane, (unsigned)(padded(tab) * (int)sizeof(W)), buf, A.src + m.blk);
  }
  __device__ static void compute(const DevPlan& Pl, const Args&, int visit, int, int, int lane, const Meta<P>& m,
                                 unsigned char* buf, const Prev&, unsigned char*, int) {
    if (visit == 0) return;
    const int* tab = reinterpret_cast<const int*>(buf + kTab);
    W* sr = rows_of(buf);
    W* sc = cols_of(buf);
    Bulk::wait(Pl, buf, lane);
    for_lane_slots(m, lane, tab, [&](int q, int c) { sc[c] = sr[q]; });
  }
  __device__ static void copy_out(const DevPlan&, const Args& A, int visit, const Meta<P>& m, int n, int lane,
                                  unsigned char* buf) {
    if (visit == 0) return;
    const int* tab = reinterpret_cast<const int*>(buf + kTab);
    const W* sc = cols_of(buf);
    for_chunk_elements(m, n, lane, [&](int i, int t, int row, long long g, bool) {
      const W v = sc[i * kPitch + t];
      if constexpr (kMapped) {
        const long long c = __ldg(A.map + m.blk + tab[row] + i);
        if (c >= 0) A.dst[c] = v;
      } else {
        A.dst[g] = v;
      }
    });
  }
};

template <typename W, int P, bool kMapped>
cudaError_t unpack_by_chunks(const DevPlan& Pd, const W* pk, W* nat, cudaStream_t s) {
  using M = UnpackMode<W, P, kMapped>;
  int grid = 0;
  cudaError_t e = grid_of<M>(Pd, &grid);
  if (e != cudaSuccess) return e;
  return launch_phases<M>(Pd, typename M::Args{pk, nat, Pd.pk_perm}, grid, s);
}

template <typename W>
cudaError_t unpack(const DevPlan& Pd, const void* packed, void* natural, cudaStream_t s) {
  const bool mapped = Pd.pk_edge != Pd.pk_perm;  // re-rooted: the plan's numbering is its own
  const W* pk = static_cast<const W*>(packed);
  W* nat = static_cast<W*>(natural);
  if (Pd.per_lane == 2)
    return mapped ? unpack_by_chunks<W, 2, true>(Pd, pk, nat, s) : unpack_by_chunks<W, 2, false>(Pd, pk, nat, s);
  return mapped ? unpack_by_chunks<W, 1, true>(Pd, pk, nat, s) : unpack_by_chunks<W, 1, false>(Pd, pk, nat, s);
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
  return elem_bytes == 8 ? unpack<uint64_t>(P, packed, natural, s) : unpack<uint32_t>(P, packed, natural, s);
}

}  // namespace hines
