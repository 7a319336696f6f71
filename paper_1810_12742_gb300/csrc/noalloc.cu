// Allocation-free FP64 solve.
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool that forbids cudaMalloc, an allocator-hooked host runtime, or a
// library entry point that must not change the device's memory footprint
// after start-up.  They cannot create a plan (plan creation allocates the
// metadata and the workspace), so this entry point needs neither: it takes
// the batch's structure as device arrays and solves every cell with one
// thread.  Its only scratch -- a validity word and the eliminated diagonal --
// lives in a fixed file-scope device array.  It never calls cudaMalloc,
// cudaFree or an allocating library routine.
//
// The scratch array holds kNoAllocMaxUnknowns doubles of diagonal plus a
// 256-byte header (16 MiB in all).  It is part of the library's device image,
// so every GPU that loads libhines holds it until the process exits.  Every
// call shares it and finds the previous call's values in it; each call
// rewrites the header and every diagonal entry it reads before reading it,
// so nothing needs clearing, but calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hines.h"

namespace {

constexpr long long kNoAllocMaxUnknowns = 1LL << 21;
constexpr long long kHeader = 32;  // doubles (256 bytes) before the diagonal: the validity word
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kHeader + kNoAllocMaxUnknowns];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory, so the device address is looked up once per device, with that
// device current, and passed to the kernels.
hines_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HINES_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HINES_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return HINES_OK;
}

// One block checks the offsets: off[0] = 0, non-decreasing, off[n_cells] <=
// n_unknowns.  The header word becomes 1 when they are not (then no cell is
// solved and every entry of b is set to NaN), else 0.
__global__ void k_noalloc_check(long long n_unknowns, int n_cells, const long long* __restrict__ off,
                                unsigned long long* __restrict__ bad_word) {
  int bad = 0;
  for (int c = threadIdx.x; c <= n_cells; c += blockDim.x) {
    const long long o = off[c];
    if (o < 0 || o > n_unknowns || (c == 0 && o != 0) || (c > 0 && o < off[c - 1])) bad = 1;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) *bad_word = bad ? 1ull : 0ull;
}

// One thread per cell.  Elimination from the last compartment to the first:
// an unbranched run (parent[i] == i - 1) is a Thomas chain whose pivot and
// right-hand side pass to the next compartment in registers; where a branch
// starts (parent[i] != i - 1) the row is folded into its parent row in
// memory (the parent's pivot in the scratch diagonal, its right-hand side in
// b), to be picked up when the walk reaches the parent.  Substitution from
// the root outwards, the chain's last solution again kept in a register.
// A cell whose parent array breaks Hines order (p[0] = -1, 0 <= p[i] < i)
// is set to NaN and not solved, so no index ever leaves the cell.
__global__ void k_noalloc_solve(long long n_unknowns, int n_cells, const long long* __restrict__ off,
                                const int* __restrict__ p, const double* __restrict__ d,
                                const double* __restrict__ u, double* __restrict__ b, double* __restrict__ scratch) {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (*reinterpret_cast<const unsigned long long*>(scratch) != 0ull) {  // offsets rejected by k_noalloc_check
    for (long long i = tid; i < n_unknowns; i += stride) b[i] = nan;
    return;
  }
  if (tid >= n_cells) return;
  const long long lo = off[tid], n = off[tid + 1] - lo;
  if (n == 0) return;
  const int* pc = p + lo;
  const double* dc = d + lo;
  const double* uc = u + lo;
  double* bc = b + lo;
  double* piv = scratch + kHeader + lo;
  bool ok = pc[0] == -1;
  for (long long i = 1; i < n && ok; ++i) ok = pc[i] >= 0 && (long long)pc[i] < i;
  if (!ok) {
    for (long long i = 0; i < n; ++i) bc[i] = nan;
    return;
  }
  for (long long i = 0; i < n; ++i) piv[i] = dc[i];
  double D = piv[n - 1], B = bc[n - 1];
  for (long long i = n - 1; i > 0; --i) {
    piv[i] = D;
    bc[i] = B;
    const double f = uc[i] / D;
    const long long q = pc[i];
    if (q == i - 1) {  // chain: the parent is the next row of the walk
      D = piv[i - 1] - f * uc[i];
      B = bc[i - 1] - f * B;
    } else {  // branch start: fold into the parent row, continue with row i - 1 as it stands
      piv[q] -= f * uc[i];
      bc[q] -= f * B;
      D = piv[i - 1];
      B = bc[i - 1];
    }
  }
  double x = B / D;  // the root
  bc[0] = x;
  for (long long i = 1; i < n; ++i) {
    const long long q = pc[i];
    const double xp = q == i - 1 ? x : bc[q];
    x = (bc[i] - uc[i] * xp) / piv[i];
    bc[i] = x;
  }
}

}  // namespace

extern "C" hines_status hines_solve_f64_noalloc(int64_t n_unknowns, int32_t n_cells, const int64_t* cell_offsets,
                                                const int32_t* parent, const double* d, const double* u,
                                                double* b_inout, hines_stream_t stream) {
  if (n_unknowns < 0 || n_cells < 0) return HINES_ERR_INVALID_ARG;
  if (n_unknowns > kNoAllocMaxUnknowns) return HINES_ERR_INVALID_ARG;
  if (n_cells == 0 || n_unknowns == 0) return HINES_OK;
  if (!cell_offsets || !parent || !d || !u || !b_inout) return HINES_ERR_INVALID_ARG;
  double* scratch = nullptr;
  hines_status st = scratch_for_current_device(&scratch);
  if (st != HINES_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long* off = reinterpret_cast<const long long*>(cell_offsets);
  k_noalloc_check<<<1, 256, 0, s>>>((long long)n_unknowns, n_cells, off,
                                    reinterpret_cast<unsigned long long*>(scratch));
  const int threads = 128;
  const int blocks = (n_cells + threads - 1) / threads;
  k_noalloc_solve<<<blocks, threads, 0, s>>>((long long)n_unknowns, n_cells, off, parent, d, u, b_inout, scratch);
  return cudaGetLastError() == cudaSuccess ? HINES_OK : HINES_ERR_CUDA;
}
