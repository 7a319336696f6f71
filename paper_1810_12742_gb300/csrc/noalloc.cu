// Allocation-free FP64 solve.
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool that forbids cudaMalloc, an allocator-hooked host runtime, or a
// library entry point that must not change the device's memory footprint
// after start-up.  They cannot create a plan (plan creation allocates the
// metadata and the workspace), so this entry point needs neither: it takes
// the batch's structure as device arrays and solves every cell with one
// thread, keeping the eliminated diagonal -- the only scratch the solve
// needs -- in a fixed file-scope device array.  It never calls cudaMalloc,
// cudaFree or an allocating library routine.
//
// The scratch array holds kNoAllocMaxUnknowns doubles (16 MiB).  It is part
// of the library's device image, so every GPU that loads libhines holds it
// until the process exits.  Every call shares it and finds the previous
// call's values in it; the solve overwrites every entry it reads before
// reading it, so nothing needs clearing, but calls whose kernels overlap on
// the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hines.h"

namespace {

constexpr long long kNoAllocMaxUnknowns = 1LL << 21;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_diag[kNoAllocMaxUnknowns];

std::mutex g_setup_mutex;
double* g_diag_addr[kMaxDevices] = {};

// In host code g_noalloc_diag names a host-side stand-in, not device memory,
// so the device address is looked up once per device, with that device
// current, and passed to the kernel.
hines_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HINES_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_diag_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_diag) != cudaSuccess || !p) {
      cudaGetLastError();
      return HINES_ERR_CUDA;
    }
    g_diag_addr[dev] = static_cast<double*>(p);
  }
  *out = g_diag_addr[dev];
  return HINES_OK;
}

// One thread per cell solves it serially (Section 2's Hines algorithm, with
// the per-child coupling u[i] = A[i][p[i]]): rows are folded into their parent
// rows from the last to the first, which leaves one coupling per row, to the
// parent, and the rows are then solved from the root outwards.  The eliminated
// diagonal lives in the scratch array at the cell's natural-layout offsets.  A
// cell whose offsets or parent indices are out of range is left unsolved and
// its right-hand side is set to NaN, so a bad input never leads to an access
// outside the arrays.
__global__ void k_noalloc_solve(long long n_unknowns, int n_cells, const long long* __restrict__ off,
                                const int* __restrict__ p, const double* __restrict__ d,
                                const double* __restrict__ u, double* __restrict__ b, double* __restrict__ dd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const long long lo = off[c], hi = off[c + 1];
  if (lo < 0 || hi < lo || hi > n_unknowns) return;
  const long long n = hi - lo;
  if (n == 0) return;
  const int* pc = p + lo;
  const double* uc = u + lo;
  double* bc = b + lo;
  double* diag = dd + lo;
  bool ok = pc[0] == -1;
  for (long long i = 1; i < n && ok; ++i) ok = pc[i] >= 0 && (long long)pc[i] < i;
  if (!ok) {
    for (long long i = 0; i < n; ++i) bc[i] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  for (long long i = 0; i < n; ++i) diag[i] = d[lo + i];
  for (long long row = n - 1; row > 0; --row) {  // fold row into its parent row
    const int par = pc[row];
    const double l = uc[row] / diag[row];
    diag[par] -= l * uc[row];
    bc[par] -= l * bc[row];
  }
  for (long long row = 0; row < n; ++row) {  // root outwards: the parent's unknown is known
    const double known = row == 0 ? 0.0 : uc[row] * bc[pc[row]];
    bc[row] = (bc[row] - known) / diag[row];
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
  double* dd = nullptr;
  hines_status st = scratch_for_current_device(&dd);
  if (st != HINES_OK) return st;
  const int threads = 128;
  const int blocks = (n_cells + threads - 1) / threads;
  k_noalloc_solve<<<blocks, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      (long long)n_unknowns, n_cells, reinterpret_cast<const long long*>(cell_offsets), parent, d, u, b_inout, dd);
  return cudaGetLastError() == cudaSuccess ? HINES_OK : HINES_ERR_CUDA;
}
