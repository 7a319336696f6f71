// Host pipeline: the compensated solve from host arrays, with the transfers
// overlapped (hines_pipeline_*).
//
// The batch is cut into runs of consecutive cells of about equal size, each
// with its own plan and device buffers.  A solve enqueues, per piece, the
// host-to-device copies of d, u, b on one stream, the device solve on a
// second and the device-to-host copy of x on a third, joined by events, so
// that piece k is solved while piece k+1 arrives and piece k-1 leaves.  All
// of it is ordered after the caller's stream and the caller's stream waits
// for all of it, so the call behaves like one stream-ordered operation.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/hines.h"

struct hines_pipeline_s {
  struct Piece {
    int64_t lo = 0, n = 0;  // first compartment in the batch, compartments
    hines_plan_t plan = nullptr;
    float *d = nullptr, *u = nullptr, *b = nullptr;
    double* x = nullptr;
    cudaEvent_t in = nullptr, done = nullptr;
  };
  std::vector<Piece> pieces;
  int64_t n_unknowns = 0;
  int32_t n_cells = 0;
  int device = -1;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  cudaEvent_t start = nullptr, end_in = nullptr, end_run = nullptr, end_out = nullptr;
};

namespace {

void release(hines_pipeline_s* p) {
  if (!p) return;
  for (cudaStream_t s : {p->s_in, p->s_run, p->s_out})
    if (s) cudaStreamSynchronize(s);
  for (auto& q : p->pieces) {
    if (q.plan) hines_plan_destroy(q.plan);
    for (void* a : {(void*)q.d, (void*)q.u, (void*)q.b, (void*)q.x})
      if (a) cudaFree(a);
    for (cudaEvent_t e : {q.in, q.done})
      if (e) cudaEventDestroy(e);
  }
  for (cudaEvent_t e : {p->start, p->end_in, p->end_run, p->end_out})
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : {p->s_in, p->s_run, p->s_out})
    if (s) cudaStreamDestroy(s);
  cudaGetLastError();
  delete p;
}

bool make_event(cudaEvent_t* e) { return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess; }

}  // namespace

extern "C" {

hines_status hines_pipeline_create(hines_pipeline_t* out, int32_t n_cells, const int32_t* ncomp,
                                   const int32_t* parent, int32_t pieces, const hines_plan_opts* opts) {
  if (!out) return HINES_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_cells < 0 || pieces < 1 || (n_cells > 0 && (!ncomp || !parent))) return HINES_ERR_INVALID_ARG;
  if (opts && opts->host_only) return HINES_ERR_INVALID_ARG;
  std::vector<int64_t> off((size_t)n_cells + 1, 0);
  for (int32_t c = 0; c < n_cells; ++c) {
    if (ncomp[c] < 0) return HINES_ERR_INVALID_ARG;
    off[(size_t)c + 1] = off[(size_t)c] + ncomp[c];
  }
  const int64_t total = off[(size_t)n_cells];
  // cell boundaries closest to equal compartment counts (first boundary at
  // or above each k / pieces of the total), duplicates dropped
  std::vector<int32_t> bounds{0};
  const int32_t np = std::max(1, std::min(pieces, std::max(n_cells, 1)));
  for (int32_t k = 1; k < np; ++k) {
    const int64_t target = (total * k) / np;
    const int32_t c = (int32_t)(std::lower_bound(off.begin(), off.end(), target) - off.begin());
    if (c > bounds.back() && c < n_cells) bounds.push_back(c);
  }
  if (n_cells > bounds.back()) bounds.push_back(n_cells);
  auto* p = new (std::nothrow) hines_pipeline_s;
  if (!p) return HINES_ERR_OOM;
  p->n_unknowns = total;
  p->n_cells = n_cells;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    release(p);
    return HINES_ERR_CUDA;
  }
  bool ok = true;
  for (cudaStream_t* s : {&p->s_in, &p->s_run, &p->s_out})
    ok = ok && cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) == cudaSuccess;
  for (cudaEvent_t* e : {&p->start, &p->end_in, &p->end_run, &p->end_out}) ok = ok && make_event(e);
  if (!ok) {
    release(p);
    return HINES_ERR_CUDA;
  }
  for (size_t k = 0; k + 1 < bounds.size(); ++k) {
    hines_pipeline_s::Piece q;
    const int32_t c0 = bounds[k], c1 = bounds[k + 1];
    q.lo = off[(size_t)c0];
    q.n = off[(size_t)c1] - q.lo;
    p->pieces.push_back(q);
    hines_pipeline_s::Piece& r = p->pieces.back();
    hines_status st = hines_plan_create(&r.plan, c1 - c0, ncomp + c0, parent + r.lo, opts);
    if (st != HINES_OK) {
      release(p);
      return st;
    }
    const size_t n = (size_t)std::max<int64_t>(r.n, 1);
    if (cudaMalloc(&r.d, n * 4) != cudaSuccess || cudaMalloc(&r.u, n * 4) != cudaSuccess ||
        cudaMalloc(&r.b, n * 4) != cudaSuccess || cudaMalloc(&r.x, n * 8) != cudaSuccess) {
      release(p);
      return HINES_ERR_OOM;
    }
    if (!make_event(&r.in) || !make_event(&r.done)) {
      release(p);
      return HINES_ERR_CUDA;
    }
  }
  *out = p;
  return HINES_OK;
}

hines_status hines_pipeline_info(hines_pipeline_t p, int32_t* pieces, int64_t* n_unknowns) {
  if (!p) return HINES_ERR_INVALID_ARG;
  if (pieces) *pieces = (int32_t)p->pieces.size();
  if (n_unknowns) *n_unknowns = p->n_unknowns;
  return HINES_OK;
}

hines_status hines_pipeline_solve_compensated(hines_pipeline_t p, const float* d, const float* u, const float* b,
                                              double* x_out, hines_stream_t stream) {
  if (!p) return HINES_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HINES_ERR_CUDA;
  if (dev != p->device) return HINES_ERR_DEVICE;
  if (p->n_unknowns == 0) return HINES_OK;
  if (!d || !u || !b || !x_out) return HINES_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventRecord(p->start, s);
  for (cudaStream_t t : {p->s_in, p->s_run, p->s_out})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(t, p->start, 0);
  for (auto& q : p->pieces) {
    if (e != cudaSuccess) break;
    if (q.n == 0) continue;
    const size_t n = (size_t)q.n;
    e = cudaMemcpyAsync(q.d, d + q.lo, n * 4, cudaMemcpyHostToDevice, p->s_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q.u, u + q.lo, n * 4, cudaMemcpyHostToDevice, p->s_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q.b, b + q.lo, n * 4, cudaMemcpyHostToDevice, p->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(q.in, p->s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_run, q.in, 0);
    if (e != cudaSuccess) break;
    const hines_status st =
        hines_solve_compensated(q.plan, q.d, q.u, q.b, q.x, reinterpret_cast<hines_stream_t>(p->s_run));
    if (st != HINES_OK) return st;
    e = cudaEventRecord(q.done, p->s_run);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_out, q.done, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x_out + q.lo, q.x, n * 8, cudaMemcpyDeviceToHost, p->s_out);
  }
  // the caller's stream waits for all three
  if (e == cudaSuccess) e = cudaEventRecord(p->end_in, p->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(p->end_run, p->s_run);
  if (e == cudaSuccess) e = cudaEventRecord(p->end_out, p->s_out);
  for (cudaEvent_t ev : {p->end_in, p->end_run, p->end_out})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HINES_ERR_CUDA;
  }
  return HINES_OK;
}

hines_status hines_pipeline_status(hines_pipeline_t p, int32_t* status) {
  if (!p || !status) return HINES_ERR_INVALID_ARG;
  *status = 0;
  for (auto& q : p->pieces) {
    int32_t s = 0;
    const hines_status st = hines_plan_status(q.plan, &s);
    if (st != HINES_OK) return st;
    if (s > *status) *status = s;
  }
  return HINES_OK;
}

hines_status hines_pipeline_destroy(hines_pipeline_t p) {
  release(p);
  return HINES_OK;
}

}  // extern "C"
