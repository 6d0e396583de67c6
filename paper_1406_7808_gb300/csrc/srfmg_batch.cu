// Batched solves: many right-hand sides, on grids of different sizes, solved
// by one CUDA graph launch.
//
// A batch holds a set of solver handles (each with its own plan and
// workspace, so problems of any size and precision mix).  The first solve
// for a given set of f / u pointers captures every handle's solve into one
// CUDA graph on the batch's own origin stream (the caller's stream may be the
// legacy default stream, which cannot be captured; events order the graph
// after the caller's earlier work and the caller's later work after it): the
// problems are spread over `streams` capture streams that fork from and join
// back to the origin stream, biggest problems first,
// each stream taking the next problem when its queued work (n^3 summed) is
// the smallest, so the graph's branches are balanced.  Later solves with the
// same pointers relaunch the graph.  sr_fmg_batch_autotune times the graph
// for 1, 2, 4, ... streams and keeps the fastest; the results do not depend
// on the choice (every problem runs the same kernels in the same order).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "srfmg.h"
#include "srfmg_internal.cuh"

struct sr_fmg_batch_s {
  std::vector<sr_fmg_t> hs;
  int device = 0;
  int streams = 1;                       // branches of the captured graph
  std::vector<cudaStream_t> side;        // capture streams
  std::vector<cudaEvent_t> events;       // fork / join events
  cudaStream_t origin = nullptr;         // stream the graph is captured and launched on
  cudaEvent_t before = nullptr, after = nullptr;  // caller stream <-> origin ordering
  cudaGraphExec_t exec = nullptr;
  std::vector<const double*> f_cached;   // pointers the graph was captured with
  std::vector<double*> u_cached;
  std::vector<long long> gen_cached;     // the handles' generations at capture
  int captured_streams = 0;
};

namespace {

bool device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void drop_graph(sr_fmg_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->captured_streams = 0;
}

int ensure_streams(sr_fmg_batch_s* b, int streams) {
  while ((int)b->side.size() < streams) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SR_ERR_CUDA;
    b->side.push_back(s);
  }
  while ((int)b->events.size() < streams + 1) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SR_ERR_CUDA;
    b->events.push_back(e);
  }
  return SR_OK;
}

// problem -> branch: biggest first, each to the least loaded branch
std::vector<std::vector<int>> assign(const sr_fmg_batch_s* b, int streams) {
  std::vector<int> order(b->hs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  auto work = [&](int i) {
    return (double)srfmg::handle_cells(b->hs[i]);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work(a) > work(c); });
  std::vector<std::vector<int>> lanes(streams);
  std::vector<double> load(streams, 0.0);
  for (int i : order) {
    int best = 0;
    for (int s = 1; s < streams; ++s)
      if (load[s] < load[best]) best = s;
    lanes[best].push_back(i);
    load[best] += work(i);
  }
  return lanes;
}

int capture(sr_fmg_batch_s* b, const double* const* f, double* const* u, int streams) {
  cudaStream_t main = b->origin;
  drop_graph(b);
  int rc = ensure_streams(b, streams);
  if (rc) return rc;
  const auto lanes = assign(b, streams);
  if (cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return SR_ERR_CUDA;
  cudaError_t err = cudaEventRecord(b->events[0], main);
  for (int s = 0; s < streams && err == cudaSuccess; ++s)
    err = cudaStreamWaitEvent(b->side[s], b->events[0], 0);
  for (int s = 0; s < streams && err == cudaSuccess && !rc; ++s)
    for (int i : lanes[s]) {
      rc = srfmg::enqueue_solve_unchecked(b->hs[i], f[i], u[i], b->side[s]);
      if (rc) break;
    }
  for (int s = 0; s < streams && err == cudaSuccess; ++s) {
    err = cudaEventRecord(b->events[s + 1], b->side[s]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(main, b->events[s + 1], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t end = cudaStreamEndCapture(main, &graph);
  if (rc || err != cudaSuccess || end != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc ? rc : SR_ERR_CUDA;
  }
  err = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (err != cudaSuccess) {
    b->exec = nullptr;
    return SR_ERR_CUDA;
  }
  b->f_cached.assign(f, f + b->hs.size());
  b->u_cached.assign(u, u + b->hs.size());
  b->gen_cached.clear();
  for (sr_fmg_t h : b->hs) b->gen_cached.push_back(srfmg::handle_generation(h));
  b->captured_streams = streams;
  return SR_OK;
}

int validate(const sr_fmg_batch_s* b, const double* const* f, double* const* u) {
  if (!f || !u) return SR_ERR_INVALID;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    if (!device_ptr(f[i]) || !device_ptr(u[i])) return SR_ERR_INVALID;
    const size_t bytes = (size_t)srfmg::handle_cells(b->hs[i]) * sizeof(double);
    const char* fa = (const char*)f[i];
    const char* ua = (const char*)u[i];
    if (fa < ua + bytes && ua < fa + bytes) return SR_ERR_INVALID;
    for (size_t j = 0; j < i; ++j)
      if (u[j] == u[i] || b->hs[j] == b->hs[i]) return SR_ERR_INVALID;
  }
  return SR_OK;
}

int launch_graph(sr_fmg_batch_s* b, const double* const* f, double* const* u, cudaStream_t s) {
  bool same = b->exec && b->captured_streams == b->streams;
  for (size_t i = 0; same && i < b->hs.size(); ++i)
    same = b->f_cached[i] == f[i] && b->u_cached[i] == u[i] &&
           b->gen_cached[i] == srfmg::handle_generation(b->hs[i]);
  if (!same) {
    int rc = capture(b, f, u, b->streams);
    if (rc) return rc;
  }
  if (cudaEventRecord(b->before, s) != cudaSuccess) return SR_ERR_CUDA;
  if (cudaStreamWaitEvent(b->origin, b->before, 0) != cudaSuccess) return SR_ERR_CUDA;
  if (cudaGraphLaunch(b->exec, b->origin) != cudaSuccess) return SR_ERR_CUDA;
  if (cudaEventRecord(b->after, b->origin) != cudaSuccess) return SR_ERR_CUDA;
  return cudaStreamWaitEvent(s, b->after, 0) == cudaSuccess ? SR_OK : SR_ERR_CUDA;
}

}  // namespace

extern "C" {

int sr_fmg_batch_create(sr_fmg_batch_t* out, const sr_fmg_t* hs, int count) {
  if (!out) return SR_ERR_INVALID;
  *out = nullptr;
  if (!hs || count < 1 || count > 4096) return SR_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (!hs[i]) return SR_ERR_INVALID;
  sr_fmg_batch_s* b = new (std::nothrow) sr_fmg_batch_s();
  if (!b) return SR_ERR_OOM;
  b->hs.assign(hs, hs + count);
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return SR_ERR_CUDA;
  }
  b->streams = count < 4 ? count : 4;
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->before, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->after, cudaEventDisableTiming) != cudaSuccess) {
    sr_fmg_batch_destroy(b);
    return SR_ERR_CUDA;
  }
  *out = b;
  return SR_OK;
}

int sr_fmg_batch_destroy(sr_fmg_batch_t b) {
  if (!b) return SR_OK;
  drop_graph(b);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->before) cudaEventDestroy(b->before);
  if (b->after) cudaEventDestroy(b->after);
  delete b;
  return SR_OK;
}

int sr_fmg_batch_solve_async(sr_fmg_batch_t b, const double* const* f, double* const* u,
                             void* stream) {
  if (!b) return SR_ERR_INVALID;
  int rc = validate(b, f, u);
  if (rc) return rc;
  return launch_graph(b, f, u, (cudaStream_t)stream);
}

int sr_fmg_batch_check(sr_fmg_batch_t b, void* stream) {
  if (!b) return SR_ERR_INVALID;
  int worst = SR_OK;
  for (sr_fmg_t h : b->hs) {
    const int rc = sr_fmg_check(h, stream);
    if (rc != SR_OK && worst == SR_OK) worst = rc;
  }
  return worst;
}

int sr_fmg_batch_solve(sr_fmg_batch_t b, const double* const* f, double* const* u,
                       void* stream) {
  int rc = sr_fmg_batch_solve_async(b, f, u, stream);
  if (rc) return rc;
  return sr_fmg_batch_check(b, stream);
}

int sr_fmg_solve_batched(sr_fmg_t* hs, const double* const* f, double* const* u, int count,
                         void* stream) {
  sr_fmg_batch_t b = nullptr;
  int rc = sr_fmg_batch_create(&b, hs, count);
  if (rc) return rc;
  rc = sr_fmg_batch_solve(b, f, u, stream);
  sr_fmg_batch_destroy(b);
  return rc;
}

int sr_fmg_batch_autotune(sr_fmg_batch_t b, const double* const* f, double* const* u,
                          void* stream, int* streams_out, float* ms_out) {
  if (!b) return SR_ERR_INVALID;
  int rc = validate(b, f, u);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SR_ERR_CUDA;
  }
  int best = -1;
  float best_ms = 0.f;
  const int count = (int)b->hs.size();
  for (int streams = 1; streams <= 32 && streams <= count; streams *= 2) {
    b->streams = streams;
    rc = launch_graph(b, f, u, s);  // captures, warms up
    if (!rc) rc = sr_fmg_batch_check(b, stream);
    if (rc) break;
    float total = 0.f;
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      cudaEventRecord(e0, s);
      rc = launch_graph(b, f, u, s);
      cudaEventRecord(e1, s);
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = SR_ERR_CUDA;
      float ms = 0.f;
      if (!rc) cudaEventElapsedTime(&ms, e0, e1);
      total += ms;
    }
    if (rc) break;
    const float ms = total / 2.f;
    if (best < 0 || ms < best_ms) {
      best = streams;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->streams = best;
  drop_graph(b);
  if (streams_out) *streams_out = best;
  if (ms_out) *ms_out = best_ms;
  return SR_OK;
}

int sr_fmg_batch_set_streams(sr_fmg_batch_t b, int streams) {
  if (!b || streams < 1 || streams > 64) return SR_ERR_INVALID;
  b->streams = streams;
  return SR_OK;
}

}  // extern "C"
