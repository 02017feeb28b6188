// Batched stepping of several meshes (dg_batch_*, include/dg.h): one CUDA graph holds
// DG_BATCH_CHUNK steps of every mesh, each mesh an independent branch, and is replayed.
//
// A mesh's step sequence is stateless across calls except for the multi-rate history slots,
// which rotate with period 3 per coarse step (and the start-up, run once, outside any graph).
// A graph of 3 steps therefore leaves every mesh's host-side state as it found it, so one
// capture serves every later chunk while the slot phases and step sizes stay the same.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

static_assert(DG_BATCH_CHUNK == 3, "the multi-rate history slots rotate with period 3");

struct dg_batch {
  std::vector<dg_mesh*> m;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<cudaStream_t> br;   // capture branch of each mesh
  std::vector<cudaEvent_t> ev;    // per mesh: ordering / join
  cudaEvent_t fork = nullptr, done = nullptr;
  struct Graph {
    std::vector<int> phase;
    std::vector<double> dt;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Graph> cache;
  int64_t replays = 0, captures = 0;
};

namespace {

constexpr size_t MAX_GRAPHS = 4;

// Runs f with the mesh's work going to stream s, per-launch timing off and the element types on
// that one stream (the meshes' branches already run side by side; per-type forks would only add
// graph nodes), then restores all three.
template <class F>
cudaError_t on_stream(dg_mesh* m, cudaStream_t s, F f) {
  cudaStream_t keep = m->stream;
  const bool prof = m->profiling, ts = m->type_streams;
  m->stream = s;
  m->profiling = false;
  m->type_streams = false;
  cudaError_t e = f();
  m->stream = keep;
  m->profiling = prof;
  m->type_streams = ts;
  return e;
}

int phase_of(const dg_mesh* m) { return m->nlevels == 2 ? m->cslot[0] : 0; }

void destroy_graphs(dg_batch* b) {
  for (auto& g : b->cache)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  b->cache.clear();
}

dg_status fail(cudaError_t e) {
  dg_set_last_error(cudaGetErrorString(e));
  return DG_ECUDA;
}

// Capture DG_BATCH_CHUNK steps of every mesh into an executable graph.
cudaError_t capture(dg_batch* b, const std::vector<double>& h, cudaGraphExec_t* out) {
  *out = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(b->fork, b->stream);
  for (size_t i = 0; i < b->m.size() && e == cudaSuccess; ++i) {
    e = cudaStreamWaitEvent(b->br[i], b->fork, 0);
    if (e == cudaSuccess)
      e = on_stream(b->m[i], b->br[i], [&] { return dg_enqueue_steps(b->m[i], DG_BATCH_CHUNK, h[i]); });
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[i], b->br[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[i], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

}  // namespace

extern "C" {

dg_status dg_batch_create(dg_mesh* const* meshes, int count, void* cuda_stream, dg_batch** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  if (!meshes || count < 1) return DG_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!meshes[i]) return DG_EINVAL;
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) {
        dg_set_last_error("a mesh appears twice in the batch");
        return DG_EINVAL;
      }
  }
  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return DG_ENOMEM;
  b->m.assign(meshes, meshes + count);
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  b->br.assign(count, nullptr);
  b->ev.assign(count, nullptr);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    dg_batch_destroy(b);
    return fail(e);
  }
  *out = b;
  return DG_OK;
}

dg_status dg_batch_step(dg_batch* b, int nsteps, const double* dt, double* t_inout) {
  if (!b || nsteps < 0) return DG_EINVAL;
  if (nsteps == 0) return DG_OK;
  const size_t n = b->m.size();
  std::vector<double> h(n);
  std::vector<char> fresh(n);
  for (size_t i = 0; i < n; ++i)
    if (b->m[i]->src_e >= 0) {
      dg_set_last_error("a mesh with a point source cannot be stepped in a batch (the graph fixes the source values)");
      return DG_ENOTSUP;
    }
  for (size_t i = 0; i < n; ++i) {
    h[i] = dt && dt[i] > 0 ? dt[i] : b->m[i]->dt_min;
    fresh[i] = b->m[i]->nlevels == 2 && !b->m[i]->mr_started;
  }
  cudaError_t e = cudaSuccess;
  // the batch stream follows the work already queued on each mesh's stream
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaEventRecord(b->ev[i], b->m[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[i], 0);
  }
  // start-ups and the remainder steps, mesh after mesh on the batch stream
  const int reps = nsteps / DG_BATCH_CHUNK, rest = nsteps % DG_BATCH_CHUNK;
  for (size_t i = 0; i < n && e == cudaSuccess; ++i)
    if (fresh[i] || rest)
      e = on_stream(b->m[i], b->stream, [&] { return dg_enqueue_steps(b->m[i], rest, h[i]); });
  if (e != cudaSuccess) return fail(e);
  if (reps > 0) {
    std::vector<int> phase(n);
    for (size_t i = 0; i < n; ++i) phase[i] = phase_of(b->m[i]);
    cudaGraphExec_t exec = nullptr;
    for (auto& g : b->cache)
      if (g.phase == phase && g.dt == h) exec = g.exec;
    if (!exec) {
      e = capture(b, h, &exec);
      if (e != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        return fail(e);
      }
      if (b->cache.size() == MAX_GRAPHS) {
        cudaGraphExecDestroy(b->cache.front().exec);
        b->cache.erase(b->cache.begin());
      }
      b->cache.push_back({phase, h, exec});
      b->captures += 1;
    }
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, b->stream);
    if (e != cudaSuccess) return fail(e);
    b->replays += reps;
  }
  // each mesh's stream follows the batch
  e = cudaEventRecord(b->done, b->stream);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->m[i]->stream, b->done, 0);
  if (e != cudaSuccess) return fail(e);
  if (t_inout)
    for (size_t i = 0; i < n; ++i) t_inout[i] += dg_step_time(b->m[i], nsteps, h[i], fresh[i]);
  return DG_OK;
}

dg_status dg_batch_stats(const dg_batch* b, int64_t* replays, int64_t* captures) {
  if (!b) return DG_EINVAL;
  if (replays) *replays = b->replays;
  if (captures) *captures = b->captures;
  return DG_OK;
}

void dg_batch_destroy(dg_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  destroy_graphs(b);
  for (cudaStream_t s : b->br)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t ev : b->ev)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
