// Batched stepping of several meshes (dg_batch_*, include/dg.h): one CUDA graph holds
// DG_BATCH_CHUNK steps of every mesh, each mesh an independent branch, and is replayed.
//
// Packing: single-rate meshes of the same order and options are merged at creation into one
// combined mesh (the union of their disjoint element sets, vertex ids offset per mesh), whose
// kernels cover every member with one launch per element type and stage; each element carries
// its own mesh's time step (dg_mesh::dte), so the per-element arithmetic is that of the member
// mesh and results are bitwise those of stepping it alone.  A batch step copies the members'
// states into the combined mesh (one gather kernel over contiguous segments), steps it, and
// copies them back.  Meshes without a partner (other N or options, two time-step levels) keep
// their own graph branch.  Sec. 4.3 (Figure perDofTimes) shows the time per degree of freedom
// rising for small meshes, whose launches cannot fill the GPU: packing removes that.
//
// A mesh's step sequence is stateless across calls except for the multi-rate history slots,
// which rotate with period 3 per coarse step (and the start-up, run once, outside any graph).
// A graph of 3 steps therefore leaves every mesh's host-side state as it found it, so one
// capture serves every later chunk while the slot phases and step sizes stay the same.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
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
  // packing
  struct Group {
    dg_mesh* mm = nullptr;          // combined mesh (owned)
    std::vector<int> idx;           // member indices into m, in element order of mm
    dgk::Seg* segs = nullptr;       // device: [nseg] gather (members -> mm), then [nseg] scatter
    int nseg = 0;
    std::vector<double> dt;         // member steps held in mm->dte
    cudaStream_t br = nullptr;
    cudaEvent_t ev = nullptr;
  };
  std::vector<Group> groups;
  std::vector<int> group_of;        // per mesh: its group, or -1
  bool packed = false;              // step through the groups (true) or mesh by mesh
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

int phase_of(const dg_mesh* m) { return m->nlevels == 2 && m->integrator == 0 ? m->cslot[0] : 0; }

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
    if (b->packed && b->group_of[i] >= 0) continue;
    e = cudaStreamWaitEvent(b->br[i], b->fork, 0);
    if (e == cudaSuccess)
      e = on_stream(b->m[i], b->br[i], [&] { return dg_enqueue_steps(b->m[i], DG_BATCH_CHUNK, h[i]); });
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[i], b->br[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[i], 0);
  }
  for (size_t k = 0; k < b->groups.size() && b->packed && e == cudaSuccess; ++k) {
    dg_batch::Group& g = b->groups[k];
    e = cudaStreamWaitEvent(g.br, b->fork, 0);
    if (e == cudaSuccess)
      e = on_stream(g.mm, g.br, [&] { return dg_enqueue_steps(g.mm, DG_BATCH_CHUNK, h[g.idx[0]]); });
    if (e == cudaSuccess) e = cudaEventRecord(g.ev, g.br);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, g.ev, 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

// Meshes that may share a combined mesh: single rate, no point source, same order, bases, flux,
// precision, face exchange and run-time kernel choices (so the kernels, and therefore the
// per-element arithmetic, are the same).
using PackKey = std::tuple<int, int, int, double, int, bool, bool, bool>;
bool packable(const dg_mesh* m) { return m->nlevels == 1 && m->src_e < 0; }
PackKey pack_key(const dg_mesh* m) {
  return PackKey(m->N, m->hex_sem ? 1 : 0, m->pyr_form, m->tau_scale, m->precision, m->tri_lat, m->use_hex_tma,
                 m->use_tet_tc);
}

// The combined mesh of members idx (vertex ids offset per member), its per-element step arrays and
// the gather / scatter segments of the state.
dg_status build_group(dg_batch* b, dg_batch::Group& g) {
  const dg_mesh* m0 = b->m[g.idx[0]];
  dg_mesh_desc d = m0->host.d;
  std::vector<double> xyz;
  std::vector<int32_t> conn[4];
  std::vector<double> c2[4];
  const int nvt[4] = {8, 6, 5, 4};
  int64_t voff = 0;
  for (int i : g.idx) {
    const dg_mesh* mi = b->m[i];
    xyz.insert(xyz.end(), mi->host.xyz.begin(), mi->host.xyz.end());
    for (int t = 0; t < 4; ++t) {
      for (int32_t v : mi->host.conn[t]) conn[t].push_back((int32_t)(v + voff));
      c2[t].insert(c2[t].end(), mi->host.c2[t].begin(), mi->host.c2[t].end());
    }
    voff += (int64_t)mi->host.xyz.size() / 3;
  }
  if (voff >= (1LL << 31)) {
    dg_set_last_error("combined batch mesh exceeds 2^31 vertices");
    return DG_EINVAL;
  }
  d.nverts = voff;
  d.xyz = xyz.data();
  for (int t = 0; t < 4; ++t) {
    d.nelem[t] = (int64_t)c2[t].size();
    d.conn[t] = conn[t].data();
    d.c2[t] = c2[t].data();
  }
  d.nlevels = 1;
  dg_status st = dg_mesh_create(&d, b->stream, &g.mm);
  if (st != DG_OK) return st;
  dg_mesh* mm = g.mm;
  mm->use_hex_tma = m0->use_hex_tma;
  mm->use_tet_tc = m0->use_tet_tc;
  for (int t = 0; t < 4; ++t)
    if (mm->td[t].K > 0 && !(mm->dte[t] = static_cast<float*>(dg_alloc_owned(mm, (size_t)mm->td[t].K * sizeof(float))))) {
      dg_set_last_error("combined batch mesh: per-element step arrays do not fit");
      return DG_ENOMEM;
    }
  std::vector<dgk::Seg> gat, sca;
  int64_t eoff[4] = {0, 0, 0, 0};
  for (int i : g.idx) {
    const dg_mesh* mi = b->m[i];
    for (int t = 0; t < 4; ++t) {
      const int64_t n = (int64_t)mi->td[t].K * mi->td[t].Np;
      for (int f = 0; f < 4 && n > 0; ++f) {
        float* src = mi->q + f * mi->ndof + mi->td[t].dof_off;
        float* dst = mm->q + f * mm->ndof + mm->td[t].dof_off + eoff[t] * mm->td[t].Np;
        gat.push_back({src, dst, n});
        sca.push_back({dst, src, n});
      }
      eoff[t] += mi->td[t].K;
    }
  }
  (void)nvt;
  g.nseg = (int)gat.size();
  gat.insert(gat.end(), sca.begin(), sca.end());
  g.segs = static_cast<dgk::Seg*>(dg_alloc_owned(mm, gat.size() * sizeof(dgk::Seg)));
  if (!g.segs) return DG_ENOMEM;
  cudaError_t e = cudaMemcpy(g.segs, gat.data(), gat.size() * sizeof(dgk::Seg), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.br, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming);
  return e == cudaSuccess ? DG_OK : fail(e);
}

// Per-element steps of group g for the member steps h (uploaded when they change).
cudaError_t group_dt(dg_batch* b, dg_batch::Group& g, const std::vector<double>& h) {
  std::vector<double> want;
  for (int i : g.idx) want.push_back(h[i]);
  if (want == g.dt) return cudaSuccess;
  for (int t = 0; t < 4; ++t) {
    if (!g.mm->dte[t]) continue;
    std::vector<float> v;
    v.reserve(g.mm->td[t].K);
    for (int i : g.idx) v.insert(v.end(), (size_t)b->m[i]->td[t].K, (float)h[i]);
    // pageable source: the copy has taken v's contents when the call returns
    cudaError_t e = cudaMemcpyAsync(g.mm->dte[t], v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return e;
  }
  g.dt = want;
  return cudaSuccess;
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
  // packing: groups of at least two packable meshes with equal keys
  b->group_of.assign(count, -1);
  const char* pk = std::getenv("DG_BATCH_PACK");
  if (!(pk && pk[0] == '0')) {
    std::map<PackKey, std::vector<int>> by;
    for (int i = 0; i < count; ++i)
      if (packable(meshes[i])) by[pack_key(meshes[i])].push_back(i);
    for (auto& kv : by) {
      if (kv.second.size() < 2) continue;
      b->groups.emplace_back();
      b->groups.back().idx = kv.second;
      const dg_status st = build_group(b, b->groups.back());
      if (st != DG_OK) {
        dg_batch_destroy(b);
        return st;
      }
      for (int i : kv.second) b->group_of[i] = (int)b->groups.size() - 1;
    }
    b->packed = !b->groups.empty();
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
    fresh[i] = b->m[i]->nlevels == 2 && b->m[i]->integrator == 0 && !b->m[i]->mr_started;
  }
  cudaError_t e = cudaSuccess;
  // the batch stream follows the work already queued on each mesh's stream
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaEventRecord(b->ev[i], b->m[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[i], 0);
  }
  // packed groups: per-element steps, members' states into the combined meshes
  for (size_t k = 0; k < b->groups.size() && b->packed && e == cudaSuccess; ++k) {
    dg_batch::Group& g = b->groups[k];
    e = group_dt(b, g, h);
    if (e == cudaSuccess) e = dgk::launch_seg_copy(g.segs, g.nseg, b->stream);
  }
  // start-ups and the remainder steps, mesh after mesh (group after group) on the batch stream
  const int reps = nsteps / DG_BATCH_CHUNK, rest = nsteps % DG_BATCH_CHUNK;
  for (size_t i = 0; i < n && e == cudaSuccess; ++i)
    if ((fresh[i] || rest) && !(b->packed && b->group_of[i] >= 0))
      e = on_stream(b->m[i], b->stream, [&] { return dg_enqueue_steps(b->m[i], rest, h[i]); });
  for (size_t k = 0; k < b->groups.size() && b->packed && rest && e == cudaSuccess; ++k) {
    dg_batch::Group& g = b->groups[k];
    e = on_stream(g.mm, b->stream, [&] { return dg_enqueue_steps(g.mm, rest, h[g.idx[0]]); });
  }
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
  // combined meshes' states back into the members
  for (size_t k = 0; k < b->groups.size() && b->packed && e == cudaSuccess; ++k)
    e = dgk::launch_seg_copy(b->groups[k].segs + b->groups[k].nseg, b->groups[k].nseg, b->stream);
  if (e != cudaSuccess) return fail(e);
  // each mesh's stream follows the batch
  e = cudaEventRecord(b->done, b->stream);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->m[i]->stream, b->done, 0);
  if (e != cudaSuccess) return fail(e);
  if (t_inout)
    for (size_t i = 0; i < n; ++i) t_inout[i] += dg_step_time(b->m[i], nsteps, h[i], fresh[i]);
  return DG_OK;
}

dg_status dg_batch_set_packing(dg_batch* b, int packed) {
  if (!b) return DG_EINVAL;
  const bool p = packed != 0 && !b->groups.empty();
  if (p != b->packed) {   // the cached graphs hold the other schedule
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(e);
    destroy_graphs(b);
    b->packed = p;
  }
  return DG_OK;
}

dg_status dg_batch_autotune(dg_batch* b, int nsteps, int* packed) {
  if (!b || nsteps < 1 || nsteps > 30) return DG_EINVAL;
  nsteps = (nsteps + DG_BATCH_CHUNK - 1) / DG_BATCH_CHUNK * DG_BATCH_CHUNK;
  if (b->groups.empty()) {
    if (packed) *packed = 0;
    return DG_OK;
  }
  // scratch copies of every mesh's state, and of the multi-rate meshes' rhs history with its slot
  // phases and start-up flag (all restored after the trials)
  const size_t n = b->m.size();
  std::vector<float*> keep(n, nullptr);
  struct MrKeep {
    int c[3], f[3];
    bool started;
  };
  std::vector<MrKeep> mk(n);
  auto kbytes = [&](size_t i) { return (b->m[i]->nlevels == 2 ? 16 : 4) * (size_t)b->m[i]->ndof * sizeof(float); };
  cudaError_t e = cudaStreamSynchronize(b->stream);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    dg_mesh* mi = b->m[i];
    e = cudaMallocAsync(reinterpret_cast<void**>(&keep[i]), kbytes(i), b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(keep[i], mi->q, 4 * (size_t)mi->ndof * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess && mi->nlevels == 2)
      e = cudaMemcpyAsync(keep[i] + 4 * mi->ndof, mi->hist, 12 * (size_t)mi->ndof * sizeof(float),
                          cudaMemcpyDeviceToDevice, b->stream);
    for (int k = 0; k < 3; ++k) {
      mk[i].c[k] = mi->cslot[k];
      mk[i].f[k] = mi->fslot[k];
    }
    mk[i].started = mi->mr_started;
  }
  float best[2] = {0.f, 0.f};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const bool was = b->packed;
  for (int trial = 0; trial < 2 && e == cudaSuccess; ++trial) {
    const int p = trial == 0 ? 1 : 0;
    dg_status st = dg_batch_set_packing(b, p);
    if (st != DG_OK) break;
    float t = 1e30f;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {   // a capture, then two timed replays
      e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess && dg_batch_step(b, nsteps, nullptr, nullptr) != DG_OK) e = cudaErrorUnknown;
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && ms < t) t = ms;
    }
    best[p] = t;
  }
  for (size_t i = 0; i < n; ++i)
    if (keep[i]) {
      dg_mesh* mi = b->m[i];
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(mi->q, keep[i], 4 * (size_t)mi->ndof * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
      if (e == cudaSuccess && mi->nlevels == 2)
        e = cudaMemcpyAsync(mi->hist, keep[i] + 4 * mi->ndof, 12 * (size_t)mi->ndof * sizeof(float),
                            cudaMemcpyDeviceToDevice, b->stream);
      for (int k = 0; k < 3; ++k) {
        mi->cslot[k] = mk[i].c[k];
        mi->fslot[k] = mk[i].f[k];
      }
      mi->mr_started = mk[i].started;
      cudaFreeAsync(keep[i], b->stream);
    }
  // the members' own streams follow the restores
  if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->m[i]->stream, b->done, 0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    dg_batch_set_packing(b, was);
    return fail(e);
  }
  const int pick = best[1] <= best[0] ? 1 : 0;
  dg_status st = dg_batch_set_packing(b, pick);
  if (packed) *packed = pick;
  if (st == DG_OK) st = cudaStreamSynchronize(b->stream) == cudaSuccess ? DG_OK : DG_ECUDA;
  return st;
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
  for (auto& g : b->groups) {
    if (g.br) cudaStreamDestroy(g.br);
    if (g.ev) cudaEventDestroy(g.ev);
    dg_mesh_destroy(g.mm);
  }
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
