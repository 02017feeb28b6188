// Autotuner (dg_autotune, include/dg.h): picks, per mesh, among the kernel choices the library
// has at run time by timing them on the GPU:
//   0  TMA staging of the fused N = 4 hex kernels, or cp.async staging;
//   1  tensor-core tets (N <= 4, lattice exchange), or the warp-per-element SIMT tet kernel;
//   2  the four element types of a stage on their own streams, or on the mesh's one stream.
// Which is faster depends on the mesh: small meshes leave SMs idle (the tensor-core kernel works
// on tiles of 32 tets), large ones are bound by the per-type kernels.  Each choice is tried in
// turn, the others held at their current values (coordinate descent, one pass), on nsteps
// LSRK(5,4) steps of a scratch copy of the state (best of three runs), and taken only when it is
// at least 2 % faster than the current choice; the mesh's state is not modified.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace {

// GPU time of nsteps single-rate LSRK steps of dt on state qs (trace buffers and the residual
// of the mesh are used as scratch), measured with events on the mesh's stream.
cudaError_t time_steps(dg_mesh* m, float* qs, int nsteps, double dt, float* ms) {
  const size_t plane2 = 2 * (size_t)m->nsides * m->nq;
  float* buf[2] = {m->trace, m->trace + plane2};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, m->stream);
  if (e == cudaSuccess) e = dgk::launch_trace(m, qs, buf[0]);
  int cur = 0;
  for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
      e = dgk::launch_stage(m, qs, m->res, buf[cur], buf[cur ^ 1], (float)RK_A[k], (float)RK_B[k], (float)dt);
      cur ^= 1;
    }
  if (e == cudaSuccess) e = cudaEventRecord(e1, m->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" dg_status dg_autotune(dg_mesh* m, int nsteps, int* choice) {
  if (!m || nsteps < 0 || nsteps > 100) return DG_EINVAL;
  bool* knob[3] = {&m->use_hex_tma, &m->use_tet_tc, &m->type_streams};
  if (nsteps == 0) {   // apply the given choices (type streams only where the mesh has them)
    if (!choice) return DG_EINVAL;
    m->use_hex_tma = choice[0] != 0;
    m->use_tet_tc = choice[1] != 0;
    m->type_streams = choice[2] != 0 && m->tev[4] != nullptr;
    choice[2] = m->type_streams ? 1 : 0;
    return DG_OK;
  }
  const bool active[3] = {m->N == 4 && m->K[DG_HEX] > 0,
                          m->N <= 4 && m->tri_lat && m->K[DG_TET] > 0,
                          m->tev[4] != nullptr};
  const size_t bytes = 4 * (size_t)m->ndof * sizeof(float);
  float* qs = nullptr;
  cudaError_t e = cudaMalloc(&qs, bytes);
  if (e != cudaSuccess) {
    dg_set_last_error("dg_autotune: scratch state allocation failed");
    return DG_ENOMEM;
  }
  const bool prof = m->profiling;
  m->profiling = false;
  const double dt = m->dt_min;
  // best of three timed runs after a warm-up run (the first launches of a variant)
  auto trial = [&](float* ms) {
    cudaError_t r = cudaMemcpyAsync(qs, m->q, bytes, cudaMemcpyDeviceToDevice, m->stream);
    if (r == cudaSuccess) r = time_steps(m, qs, 1, dt, ms);
    float best = 3.4e38f;
    for (int rep = 0; rep < 3 && r == cudaSuccess; ++rep) {
      r = cudaMemcpyAsync(qs, m->q, bytes, cudaMemcpyDeviceToDevice, m->stream);
      float t = 0.f;
      if (r == cudaSuccess) r = time_steps(m, qs, nsteps, dt, &t);
      if (t < best) best = t;
    }
    *ms = best;
    return r;
  };
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
    if (!active[c]) continue;
    const bool cur = *knob[c];
    float t_cur = 0.f, t_alt = 0.f;
    e = trial(&t_cur);
    if (e != cudaSuccess) break;
    *knob[c] = !cur;
    e = trial(&t_alt);
    if (e != cudaSuccess || !(t_alt < 0.98f * t_cur)) *knob[c] = cur;   // switch on a clear gain only
  }
  m->profiling = prof;
  cudaFree(qs);
  if (e != cudaSuccess) {
    dg_set_last_error(std::string("dg_autotune: ") + cudaGetErrorString(e));
    return DG_ECUDA;
  }
  if (choice)
    for (int c = 0; c < 3; ++c) choice[c] = *knob[c] ? 1 : 0;
  return DG_OK;
}
