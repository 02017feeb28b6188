// C ABI of libdg (see include/dg.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace {
thread_local std::string g_err;

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage Runge-Kutta.
const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double RK_B[5] = {1432997174477.0 / 9575080441904.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

dg_status cuda_fail(cudaError_t e) {
  g_err = cudaGetErrorString(e);
  return DG_ECUDA;
}
}  // namespace

void dg_set_last_error(const std::string& msg) { g_err = msg; }

extern "C" {

const char* dg_status_string(dg_status s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_EINVAL: return "invalid argument";
    case DG_ENOMEM: return "out of device memory";
    case DG_ECUDA: return "CUDA error";
    case DG_EMESH: return "invalid mesh";
    case DG_ETIMEOUT: return "device wait timed out";
    case DG_ENOTSUP: return "not supported";
    case DG_ENONFINITE: return "non-finite value";
  }
  return "unknown status";
}

const char* dg_last_error(void) { return g_err.c_str(); }

dg_status dg_mesh_create(const dg_mesh_desc* d, void* stream, dg_mesh** out) {
  if (!d || !out) return DG_EINVAL;
  *out = nullptr;
  if (d->N < 1 || d->N > dgk::MAXN) {
    g_err = "N must be in 1..6";
    return DG_ENOTSUP;
  }
  if (d->hex_basis != 0 || d->nlevels > 1 || d->precision != 0) {
    g_err = "only GL hexahedra, single-rate stepping and FP32 are built";
    return DG_ENOTSUP;
  }
  if (d->nverts <= 0 || !d->xyz) return DG_EINVAL;
  for (int t = 0; t < 4; ++t) {
    if (d->nelem[t] < 0 || d->nelem[t] > (int64_t)1 << 30) return DG_EINVAL;
    if (d->nelem[t] > 0 && (!d->conn[t] || !d->c2[t])) return DG_EINVAL;
  }
  if (!(d->tau_scale >= 0.0)) return DG_EINVAL;
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return DG_ENOMEM;
  cudaGetDevice(&m->device);
  m->stream = static_cast<cudaStream_t>(stream);
  std::string err;
  dg_status st = dg_setup(m, d, err);
  if (st != DG_OK) {
    g_err = err;
    dg_free(m);
    delete m;
    return st;
  }
  *out = m;
  return DG_OK;
}

dg_status dg_host_check(const dg_mesh_desc* d, double* dt_min, double* trace_const) {
  if (!d || d->nverts <= 0 || !d->xyz) return DG_EINVAL;
  if (d->N < 1 || d->N > dgk::MAXN) return DG_ENOTSUP;
  for (int t = 0; t < 4; ++t)
    if (d->nelem[t] < 0 || (d->nelem[t] > 0 && (!d->conn[t] || !d->c2[t]))) return DG_EINVAL;
  dg_mesh m;
  std::string err;
  double ct[4];
  dg_status st = dg_setup_host_only(&m, d, err, ct);
  if (st != DG_OK) {
    g_err = err;
    return st;
  }
  if (dt_min) *dt_min = m.dt_min;
  if (trace_const)
    for (int t = 0; t < 4; ++t) trace_const[t] = ct[t];
  return DG_OK;
}

void dg_mesh_destroy(dg_mesh* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  for (cudaEvent_t ev : m->ev_pool) cudaEventDestroy(ev);
  dg_free(m);
  delete m;
}

dg_status dg_layout(const dg_mesh* m, int type, int64_t* offset, int64_t* nelem, int* Np) {
  if (!m || type < 0 || type > 3) return DG_EINVAL;
  if (offset) *offset = m->td[type].dof_off;
  if (nelem) *nelem = m->td[type].K;
  if (Np) *Np = m->td[type].Np;
  return DG_OK;
}

dg_status dg_ndof(const dg_mesh* m, int64_t* ndof) {
  if (!m || !ndof) return DG_EINVAL;
  *ndof = m->ndof;
  return DG_OK;
}

dg_status dg_state_ptr(dg_mesh* m, float** q) {
  if (!m || !q) return DG_EINVAL;
  *q = m->q;
  return DG_OK;
}

dg_status dg_set_state(dg_mesh* m, const float* q, int on_device) {
  if (!m || !q) return DG_EINVAL;
  size_t bytes = 4 * (size_t)m->ndof * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(m->q, q, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemsetAsync(m->res, 0, bytes, m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return DG_OK;
}

dg_status dg_get_state(const dg_mesh* m, float* q, int on_device) {
  if (!m || !q) return DG_EINVAL;
  size_t bytes = 4 * (size_t)m->ndof * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(q, m->q, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!on_device) {
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return DG_OK;
}

dg_status dg_rhs(dg_mesh* m, const float* q, float* rhs, double t) {
  (void)t;
  if (!m || !q || !rhs) return DG_EINVAL;
  float* tr = m->trace;  // buffer 0 used as scratch
  cudaError_t e = dgk::launch_trace(m, q, tr);
  if (e != cudaSuccess) return cuda_fail(e);
  e = dgk::launch_rhs(m, q, tr, rhs);
  if (e != cudaSuccess) return cuda_fail(e);
  return DG_OK;
}

dg_status dg_timestep(const dg_mesh* m, double* dt_min, int64_t* level_count) {
  if (!m || !dt_min) return DG_EINVAL;
  *dt_min = m->dt_min;
  if (level_count) level_count[0] = m->td[0].K + m->td[1].K + m->td[2].K + m->td[3].K;
  return DG_OK;
}

dg_status dg_step(dg_mesh* m, int nsteps, double dt, double* t_inout) {
  if (!m || nsteps < 0) return DG_EINVAL;
  if (!(dt > 0)) dt = m->dt_min;
  if (nsteps == 0) return DG_OK;
  const size_t plane2 = 2 * (size_t)m->nsides * m->nq;
  float* buf[2] = {m->trace, m->trace + plane2};
  cudaError_t e = dgk::launch_trace(m, m->q, buf[0]);
  if (e != cudaSuccess) return cuda_fail(e);
  int cur = 0;
  for (int s = 0; s < nsteps; ++s)
    for (int k = 0; k < 5; ++k) {
      e = dgk::launch_stage(m, m->q, m->res, buf[cur], buf[cur ^ 1], (float)RK_A[k], (float)RK_B[k], (float)dt);
      if (e != cudaSuccess) return cuda_fail(e);
      cur ^= 1;
    }
  if (t_inout) *t_inout += nsteps * dt;
  return DG_OK;
}

dg_status dg_energy(dg_mesh* m, const float* q, double* E) {
  if (!m || !E) return DG_EINVAL;
  if (!q) q = m->q;
  cudaError_t e = cudaMemsetAsync(m->dacc, 0, sizeof(double), m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = dgk::launch_energy(m, q, m->dacc);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemcpyAsync(E, m->dacc, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!std::isfinite(*E)) return DG_ENONFINITE;
  return DG_OK;
}

dg_status dg_profile(dg_mesh* m, int enable, double* ms, int64_t* launches) {
  if (!m) return DG_EINVAL;
  if (ms || launches) {
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int t = 0; t < 4; ++t) {
      double sum = 0.0;
      for (auto& pr : m->ev_used[t]) {
        float x = 0.f;
        if (cudaEventElapsedTime(&x, m->ev_pool[pr.first], m->ev_pool[pr.second]) == cudaSuccess) sum += x;
      }
      if (ms) ms[t] = sum;
      if (launches) launches[t] = m->launches[t];
    }
  }
  for (int t = 0; t < 4; ++t) {
    m->ev_used[t].clear();
    m->launches[t] = 0;
  }
  m->ev_next = 0;
  m->profiling = enable != 0;
  return DG_OK;
}

dg_status dg_adjoint_step(dg_mesh* m, int nsteps, float* lambda, double* g_c2, double* g_amp) {
  (void)m; (void)nsteps; (void)lambda; (void)g_c2; (void)g_amp;
  g_err = "adjoint not built";
  return DG_ENOTSUP;
}

}  // extern "C"
