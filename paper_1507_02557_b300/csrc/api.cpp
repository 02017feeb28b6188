// C ABI of libdg (see include/dg.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage Runge-Kutta.
const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double RK_B[5] = {1432997174477.0 / 9575080441904.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};
const double RK_C[5] = {0.0, 1432997174477.0 / 9575080441904.0, 2526269341429.0 / 6820363962896.0,
                        2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

namespace {
thread_local std::string g_err;

dg_status cuda_fail(cudaError_t e) {
  g_err = cudaGetErrorString(e);
  return DG_ECUDA;
}

// The device error word after a synchronization: bit 0 = a bounded device wait timed out
// (the word is cleared once reported).
dg_status device_flags(const dg_mesh* m) {
  int v = 0;
  if (!m->derr) return DG_OK;
  cudaError_t e = cudaMemcpyAsync(&v, m->derr, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if (v == 0) return DG_OK;
  cudaMemsetAsync(m->derr, 0, sizeof(int), m->stream);
  g_err = "a bounded device wait timed out";
  return DG_ETIMEOUT;
}
}  // namespace

void dg_set_last_error(const std::string& msg) { g_err = msg; }

dg_status dg_device_flags(const dg_mesh* m) { return device_flags(m); }

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
    g_err = "N must be in 1..9";
    return DG_ENOTSUP;
  }
  if ((d->hex_basis != 0 && d->hex_basis != 1) || d->nlevels > 2 || d->precision < 0 || d->precision > 2) {
    g_err = "hex_basis 0 / 1, one or two time-step levels and precision 0 / 1 / 2 are built";
    return DG_ENOTSUP;
  }
  if (d->nverts <= 0 || !d->xyz) return DG_EINVAL;
  for (int t = 0; t < 4; ++t) {
    if (d->nelem[t] < 0 || d->nelem[t] > (int64_t)1 << 30) return DG_EINVAL;
    if (d->nelem[t] > 0 && (!d->conn[t] || !d->c2[t])) return DG_EINVAL;
  }
  if (!(d->tau_scale >= 0.0)) return DG_EINVAL;
  if (d->integrator < 0 || d->integrator > 1) {
    g_err = "integrator 0 (multi-rate AB3) or 1 (multi-rate LSRK) are built";
    return DG_ENOTSUP;
  }
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return DG_ENOMEM;
  cudaGetDevice(&m->device);
  m->stream = static_cast<cudaStream_t>(stream);
  const char* ts = std::getenv("DG_TYPE_STREAMS");
  m->type_streams = !(ts && ts[0] == '0');
  std::string err;
  dg_status st = dg_setup(m, d, err);
  if (st != DG_OK) {
    g_err = err;
    dg_free(m);
    delete m;
    return st;
  }
  try {   // host copy of the description (a batch may merge the mesh with others of its kind)
    m->host.d = *d;
    m->host.xyz.assign(d->xyz, d->xyz + 3 * d->nverts);
    for (int t = 0; t < 4; ++t) {
      const int nv = t == DG_HEX ? 8 : t == DG_WEDGE ? 6 : t == DG_PYR ? 5 : 4;
      m->host.conn[t].assign(d->conn[t], d->conn[t] + nv * d->nelem[t]);
      m->host.c2[t].assign(d->c2[t], d->c2[t] + d->nelem[t]);
      m->host.d.conn[t] = nullptr;
      m->host.d.c2[t] = nullptr;
    }
    m->host.d.xyz = nullptr;
  } catch (const std::bad_alloc&) {
    dg_free(m);
    delete m;
    return DG_ENOMEM;
  }
  if (m->type_streams) {   // created here, not inside a later stream capture
    bool ok = true;
    for (int t = 0; t < 4 && ok; ++t) ok = cudaStreamCreateWithFlags(&m->tstream[t], cudaStreamNonBlocking) == cudaSuccess;
    for (int t = 0; t < 5 && ok; ++t) ok = cudaEventCreateWithFlags(&m->tev[t], cudaEventDisableTiming) == cudaSuccess;
    m->type_streams = ok;
  }
  *out = m;
  return DG_OK;
}

dg_status dg_host_check(const dg_mesh_desc* d, double* dt_min, double* trace_const, int64_t* level_count) {
  if (!d || d->nverts <= 0 || !d->xyz) return DG_EINVAL;
  if (d->N < 1 || d->N > dgk::MAXN || d->nlevels > 2) return DG_ENOTSUP;
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
  if (level_count)
    for (int L = 0; L < m.nlevels; ++L) level_count[L] = m.level_count[L];
  return DG_OK;
}

void dg_mesh_destroy(dg_mesh* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  for (cudaEvent_t ev : m->ev_pool) cudaEventDestroy(ev);
  for (int t = 0; t < 4; ++t)
    if (m->tstream[t]) cudaStreamSynchronize(m->tstream[t]), cudaStreamDestroy(m->tstream[t]);
  for (int t = 0; t < 5; ++t)
    if (m->tev[t]) cudaEventDestroy(m->tev[t]);
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

dg_status dg_level_counts(const dg_mesh* m, int level, int64_t* counts) {
  if (m && counts && level == 0 && m->integrator == 1) {   // multi-rate LSRK: the set S
    for (int t = 0; t < 4; ++t) counts[t] = m->mr_s.count[t];
    return DG_OK;
  }
  if (m && counts && level == -1 && m->nlevels == 2) {   // coarse elements next to fine ones
    for (int t = 0; t < 4; ++t) counts[t] = m->mr_pred_count[t];
    return DG_OK;
  }
  if (!m || !counts || level < 1 || level > m->nlevels) return DG_EINVAL;
  for (int t = 0; t < 4; ++t) counts[t] = m->nlevels == 1 ? m->td[t].K : m->lev[level - 1].count[t];
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
  m->mr_started = false;
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
    return device_flags(m);
  }
  return DG_OK;
}

dg_status dg_rhs(dg_mesh* m, const float* q, float* rhs, double t) {
  if (!m || !q || !rhs) return DG_EINVAL;
  float* tr = m->trace;  // buffer 0 used as scratch
  cudaError_t e = dgk::launch_trace(m, q, tr);
  if (e != cudaSuccess) return cuda_fail(e);
  dg_source_at(m, t);
  e = dgk::launch_rhs(m, q, tr, rhs);
  m->src_now = 0.f;
  if (e != cudaSuccess) return cuda_fail(e);
  return DG_OK;
}

dg_status dg_timestep(const dg_mesh* m, double* dt_min, int64_t* level_count) {
  if (!m || !dt_min) return DG_EINVAL;
  *dt_min = m->dt_min;
  if (level_count)
    for (int L = 0; L < m->nlevels; ++L) level_count[L] = m->level_count[L];
  return DG_OK;
}

}  // extern "C"

namespace {

// nsteps single-rate LSRK(5,4) steps: one trace launch, then fused stage kernels (ping-pong traces).
cudaError_t lsrk_steps(dg_mesh* m, int nsteps, double dt, double t0 = 0.0) {
  const size_t plane2 = 2 * (size_t)m->nsides * m->nq;
  float* buf[2] = {m->trace, m->trace + plane2};
  cudaError_t e = dgk::launch_trace(m, m->q, buf[0]);
  if (e != cudaSuccess) return e;
  int cur = 0;
  for (int s = 0; s < nsteps; ++s)
    for (int k = 0; k < 5; ++k) {
      dg_source_at(m, t0 + (s + RK_C[k]) * dt);
      e = dgk::launch_stage(m, m->q, m->res, buf[cur], buf[cur ^ 1], (float)RK_A[k], (float)RK_B[k], (float)dt);
      m->src_now = 0.f;
      if (e != cudaSuccess) return e;
      cur ^= 1;
    }
  return cudaSuccess;
}

// rhs of the current state for the elements of sel, into slot (all traces refreshed first).
cudaError_t rhs_to(dg_mesh* m, const float* q, float* slot, const dgk::Sel& sel) {
  cudaError_t e = dgk::launch_trace(m, q, m->trace);
  if (e != cudaSuccess) return e;
  return dgk::launch_rhs_sel(m, q, m->trace, slot, sel);
}

// Two-level multi-rate AB3 (reading of Sec. 2.4), fine step h, coarse step 2h.
// Start-up: four LSRK(5,4) steps of size h, recording rhs at t = 0, 2h, 3h.
cudaError_t mrab3(dg_mesh* m, int nsteps, double h) {
  const size_t fs = 4 * (size_t)m->ndof;
  float* H[3] = {m->hist, m->hist + fs, m->hist + 2 * fs};
  const dgk::Sel &C = m->lev[0], &F = m->lev[1];
  cudaError_t e;
  if (!m->mr_started) {
    if ((e = rhs_to(m, m->q, H[2], m->all)) != cudaSuccess) return e;   // r(0)
    if ((e = lsrk_steps(m, 2, h)) != cudaSuccess) return e;
    if ((e = rhs_to(m, m->q, H[1], m->all)) != cudaSuccess) return e;   // r(2h)
    if ((e = lsrk_steps(m, 1, h)) != cudaSuccess) return e;
    if ((e = rhs_to(m, m->q, H[0], m->all)) != cudaSuccess) return e;   // r(3h)
    if ((e = lsrk_steps(m, 1, h)) != cudaSuccess) return e;
    m->cslot[0] = 0; m->cslot[1] = 1; m->cslot[2] = 2;   // coarse: new r^n, r(2h), r(0)
    m->fslot[0] = 2; m->fslot[1] = 0; m->fslot[2] = 1;   // fine:   new r^n, r(3h), r(2h)
    m->mr_started = true;
  }
  const float a0 = 23.f / 12.f, a1 = -16.f / 12.f, a2 = 5.f / 12.f;
  const float b0 = 17.f / 24.f, b1 = -7.f / 24.f, b2 = 2.f / 24.f;
  const float hf = (float)h, hc = (float)(2 * h);
  float* pred = m->res;   // predicted coarse state (the LSRK residual is free between start-ups)
  for (int s = 0; s < nsteps; ++s) {
    int* c = m->cslot;
    int* f = m->fslot;
    // rhs at t_n: coarse -> H[c0], fine -> H[f0]
    if ((e = dgk::launch_trace(m, m->q, m->trace)) != cudaSuccess) return e;
    if ((e = dgk::launch_rhs_sel(m, m->q, m->trace, H[c[0]], C)) != cudaSuccess) return e;
    if ((e = dgk::launch_rhs_sel(m, m->q, m->trace, H[f[0]], F)) != cudaSuccess) return e;
    // fine AB3 to t_n + h; coarse prediction at t_n + h
    if ((e = dgk::launch_ab(m, F, m->q, m->q, H[f[0]], H[f[1]], H[f[2]], hf * a0, hf * a1, hf * a2)) != cudaSuccess) return e;
    if ((e = dgk::launch_ab(m, C, m->q, pred, H[c[0]], H[c[1]], H[c[2]], hc * b0, hc * b1, hc * b2)) != cudaSuccess) return e;
    // traces at t_n + h (fine: state, coarse: prediction), fine rhs -> H[f2]
    if ((e = dgk::launch_trace_sel(m, m->q, m->trace, F)) != cudaSuccess) return e;
    if ((e = dgk::launch_trace_sel(m, pred, m->trace, C)) != cudaSuccess) return e;
    if ((e = dgk::launch_rhs_sel(m, m->q, m->trace, H[f[2]], F)) != cudaSuccess) return e;
    // fine AB3 to t_n + 2h; coarse AB3 to t_n + 2h
    if ((e = dgk::launch_ab(m, F, m->q, m->q, H[f[2]], H[f[0]], H[f[1]], hf * a0, hf * a1, hf * a2)) != cudaSuccess) return e;
    if ((e = dgk::launch_ab(m, C, m->q, m->q, H[c[0]], H[c[1]], H[c[2]], hc * a0, hc * a1, hc * a2)) != cudaSuccess) return e;
    // rotate histories
    int f0 = f[0], f1 = f[1], f2 = f[2];
    f[0] = f1; f[1] = f2; f[2] = f0;
    int c0 = c[0], c1 = c[1], c2 = c[2];
    c[0] = c2; c[1] = c0; c[2] = c1;
  }
  return cudaSuccess;
}

// Fused form of mrab3 for N <= 4: one kernel per type and level and substep computes the rhs,
// stores it in the history, applies the AB3 update (and the coarse half-step prediction) and
// deposits the traces for the next substep.  Trace buffers: A (t_n), B (t_n + h), C (t_n + 2h).
cudaError_t mrab3_fused(dg_mesh* m, int nsteps, double h) {
  const size_t fs = 4 * (size_t)m->ndof;
  float* H[3] = {m->hist, m->hist + fs, m->hist + 2 * fs};
  const dgk::Sel &C = m->lev[0], &F = m->lev[1];
  cudaError_t e;
  if (!m->mr_started) {
    if ((e = rhs_to(m, m->q, H[2], m->all)) != cudaSuccess) return e;   // r(0)
    if ((e = lsrk_steps(m, 2, h)) != cudaSuccess) return e;
    if ((e = rhs_to(m, m->q, H[1], m->all)) != cudaSuccess) return e;   // r(2h)
    if ((e = lsrk_steps(m, 1, h)) != cudaSuccess) return e;
    if ((e = rhs_to(m, m->q, H[0], m->all)) != cudaSuccess) return e;   // r(3h)
    if ((e = lsrk_steps(m, 1, h)) != cudaSuccess) return e;
    m->cslot[0] = 0; m->cslot[1] = 1; m->cslot[2] = 2;
    m->fslot[0] = 2; m->fslot[1] = 0; m->fslot[2] = 1;
    m->mr_started = true;
  }
  const size_t plane2 = 2 * (size_t)m->nsides * m->nq;
  float* TA = m->trace;
  float* TB = m->trace + plane2;
  float* TC = m->trace3;
  if ((e = dgk::launch_trace(m, m->q, TA)) != cudaSuccess) return e;
  const float hc = (float)(2 * h), hf = (float)h;
  const float ac[3] = {hc * 23.f / 12.f, -hc * 16.f / 12.f, hc * 5.f / 12.f};
  const float pc[3] = {hc * 17.f / 24.f, -hc * 7.f / 24.f, hc * 2.f / 24.f};
  const float af[3] = {hf * 23.f / 12.f, -hf * 16.f / 12.f, hf * 5.f / 12.f};
  const float zero[3] = {0.f, 0.f, 0.f};
  for (int s = 0; s < nsteps; ++s) {
    int* c = m->cslot;
    int* f = m->fslot;
    if ((e = dgk::launch_mr(m, true, C, m->q, TA, TB, TC, H[c[0]], H[c[1]], H[c[2]], ac, pc)) != cudaSuccess)
      return e;
    if ((e = dgk::launch_mr(m, false, F, m->q, TA, TB, nullptr, H[f[0]], H[f[1]], H[f[2]], af, zero)) !=
        cudaSuccess)
      return e;
    if ((e = dgk::launch_mr(m, false, F, m->q, TB, TC, nullptr, H[f[2]], H[f[0]], H[f[1]], af, zero)) !=
        cudaSuccess)
      return e;
    int f0 = f[0], f1 = f[1], f2 = f[2];
    f[0] = f1; f[1] = f2; f[2] = f0;
    int c0 = c[0], c1 = c[1], c2 = c[2];
    c[0] = c2; c[1] = c0; c[2] = c1;
    float* tmp = TA;
    TA = TC;
    TC = tmp;
  }
  return cudaSuccess;
}

}  // namespace

namespace dgk {
cudaError_t launch_watchdog(int* err, long long limit, cudaStream_t s);   // kernels_tc.cu
}

extern "C" dg_status dg_watchdog_selftest(dg_mesh* m, int64_t limit_cycles) {
  if (!m || !m->derr || limit_cycles < 1 || limit_cycles > (1LL << 32)) return DG_EINVAL;
  cudaError_t e = dgk::launch_watchdog(m->derr, (long long)limit_cycles, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return device_flags(m);
}

cudaError_t dg_enqueue_steps(dg_mesh* m, int nsteps, double dt, double t0) {
  if (m->nlevels == 2 && m->integrator == 1) return dg_mrlsrk_steps(m, nsteps, dt);
  if (m->nlevels == 2)   // fused kernels: N <= 4 with lattice exchange on tet / pyramid triangle faces
    return m->N <= 4 && m->tri_lat ? mrab3_fused(m, nsteps, dt) : mrab3(m, nsteps, dt);
  return nsteps > 0 ? lsrk_steps(m, nsteps, dt, t0) : cudaSuccess;
}

double dg_step_time(const dg_mesh* m, int nsteps, double dt, bool fresh) {
  if (m->nlevels == 2 && m->integrator == 1) return nsteps * 2 * dt;
  if (m->nlevels == 2) return (fresh ? 4 * dt : 0.0) + nsteps * 2 * dt;
  return nsteps * dt;
}

extern "C" dg_status dg_step(dg_mesh* m, int nsteps, double dt, double* t_inout) {
  if (!m || nsteps < 0) return DG_EINVAL;
  if (!(dt > 0)) dt = m->dt_min;
  if (nsteps == 0) return DG_OK;
  if (m->src_e >= 0) {
    if (m->nlevels != 1) {
      g_err = "a point source is built for single-rate LSRK";
      return DG_ENOTSUP;
    }
    if (!t_inout) {
      g_err = "a point source needs the start time (t_inout)";
      return DG_EINVAL;
    }
  }
  const bool fresh = m->nlevels == 2 && m->integrator == 0 && !m->mr_started;
  cudaError_t e = dg_enqueue_steps(m, nsteps, dt, t_inout ? *t_inout : 0.0);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    g_err = "dg_step: the multi-rate LSRK buffers (15 states) do not fit";
    return DG_ENOMEM;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (t_inout) *t_inout += dg_step_time(m, nsteps, dt, fresh);
  return DG_OK;
}

extern "C" {

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
  const dg_status st = device_flags(m);
  if (st != DG_OK) return st;
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

dg_status dg_adjoint_step(dg_mesh* m, int nsteps, double dt, double t0, float* lambda, const float* resid,
                          double* g_c2, double* g_amp) {
  if (!m || nsteps < 0 || !lambda) return DG_EINVAL;
  if (g_amp && m->src_e < 0) {
    g_err = "grad_amp needs a point source (dg_set_source)";
    return DG_EINVAL;
  }
  if (resid && m->nrec == 0) {
    g_err = "receiver residuals need receivers (dg_set_receivers)";
    return DG_EINVAL;
  }
  if (m->nlevels != 1 || m->hex_sem || m->pyr_form != 0 || m->precision != 0) {
    g_err = "adjoint built for single-rate LSRK with GL hexahedra, skew-form pyramids and FP32 products";
    return DG_ENOTSUP;
  }
  if (!(dt > 0)) dt = m->dt_min;
  if (nsteps == 0) return DG_OK;
  cudaError_t e = dg_adjoint_run(m, nsteps, dt, t0, lambda, resid, g_c2, g_amp);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();   // clear the (non-sticky) allocation error
    g_err = "dg_adjoint_step: scratch of nsteps + 9 states does not fit; use shorter windows";
    return DG_ENOMEM;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  return DG_OK;
}

}  // extern "C"
