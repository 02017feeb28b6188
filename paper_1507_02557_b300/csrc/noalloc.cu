// dg_energy_noalloc: the discrete energy without any device allocation.
//
// For callers that must not allocate device memory while they run: real-time loops that cannot
// take the latency of cudaMalloc (it may synchronise the device) and frameworks that have
// reserved all device memory for their own pool, so that a cudaMalloc of the library would fail
// or evict their data.  The per-element partial sums live in a file-scope static device array
// instead of the mesh's accumulator, and are reduced in a fixed order, so repeated calls on the
// same state return bitwise-equal results.
//
// The static array (DG_NOALLOC_MAX_ELEMS + 1 doubles, 8 MiB) is held by every GPU that loads
// libdg until the process exits.  Its device address is looked up with cudaGetSymbolAddress once
// per device, on the first call made with that device current.  All calls share the array and
// it keeps the last call's contents (every call overwrites the entries it sums, so nothing needs
// clearing): calls whose work overlaps on the GPU (different streams, meshes or host threads)
// race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"

#define DG_NOALLOC_MAX_ELEMS (1 << 20)

namespace {

static __device__ __align__(256) double g_energy_scratch[DG_NOALLOC_MAX_ELEMS + 1];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch_ptr[MAX_DEVICES] = {};

// Element energy 1/2 (p^T M p + (1/c^2) sum_d u_d^T M u_d), one block per element.
template <int T, int N>
__global__ void __launch_bounds__(128) element_energy(const float* q, int64_t ndof, int64_t dof_off,
                                                      const float* geo, const float* c2, const float* hexc,
                                                      const float* mhat, double* part, int64_t part_off) {
  constexpr int n1 = N + 1;
  constexpr int NP = T == DG_HEX ? n1 * n1 * n1
                     : T == DG_WEDGE ? n1 * n1 * (N + 2) / 2
                     : T == DG_PYR ? n1 * (N + 2) * (2 * N + 3) / 6
                                   : n1 * (N + 2) * (N + 3) / 6;
  __shared__ double s_red[128];
  const int64_t e = blockIdx.x;
  const int64_t base = dof_off + e * NP;
  const int tid = threadIdx.x;
  const double ic2 = 1.0 / (double)c2[e];
  double loc = 0.0;
  for (int n = tid; n < NP; n += 128) {
    double qv[4];
    for (int f = 0; f < 4; ++f) qv[f] = q[f * ndof + base + n];
    double wsq = qv[0] * qv[0] + ic2 * (qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
    if (T == DG_HEX) {
      const float* g = geo + e * 24;
      const float* r1 = hexc + n1 * n1 + 3 * n1;
      const float* w1 = hexc + n1 * n1 + 2 * n1;
      int i = n % n1, j = (n / n1) % n1, k = n / (n1 * n1);
      float r = r1[i], s = r1[j], t = r1[k], xr[3], xs[3], xt[3];
      for (int d = 0; d < 3; ++d) {
        xr[d] = g[d] + g[9 + d] * s + g[12 + d] * t + g[18 + d] * s * t;
        xs[d] = g[3 + d] + g[9 + d] * r + g[15 + d] * t + g[18 + d] * r * t;
        xt[d] = g[6 + d] + g[12 + d] * r + g[15 + d] * s + g[18 + d] * r * s;
      }
      double J = (double)xr[0] * (xs[1] * xt[2] - xs[2] * xt[1]) + (double)xr[1] * (xs[2] * xt[0] - xs[0] * xt[2]) +
                 (double)xr[2] * (xs[0] * xt[1] - xs[1] * xt[0]);
      loc += (double)w1[i] * w1[j] * w1[k] * J * wsq;
    } else if (T == DG_WEDGE) {
      loc += wsq;
    } else if (T == DG_PYR) {
      loc += (double)geo[(e * 10 + 9) * NP + n] * wsq;
    } else {
      double s = 0.0;
      for (int m = 0; m < NP; ++m) {
        double o = (double)q[base + m] * qv[0];
        for (int f = 1; f < 4; ++f) o += ic2 * (double)q[f * ndof + base + m] * qv[f];
        s += (double)mhat[n * NP + m] * o;
      }
      loc += (double)geo[e * 12 + 9] * s;
    }
  }
  s_red[tid] = loc;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (tid < s) s_red[tid] += s_red[tid + s];
    __syncthreads();
  }
  if (tid == 0) part[part_off + e] = 0.5 * s_red[0];
}

// Fixed-order sum of part[0..n) into part[DG_NOALLOC_MAX_ELEMS].
__global__ void __launch_bounds__(1024) ordered_sum(double* part, int64_t n) {
  __shared__ double s[1024];
  double loc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) loc += part[i];
  s[threadIdx.x] = loc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[DG_NOALLOC_MAX_ELEMS] = s[0];
}

template <int N>
void launch_parts(const dg_mesh* m, const float* q, double* part) {
  int64_t off = 0;
  const dgk::TypeDev* td = m->td;
  cudaStream_t s = m->stream;
  if (td[0].K) element_energy<DG_HEX, N><<<td[0].K, 128, 0, s>>>(q, m->ndof, td[0].dof_off, td[0].geo, td[0].c2, m->hexc, nullptr, part, off);
  off += td[0].K;
  if (td[1].K) element_energy<DG_WEDGE, N><<<td[1].K, 128, 0, s>>>(q, m->ndof, td[1].dof_off, td[1].geo, td[1].c2, nullptr, nullptr, part, off);
  off += td[1].K;
  if (td[2].K) element_energy<DG_PYR, N><<<td[2].K, 128, 0, s>>>(q, m->ndof, td[2].dof_off, td[2].geo, td[2].c2, nullptr, nullptr, part, off);
  off += td[2].K;
  if (td[3].K) element_energy<DG_TET, N><<<td[3].K, 128, 0, s>>>(q, m->ndof, td[3].dof_off, td[3].geo, td[3].c2, nullptr, m->tet_mhat_dev, part, off);
}

}  // namespace

extern "C" dg_status dg_energy_noalloc(dg_mesh* m, const float* q, double* E) {
  if (!m || !E) return DG_EINVAL;
  if (!q) q = m->q;
  const int64_t nel = m->td[0].K + m->td[1].K + m->td[2].K + m->td[3].K;
  if (nel > DG_NOALLOC_MAX_ELEMS) {
    dg_set_last_error("dg_energy_noalloc: mesh has more than 1048576 elements (static scratch limit)");
    return DG_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES || dev != m->device) {
    dg_set_last_error("dg_energy_noalloc: the mesh's device must be the current device");
    return DG_EINVAL;
  }
  double* part = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      e = cudaGetSymbolAddress((void**)&g_scratch_ptr[dev], g_energy_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        dg_set_last_error(std::string("dg_energy_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return DG_ECUDA;
      }
    }
    part = g_scratch_ptr[dev];
  }
  switch (m->N) {
    case 1: launch_parts<1>(m, q, part); break;
    case 2: launch_parts<2>(m, q, part); break;
    case 3: launch_parts<3>(m, q, part); break;
    case 4: launch_parts<4>(m, q, part); break;
    case 5: launch_parts<5>(m, q, part); break;
    case 6: launch_parts<6>(m, q, part); break;
    case 7: launch_parts<7>(m, q, part); break;
    case 8: launch_parts<8>(m, q, part); break;
    case 9: launch_parts<9>(m, q, part); break;
    default:
      dg_set_last_error("dg_energy_noalloc: N must be in 1..9");
      return DG_ENOTSUP;
  }
  ordered_sum<<<1, 1024, 0, m->stream>>>(part, nel);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(E, part + DG_NOALLOC_MAX_ELEMS, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    dg_set_last_error(std::string("dg_energy_noalloc: ") + cudaGetErrorString(e));
    return DG_ECUDA;
  }
  // the same reports as dg_energy: a timed-out device wait, then a non-finite energy
  const dg_status st = dg_device_flags(m);
  if (st != DG_OK) return st;
  if (!std::isfinite(*E)) {
    dg_set_last_error("dg_energy_noalloc: the energy is not finite");
    return DG_ENONFINITE;
  }
  return DG_OK;
}
