// Two-level multi-rate LSRK(5,4) (integrator 1; include/dg.h, dg_step): a local time-stepping
// Runge-Kutta scheme read for the multi-rate level schedule of Sec. 2.4, in the manner of the
// LTS-RK methods of Grote, Mehlin & Mitkova (2015).  Fine step h, coarse step H = 2h, B the rhs
// operator (dg_rhs), P the restriction to the fine elements, R(z) = sum rho_i z^i the LSRK(5,4)
// amplification.  Per coarse step from y:
//   z_j = B^j y (j = 1..5)                                      full trace + rhs launches
//   u_j = B (I - P) z_j (j = 0..4) on S                         X = coarse part of z_j on T
//   W(tau) = sum_j rho_{j+1} tau^{j+1} u_j
//   v' = B P (y + W(tau) + v), v(0) = 0: two LSRK(5,4) steps of h on S, the input's fine part in Y
//   y += W(H) + v
// S = fine elements and the coarse elements sharing a face with one: outside S, B (I - P) z_j =
// z_{j+1} and B P (...) = 0, so the final combination takes z_{j+1} there.  T = S and its face
// neighbours: the elements whose traces the rhs launches over S read.  X keeps zeros at the fine
// DOFs and Y at the coarse DOFs (written once, at allocation), so only the other part is copied.
// The launches reuse the trace / rhs kernels of the single-rate path on element lists, plus the
// elementwise kernels below (FP32; coefficients formed in FP64 on the host).
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace dgk {

namespace {

enum { EW_COPY = 0, EW_BUILD_Y = 1, EW_STAGE = 2, EW_ZERO = 3, EW_FINAL = 4 };

struct Ew {
  const int* list;   // element list of the type (NULL: 0..K-1)
  int K, Np;
  int64_t dof_off, ndof;
  float* y;          // FINAL: state (updated); BUILD_Y: the state y (read)
  float* out;        // COPY: destination; BUILD_Y: Y
  const float* src;  // COPY: source
  const float* u[5];
  const float* z[5];  // FINAL: z_{j+1}
  float* v;
  float* r;
  const float* R;
  float c[5];
  float a, b, h;
  const unsigned char* ins;   // FINAL: 1 for elements of S
};

template <int OP>
__global__ void __launch_bounds__(256) ew_kernel(Ew P) {
  const int64_t n = (int64_t)P.K * P.Np;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t li = x / P.Np;
    const int nn = (int)(x - li * P.Np);
    const int64_t e = P.list ? (int64_t)P.list[li] : li;
    const int64_t id0 = P.dof_off + e * P.Np + nn;
    const bool in_s = OP == EW_FINAL ? P.ins[e] != 0 : false;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int64_t id = f * P.ndof + id0;
      if (OP == EW_COPY) {
        P.out[id] = P.src[id];
      } else if (OP == EW_BUILD_Y) {
        float s = P.y[id] + P.v[id];
#pragma unroll
        for (int j = 0; j < 5; ++j) s += P.c[j] * P.u[j][id];
        P.out[id] = s;
      } else if (OP == EW_STAGE) {
        const float rr = P.a * P.r[id] + P.h * P.R[id];
        P.r[id] = rr;
        P.v[id] += P.b * rr;
      } else if (OP == EW_ZERO) {
        P.v[id] = 0.f;
        P.r[id] = 0.f;
      } else {
        float w = 0.f;
#pragma unroll
        for (int j = 0; j < 5; ++j) w += P.c[j] * (in_s ? P.u[j][id] : P.z[j][id]);
        P.y[id] += w + (in_s ? P.v[id] : 0.f);
      }
    }
  }
}

// one elementwise launch per element type over the elements of sel (NULL: all)
template <int OP>
cudaError_t ew(dg_mesh* m, const Sel* sel, Ew P) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  P.ndof = m->ndof;
  for (int t = 0; t < 4; ++t) {
    P.K = sel ? (int)sel->count[t] : m->td[t].K;
    if (P.K == 0) continue;
    P.list = sel ? sel->list[t] : nullptr;
    P.Np = m->td[t].Np;
    P.dof_off = m->td[t].dof_off;
    P.ins = m->mr_in_s[t];
    const int64_t need = ((int64_t)P.K * P.Np + 255) / 256;
    ew_kernel<OP><<<(unsigned)(need < 8 * sms ? need : 8 * sms), 256, 0, m->stream>>>(P);
  }
  return cudaGetLastError();
}

// rho_1..rho_5 of the LSRK(5,4) amplification R(z) = sum rho_i z^i
void amplification(double rho[6]) {
  double y[6] = {1, 0, 0, 0, 0, 0}, r[6] = {0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 5; ++k) {
    double nr[6];
    for (int i = 0; i < 6; ++i) nr[i] = RK_A[k] * r[i] + (i > 0 ? y[i - 1] : 0.0);
    for (int i = 0; i < 6; ++i) {
      r[i] = nr[i];
      y[i] += RK_B[k] * r[i];
    }
  }
  for (int i = 0; i < 6; ++i) rho[i] = y[i];
}

}  // namespace

}  // namespace dgk

cudaError_t dg_mrlsrk_steps(dg_mesh* m, int nsteps, double h) {
  using namespace dgk;
  const size_t fs = 4 * (size_t)m->ndof;
  cudaError_t e = cudaSuccess;
  if (!m->mrl) {
    m->mrl = static_cast<float*>(dg_alloc_owned(m, 15 * fs * sizeof(float)));
    if (!m->mrl) return cudaErrorMemoryAllocation;
    e = cudaMemsetAsync(m->mrl, 0, 15 * fs * sizeof(float), m->stream);
    if (e != cudaSuccess) return e;
  }
  float* Z[6] = {m->q, m->mrl, m->mrl + fs, m->mrl + 2 * fs, m->mrl + 3 * fs, m->mrl + 4 * fs};   // z_0..z_5
  float* U[5] = {m->mrl + 5 * fs, m->mrl + 6 * fs, m->mrl + 7 * fs, m->mrl + 8 * fs, m->mrl + 9 * fs};
  float *X = m->mrl + 10 * fs, *Y = m->mrl + 11 * fs, *R = m->mrl + 12 * fs, *V = m->mrl + 13 * fs,
        *RS = m->mrl + 14 * fs;
  float* tr = m->trace;
  double rho[6];
  amplification(rho);
  const double H = 2.0 * h;
  for (int st = 0; st < nsteps && e == cudaSuccess; ++st) {
    // z_j = B^j y
    for (int j = 1; j <= 5 && e == cudaSuccess; ++j) {
      e = launch_trace(m, Z[j - 1], tr);
      if (e == cudaSuccess) e = launch_rhs(m, Z[j - 1], tr, Z[j]);
    }
    // u_j = B (I - P) z_j on S
    for (int j = 0; j < 5 && e == cudaSuccess; ++j) {
      Ew P{};
      P.out = X;
      P.src = Z[j];
      e = ew<EW_COPY>(m, &m->mr_tc, P);
      if (e == cudaSuccess) e = launch_trace_sel(m, X, tr, m->mr_t);
      if (e == cudaSuccess) e = launch_rhs_sel(m, X, tr, U[j], m->mr_s);
    }
    // v: two LSRK(5,4) steps of h on S
    Ew Pz{};
    Pz.v = V;
    Pz.r = RS;
    if (e == cudaSuccess) e = ew<EW_ZERO>(m, &m->mr_s, Pz);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
      for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
        const double tau = (s + RK_C[k]) * h;
        Ew P{};
        P.y = m->q;
        P.out = Y;
        P.v = V;
        double tp = tau;
        for (int j = 0; j < 5; ++j, tp *= tau) {
          P.u[j] = U[j];
          P.c[j] = (float)(rho[j + 1] * tp);
        }
        e = ew<EW_BUILD_Y>(m, &m->lev[1], P);
        if (e == cudaSuccess) e = launch_trace_sel(m, Y, tr, m->mr_t);
        if (e == cudaSuccess) e = launch_rhs_sel(m, Y, tr, R, m->mr_s);
        Ew Q{};
        Q.v = V;
        Q.r = RS;
        Q.R = R;
        Q.a = (float)RK_A[k];
        Q.b = (float)RK_B[k];
        Q.h = (float)h;
        if (e == cudaSuccess) e = ew<EW_STAGE>(m, &m->mr_s, Q);
      }
    // y += W(H) + v
    Ew F{};
    F.y = m->q;
    F.v = V;
    double Hp = H;
    for (int j = 0; j < 5; ++j, Hp *= H) {
      F.u[j] = U[j];
      F.z[j] = Z[j + 1];
      F.c[j] = (float)(rho[j + 1] * Hp);
    }
    if (e == cudaSuccess) e = ew<EW_FINAL>(m, nullptr, F);
  }
  return e;
}
