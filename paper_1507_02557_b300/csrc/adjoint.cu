// Discrete adjoint of LSRK(5,4) steps (dg_adjoint_step, include/dg.h).
//
// For a loss L of the state after n steps, lambda = dL/dq_n is carried back through the
// 2N-storage stages (res^{k+1} = a_k res^k + dt R q^k, q^{k+1} = q^k + b_k res^{k+1}) in reverse:
//     rho += b_k lambda;  lambda += dt R^T rho;  g += dt rho^T d(R q^k)/dc^2;  rho *= a_k.
// R^T is applied through the forward operator: with W = blockdiag(M, M/c^2) (the energy weight
// of Sec. 3) and F = diag(1,-1,-1,-1), R^T = W F R F W^{-1}, because the central part of W R is
// skew (the energy identity), its upwind penalty symmetric, and flipping u negates the former
// and keeps the latter.  So each reverse stage is one forward rhs of F W^{-1} rho.
// The c^2 gradient of element K collects rho_u . (R q)_u / c^2_K (the 1/rho = c^2 factor of the
// u-equation) and, on every face of K, -tau_scale/2 (dtau_p/dc^2_K I_p + dtau_u/dc^2_K I_u) with
// I_p = int [q_p][v_p], I_u = int [q.n][v.n], v = W^{-1} rho, tau_p = 2/(1/c^- + 1/c^+),
// tau_u = 1/tau_p; on a wall (tau_p = c_K, mirror state) -tau_scale/(2 c_K) int q_p v_p.
// The face integrals use the traces the forward kernels exchange (canonical points, or the
// triangle lattice of tets and pyramids with its face mass).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "kcommon.cuh"

namespace dgk {
namespace {

struct TypeView {
  int K = 0, Np = 0;
  int64_t dof_off = 0, goff = 0;   // first DOF of the type; first element in the global numbering
  const float* geo = nullptr;
  const float* c2 = nullptr;
};

TypeView view(const dg_mesh* m, int t) {
  TypeView v;
  v.K = m->td[t].K;
  v.Np = m->td[t].Np;
  v.dof_off = m->td[t].dof_off;
  v.geo = m->td[t].geo;
  v.c2 = m->td[t].c2;
  for (int u = 0; u < t; ++u) v.goff += m->td[u].K;
  return v;
}

// Diagonal mass of node n of element e: hexahedron w_i w_j w_k J(r_i, s_j, t_k) (GL collocation,
// trilinear map from its coefficients c1..c7), pyramid J at the node, LSC wedge 1.
template <int T>
__device__ float node_mass(const TypeView& V, const float* hexc, int N, int64_t e, int n) {
  if (T == DG_WEDGE) return 1.f;
  if (T == DG_PYR) return V.geo[(e * 10 + 9) * V.Np + n];
  const int n1 = N + 1, i = n % n1, j = (n / n1) % n1, k = n / (n1 * n1);
  const float* w1 = hexc + n1 * n1 + 2 * n1;
  const float* r1 = w1 + n1;
  const float r = r1[i], s = r1[j], t = r1[k];
  const float* g = V.geo + e * 24;
  float F[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F[d][0] = g[d] + g[9 + d] * s + g[12 + d] * t + g[18 + d] * s * t;
    F[d][1] = g[3 + d] + g[9 + d] * r + g[15 + d] * t + g[18 + d] * r * t;
    F[d][2] = g[6 + d] + g[12 + d] * r + g[15 + d] * s + g[18 + d] * r * s;
  }
  const float J = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                  F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                  F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
  return w1[i] * w1[j] * w1[k] * J;
}

// mode 0: o1 = W^{-1} x, o2 = F W^{-1} x.   mode 1: o1 += s W F x.
template <int T>
__global__ void mass_diag_kernel(TypeView V, const float* hexc, int N, int64_t ndof, int mode,
                                 const float* x, float* o1, float* o2, float s) {
  const int64_t n_all = (int64_t)V.K * V.Np;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n_all;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = id / V.Np;
    const float mm = node_mass<T>(V, hexc, N, e, (int)(id % V.Np));
    const float c2 = V.c2[e];
    const int64_t d = V.dof_off + id;
    if (mode == 0) {
      const float p = x[d] / mm;
      o1[d] = p;
      o2[d] = p;
#pragma unroll
      for (int f = 1; f < 4; ++f) {
        const float u = c2 * x[f * ndof + d] / mm;
        o1[f * ndof + d] = u;
        o2[f * ndof + d] = -u;
      }
    } else {
      o1[d] += s * mm * x[d];
#pragma unroll
      for (int f = 1; f < 4; ++f) o1[f * ndof + d] -= s * mm * x[f * ndof + d] / c2;
    }
  }
}

// Tetrahedra: M = J_K Mhat (dense reference mass), same modes.
__global__ void mass_tet_kernel(TypeView V, const float* Mh, const float* Minv, int64_t ndof, int mode,
                                const float* x, float* o1, float* o2, float s) {
  const int Np = V.Np;
  const int64_t n_all = (int64_t)V.K * Np;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n_all;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = id / Np;
    const int n = (int)(id % Np);
    const float J = V.geo[e * 12 + 9], c2 = V.c2[e];
    const int64_t base = V.dof_off + e * Np;
    const float* row = (mode == 0 ? Minv : Mh) + (size_t)n * Np;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      float acc = 0.f;
      for (int mm = 0; mm < Np; ++mm) acc = fmaf(row[mm], x[f * ndof + base + mm], acc);
      const int64_t d = f * ndof + base + n;
      if (mode == 0) {
        const float v = (f ? c2 : 1.f) * acc / J;
        o1[d] = v;
        o2[d] = f ? -v : v;
      } else {
        o1[d] += s * J * acc * (f ? -1.f / c2 : 1.f);
      }
    }
  }
}

// traces of F v from those of v: the p plane as is, the u.n plane negated
__global__ void flip_traces_kernel(int64_t plane, const float* tv, float* tfv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * plane; i += (int64_t)gridDim.x * blockDim.x)
    tfv[i] = i < plane ? tv[i] : -tv[i];
}

// y = a y + b x over n floats
__global__ void axpby_kernel(int64_t n, float a, float* y, float b, const float* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * y[i] + (x ? b * x[i] : 0.f);
}

// g[K] += dt rho_u . y_u / c^2_K, one warp per element
__global__ void grad_vol_kernel(TypeView V, int64_t ndof, const float* rho, const float* y, double* g,
                                double dt) {
  const int lane = threadIdx.x & 31;
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < V.K;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t base = V.dof_off + e * V.Np;
    float acc = 0.f;   // FP32 products of FP32 fields; FP64 only for the accumulation into g
    for (int n = lane; n < V.Np; n += 32)
#pragma unroll
      for (int f = 1; f < 4; ++f) acc = fmaf(rho[f * ndof + base + n], y[f * ndof + base + n], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) g[V.goff + e] += dt * (double)acc / V.c2[e];
  }
}

struct FaceView {
  int64_t side_off[4] = {0, 0, 0, 0}, K[4] = {0, 0, 0, 0}, goff[4] = {0, 0, 0, 0};
  int nf[4] = {6, 5, 5, 4};
  const float* c2[4] = {nullptr, nullptr, nullptr, nullptr};
  const int* nbr = nullptr;
  const float* fw = nullptr;    // [nsides][nq]
  const float* Mf = nullptr;    // [nfn][nfn]
  int nq = 0, nfn = 0, tri_lat = 0;
  float tau_scale = 1.f;
  int64_t nsides = 0, plane = 0;
};

__device__ void side_elem(const FaceView& F, int64_t s, int& t, int64_t& e, int& f) {
  t = 3;
  for (int u = 0; u < 3; ++u)
    if (s < F.side_off[u + 1]) {
      t = u;
      break;
    }
  const int64_t r = s - F.side_off[t];
  e = r / F.nf[t];
  f = (int)(r % F.nf[t]);
}

constexpr int MAX_NFN = 36;   // (N+1)(N+2)/2 at N = 7

// One thread per face (the lower-numbered side of an interior face, every wall side).
// TQ, TV: trace buffers (p plane, u.n plane) of q and v written with wall_self.
__global__ void grad_face_kernel(FaceView F, const float* TQ, const float* TV, double* g, double dt) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= F.nsides) return;
  const int nb = F.nbr[s];
  if (nb >= 0 && nb < s) return;
  int t, f;
  int64_t e;
  side_elem(F, s, t, e, f);
  const bool lat = F.tri_lat && (t == DG_TET || (t == DG_PYR && f > 0));
  const int npt = lat ? F.nfn : F.nq;
  const int64_t o = s * F.nq, on = (int64_t)(nb >= 0 ? nb : 0) * F.nq;
  float jqp[MAX_NFN], jvp[MAX_NFN], jqn[MAX_NFN], jvn[MAX_NFN];
  float Ip = 0.f, Iu = 0.f;   // FP32 sums of FP32 trace products (FP64 is slow here)
  for (int i = 0; i < npt; ++i) {
    float qp, vp, qn = 0.f, vn = 0.f;
    if (nb >= 0) {   // jumps [x] = x(neighbour) - x(own); u.n planes carry each writer's normal
      qp = TQ[o + i] - TQ[on + i];
      vp = TV[o + i] - TV[on + i];
      qn = -TQ[F.plane + o + i] - TQ[F.plane + on + i];
      vn = -TV[F.plane + o + i] - TV[F.plane + on + i];
    } else {         // wall: own values (written into the side's own slot)
      qp = TQ[o + i];
      vp = TV[o + i];
    }
    if (lat) {
      jqp[i] = qp; jvp[i] = vp; jqn[i] = qn; jvn[i] = vn;
    } else {
      const float w = F.fw[o + i];
      Ip = fmaf(w * qp, vp, Ip);
      Iu = fmaf(w * qn, vn, Iu);
    }
  }
  if (lat) {
    for (int i = 0; i < npt; ++i) {
      float sp = 0.f, su = 0.f;
      for (int j = 0; j < npt; ++j) {
        sp = fmaf(F.Mf[i * F.nfn + j], jvp[j], sp);
        su = fmaf(F.Mf[i * F.nfn + j], jvn[j], su);
      }
      Ip = fmaf(jqp[i], sp, Ip);
      Iu = fmaf(jqn[i], su, Iu);
    }
    Ip *= F.fw[o];
    Iu *= F.fw[o];
  }
  const double cK = sqrt((double)F.c2[t][e]);
  if (nb < 0) {
    atomicAdd(&g[F.goff[t] + e], dt * (-0.5 * F.tau_scale * Ip / cK));
    return;
  }
  int t2, f2;
  int64_t e2;
  side_elem(F, nb, t2, e2, f2);
  const double cO = sqrt((double)F.c2[t2][e2]);
  const double sig = 1.0 / cK + 1.0 / cO;
  const double cs[2] = {cK, cO};
  const int64_t gi[2] = {F.goff[t] + e, F.goff[t2] + e2};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double c = cs[k];
    const double dtp = 1.0 / (sig * sig * c * c * c), dtu = -0.25 / (c * c * c);
    atomicAdd(&g[gi[k]], dt * (-0.5 * F.tau_scale * (dtp * Ip + dtu * Iu)));
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 148 * 32) b = 148 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

template <class Tv>
cudaError_t upload_lazy(dg_mesh* m, float*& dev, const std::vector<Tv>& h) {
  if (dev || h.empty()) return cudaSuccess;
  std::vector<float> f(h.begin(), h.end());
  dev = static_cast<float*>(dg_alloc_owned(m, f.size() * sizeof(float)));
  if (!dev) return cudaErrorMemoryAllocation;
  return cudaMemcpy(dev, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
}

// mode 0: o1 = W^{-1} x, o2 = F W^{-1} x; mode 1: o1 += s W F x (every element type)
cudaError_t apply_mass(dg_mesh* m, int mode, const float* x, float* o1, float* o2, float s) {
  for (int t = 0; t < 4; ++t) {
    const TypeView V = view(m, t);
    if (V.K == 0) continue;
    const unsigned gr = grid_for((int64_t)V.K * V.Np, 256);
    if (t == DG_HEX) mass_diag_kernel<DG_HEX><<<gr, 256, 0, m->stream>>>(V, m->hexc, m->N, m->ndof, mode, x, o1, o2, s);
    else if (t == DG_WEDGE) mass_diag_kernel<DG_WEDGE><<<gr, 256, 0, m->stream>>>(V, m->hexc, m->N, m->ndof, mode, x, o1, o2, s);
    else if (t == DG_PYR) mass_diag_kernel<DG_PYR><<<gr, 256, 0, m->stream>>>(V, m->hexc, m->N, m->ndof, mode, x, o1, o2, s);
    else mass_tet_kernel<<<gr, 256, 0, m->stream>>>(V, m->tet_mhat_dev, m->tet_minv_dev, m->ndof, mode, x, o1, o2, s);
  }
  return cudaGetLastError();
}

cudaError_t axpby(dg_mesh* m, int64_t n, float a, float* y, float b, const float* x) {
  axpby_kernel<<<grid_for(n, 256), 256, 0, m->stream>>>(n, a, y, b, x);
  return cudaGetLastError();
}

// traces of x into tout, wall sides included (their own slot)
cudaError_t traces_all(dg_mesh* m, const float* x, float* tout) {
  m->wall_self = true;
  cudaError_t e = launch_trace(m, x, tout);
  m->wall_self = false;
  return e;
}

}  // namespace
}  // namespace dgk

cudaError_t dg_adjoint_run(dg_mesh* m, int nsteps, double dt, double t0, float* lam, const float* resid,
                           double* grad, double* grad_amp) {
  using namespace dgk;
  const int64_t fs = 4 * m->ndof;
  const size_t need = (size_t)nsteps + 9;   // step states S[0..n-1], Q1..Q4, rho, v, fv, y, z
  cudaError_t e = cudaSuccess;
  if (m->adj_states < need) {
    if (m->adj_buf) cudaFree(m->adj_buf);
    m->adj_buf = nullptr;
    m->adj_states = 0;
    e = cudaMalloc(&m->adj_buf, need * fs * sizeof(float));
    if (e != cudaSuccess) {
      m->adj_buf = nullptr;
      return e;
    }
    m->adj_states = need;
  }
  if ((e = upload_lazy(m, m->face_w_dev, m->face_w)) != cudaSuccess) return e;
  if ((e = upload_lazy(m, m->face_mass_dev, m->face_mass)) != cudaSuccess) return e;
  if ((e = upload_lazy(m, m->tet_minv_dev, m->tet_mhat_inv)) != cudaSuccess) return e;
  float* S = m->adj_buf;
  float* Q = S + (size_t)nsteps * fs;   // Q1..Q4
  float* rho = Q + 4 * fs;
  float* v = rho + fs;
  float* fv = v + fs;
  float* y = fv + fs;
  float* z = y + fs;
  const size_t plane = (size_t)m->nsides * m->nq;
  float* TB[2] = {m->trace, m->trace + 2 * plane};
  cudaStream_t st = m->stream;
  auto stage_state = [&](int k) { return k == 0 ? nullptr : Q + (size_t)(k - 1) * fs; };

  FaceView F;
  for (int t = 0; t < 4; ++t) {
    F.side_off[t] = m->td[t].side_off;
    F.K[t] = m->td[t].K;
    F.c2[t] = m->td[t].c2;
    F.goff[t] = view(m, t).goff;
  }
  F.nbr = m->side_nbr;
  F.fw = m->face_w_dev;
  F.Mf = m->face_mass_dev;
  F.nq = m->nq;
  F.nfn = (m->N + 1) * (m->N + 2) / 2;
  F.tri_lat = m->tri_lat ? 1 : 0;
  F.tau_scale = (float)m->tau_scale;
  F.nsides = m->nsides;
  F.plane = (int64_t)plane;

  // step states S[j] = q_j, j < nsteps
  if ((e = cudaMemcpyAsync(S, m->q, fs * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  for (int j = 0; j + 1 < nsteps; ++j) {
    float* qp = S + (size_t)j * fs;
    float* qj = S + (size_t)(j + 1) * fs;
    if ((e = launch_trace(m, qp, TB[0])) != cudaSuccess) return e;
    int cur = 0;
    for (int k = 0; k < 5; ++k) {   // the first stage writes q_{j+1} from q_j, the others update it
      dg_source_at(m, t0 + (j + RK_C[k]) * dt);
      e = launch_stage(m, k == 0 ? qp : qj, m->res, TB[cur], TB[cur ^ 1], (float)RK_A[k], (float)RK_B[k], (float)dt,
                       qj);
      m->src_now = 0.f;
      if (e != cudaSuccess) return e;
      cur ^= 1;
    }
  }
  for (int j = nsteps - 1; j >= 0; --j) {
    float* Sj = S + (size_t)j * fs;
    // receiver forcing of the state after step j
    if (resid && (e = dg_receiver_inject(m, resid + (size_t)j * m->nrec, lam)) != cudaSuccess) return e;
    // stage inputs q^1..q^4 of step j (the stage kernels update in place)
    if ((e = launch_trace(m, Sj, TB[0])) != cudaSuccess) return e;
    int cur = 0;
    for (int k = 0; k < 4; ++k) {   // out of place: q^{k+1} from q^k
      float* src = k == 0 ? Sj : stage_state(k);
      dg_source_at(m, t0 + (j + RK_C[k]) * dt);
      e = launch_stage(m, src, m->res, TB[cur], TB[cur ^ 1], (float)RK_A[k], (float)RK_B[k], (float)dt,
                       stage_state(k + 1));
      m->src_now = 0.f;
      if (e != cudaSuccess) return e;
      cur ^= 1;
    }
    if ((e = cudaMemsetAsync(rho, 0, fs * sizeof(float), st)) != cudaSuccess) return e;
    for (int k = 4; k >= 0; --k) {
      const float* qk = k == 0 ? Sj : stage_state(k);
      if ((e = axpby(m, fs, 1.f, rho, (float)RK_B[k], lam)) != cudaSuccess) return e;
      if (grad_amp && m->src_e >= 0) {   // d(stage source dt amp ricker(t_k) g)/d amp against rho
        const double tk = t0 + (j + RK_C[k]) * dt;
        if ((e = dg_source_amp_grad(m, rho, dt * dg_ricker(tk, m->src_f0, m->src_t0), grad_amp)) != cudaSuccess)
          return e;
      }
      if ((e = apply_mass(m, 0, rho, v, fv, 0.f)) != cudaSuccess) return e;
      if (grad) {
        if ((e = traces_all(m, qk, TB[0])) != cudaSuccess) return e;
        if ((e = traces_all(m, v, TB[1])) != cudaSuccess) return e;
        if ((e = launch_rhs(m, qk, TB[0], y)) != cudaSuccess) return e;
        for (int t = 0; t < 4; ++t) {
          const TypeView V = view(m, t);
          if (V.K) grad_vol_kernel<<<grid_for((int64_t)V.K * 32, 256), 256, 0, st>>>(V, m->ndof, rho, y, grad, dt);
        }
        grad_face_kernel<<<(unsigned)((m->nsides + 255) / 256), 256, 0, st>>>(F, TB[0], TB[1], grad, dt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      if (grad) {   // traces of F v = those of v (in TB[1]) with u.n negated: no trace launch
        flip_traces_kernel<<<grid_for(2 * (int64_t)plane, 256), 256, 0, st>>>((int64_t)plane, TB[1], TB[0]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      } else if ((e = launch_trace(m, fv, TB[0])) != cudaSuccess) {
        return e;
      }
      if ((e = launch_rhs(m, fv, TB[0], z)) != cudaSuccess) return e;
      if ((e = apply_mass(m, 1, z, lam, nullptr, (float)dt)) != cudaSuccess) return e;
      if (k > 0 && (e = axpby(m, fs, (float)RK_A[k], rho, 0.f, nullptr)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}
