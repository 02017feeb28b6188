// Point source and receivers in hexahedra (dg_set_source, dg_set_receivers, dg_sample_receivers;
// include/dg.h) and the adjoint's receiver forcing and source-amplitude terms.
//
// The pressure equation (1/kappa) p_t + div u = f of Sec. 2.2 with f = amp ricker(t) delta(x - x_s):
// its weak form adds amp ricker(t) M_K^{-1} phi(x_s) to the p rhs of the hexahedron K holding
// x_s (GL-collocated mass w_n J_n).  A receiver reads p(x_r) = sum_n phi_n(x_r) p_n.  A point is
// located by Newton's method on the trilinear map of the hexahedra whose corner box contains it;
// a point on a face shared by two hexahedra belongs to the one of lower index.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "kcommon.cuh"
#include "refelem.h"

namespace {

// x(r) of the trilinear map with coefficients c[8][3] (c0, c1 r, c2 s, c3 t, c4 rs, c5 rt, c6 st,
// c7 rst) and its Jacobian F[d][a] = dx_d/dr_a.
void hex_map(const double* c, const double r[3], double x[3], double F[3][3]) {
  const double mon[8] = {1, r[0], r[1], r[2], r[0] * r[1], r[0] * r[2], r[1] * r[2], r[0] * r[1] * r[2]};
  const double dr[8] = {0, 1, 0, 0, r[1], r[2], 0, r[1] * r[2]};
  const double ds[8] = {0, 0, 1, 0, r[0], 0, r[2], r[0] * r[2]};
  const double dt[8] = {0, 0, 0, 1, 0, r[0], r[1], r[0] * r[1]};
  for (int d = 0; d < 3; ++d) {
    x[d] = F[d][0] = F[d][1] = F[d][2] = 0.0;
    for (int m = 0; m < 8; ++m) {
      x[d] += c[3 * m + d] * mon[m];
      F[d][0] += c[3 * m + d] * dr[m];
      F[d][1] += c[3 * m + d] * ds[m];
      F[d][2] += c[3 * m + d] * dt[m];
    }
  }
}

double det3(const double F[3][3]) {
  return F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
         F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
}

// lowest-index hexahedron containing x and the reference point there; false if none
bool locate(const dg_mesh* m, const double x[3], int64_t& e_out, double r_out[3]) {
  const int64_t K = m->td[DG_HEX].K;
  for (int64_t e = 0; e < K; ++e) {
    const double* c = m->hex_coef.data() + (size_t)e * 24;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v < 8; ++v) {
      const double r[3] = {(v & 1) ? 1.0 : -1.0, (v & 2) ? 1.0 : -1.0, (v & 4) ? 1.0 : -1.0};
      double xv[3], F[3][3];
      hex_map(c, r, xv, F);
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], xv[d]);
        hi[d] = std::max(hi[d], xv[d]);
      }
    }
    bool in = true;
    for (int d = 0; d < 3; ++d) in = in && x[d] >= lo[d] - 1e-9 && x[d] <= hi[d] + 1e-9;
    if (!in) continue;
    double r[3] = {0, 0, 0};
    for (int it = 0; it < 50; ++it) {
      double xr[3], F[3][3];
      hex_map(c, r, xr, F);
      const double b[3] = {x[0] - xr[0], x[1] - xr[1], x[2] - xr[2]};
      const double D = det3(F);
      if (!(std::fabs(D) > 0)) break;
      double dr[3];
      for (int a = 0; a < 3; ++a) {   // Cramer's rule
        double G[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) G[i][j] = j == a ? b[i] : F[i][j];
        dr[a] = det3(G) / D;
      }
      for (int a = 0; a < 3; ++a) r[a] += dr[a];
      if (std::max(std::fabs(dr[0]), std::max(std::fabs(dr[1]), std::fabs(dr[2]))) < 1e-14) break;
    }
    if (std::fabs(r[0]) <= 1 + 1e-10 && std::fabs(r[1]) <= 1 + 1e-10 && std::fabs(r[2]) <= 1 + 1e-10) {
      e_out = e;
      for (int a = 0; a < 3; ++a) r_out[a] = r[a];
      return true;
    }
  }
  return false;
}

// phi_n(r) of the nodal hexahedron basis, node n = i + n1 (j + n1 k)
std::vector<double> hex_basis_at(const dg_mesh* m, const double r[3]) {
  const int n1 = m->N + 1;
  std::vector<double> l[3];
  for (int a = 0; a < 3; ++a) {
    l[a].resize(n1);
    dgref::lagrange(m->hex_r1, r[a], l[a].data(), nullptr);
  }
  std::vector<double> phi((size_t)n1 * n1 * n1);
  for (int k = 0; k < n1; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) phi[i + n1 * (j + n1 * k)] = l[0][i] * l[1][j] * l[2][k];
  return phi;
}

template <class T>
T* to_device(dg_mesh* m, const std::vector<T>& h) {
  T* p = static_cast<T*>(dg_alloc_owned(m, h.size() * sizeof(T)));
  if (p && cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
  return p;
}

// out[r] = sum_n rows[r][n] p[dof_off + e_r Np + n], one warp per receiver
__global__ void sample_kernel(int nrec, const int* rec_e, const float* rows, int Np, int64_t dof_off,
                              const float* q, float* out) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nrec) return;
  const float* p = q + dof_off + (int64_t)rec_e[r] * Np;
  float acc = 0.f;
  for (int n = lane; n < Np; n += 32) acc = fmaf(rows[(size_t)r * Np + n], p[n], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[r] = acc;
}

// lambda_p[e_r, n] += resid[r] rows[r][n] (the transpose of sample_kernel)
__global__ void inject_kernel(int nrec, const int* rec_e, const float* rows, int Np, int64_t dof_off,
                              const float* resid, float* lam) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)nrec * Np) return;
  const int r = (int)(id / Np), n = (int)(id % Np);
  atomicAdd(lam + dof_off + (int64_t)rec_e[r] * Np + n, resid[r] * rows[(size_t)r * Np + n]);
}

// *g += coef sum_n rho_p[e_s, n] g_s[n], one block
__global__ void amp_grad_kernel(const float* rho, int64_t base, const float* gs, int Np, double coef, double* g) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int n = threadIdx.x; n < Np; n += blockDim.x) acc += (double)rho[base + n] * gs[n];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *g += coef * s[0];
}

}  // namespace

double dg_ricker(double t, double f0, double t0) {
  const double a = M_PI * M_PI * f0 * f0 * (t - t0) * (t - t0);
  return (1.0 - 2.0 * a) * std::exp(-a);
}

void dg_source_at(dg_mesh* m, double t) {
  m->src_now = m->src_e >= 0 ? (float)(m->src_amp * dg_ricker(t, m->src_f0, m->src_t0)) : 0.f;
}

cudaError_t dg_receiver_inject(dg_mesh* m, const float* resid, float* lam) {
  if (m->nrec == 0) return cudaSuccess;
  const int Np = m->td[DG_HEX].Np;
  const int64_t n = (int64_t)m->nrec * Np;
  inject_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->nrec, m->rec_e, m->rec_rows, Np,
                                                                    m->td[DG_HEX].dof_off, resid, lam);
  return cudaGetLastError();
}

cudaError_t dg_source_amp_grad(dg_mesh* m, const float* rho, double coef, double* g) {
  const int Np = m->td[DG_HEX].Np;
  amp_grad_kernel<<<1, 256, 0, m->stream>>>(rho, m->td[DG_HEX].dof_off + m->src_e * Np, m->src_g, Np, coef, g);
  return cudaGetLastError();
}

extern "C" {

dg_status dg_set_source(dg_mesh* m, const double* x, double amp, double f0, double t0) {
  if (!m || !x || !(f0 > 0) || !std::isfinite(amp) || !std::isfinite(t0)) return DG_EINVAL;
  int64_t e;
  double r[3];
  if (!locate(m, x, e, r)) {
    dg_set_last_error("the source point is not inside a hexahedron");
    return DG_EINVAL;
  }
  const int n1 = m->N + 1, Np = n1 * n1 * n1;
  std::vector<double> phi = hex_basis_at(m, r);
  const double* c = m->hex_coef.data() + (size_t)e * 24;
  std::vector<float> g(Np);
  for (int n = 0; n < Np; ++n) {   // M^{-1} phi(x_s), M = w_i w_j w_k J(r_i, s_j, t_k)
    const int i = n % n1, j = (n / n1) % n1, k = n / (n1 * n1);
    const double rn[3] = {m->hex_r1[i], m->hex_r1[j], m->hex_r1[k]};
    double xn[3], F[3][3];
    hex_map(c, rn, xn, F);
    g[n] = (float)(phi[n] / (m->hex_w1[i] * m->hex_w1[j] * m->hex_w1[k] * det3(F)));
  }
  if (!m->src_g) m->src_g = static_cast<float*>(dg_alloc_owned(m, Np * sizeof(float)));
  if (!m->src_g || cudaMemcpy(m->src_g, g.data(), Np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    dg_set_last_error("source upload failed");
    return DG_ECUDA;
  }
  m->src_e = e;
  m->src_amp = amp;
  m->src_f0 = f0;
  m->src_t0 = t0;
  return DG_OK;
}

dg_status dg_set_receivers(dg_mesh* m, int nrec, const double* xyz) {
  if (!m || nrec < 0 || (nrec > 0 && !xyz)) return DG_EINVAL;
  const int Np = m->td[DG_HEX].Np;
  std::vector<int> re(nrec);
  std::vector<float> rows((size_t)nrec * Np);
  for (int r = 0; r < nrec; ++r) {
    int64_t e;
    double rr[3];
    if (!locate(m, xyz + 3 * r, e, rr)) {
      dg_set_last_error("receiver " + std::to_string(r) + " is not inside a hexahedron");
      return DG_EINVAL;
    }
    re[r] = (int)e;
    std::vector<double> phi = hex_basis_at(m, rr);
    for (int n = 0; n < Np; ++n) rows[(size_t)r * Np + n] = (float)phi[n];
  }
  m->nrec = 0;
  if (nrec == 0) return DG_OK;
  m->rec_e = to_device(m, re);
  m->rec_rows = to_device(m, rows);
  if (!m->rec_e || !m->rec_rows) {
    dg_set_last_error("receiver upload failed");
    return DG_ECUDA;
  }
  m->nrec = nrec;
  return DG_OK;
}

dg_status dg_sample_receivers(dg_mesh* m, const float* q, float* out) {
  if (!m || !out) return DG_EINVAL;
  if (m->nrec == 0) return DG_OK;
  if (!q) q = m->q;
  sample_kernel<<<(unsigned)((m->nrec * 32 + 255) / 256), 256, 0, m->stream>>>(
      m->nrec, m->rec_e, m->rec_rows, m->td[DG_HEX].Np, m->td[DG_HEX].dof_off, q, out);
  if (cudaGetLastError() != cudaSuccess) {
    dg_set_last_error("receiver sampling launch failed");
    return DG_ECUDA;
  }
  return DG_OK;
}

}  // extern "C"
