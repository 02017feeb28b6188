// CUDA kernels of the hybrid DG right-hand side and LSRK stage (sm_103a).
//
// One stage is one kernel per element type.  Each kernel reads its element's
// state, recomputes the volume term, reads the neighbour traces (p, u.n) that
// the neighbours deposited in this element's face "inbox" during the previous
// launch, computes the upwind flux and lift, applies the inverse mass matrix and
// the LSRK(5,4) update, then evaluates the traces of the updated state and
// deposits them in the neighbours' inboxes of the other trace buffer
// (ping-pong).  Kernel boundaries give the grid-wide ordering between stages.
//
// Flux (Sec. 2.2): with [p] = p+ - p-, [u].n- = -(u+.n+) - (u-.n-):
//   strong form  f_p = 1/2 (tau_p [p] - [u].n-)
//   skew form    f_p = 1/2 tau_p [p] - n-.{u}
//   u-equation   f_u = 1/2 (tau_u [u].n- - [p]),  vector flux f_u n-
// Wall faces (p = 0): mirror state p+ = -p-, u+ = u-.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "kcommon.cuh"

namespace dgk {

// ============================================================================ hexahedra
template <int N>
struct HexCfg {
  static constexpr int n1 = N + 1, NP = n1 * n1 * n1, NQ = n1 * n1;
  static constexpr int TPE = ((NP + 31) / 32) * 32;
  static constexpr int EPB = TPE >= 256 ? 1 : 256 / TPE;
  static constexpr int NT = TPE * EPB;
};

// x_r, x_s, x_t of the trilinear map at (r,s,t); g = c1..c7 (3 floats each)
__device__ __forceinline__ void hex_jac(const float* g, float r, float s, float t, float xr[3],
                                        float xs[3], float xt[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float c1 = g[d], c2 = g[3 + d], c3 = g[6 + d], c4 = g[9 + d], c5 = g[12 + d], c6 = g[15 + d],
          c7 = g[18 + d];
    xr[d] = c1 + c4 * s + c5 * t + c7 * s * t;
    xs[d] = c2 + c4 * r + c6 * t + c7 * r * t;
    xt[d] = c3 + c5 * r + c6 * s + c7 * r * s;
  }
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

template <int N, int MODE>
__global__ void __launch_bounds__(HexCfg<N>::NT) hex_kernel(Args A) {
  using C = HexCfg<N>;
  constexpr int n1 = C::n1, NP = C::NP, NQ = C::NQ, EPB = C::EPB, TPE = C::TPE;
  __shared__ float s_q[EPB][4][NP];
  __shared__ float s_geo[EPB][24];
  __shared__ float s_F[EPB][6][4][NQ];
  __shared__ float s_n[EPB][6][3][NQ];
  __shared__ float s_D[n1 * n1], s_Vm[n1], s_Vp[n1], s_w[n1], s_r[n1];
  __shared__ int s_perm[8 * NQ];

  const int le = threadIdx.x / TPE, tid = threadIdx.x % TPE;
  const int64_t li = (int64_t)blockIdx.x * EPB + le;
  const bool valid = li < A.K;
  const int64_t e = valid ? (A.elist ? (int64_t)A.elist[li] : li) : 0;
  for (int i = threadIdx.x; i < n1 * n1; i += blockDim.x) s_D[i] = A.hexc[i];
  for (int i = threadIdx.x; i < n1; i += blockDim.x) {
    s_Vm[i] = A.hexc[n1 * n1 + i];
    s_Vp[i] = A.hexc[n1 * n1 + n1 + i];
    s_w[i] = A.hexc[n1 * n1 + 2 * n1 + i];
    s_r[i] = A.hexc[n1 * n1 + 3 * n1 + i];
  }
  for (int i = threadIdx.x; i < 8 * NQ; i += blockDim.x) s_perm[i] = A.perm[i];
  const int64_t base = A.dof_off + e * NP;
  if (valid && tid < NP) {
#pragma unroll
    for (int f = 0; f < 4; ++f) s_q[le][f][tid] = A.q[f * A.ndof + base + tid];
  }
  if (valid && tid < 24) s_geo[le][tid] = A.geo[e * 24 + tid];
  __syncthreads();

  const int i = tid % n1, j = (tid / n1) % n1, k = tid / (n1 * n1);
  float rhs[4] = {0.f, 0.f, 0.f, 0.f};
  float Jn = 1.f;
  const float c2 = valid ? A.c2[e] : 0.f;

  if (MODE != MODE_TRACE) {
    // ---- volume term, Alg. hex_vol: collocated strong form (M^{-1} cancels w J)
    if (valid && tid < NP) {
      float dr[4], ds[4], dt[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          a0 += s_D[i * n1 + m] * s_q[le][f][m + n1 * (j + n1 * k)];
          a1 += s_D[j * n1 + m] * s_q[le][f][i + n1 * (m + n1 * k)];
          a2 += s_D[k * n1 + m] * s_q[le][f][i + n1 * (j + n1 * m)];
        }
        dr[f] = a0;
        ds[f] = a1;
        dt[f] = a2;
      }
      float xr[3], xs[3], xt[3], g0[3], g1[3], g2[3];
      hex_jac(s_geo[le], s_r[i], s_r[j], s_r[k], xr, xs, xt);
      cross3(xs, xt, g0);
      cross3(xt, xr, g1);
      cross3(xr, xs, g2);
      Jn = xr[0] * g0[0] + xr[1] * g0[1] + xr[2] * g0[2];
      const float iJ = 1.f / Jn;
      float grad[4][3];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int d = 0; d < 3; ++d) grad[f][d] = (g0[d] * dr[f] + g1[d] * ds[f] + g2[d] * dt[f]) * iJ;
      rhs[0] = -(grad[1][0] + grad[2][1] + grad[3][2]);
      rhs[1] = -c2 * grad[0][0];
      rhs[2] = -c2 * grad[0][1];
      rhs[3] = -c2 * grad[0][2];
    }
    // ---- face fluxes at the 6 (N+1)^2 face points
    for (int fq = tid; fq < 6 * NQ; fq += TPE) {
      if (!valid) break;
      const int f = fq / NQ, lp = fq % NQ, a = lp % n1, b = lp / n1;
      const int ax = f >> 1;
      const float sg = (f & 1) ? 1.f : -1.f;
      const float* V = (f & 1) ? s_Vp : s_Vm;
      float r, s, t;
      if (ax == 0) { r = sg; s = s_r[a]; t = s_r[b]; }
      else if (ax == 1) { r = s_r[a]; s = sg; t = s_r[b]; }
      else { r = s_r[a]; s = s_r[b]; t = sg; }
      float xr[3], xs[3], xt[3], nv[3];
      hex_jac(s_geo[le], r, s, t, xr, xs, xt);
      if (ax == 0) cross3(xs, xt, nv);
      else if (ax == 1) cross3(xt, xr, nv);
      else cross3(xr, xs, nv);
      const float Js = sqrtf(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      const float inv = sg / Js;
      nv[0] *= inv; nv[1] *= inv; nv[2] *= inv;
      float tr[4];
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          int id = ax == 0 ? m + n1 * (a + n1 * b) : ax == 1 ? a + n1 * (m + n1 * b) : a + n1 * (b + n1 * m);
          acc += V[m] * s_q[le][fl][id];
        }
        tr[fl] = acc;
      }
      const float unm = nv[0] * tr[1] + nv[1] * tr[2] + nv[2] * tr[3];
      const int64_t gs = A.side_off + e * 6 + f;
      const int nb = A.nbr[gs];
      const int cidx = s_perm[A.code[gs] * NQ + lp];
      float P = 0.f, UN = 0.f;
      if (nb >= 0) {
        P = A.tin[gs * NQ + cidx];
        UN = A.tin[A.plane + gs * NQ + cidx];
      }
      const float tp = A.tau_scale * A.tau[gs], tu = A.tau_scale / A.tau[gs];
      float fp, fu;
      flux(nb < 0, tr[0], unm, P, UN, tp, tu, false, fp, fu);
      const float wgt = s_w[a] * s_w[b] * Js;
      s_F[le][f][0][lp] = wgt * fp;
      s_F[le][f][1][lp] = wgt * fu * nv[0];
      s_F[le][f][2][lp] = wgt * fu * nv[1];
      s_F[le][f][3][lp] = wgt * fu * nv[2];
      s_n[le][f][0][lp] = nv[0];
      s_n[le][f][1][lp] = nv[1];
      s_n[le][f][2][lp] = nv[2];
    }
    __syncthreads();
    // ---- lift, Alg. hex_surf: M^{-1} w w J^s l(+-1) flux
    if (valid && tid < NP) {
      const float iM = 1.f / (s_w[i] * s_w[j] * s_w[k] * Jn);
      const int jk = j + n1 * k, ik = i + n1 * k, ij = i + n1 * j;
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        float sum = s_Vm[i] * s_F[le][0][fl][jk] + s_Vp[i] * s_F[le][1][fl][jk] +
                    s_Vm[j] * s_F[le][2][fl][ik] + s_Vp[j] * s_F[le][3][fl][ik] +
                    s_Vm[k] * s_F[le][4][fl][ij] + s_Vp[k] * s_F[le][5][fl][ij];
        rhs[fl] += (fl == 0 ? 1.f : c2) * iM * sum;
      }
      if (MODE == MODE_RHS) {
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) A.rhs[fl * A.ndof + base + tid] = rhs[fl];
      } else {
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
          const int64_t id = fl * A.ndof + base + tid;
          float r = A.a * A.res[id] + A.dt * rhs[fl];
          float qn = s_q[le][fl][tid] + A.b * r;
          A.res[id] = r;
          A.qout[id] = qn;
          rhs[fl] = qn;
        }
      }
    }
    if (MODE == MODE_STAGE) {
      __syncthreads();
      if (valid && tid < NP) {
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) s_q[le][fl][tid] = rhs[fl];
      }
    }
  }
  if (MODE == MODE_TRACE || MODE == MODE_STAGE) {
    __syncthreads();
    // ---- traces of the (updated) state, deposited in the neighbours' inboxes
    for (int fq = tid; fq < 6 * NQ; fq += TPE) {
      if (!valid) break;
      const int f = fq / NQ, lp = fq % NQ, a = lp % n1, b = lp / n1;
      const int ax = f >> 1;
      const int64_t gs = A.side_off + e * 6 + f;
      const int nb = A.nbr[gs];
      if (nb < 0) continue;
      const float* V = (f & 1) ? s_Vp : s_Vm;
      float nv[3];
      if (MODE == MODE_STAGE) {
        nv[0] = s_n[le][f][0][lp];
        nv[1] = s_n[le][f][1][lp];
        nv[2] = s_n[le][f][2][lp];
      } else {
        const float sg = (f & 1) ? 1.f : -1.f;
        float r, s, t;
        if (ax == 0) { r = sg; s = s_r[a]; t = s_r[b]; }
        else if (ax == 1) { r = s_r[a]; s = sg; t = s_r[b]; }
        else { r = s_r[a]; s = s_r[b]; t = sg; }
        float xr[3], xs[3], xt[3];
        hex_jac(s_geo[le], r, s, t, xr, xs, xt);
        if (ax == 0) cross3(xs, xt, nv);
        else if (ax == 1) cross3(xt, xr, nv);
        else cross3(xr, xs, nv);
        const float inv = sg / sqrtf(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        nv[0] *= inv; nv[1] *= inv; nv[2] *= inv;
      }
      float tr[4];
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          int id = ax == 0 ? m + n1 * (a + n1 * b) : ax == 1 ? a + n1 * (m + n1 * b) : a + n1 * (b + n1 * m);
          acc += V[m] * s_q[le][fl][id];
        }
        tr[fl] = acc;
      }
      const int cidx = s_perm[A.code[gs] * NQ + lp];
      A.tout[(int64_t)nb * NQ + cidx] = tr[0];
      A.tout[A.plane + (int64_t)nb * NQ + cidx] = nv[0] * tr[1] + nv[1] * tr[2] + nv[2] * tr[3];
    }
  }
}

// ============================================================================ hexahedra, warp per element
// For N <= 4: a warp owns EPW = 32 / (N+1)^2 elements; lane (i,j) of an element keeps
// the column (i,j,0..N) of all four fields in registers.  t-derivatives and the
// t-face traces come from registers; r/s-derivatives and r/s-face traces read the
// element's nodes as float4 (p,u,v,w) from shared memory.  Only warp-level
// synchronisation after the start of the block.
__constant__ float c_hexw[5][64];   // per N: D1[n1*n1] (row = node), Vm[n1], Vp[n1], w[n1], r[n1]

cudaError_t upload_hex_constants(int N, const float* hc, int count) {
  if (N < 1 || N > 4 || count > 64) return cudaSuccess;
  return cudaMemcpyToSymbol(c_hexw, hc, count * sizeof(float), N * 64 * sizeof(float));
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int N>
struct HexW {
  static constexpr int n1 = N + 1, NP = n1 * n1 * n1, NQ = n1 * n1;
  static constexpr int EPW = 32 / NQ;   // elements per warp
  static constexpr int WPB = 4;         // warps per block
  static constexpr int EPB = EPW * WPB;
};

__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// Outward unit normal and surface Jacobian at point (a,b) of hex face f (local face parameters).
template <int N>
__device__ __forceinline__ void hexw_face_geom(const float* g, const float* rr, int f, int a, int b, float nv[3],
                                               float& Js) {
  const int ax = f >> 1;
  const float sg = (f & 1) ? 1.f : -1.f;
  float u[3], v[3];
  if (ax == 0) {   // r = sg: x_s x x_t
    const float s = rr[a], t = rr[b];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = g[3 + d] + g[9 + d] * sg + (g[15 + d] + g[18 + d] * sg) * t;
      v[d] = g[6 + d] + g[12 + d] * sg + (g[15 + d] + g[18 + d] * sg) * s;
    }
  } else if (ax == 1) {   // s = sg: x_t x x_r
    const float r = rr[a], t = rr[b];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = g[6 + d] + g[15 + d] * sg + (g[12 + d] + g[18 + d] * sg) * r;
      v[d] = g[d] + g[9 + d] * sg + (g[12 + d] + g[18 + d] * sg) * t;
    }
  } else {   // t = sg: x_r x x_s
    const float r = rr[a], s = rr[b];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = g[d] + g[12 + d] * sg + (g[9 + d] + g[18 + d] * sg) * s;
      v[d] = g[3 + d] + g[15 + d] * sg + (g[9 + d] + g[18 + d] * sg) * r;
    }
  }
  cross3(u, v, nv);
  Js = sqrtf(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
  const float inv = sg / Js;
  nv[0] *= inv;
  nv[1] *= inv;
  nv[2] *= inv;
}

#ifndef DG_HEXW_MINB
#define DG_HEXW_MINB 4
#endif
template <int N, int MODE>
__global__ void __launch_bounds__(128, DG_HEXW_MINB) hexw_kernel(Args A) {
  using H = HexW<N>;
  constexpr int n1 = H::n1, NP = H::NP, NQ = H::NQ, EPW = H::EPW, WPB = H::WPB;
  __shared__ float4 s_q[WPB][EPW][NP];
  __shared__ float4 s_F[WPB][EPW][4][NQ];
  __shared__ float4 s_N[WPB][EPW][6][NQ];
  __shared__ float s_g[WPB][EPW][24];
  __shared__ int s_nb[WPB][EPW][6], s_code[WPB][EPW][6];
  __shared__ float s_tau[WPB][EPW][6];
  __shared__ int s_perm[8 * NQ];

  const float* Dm = c_hexw[N];
  const float* Vm = Dm + n1 * n1;
  const float* Vp = Vm + n1;
  const float* W1 = Vp + n1;
  const float* R1 = W1 + n1;

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / NQ, col = lane % NQ;
  const int i = col % n1, j = col / n1;
  const int64_t li = ((int64_t)blockIdx.x * WPB + w) * EPW + sub;
  const bool act = sub < EPW && li < A.K;
  const int64_t e = act ? (A.elist ? (int64_t)A.elist[li] : li) : 0;
  const int su = sub < EPW ? sub : 0;
  const int64_t base = A.dof_off + e * NP;

  for (int x = threadIdx.x; x < 8 * NQ; x += blockDim.x) s_perm[x] = A.perm[x];
  float q[4][n1], res[4][n1];
  if (act) {
#pragma unroll
    for (int k = 0; k < n1; ++k)
#pragma unroll
      for (int f = 0; f < 4; ++f) q[f][k] = A.q[f * A.ndof + base + col + NQ * k];
#ifdef DG_HEXW_RES_EARLY
    if (MODE == MODE_STAGE) {
#pragma unroll
      for (int k = 0; k < n1; ++k)
#pragma unroll
        for (int f = 0; f < 4; ++f) res[f][k] = A.res[f * A.ndof + base + col + NQ * k];
    }
#endif
    if (col < 24) s_g[w][su][col] = A.geo[e * 24 + col];
    if (NQ < 24 && col < NQ) {   // small N: fewer lanes than coefficients
      for (int x = col + NQ; x < 24; x += NQ) s_g[w][su][x] = A.geo[e * 24 + x];
    }
    if (col < 6) {
      const int64_t gs = A.side_off + e * 6 + col;
      s_nb[w][su][col] = A.nbr[gs];
      s_code[w][su][col] = A.code[gs];
      s_tau[w][su][col] = A.tau[gs];
    }
#pragma unroll
    for (int k = 0; k < n1; ++k) s_q[w][su][col + NQ * k] = make_float4(q[0][k], q[1][k], q[2][k], q[3][k]);
  }
  if (NQ < 6 && act) {   // N = 1: 4 lanes per element, 6 faces
    for (int x = col + NQ; x < 6; x += NQ) {
      const int64_t gs = A.side_off + e * 6 + x;
      s_nb[w][su][x] = A.nbr[gs];
      s_code[w][su][x] = A.code[gs];
      s_tau[w][su][x] = A.tau[gs];
    }
  }
  // L2 prefetch of what this element reads late: the residual (or the two history slots)
  // and its face inboxes; one 128-byte line per lane
  if (act && MODE != MODE_TRACE) {
    constexpr int LPF = (NP * 4 + 127) / 128 + 1;         // lines per field array of one element
    const int64_t b4 = base * 4;
    for (int x = col; x < 4 * LPF; x += NQ) {
      const int f = x / LPF, l = x % LPF;
      const int64_t line = (b4 & ~127LL) + 128LL * l;
      if (line >= b4 + NP * 4) continue;                 // only lines holding this element's values
      const int64_t off = f * A.ndof * 4 + (line < b4 ? b4 : line);
      if (MODE == MODE_STAGE) prefetch_l2(reinterpret_cast<const char*>(A.res) + off);
      if (MODE == MODE_MRC || MODE == MODE_MRF) {
        prefetch_l2(reinterpret_cast<const char*>(A.h1) + off);
        prefetch_l2(reinterpret_cast<const char*>(A.h2) + off);
      }
    }
    if (col < 12) {   // inboxes of the six faces, both planes (NQ floats each, <= 2 lines)
      const int64_t gs0 = (A.side_off + e * 6) * NQ * 4;
      const int64_t o = gs0 + (col % 6) * NQ * 4 + (col >= 6 ? A.plane * 4 : 0);
      prefetch_l2(reinterpret_cast<const char*>(A.tin) + o);
      prefetch_l2(reinterpret_cast<const char*>(A.tin) + o + NQ * 4 - 4);
    }
  }
  __syncthreads();
  const float* g = s_g[w][su];
  const float c2 = act ? A.c2[e] : 0.f;
  float rhs[4][n1];
  float Jn[n1];

  if (MODE != MODE_TRACE && act) {
    // ---- volume: collocated strong form (Alg. hex_vol), metrics built along the column
    float Dri[n1], Dsj[n1];
#pragma unroll
    for (int m = 0; m < n1; ++m) {
      Dri[m] = Dm[i * n1 + m];
      Dsj[m] = Dm[j * n1 + m];
    }
    const float r = R1[i], s = R1[j];
    float Ar[3], Br[3], As[3], Bs[3], xt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Ar[d] = g[d] + g[9 + d] * s;
      Br[d] = g[12 + d] + g[18 + d] * s;
      As[d] = g[3 + d] + g[9 + d] * r;
      Bs[d] = g[15 + d] + g[18 + d] * r;
      xt[d] = g[6 + d] + g[12 + d] * r + g[15 + d] * s + g[18 + d] * r * s;
    }
    float G0a[3], G0b[3], G1a[3], G1b[3], G2a[3], G2b[3], G2c[3], tmp[3];
    cross3(As, xt, G0a);
    cross3(Bs, xt, G0b);
    cross3(xt, Ar, G1a);
    cross3(xt, Br, G1b);
    cross3(Ar, As, G2a);
    cross3(Ar, Bs, G2b);
    cross3(Br, As, tmp);
    G2b[0] += tmp[0]; G2b[1] += tmp[1]; G2b[2] += tmp[2];
    cross3(Br, Bs, G2c);
#pragma unroll
    for (int k = 0; k < n1; ++k) {
      const float t = R1[k];
      float g0[3], g1[3], g2[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        g0[d] = G0a[d] + t * G0b[d];
        g1[d] = G1a[d] + t * G1b[d];
        g2[d] = G2a[d] + t * (G2b[d] + t * G2c[d]);
      }
      const float J = (Ar[0] + t * Br[0]) * g0[0] + (Ar[1] + t * Br[1]) * g0[1] + (Ar[2] + t * Br[2]) * g0[2];
      Jn[k] = J;
      const float iJ = 1.f / J;
      float4 dr = make_float4(0.f, 0.f, 0.f, 0.f), ds = dr;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        dr = f4fma(Dri[m], s_q[w][su][m + n1 * j + NQ * k], dr);
        ds = f4fma(Dsj[m], s_q[w][su][i + n1 * m + NQ * k], ds);
      }
      float dt[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        const float dk = Dm[k * n1 + m];
#pragma unroll
        for (int f = 0; f < 4; ++f) dt[f] = fmaf(dk, q[f][m], dt[f]);
      }
      const float drf[4] = {dr.x, dr.y, dr.z, dr.w}, dsf[4] = {ds.x, ds.y, ds.z, ds.w};
      // -div u and -c^2 grad p
      float div = 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) div += g0[d] * drf[1 + d] + g1[d] * dsf[1 + d] + g2[d] * dt[1 + d];
      rhs[0][k] = -div * iJ;
#pragma unroll
      for (int d = 0; d < 3; ++d) rhs[1 + d][k] = -c2 * iJ * (g0[d] * drf[0] + g1[d] * dsf[0] + g2[d] * dt[0]);
    }
  }
  if (MODE != MODE_TRACE) {
    // ---- fluxes at this lane's point (a,b) = (i,j) of all six faces
    float4 F45[2];
    if (act) {
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        float4 tm = make_float4(0.f, 0.f, 0.f, 0.f), tp = tm;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          float4 v;
          if (ax == 0) v = s_q[w][su][m + n1 * i + NQ * j];
          else if (ax == 1) v = s_q[w][su][i + n1 * m + NQ * j];
          else v = make_float4(q[0][m], q[1][m], q[2][m], q[3][m]);
          tm = f4fma(Vm[m], v, tm);
          tp = f4fma(Vp[m], v, tp);
        }
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const int f = 2 * ax + sd;
          const float4 tr = sd ? tp : tm;
          float nv[3], Js;
          hexw_face_geom<N>(g, R1, f, i, j, nv, Js);
          s_N[w][su][f][col] = make_float4(nv[0], nv[1], nv[2], Js);
          const float unm = nv[0] * tr.y + nv[1] * tr.z + nv[2] * tr.w;
          const int nb = s_nb[w][su][f];
          float P = 0.f, UN = 0.f;
          if (nb >= 0) {
            const int64_t gs = A.side_off + e * 6 + f;
            const int cidx = s_perm[s_code[w][su][f] * NQ + col];
            P = A.tin[gs * NQ + cidx];
            UN = A.tin[A.plane + gs * NQ + cidx];
          }
          const float ta = s_tau[w][su][f];
          float fp, fu;
          flux(nb < 0, tr.x, unm, P, UN, A.tau_scale * ta, A.tau_scale / ta, false, fp, fu);
          const float wg = W1[i] * W1[j] * Js;
          const float4 Fv = make_float4(wg * fp, wg * fu * nv[0], wg * fu * nv[1], wg * fu * nv[2]);
          if (ax < 2) s_F[w][su][f][col] = Fv;
          else F45[sd] = Fv;
        }
      }
    }
    __syncwarp();
    if (act) {
      // ---- lift (Alg. hex_surf), M^{-1} = 1/(w w w J), LSRK update
#pragma unroll
      for (int k = 0; k < n1; ++k) {
        const float4 F0 = s_F[w][su][0][j + n1 * k], F1 = s_F[w][su][1][j + n1 * k];
        const float4 F2 = s_F[w][su][2][i + n1 * k], F3 = s_F[w][su][3][i + n1 * k];
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        sum = f4fma(Vm[i], F0, sum);
        sum = f4fma(Vp[i], F1, sum);
        sum = f4fma(Vm[j], F2, sum);
        sum = f4fma(Vp[j], F3, sum);
        sum = f4fma(Vm[k], F45[0], sum);
        sum = f4fma(Vp[k], F45[1], sum);
        const float iM = 1.f / (W1[i] * W1[j] * W1[k] * Jn[k]);
        rhs[0][k] += iM * sum.x;
        rhs[1][k] += c2 * iM * sum.y;
        rhs[2][k] += c2 * iM * sum.z;
        rhs[3][k] += c2 * iM * sum.w;
      }
      if (MODE == MODE_RHS) {
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) A.rhs[f * A.ndof + base + col + NQ * k] = rhs[f][k];
      } else if (MODE == MODE_STAGE) {
#ifndef DG_HEXW_RES_EARLY
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) res[f][k] = A.res[f * A.ndof + base + col + NQ * k];
#endif
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const int64_t id = f * A.ndof + base + col + NQ * k;
            const float rr = A.a * res[f][k] + A.dt * rhs[f][k];
            q[f][k] += A.b * rr;
            A.res[id] = rr;
            A.qout[id] = q[f][k];
          }
      } else {   // MRC / MRF: AB3 update; MRC keeps the new state in res[] and the prediction in q[]
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const int64_t id = f * A.ndof + base + col + NQ * k;
            const float r0 = rhs[f][k], r1 = A.h1[id], r2 = A.h2[id];
            A.hw[id] = r0;
            const float qn = q[f][k] + A.ab0 * r0 + A.ab1 * r1 + A.ab2 * r2;
            A.qout[id] = qn;
            if (MODE == MODE_MRC) {
              res[f][k] = qn;
              q[f][k] += A.pr0 * r0 + A.pr1 * r1 + A.pr2 * r2;
            } else {
              q[f][k] = qn;
            }
          }
      }
    }
  }
  // ---- traces of the state in q[] / s_q into the neighbours' inboxes
  auto emit = [&](float* tout) {
    __syncwarp();
    if (act) {
#pragma unroll
      for (int k = 0; k < n1; ++k) s_q[w][su][col + NQ * k] = make_float4(q[0][k], q[1][k], q[2][k], q[3][k]);
    }
    __syncwarp();
    if (!act) return;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      float4 tm = make_float4(0.f, 0.f, 0.f, 0.f), tp = tm;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        float4 v;
        if (ax == 0) v = s_q[w][su][m + n1 * i + NQ * j];
        else if (ax == 1) v = s_q[w][su][i + n1 * m + NQ * j];
        else v = make_float4(q[0][m], q[1][m], q[2][m], q[3][m]);
        tm = f4fma(Vm[m], v, tm);
        tp = f4fma(Vp[m], v, tp);
      }
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int f = 2 * ax + sd;
        const int nb = s_nb[w][su][f];
        if (nb < 0) continue;
        float nv[3];
        if (MODE != MODE_TRACE) {
          const float4 nn = s_N[w][su][f][col];
          nv[0] = nn.x; nv[1] = nn.y; nv[2] = nn.z;
        } else {
          float Js;
          hexw_face_geom<N>(g, R1, f, i, j, nv, Js);
        }
        const float4 tr = sd ? tp : tm;
        const int cidx = s_perm[s_code[w][su][f] * NQ + col];
        tout[(int64_t)nb * NQ + cidx] = tr.x;
        tout[A.plane + (int64_t)nb * NQ + cidx] = nv[0] * tr.y + nv[1] * tr.z + nv[2] * tr.w;
      }
    }
  };
  if (MODE != MODE_RHS) emit(A.tout);
  if (MODE == MODE_MRC) {
    if (act) {
#pragma unroll
      for (int k = 0; k < n1; ++k)
#pragma unroll
        for (int f = 0; f < 4; ++f) q[f][k] = res[f][k];
    }
    emit(A.tout2);
  }
}

template <int N, int MODE>
static void launch_hexw_n(const Args& A, cudaStream_t s) {
  using H = HexW<N>;
  if (A.K == 0) return;
  dim3 grid((A.K + H::EPB - 1) / H::EPB);
  hexw_kernel<N, MODE><<<grid, 32 * H::WPB, 0, s>>>(A);
}

// ============================================================================ wedge, pyramid, tet

template <int T, int N>
struct GenCfg {
  static constexpr int NP = np_of(T, N), NQ = (N + 1) * (N + 1), NF = T == DG_TET ? 4 : 5;
  static constexpr int NC = T == DG_WEDGE ? (N + 1) * (N + 1) * (N + 1) : 1;
  static constexpr int NT = 128;
};

template <int T, int N, int MODE>
__global__ void __launch_bounds__(128) gen_kernel(Args A) {
  using C = GenCfg<T, N>;
  constexpr int NP = C::NP, NQ = C::NQ, NF = C::NF, NC = C::NC, NT = C::NT;
  __shared__ float s_q[4][NP];
  __shared__ float s_r[4][NP];
  __shared__ float s_F[NF][4][NQ];
  __shared__ float s_w[7][T == DG_WEDGE ? NC : (T == DG_PYR ? NP : 3 * NP / 7 + 1)];
  __shared__ float s_e[12];
  __shared__ int s_code[NF];

  const int tid = threadIdx.x;
  const int64_t e = A.elist ? (int64_t)A.elist[blockIdx.x] : (int64_t)blockIdx.x;
  const int64_t base = A.dof_off + e * NP;
  for (int x = tid; x < 4 * NP; x += NT) s_q[x / NP][x % NP] = A.q[(x / NP) * A.ndof + base + x % NP];
  if (tid < NF) s_code[tid] = A.code[A.side_off + e * NF + tid];
  if (T == DG_TET && tid < 12) s_e[tid] = A.geo[e * 12 + tid];
  __syncthreads();
  const float c2 = A.c2[e];

  if (MODE != MODE_TRACE) {
    // ---------------------------------------------------------------- volume
    if (T == DG_TET) {
      // Alg. tet_vol with constant metrics: -div u = -sum_a D^a (sum_d G_ad u_d), -c^2 grad p
      float* W = &s_w[0][0];
      for (int x = tid; x < 3 * NP; x += NT) {
        int a = x / NP, m = x % NP;
        W[x] = s_e[3 * a] * s_q[1][m] + s_e[3 * a + 1] * s_q[2][m] + s_e[3 * a + 2] * s_q[3][m];
      }
      __syncthreads();
      for (int n = tid; n < NP; n += NT) {
        float div = 0.f, dp[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < 3; ++a) {
          const float* DT = A.ops + a * NP * NP;
          float s1 = 0.f, s2 = 0.f;
          for (int m = 0; m < NP; ++m) {
            float dv = DT[m * NP + n];
            s1 += dv * W[a * NP + m];
            s2 += dv * s_q[0][m];
          }
          div += s1;
          dp[a] = s2;
        }
        s_r[0][n] = -div;
        for (int d = 0; d < 3; ++d)
          s_r[1 + d][n] = -c2 * (s_e[d] * dp[0] + s_e[3 + d] * dp[1] + s_e[6 + d] * dp[2]);
      }
    } else if (T == DG_PYR) {
      // Alg. pyr_vol (skew): u^a_m = J_m sum_d G_ad(m) u_d(m); p-eq (1/J) sum_a (D^a)^T u^a;
      // u-eq -c^2 sum_a G_ad (D^a p)  (J cancels with M^{-1} = 1/J)
      const float* geo = A.geo + e * NP * 10;
      for (int x = tid; x < 3 * NP; x += NT) {
        int a = x / NP, m = x % NP;
        const float* g = geo + m * 10;
        s_w[a][m] = g[9] * (g[3 * a] * s_q[1][m] + g[3 * a + 1] * s_q[2][m] + g[3 * a + 2] * s_q[3][m]);
      }
      __syncthreads();
      for (int n = tid; n < NP; n += NT) {
        const float* g = geo + n * 10;
        float pint = 0.f, dp[3];
        for (int a = 0; a < 3; ++a) {
          const float* D = A.ops + a * NP * NP;            // D[m][n] = D^a_{mn}
          const float* DT = A.ops + (3 + a) * NP * NP;     // DT[m][n] = D^a_{nm}
          float s1 = 0.f, s2 = 0.f;
          for (int m = 0; m < NP; ++m) {
            s1 += D[m * NP + n] * s_w[a][m];
            s2 += DT[m * NP + n] * s_q[0][m];
          }
          pint += s1;
          dp[a] = s2;
        }
        s_r[0][n] = pint / g[9];
        for (int d = 0; d < 3; ++d) s_r[1 + d][n] = -c2 * (g[d] * dp[0] + g[3 + d] * dp[1] + g[6 + d] * dp[2]);
      }
    } else {
      // Alg. wedge_vol1/2 (LSC-DG skew form) at the (N+1)^3 cubature points, M = I
      const float* V = A.ops;                              // [NC][NP]
      const float* VT = A.ops + 4 * NC * NP;               // [NP][NC]
      const float* wq = A.ops + 8 * NC * NP;
      const float* geo = A.geo + e * NC * 12;
      for (int q = tid; q < NC; q += NT) {
        float P = 0.f, Pa[3] = {0.f, 0.f, 0.f}, U[3] = {0.f, 0.f, 0.f};
        for (int m = 0; m < NP; ++m) {
          float v = VT[m * NC + q];
          P += v * s_q[0][m];
          U[0] += v * s_q[1][m];
          U[1] += v * s_q[2][m];
          U[2] += v * s_q[3][m];
#pragma unroll
          for (int a = 0; a < 3; ++a) Pa[a] += VT[(1 + a) * NC * NP + m * NC + q] * s_q[0][m];
        }
        const float* g = geo + q * 12;
        const float w = wq[q];
        float UJ = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float Ad = g[d] * Pa[0] + g[3 + d] * Pa[1] + g[6 + d] * Pa[2] - P * g[9 + d];
          s_w[d][q] = w * Ad;
          UJ += U[d] * g[9 + d];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) s_w[3 + a][q] = w * (g[3 * a] * U[0] + g[3 * a + 1] * U[1] + g[3 * a + 2] * U[2]);
        s_w[6][q] = w * UJ;
      }
      __syncthreads();
      for (int n = tid; n < NP; n += NT) {
        float up[3] = {0.f, 0.f, 0.f}, pp = 0.f;
        for (int q = 0; q < NC; ++q) {
          float v = V[q * NP + n];
          up[0] += v * s_w[0][q];
          up[1] += v * s_w[1][q];
          up[2] += v * s_w[2][q];
          pp += V[(1) * NC * NP + q * NP + n] * s_w[3][q] + V[(2) * NC * NP + q * NP + n] * s_w[4][q] +
                V[(3) * NC * NP + q * NP + n] * s_w[5][q] - v * s_w[6][q];
        }
        s_r[0][n] = pp;
        for (int d = 0; d < 3; ++d) s_r[1 + d][n] = -c2 * up[d];
      }
    }
    // ---------------------------------------------------------------- face fluxes
    for (int fq = tid; fq < NF * NQ; fq += NT) {
      const int f = fq / NQ, qq = fq % NQ;
      const int64_t gs = A.side_off + e * NF + f;
      const int c = s_code[f];
      const float* Tt = A.Tt + ((size_t)(f * NCODES + c) * NP) * NQ;
      float tr[4] = {0.f, 0.f, 0.f, 0.f};
      for (int m = 0; m < NP; ++m) {
        float v = Tt[m * NQ + qq];
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) tr[fl] += v * s_q[fl][m];
      }
      const int64_t sp = (e * NF + f) * NQ + qq;
      if (T == DG_WEDGE) {
        float is = A.sisq[sp];
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) tr[fl] *= is;
      }
      const float4 sg = A.sgeo[sp];
      const float unm = sg.x * tr[1] + sg.y * tr[2] + sg.z * tr[3];
      const int nb = A.nbr[gs];
      float P = 0.f, UN = 0.f;
      if (nb >= 0) {
        P = A.tin[gs * NQ + qq];
        UN = A.tin[A.plane + gs * NQ + qq];
      }
      const float tp = A.tau_scale * A.tau[gs], tu = A.tau_scale / A.tau[gs];
      float fp, fu;
      flux(nb < 0, tr[0], unm, P, UN, tp, tu, T != DG_TET && A.skew, fp, fu);
      s_F[f][0][qq] = sg.w * fp;
      s_F[f][1][qq] = sg.w * fu * sg.x;
      s_F[f][2][qq] = sg.w * fu * sg.y;
      s_F[f][3][qq] = sg.w * fu * sg.z;
    }
    __syncthreads();
    // ---------------------------------------------------------------- lift, M^{-1}, update
    for (int n = tid; n < NP; n += NT) {
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      for (int f = 0; f < NF; ++f) {
        const float* L = A.L + ((size_t)(f * NCODES + s_code[f]) * NQ) * NP;
        for (int qq = 0; qq < NQ; ++qq) {
          float l = L[qq * NP + n];
#pragma unroll
          for (int fl = 0; fl < 4; ++fl) sum[fl] += l * s_F[f][fl][qq];
        }
      }
      float iM = 1.f;
      if (T == DG_TET) iM = 1.f / s_e[9];
      if (T == DG_PYR) iM = 1.f / A.geo[(e * NP + n) * 10 + 9];
      float r[4];
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) r[fl] = s_r[fl][n] + (fl == 0 ? 1.f : c2) * iM * sum[fl];
      if (MODE == MODE_RHS) {
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) A.rhs[fl * A.ndof + base + n] = r[fl];
      } else {
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
          const int64_t id = fl * A.ndof + base + n;
          float rr = A.a * A.res[id] + A.dt * r[fl];
          float qn = s_q[fl][n] + A.b * rr;
          A.res[id] = rr;
          A.qout[id] = qn;
          s_r[fl][n] = qn;
        }
      }
    }
    if (MODE == MODE_STAGE) {
      __syncthreads();
      for (int x = tid; x < 4 * NP; x += NT) s_q[x / NP][x % NP] = s_r[x / NP][x % NP];
    }
  }
  if (MODE == MODE_TRACE || MODE == MODE_STAGE) {
    __syncthreads();
    for (int fq = tid; fq < NF * NQ; fq += NT) {
      const int f = fq / NQ, qq = fq % NQ;
      const int64_t gs = A.side_off + e * NF + f;
      const int nb = A.nbr[gs];
      if (nb < 0) continue;
      const float* Tt = A.Tt + ((size_t)(f * NCODES + s_code[f]) * NP) * NQ;
      float tr[4] = {0.f, 0.f, 0.f, 0.f};
      for (int m = 0; m < NP; ++m) {
        float v = Tt[m * NQ + qq];
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) tr[fl] += v * s_q[fl][m];
      }
      const int64_t sp = (e * NF + f) * NQ + qq;
      if (T == DG_WEDGE) {
        float is = A.sisq[sp];
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) tr[fl] *= is;
      }
      const float4 sg = A.sgeo[sp];
      A.tout[(int64_t)nb * NQ + qq] = tr[0];
      A.tout[A.plane + (int64_t)nb * NQ + qq] = sg.x * tr[1] + sg.y * tr[2] + sg.z * tr[3];
    }
  }
}

// ============================================================================ energy
// E_K = 1/2 (p^T M p + (1/c^2) sum_d u_d^T M u_d), FP64, one block per element.
template <int T, int N>
__global__ void __launch_bounds__(128) energy_kernel(Args A, const float* mhat, double* acc) {
  constexpr int NP = T == DG_HEX ? (N + 1) * (N + 1) * (N + 1) : np_of(T, N);
  constexpr int n1 = N + 1;
  __shared__ double s_red[128];
  __shared__ float s_geo[24];
  const int64_t e = blockIdx.x;
  const int64_t base = A.dof_off + e * NP;
  const int tid = threadIdx.x;
  if (T == DG_HEX && tid < 24) s_geo[tid] = A.geo[e * 24 + tid];
  __syncthreads();
  const double ic2 = 1.0 / (double)A.c2[e];
  double loc = 0.0;
  for (int n = tid; n < NP; n += 128) {
    double qv[4];
    for (int f = 0; f < 4; ++f) qv[f] = A.q[f * A.ndof + base + n];
    double wsq = qv[0] * qv[0] + ic2 * (qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
    if (T == DG_HEX) {
      const float* hc = A.hexc;
      int i = n % n1, j = (n / n1) % n1, k = n / (n1 * n1);
      float xr[3], xs[3], xt[3], g0[3];
      hex_jac(s_geo, hc[n1 * n1 + 3 * n1 + i], hc[n1 * n1 + 3 * n1 + j], hc[n1 * n1 + 3 * n1 + k], xr, xs, xt);
      cross3(xs, xt, g0);
      double J = (double)xr[0] * g0[0] + (double)xr[1] * g0[1] + (double)xr[2] * g0[2];
      double w = (double)hc[n1 * n1 + 2 * n1 + i] * hc[n1 * n1 + 2 * n1 + j] * hc[n1 * n1 + 2 * n1 + k];
      loc += w * J * wsq;
    } else if (T == DG_WEDGE) {
      loc += wsq;
    } else if (T == DG_PYR) {
      loc += (double)A.geo[(e * NP + n) * 10 + 9] * wsq;
    } else {
      double J = A.geo[e * 12 + 9];
      double s = 0.0;
      for (int m = 0; m < NP; ++m) {
        double mm = mhat[n * NP + m];
        double o = (double)A.q[base + m] * qv[0];
        for (int f = 1; f < 4; ++f) o += ic2 * (double)A.q[f * A.ndof + base + m] * qv[f];
        s += mm * o;
      }
      loc += J * s;
    }
  }
  s_red[tid] = loc;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (tid < s) s_red[tid] += s_red[tid + s];
    __syncthreads();
  }
  if (tid == 0) atomicAdd(acc, 0.5 * s_red[0]);
}

// ============================================================================ multi-rate AB3 update
// q_out = q_in + h0*r0 + h1*r1 + h2*r2 on the DOFs of the listed elements (all four fields).
__global__ void __launch_bounds__(256) ab_update_kernel(const int* elist, int K, int Np, int64_t dof_off,
                                                        int64_t ndof, const float* qin, float* qout,
                                                        const float* r0, const float* r1, const float* r2,
                                                        float h0, float h1, float h2) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (int64_t)K * Np) return;
  const int64_t li = x / Np;
  const int n = (int)(x % Np);
  const int64_t e = elist ? (int64_t)elist[li] : li;
  const int64_t id = dof_off + e * Np + n;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int64_t k = f * ndof + id;
    qout[k] = qin[k] + h0 * r0[k] + h1 * r1[k] + h2 * r2[k];
  }
}

// ============================================================================ launchers
static Args make_args(dg_mesh* m, int t) {
  const TypeDev& td = m->td[t];
  Args A{};
  A.plane = m->nsides * (int64_t)m->nq;
  A.geo = td.geo;
  A.sgeo = td.sgeo;
  A.sisq = td.sisq;
  A.c2 = td.c2;
  A.Tt = td.Tt;
  A.L = td.L;
  A.ops = td.ops;
  A.nbr = m->side_nbr;
  A.code = m->side_code;
  A.tau = m->side_tau;
  A.hexc = m->hexc;
  A.perm = m->hexperm;
  A.sgeo2 = td.sgeo2;
  A.sisq2 = td.sisq2;
  A.ops2 = td.ops2;
  A.iops2 = td.iops2;
  A.K = td.K;
  A.elist = nullptr;
  A.dof_off = td.dof_off;
  A.ndof = m->ndof;
  A.side_off = td.side_off;
  A.tau_scale = (float)m->tau_scale;
  A.skew = 1;
  return A;
}

template <int N, int MODE>
static void launch_hex_n(const Args& A, cudaStream_t s) {
  using C = HexCfg<N>;
  if (A.K == 0) return;
  dim3 grid((A.K + C::EPB - 1) / C::EPB);
  hex_kernel<N, MODE><<<grid, C::NT, 0, s>>>(A);
}

template <int T, int N, int MODE>
static void launch_gen_n(const Args& A, cudaStream_t s) {
  if (A.K == 0) return;
  gen_kernel<T, N, MODE><<<A.K, 128, 0, s>>>(A);
}

template <int MODE>
bool launch_gen2(int t, int N, const Args& A, cudaStream_t s);   // kernels_gen2.cu

// Event pair around one type's launch when dg_profile is on.
static int ev_take(dg_mesh* m) {
  if (m->ev_next == m->ev_pool.size()) {
    cudaEvent_t ev;
    cudaEventCreate(&ev);
    m->ev_pool.push_back(ev);
  }
  return (int)m->ev_next++;
}

template <int MODE>
static void launch_type(dg_mesh* m, const Args& A, int t) {
  if (A.K == 0) return;
  if (MODE >= MODE_MRC && m->N > 4) return;   // fused multi-rate kernels exist for N <= 4 only
  cudaStream_t s = m->stream;
  int e0 = -1;
  if (m->profiling) {
    e0 = ev_take(m);
    cudaEventRecord(m->ev_pool[e0], s);
  }
  switch (m->N) {
#define DG_CASE(NN)                                                   \
  case NN:                                                            \
    if (t == DG_HEX) { if (NN <= 4) launch_hexw_n<(NN <= 4 ? NN : 4), MODE>(A, s); else launch_hex_n<NN, (MODE > 2 ? 1 : MODE)>(A, s); } \
    else if (launch_gen2<MODE>(t, NN, A, s)) {}                       \
    else if (t == DG_WEDGE) launch_gen_n<DG_WEDGE, NN, (MODE > 2 ? 1 : MODE)>(A, s);   \
    else if (t == DG_PYR) launch_gen_n<DG_PYR, NN, (MODE > 2 ? 1 : MODE)>(A, s);       \
    else launch_gen_n<DG_TET, NN, (MODE > 2 ? 1 : MODE)>(A, s);                        \
    break;
    DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6)
#undef DG_CASE
    default: break;
  }
  m->launches[t] += 1;
  if (m->profiling) {
    int e1 = ev_take(m);
    cudaEventRecord(m->ev_pool[e1], s);
    m->ev_used[t].push_back({e0, e1});
  }
}

template <int MODE>
static void launch_all(dg_mesh* m, Args* A, const Sel* sel = nullptr) {
  for (int t = 0; t < 4; ++t) {
    if (sel) {
      A[t].elist = sel->list[t];
      A[t].K = (int)sel->count[t];
    }
    launch_type<MODE>(m, A[t], t);
  }
}

cudaError_t launch_trace_sel(dg_mesh* m, const float* q, float* tout, const Sel& sel) {
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
    A[t].tout = tout;
  }
  launch_all<MODE_TRACE>(m, A, &sel);
  return cudaGetLastError();
}

cudaError_t launch_rhs_sel(dg_mesh* m, const float* q, const float* tin, float* rhs, const Sel& sel) {
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
    A[t].tin = tin;
    A[t].rhs = rhs;
  }
  launch_all<MODE_RHS>(m, A, &sel);
  return cudaGetLastError();
}

cudaError_t launch_ab(dg_mesh* m, const Sel& sel, const float* qin, float* qout, const float* r0,
                      const float* r1, const float* r2, float h0, float h1, float h2) {
  for (int t = 0; t < 4; ++t) {
    const int64_t n = sel.count[t] * (int64_t)m->td[t].Np;
    if (n == 0) continue;
    ab_update_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(
        sel.list[t], (int)sel.count[t], m->td[t].Np, m->td[t].dof_off, m->ndof, qin, qout, r0, r1, r2, h0, h1, h2);
  }
  return cudaGetLastError();
}

cudaError_t launch_mr(dg_mesh* m, bool coarse, const Sel& sel, float* q, const float* tin, float* tout,
                      float* tout2, float* hw, const float* h1, const float* h2, const float c[3],
                      const float p[3]) {
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
    A[t].qout = q;
    A[t].tin = tin;
    A[t].tout = tout;
    A[t].tout2 = tout2;
    A[t].hw = hw;
    A[t].h1 = h1;
    A[t].h2 = h2;
    A[t].ab0 = c[0]; A[t].ab1 = c[1]; A[t].ab2 = c[2];
    A[t].pr0 = p[0]; A[t].pr1 = p[1]; A[t].pr2 = p[2];
  }
  if (coarse) launch_all<MODE_MRC>(m, A, &sel);
  else launch_all<MODE_MRF>(m, A, &sel);
  return cudaGetLastError();
}

cudaError_t launch_trace(dg_mesh* m, const float* q, float* tout) {
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
    A[t].tout = tout;
  }
  launch_all<MODE_TRACE>(m, A);
  return cudaGetLastError();
}

cudaError_t launch_rhs(dg_mesh* m, const float* q, const float* tin, float* rhs) {
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
    A[t].tin = tin;
    A[t].rhs = rhs;
  }
  launch_all<MODE_RHS>(m, A);
  return cudaGetLastError();
}

cudaError_t launch_stage(dg_mesh* m, float* q, float* res, const float* tin, float* tout, float a,
                         float b, float dt) {
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
    A[t].qout = q;
    A[t].res = res;
    A[t].tin = tin;
    A[t].tout = tout;
    A[t].a = a;
    A[t].b = b;
    A[t].dt = dt;
  }
  launch_all<MODE_STAGE>(m, A);
  return cudaGetLastError();
}

cudaError_t launch_energy(dg_mesh* m, const float* q, double* acc) {
  cudaStream_t s = m->stream;
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
  }
  switch (m->N) {
#define DG_CASE(NN)                                                                                  \
  case NN:                                                                                           \
    if (A[0].K) energy_kernel<DG_HEX, NN><<<A[0].K, 128, 0, s>>>(A[0], nullptr, acc);                \
    if (A[1].K) energy_kernel<DG_WEDGE, NN><<<A[1].K, 128, 0, s>>>(A[1], nullptr, acc);              \
    if (A[2].K) energy_kernel<DG_PYR, NN><<<A[2].K, 128, 0, s>>>(A[2], nullptr, acc);                \
    if (A[3].K) energy_kernel<DG_TET, NN><<<A[3].K, 128, 0, s>>>(A[3], m->tet_mhat_dev, acc);        \
    break;
    DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6)
#undef DG_CASE
    default: break;
  }
  return cudaGetLastError();
}

}  // namespace dgk
