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
  // resident blocks per SM the register allocation aims at (measured best: N = 5..7: 8, 5, 3; one
  // more block at N = 7 spills enough to lose).  The launchers run this kernel at N = 5 only; N = 6..9
  // run the column kernel hexc_kernel below.
  static constexpr int MINB = N >= 8 ? 1 : N == 7 ? 3 : N == 6 ? 5 : N == 5 ? 8 : 1;
};

// a x + y on the four fields as two packed FP32 pair FMAs (round to nearest, the same values as
// four fmaf)
__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
  const float2 aa = make_float2(a, a);
  const float2 lo = __ffma2_rn(aa, make_float2(x.x, x.y), make_float2(y.x, y.y));
  const float2 hi = __ffma2_rn(aa, make_float2(x.z, x.w), make_float2(y.z, y.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

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
__global__ void __launch_bounds__(HexCfg<N>::NT, HexCfg<N>::MINB) hex_kernel(Args A) {
  using C = HexCfg<N>;
  constexpr int n1 = C::n1, NP = C::NP, NQ = C::NQ, EPB = C::EPB, TPE = C::TPE;
  __shared__ float4 s_q4[EPB][NP];   // (p, u, v, w) per node
  __shared__ float s_geo[EPB][24];
  __shared__ float4 s_F4[EPB][6][NQ];   // J^s-weighted fluxes (p, u, v, w) per face point
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
    s_q4[le][tid] = make_float4(A.q[base + tid], A.q[A.ndof + base + tid], A.q[2 * A.ndof + base + tid],
                                A.q[3 * A.ndof + base + tid]);
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
      float4 dr4 = make_float4(0.f, 0.f, 0.f, 0.f), ds4 = dr4, dt4 = dr4;
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        dr4 = f4fma(s_D[i * n1 + m], s_q4[le][m + n1 * (j + n1 * k)], dr4);
        ds4 = f4fma(s_D[j * n1 + m], s_q4[le][i + n1 * (m + n1 * k)], ds4);
        dt4 = f4fma(s_D[k * n1 + m], s_q4[le][i + n1 * (j + n1 * m)], dt4);
      }
      const float dr[4] = {dr4.x, dr4.y, dr4.z, dr4.w}, ds[4] = {ds4.x, ds4.y, ds4.z, ds4.w};
      const float dt[4] = {dt4.x, dt4.y, dt4.z, dt4.w};
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
      float4 tr4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        const int id = ax == 0 ? m + n1 * (a + n1 * b) : ax == 1 ? a + n1 * (m + n1 * b) : a + n1 * (b + n1 * m);
        tr4 = f4fma(V[m], s_q4[le][id], tr4);
      }
      const float tr[4] = {tr4.x, tr4.y, tr4.z, tr4.w};
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
      s_F4[le][f][lp] = make_float4(wgt * fp, wgt * fu * nv[0], wgt * fu * nv[1], wgt * fu * nv[2]);
      s_n[le][f][0][lp] = nv[0];
      s_n[le][f][1][lp] = nv[1];
      s_n[le][f][2][lp] = nv[2];
    }
    __syncthreads();
    // ---- lift, Alg. hex_surf: M^{-1} w w J^s l(+-1) flux
    if (valid && tid < NP) {
      const float iM = 1.f / (s_w[i] * s_w[j] * s_w[k] * Jn);
      const int jk = j + n1 * k, ik = i + n1 * k, ij = i + n1 * j;
      float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
      sum = f4fma(s_Vm[i], s_F4[le][0][jk], sum);
      sum = f4fma(s_Vp[i], s_F4[le][1][jk], sum);
      sum = f4fma(s_Vm[j], s_F4[le][2][ik], sum);
      sum = f4fma(s_Vp[j], s_F4[le][3][ik], sum);
      sum = f4fma(s_Vm[k], s_F4[le][4][ij], sum);
      sum = f4fma(s_Vp[k], s_F4[le][5][ij], sum);
      const float sf[4] = {sum.x, sum.y, sum.z, sum.w};
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) rhs[fl] += (fl == 0 ? 1.f : c2) * iM * sf[fl];
      if (e == A.src_e) rhs[0] += A.src_s * A.src_g[tid];   // point source on p
      if (MODE == MODE_RHS) {
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) A.rhs[fl * A.ndof + base + tid] = rhs[fl];
      } else {
        const float4 qo = s_q4[le][tid];
        const float qv[4] = {qo.x, qo.y, qo.z, qo.w};
        const float dte = A.dtE ? A.dtE[e] : A.dt;
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
          const int64_t id = fl * A.ndof + base + tid;
          float r = A.a * A.res[id] + dte * rhs[fl];
          float qn = qv[fl] + A.b * r;
          A.res[id] = r;
          A.qout[id] = qn;
          rhs[fl] = qn;
        }
      }
    }
    if (MODE == MODE_STAGE) {
      __syncthreads();
      if (valid && tid < NP) {
        s_q4[le][tid] = make_float4(rhs[0], rhs[1], rhs[2], rhs[3]);
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
      const int64_t dst = nb >= 0 ? (int64_t)nb : ((MODE == MODE_TRACE && A.wall_self) ? gs : -1);
      if (dst < 0) continue;
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
      float4 tr4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        const int id = ax == 0 ? m + n1 * (a + n1 * b) : ax == 1 ? a + n1 * (m + n1 * b) : a + n1 * (b + n1 * m);
        tr4 = f4fma(V[m], s_q4[le][id], tr4);
      }
      const float tr[4] = {tr4.x, tr4.y, tr4.z, tr4.w};
      const int cidx = s_perm[A.code[gs] * NQ + lp];
      A.tout[dst * NQ + cidx] = tr[0];
      A.tout[A.plane + dst * NQ + cidx] = nv[0] * tr[1] + nv[1] * tr[2] + nv[2] * tr[3];
    }
  }
}

// ============================================================================ hexahedra, warp per element
// For N <= 4: a warp owns EPW = 32 / (N+1)^2 elements; lane (i,j) of an element keeps
// the column (i,j,0..N) of all four fields in registers.  t-derivatives and the
// t-face traces come from registers; r/s-derivatives and r/s-face traces read the
// element's nodes as float4 (p,u,v,w) from shared memory.  Only warp-level
// synchronisation after the start of the block.
// per node set (0 = GL, 1 = GLL) and N: D1[n1*n1] (row = node), Vm[n1], Vp[n1], w[n1], r[n1], 1/w[n1]
__constant__ float c_hexw[2][5][64];

cudaError_t upload_hex_constants(int N, bool sem, const float* hc, int count) {
  if (N < 1 || N > 4 || count > 64) return cudaSuccess;
  return cudaMemcpyToSymbol(c_hexw, hc, count * sizeof(float), ((sem ? 5 : 0) + N) * 64 * sizeof(float));
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
  const float inv = sg * __frcp_rn(Js);
  nv[0] *= inv;
  nv[1] *= inv;
  nv[2] *= inv;
}

// ---------------------------------------------------------------------------- pipelined hex kernel
// Persistent warp-per-element kernel for N <= 4.  Lane (i,j) owns the node column (i,j,:).
// While a warp computes element g, the copies of the next element's operands into shared
// memory are in flight:
//   main(g')  node values and side data (geometry coefficients, neighbours, codes, tau, c^2);
//             double-buffered, issued at the start of element g
//   in(g')    the two inbox planes (p, u.n) of its six faces; issued after g's flux phase
//   aux(g')   the residual (LSRK stage) or the two history slots (multi-rate); issued after
//             g's update
// so every global read of the element loop is a shared-memory read of data requested one
// element earlier.  Writes (state, residual / history, traces) go straight to global memory.
// Two copy engines:
//   TMA = false  4-byte cp.async by every lane (any N <= 4, any buffers)
//   TMA = true   N = 4, EPW = 1: one lane issues 1D bulk tensor copies (cp.async.bulk.tensor)
//                of whole field slices into planar staging buffers, completing on per-warp
//                mbarriers; the start coordinate of each slice is rounded down to 16 bytes
//                and the slice read from the remainder (boxes of 128 / 160 floats cover the
//                125-node field slice / the 150-point inbox plane plus that remainder; reads
//                past the end of an array are zero-filled by the copy engine).
//                Side data still uses cp.async.
// Waits on mbarriers are bounded (~1 s of SM clock); on a timeout the warp sets bit 0 of the
// device error word, waits (bounded) for its own copies in flight and leaves the loop.
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory");
}
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* map, int x, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_u32(bar))
      : "memory");
}
// Wait for the completion of phase `parity` of an mbarrier; false after ~2^31 SM clocks.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1LL << 31)) return false;
  }
}

// 3 resident blocks of 4 warps per SM: the register budget that needs no spills
#ifndef DG_HEXP_MINB
#define DG_HEXP_MINB 3
#endif
template <int N, int MODE, bool TMA>
struct HexP {
  static constexpr int n1 = N + 1, NP = n1 * n1 * n1, NQ = n1 * n1;
  static constexpr int EPW = 32 / NQ, WPB = 4;
  static constexpr int NAUX = MODE == MODE_STAGE ? 1 : (MODE == MODE_MRC || MODE == MODE_MRF) ? 2 : 0;
  static constexpr int SD = 44;   // side data words: geometry [24], nbr [6], code [6], tau [6], c2
  static constexpr int R128(int x) { return (x + 127) / 128 * 128; }
  // cp.async layout (bytes, per warp): q [2][EPW][NP] float4, aux [EPW][NAUX][NP] float4,
  // F [EPW][4][NQ] float4, Nrm [EPW][6][NQ] float4, in [EPW][2][6 NQ] float, sd [2][EPW][SD]
  static constexpr int C_AUX = 2 * EPW * NP * 16;
  static constexpr int C_F = C_AUX + EPW * NAUX * NP * 16;
  static constexpr int C_N = C_F + EPW * 4 * NQ * 16;
  static constexpr int C_IN = C_N + EPW * 6 * NQ * 16;
  static constexpr int C_SD = C_IN + EPW * 12 * NQ * 4;
  static constexpr int C_PW = ((C_SD + 2 * EPW * SD * 4 + 15) / 16) * 16;
  // TMA layout (EPW = 1): planar staging qp [2][4][QB], node-major copy q4 [NP] float4,
  // aux [NAUX][4][QB], in [2][IB], F, Nrm, sd [2][SD], 4 mbarriers (main[2], in, aux)
  static constexpr int QB = 128, IB = 160;
  static constexpr int T_Q4 = 2 * 4 * QB * 4;
  static constexpr int T_AUX = T_Q4 + R128(NP * 16);
  static constexpr int T_IN = T_AUX + NAUX * 4 * QB * 4;
  static constexpr int T_F = T_IN + 2 * IB * 4;
  static constexpr int T_N = T_F + 4 * NQ * 16;
  static constexpr int T_SD = T_N + 6 * NQ * 16;
  static constexpr int T_BAR = ((T_SD + 2 * SD * 4 + 7) / 8) * 8;
  static constexpr int T_PW = R128(T_BAR + 4 * 8);
  static constexpr int PW = TMA ? T_PW : C_PW;
  static constexpr int PERM_B = R128(8 * NQ * 4);
  static constexpr int SMEM = PERM_B + WPB * PW;
  static_assert(!TMA || (EPW == 1 && NP + 3 <= QB && 6 * NQ + 3 <= IB && NAUX > 0), "TMA path: N = 4 updates");
};

// 1D tensor maps of the arrays the TMA path reads, with the float offsets of the kernel's
// pointers inside them
struct HexMaps {
  CUtensorMap q, a0, a1, in;
  long long qoff, a0off, a1off, inoff;
};

// SEM = true: GLL nodes, the faces carry the end nodes; traces are node values and the lift only
// touches the boundary nodes (the cost advantage of the SEM hexahedron, Sec. 2.1.1)
template <int N, int MODE, bool TMA, bool SEM>
__global__ void __launch_bounds__(128, DG_HEXP_MINB) hexw_kernel(Args A, const __grid_constant__ HexMaps M) {
  using H = HexP<N, MODE, TMA>;
  constexpr int n1 = H::n1, NP = H::NP, NQ = H::NQ, EPW = H::EPW, WPB = H::WPB, SD = H::SD;
  constexpr int QB = H::QB, IB = H::IB;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int* s_perm = reinterpret_cast<int*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* pw = smem_raw + H::PERM_B + w * H::PW;
  const int sub = lane / NQ, col = lane % NQ;
  const int i = col % n1, j = col / n1;
  const int su = sub < EPW ? sub : 0;
  // cp.async layout
  auto SQ = [&](int b) { return reinterpret_cast<float4*>(pw) + (b * EPW + su) * NP; };
  float4* c_aux = reinterpret_cast<float4*>(pw + H::C_AUX) + su * H::NAUX * NP;
  float* c_in = reinterpret_cast<float*>(pw + H::C_IN) + su * 12 * NQ;
  // TMA layout
  float* t_qp = reinterpret_cast<float*>(pw);
  float4* t_q4 = reinterpret_cast<float4*>(pw + H::T_Q4);
  float* t_aux = reinterpret_cast<float*>(pw + H::T_AUX);
  float* t_in = reinterpret_cast<float*>(pw + H::T_IN);
  uint64_t* bar = reinterpret_cast<uint64_t*>(pw + H::T_BAR);
  // both
  float4* s_F = reinterpret_cast<float4*>(pw + (TMA ? H::T_F : H::C_F)) + su * 4 * NQ;
  float4* s_N = reinterpret_cast<float4*>(pw + (TMA ? H::T_N : H::C_N)) + su * 6 * NQ;
  auto SDp = [&](int b) { return reinterpret_cast<float*>(pw + (TMA ? H::T_SD : H::C_SD)) + (b * EPW + su) * SD; };

  const float* Dm = c_hexw[SEM ? 1 : 0][N];
  const float* Vm = Dm + n1 * n1;
  const float* Vp = Vm + n1;
  const float* W1 = Vp + n1;
  const float* R1 = W1 + n1;
  const float* iW = R1 + n1;

  for (int x = threadIdx.x; x < 8 * NQ; x += blockDim.x) s_perm[x] = A.perm[x];
  if (TMA && lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) mbar_init(bar + k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  // element of this lane in group g (or -1)
  auto elem = [&](int g) -> int {
    const int li = (g * WPB + w) * EPW + sub;
    if (sub >= EPW || li >= A.K) return -1;
    return A.elist ? A.elist[li] : li;
  };
  unsigned pend = 0;    // TMA: barriers with copies in flight (bit k = bar[k])
  unsigned phase = 0;   // TMA: parity of the next completion of each barrier
  // start coordinate of a TMA slice, rounded down to 16 bytes
  auto x16 = [](long long x) { return (int)(x & ~3LL); };
  auto stage_main = [&](int b, int e) {
    if (e >= 0) {
      if (TMA) {
        if (lane == 0) {
          const long long x = M.qoff + A.dof_off + (long long)e * NP;
          mbar_expect_tx(bar + b, 4 * QB * 4);
#pragma unroll
          for (int f = 0; f < 4; ++f) tma_load_1d(t_qp + (b * 4 + f) * QB, &M.q, x16(x + f * A.ndof), bar + b);
        }
      } else {
        const float* qs = A.q + A.dof_off + (int64_t)e * NP + col;
        float* dq = reinterpret_cast<float*>(SQ(b)) + 4 * col;
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) cp_async4(dq + 4 * NQ * k + f, qs + f * A.ndof + NQ * k);
      }
      const int64_t gs0 = A.side_off + (int64_t)e * 6;
      float* ds = SDp(b);
      for (int x = col; x < SD - 1; x += NQ) {
        const void* src = x < 24   ? static_cast<const void*>(A.geo + (int64_t)e * 24 + x)
                          : x < 30 ? static_cast<const void*>(A.nbr + gs0 + (x - 24))
                          : x < 36 ? static_cast<const void*>(A.code + gs0 + (x - 30))
                          : x < 42 ? static_cast<const void*>(A.tau + gs0 + (x - 36))
                                   : static_cast<const void*>(A.c2 + e);
        cp_async4(ds + x, src);
      }
      if (TMA) pend |= 1u << b;
    }
    cp_async_commit();
  };
  auto stage_in = [&](int e) {
    if (MODE != MODE_TRACE && e >= 0) {
      const long long x = (A.side_off + (long long)e * 6) * NQ;
      if (TMA) {
        if (lane == 0) {
          mbar_expect_tx(bar + 2, 2 * IB * 4);
          tma_load_1d(t_in, &M.in, x16(M.inoff + x), bar + 2);
          tma_load_1d(t_in + IB, &M.in, x16(M.inoff + A.plane + x), bar + 2);
        }
        pend |= 4u;
      } else {
        const float* src = A.tin + x;
        for (int y = col; y < 12 * NQ; y += NQ) cp_async4(c_in + y, src + (y >= 6 * NQ ? A.plane - 6 * NQ : 0) + y);
      }
    }
    cp_async_commit();
  };
  auto stage_aux = [&](int e) {
    if (H::NAUX > 0 && e >= 0) {
      if (TMA) {
        if (lane == 0) {
          const long long x = A.dof_off + (long long)e * NP;
          mbar_expect_tx(bar + 3, H::NAUX * 4 * QB * 4);
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            tma_load_1d(t_aux + f * QB, &M.a0, x16(M.a0off + x + f * A.ndof), bar + 3);
            if (H::NAUX > 1) tma_load_1d(t_aux + (4 + f) * QB, &M.a1, x16(M.a1off + x + f * A.ndof), bar + 3);
          }
        }
        pend |= 8u;
      } else {
        const float* s0 = (MODE == MODE_STAGE ? A.res : A.h1) + A.dof_off + (int64_t)e * NP + col;
        const float* s1 = A.h2 + A.dof_off + (int64_t)e * NP + col;
        float* d = reinterpret_cast<float*>(c_aux) + 4 * col;
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            cp_async4(d + 4 * NQ * k + f, s0 + f * A.ndof + NQ * k);
            if (H::NAUX > 1) cp_async4(d + 4 * NP + 4 * NQ * k + f, s1 + f * A.ndof + NQ * k);
          }
      }
    }
    cp_async_commit();
  };
  // TMA: wait for barrier k (warp-uniform); false on a timeout
  auto wait_bar = [&](int k) -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar + k, (phase >> k) & 1u));
    if (ok) {
      phase ^= 1u << k;
      pend &= ~(1u << k);
    }
    return ok;
  };

  int g = blockIdx.x;
  const int gstride = gridDim.x;
  // TMA (EPW = 1): the warp's element is lane 0's
  auto welem = [&](int e) { return TMA ? __shfl_sync(0xffffffffu, e, 0) : e; };
  int e_c = elem(g), e_n = elem(g + gstride);
  stage_main(0, welem(e_c));
  stage_in(welem(e_c));
  stage_aux(welem(e_c));
  int b = 0;
  bool bail = false;
  for (; (g * WPB + w) * EPW < A.K; g += gstride, b ^= 1) {
    const int e_nn = elem(g + 2 * gstride);   // consumed one element later
    stage_main(b ^ 1, welem(e_n));
    cp_async_wait<2>();                       // main(g) and in(g) have landed
    if (TMA && !(wait_bar(b) && wait_bar(2))) {
      bail = true;
      break;
    }
    __syncwarp();
    const bool act = e_c >= 0;
    const int64_t e = act ? e_c : 0;
    const int64_t base = A.dof_off + e * NP;
    const float* g_ = SDp(b);
    const int* s_nb = reinterpret_cast<const int*>(g_ + 24);
    const int* s_code = reinterpret_cast<const int*>(g_ + 30);
    const float* s_tau = g_ + 36;
    const float c2 = act ? g_[42] : 0.f;
    float4* s_q = TMA ? t_q4 : SQ(b);
    float q[4][n1];
    if (TMA) {   // planar slices -> registers and the node-major copy
      int o[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) o[f] = (int)((M.qoff + base + f * A.ndof) & 3) + (b * 4 + f) * QB;
      if (act) {
#pragma unroll
        for (int k = 0; k < n1; ++k) {
#pragma unroll
          for (int f = 0; f < 4; ++f) q[f][k] = t_qp[o[f] + col + NQ * k];
          s_q[col + NQ * k] = make_float4(q[0][k], q[1][k], q[2][k], q[3][k]);
        }
      }
      __syncwarp();
    } else {
#pragma unroll
      for (int k = 0; k < n1; ++k) {
        const float4 v = s_q[col + NQ * k];
        q[0][k] = v.x;
        q[1][k] = v.y;
        q[2][k] = v.z;
        q[3][k] = v.w;
      }
    }
    float rhs[4][n1];
    float iJn[n1];   // 1/J at the column's nodes

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
        Ar[d] = g_[d] + g_[9 + d] * s;
        Br[d] = g_[12 + d] + g_[18 + d] * s;
        As[d] = g_[3 + d] + g_[9 + d] * r;
        Bs[d] = g_[15 + d] + g_[18 + d] * r;
        xt[d] = g_[6 + d] + g_[12 + d] * r + g_[15 + d] * s + g_[18 + d] * r * s;
      }
      float G0a[3], G0b[3], G1a[3], G1b[3], G2a[3], G2b[3], G2c[3], tmp[3];
      cross3(As, xt, G0a);
      cross3(Bs, xt, G0b);
      cross3(xt, Ar, G1a);
      cross3(xt, Br, G1b);
      cross3(Ar, As, G2a);
      cross3(Ar, Bs, G2b);
      cross3(Br, As, tmp);
      G2b[0] += tmp[0];
      G2b[1] += tmp[1];
      G2b[2] += tmp[2];
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
        const float iJ = __frcp_rn(J);
        iJn[k] = iJ;
        float4 dr = make_float4(0.f, 0.f, 0.f, 0.f), ds = dr;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          dr = f4fma(Dri[m], s_q[m + n1 * j + NQ * k], dr);
          ds = f4fma(Dsj[m], s_q[i + n1 * m + NQ * k], ds);
        }
        float4 dt4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int m = 0; m < n1; ++m) dt4 = f4fma(Dm[k * n1 + m], make_float4(q[0][m], q[1][m], q[2][m], q[3][m]), dt4);
        const float dt[4] = {dt4.x, dt4.y, dt4.z, dt4.w};
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
    float4 F45[2];
    if (MODE != MODE_TRACE && act) {
      // inbox offsets: TMA slices start at the 16-byte boundary below the element's first point
      int oi0 = 0, oi1 = 6 * NQ;
      const float* sin_ = c_in;
      if (TMA) {
        const long long x = (A.side_off + e * 6) * NQ;
        oi0 = (int)((M.inoff + x) & 3);
        oi1 = IB + (int)((M.inoff + A.plane + x) & 3);
        sin_ = t_in;
      }
      // ---- fluxes at this lane's point (a,b) = (i,j) of all six faces
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        float4 tm = make_float4(0.f, 0.f, 0.f, 0.f), tp = tm;
        auto node = [&](int m) {
          if (ax == 0) return s_q[m + n1 * i + NQ * j];
          if (ax == 1) return s_q[i + n1 * m + NQ * j];
          return make_float4(q[0][m], q[1][m], q[2][m], q[3][m]);
        };
        if constexpr (SEM) {
          tm = node(0);
          tp = node(N);
        } else {
#pragma unroll
          for (int m = 0; m < n1; ++m) {
            const float4 v = node(m);
            tm = f4fma(Vm[m], v, tm);
            tp = f4fma(Vp[m], v, tp);
          }
        }
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const int f = 2 * ax + sd;
          const float4 tr = sd ? tp : tm;
          float nv[3], Js;
          hexw_face_geom<N>(g_, R1, f, i, j, nv, Js);
          s_N[f * NQ + col] = make_float4(nv[0], nv[1], nv[2], Js);
          const float unm = nv[0] * tr.y + nv[1] * tr.z + nv[2] * tr.w;
          const int nb = s_nb[f];
          float P = 0.f, UN = 0.f;
          if (nb >= 0) {
            const int cidx = s_perm[s_code[f] * NQ + col];
            P = sin_[oi0 + f * NQ + cidx];
            UN = sin_[oi1 + f * NQ + cidx];
          }
          const float ta = s_tau[f];
          float fp, fu;
          flux(nb < 0, tr.x, unm, P, UN, A.tau_scale * ta, A.tau_scale * __frcp_rn(ta), false, fp, fu);
          const float wg = W1[i] * W1[j] * Js;
          const float4 Fv = make_float4(wg * fp, wg * fu * nv[0], wg * fu * nv[1], wg * fu * nv[2]);
          if (ax < 2) s_F[f * NQ + col] = Fv;
          else F45[sd] = Fv;
        }
      }
    }
    __syncwarp();
    stage_in(welem(e_n));   // the inbox buffer is free again
    if (MODE != MODE_TRACE) {
      if (act) {
        // ---- lift (Alg. hex_surf), M^{-1} = 1/(w w w J)
#pragma unroll
        for (int k = 0; k < n1; ++k) {
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
          if constexpr (SEM) {   // l_m(-1) = delta_{m0}, l_m(+1) = delta_{mN}
            if (i == 0) sum = f4fma(1.f, s_F[0 * NQ + j + n1 * k], sum);
            if (i == N) sum = f4fma(1.f, s_F[1 * NQ + j + n1 * k], sum);
            if (j == 0) sum = f4fma(1.f, s_F[2 * NQ + i + n1 * k], sum);
            if (j == N) sum = f4fma(1.f, s_F[3 * NQ + i + n1 * k], sum);
            if (k == 0) sum = f4fma(1.f, F45[0], sum);
            if (k == N) sum = f4fma(1.f, F45[1], sum);
          } else {
            const float4 F0 = s_F[0 * NQ + j + n1 * k], F1 = s_F[1 * NQ + j + n1 * k];
            const float4 F2 = s_F[2 * NQ + i + n1 * k], F3 = s_F[3 * NQ + i + n1 * k];
            sum = f4fma(Vm[i], F0, sum);
            sum = f4fma(Vp[i], F1, sum);
            sum = f4fma(Vm[j], F2, sum);
            sum = f4fma(Vp[j], F3, sum);
            sum = f4fma(Vm[k], F45[0], sum);
            sum = f4fma(Vp[k], F45[1], sum);
          }
          const float iM = iW[i] * iW[j] * iW[k] * iJn[k];
          rhs[0][k] += iM * sum.x;
          rhs[1][k] += c2 * iM * sum.y;
          rhs[2][k] += c2 * iM * sum.z;
          rhs[3][k] += c2 * iM * sum.w;
        }
        if ((MODE == MODE_RHS || MODE == MODE_STAGE) && e == A.src_e) {   // point source on p
#pragma unroll
          for (int k = 0; k < n1; ++k) rhs[0][k] += A.src_s * A.src_g[col + NQ * k];
        }
      }
      cp_async_wait<2>();   // aux(g) has landed
      if (TMA && H::NAUX > 0 && !wait_bar(3)) {
        bail = true;
        break;
      }
      __syncwarp();
      // aux value of field f, node (col, k), slot a
      int oa[2][4];
      if (TMA) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          oa[0][f] = (int)((M.a0off + base + f * A.ndof) & 3) + f * QB + col;
          oa[1][f] = (int)((M.a1off + base + f * A.ndof) & 3) + (4 + f) * QB + col;
        }
      }
      auto auxv = [&](int a, int f, int k) -> float {
        if (TMA) return t_aux[oa[a][f] + NQ * k];
        const float* c = reinterpret_cast<const float*>(c_aux + a * NP + col + NQ * k);
        return c[f];
      };
      if (act) {
        if (MODE == MODE_RHS) {
#pragma unroll
          for (int k = 0; k < n1; ++k)
#pragma unroll
            for (int f = 0; f < 4; ++f) A.rhs[f * A.ndof + base + col + NQ * k] = rhs[f][k];
        } else if (MODE == MODE_STAGE) {   // LSRK(5,4) 2N-storage update
          const float dte = A.dtE ? A.dtE[e] : A.dt;
#pragma unroll
          for (int k = 0; k < n1; ++k)
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              const int64_t id = f * A.ndof + base + col + NQ * k;
              const float rr = A.a * auxv(0, f, k) + dte * rhs[f][k];
              q[f][k] += A.b * rr;
              A.res[id] = rr;
              A.qout[id] = q[f][k];
            }
        } else {   // MRC / MRF: AB3 update; MRC keeps the new state in rhs[] and the prediction in q[]
#pragma unroll
          for (int k = 0; k < n1; ++k)
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              const int64_t id = f * A.ndof + base + col + NQ * k;
              const float r0 = rhs[f][k], r1 = auxv(0, f, k), r2 = auxv(1, f, k);
              A.hw[id] = r0;
              const float qn = q[f][k] + A.ab0 * r0 + A.ab1 * r1 + A.ab2 * r2;
              A.qout[id] = qn;
              if (MODE == MODE_MRC) {
                rhs[f][k] = qn;
                q[f][k] += A.pr0 * r0 + A.pr1 * r1 + A.pr2 * r2;
              } else {
                q[f][k] = qn;
              }
            }
        }
      }
      __syncwarp();
    }
    stage_aux(welem(e_n));   // the aux buffer is free again

    // ---- traces of the state in q[] into the neighbours' inboxes (MRC: the half-step
    // prediction into tout, then the new state into tout2)
    constexpr int NPASS = MODE == MODE_RHS ? 0 : MODE == MODE_MRC ? 2 : 1;
#pragma unroll 1
    for (int pass = 0; pass < NPASS; ++pass) {
      float* tout = pass ? A.tout2 : A.tout;
      // the half-step traces only where a fine neighbour reads them
      const bool em = act && (MODE != MODE_MRC || pass == 1 || !A.pred || A.pred[e]);
      if (em) {
#pragma unroll
        for (int k = 0; k < n1; ++k) s_q[col + NQ * k] = make_float4(q[0][k], q[1][k], q[2][k], q[3][k]);
      }
      __syncwarp();
      if (em) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          float4 tm = make_float4(0.f, 0.f, 0.f, 0.f), tp = tm;
          auto node = [&](int m) {
            if (ax == 0) return s_q[m + n1 * i + NQ * j];
            if (ax == 1) return s_q[i + n1 * m + NQ * j];
            return make_float4(q[0][m], q[1][m], q[2][m], q[3][m]);
          };
          if constexpr (SEM) {
            tm = node(0);
            tp = node(N);
          } else {
#pragma unroll
            for (int m = 0; m < n1; ++m) {
              const float4 v = node(m);
              tm = f4fma(Vm[m], v, tm);
              tp = f4fma(Vp[m], v, tp);
            }
          }
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            const int f = 2 * ax + sd;
            const int nb = s_nb[f];
            const int64_t dst = nb >= 0 ? (int64_t)nb : ((MODE == MODE_TRACE && A.wall_self) ? A.side_off + e * 6 + f : -1);
            if (dst < 0) continue;
            float nv[3];
            if (MODE != MODE_TRACE) {
              const float4 nn = s_N[f * NQ + col];
              nv[0] = nn.x;
              nv[1] = nn.y;
              nv[2] = nn.z;
            } else {
              float Js;
              hexw_face_geom<N>(g_, R1, f, i, j, nv, Js);
            }
            const float4 tr = sd ? tp : tm;
            const int cidx = s_perm[s_code[f] * NQ + col];
            tout[dst * NQ + cidx] = tr.x;
            tout[A.plane + dst * NQ + cidx] = nv[0] * tr.y + nv[1] * tr.z + nv[2] * tr.w;
          }
        }
      }
      __syncwarp();
      if (MODE == MODE_MRC && act) {
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) q[f][k] = rhs[f][k];
      }
    }
    if (MODE == MODE_RHS) __syncwarp();
    e_c = e_n;
    e_n = e_nn;
  }
  cp_async_wait<0>();
  if (TMA && bail) {   // report, then wait (bounded) for this warp's copies still in flight
    if (lane == 0) atomicOr(A.err, 1);
#pragma unroll 1
    for (int k = 0; k < 4; ++k)
      if (pend & (1u << k)) mbar_wait(bar + k, (phase >> k) & 1u);
  }
}

template <int N, int MODE, bool TMA, bool SEM>
static void launch_hexw_n(const Args& A, const HexMaps& M, cudaStream_t s) {
  using H = HexP<N, MODE, TMA>;
  if (A.K == 0) return;
  static int blocks = 0;   // persistent grid: resident blocks per SM x SMs (computed once)
  if (blocks == 0) {
    cudaFuncSetAttribute(hexw_kernel<N, MODE, TMA, SEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, H::SMEM);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hexw_kernel<N, MODE, TMA, SEM>, 32 * H::WPB, H::SMEM);
    blocks = (per < 1 ? 1 : per) * sms;
  }
  const int64_t per_block = (int64_t)H::WPB * H::EPW;
  const int64_t need = ((int64_t)A.K + per_block - 1) / per_block;
  const int grid = (int)(need < blocks ? need : blocks);
  hexw_kernel<N, MODE, TMA, SEM><<<grid, 32 * H::WPB, H::SMEM, s>>>(A, M);
}

// ---------------------------------------------------------------------------- hex, N >= 6, columns
// Column kernel for N = 6..9 (rhs, LSRK stage, traces; at N = 5 its 36 columns fill 2 warps too
// sparsely and the thread-per-node kernel is 5 % faster): an element's (N+1)^2 node columns are
// spread over WPE = ceil((N+1)^2 / 32) warps, thread = column (i, j) with the column's N+1 nodes
// in registers (t-derivatives, t-face traces and the update from registers; r/s-derivatives and
// r/s-face traces read the element's node values from shared memory), as in the N <= 4 kernel
// above.  A block holds G element groups of WPE warps; each group walks its own elements and
// synchronises on its own named barrier, so the groups stay independent.  While a group computes
// element g, the cp.async copies of the next element's state and side data (double-buffered), of
// its inbox planes (after g's flux phase) and of its residual (after g's update) are in flight.
#ifndef DG_HEXC_MINB
#define DG_HEXC_MINB 1
#endif
template <int N, int MODE>
struct HexC {
  static constexpr int n1 = N + 1, NP = n1 * n1 * n1, NQ = n1 * n1;
  static constexpr int WPE = (NQ + 31) / 32, GT = WPE * 32;
  static constexpr int G = WPE >= 3 ? 1 : 4 / WPE;        // N = 6, 7: 2 groups of 2 warps; N = 8, 9: 1
  static constexpr int NT = G * GT;
  static constexpr int NAUX = MODE == MODE_STAGE ? 1 : 0;
  static constexpr int SD = 44;   // geometry [24], nbr [6], code [6], tau [6], c2
  // per group (bytes): q [2][NP] float4, aux [NAUX][NP] float4, F [4][NQ] float4, Nrm [6][NQ]
  // float4, in [12 NQ] float, sd [2][SD] float
  static constexpr int O_AUX = 2 * NP * 16;
  static constexpr int O_F = O_AUX + NAUX * NP * 16;
  static constexpr int O_N = O_F + 4 * NQ * 16;
  static constexpr int O_IN = O_N + 6 * NQ * 16;
  static constexpr int O_SD = O_IN + 12 * NQ * 4;
  static constexpr int PG = ((O_SD + 2 * SD * 4 + 15) / 16) * 16;
  static constexpr int CB = ((n1 * n1 + 5 * n1) * 4 + 15) / 16 * 16;   // D, Vm, Vp, w, r, 1/w
  static constexpr int PERM_B = 8 * NQ * 4;
  static constexpr int SMEM = CB + PERM_B + G * PG;
  static_assert(SMEM <= 227 * 1024, "hex column kernel: shared memory");
};

template <int N, int MODE>
__global__ void __launch_bounds__(HexC<N, MODE>::NT, DG_HEXC_MINB) hexc_kernel(Args A) {
  using H = HexC<N, MODE>;
  constexpr int n1 = H::n1, NP = H::NP, NQ = H::NQ, GT = H::GT, G = H::G, SD = H::SD;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sc = reinterpret_cast<float*>(smem_raw);
  const float* Dm = sc;
  const float* Vm = Dm + n1 * n1;
  const float* Vp = Vm + n1;
  const float* W1 = Vp + n1;
  const float* R1 = W1 + n1;
  const float* iW = R1 + n1;
  int* s_perm = reinterpret_cast<int*>(smem_raw + H::CB);
  const int grp = threadIdx.x / GT, col = threadIdx.x % GT;
  const bool own = col < NQ;            // threads past the last column only copy and synchronise
  const int cl = own ? col : 0;
  const int i = cl % n1, j = cl / n1;
  unsigned char* pg = smem_raw + H::CB + H::PERM_B + grp * H::PG;
  auto SQ = [&](int b) { return reinterpret_cast<float4*>(pg) + b * NP; };
  float4* c_aux = reinterpret_cast<float4*>(pg + H::O_AUX);
  float4* s_F = reinterpret_cast<float4*>(pg + H::O_F);
  float4* s_N = reinterpret_cast<float4*>(pg + H::O_N);
  float* c_in = reinterpret_cast<float*>(pg + H::O_IN);
  auto SDp = [&](int b) { return reinterpret_cast<float*>(pg + H::O_SD) + b * SD; };
  const unsigned bid = 1 + grp;   // named barrier of the group
  auto gsync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(bid), "r"(GT) : "memory"); };

  for (int x = threadIdx.x; x < n1 * n1 + 5 * n1; x += blockDim.x) sc[x] = A.hexc[x];
  for (int x = threadIdx.x; x < 8 * NQ; x += blockDim.x) s_perm[x] = A.perm[x];
  __syncthreads();

  auto elem = [&](int64_t g) -> int64_t {
    const int64_t li = g * G + grp;
    if (li >= A.K) return -1;
    return A.elist ? (int64_t)A.elist[li] : li;
  };
  // copies by every thread of the group: columns col, col + GT, ... of the NQ columns
  auto stage_main = [&](int b, int64_t e) {
    if (e >= 0) {
      float* dq = reinterpret_cast<float*>(SQ(b));
      for (int c = col; c < NQ; c += GT) {
        const float* qs = A.q + A.dof_off + e * NP + c;
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) cp_async4(dq + 4 * (c + NQ * k) + f, qs + f * A.ndof + NQ * k);
      }
      const int64_t gs0 = A.side_off + e * 6;
      float* ds = SDp(b);
      for (int x = col; x < SD - 1; x += GT) {
        const void* src = x < 24   ? static_cast<const void*>(A.geo + e * 24 + x)
                          : x < 30 ? static_cast<const void*>(A.nbr + gs0 + (x - 24))
                          : x < 36 ? static_cast<const void*>(A.code + gs0 + (x - 30))
                          : x < 42 ? static_cast<const void*>(A.tau + gs0 + (x - 36))
                                   : static_cast<const void*>(A.c2 + e);
        cp_async4(ds + x, src);
      }
    }
    cp_async_commit();
  };
  auto stage_in = [&](int64_t e) {
    if (MODE != MODE_TRACE && e >= 0) {
      const float* src = A.tin + (A.side_off + e * 6) * NQ;
      for (int y = col; y < 12 * NQ; y += GT) cp_async4(c_in + y, src + (y >= 6 * NQ ? A.plane - 6 * NQ : 0) + y);
    }
    cp_async_commit();
  };
  auto stage_aux = [&](int64_t e) {
    if (H::NAUX > 0 && e >= 0) {
      float* d = reinterpret_cast<float*>(c_aux);
      for (int c = col; c < NQ; c += GT) {
        const float* s0 = A.res + A.dof_off + e * NP + c;
#pragma unroll
        for (int k = 0; k < n1; ++k)
#pragma unroll
          for (int f = 0; f < 4; ++f) cp_async4(d + 4 * (c + NQ * k) + f, s0 + f * A.ndof + NQ * k);
      }
    }
    cp_async_commit();
  };

  int64_t g = blockIdx.x;
  const int64_t gstride = gridDim.x;
  int64_t e_c = elem(g), e_n = elem(g + gstride);
  stage_main(0, e_c);
  stage_in(e_c);
  stage_aux(e_c);
  int b = 0;
  for (; g * G + grp < A.K; g += gstride, b ^= 1) {
    const int64_t e_nn = elem(g + 2 * gstride);   // consumed one element later
    stage_main(b ^ 1, e_n);
    cp_async_wait<2>();                           // main(g) and in(g) have landed
    gsync();
    const int64_t e = e_c;
    const int64_t base = A.dof_off + e * NP;
    const float* g_ = SDp(b);
    const int* s_nb = reinterpret_cast<const int*>(g_ + 24);
    const int* s_code = reinterpret_cast<const int*>(g_ + 30);
    const float* s_tau = g_ + 36;
    const float c2 = g_[42];
    float4* s_q = SQ(b);
    float q[4][n1];
#pragma unroll
    for (int k = 0; k < n1; ++k) {
      const float4 v = s_q[cl + NQ * k];
      q[0][k] = v.x;
      q[1][k] = v.y;
      q[2][k] = v.z;
      q[3][k] = v.w;
    }
    float rhs[4][n1];
    float iJn[n1];
    if (MODE != MODE_TRACE && own) {
      // ---- volume: collocated strong form (Alg. hex_vol), metrics built along the column
      const float r = R1[i], s = R1[j];
      float Ar[3], Br[3], As[3], Bs[3], xt[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Ar[d] = g_[d] + g_[9 + d] * s;
        Br[d] = g_[12 + d] + g_[18 + d] * s;
        As[d] = g_[3 + d] + g_[9 + d] * r;
        Bs[d] = g_[15 + d] + g_[18 + d] * r;
        xt[d] = g_[6 + d] + g_[12 + d] * r + g_[15 + d] * s + g_[18 + d] * r * s;
      }
      float G0a[3], G0b[3], G1a[3], G1b[3], G2a[3], G2b[3], G2c[3], tmp[3];
      cross3(As, xt, G0a);
      cross3(Bs, xt, G0b);
      cross3(xt, Ar, G1a);
      cross3(xt, Br, G1b);
      cross3(Ar, As, G2a);
      cross3(Ar, Bs, G2b);
      cross3(Br, As, tmp);
      G2b[0] += tmp[0];
      G2b[1] += tmp[1];
      G2b[2] += tmp[2];
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
        const float iJ = __frcp_rn(J);
        iJn[k] = iJ;
        float4 dr = make_float4(0.f, 0.f, 0.f, 0.f), ds = dr, dt4 = dr;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          dr = f4fma(Dm[i * n1 + m], s_q[m + n1 * j + NQ * k], dr);
          ds = f4fma(Dm[j * n1 + m], s_q[i + n1 * m + NQ * k], ds);
          dt4 = f4fma(Dm[k * n1 + m], make_float4(q[0][m], q[1][m], q[2][m], q[3][m]), dt4);
        }
        const float dt[4] = {dt4.x, dt4.y, dt4.z, dt4.w};
        const float drf[4] = {dr.x, dr.y, dr.z, dr.w}, dsf[4] = {ds.x, ds.y, ds.z, ds.w};
        float div = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) div += g0[d] * drf[1 + d] + g1[d] * dsf[1 + d] + g2[d] * dt[1 + d];
        rhs[0][k] = -div * iJ;
#pragma unroll
        for (int d = 0; d < 3; ++d) rhs[1 + d][k] = -c2 * iJ * (g0[d] * drf[0] + g1[d] * dsf[0] + g2[d] * dt[0]);
      }
    }
    float4 F45[2];
    if (MODE != MODE_TRACE && own) {
      // ---- fluxes at this thread's point (a,b) = (i,j) of all six faces
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        float4 tm = make_float4(0.f, 0.f, 0.f, 0.f), tp = tm;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          const float4 v = ax == 0 ? s_q[m + n1 * i + NQ * j]
                           : ax == 1 ? s_q[i + n1 * m + NQ * j]
                                     : make_float4(q[0][m], q[1][m], q[2][m], q[3][m]);
          tm = f4fma(Vm[m], v, tm);
          tp = f4fma(Vp[m], v, tp);
        }
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const int f = 2 * ax + sd;
          const float4 tr = sd ? tp : tm;
          float nv[3], Js;
          hexw_face_geom<N>(g_, R1, f, i, j, nv, Js);
          s_N[f * NQ + cl] = make_float4(nv[0], nv[1], nv[2], Js);
          const float unm = nv[0] * tr.y + nv[1] * tr.z + nv[2] * tr.w;
          const int nb = s_nb[f];
          float P = 0.f, UN = 0.f;
          if (nb >= 0) {
            const int cidx = s_perm[s_code[f] * NQ + cl];
            P = c_in[f * NQ + cidx];
            UN = c_in[6 * NQ + f * NQ + cidx];
          }
          const float ta = s_tau[f];
          float fp, fu;
          flux(nb < 0, tr.x, unm, P, UN, A.tau_scale * ta, A.tau_scale * __frcp_rn(ta), false, fp, fu);
          const float wg = W1[i] * W1[j] * Js;
          const float4 Fv = make_float4(wg * fp, wg * fu * nv[0], wg * fu * nv[1], wg * fu * nv[2]);
          if (ax < 2) s_F[f * NQ + cl] = Fv;
          else F45[sd] = Fv;
        }
      }
    }
    gsync();
    stage_in(e_n);   // the inbox buffer is free again
    if (MODE != MODE_TRACE) {
      if (own) {
        // ---- lift (Alg. hex_surf), M^{-1} = 1/(w w w J)
#pragma unroll
        for (int k = 0; k < n1; ++k) {
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
          sum = f4fma(Vm[i], s_F[0 * NQ + j + n1 * k], sum);
          sum = f4fma(Vp[i], s_F[1 * NQ + j + n1 * k], sum);
          sum = f4fma(Vm[j], s_F[2 * NQ + i + n1 * k], sum);
          sum = f4fma(Vp[j], s_F[3 * NQ + i + n1 * k], sum);
          sum = f4fma(Vm[k], F45[0], sum);
          sum = f4fma(Vp[k], F45[1], sum);
          const float iM = iW[i] * iW[j] * iW[k] * iJn[k];
          rhs[0][k] += iM * sum.x;
          rhs[1][k] += c2 * iM * sum.y;
          rhs[2][k] += c2 * iM * sum.z;
          rhs[3][k] += c2 * iM * sum.w;
        }
        if (e == A.src_e) {   // point source on p
#pragma unroll
          for (int k = 0; k < n1; ++k) rhs[0][k] += A.src_s * A.src_g[cl + NQ * k];
        }
      }
      cp_async_wait<2>();   // aux(g) has landed
      gsync();
      if (own) {
        if (MODE == MODE_RHS) {
#pragma unroll
          for (int k = 0; k < n1; ++k)
#pragma unroll
            for (int f = 0; f < 4; ++f) A.rhs[f * A.ndof + base + cl + NQ * k] = rhs[f][k];
        } else {   // LSRK(5,4) 2N-storage update
          const float dte = A.dtE ? A.dtE[e] : A.dt;
#pragma unroll
          for (int k = 0; k < n1; ++k) {
            const float4 rv = c_aux[cl + NQ * k];
            const float ro[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              const int64_t id = f * A.ndof + base + cl + NQ * k;
              const float rr = A.a * ro[f] + dte * rhs[f][k];
              q[f][k] += A.b * rr;
              A.res[id] = rr;
              A.qout[id] = q[f][k];
            }
          }
        }
      }
      gsync();
    }
    stage_aux(e_n);   // the aux buffer is free again

    // ---- traces of the state in q[] into the neighbours' inboxes
    if (MODE != MODE_RHS) {
      if (MODE == MODE_STAGE) {
        if (own) {
#pragma unroll
          for (int k = 0; k < n1; ++k) s_q[cl + NQ * k] = make_float4(q[0][k], q[1][k], q[2][k], q[3][k]);
        }
        gsync();
      }
      if (own) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          float4 tm = make_float4(0.f, 0.f, 0.f, 0.f), tp = tm;
#pragma unroll
          for (int m = 0; m < n1; ++m) {
            const float4 v = ax == 0 ? s_q[m + n1 * i + NQ * j]
                             : ax == 1 ? s_q[i + n1 * m + NQ * j]
                                       : make_float4(q[0][m], q[1][m], q[2][m], q[3][m]);
            tm = f4fma(Vm[m], v, tm);
            tp = f4fma(Vp[m], v, tp);
          }
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            const int f = 2 * ax + sd;
            const int nb = s_nb[f];
            const int64_t dst = nb >= 0 ? (int64_t)nb : ((MODE == MODE_TRACE && A.wall_self) ? A.side_off + e * 6 + f : -1);
            if (dst < 0) continue;
            float nv[3];
            if (MODE != MODE_TRACE) {
              const float4 nn = s_N[f * NQ + cl];
              nv[0] = nn.x;
              nv[1] = nn.y;
              nv[2] = nn.z;
            } else {
              float Js;
              hexw_face_geom<N>(g_, R1, f, i, j, nv, Js);
            }
            const float4 tr = sd ? tp : tm;
            const int cidx = s_perm[s_code[f] * NQ + cl];
            A.tout[dst * NQ + cidx] = tr.x;
            A.tout[A.plane + dst * NQ + cidx] = nv[0] * tr.y + nv[1] * tr.z + nv[2] * tr.w;
          }
        }
      }
    }
    gsync();   // the state buffer is refilled two elements later; side data and faces next element
    e_c = e_n;
    e_n = e_nn;
  }
  cp_async_wait<0>();
}

template <int N, int MODE>
static void launch_hexc_n(const Args& A, cudaStream_t s) {
  using H = HexC<N, MODE>;
  if (A.K == 0) return;
  static int blocks = 0;   // persistent grid: resident blocks per SM x SMs (computed once)
  if (blocks == 0) {
    cudaFuncSetAttribute(hexc_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, H::SMEM);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hexc_kernel<N, MODE>, H::NT, H::SMEM);
    blocks = (per < 1 ? 1 : per) * sms;
  }
  const int64_t need = ((int64_t)A.K + H::G - 1) / H::G;
  const int grid = (int)(need < blocks ? need : blocks);
  hexc_kernel<N, MODE><<<grid, H::NT, H::SMEM, s>>>(A);
}

// ---------------------------------------------------------------------------- TMA descriptors
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<EncodeTiledFn>(nullptr);
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// 1D descriptor of n floats at base, box of `box` floats; false where TMA cannot address it.
bool tma_map_1d(TmaArr& t, const float* base, int64_t n, int box) {
  t.ok = false;
  t.base = base;
  t.n = n;
  t.box = box;
  EncodeTiledFn enc = encode_fn();
  if (!enc || !base || n <= 0 || n >= (1LL << 31) || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t dim[1] = {static_cast<cuuint64_t>(n)};
  const cuuint64_t stride[1] = {4};
  const cuuint32_t boxd[1] = {static_cast<cuuint32_t>(box)};
  const cuuint32_t es[1] = {1};
  t.ok = enc(&t.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, const_cast<float*>(base), dim, stride, boxd, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  return t.ok;
}

// 2D descriptors of the tensor-core volume operands: X [rows][4 npk] and B [4 npp][4 npk], 16-bit,
// copied in boxes of 8 values (16 bytes: one K-major core-matrix row) x 128 (X) or npp (B) rows
bool prec_maps(PrecMaps& M, const PrecDev& P, int64_t rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc || rows <= 0 || rows >= (1LL << 31)) return false;
  auto map2 = [&](CUtensorMap* m, const void* base, int64_t nrow, int box_rows) {
    const cuuint64_t dim[2] = {static_cast<cuuint64_t>(P.kx), static_cast<cuuint64_t>(nrow)};
    const cuuint64_t stride[1] = {static_cast<cuuint64_t>(P.kx * 2)};
    const cuuint32_t boxd[2] = {8, static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dim, stride, boxd, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  return map2(&M.xh, P.xh, rows, 128) && map2(&M.xl, P.xl, rows, 128) &&
         map2(&M.bh, P.bh, (int64_t)P.nblk * P.npp, P.npp) && map2(&M.bl, P.bl, (int64_t)P.nblk * P.npp, P.npp);
}

// the registered array holding p (with p's offset in floats), or null
static const TmaArr* tma_find(const dg_mesh* m, const float* p, long long* off) {
  for (const TmaArr& t : m->tma)
    if (t.ok && p >= t.base && p < t.base + t.n) {
      *off = p - t.base;
      return &t;
    }
  return nullptr;
}

// TMA operands of a fused hex update launch, or false (then the cp.async kernel runs)
template <int MODE>
static bool hex_maps(const dg_mesh* m, const Args& A, HexMaps* M) {
  if (m->N != 4 || !(MODE == MODE_STAGE || MODE == MODE_MRC || MODE == MODE_MRF)) return false;
  const TmaArr *q = tma_find(m, A.q, &M->qoff), *in = tma_find(m, A.tin, &M->inoff);
  const TmaArr* a0 = tma_find(m, MODE == MODE_STAGE ? A.res : A.h1, &M->a0off);
  const TmaArr* a1 = MODE == MODE_STAGE ? a0 : tma_find(m, A.h2, &M->a1off);
  if (MODE == MODE_STAGE) M->a1off = M->a0off;
  if (!q || !in || !a0 || !a1 || q->box != 128 || a0->box != 128 || a1->box != 128 || in->box != 160) return false;
  M->q = q->map;
  M->in = in->map;
  M->a0 = a0->map;
  M->a1 = a1->map;
  return true;
}

// ============================================================================ wedge, pyramid, tet

template <int T, int N>
struct GenCfg {
  static constexpr int NP = np_of(T, N), NQ = (N + 1) * (N + 1), NF = T == DG_TET ? 4 : 5;
  static constexpr int NC = T == DG_WEDGE ? (N + 1) * (N + 1) * (N + 1) : 1;
  static constexpr int NT = 128;
  // volume intermediates [7][SW] in dynamic shared memory (the wedge's exceed the static limit at N = 9)
  static constexpr int SW = T == DG_WEDGE ? NC : (T == DG_PYR ? NP : 3 * NP / 7 + 1);
  static constexpr int DYN = 7 * SW * 4;
};

template <int T, int N, int MODE>
__global__ void __launch_bounds__(128) gen_kernel(Args A) {
  using C = GenCfg<T, N>;
  constexpr int NP = C::NP, NQ = C::NQ, NF = C::NF, NC = C::NC, NT = C::NT;
  __shared__ float s_q[4][NP];
  __shared__ float s_r[4][NP];
  __shared__ float s_F[NF][4][NQ];
  extern __shared__ __align__(16) float gen_dyn[];
  float(*s_w)[C::SW] = reinterpret_cast<float(*)[C::SW]>(gen_dyn);
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
      const float* geo = A.geo + e * NP * 10;   // [10][NP]: component c of node m at c * NP + m
      for (int x = tid; x < 3 * NP; x += NT) {
        int a = x / NP, m = x % NP;
        const float* g = geo + m;
        s_w[a][m] = g[9 * NP] * (g[3 * a * NP] * s_q[1][m] + g[(3 * a + 1) * NP] * s_q[2][m] +
                                 g[(3 * a + 2) * NP] * s_q[3][m]);
      }
      __syncthreads();
      for (int n = tid; n < NP; n += NT) {
        const float* g = geo + n;
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
        s_r[0][n] = pint / g[9 * NP];
        for (int d = 0; d < 3; ++d)
          s_r[1 + d][n] = -c2 * (g[d * NP] * dp[0] + g[(3 + d) * NP] * dp[1] + g[(6 + d) * NP] * dp[2]);
      }
    } else {
      // Alg. wedge_vol1/2 (LSC-DG skew form) at the (N+1)^3 cubature points, M = I
      const float* V = A.ops;                              // [NC][NP]
      const float* VT = A.ops + 4 * NC * NP;               // [NP][NC]
      const float* wq = A.ops + 8 * NC * NP;
      constexpr int NQT = NC / (N + 1) > 0 ? NC / (N + 1) : 1;   // triangle points; point q = (q % NQT, q / NQT)
      const float* wc = A.geo + e * 16;
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
        float g[12];
        wedge_metrics(wc, A.wpts[2 * (q % NQT)], A.wpts[2 * NQT + q / NQT], A.wpts[2 * (q % NQT) + 1], g);
        const float w = wq[q];
        float UJ = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float Ad = g[d] * Pa[0] + g[3 + d] * Pa[1] + g[6 + d] * Pa[2] - P * g[9 + d];
          s_w[d][q] = w * Ad;
          UJ += U[d] * g[9 + d];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
          s_w[3 + a][q] = w * (g[3 * a] * U[0] + g[3 * a + 1] * U[1] + g[3 * a + 2] * U[2]);
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
      if (T == DG_PYR) iM = 1.f / A.geo[(e * 10 + 9) * NP + n];
      float r[4];
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) r[fl] = s_r[fl][n] + (fl == 0 ? 1.f : c2) * iM * sum[fl];
      if (MODE == MODE_RHS) {
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) A.rhs[fl * A.ndof + base + n] = r[fl];
      } else {
        const float dte = A.dtE ? A.dtE[e] : A.dt;
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
          const int64_t id = fl * A.ndof + base + n;
          float rr = A.a * A.res[id] + dte * r[fl];
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
      const int64_t dst = nb >= 0 ? (int64_t)nb : ((MODE == MODE_TRACE && A.wall_self) ? gs : -1);
      if (dst < 0) continue;
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
      A.tout[dst * NQ + qq] = tr[0];
      A.tout[A.plane + dst * NQ + qq] = sg.x * tr[1] + sg.y * tr[2] + sg.z * tr[3];
    }
  }
}

// ============================================================================ energy
// E = 1/2 sum_K (p^T M p + (1/c^2) sum_d u_d^T M u_d).  Flat grid-stride loop over (element,
// node): FP32 per-node terms (hex w J, pyramid J, wedge 1; tet: row n of R q with M_hat = R^T R,
// so p^T M p = J |R p|^2), FP64 accumulation, one atomic per block.
template <int T, int N>
__global__ void __launch_bounds__(256) energy_kernel(Args A, const float* chol, double* acc) {
  constexpr int NP = T == DG_HEX ? (N + 1) * (N + 1) * (N + 1) : np_of(T, N);
  constexpr int n1 = N + 1;
  __shared__ double s_red[256];
  const int tid = threadIdx.x;
  double loc = 0.0;
  const int64_t total = (int64_t)A.K * NP;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + tid; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = x / NP;
    const int n = (int)(x % NP);
    const int64_t b = A.dof_off + e * NP;
    const float ic2 = 1.f / A.c2[e];
    float term;
    if (T == DG_TET) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      for (int m = n; m < NP; ++m) {
        const float r = __ldg(chol + n * NP + m);
#pragma unroll
        for (int f = 0; f < 4; ++f) c[f] = fmaf(r, A.q[f * A.ndof + b + m], c[f]);
      }
      term = A.geo[e * 12 + 9] * (c[0] * c[0] + ic2 * (c[1] * c[1] + c[2] * c[2] + c[3] * c[3]));
    } else {
      const float qv[4] = {A.q[b + n], A.q[A.ndof + b + n], A.q[2 * A.ndof + b + n], A.q[3 * A.ndof + b + n]};
      const float wsq = qv[0] * qv[0] + ic2 * (qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
      if (T == DG_HEX) {
        const float* g = A.geo + e * 24;
        const float* hc = A.hexc;
        const int i = n % n1, j = (n / n1) % n1, k = n / (n1 * n1);
        float xr[3], xs[3], xt[3], g0[3];
        hex_jac(g, hc[n1 * n1 + 3 * n1 + i], hc[n1 * n1 + 3 * n1 + j], hc[n1 * n1 + 3 * n1 + k], xr, xs, xt);
        cross3(xs, xt, g0);
        const float J = xr[0] * g0[0] + xr[1] * g0[1] + xr[2] * g0[2];
        term = hc[n1 * n1 + 2 * n1 + i] * hc[n1 * n1 + 2 * n1 + j] * hc[n1 * n1 + 2 * n1 + k] * J * wsq;
      } else if (T == DG_WEDGE) {
        term = wsq;
      } else {
        term = A.geo[(e * 10 + 9) * NP + n] * wsq;
      }
    }
    loc += (double)term;
  }
  s_red[tid] = loc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st) s_red[tid] += s_red[tid + st];
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
  A.wpts = td.wpts;
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
  A.nops2 = td.nops2;
  A.wall_self = m->wall_self ? 1 : 0;
  A.src_e = (t == DG_HEX && m->src_e >= 0 && m->src_now != 0.f) ? m->src_e : -1;
  A.src_s = m->src_now;
  A.src_g = m->src_g;
  A.K = td.K;
  A.elist = nullptr;
  A.err = m->derr;
  A.dof_off = td.dof_off;
  A.ndof = m->ndof;
  A.side_off = td.side_off;
  A.tau_scale = (float)m->tau_scale;
  A.skew = 1;
  A.dtE = m->dte[t];
  A.pred = m->mr_pred[t];
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
  using C = GenCfg<T, N>;
  if (A.K == 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gen_kernel<T, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::DYN);
    attr = true;
  }
  gen_kernel<T, N, MODE><<<A.K, C::NT, C::DYN, s>>>(A);
}

template <int MODE>
bool launch_gen2(int t, int N, const Args& A, cudaStream_t s);   // kernels_gen2.cu
template <int MODE>
bool launch_tet_tc(int N, const Args& A, cudaStream_t s);        // kernels_tc.cu
#ifndef DG_TET_TC
#define DG_TET_TC 1
#endif

// Event pair around one type's launch when dg_profile is on.
static int ev_take(dg_mesh* m) {
  if (m->ev_next == m->ev_pool.size()) {
    cudaEvent_t ev;
    cudaEventCreate(&ev);
    m->ev_pool.push_back(ev);
  }
  return (int)m->ev_next++;
}

// N <= 4 hexahedra: the TMA kernel for the fused N = 4 updates when every staged array has a
// descriptor, the cp.async kernel otherwise
template <int N, int MODE, bool SEM>
static void launch_hex_fast_b(dg_mesh* m, const Args& A, cudaStream_t s) {
  HexMaps M{};
  if constexpr (N == 4 && (MODE == MODE_STAGE || MODE == MODE_MRC || MODE == MODE_MRF)) {
    if (m->use_hex_tma && hex_maps<MODE>(m, A, &M)) {
      launch_hexw_n<N, MODE, true, SEM>(A, M, s);
      return;
    }
  }
  launch_hexw_n<N, MODE, false, SEM>(A, M, s);
}
template <int N, int MODE>
static void launch_hex_fast(dg_mesh* m, const Args& A, cudaStream_t s) {
  if (m->hex_sem) launch_hex_fast_b<N, MODE, true>(m, A, s);
  else launch_hex_fast_b<N, MODE, false>(m, A, s);
}

template <int MODE>
static void launch_type(dg_mesh* m, const Args& A0, int t) {
  if (A0.K == 0) return;
  if (MODE >= MODE_MRC && m->N > 4) return;   // fused multi-rate kernels exist for N <= 4 only
  cudaStream_t s = m->stream;
  int e0 = -1;
  if (m->profiling) {
    e0 = ev_take(m);
    cudaEventRecord(m->ev_pool[e0], s);
  }
  // precision > 0: the volume products of tets and pyramids (lattice-exchange meshes) and the
  // wedges' first contraction on the tensor cores in split 16-bit form, then the type's warp
  // kernel with those products as input.  (The wedge warp kernel's fused multi-rate modes exist
  // for N <= 4 only; at higher N those modes run a kernel that forms its own products.)
  Args A = A0;
  const bool tcv = m->precision > 0 && MODE != MODE_TRACE &&
                   (((t == DG_TET || t == DG_PYR) && m->tri_lat) ||
                    (t == DG_WEDGE && (MODE <= MODE_STAGE || m->N <= 4))) &&
                   m->prec[prec_slot(t)].y != nullptr;
  if (tcv) launch_prec_volume(m, t, A, s);
  switch (m->N) {
#define DG_CASE(NN)                                                   \
  case NN:                                                            \
    if (t == DG_HEX) { if (NN <= 4) launch_hex_fast<(NN <= 4 ? NN : 4), MODE>(m, A, s); else if (NN == 5) launch_hex_n<(NN < 6 ? NN : 5), (MODE > 2 ? 1 : MODE)>(A, s); else launch_hexc_n<(NN > 5 ? NN : 6), (MODE > 2 ? 1 : MODE)>(A, s); } \
    else if (DG_TET_TC && !tcv && t == DG_TET && m->tri_lat && m->use_tet_tc && launch_tet_tc<MODE>(NN, A, s)) {}   \
    else if ((t == DG_WEDGE || m->tri_lat) && launch_gen2<MODE>(t, NN, A, s)) {}   \
    else if (t == DG_WEDGE) launch_gen_n<DG_WEDGE, NN, (MODE > 2 ? 1 : MODE)>(A, s);   \
    else if (t == DG_PYR) launch_gen_n<DG_PYR, NN, (MODE > 2 ? 1 : MODE)>(A, s);       \
    else launch_gen_n<DG_TET, NN, (MODE > 2 ? 1 : MODE)>(A, s);                        \
    break;
    DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8) DG_CASE(9)
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
  // the four types of one launch group read the previous trace buffer and write disjoint slots of
  // the next, so they may run side by side (per-type timing keeps them on one stream)
  const bool par = m->type_streams && !m->profiling && m->tev[4];
  if (par) cudaEventRecord(m->tev[4], m->stream);
  for (int t = 0; t < 4; ++t) {
    if (sel) {
      A[t].elist = sel->list[t];
      A[t].K = (int)sel->count[t];
    }
    if (par && A[t].K > 0) {
      cudaStream_t home = m->stream;
      cudaStreamWaitEvent(m->tstream[t], m->tev[4], 0);
      m->stream = m->tstream[t];
      launch_type<MODE>(m, A[t], t);
      m->stream = home;
      cudaEventRecord(m->tev[t], m->tstream[t]);
      cudaStreamWaitEvent(home, m->tev[t], 0);
    } else {
      launch_type<MODE>(m, A[t], t);
    }
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
                         float b, float dt, float* qout) {
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
    A[t].qout = qout ? qout : q;
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

// one row of blocks per segment (blockIdx.y), grid-stride within it
__global__ void __launch_bounds__(256) seg_copy_kernel(const Seg* segs) {
  const Seg g = segs[blockIdx.y];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < g.n; k += (int64_t)gridDim.x * blockDim.x)
    g.dst[k] = g.src[k];
}

cudaError_t launch_seg_copy(const Seg* segs_dev, int nseg, cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  seg_copy_kernel<<<dim3(16, (unsigned)nseg), 256, 0, s>>>(segs_dev);
  return cudaGetLastError();
}

cudaError_t launch_energy(dg_mesh* m, const float* q, double* acc) {
  cudaStream_t s = m->stream;
  Args A[4];
  for (int t = 0; t < 4; ++t) {
    A[t] = make_args(m, t);
    A[t].q = q;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto egrid = [&](int t) {   // blocks of 256 (element, node) pairs, at most 8 per SM
    const int64_t need = ((int64_t)A[t].K * m->td[t].Np + 255) / 256;
    return (unsigned)(need < 8 * sms ? need : 8 * sms);
  };
  switch (m->N) {
#define DG_CASE(NN)                                                                                  \
  case NN:                                                                                           \
    if (A[0].K) energy_kernel<DG_HEX, NN><<<egrid(0), 256, 0, s>>>(A[0], nullptr, acc);              \
    if (A[1].K) energy_kernel<DG_WEDGE, NN><<<egrid(1), 256, 0, s>>>(A[1], nullptr, acc);            \
    if (A[2].K) energy_kernel<DG_PYR, NN><<<egrid(2), 256, 0, s>>>(A[2], nullptr, acc);              \
    if (A[3].K) energy_kernel<DG_TET, NN><<<egrid(3), 256, 0, s>>>(A[3], m->tet_chol_dev, acc);      \
    break;
    DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7) DG_CASE(8) DG_CASE(9)
#undef DG_CASE
    default: break;
  }
  return cudaGetLastError();
}

}  // namespace dgk
