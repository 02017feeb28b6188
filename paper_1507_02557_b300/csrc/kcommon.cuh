// Shared definitions of the CUDA kernels (kernels.cu, kernels_gen2.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace dgk {

// TRACE: traces only; RHS: write rhs; STAGE: fused LSRK stage;
// MRC / MRF: fused multi-rate AB3 step of a coarse / fine element (see api.cpp).
enum { MODE_TRACE = 0, MODE_RHS = 1, MODE_STAGE = 2, MODE_MRC = 3, MODE_MRF = 4 };

struct Args {
  const float* q;     // state in  [4][ndof]
  float* qout;        // state out (stage: may alias q)
  float* res;         // LSRK residual [4][ndof]
  float* rhs;         // rhs out [4][ndof]
  const float* tin;   // inbox to read: plane 0 = p, plane 1 = u.n
  float* tout;        // inboxes to write
  int64_t plane;      // nsides * nq
  const float* geo;
  const float4* sgeo;
  const float* sisq;
  const float* c2;
  const float* Tt;
  const float* L;
  const float* ops;
  const int* nbr;
  const int* code;
  const float* tau;
  const float* hexc;
  const int* perm;
  const float4* sgeo2;  // orientation-free kernels: face geometry in their point order
  const float* sisq2;
  const float* ops2;
  const int* iops2;
  int nops2;          // floats in ops2 (layout check of the orientation-free kernels)
  int wall_self;      // trace launches (MODE_TRACE): a wall side's own trace also goes to its own slot
  // point source (hexahedra, RHS / STAGE): rhs_p += src_s src_g[node] in element src_e (-1: none)
  int64_t src_e;
  float src_s;
  const float* src_g;
  int* err;           // device error word (bit 0: a bounded wait timed out)
  const int* elist;   // optional element list (multi-rate levels); NULL = elements 0..K-1
  int K;              // number of elements processed
  int64_t dof_off, ndof, side_off;
  float a, b, dt, tau_scale;
  int skew;
  // multi-rate AB3 (MRC, MRF): rhs written to hw; q <- q + ab0 r + ab1 h1 + ab2 h2; coarse elements
  // also emit the traces of the prediction q + pr0 r + pr1 h1 + pr2 h2 to tout and of the new q to tout2
  float* hw;
  const float* h1;
  const float* h2;
  float ab0, ab1, ab2, pr0, pr1, pr2;
  float* tout2;
  // tensor-core volume terms (precision > 0), each block vol_np floats wide; NULL = computed in
  // the kernel.  Tets and pyramids: row li (element of list index li) holds
  // [sum_a D^a w_a | D^r p | D^s p | D^t p] (pyramid: the first block with the transposes
  // (D^a)^T).  Wedges: row li (N + 1) + l (1D level l) holds the seven products at the triangle
  // cubature points [V y_p | V_r y_p | V_t y_p | V y_s | V y_u | V y_v | V y_w], y_f the
  // triangle-mode vector of field f at level l (the 1D factor V1 applied; y_s: its derivative D1
  // applied to p)
  const float* vol;
  int vol_np;
  // per-element LSRK step (element index of the type), NULL = dt
  const float* dtE;
  const float* wpts;   // wedge cubature points (TypeDev::wpts)
  // MRC: per element of the type, 1 if it has a fine face neighbour; the others skip the half-step
  // traces, which no launch reads (NULL: every element writes them)
  const unsigned char* pred;
};

// Wedge metric terms at reference point (r, s, t) from the element's map coefficients c[15]
// (TypeDev::geo): g[0..8] = d(r,s,t)/d(x,y,z) row-major, g[9..11] = grad_x J / (2 J) (the LSC-DG
// term of Sec. 2.3.3), with J the map's Jacobian determinant.
__device__ __forceinline__ void wedge_metrics(const float* c, float r, float s, float t, float g[12]) {
  float xr[3], xs[3], xt[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xr[d] = fmaf(s, c[3 + d], c[d]);
    xt[d] = fmaf(s, c[9 + d], c[6 + d]);
    xs[d] = fmaf(t, c[9 + d], fmaf(r, c[3 + d], c[12 + d]));
  }
  auto cr = [](const float* a, const float* b, float* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
  };
  float gr[3], gs[3], gt[3];
  cr(xs, xt, gr);
  cr(xt, xr, gs);
  cr(xr, xs, gt);
  const float J = xr[0] * gr[0] + xr[1] * gr[1] + xr[2] * gr[2];
  const float iJ = 1.f / J;
  // dJ/dr = det(x_rs, x_s, x_t) + det(x_r, x_ss, x_t) + ... with x_rr = x_ss = x_tt = x_rt = 0:
  // dJ/dr = det(x_r, x_rs, x_t), dJ/ds = det(x_rs, x_s, x_t) + det(x_r, x_s, x_ts),
  // dJ/dt = det(x_r, x_ts, x_t); x_rs = b_r, x_ts = b_t
  const float* brs = c + 3;
  const float* bts = c + 9;
  float u[3];
  cr(brs, xt, u);
  const float Jr = xr[0] * u[0] + xr[1] * u[1] + xr[2] * u[2];
  const float Js = brs[0] * gr[0] + brs[1] * gr[1] + brs[2] * gr[2] + bts[0] * gt[0] + bts[1] * gt[1] +
                   bts[2] * gt[2];
  cr(bts, xt, u);
  const float Jt = xr[0] * u[0] + xr[1] * u[1] + xr[2] * u[2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g[d] = gr[d] * iJ;
    g[3 + d] = gs[d] * iJ;
    g[6 + d] = gt[d] * iJ;
  }
  const float h = 0.5f * iJ;
#pragma unroll
  for (int d = 0; d < 3; ++d) g[9 + d] = h * (g[d] * Jr + g[3 + d] * Js + g[6 + d] * Jt);
}

__device__ __forceinline__ void flux(bool wall, float pm, float unm, float P, float UN, float tp,
                                     float tu, bool skew, float& fp, float& fu) {
  if (wall) {
    P = -pm;
    UN = -unm;
  }
  float jp = P - pm;
  float jun = -UN - unm;
  fp = skew ? 0.5f * tp * jp - 0.5f * (unm - UN) : 0.5f * (tp * jp - jun);
  fu = 0.5f * (tu * jun - jp);
}


__host__ __device__ constexpr int np_of(int t, int N) {
  return t == DG_WEDGE ? (N + 1) * (N + 1) * (N + 2) / 2
         : t == DG_PYR ? (N + 1) * (N + 2) * (2 * N + 3) / 6
                       : (N + 1) * (N + 2) * (N + 3) / 6;
}

}  // namespace dgk
