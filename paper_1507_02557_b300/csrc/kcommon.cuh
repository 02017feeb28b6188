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
  // tensor-core volume terms (precision > 0, tets and pyramids): row li of vol holds, for the
  // element of list index li, [sum_a D^a w_a | D^r p | D^s p | D^t p] (pyramid: the first block
  // with the transposes (D^a)^T), each block vol_np floats wide; NULL = computed in the kernel
  const float* vol;
  int vol_np;
  // per-element LSRK step (element index of the type), NULL = dt
  const float* dtE;
};

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
