// Warp-per-element kernels for tetrahedra, pyramids and wedges (sm_103a).
//
// Persistent blocks stage the element type's reference operators in shared memory
// once; each warp then walks over elements.  All operators are independent of the
// face orientation:
//   tet / pyramid triangle faces (affine: n, J^s and tau constant over the face)
//                   the trace is taken at the equispaced face lattice (a gather for the
//                   nodal tet, a small matrix for the pyramid) and exchanged there: the
//                   neighbour's value at local lattice node l sits at its canonical index.
//                   The flux is linear with constant coefficients, so its values at the
//                   lattice nodes determine it; the face quadrature of Sec. 2.3 of the
//                   P_N flux against P_N test traces is then the face mass matrix of the
//                   lattice basis, folded into the lift operators (Lf, Tn2) at setup;
//   wedge triangle faces (trace divided by sqrt J, not a polynomial)
//                   lattice values permuted into the canonical frame, interpolated to
//                   the canonical face quadrature points (matrix E); the lift applies
//                   E^T, the inverse permutation and the transposed lattice evaluation;
//   quad faces      the trace is taken at the local GL points and permuted.
// The four fields p,u,v,w travel together as float4, so every operator entry read
// from shared memory feeds four FMAs.
// Volume terms: Alg. tet_vol (strong form, constant metrics), Alg. pyr_vol (skew
// form with transposed operators), Alg. wedge_vol1/2 (LSC-DG skew form at the
// wedge cubature points).  Flux, walls and M^{-1} as in kernels.cu.
// The wedge's volume term is sum-factorised over triangle x 1D: the triangle modes of each 1D
// level are contracted to the triangle cubature points (or taken from the tensor-core pass,
// Args.vol), the metric terms are applied point by point, and a second contraction takes the
// points back to the modes; at N >= 5 one 1D plane of points at a time.  Where a plane's points
// or modes leave a partial warp pass, the leftover items share the warp (several lanes each,
// then a butterfly sum).
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace dgk {

// fewest warps per block for which the N >= 5 kernels keep their operators in shared memory
// (measured at N = 5..7: the tets do better with 16 warps and operators read through L1, the
// wedges with their operators in shared memory)
#ifndef DG_G2_MIN_WARPS
#define DG_G2_MIN_WARPS 6
#endif
#ifndef DG_G2_MIN_WARPS_TET
#define DG_G2_MIN_WARPS_TET 12
#endif

template <int T, int N>
struct G2 {
  static constexpr int NP = np_of(T, N), NQ = (N + 1) * (N + 1), NFN = (N + 1) * (N + 2) / 2;
  static constexpr int NF = T == DG_TET ? 4 : 5;
  static constexpr int NTRI = T == DG_WEDGE ? 2 : 4;
  static constexpr int NQUAD = NF - NTRI;
  static constexpr int NC = T == DG_WEDGE ? (N + 1) * (N + 1) * (N + 1) : 0;
  static constexpr int N1 = N + 1, NT = NFN;                            // wedge: 1D points, triangle modes
  // pyramid: work items of the sum-factorised volume products (level pairs (q, k) with k <= q + 1,
  // (k + 1)(q + 1) items each) and the factor tables FE, FD [N1]^4, CR, CC, AH [N1]^2
  static constexpr int pyr_items() {
    int s = 0;
    for (int q = 0; q <= N; ++q)
      for (int k = 0; k <= (q + 1 < N ? q + 1 : N); ++k) s += (k + 1) * (q + 1);
    return s;
  }
  static constexpr int NIT = T == DG_PYR ? pyr_items() : 0;
  static constexpr int VOL = T == DG_WEDGE ? NQ * NT * 4 + 2 * N1 * N1 + NQ * N1
                             : T == DG_PYR ? 2 * N1 * N1 * N1 * N1 + 3 * N1 * N1 : NP * NP * 4;
  static constexpr int NKL = (N + 1) * (N + 2) / 2;                   // pyramid (level k, index l <= k)
  // tet: lattice lift; pyramid: EF [4][NKL] | PF [4][NFN][NKL] | PF2 [4][NFN][NKL]; wedge: Vtl [2][NFN][NT]
  static constexpr int TN = T == DG_WEDGE ? NTRI * NFN * NT
                            : T == DG_PYR ? NTRI * NKL + 2 * NTRI * NFN * NKL : NTRI * NFN * NP;
  // pyramid: LA [N1][NKL] | GC [N1]; wedge: Ve [3][N1][NT] | V1e [2][N1] | V1q [N1][N1]
  static constexpr int TQ = T == DG_WEDGE ? NQUAD * N1 * NT + 2 * N1 + N1 * N1 : T == DG_PYR ? N1 * NKL + N1 : 0;
  static constexpr bool LAT = T != DG_WEDGE;                            // lattice-point face exchange
  static constexpr int TN2 = 0;
  static constexpr int NFX = LAT ? NTRI * NFN + NQUAD * NQ : NF * NQ;   // face flux points
  // pyramid N <= 4: the volume loop reads D^a[m][n] (a = r, s, t) and D^t[n][m] as one float4
  // (the .w of the operator entry) and D^r[n][m], D^s[n][m] as a float2 from PV2, laid out
  // [m][n] so that the lanes' reads are contiguous: 6 words instead of two float4 per product
  static constexpr int PV2 = 0;
  static constexpr int OPS = VOL + PV2 + TN + TQ + TN2 + NQ * NFN;
  static constexpr int IOPS = 12 * NFN + 8 * NQ + (T == DG_TET ? 4 * NFN : 0) + (T == DG_PYR ? N1 * N1 + NIT : 0);
  static constexpr int OPS_B = ((OPS * 4 + 15) / 16) * 16;
  static constexpr int IOPS_B = ((IOPS * 4 + 15) / 16) * 16;
  // per-warp float4 buffers: q4, W4 (wedge: Y/Z pair + X1,X2), F4, G4 (local-order moments),
  // V4 (canonical lattice values)
  // wedge volume scratch: Y/Z pairs [2][NT][N1] and the cubature-point intermediates X1, X2, all
  // NC points at once (N <= 4) or one 1D plane of NQ points at a time (N >= 5); also holds the face
  // values (Z [2][NT], Y [3][N1][N1], quad traces [3][NQ]) and the lift factors
  static constexpr bool WPLANE = N >= 5;
  static constexpr int WXN = WPLANE ? NQ : NC;
  static constexpr int WV0 = 2 * NT * N1 + 2 * WXN, WV1 = 2 * NT + 3 * N1 * N1 + 3 * NQ;
  static constexpr int WV = T == DG_WEDGE ? (WV0 > WV1 ? WV0 : WV1) : NP;
  static constexpr int WB0 = NP + WV + NFX + 2 * NTRI * NFN + (T == DG_PYR ? NKL * N1 + NQ : 0);   // F4: NFX
  // pyramid: the volume products' scratch (3 NIT floats from F4 on) may run past the face buffers
  // (N = 9): extra float4 at the end of the warp's buffer
  static constexpr int PEX0 = T == DG_PYR ? 3 * NIT - 4 * (WB0 - NP - WV) : 0;
  // wedge N <= 4: the element's face-point data (sgeo2 [NF][NQ] float4, sisq2 [NF][NQ] float)
  // copied into the end of the warp's buffer once per element (cp.async, during the volume
  // terms) and read there by the flux pass and the trace passes
  static constexpr bool WSG = T == DG_WEDGE && N <= 4;
  static constexpr int WSGB = WSG ? NF * NQ + (NF * NQ + 3) / 4 : 0;
  static constexpr int WB = WB0 + (PEX0 > 0 ? (PEX0 + 3) / 4 : 0) + WSGB;
  // tet / pyramid: the volume operator transposed, (D^T)[m][n] = D[n][m] as float4, follows the
  // operators in global memory at float offset OPS_T (host layout size NOPS)
  static constexpr int OPS_T = ((OPS + 3) / 4) * 4;
  static constexpr int NOPS = OPS_T + (T == DG_TET ? VOL : 0);
  // one block per SM.  Warps per block: 16 (pyramid 22, which fill the shared memory at N = 4),
  // fewer where the per-warp buffers do not fit.  The operators sit in shared memory while at
  // least 6 warps fit beside them (N <= 4: all of them); otherwise the kernel reads them from
  // global memory through L1, the volume operator in its transposed copy so that the lanes'
  // reads of one column are contiguous.
  static constexpr int SMEM_CAP = 226 * 1024;
  static constexpr int NW_DEF = T == DG_PYR ? 28 : 16;
  static constexpr int WB_B = WB * 16;
  // pyramid N <= 7: the first pass of the factorised face values as uniform work items, from a
  // block-shared table built at block start: per item the first node and the node stride (start |
  // stride << 16) and N1 coefficients, zero past the item's level size (the padded terms read nodes
  // that exist: the largest index is NP - 1)
  static constexpr bool PTAB = T == DG_PYR && N <= 7;   // (N = 8, 9: the table would cost warps)
  static constexpr int PL1 = PTAB ? NTRI * NKL + NKL * N1 : 0;
  static constexpr int PT_B = PTAB ? (((PL1 * (N1 + 1) + NP) * 4 + 15) / 16) * 16 : 0;   // + node decode [NP]
  static constexpr int NW_SM = (SMEM_CAP - OPS_B - IOPS_B - PT_B) / WB_B;
  static constexpr bool OPS_SMEM =
      NW_SM >= (N <= 4 ? NW_DEF : T == DG_TET ? DG_G2_MIN_WARPS_TET : DG_G2_MIN_WARPS);
  static constexpr int UNR = 4;   // volume loops (8 measured no faster from L2, slower for pyramids)
  // Tets whose operators are read from global memory: the block stages the volume operator in
  // chunks of CM rows that all its warps use, so each operator entry crosses from L2 once per
  // block iteration instead of once per element (N = 6: 14.3 -> 11.9 ms, N = 7: 30.8 -> 22.1 ms
  // per step on the throughput mesh).  Pyramids stage D and D^T per chunk: at N = 6 (10-row
  // chunks) that pays (17.7 -> 15.5 ms); at N = 7 the chunks are 7 rows and the block barriers
  // cost more than the L2 reads saved (29.9 -> 36.1 ms), so there they read through L1.
  static constexpr bool CHUNK = !OPS_SMEM && T == DG_TET;
  static constexpr int NOPV = 1;
  static constexpr int CM0 = 49152 / (NP * 16 * NOPV);
  static constexpr int CM = CM0 < 4 ? 4 : (CM0 > NP ? NP : CM0);
  static constexpr int CHUNK_B = CHUNK ? CM * NP * 16 * NOPV : 0;
  static constexpr int NW_FIT = OPS_SMEM ? NW_SM : (SMEM_CAP - IOPS_B - CHUNK_B - PT_B) / WB_B;
  static constexpr int NW = NW_FIT < NW_DEF ? NW_FIT : NW_DEF;
  static constexpr int SMEM = (OPS_SMEM ? OPS_B : 0) + IOPS_B + CHUNK_B + PT_B + NW * WB_B;
  static constexpr int R = (NP + 31) / 32;
  static_assert(N > 4 || (OPS_SMEM && NW == NW_DEF), "N <= 4 keeps its operators and warps in shared memory");
  static_assert(T != DG_PYR || 3 * NIT <= 4 * (WB - NP - WV), "pyramid product scratch exceeds the free warp buffers");
  static_assert(NW >= 1, "per-warp buffers exceed the shared memory");
};

__device__ __forceinline__ float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
// s += c v on the four fields as two packed FP32 pair FMAs (the same values as four fmaf)
__device__ __forceinline__ void f4acc(float4& s, float c, const float4& v) {
  const float2 cc = make_float2(c, c);
  const float2 lo = __ffma2_rn(cc, make_float2(v.x, v.y), make_float2(s.x, s.y));
  const float2 hi = __ffma2_rn(cc, make_float2(v.z, v.w), make_float2(s.z, s.w));
  s = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// face f of type T: triangle index (or -1) and quad index (or -1)
template <int T>
__device__ __forceinline__ int tri_of(int f) {
  return T == DG_TET ? f : T == DG_PYR ? (f == 0 ? -1 : f - 1) : (f < 2 ? f : -1);
}
template <int T>
__device__ __forceinline__ int quad_of(int f) {
  return T == DG_TET ? -1 : T == DG_PYR ? (f == 0 ? 0 : -1) : (f >= 2 ? f - 2 : -1);
}
template <int T>
__device__ __forceinline__ int face_of_tri(int ti) {
  return T == DG_PYR ? ti + 1 : ti;
}

template <int T, int N, int MODE>
__global__ void __launch_bounds__(G2<T, N>::NW * 32, 1) gen2_kernel(Args A) {
  using C = G2<T, N>;
  constexpr int NP = C::NP, NQ = C::NQ, NFN = C::NFN, NF = C::NF, NTRI = C::NTRI, NQUAD = C::NQUAD;
  constexpr int NC = C::NC, NW = C::NW, R = C::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int OPS_SB = C::OPS_SMEM ? C::OPS_B : 0;
  int* sio = reinterpret_cast<int*>(smem_raw + OPS_SB);
  float4* sch = reinterpret_cast<float4*>(smem_raw + OPS_SB + C::IOPS_B);   // [NOPV][CM][NP] (CHUNK)
  int* ptd = reinterpret_cast<int*>(smem_raw + OPS_SB + C::IOPS_B + C::CHUNK_B);   // [PL1] (PTAB)
  const float* ptc = reinterpret_cast<const float*>(ptd + C::PL1);                   // [PL1][N1]
  // pyramid node n = off_k + row (k + 1) + col: k | row << 4 | col << 8 (PTAB)
  const int* pnd = reinterpret_cast<const int*>(ptc + C::PL1 * C::N1);
  float4* swarp = reinterpret_cast<float4*>(smem_raw + OPS_SB + C::IOPS_B + C::CHUNK_B + C::PT_B);
  if constexpr (C::OPS_SMEM) {
    float* sops = reinterpret_cast<float*>(smem_raw);
    for (int x = threadIdx.x; x < C::OPS; x += blockDim.x) sops[x] = A.ops2[x];
  }
  for (int x = threadIdx.x; x < C::IOPS; x += blockDim.x) sio[x] = A.iops2[x];
  __syncthreads();
  const float* sop = C::OPS_SMEM ? reinterpret_cast<const float*>(smem_raw) : A.ops2;
  const float4* DT4 = reinterpret_cast<const float4*>(A.ops2 + C::OPS_T);   // global: D^T (tet, pyramid)

  const float4* DV4 = reinterpret_cast<const float4*>(sop);     // tet/pyr [NP][NP]; wedge Vt4 [NQ][NT]
  const float* V1 = sop + NQ * C::NT * 4;                        // wedge [N1][N1] (l, j)
  const float* D1 = V1 + C::N1 * C::N1;
  const float* wq = D1 + C::N1 * C::N1;                          // wedge weights [NQ][N1]
  const float2* P2 = reinterpret_cast<const float2*>(sop + C::VOL);   // pyramid N <= 4 [NP][NP]
  const float* Tn = sop + C::VOL + C::PV2;                      // [NTRI][NFN][NP]
  const float* Tq = Tn + C::TN;                                  // [NQUAD][NQ][NP]
  const float* E = Tq + C::TQ;                                   // [NQ][NFN]
  constexpr bool LAT = C::LAT;
  constexpr int NFX = C::NFX, NLT = NTRI * NFN;
  const float* Vtl = Tn;                                         // wedge [2][NFN][NT]
  const float* Ve = Tq;                                          // wedge [3][N1][NT]
  const float* V1e = Tq + NQUAD * C::N1 * C::NT;                 // wedge [2][N1]
  const float* V1q = V1e + 2 * C::N1;                            // wedge [N1][N1]: 1D basis at quad-face s points
  constexpr int NKL = C::NKL;
  const float* EF = Tn;                                          // pyramid [4][NKL]
  const float* PF = Tn + NTRI * NKL;                             // pyramid [4][NFN][NKL]
  const float* PF2 = PF + NTRI * NFN * NKL;                      // pyramid [4][NFN][NKL]
  const float* LA = Tq;                                          // pyramid [N1][NKL]
  const float* GC = Tq + C::N1 * NKL;                            // pyramid [N1]
  const int* tperm = sio;                                        // [6][NFN] local lattice -> canonical
  const int* qperm = sio + 12 * NFN;                             // [8][NQ] local GL point -> canonical
  const int* fnode = qperm + 8 * NQ;                             // tet [4][NFN]
  if constexpr (C::PTAB) {   // uniform items of the first face-value pass (see G2::PTAB)
    constexpr int PN1 = C::N1;
    float* pc = const_cast<float*>(ptc);
    for (int x = threadIdx.x; x < C::PL1; x += blockDim.x) {
      const bool face = x < NTRI * NKL;
      const int kl = face ? x % NKL : (x - NTRI * NKL) / PN1;
      int k = 0;
      while ((k + 1) * (k + 2) / 2 <= kl) ++k;
      const int l = kl - k * (k + 1) / 2, k1 = k + 1, off = k * (k + 1) * (2 * k + 1) / 6, kb = k * (k + 1) / 2;
      const int ti = x / NKL;
      const bool alongi = face && (ti & 1);   // odd triangle faces sum over i, the others over j
      const float* src = face ? EF + ti * NKL + kb : LA + ((x - NTRI * NKL) % PN1) * NKL + kb;
      const float g = face ? 1.f : GC[k];
      ptd[x] = (alongi ? off + l * k1 : off + l) | ((alongi ? 1 : k1) << 16);
      for (int t = 0; t < PN1; ++t) pc[x * PN1 + t] = t < k1 ? g * src[t] : 0.f;
    }
    int* nd = const_cast<int*>(pnd);
    for (int n = threadIdx.x; n < NP; n += blockDim.x) {
      int k = 0;
      while ((k + 1) * (k + 2) * (2 * k + 3) / 6 <= n) ++k;
      const int rem = n - k * (k + 1) * (2 * k + 1) / 6;
      nd[n] = k | ((rem / (k + 1)) << 4) | ((rem % (k + 1)) << 8);
    }
    __syncthreads();
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int s_code[NW][NF];
  int* code = s_code[warp];
  float4* q4 = swarp + warp * C::WB;
  float4* W4 = q4 + NP;
  float4* F4 = W4 + C::WV;
  float4* G4 = F4 + NFX;
  float4* V4 = G4 + NTRI * NFN;
  float4* PZB = V4 + NTRI * NFN;                                 // pyramid [NKL][N1]
  float4* PTQB = PZB + NKL * C::N1;                              // pyramid [NQ] base traces
  float4* SGw = q4 + (C::WB - C::WSGB);                          // wedge (WSG): face data [NF][NQ]
  float* SIw = reinterpret_cast<float*>(SGw + NF * NQ);          // wedge (WSG): 1/sqrt J [NF][NQ]

  // CHUNK: the block's warps walk their elements in step (lb is the block's first) and every warp
  // takes part in every operator chunk (block barriers); a warp past the end redoes the last
  // element and stores nothing.  Otherwise each warp walks its own elements (lb is the warp's).
  for (int64_t lb = (int64_t)blockIdx.x * NW + (C::CHUNK ? 0 : warp); lb < A.K; lb += (int64_t)gridDim.x * NW) {
    const int64_t li_raw = C::CHUNK ? lb + warp : lb;
    const bool act = C::CHUNK ? li_raw < A.K : true;
    const int64_t li = act ? li_raw : A.K - 1;
    const int64_t e = A.elist ? (int64_t)A.elist[li] : li;
    const int64_t base = A.dof_off + e * NP;
    const float c2 = A.c2[e];
    if (lane < NF) code[lane] = A.code[A.side_off + e * NF + lane];
    for (int n = lane; n < NP; n += 32)
      q4[n] = f4(A.q[base + n], A.q[A.ndof + base + n], A.q[2 * A.ndof + base + n], A.q[3 * A.ndof + base + n]);
    if constexpr (C::WSG) {
      const float4* sgs = A.sgeo2 + e * NF * NQ;
      const float* sis = A.sisq2 + e * NF * NQ;
      for (int x = lane; x < NF * NQ; x += 32) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(SGw + x)),
                     "l"(sgs + x) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(SIw + x)),
                     "l"(sis + x) : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    __syncwarp();
    // the element's face data: staged copies (wedge N <= 4) or global memory
    auto face_ready = [&]() {
      if constexpr (C::WSG) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
      }
    };
    auto sg_at = [&](int f, int idx) -> float4 {
      if constexpr (C::WSG) return SGw[f * NQ + idx];
      else return A.sgeo2[(e * NF + f) * NQ + idx];
    };
    auto is_at = [&](int f, int idx) -> float {
      if constexpr (C::WSG) return SIw[f * NQ + idx];
      else return A.sisq2[(e * NF + f) * NQ + idx];
    };

    // wedge, factorised over triangle x 1D: lattice values of the two triangle faces (V4,
    // canonical order) and traces at the local GL points of the three quad faces (TQ), with
    // Z_f[mt] = sum_j phi_1D_j(s_f) q[mt, j] and Y_qf[ia][j] = sum_mt phi_tri_mt(edge_ia) q[mt, j]
    // staged in the (then free) volume scratch
    constexpr int WN1 = C::N1, WNT = C::NT;
    float4* ZB = W4;
    float4* YB = W4 + 2 * WNT;
    float4* TQB = YB + 3 * WN1 * WN1;
    auto wedge_face_values = [&]() {
      {
        auto item = [&](int x) {
          float4 v = f4(0.f, 0.f, 0.f, 0.f);
          if (x < 2 * WNT) {
            const int f = x / WNT, mt = x % WNT;
#pragma unroll
            for (int j = 0; j < WN1; ++j) f4acc(v, V1e[f * WN1 + j], q4[mt + WNT * j]);
            ZB[x] = v;
          } else {
            const int y = x - 2 * WNT, qf = y / (WN1 * WN1), ia = (y / WN1) % WN1, j = y % WN1;
            const float* ve = Ve + (qf * WN1 + ia) * WNT;
#pragma unroll 5
            for (int mt = 0; mt < WNT; ++mt) f4acc(v, ve[mt], q4[mt + WNT * j]);
            YB[y] = v;
          }
        };
        for (int x = lane; x < 2 * WNT; x += 32) item(x);   // one kind of item per warp pass
        for (int x = 2 * WNT + lane; x < 2 * WNT + 3 * WN1 * WN1; x += 32) item(x);
      }
      __syncwarp();
      {
        auto item = [&](int x) {
          float4 v = f4(0.f, 0.f, 0.f, 0.f);
          if (x < 2 * NFN) {
            const int ti = x / NFN, nl = x % NFN;
            const float* vt = Vtl + (ti * NFN + nl) * WNT;
#pragma unroll 5
            for (int mt = 0; mt < WNT; ++mt) f4acc(v, vt[mt], ZB[ti * WNT + mt]);
            V4[ti * NFN + tperm[code[ti] * NFN + nl]] = v;
          } else {
            const int y = x - 2 * NFN, qf = y / NQ, idx = y % NQ, ia = idx % WN1, ib = idx / WN1;
#pragma unroll
            for (int j = 0; j < WN1; ++j) f4acc(v, V1q[ib * WN1 + j], YB[(qf * WN1 + ia) * WN1 + j]);
            TQB[y] = v;
          }
        };
        for (int x = lane; x < 2 * NFN; x += 32) item(x);   // one kind of item per warp pass
        for (int x = 2 * NFN + lane; x < 2 * NFN + 3 * NQ; x += 32) item(x);
      }
    };
    // canonical lattice values of the triangle faces (V4) from q4
    // pyramid, factorised over the levels of the semi-nodal basis: triangle face ti fixes
    // b (ti even) or a (ti odd); Y_ti[k][l] = sum over the fixed direction of its factor times q
    // (into G4), then lattice values (local order) = sum_kl PF[x][kl] Y_ti[kl]; base:
    // Z[k][i][q] = GC_k sum_j LA[q][k][j] q_kji (PZB), traces = sum_kl LA[p][kl] Z[kl][q] (PTQB)
    auto pyr_face_values = [&]() {
      constexpr int PN1 = C::N1;
      if constexpr (C::PTAB) {
        for (int x = lane; x < C::PL1; x += 32) {
          const int d = ptd[x], n0 = d & 0xFFFF, ns = d >> 16;
          const float* pc = ptc + x * PN1;
          float4 v = f4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int t = 0; t < PN1; ++t) f4acc(v, pc[t], q4[n0 + t * ns]);
          if (x < NTRI * NKL) G4[x] = v;
          else PZB[x - NTRI * NKL] = v;
        }
      } else {
        auto item = [&](int x) {
          const bool face = x < NTRI * NKL;
          const int kl = face ? x % NKL : (x - NTRI * NKL) / PN1;
          int k = 0;
          while ((k + 1) * (k + 2) / 2 <= kl) ++k;
          const int l = kl - k * (k + 1) / 2, k1 = k + 1, off = k * (k + 1) * (2 * k + 1) / 6, kb = k * (k + 1) / 2;
          float4 v = f4(0.f, 0.f, 0.f, 0.f);
          if (face) {
            const int ti = x / NKL;
            const float* ef = EF + ti * NKL + kb;
            if (ti & 1) {
              for (int i = 0; i < k1; ++i) f4acc(v, ef[i], q4[off + l * k1 + i]);
            } else {
              for (int j = 0; j < k1; ++j) f4acc(v, ef[j], q4[off + j * k1 + l]);
            }
            G4[x] = v;
          } else {
            const float* la = LA + ((x - NTRI * NKL) % PN1) * NKL + kb;
            for (int j = 0; j < k1; ++j) f4acc(v, la[j], q4[off + j * k1 + l]);
            const float g = GC[k];
            PZB[x - NTRI * NKL] = f4(g * v.x, g * v.y, g * v.z, g * v.w);
          }
        };
        for (int x = lane; x < NTRI * NKL; x += 32) item(x);   // one kind of item per warp pass
        for (int x = NTRI * NKL + lane; x < NTRI * NKL + NKL * PN1; x += 32) item(x);
      }
      __syncwarp();
      {
        auto item = [&](int x) {
          float4 v = f4(0.f, 0.f, 0.f, 0.f);
          if (x < NTRI * NFN) {
            const float* pf = PF + x * NKL;
            const float4* y = G4 + (x / NFN) * NKL;
#pragma unroll 5
            for (int kl = 0; kl < NKL; ++kl) f4acc(v, pf[kl], y[kl]);
            V4[x] = v;
          } else {
            const int idx = x - NTRI * NFN, pp = idx % PN1, qq = idx / PN1;
            const float* la = LA + pp * NKL;
#pragma unroll 5
            for (int kl = 0; kl < NKL; ++kl) f4acc(v, la[kl], PZB[kl * PN1 + qq]);
            PTQB[idx] = v;
          }
        };
        for (int x = lane; x < NTRI * NFN; x += 32) item(x);   // one kind of item per warp pass
        for (int x = NTRI * NFN + lane; x < NTRI * NFN + NQ; x += 32) item(x);
      }
    };
    // (tet, pyramid: local order; the wedge also fills the quad-face traces)
    auto lattice_values = [&]() {
      if constexpr (T == DG_WEDGE) {
        wedge_face_values();
      } else if constexpr (T == DG_PYR) {
        pyr_face_values();
      } else {
        for (int x = lane; x < NTRI * NFN; x += 32) {
          float4 v;
          if (T == DG_TET) {
            v = q4[fnode[x]];
          } else {
            v = f4(0.f, 0.f, 0.f, 0.f);
            const float* row = Tn + x * NP;
#pragma unroll 4
            for (int m = 0; m < NP; ++m) f4acc(v, row[m], q4[m]);
          }
          V4[x] = v;
        }
      }
    };
    // trace (p,u,v,w) at point idx of face f (triangle: canonical point; quad: local point)
    auto trace_at = [&](int f, int idx) {
      float4 tr = f4(0.f, 0.f, 0.f, 0.f);
      const int ti = tri_of<T>(f);
      if (ti >= 0) {
        const float* er = E + idx * NFN;
        const float4* vc = V4 + ti * NFN;
        #pragma unroll 4
        for (int n = 0; n < NFN; ++n) f4acc(tr, er[n], vc[n]);
      } else if (T == DG_WEDGE) {
        tr = TQB[quad_of<T>(f) * NQ + idx];
      } else if (T == DG_PYR) {
        tr = PTQB[idx];
      } else {
        const float* row = Tq + (quad_of<T>(f) * NQ + idx) * NP;
        #pragma unroll 4
        for (int m = 0; m < NP; ++m) f4acc(tr, row[m], q4[m]);
      }
      if (T == DG_WEDGE) {
        const float is = is_at(f, idx);
        tr.x *= is; tr.y *= is; tr.z *= is; tr.w *= is;
      }
      return tr;
    };
    // LAT: trace at face-flux point x (lattice node of a triangle face, local order, or local
    // GL point of a quad face), its face, the inbox index and the face data (n, J^s or w J^s)
    auto lat_point = [&](int x, int& f, int& ci, float4& tr, float4& sg) {
      if (x < NLT) {
        const int ti = x / NFN, nl = x % NFN;
        f = face_of_tri<T>(ti);
        tr = T == DG_TET ? q4[fnode[x]] : V4[x];
        ci = tperm[code[f] * NFN + nl];
        sg = sg_at(f, 0);
      } else {
        const int idx = (x - NLT) % NQ;
        f = T == DG_PYR ? 0 : 2 + (x - NLT) / NQ;
        tr = trace_at(f, idx);
        ci = qperm[code[f] * NQ + idx];
        sg = sg_at(f, idx);
      }
    };

    float4 acc[R], pred[R];
    if (MODE != MODE_TRACE) {
      // ---------------------------------------------------------------- volume
      if (T == DG_TET) {
        const float* g = A.geo + e * 12;
        float G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) G[i] = g[i];
        for (int n = lane; n < NP && !A.vol; n += 32) {
          const float4 v = q4[n];
          W4[n] = f4(G[0] * v.y + G[1] * v.z + G[2] * v.w, G[3] * v.y + G[4] * v.z + G[5] * v.w,
                     G[6] * v.y + G[7] * v.z + G[8] * v.w, v.x);
        }
        __syncwarp();
        auto tet_acc = [&](float* a, const float4& d, const float4& w) {
          a[0] = fmaf(d.x, w.x, a[0]);
          a[1] = fmaf(d.y, w.y, a[1]);
          a[2] = fmaf(d.z, w.z, a[2]);
          a[3] = fmaf(d.x, w.w, a[3]);
          a[4] = fmaf(d.y, w.w, a[4]);
          a[5] = fmaf(d.z, w.w, a[5]);
        };
        auto tet_out = [&](int r, const float* a) {
          const float div = a[0] + a[1] + a[2];
          acc[r] = f4(-div, -c2 * (G[0] * a[3] + G[3] * a[4] + G[6] * a[5]),
                      -c2 * (G[1] * a[3] + G[4] * a[4] + G[7] * a[5]), -c2 * (G[2] * a[3] + G[5] * a[4] + G[8] * a[5]));
        };
        if (A.vol) {   // products from the tensor-core pass (row li: sum_a D^a w_a, D^r p, D^s p, D^t p)
          const float* vr = A.vol + li * 4 * (int64_t)A.vol_np;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            if (n >= NP) break;
            const float a[6] = {vr[n], 0.f, 0.f, vr[A.vol_np + n], vr[2 * A.vol_np + n], vr[3 * A.vol_np + n]};
            tet_out(r, a);
          }
        } else if constexpr (C::CHUNK) {   // all rows accumulate across the block's operator chunks
          float s6[R][6];
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < 6; ++c) s6[r][c] = 0.f;
          for (int m0 = 0; m0 < NP; m0 += C::CM) {
            const int mc = NP - m0 < C::CM ? NP - m0 : C::CM;
            __syncthreads();
            for (int x = threadIdx.x; x < mc * NP; x += blockDim.x) sch[x] = __ldg(DT4 + (size_t)m0 * NP + x);
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int n = lane + 32 * r;
              if (n >= NP) break;
#pragma unroll 4
              for (int mm = 0; mm < mc; ++mm) tet_acc(s6[r], sch[mm * NP + n], W4[m0 + mm]);
            }
          }
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (lane + 32 * r < NP) tet_out(r, s6[r]);
        } else {   // one row at a time
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            if (n >= NP) break;
            float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const float4* drow = DV4 + n * NP;
#pragma unroll C::UNR
            for (int m = 0; m < NP; ++m) tet_acc(a, C::OPS_SMEM ? drow[m] : __ldg(DT4 + m * NP + n), W4[m]);
            tet_out(r, a);
          }
        }
      } else if (T == DG_PYR) {
        const float* geo = A.geo + e * NP * 10;   // [10][NP]: component c of node m at c * NP + m
        auto geo_at = [&](int m, float (&g)[10]) {   // lanes read consecutive nodes: coalesced
#pragma unroll
          for (int c = 0; c < 10; ++c) g[c] = geo[c * NP + m];
        };
        for (int m = lane; m < NP && !A.vol; m += 32) {
          float g[10];
          geo_at(m, g);
          const float4 v = q4[m];
          const float J = g[9];
          W4[m] = f4(J * (g[0] * v.y + g[1] * v.z + g[2] * v.w), J * (g[3] * v.y + g[4] * v.z + g[5] * v.w),
                     J * (g[6] * v.y + g[7] * v.z + g[8] * v.w), v.x);
        }
        __syncwarp();
        // a[0] = sum_a ((D^a)^T J G u_a)[n] (skew part), a[3..5] = (D^a p)[n]
        auto pyr_out = [&](int r, const float* a) {
          float g[10];
          geo_at(lane + 32 * r, g);
          acc[r] = f4((a[0] + a[1] + a[2]) / g[9], -c2 * (g[0] * a[3] + g[3] * a[4] + g[6] * a[5]),
                      -c2 * (g[1] * a[3] + g[4] * a[4] + g[7] * a[5]), -c2 * (g[2] * a[3] + g[5] * a[4] + g[8] * a[5]));
        };
        if (A.vol) {   // products from the tensor-core pass (row li: sum_a (D^a)^T J G u_a, D^r p, D^s p, D^t p)
          const float* vr = A.vol + li * 4 * (int64_t)A.vol_np;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            if (n >= NP) break;
            const float a[6] = {vr[n], 0.f, 0.f, vr[A.vol_np + n], vr[2 * A.vol_np + n], vr[3 * A.vol_np + n]};
            pyr_out(r, a);
          }
        } else {
          // Sum-factorised skew volume terms (factor tables of the level pairs (q, k), see the host
          // layout): node (i, j, k) = off_k + j (k + 1) + i with off_k = k (k + 1)(2k + 1) / 6.
          constexpr int N1 = C::N1, NIT = C::NIT;
          const float* FE = sop;                                   // [q][k][l][i]
          const float* FD = FE + N1 * N1 * N1 * N1;
          const float* CR = FD + N1 * N1 * N1 * N1;
          const float* CC = CR + N1 * N1;
          const float* AH = CC + N1 * N1;
          const int* PB = sio + 12 * NFN + 8 * NQ;                 // [q][k] first item of the pair
          const int* IT = PB + N1 * N1;                            // items q | k<<4 | a<<8 | b<<12
          float* TT = reinterpret_cast<float*>(F4);                // scratch: the free face buffers
          auto off = [](int k) { return k * (k + 1) * (2 * k + 1) / 6; };
          auto lev = [&](int n) {
            int k = 0;
            while (off(k + 1) <= n) ++k;
            return k;
          };
          // (A) T[q][k][i][b] = sum_j E[q][k][b][j] p(i,j,k); T' with E' (b: test-level index)
          for (int x = lane; x < NIT; x += 32) {
            const int it = IT[x], q = it & 15, k = (it >> 4) & 15, i = (it >> 8) & 15, b = (it >> 12) & 15;
            const float* fe = FE + ((q * N1 + k) * N1 + b) * N1;
            const float* fd = FD + ((q * N1 + k) * N1 + b) * N1;
            const float4* pk = q4 + off(k) + i;
            float t = 0.f, td = 0.f;
            for (int j = 0; j <= k; ++j) {
              const float pv = pk[j * (k + 1)].x;
              t = fmaf(fe[j], pv, t);
              td = fmaf(fd[j], pv, td);
            }
            TT[x] = t;
            TT[NIT + x] = td;
          }
          __syncwarp();
          // (B) test node n = (l, b, q): D^r p, D^s p, D^t p
          float yg[R][3];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            yg[r][0] = yg[r][1] = yg[r][2] = 0.f;
            if (n >= NP) continue;
            int q, b, l;
            if constexpr (C::PTAB) {
              const int d = pnd[n];
              q = d & 15, b = (d >> 4) & 15, l = d >> 8;
            } else {
              q = lev(n);
              const int rem = n - off(q);
              b = rem / (q + 1), l = rem - b * (q + 1);
            }
            float yr = 0.f, ys = 0.f, yc = 0.f;
            for (int k = 0; k <= (q + 1 < N ? q + 1 : N); ++k) {
              const int base = PB[q * N1 + k];
              const float cr = CR[q * N1 + k], cc = CC[q * N1 + k];
              const float* fe = FE + ((q * N1 + k) * N1 + l) * N1;
              const float* fd = FD + ((q * N1 + k) * N1 + l) * N1;
              float sr = 0.f, ss = 0.f, sc = 0.f;
              for (int i = 0; i <= k; ++i) {
                const float t = TT[base + i * (q + 1) + b], td = TT[NIT + base + i * (q + 1) + b];
                sr = fmaf(fd[i], t, sr);
                ss = fmaf(fe[i], td, ss);
                sc = fmaf(fe[i], t, sc);
              }
              yr = fmaf(cr, sr, yr);
              ys = fmaf(cr, ss, ys);
              yc = fmaf(cc, sc, yc);
            }
            yg[r][0] = yr;
            yg[r][1] = ys;
            yg[r][2] = AH[q * N1 + l] * yr + AH[q * N1 + b] * ys + yc;
          }
          __syncwarp();
          // (C) W_r + (1+a_l)/2 W_t, W_s + (1+a_b)/2 W_t, W_t at each node (in place), then
          // A1[q][k][j][l] = sum_b E[q][k][b][j] (..)_r(l,b,q), A2 with E' and (..)_s, A3 with E and W_t
          for (int m = lane; m < NP; m += 32) {
            int q, b, l;
            if constexpr (C::PTAB) {
              const int d = pnd[m];
              q = d & 15, b = (d >> 4) & 15, l = d >> 8;
            } else {
              q = lev(m);
              const int rem = m - off(q);
              b = rem / (q + 1), l = rem - b * (q + 1);
            }
            const float4 w = W4[m];
            W4[m] = f4(fmaf(AH[q * N1 + l], w.z, w.x), fmaf(AH[q * N1 + b], w.z, w.y), w.z, w.w);
          }
          __syncwarp();
          for (int x = lane; x < NIT; x += 32) {
            const int it = IT[x], q = it & 15, k = (it >> 4) & 15, j = (it >> 8) & 15, l = (it >> 12) & 15;
            const float4* wq4 = W4 + off(q) + l;
            float a1 = 0.f, a2 = 0.f, a3 = 0.f;
            for (int b = 0; b <= q; ++b) {
              const float e1 = FE[((q * N1 + k) * N1 + b) * N1 + j], d1 = FD[((q * N1 + k) * N1 + b) * N1 + j];
              const float4 w = wq4[b * (q + 1)];
              a1 = fmaf(e1, w.x, a1);
              a2 = fmaf(d1, w.y, a2);
              a3 = fmaf(e1, w.z, a3);
            }
            TT[x] = a1;
            TT[NIT + x] = a2;
            TT[2 * NIT + x] = a3;
          }
          __syncwarp();
          // (D) trial node m = (i, j, k): sum over the test levels q >= k - 1
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m >= NP) break;
            int k, j, i;
            if constexpr (C::PTAB) {
              const int d = pnd[m];
              k = d & 15, j = (d >> 4) & 15, i = d >> 8;
            } else {
              k = lev(m);
              const int rem = m - off(k);
              j = rem / (k + 1), i = rem - j * (k + 1);
            }
            float z = 0.f;
            for (int q = (k > 0 ? k - 1 : 0); q <= N; ++q) {
              const int base = PB[q * N1 + k] + j * (q + 1);
              const float cr = CR[q * N1 + k], cc = CC[q * N1 + k];
              float s1 = 0.f, s3 = 0.f;
              for (int l = 0; l <= q; ++l) {
                const float e1 = FE[((q * N1 + k) * N1 + l) * N1 + i], d1 = FD[((q * N1 + k) * N1 + l) * N1 + i];
                s1 = fmaf(d1, TT[base + l], fmaf(e1, TT[NIT + base + l], s1));
                s3 = fmaf(e1, TT[2 * NIT + base + l], s3);
              }
              z = fmaf(cr, s1, fmaf(cc, s3, z));
            }
            const float a[6] = {z, 0.f, 0.f, yg[r][0], yg[r][1], yg[r][2]};
            pyr_out(r, a);
          }
        }
      } else {   // wedge, sum-factorised (triangle x 1D) form of Alg. wedge_vol1/2
        constexpr int NT = C::NT, N1 = C::N1;
        float4* Y4 = W4;                  // phase 1: [NT][N1] sum_j V1 q ; phase 2: ZA
        float4* Ys4 = W4 + NT * N1;       // phase 1: [NT][N1] sum_j D1 p (x); phase 2: ZB
        float4* X1 = W4 + 2 * NT * N1;    // [WXN] w (A0, A1, A2, UJ)
        float4* X2 = X1 + C::WXN;         // [WXN] w (GU0, GU1, GU2, 0)
        float wc[15];   // the element's map coefficients; metric terms rebuilt at each point
#pragma unroll
        for (int c = 0; c < 15; ++c) wc[c] = A.geo[e * 16 + c];
        for (int x = lane; x < NT * N1 && !A.vol; x += 32) {
          const int mt = x / N1, l = x % N1;
          float4 y = f4(0.f, 0.f, 0.f, 0.f);
          float ys = 0.f;
#pragma unroll
          for (int j = 0; j < N1; ++j) {
            const float4 v = q4[mt + NT * j];
            f4acc(y, V1[l * N1 + j], v);
            ys = fmaf(D1[l * N1 + j], v.x, ys);
          }
          Y4[x] = y;
          Ys4[x] = f4(ys, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        constexpr bool PL = C::WPLANE;
        float4* ZA = Y4;
        float4* ZB = Ys4;
#pragma unroll 1
        for (int lp = 0; lp < (PL ? N1 : 1); ++lp) {
        const int q0 = PL ? lp * NQ : 0, q1 = PL ? q0 + NQ : NC;
        // the seven first-contraction products at point qc (modes mt = part, part + step, ...)
        auto wprod = [&](int qc, int part, int step, float (&pr)[7]) {
          const int qt = qc % NQ, l = qc / NQ;
#pragma unroll
          for (int c = 0; c < 7; ++c) pr[c] = 0.f;
          if (A.vol) {   // the tensor-core pass: row (li, l) holds the seven products at point qt
            const float* yr = A.vol + ((int64_t)li * N1 + l) * 7 * A.vol_np + qt;
#pragma unroll
            for (int c = 0; c < 7; ++c) pr[c] = yr[c * A.vol_np];
          } else {
            const float4* vrow = DV4 + qt * NT;
#pragma unroll 5
            for (int mt = part; mt < NT; mt += step) {
              const float4 v = vrow[mt], y = Y4[mt * N1 + l];
              pr[0] = fmaf(v.x, y.x, pr[0]);              // V y_p
              pr[1] = fmaf(v.y, y.x, pr[1]);              // V_r y_p
              pr[2] = fmaf(v.z, y.x, pr[2]);              // V_t y_p
              pr[3] = fmaf(v.x, Ys4[mt * N1 + l].x, pr[3]);   // V y_s
              pr[4] = fmaf(v.x, y.y, pr[4]);              // V y_u, V y_v, V y_w
              pr[5] = fmaf(v.x, y.z, pr[5]);
              pr[6] = fmaf(v.x, y.w, pr[6]);
            }
          }
        };
        // metric terms at point qc and the weighted intermediates X1, X2
        auto wout = [&](int qc, const float (&pr)[7]) {
          const int qt = qc % NQ, l = qc / NQ;
          float g[12];
          wedge_metrics(wc, __ldg(A.wpts + 2 * qt), __ldg(A.wpts + 2 * NQ + l), __ldg(A.wpts + 2 * qt + 1), g);
          const float P = pr[0], Pr = pr[1], Pt = pr[2], Ps = pr[3], U0 = pr[4], U1 = pr[5], U2 = pr[6];
          const float w = wq[qt * N1 + l];
          const float A0 = g[0] * Pr + g[3] * Ps + g[6] * Pt - P * g[9];
          const float A1 = g[1] * Pr + g[4] * Ps + g[7] * Pt - P * g[10];
          const float A2 = g[2] * Pr + g[5] * Ps + g[8] * Pt - P * g[11];
          const float UJ = U0 * g[9] + U1 * g[10] + U2 * g[11];
          X1[qc - q0] = f4(w * A0, w * A1, w * A2, w * UJ);
          X2[qc - q0] = f4(w * (g[0] * U0 + g[1] * U1 + g[2] * U2), w * (g[3] * U0 + g[4] * U1 + g[5] * U2),
                           w * (g[6] * U0 + g[7] * U1 + g[8] * U2), 0.f);
        };
        // points one per lane in full warp passes; plane by plane (N >= 5) and without the
        // tensor-core products, the QR points left over share the warp, QS lanes each (strided
        // over the modes, then a butterfly sum): N = 5, 36 points, take 32 + 4 x 8 lanes
        constexpr int QI = PL ? NQ : NC, QF = QI / 32 * 32, QR = QI - QF;
        constexpr int QS = !PL || QR == 0 ? 1 : QR <= 2 ? 16 : QR <= 4 ? 8 : QR <= 8 ? 4 : QR <= 16 ? 2 : 1;
        const bool qsplit = QS > 1 && !A.vol;
        for (int qc = q0 + lane; qc < (qsplit ? q0 + QF : q1); qc += 32) {
          float pr[7];
          wprod(qc, 0, 1, pr);
          wout(qc, pr);
        }
        if (QS > 1 && qsplit) {
          const int qc = q0 + QF + lane / QS, part = lane % QS;
          float pr[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          if (qc < q1) wprod(qc, part, QS, pr);
#pragma unroll
          for (int o = QS / 2; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 7; ++c) pr[c] += __shfl_xor_sync(0xffffffffu, pr[c], o);
          if (qc < q1 && part == 0) wout(qc, pr);
        }
        __syncwarp();
        // Z of plane l overwrites Y of plane l, whose last reads precede the warp barrier above.
        // Items (mt, l) one per lane in full warp passes; plane by plane (N >= 5), the ZR items
        // left over share the warp, ZS lanes each (strided over the points, then a butterfly sum
        // over those lanes): N = 7, 36 items, takes 32 + 4 x 8 lanes instead of 32 + 4
        constexpr int ZI = NT * (PL ? 1 : N1), ZF = ZI / 32 * 32, ZR = ZI - ZF;
        constexpr int ZS = !PL || ZR == 0 ? 1 : ZR <= 2 ? 16 : ZR <= 4 ? 8 : ZR <= 8 ? 4 : ZR <= 16 ? 2 : 1;
        constexpr int ZL = ZS > 1 ? ZF : ZI;   // items taken one per lane
        auto zitem = [&](int x, int part, int step, float4& za, float& zr, float& zs) {
          const int mt = PL ? x : x / N1, l = PL ? lp : x % N1;
          const int xo = PL ? 0 : NQ * l;
#pragma unroll 5
          for (int qt = part; qt < NQ; qt += step) {
            const float4 v = DV4[qt * NT + mt], x1 = X1[qt + xo], x2 = X2[qt + xo];
            f4acc(za, v.x, x1);
            zr = fmaf(v.y, x2.x, fmaf(v.z, x2.z, zr));
            zs = fmaf(v.x, x2.y, zs);
          }
        };
        auto zstore = [&](int x, const float4& za, float zr, float zs) {
          const int mt = PL ? x : x / N1, l = PL ? lp : x % N1;
          ZA[mt * N1 + l] = za;
          ZB[mt * N1 + l] = f4(zr, zs, 0.f, 0.f);
        };
        for (int x = lane; x < ZL; x += 32) {
          float4 za = f4(0.f, 0.f, 0.f, 0.f);
          float zr = 0.f, zs = 0.f;
          zitem(x, 0, 1, za, zr, zs);
          zstore(x, za, zr, zs);
        }
        if constexpr (ZS > 1) {
          const int x = ZF + lane / ZS, part = lane % ZS;
          float4 za = f4(0.f, 0.f, 0.f, 0.f);
          float zr = 0.f, zs = 0.f;
          if (x < ZI) zitem(x, part, ZS, za, zr, zs);
#pragma unroll
          for (int o = ZS / 2; o > 0; o >>= 1) {
            za.x += __shfl_xor_sync(0xffffffffu, za.x, o);
            za.y += __shfl_xor_sync(0xffffffffu, za.y, o);
            za.z += __shfl_xor_sync(0xffffffffu, za.z, o);
            za.w += __shfl_xor_sync(0xffffffffu, za.w, o);
            zr += __shfl_xor_sync(0xffffffffu, zr, o);
            zs += __shfl_xor_sync(0xffffffffu, zs, o);
          }
          if (x < ZI && part == 0) zstore(x, za, zr, zs);
        }
        __syncwarp();
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = lane + 32 * r;
          if (n >= NP) break;
          const int mt = n % NT, j = n / NT;
          float u0 = 0.f, u1 = 0.f, u2 = 0.f, pp = 0.f;
#pragma unroll
          for (int l = 0; l < N1; ++l) {
            const float v1 = V1[l * N1 + j], d1 = D1[l * N1 + j];
            const float4 za = ZA[mt * N1 + l], zb = ZB[mt * N1 + l];
            u0 = fmaf(v1, za.x, u0);
            u1 = fmaf(v1, za.y, u1);
            u2 = fmaf(v1, za.z, u2);
            pp = fmaf(v1, zb.x - za.w, fmaf(d1, zb.y, pp));
          }
          acc[r] = f4(pp, -c2 * u0, -c2 * u1, -c2 * u2);
        }
      }
      // ---------------------------------------------------------------- face fluxes
      // In the fused modes (stage, multi-rate) the element's own trace (p, u.n) at a face with a
      // neighbour sits in the neighbour's inbox slot of the buffer read here: this element wrote it
      // at the end of its previous launch, from the state it starts from now (and dg_step begins
      // with a traces-only launch).  Elements without a wall face read it there instead of
      // evaluating their own face values.
      constexpr bool OWN_IN = T != DG_TET && (MODE == MODE_STAGE || MODE == MODE_MRC || MODE == MODE_MRF);
      bool inner = false;
      if (OWN_IN) {
        const int nbf = lane < NF ? A.nbr[A.side_off + e * NF + lane] : 0;
        inner = __all_sync(0xffffffffu, nbf >= 0);
      }
      face_ready();
      if (T != DG_TET && !inner) lattice_values();
      __syncwarp();
      {   // triangle-face points, then quad-face points: one kind per warp pass
        auto point = [&](int fq) {
          int f, ci;
          float4 tr, sg;
          if (inner) {   // face, canonical index and face data only
            if (LAT && fq < NLT) {
              f = face_of_tri<T>(fq / NFN);
              ci = tperm[code[f] * NFN + fq % NFN];
              sg = sg_at(f, 0);
            } else {
              const int x = LAT ? fq - NLT : fq, idx = x % NQ;
              f = LAT ? (T == DG_PYR ? 0 : 2 + x / NQ) : x / NQ;
              ci = (!LAT && tri_of<T>(f) >= 0) ? idx : qperm[code[f] * NQ + idx];
              sg = sg_at(f, idx);
            }
          } else if (LAT) {
            lat_point(fq, f, ci, tr, sg);
          } else {
            f = fq / NQ;
            const int idx = fq % NQ;
            tr = trace_at(f, idx);
            ci = tri_of<T>(f) >= 0 ? idx : qperm[code[f] * NQ + idx];
            sg = sg_at(f, idx);
          }
          const int64_t gs = A.side_off + e * NF + f;
          const int nb = A.nbr[gs];
          float pm, unm;
          if (inner) {
            pm = A.tin[(int64_t)nb * NQ + ci];
            unm = A.tin[A.plane + (int64_t)nb * NQ + ci];
          } else {
            pm = tr.x;
            unm = sg.x * tr.y + sg.y * tr.z + sg.z * tr.w;
          }
          float P = 0.f, UN = 0.f;
          if (nb >= 0) {
            P = A.tin[gs * NQ + ci];
            UN = A.tin[A.plane + gs * NQ + ci];
          }
          const float ta = A.tau[gs];
          float fp, fu;
          flux(nb < 0, pm, unm, P, UN, A.tau_scale * ta, A.tau_scale / ta, T != DG_TET && A.skew, fp, fu);
          F4[fq] = f4(sg.w * fp, sg.w * fu * sg.x, sg.w * fu * sg.y, sg.w * fu * sg.z);
        };
        constexpr int NTP = LAT ? NLT : NTRI * NQ;
        for (int fq = lane; fq < NTP; fq += 32) point(fq);
        for (int fq = NTP + lane; fq < NFX; fq += 32) point(fq);
      }
      __syncwarp();
      if (!LAT) {
        // lattice moments of the triangle-face fluxes, in local lattice order
        for (int x = lane; x < NTRI * NFN; x += 32) {
          const int ti = x / NFN, nl = x % NFN;
          const int f = face_of_tri<T>(ti);
          const int nc = tperm[code[f] * NFN + nl];
          float4 gsum = f4(0.f, 0.f, 0.f, 0.f);
          const float4* fr = F4 + f * NQ;
#pragma unroll 4
          for (int q = 0; q < NQ; ++q) f4acc(gsum, E[q * NFN + nc], fr[q]);
          G4[x] = gsum;
        }
        __syncwarp();
      }
      // ---------------------------------------------------------------- lift, M^{-1}, update
      float4* HB = W4;              // wedge: H_f[mt] = sum_nl phi_tri_mt(lattice_nl) G_f[nl]
      float4* PB = W4 + 2 * WNT;    // wedge: P_qf[ia][j] = sum_ib phi_1D_j(x_ib) F_qf[ia, ib]
      if (T == DG_WEDGE) {
        {
          auto item = [&](int x) {
            float4 v = f4(0.f, 0.f, 0.f, 0.f);
            if (x < 2 * WNT) {
              const int f = x / WNT, mt = x % WNT;
#pragma unroll 5
              for (int nl = 0; nl < NFN; ++nl) f4acc(v, Vtl[(f * NFN + nl) * WNT + mt], G4[f * NFN + nl]);
              HB[x] = v;
            } else {
              const int y = x - 2 * WNT, qf = y / (WN1 * WN1), ia = (y / WN1) % WN1, j = y % WN1;
#pragma unroll
              for (int ib = 0; ib < WN1; ++ib) f4acc(v, V1q[ib * WN1 + j], F4[(2 + qf) * NQ + ia + WN1 * ib]);
              PB[y] = v;
            }
          };
          for (int x = lane; x < 2 * WNT; x += 32) item(x);   // one kind of item per warp pass
          for (int x = 2 * WNT + lane; x < 2 * WNT + 3 * WN1 * WN1; x += 32) item(x);
        }
        __syncwarp();
      }
      if (T == DG_PYR) {
        // H_ti[kl] = sum_n PF2[ti][n][kl] F_ti[n] (G4); Wb[(k,j)][p] = sum_q LA[q][(k,j)] F_base[p, q] (PZB)
        constexpr int PN1 = C::N1;
        {
          auto item = [&](int x) {
            float4 v = f4(0.f, 0.f, 0.f, 0.f);
            if (x < NTRI * NKL) {
              const int ti = x / NKL, kl = x % NKL;
              const float* pf2 = PF2 + ti * NFN * NKL + kl;
#pragma unroll 5
              for (int n = 0; n < NFN; ++n) f4acc(v, pf2[n * NKL], F4[ti * NFN + n]);
              G4[x] = v;
            } else {
              const int y = x - NTRI * NKL, kl = y / PN1, pp = y % PN1;
#pragma unroll
              for (int qq = 0; qq < PN1; ++qq) f4acc(v, LA[qq * NKL + kl], F4[NLT + pp + PN1 * qq]);
              PZB[y] = v;
            }
          };
          for (int x = lane; x < NTRI * NKL; x += 32) item(x);   // one kind of item per warp pass
          for (int x = NTRI * NKL + lane; x < NTRI * NKL + NKL * PN1; x += 32) item(x);
        }
        __syncwarp();
      }
      // tets whose operators stay in global memory: the lattice lift operator crosses from L2 in
      // row chunks staged once per block iteration for all its warps (as the volume operator)
      float4 lsum[R];
      if constexpr (C::CHUNK && T == DG_TET) {
        constexpr int CL = 4 * C::CM;   // rows of NP floats per chunk
        float* schf = reinterpret_cast<float*>(sch);
#pragma unroll
        for (int r = 0; r < R; ++r) lsum[r] = f4(0.f, 0.f, 0.f, 0.f);
        for (int x0 = 0; x0 < NLT; x0 += CL) {
          const int xc = NLT - x0 < CL ? NLT - x0 : CL;
          __syncthreads();
          for (int y = threadIdx.x; y < xc * NP; y += blockDim.x) schf[y] = __ldg(Tn + (size_t)x0 * NP + y);
          __syncthreads();
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            if (n >= NP) break;
#pragma unroll 4
            for (int xx = 0; xx < xc; ++xx) f4acc(lsum[r], schf[xx * NP + n], F4[x0 + xx]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int n = lane + 32 * r;
        if (n >= NP) break;
        float4 sum = f4(0.f, 0.f, 0.f, 0.f);
        if (T == DG_PYR) {   // node (k, j, i): four triangle faces, then the base
          constexpr int PN1 = C::N1;
          int k = 0, j, i;
          if constexpr (C::PTAB) {
            const int d = pnd[n];
            k = d & 15, j = (d >> 4) & 15, i = d >> 8;
          } else {
            while ((k + 1) * (k + 2) * (2 * k + 3) / 6 <= n) ++k;
            const int r0 = n - k * (k + 1) * (2 * k + 1) / 6;
            j = r0 / (k + 1), i = r0 % (k + 1);
          }
          const int kb = k * (k + 1) / 2;
          f4acc(sum, EF[0 * NKL + kb + j], G4[0 * NKL + kb + i]);
          f4acc(sum, EF[1 * NKL + kb + i], G4[1 * NKL + kb + j]);
          f4acc(sum, EF[2 * NKL + kb + j], G4[2 * NKL + kb + i]);
          f4acc(sum, EF[3 * NKL + kb + i], G4[3 * NKL + kb + j]);
          float4 bsum = f4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int pp = 0; pp < PN1; ++pp) f4acc(bsum, LA[pp * NKL + kb + i], PZB[(kb + j) * PN1 + pp]);
          f4acc(sum, GC[k], bsum);
        } else if (T == DG_WEDGE) {   // node (mt, j): triangle faces, then quad faces (edge x 1D)
          const int mt = n % WNT, j = n / WNT;
          f4acc(sum, V1e[j], HB[mt]);
          f4acc(sum, V1e[WN1 + j], HB[WNT + mt]);
#pragma unroll
          for (int qf = 0; qf < 3; ++qf)
#pragma unroll
            for (int ia = 0; ia < WN1; ++ia)
              f4acc(sum, Ve[(qf * WN1 + ia) * WNT + mt], PB[(qf * WN1 + ia) * WN1 + j]);
        } else if constexpr (C::CHUNK) {   // tet, lift from the staged chunks above
          sum = lsum[r];
        } else {   // tet: lattice-point fluxes (Lf holds the face mass)
#pragma unroll 4
          for (int x = 0; x < NLT; ++x) f4acc(sum, Tn[x * NP + n], F4[x]);
        }
        float iM = 1.f;
        if (T == DG_TET) iM = 1.f / A.geo[e * 12 + 9];
        if (T == DG_PYR) iM = 1.f / A.geo[(e * 10 + 9) * NP + n];
        acc[r].x += iM * sum.x;
        acc[r].y += c2 * iM * sum.y;
        acc[r].z += c2 * iM * sum.z;
        acc[r].w += c2 * iM * sum.w;
      }
      if (!act) {
      } else if (MODE == MODE_RHS) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = lane + 32 * r;
          if (n >= NP) break;
          A.rhs[base + n] = acc[r].x;
          A.rhs[A.ndof + base + n] = acc[r].y;
          A.rhs[2 * A.ndof + base + n] = acc[r].z;
          A.rhs[3 * A.ndof + base + n] = acc[r].w;
        }
      } else if (MODE == MODE_STAGE) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = lane + 32 * r;
          if (n >= NP) break;
          const float rv[4] = {acc[r].x, acc[r].y, acc[r].z, acc[r].w};
          const float4 qo = q4[n];
          const float qv[4] = {qo.x, qo.y, qo.z, qo.w};
          float qn[4];
          const float dte = A.dtE ? A.dtE[e] : A.dt;
#pragma unroll
          for (int fl = 0; fl < 4; ++fl) {
            const int64_t id = fl * A.ndof + base + n;
            const float rr = A.a * A.res[id] + dte * rv[fl];
            qn[fl] = qv[fl] + A.b * rr;
            A.res[id] = rr;
            A.qout[id] = qn[fl];
          }
          acc[r] = f4(qn[0], qn[1], qn[2], qn[3]);
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = lane + 32 * r;
          if (n < NP) q4[n] = acc[r];
        }
        __syncwarp();
      } else {   // MRC / MRF: AB3 update; q4 <- prediction (MRC) or new state (MRF), acc <- new state
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = lane + 32 * r;
          if (n >= NP) break;
          const float rv[4] = {acc[r].x, acc[r].y, acc[r].z, acc[r].w};
          const float4 qo = q4[n];
          const float qv[4] = {qo.x, qo.y, qo.z, qo.w};
          float qn[4], qp[4];
#pragma unroll
          for (int fl = 0; fl < 4; ++fl) {
            const int64_t id = fl * A.ndof + base + n;
            const float r0 = rv[fl], r1 = A.h1[id], r2 = A.h2[id];
            A.hw[id] = r0;
            qn[fl] = qv[fl] + A.ab0 * r0 + A.ab1 * r1 + A.ab2 * r2;
            qp[fl] = qv[fl] + A.pr0 * r0 + A.pr1 * r1 + A.pr2 * r2;
            A.qout[id] = qn[fl];
          }
          acc[r] = f4(qn[0], qn[1], qn[2], qn[3]);
          pred[r] = f4(qp[0], qp[1], qp[2], qp[3]);
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int n = lane + 32 * r;
          if (n < NP) q4[n] = MODE == MODE_MRC ? pred[r] : acc[r];
        }
        __syncwarp();
      }
    }
    // traces of the state in q4 into the neighbours' inboxes
    auto emit = [&](float* tout) {
      face_ready();
      if (T != DG_TET) lattice_values();
      __syncwarp();
      {   // triangle-face points, then quad-face points: one kind per warp pass
        auto point = [&](int fq) {
          int f, ci;
          float4 tr, sg;
          if (LAT) {
            f = fq < NLT ? face_of_tri<T>(fq / NFN) : (T == DG_PYR ? 0 : 2 + (fq - NLT) / NQ);
          } else {
            f = fq / NQ;
          }
          const int64_t gs = A.side_off + e * NF + f;
          const int nb = A.nbr[gs];
          const int64_t dst = nb >= 0 ? (int64_t)nb : ((MODE == MODE_TRACE && A.wall_self) ? gs : -1);
          if (dst < 0) return;
          if (LAT) {
            lat_point(fq, f, ci, tr, sg);
          } else {
            const int idx = fq % NQ;
            tr = trace_at(f, idx);
            ci = tri_of<T>(f) >= 0 ? idx : qperm[code[f] * NQ + idx];
            sg = sg_at(f, idx);
          }
          tout[dst * NQ + ci] = tr.x;
          tout[A.plane + dst * NQ + ci] = sg.x * tr.y + sg.y * tr.z + sg.z * tr.w;
        };
        constexpr int NTP = LAT ? NLT : NTRI * NQ;
        for (int fq = lane; fq < NTP; fq += 32) point(fq);
        for (int fq = NTP + lane; fq < NFX; fq += 32) point(fq);
      }
      __syncwarp();
    };
    // (multi-rate coarse step: the half-step traces only where a fine neighbour reads them)
    if (MODE != MODE_RHS && act && (MODE != MODE_MRC || !A.pred || A.pred[e])) emit(A.tout);
    if (MODE == MODE_MRC && act) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int n = lane + 32 * r;
        if (n < NP) q4[n] = acc[r];
      }
      __syncwarp();
      emit(A.tout2);
    }
    __syncwarp();
  }
}

template <int T, int N, int MODE>
static bool launch_one(const Args& A, cudaStream_t s) {
  using C = G2<T, N>;
  if constexpr (N > 4 && (MODE == MODE_MRC || MODE == MODE_MRF)) {
    return false;   // the fused multi-rate modes exist for N <= 4 only (not instantiated above)
  } else {
  if (A.nops2 != C::NOPS) return false;   // host operator layout of another (type, N)
  static int blocks = 0;   // persistent grid: resident blocks per SM x SMs (computed once)
  if (blocks == 0) {
    if (cudaFuncSetAttribute(gen2_kernel<T, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) !=
        cudaSuccess)
      return false;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gen2_kernel<T, N, MODE>, C::NW * 32, C::SMEM);
    if (per < 1) return false;
    blocks = per * sms;
  }
  const int64_t need = ((int64_t)A.K + C::NW - 1) / C::NW;
  const int grid = (int)(need < blocks ? need : blocks);
  gen2_kernel<T, N, MODE><<<grid, C::NW * 32, C::SMEM, s>>>(A);
  return true;
  }
}

template <int MODE>
bool launch_gen2(int t, int N, const Args& A, cudaStream_t s) {
  if (A.K == 0) return true;
  if (!A.ops2) return false;
  switch (N) {
#define G2_CASE(NN)                                                        \
  case NN:                                                                 \
    if (t == DG_TET) return launch_one<DG_TET, NN, MODE>(A, s);            \
    if (t == DG_PYR) return launch_one<DG_PYR, NN, MODE>(A, s);            \
    if (t == DG_WEDGE) return launch_one<DG_WEDGE, NN, MODE>(A, s);        \
    return false;
    G2_CASE(1) G2_CASE(2) G2_CASE(3) G2_CASE(4) G2_CASE(5) G2_CASE(6) G2_CASE(7) G2_CASE(8) G2_CASE(9)
#undef G2_CASE
    default: return false;
  }
}

template bool launch_gen2<MODE_TRACE>(int, int, const Args&, cudaStream_t);
template bool launch_gen2<MODE_RHS>(int, int, const Args&, cudaStream_t);
template bool launch_gen2<MODE_STAGE>(int, int, const Args&, cudaStream_t);
template bool launch_gen2<MODE_MRC>(int, int, const Args&, cudaStream_t);
template bool launch_gen2<MODE_MRF>(int, int, const Args&, cudaStream_t);

}  // namespace dgk
