// Tensor-core tetrahedron kernel (sm_103a): 5th-generation tensor cores (tcgen05.mma, TF32 with a
// three-term split for FP32 accuracy, accumulators in tensor memory).
//
// With the lattice-point face exchange (kernels_gen2.cu), the whole right-hand side of a tet is one
// product of a fixed operator with a per-element vector:
//   rhs_f[n] = sum_k Op[n][k] X_f[k],   Op = [ D^r | D^s | D^t | Lf ]   (NP x (3 NP + 4 NFN))
// where, with the constant metrics G = d(rst)/d(xyz), J and c^2 of the element (Alg. tet_vol),
//   X_p  = [ -w_r, -w_s, -w_t, F_p / J ],            w_a = G[a][0] u + G[a][1] v + G[a][2] w
//   X_ud = [ -c^2 G[a][d] p (a = r,s,t),  c^2 F_ud / J ]
// and F holds the J^s-scaled upwind fluxes at the face-lattice nodes (Sec. 2.2; Lf folds the face
// mass and M_hat^{-1}).  The metric terms are applied on the input side because they are constant
// per element.
//
// A persistent block of 16 warps owns all 512 columns of the SM's tensor memory and walks over
// tiles of 32 elements: TMEM lane r = 4 (element) + field holds X (hi and lo TF32 parts, written by
// tcgen05.st); the operator (hi, lo) sits in shared memory in the K-major canonical layout; one
// thread issues D = X_hi Op_hi + X_hi Op_lo + X_lo Op_hi (3 x K/8 MMAs of 128 x NPP x 8) and
// commits them to an mbarrier; the accumulators come back with tcgen05.ld and go through shared
// memory so that the update and the trace writes are coalesced.  Two staging buffers: the copies
// of tile i+1 (state, side data, inbox values) are issued as soon as tile i's flux phase is done,
// so they land while tile i's operands, products, update and traces run; tile i's residual /
// history rows are loaded into registers before its products and used by its update.  The waits
// are bounded (~1 s of SM clock); on a timeout the block reports through the device error word,
// lets its copies in flight complete and stops.
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace dgk {

namespace {

__device__ __forceinline__ unsigned su32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ float tf32r(float x) {
  unsigned u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}
// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte stride between core matrices
// along K, sbo = byte stride between 8-row groups; bit 46 = descriptor version of tcgen05
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFF) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (static_cast<uint64_t>(1) << 46);
}
__device__ __forceinline__ void mma_tf32(unsigned d, unsigned a, uint64_t b, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_st8(unsigned taddr, const unsigned (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(unsigned taddr, unsigned (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = su32(bar);
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

constexpr int a128(int x) { return (x + 127) / 128 * 128; }
constexpr int pow2_cols(int x) { return x <= 32 ? 32 : x <= 64 ? 64 : x <= 128 ? 128 : x <= 256 ? 256 : 512; }

}  // namespace

template <int N>
struct TetTC {
  static constexpr int NP = (N + 1) * (N + 2) * (N + 3) / 6, NFN = (N + 1) * (N + 2) / 2, NQ = (N + 1) * (N + 1);
  static constexpr int TE = 32, NT = 512;                 // elements per tile (128 TMEM lanes), threads
  static constexpr int KV = 3 * NP, KL = 4 * NFN;         // volume and lift columns of X
  // K layout: each of the blocks D^r, D^s, D^t, Lf padded to a multiple of the MMA's 8, so that an
  // 8-column chunk of X lies in one block
  static constexpr int NP8 = (NP + 7) / 8 * 8, KL8 = (KL + 7) / 8 * 8;
  static constexpr int KV8 = 3 * NP8;
  static constexpr int KP = KV8 + KL8;
  static constexpr int NPP = (NP + 15) / 16 * 16;         // MMA N: multiple of 16 for M = 128
  static constexpr int XHI = 0, XLO = KP, DCOL = 2 * KP;  // tensor-memory columns
  static constexpr int TCOLS = pow2_cols(DCOL + NPP);
  static_assert(DCOL + NPP <= 512, "tile does not fit tensor memory");
  static constexpr int NJ = (NP + 3) / 4;                 // values per thread of a (element, field) row
  static constexpr int OPB = NPP * KP * 4;                // one operator copy (bytes)
  static constexpr int S_OPH = 0, S_OPL = a128(OPB);
  static constexpr int S_R = S_OPL + a128(OPB);            // [TE][4][NP] rhs (MRC: new state); -w_a before
  static constexpr int S_F = S_R + a128(TE * 4 * NP * 4);  // [TE][4 comps][KL + 1] lattice fluxes
  static constexpr int S_I = S_F + a128(TE * 4 * (KL + 1) * 4);   // tperm [6][NFN], fnode [4][NFN]
  static constexpr int S_BUF = a128(S_I + 10 * NFN * 4);   // two tile buffers: tile i+1 lands while i runs
  static constexpr int B_Q = 0;                             // [TE][4][NP] state
  static constexpr int B_G = a128(TE * 4 * NP * 4);         // [TE][16]: G[9], J, -, -, c^2
  static constexpr int B_SD = B_G + TE * 16 * 4;            // [TE][4] code, [TE][4] nbr, [TE][4] tau, [TE] element
  static constexpr int B_N = a128(B_SD + TE * 13 * 4);      // [TE][4] float4 (n, J^s) of the faces
  static constexpr int B_IN = B_N + TE * 4 * 16;            // [TE][4][2][NFN] inbox lattice values
  static constexpr int BUFB = a128(B_IN + TE * 8 * NFN * 4);
  static constexpr int S_BAR = S_BUF + 2 * BUFB;
  static constexpr int SMEM = S_BAR + 16;
  static_assert(SMEM <= 227 * 1024, "tet tile buffers exceed shared memory");
};

__device__ __forceinline__ void cpa4(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(sdst)), "l"(gsrc) : "memory");
}

// One tile's staging buffer in shared memory.
template <int N>
struct TetBuf {
  float* q;
  float* g;
  int *code, *nb, *e;
  float* tau;
  float4* n;
  float* in;
  __device__ TetBuf(unsigned char* base) {
    using C = TetTC<N>;
    q = reinterpret_cast<float*>(base + C::B_Q);
    g = reinterpret_cast<float*>(base + C::B_G);
    code = reinterpret_cast<int*>(base + C::B_SD);
    nb = code + 4 * C::TE;
    tau = reinterpret_cast<float*>(nb + 4 * C::TE);
    e = reinterpret_cast<int*>(tau + 4 * C::TE);
    n = reinterpret_cast<float4*>(base + C::B_N);
    in = reinterpret_cast<float*>(base + C::B_IN);
  }
};

// Every global read of a tile except the residual / history, as asynchronous copies (one commit
// group): state, metrics and c^2, side data, face (n, J^s), inbox lattice values.  Rows
// (element, field) of NP contiguous values, 4 threads per row; absent elements are zero-filled.
template <int N>
__device__ __forceinline__ void tet_issue_tile(const Args& A, const TetBuf<N>& B, int tid) {
  using C = TetTC<N>;
  constexpr int NP = C::NP, NFN = C::NFN, NQ = C::NQ, TE = C::TE;
  {
    const int row = tid >> 2, sub = tid & 3, el = row >> 2, f = row & 3;
    const int e = B.e[el];
    if (e >= 0) {
      const float* src = A.q + f * A.ndof + A.dof_off + (int64_t)e * NP;
      for (int n = sub; n < NP; n += 4) cpa4(B.q + row * NP + n, src + n);
    } else {
      for (int n = sub; n < NP; n += 4) B.q[row * NP + n] = 0.f;
    }
  }
  if (tid < TE * 16) {
    const int el = tid >> 4, i = tid & 15;
    const int e = B.e[el];
    if (i < 13) {
      if (e >= 0) cpa4(B.g + el * 16 + i, i < 12 ? A.geo + (int64_t)e * 12 + i : A.c2 + e);
      else B.g[el * 16 + i] = i == 9 ? 1.f : 0.f;
    }
  }
  if (tid < TE * 4) {
    const int e = B.e[tid >> 2];
    if (e >= 0) {
      const int64_t gs = A.side_off + (int64_t)e * 4 + (tid & 3);
      cpa4(B.code + tid, A.code + gs);
      cpa4(B.nb + tid, A.nbr + gs);
      cpa4(B.tau + tid, A.tau + gs);
      cpa16(B.n + tid, A.sgeo2 + ((int64_t)e * 4 + (tid & 3)) * NQ);
    } else {
      B.code[tid] = 0;
      B.nb[tid] = -1;
      B.tau[tid] = 1.f;
      B.n[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  {   // inbox lattice slots: rows (element, face, plane) of NFN values, 2 threads per row
    const int row = tid >> 1, sub = tid & 1, el = row >> 3, f = (row >> 1) & 3, pl = row & 1;
    const int e = B.e[el];
    if (e >= 0) {
      const float* src = A.tin + pl * A.plane + (A.side_off + (int64_t)e * 4 + f) * NQ;
      for (int c = sub; c < NFN; c += 2) cpa4(B.in + row * NFN + c, src + c);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N, int MODE>
__global__ void __launch_bounds__(512, 1) tet_tc_kernel(Args A) {
  using C = TetTC<N>;
  constexpr int NP = C::NP, NFN = C::NFN, NQ = C::NQ, TE = C::TE, NT = C::NT, KV = C::KV, KL = C::KL, KP = C::KP,
                NPP = C::NPP, NJ = C::NJ;
  constexpr int NAUX = MODE == MODE_STAGE ? 1 : (MODE == MODE_MRC || MODE == MODE_MRF) ? 2 : 0;
  extern __shared__ __align__(1024) unsigned char sm[];
  float* opH = reinterpret_cast<float*>(sm + C::S_OPH);
  float* opL = reinterpret_cast<float*>(sm + C::S_OPL);
  float* sr = reinterpret_cast<float*>(sm + C::S_R);
  float* sfc = reinterpret_cast<float*>(sm + C::S_F);
  int* stp = reinterpret_cast<int*>(sm + C::S_I);
  int* sfn = stp + 6 * NFN;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + C::S_BAR);
  unsigned* stm = reinterpret_cast<unsigned*>(sm + C::S_BAR + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // operator Op[n][k] (hi, lo) from the tet operators of the warp kernels:
  // DV4 [NP][NP] = (D^r, D^s, D^t, 0)[n][m] | Lf [4 NFN][NP]; element (n, k) of the K-major canonical
  // layout sits in core matrix (n / 8, k / 4), core matrices ordered K-block-major
  {
    const float4* DV4 = reinterpret_cast<const float4*>(A.ops2);
    const float* Lf = A.ops2 + 4 * NP * NP;
    for (int x = tid; x < NPP * KP; x += NT) {
      const int n = x / KP, k = x % KP;
      float v = 0.f;
      if (n < NP) {
        if (k < C::KV8) {
          const int a = k / C::NP8, m = k - a * C::NP8;
          if (m < NP) {
            const float4 d = DV4[n * NP + m];
            v = a == 0 ? d.x : a == 1 ? d.y : d.z;
          }
        } else if (k - C::KV8 < KL) {
          v = Lf[(k - C::KV8) * NP + n];
        }
      }
      const float h = tf32r(v);
      const int o = ((k >> 2) * (NPP / 8) + (n >> 3)) * 32 + (n & 7) * 4 + (k & 3);
      opH[o] = h;
      opL[o] = tf32r(v - h);
    }
    for (int x = tid; x < 6 * NFN; x += NT) stp[x] = A.iops2[x];
    for (int x = tid; x < 4 * NFN; x += NT) sfn[x] = A.iops2[12 * NFN + 8 * NQ + x];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(stm)), "r"(C::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int ntiles = (A.K + TE - 1) / TE;
  auto tile_elem = [&](int tile, int i) -> int {
    const int li = tile * TE + i;
    return tile < ntiles && li < A.K ? (A.elist ? A.elist[li] : li) : -1;
  };
  {   // the first tile's copies start before the block's set-up completes
    TetBuf<N> B0(sm + C::S_BUF);
    if (tid < TE) B0.e[tid] = tile_elem(blockIdx.x, tid);
    __syncthreads();
    if (blockIdx.x < ntiles) tet_issue_tile<N>(A, B0, tid);
  }
  int pe = tid < TE ? tile_elem(blockIdx.x + gridDim.x, tid) : -1;   // element ids one tile ahead
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operator visible to the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tb = *stm;
  unsigned phase = 0;
  bool bail = false;
  // instruction descriptor: D f32, A and B tf32, both K-major, N = NPP, M = 128
  constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(NPP >> 3) << 17) | (8u << 24);
  constexpr unsigned LBO = (NPP / 8) * 128, SBO = 128;
  const int q4 = warp & 3, wq = warp >> 2;   // TMEM lane quarter of this warp; column share
  const unsigned lanebase = tb + ((unsigned)(q4 * 32) << 16);

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles && !bail; tile += gridDim.x, ++it) {
    const TetBuf<N> B(sm + C::S_BUF + (it & 1) * C::BUFB);
    const TetBuf<N> BN(sm + C::S_BUF + ((it & 1) ^ 1) * C::BUFB);
    const int next = tile + gridDim.x;
    if (tid < TE) BN.e[tid] = pe;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // ---- per element: 16 threads; fluxes at the 4 NFN face-lattice nodes (strong form, scaled
    // by J^s, component planes) and the metric-transformed velocities -w_a (into sr)
    {
      const int el = tid >> 4, t16 = tid & 15;
      const int e = B.e[el];
      const float* qe = B.q + el * 4 * NP;
      float* fe = sfc + el * 4 * (KL + 1);
      for (int y = t16; y < KL; y += 16) {
        const int f = y / NFN, nl = y - f * NFN;
        float fp = 0.f, fu = 0.f;
        const float4 sgv = B.n[el * 4 + f];   // (n, J^s), constant on the face
        if (e >= 0) {
          const int node = sfn[y];
          const float pm = qe[node];
          const float unm = sgv.x * qe[NP + node] + sgv.y * qe[2 * NP + node] + sgv.z * qe[3 * NP + node];
          const int nb = B.nb[el * 4 + f];
          float P = 0.f, UN = 0.f;
          if (nb >= 0) {
            const int ci = stp[B.code[el * 4 + f] * NFN + nl];
            P = B.in[(el * 8 + f * 2) * NFN + ci];
            UN = B.in[(el * 8 + f * 2 + 1) * NFN + ci];
          }
          const float ta = B.tau[el * 4 + f];
          flux(nb < 0, pm, unm, P, UN, A.tau_scale * ta, A.tau_scale / ta, false, fp, fu);
        }
        fe[y] = sgv.w * fp;
        fe[(KL + 1) + y] = sgv.w * fu * sgv.x;
        fe[2 * (KL + 1) + y] = sgv.w * fu * sgv.y;
        fe[3 * (KL + 1) + y] = sgv.w * fu * sgv.z;
      }
      const float* G = B.g + el * 16;
      float* we = sr + el * KV;
      for (int m = t16; m < NP; m += 16) {
        const float u = qe[NP + m], v = qe[2 * NP + m], w = qe[3 * NP + m];
#pragma unroll
        for (int a = 0; a < 3; ++a) we[a * NP + m] = -(G[3 * a] * u + G[3 * a + 1] * v + G[3 * a + 2] * w);
      }
    }
    __syncthreads();
    // ---- the next tile's copies run while this tile's products and update proceed; the residual /
    // history rows of this tile come into registers (used by the update)
    if (next < ntiles) tet_issue_tile<N>(A, BN, tid);
    if (tid < TE) pe = tile_elem(next + gridDim.x, tid);
    const int urow = tid >> 2, usub = tid & 3, uel = urow >> 2, uf = urow & 3;
    const int ue = B.e[uel];
    const int64_t ug0 = uf * A.ndof + A.dof_off + (int64_t)(ue >= 0 ? ue : 0) * NP;
    float ax[NAUX > 0 ? NAUX : 1][NJ];
    if (NAUX > 0) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int n = usub + 4 * j;
        const bool ok = ue >= 0 && n < NP;
        ax[0][j] = ok ? (MODE == MODE_STAGE ? A.res : A.h1)[ug0 + n] : 0.f;
        if (NAUX > 1) ax[NAUX - 1][j] = ok ? A.h2[ug0 + n] : 0.f;
      }
    }
    // ---- X rows (hi, lo) into tensor memory: lane r = 4 el + field, 8-column chunks shared by
    // the four warps of each lane quarter.  p row: [-w_r, -w_s, -w_t, F_p / J];
    // u_d rows: [-c^2 G[a][d] p (a = r,s,t), c^2 F_d / J]
    {
      const int row = q4 * 32 + lane, el = row >> 2, fld = row & 3;
      const float* G = B.g + el * 16;
      const float iJ = 1.f / G[9], c2 = G[12];
      const float sl = fld == 0 ? iJ : c2 * iJ;
      const int d = fld == 0 ? 0 : fld - 1;
      const float cf0 = -c2 * G[d], cf1 = -c2 * G[3 + d], cf2 = -c2 * G[6 + d];
      const float* fsrc = sfc + row * (KL + 1);                           // lift source row
      for (int ch = wq; ch < KP / 8; ch += 4) {
        // the chunk's block: volume a (source, scale, first node) or the lift
        const bool vol = ch < C::KV8 / 8;
        const int a = vol ? ch / (C::NP8 / 8) : 0;
        const int m0 = vol ? (ch - a * (C::NP8 / 8)) * 8 : ch * 8 - C::KV8;
        const int lim = vol ? NP : KL;
        const float mul = vol ? (fld == 0 ? 1.f : (a == 0 ? cf0 : a == 1 ? cf1 : cf2)) : sl;
        const float* src = vol ? (fld == 0 ? sr + el * KV + a * NP : B.q + el * 4 * NP) : fsrc;
        unsigned vh[8], vl[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float v = m0 + c < lim ? mul * src[m0 + c] : 0.f;
          const float h = tf32r(v);
          vh[c] = __float_as_uint(h);
          vl[c] = __float_as_uint(tf32r(v - h));
        }
        tmem_st8(lanebase + C::XHI + ch * 8, vh);
        tmem_st8(lanebase + C::XLO + ch * 8, vl);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // ---- D = X_hi Op_hi + X_hi Op_lo + X_lo Op_hi
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned ah0 = su32(opH), al0 = su32(opL);
#pragma unroll 1
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint64_t bh = smem_desc(ah0 + ks * 2 * LBO, LBO, SBO), bl = smem_desc(al0 + ks * 2 * LBO, LBO, SBO);
        mma_tf32(tb + C::DCOL, tb + C::XHI + ks * 8, bh, IDESC, ks > 0);
        mma_tf32(tb + C::DCOL, tb + C::XHI + ks * 8, bl, IDESC, 1u);
        mma_tf32(tb + C::DCOL, tb + C::XLO + ks * 8, bh, IDESC, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                   : "memory");
    }
    if (!__syncthreads_and(bar_wait(bar, phase))) {
      bail = true;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- accumulators -> shared memory
    {
      const int row = q4 * 32 + lane;
      for (int ch = wq; ch < NPP / 8; ch += 4) {
        unsigned v[8];
        tmem_ld8(lanebase + C::DCOL + ch * 8, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int n = ch * 8 + c;
          if (n < NP) sr[row * NP + n] = __uint_as_float(v[c]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // ---- update: rows (element, field), 4 threads per row
    if (ue >= 0) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int n = usub + 4 * j;
        if (n >= NP) break;
        const int x = urow * NP + n;
        const int64_t id = ug0 + n;
        const float rv = sr[x], qo = B.q[x];
        if (MODE == MODE_RHS) {
          A.rhs[id] = rv;
        } else if (MODE == MODE_STAGE) {
          const float rr = A.a * ax[0][j] + (A.dtE ? A.dtE[ue] : A.dt) * rv;
          const float qn = qo + A.b * rr;
          A.res[id] = rr;
          A.qout[id] = qn;
          B.q[x] = qn;
        } else {   // MRC / MRF: AB3; MRC: prediction -> B.q, new state -> sr
          const float r1 = ax[0][j], r2 = ax[NAUX - 1][j];
          A.hw[id] = rv;
          const float qn = qo + A.ab0 * rv + A.ab1 * r1 + A.ab2 * r2;
          A.qout[id] = qn;
          if (MODE == MODE_MRC) {
            B.q[x] = qo + A.pr0 * rv + A.pr1 * r1 + A.pr2 * r2;
            sr[x] = qn;
          } else {
            B.q[x] = qn;
          }
        }
      }
    }
    __syncthreads();
    // ---- traces of the new state (MRC: prediction, then new state) into the neighbours' inboxes
    if (MODE != MODE_RHS) {
      const int el = tid >> 4, t16 = tid & 15;
      const int e = B.e[el];
#pragma unroll 1
      for (int pass = 0; pass < (MODE == MODE_MRC ? 2 : 1); ++pass) {
        const float* qe = (pass ? sr : B.q) + el * 4 * NP;
        float* tout = pass ? A.tout2 : A.tout;
        // (multi-rate coarse step: the half-step traces only where a fine neighbour reads them)
        const bool em = e >= 0 && (MODE != MODE_MRC || pass == 1 || !A.pred || A.pred[e]);
        for (int y = t16; y < KL && em; y += 16) {
          const int f = y / NFN, nl = y - f * NFN;
          const int nb = B.nb[el * 4 + f];
          if (nb < 0) continue;
          const int node = sfn[y];
          const float4 sgv = B.n[el * 4 + f];
          const int ci = stp[B.code[el * 4 + f] * NFN + nl];
          tout[(int64_t)nb * NQ + ci] = qe[node];
          tout[A.plane + (int64_t)nb * NQ + ci] =
              sgv.x * qe[NP + node] + sgv.y * qe[2 * NP + node] + sgv.z * qe[3 * NP + node];
        }
      }
    }
    __syncthreads();
  }
  // copies still in flight (a bail-out, or none) complete before the block exits
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (bail) {   // report; wait (bounded) for the MMAs in flight before freeing tensor memory
    if (tid == 0) atomicOr(A.err, 1);
    bar_wait(bar, phase);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(C::TCOLS) : "memory");
}

template <int N, int MODE>
static void launch_tet_tc_n(const Args& A, cudaStream_t s) {
  using C = TetTC<N>;
  static int sms = 0;
  if (sms == 0) {
    cudaFuncSetAttribute(tet_tc_kernel<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int ntiles = (A.K + C::TE - 1) / C::TE;
  tet_tc_kernel<N, MODE><<<ntiles < sms ? ntiles : sms, C::NT, C::SMEM, s>>>(A);
}

// Tets through the tensor cores: rhs, LSRK stage and the fused multi-rate modes, N <= 4.
template <int MODE>
bool launch_tet_tc(int N, const Args& A, cudaStream_t s) {
  if (MODE == MODE_TRACE || A.K == 0 || !A.ops2) return false;
  switch (N) {
    case 1: launch_tet_tc_n<1, MODE>(A, s); return true;
    case 2: launch_tet_tc_n<2, MODE>(A, s); return true;
    case 3: launch_tet_tc_n<3, MODE>(A, s); return true;
    case 4: launch_tet_tc_n<4, MODE>(A, s); return true;
    default: return false;
  }
}

// Watchdog self-test: a bounded wait on an mbarrier that nothing arrives on; the timeout is
// recorded in the device error word as in the production kernels.
__global__ void watchdog_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const unsigned a = su32(&bar);
  const long long t0 = clock64();
  unsigned done = 0;
  while (!done && clock64() - t0 < limit)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a)
        : "memory");
  if (!__syncthreads_or(done == 0) || threadIdx.x != 0) return;
  atomicOr(err, 1);
}

cudaError_t launch_watchdog(int* err, long long limit, cudaStream_t s) {
  watchdog_kernel<<<1, 32, 0, s>>>(err, limit);
  return cudaGetLastError();
}

template bool launch_tet_tc<MODE_TRACE>(int, const Args&, cudaStream_t);
template bool launch_tet_tc<MODE_RHS>(int, const Args&, cudaStream_t);
template bool launch_tet_tc<MODE_STAGE>(int, const Args&, cudaStream_t);
template bool launch_tet_tc<MODE_MRC>(int, const Args&, cudaStream_t);
template bool launch_tet_tc<MODE_MRF>(int, const Args&, cudaStream_t);

}  // namespace dgk
