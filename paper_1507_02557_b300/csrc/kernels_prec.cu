// Tensor-core volume terms of tetrahedra, pyramids and wedges in split 16-bit precision (sm_103a).
//
// The volume terms of tets and pyramids are products of fixed reference operators with per-element
// vectors (Alg. tet_vol, Sec. 2.3.2; Alg. pyr_vol, Sec. 2.3.4).  Per element, with the metric
// terms G = d(rst)/d(xyz) (tet: constant; pyramid: at the semi-nodal points, with J):
//   X = [ W_r | W_s | W_t | p ],   W_a = (G u)_a (tet),  W_a = J (G u)_a (pyramid)
//   Y = [ sum_a D^a W_a | D^r p | D^s p | D^t p ]          (pyramid: (D^a)^T in the first block)
// i.e. Y = B X with a fixed block operator B (4 NP x 4 NP, half of its blocks zero).  The
// warp-per-element kernels (kernels_gen2.cu) then form -div u and -c^2 grad p from Y at the
// nodes and add the face terms as before.
//
// Precision: X and B are split into 16-bit parts, x = x_hi + x_lo with x_hi = rn16(x) and
// x_lo = rn16(x - x_hi), and the product is formed as X_hi B_hi + X_hi B_lo + X_lo B_hi in FP32
// (the lo x lo term is dropped): BF16 (8 significant bits per part; about 2^-17 relative per
// product) or FP16 (11 bits per part; about 2^-22, FP32-class).  The published technique is the
// split-precision emulation of Markidis et al. (2018) and Ootomo & Yokota (2022).  Every row of X
// and the operator are scaled by powers of two so that their largest entries lie in [2^14, 2^15):
// FP16's range then holds the hi and lo parts of all entries that matter (the scaling is exact).
//
// Three kernels per launch group:
//   pack_kernel   one warp per element: X (scaled, hi and lo) and 1 / scale of the row
//   vgemm_kernel  one CTA per (128-row tile, output block): TMA loads the 16-bit operand slabs
//                 (boxes of 8 K-values x rows, i.e. the K-major core matrices of the MMA),
//                 one thread issues tcgen05.mma.kind::f16 (M = 128, N = NP padded to 16,
//                 K = 16) into a tensor-memory accumulator, the four warps read it back with
//                 tcgen05.ld and store Y = acc / (scale_row scale_B) in FP32
//   gen2_kernel   (kernels_gen2.cu) with Args.vol = Y
// The output blocks of B are the four column blocks of Y: block 0 reads the W part of X (K =
// 3 NPK), blocks 1..3 the p part (K = NPK), so the zero blocks of B are never multiplied.
// Wedges at N >= 7 (Alg. wedge_vol1/2, Sec. 2.3.3, sum-factorised over triangle x 1D): the first
// of their two contractions, triangle modes -> triangle cubature points, runs here on rows
// (element, 1D level): wpack_kernel forms the level's triangle-mode vectors, vgemm_kernel the
// seven products (seven output blocks of B, each reading one vector); the wedge warp kernel takes
// them as its cubature-point values and does the metric terms and the second contraction.
// Every mbarrier wait is bounded (~1 s of SM clock); on a timeout the CTA sets bit 0 of the
// device error word, waits (bounded) for its copies and MMAs in flight and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace dgk {

namespace {

__device__ __forceinline__ unsigned sa32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

template <bool BF>
__device__ __forceinline__ unsigned short rn16(float x) {
  if constexpr (BF) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  else return __half_as_ushort(__float2half_rn(x));
}
template <bool BF>
__device__ __forceinline__ float f16f(unsigned short h) {
  if constexpr (BF) return __bfloat162float(__ushort_as_bfloat16(h));
  else return __half2float(__ushort_as_half(h));
}

// K-major shared-memory matrix descriptor without swizzle: lbo = bytes between core matrices
// adjacent in K, sbo = bytes between 8-row groups; bit 46: tcgen05 descriptor version
__device__ __forceinline__ uint64_t kdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFF) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (static_cast<uint64_t>(1) << 46);
}
__device__ __forceinline__ void mma_f16(unsigned d, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tld8(unsigned taddr, unsigned (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void bar_init(uint64_t* b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa32(b)), "r"(bytes) : "memory");
}
// phase `parity` of an mbarrier completed; false after ~2^31 SM clocks
__device__ __forceinline__ bool bar_wait_b(uint64_t* b, unsigned parity) {
  const unsigned a = sa32(b);
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
__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          sa32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sa32(b))
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa32(b)) : "memory");
}

}  // namespace

// ---------------------------------------------------------------------------- X = [W_r W_s W_t p]
template <int T, int N, bool BF>
__global__ void __launch_bounds__(256) pack_kernel(Args A, PrecDev P) {
  constexpr int NP = np_of(T, N);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int npk = P.npk, kx = 4 * npk;
  for (int64_t li = w0; li < A.K; li += nw) {
    const int64_t e = A.elist ? (int64_t)A.elist[li] : li;
    const int64_t base = A.dof_off + e * NP;
    const float* gt = A.geo + e * 12;
    // the four blocks of X at node m (lane-strided); first pass: the row's largest magnitude
    auto value = [&](int k) -> float {
      const int blk = k / npk, m = k - blk * npk;
      if (m >= NP) return 0.f;
      if (blk == 3) return A.q[base + m];
      const float u = A.q[A.ndof + base + m], v = A.q[2 * A.ndof + base + m], w = A.q[3 * A.ndof + base + m];
      if (T == DG_TET) return gt[3 * blk] * u + gt[3 * blk + 1] * v + gt[3 * blk + 2] * w;
      const float* g = A.geo + e * 10 * NP + m;   // [10][NP] per element
      return g[9 * NP] * (g[3 * blk * NP] * u + g[(3 * blk + 1) * NP] * v + g[(3 * blk + 2) * NP] * w);
    };
    float mx = 0.f;
    for (int k = lane; k < kx; k += 32) mx = fmaxf(mx, fabsf(value(k)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // scale = 2^(14 - floor(log2 mx)): the largest entry lands in [2^14, 2^15)
    const float s = mx > 0.f ? ldexpf(1.f, 14 - ilogbf(mx)) : 1.f;
    unsigned short* xh = P.xh + li * kx;
    unsigned short* xl = P.xl + li * kx;
    for (int k = lane; k < kx; k += 32) {
      const float v = s * value(k);
      const unsigned short h = rn16<BF>(v);
      xh[k] = h;
      xl[k] = rn16<BF>(v - f16f<BF>(h));
    }
    if (lane == 0) P.xis[li] = 1.f / s;
  }
}

// ---------------------------------------------------------------------------- wedges
// Rows (element li, 1D level l): the triangle-mode vectors of the first factor of the wedge's
// sum-factorised volume terms (Alg. wedge_vol1/2): y_f[mt] = sum_j V1[l][j] q_f[mt + NT j] for the
// four fields and y_s[mt] = sum_j D1[l][j] p[mt + NT j], laid out [y_p | y_s | y_u | y_v | y_w]
// (blocks of NPK); Y = B X then holds, per row, the seven cubature-point products of level l
// (V y_p, V_r y_p, V_t y_p, V y_s, V y_u, V y_v, V y_w at the NQ triangle points).
template <int N, bool BF>
__global__ void __launch_bounds__(256) wpack_kernel(Args A, PrecDev P) {
  constexpr int N1 = N + 1, NT = N1 * (N + 2) / 2, NP = NT * N1, NQ = N1 * N1;
  constexpr int NPK = (NT + 15) / 16 * 16, KX = 5 * NPK, NV = (KX + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float* V1 = A.ops2 + NQ * NT * 4;   // [N1 (l)][N1 (j)]
  const float* D1 = V1 + N1 * N1;
  for (int64_t li = w0; li < A.K; li += nw) {
    const int64_t e = A.elist ? (int64_t)A.elist[li] : li;
    const int64_t base = A.dof_off + e * NP;
    for (int l = 0; l < N1; ++l) {
      float v[NV];
      float mx = 0.f;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int k = lane + 32 * i;
        const int blk = k / NPK, mt = k - blk * NPK;
        float s = 0.f;
        if (k < KX && mt < NT) {
          const int f = blk == 0 || blk == 1 ? 0 : blk - 1;   // field: p, p (D1), u, v, w
          const float* c = blk == 1 ? D1 + l * N1 : V1 + l * N1;
          const float* q = A.q + f * A.ndof + base + mt;
#pragma unroll
          for (int j = 0; j < N1; ++j) s = fmaf(c[j], q[NT * j], s);
        }
        v[i] = s;
        mx = fmaxf(mx, fabsf(s));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float sc = mx > 0.f ? ldexpf(1.f, 14 - ilogbf(mx)) : 1.f;
      const int64_t row = li * N1 + l;
      unsigned short* xh = P.xh + row * KX;
      unsigned short* xl = P.xl + row * KX;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int k = lane + 32 * i;
        if (k >= KX) break;
        const float x = sc * v[i];
        const unsigned short h = rn16<BF>(x);
        xh[k] = h;
        xl[k] = rn16<BF>(x - f16f<BF>(h));
      }
      if (lane == 0) P.xis[row] = 1.f / sc;
    }
  }
}

// ---------------------------------------------------------------------------- Y = B X (tcgen05)
constexpr int VG_BM = 128, VG_BK = 64, VG_ST = 2;

__host__ __device__ constexpr int vg_stage_bytes(int npp) { return 2 * VG_BM * VG_BK * 2 + 2 * npp * VG_BK * 2; }
__host__ __device__ constexpr int vg_smem(int npp) { return VG_ST * vg_stage_bytes(npp) + 1024 + 64; }

template <bool BF>
__global__ void __launch_bounds__(128) vgemm_kernel(const __grid_constant__ PrecMaps G, PrecDev P, int M, int* err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int npp = P.npp;
  const int SA = VG_BM * VG_BK * 2, SB = npp * VG_BK * 2, SST = 2 * SA + 2 * SB;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + VG_ST * SST);
  uint64_t* done = full + VG_ST;
  uint64_t* fin = done + VG_ST;
  unsigned* tslot = reinterpret_cast<unsigned*>(fin + 1);
  volatile int* sbail = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = blockIdx.x / P.nblk, blk = blockIdx.x % P.nblk;
  const int k0 = P.kb0[blk], kn = P.kbn[blk];
  const int nch = (kn + VG_BK - 1) / VG_BK;
  const unsigned ncols = npp <= 32 ? 32 : npp <= 64 ? 64 : npp <= 128 ? 128 : 256;
  if (tid == 0) {
    for (int s = 0; s < VG_ST; ++s) {
      bar_init(full + s, 1);
      bar_init(done + s, 1);
    }
    bar_init(fin, 1);
    *sbail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa32(tslot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tb = *tslot;
  // D f32 (bit 4), A and B BF16 (1) or FP16 (0) at bits 7 and 10, both K-major, N >> 3 at 17, M >> 4 at 24
  const unsigned fmt = BF ? 1u : 0u;
  const unsigned idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(npp >> 3) << 17) | ((unsigned)(VG_BM >> 4) << 24);
  unsigned ph_full = 0, ph_done = 0, inflight = 0;   // parity bit and copies-in-flight bit per stage
  if (tid == 0) {
    const int row0 = mt * VG_BM, brow0 = blk * npp;
    auto load = [&](int c, int s) {
      const int kc = k0 + c * VG_BK, len = kn - c * VG_BK < VG_BK ? kn - c * VG_BK : VG_BK, sl = len / 8;
      unsigned char* st = sm + s * SST;
      bar_expect(full + s, (unsigned)(sl * (2 * VG_BM * 16 + 2 * npp * 16)));
      for (int j = 0; j < sl; ++j) {
        tma2d(st + j * VG_BM * 16, &G.xh, kc + 8 * j, row0, full + s);
        tma2d(st + SA + j * VG_BM * 16, &G.xl, kc + 8 * j, row0, full + s);
        tma2d(st + 2 * SA + j * npp * 16, &G.bh, kc + 8 * j, brow0, full + s);
        tma2d(st + 2 * SA + SB + j * npp * 16, &G.bl, kc + 8 * j, brow0, full + s);
      }
      inflight |= 1u << s;
    };
    for (int c = 0; c < nch && c < VG_ST; ++c) load(c, c);
    for (int c = 0; c < nch; ++c) {
      const int s = c % VG_ST;
      if (!bar_wait_b(full + s, (ph_full >> s) & 1u)) {
        *sbail = 1;
        break;
      }
      ph_full ^= 1u << s;
      inflight &= ~(1u << s);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int len = kn - c * VG_BK < VG_BK ? kn - c * VG_BK : VG_BK;
      const unsigned st = sa32(sm + s * SST);
      for (int kk = 0; kk < len / 16; ++kk) {
        const uint64_t ah = kdesc(st + 2 * kk * VG_BM * 16, VG_BM * 16, 128);
        const uint64_t al = kdesc(st + SA + 2 * kk * VG_BM * 16, VG_BM * 16, 128);
        const uint64_t bh = kdesc(st + 2 * SA + 2 * kk * npp * 16, npp * 16, 128);
        const uint64_t bl = kdesc(st + 2 * SA + SB + 2 * kk * npp * 16, npp * 16, 128);
        mma_f16(tb, ah, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
        mma_f16(tb, ah, bl, idesc, 1u);
        mma_f16(tb, al, bh, idesc, 1u);
      }
      mma_commit(done + s);
      if (c + VG_ST < nch) {   // the stage is refilled once its MMAs have read it
        if (!bar_wait_b(done + s, (ph_done >> s) & 1u)) {
          *sbail = 1;
          break;
        }
        ph_done ^= 1u << s;
        load(c + VG_ST, s);
      }
    }
    mma_commit(fin);   // completes when every MMA issued above has
  }
  __syncthreads();
  const bool ok = bar_wait_b(fin, 0) && !*sbail;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = mt * VG_BM + tid;
    const unsigned lb = tb + ((unsigned)(warp * 32) << 16);
    const float sc = row < M ? P.xis[row] * P.bis : 0.f;
    float* yr = P.y + (int64_t)row * P.nblk * npp + blk * npp;
    for (int ch = 0; ch < npp / 8; ++ch) {
      unsigned v[8];
      tld8(lb + ch * 8, v);
      if (row < M) {
        float4 a = make_float4(sc * __uint_as_float(v[0]), sc * __uint_as_float(v[1]), sc * __uint_as_float(v[2]),
                               sc * __uint_as_float(v[3]));
        float4 b = make_float4(sc * __uint_as_float(v[4]), sc * __uint_as_float(v[5]), sc * __uint_as_float(v[6]),
                               sc * __uint_as_float(v[7]));
        reinterpret_cast<float4*>(yr + ch * 8)[0] = a;
        reinterpret_cast<float4*>(yr + ch * 8)[1] = b;
      }
    }
  } else if (tid == 0) {   // report; wait (bounded) for the copies still in flight
    atomicOr(err, 1);
    for (int s = 0; s < VG_ST; ++s)
      if (inflight & (1u << s)) bar_wait_b(full + s, (ph_full >> s) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------- operator split
// B (FP32, [nblk NPP][kx]) scaled by 1 / P.bis into its 16-bit hi and lo parts
template <bool BF>
__global__ void split_op_kernel(const float* b, unsigned short* bh, unsigned short* bl, int64_t n, float s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = s * b[i];
    const unsigned short h = rn16<BF>(v);
    bh[i] = h;
    bl[i] = rn16<BF>(v - f16f<BF>(h));
  }
}

cudaError_t prec_split_operator(PrecDev& P, const float* b, bool bf, cudaStream_t s) {
  const int64_t n = (int64_t)P.nblk * P.npp * P.kx;
  if (bf) split_op_kernel<true><<<256, 256, 0, s>>>(b, P.bh, P.bl, n, 1.f / P.bis);
  else split_op_kernel<false><<<256, 256, 0, s>>>(b, P.bh, P.bl, n, 1.f / P.bis);
  return cudaGetLastError();
}

template <int N, bool BF>
static void wpack_n(const Args& A, const PrecDev& P, cudaStream_t s, int sms) {
  const int64_t blocks = ((int64_t)A.K * 32 + 255) / 256;
  const int grid = (int)(blocks < 16 * sms ? blocks : 16 * sms);
  wpack_kernel<N, BF><<<grid, 256, 0, s>>>(A, P);
}

template <int T, int N, bool BF>
static void pack_n(const Args& A, const PrecDev& P, cudaStream_t s, int sms) {
  const int64_t blocks = ((int64_t)A.K * 32 + 255) / 256;
  const int grid = (int)(blocks < 16 * sms ? blocks : 16 * sms);
  pack_kernel<T, N, BF><<<grid, 256, 0, s>>>(A, P);
}

// pack, multiply; afterwards Args.vol / vol_np point at Y for the type's warp kernel.  An empty
// selection launches nothing.  A launch error is left pending (not cleared) for the launch group's
// check, and Args.vol stays NULL then (the warp kernel forms its products itself).
cudaError_t launch_prec_volume(dg_mesh* m, int t, Args& A, cudaStream_t s) {
  if (A.K == 0) return cudaSuccess;
  PrecDev& P = m->prec[prec_slot(t)];
  const PrecMaps& G = m->prec_maps[prec_slot(t)];
  const bool bf = m->precision == 1;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  switch (m->N) {
#define PK_CASE(NN)                                                             \
  case NN:                                                                      \
    if (t == DG_TET) bf ? pack_n<DG_TET, NN, true>(A, P, s, sms) : pack_n<DG_TET, NN, false>(A, P, s, sms); \
    else if (t == DG_PYR) bf ? pack_n<DG_PYR, NN, true>(A, P, s, sms) : pack_n<DG_PYR, NN, false>(A, P, s, sms); \
    else bf ? wpack_n<NN, true>(A, P, s, sms) : wpack_n<NN, false>(A, P, s, sms);                          \
    break;
    PK_CASE(1) PK_CASE(2) PK_CASE(3) PK_CASE(4) PK_CASE(5) PK_CASE(6) PK_CASE(7) PK_CASE(8) PK_CASE(9)
#undef PK_CASE
    default: return cudaErrorInvalidValue;
  }
  const int smem = vg_smem(P.npp);
  static bool attr[2] = {false, false};
  if (!attr[bf]) {
    cudaError_t e = cudaFuncSetAttribute(bf ? vgemm_kernel<true> : vgemm_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr[bf] = true;
  }
  const int rows = t == DG_WEDGE ? A.K * (m->N + 1) : A.K;   // wedges: a row per element and 1D level
  const int mtiles = (rows + VG_BM - 1) / VG_BM;
  if (bf) vgemm_kernel<true><<<mtiles * P.nblk, 128, smem, s>>>(G, P, rows, m->derr);
  else vgemm_kernel<false><<<mtiles * P.nblk, 128, smem, s>>>(G, P, rows, m->derr);
  const cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess) {
    A.vol = P.y;
    A.vol_np = P.vnp;
  }
  return e;
}

}  // namespace dgk
