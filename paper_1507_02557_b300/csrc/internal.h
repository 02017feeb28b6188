// Internal state of a dg_mesh and the kernel launch interface.
#pragma once
#include <cuda.h>   // CUtensorMap (TMA descriptors)
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dg.h"

namespace dgk {

constexpr int MAXN = 9;       // kernels are instantiated for N = 1..MAXN
constexpr int NCODES = 8;     // face orientation codes (6 used for triangles)

// Device data of one element type.
struct TypeDev {
  int K = 0, Np = 0, nf = 0, nc = 0;
  int64_t dof_off = 0;        // first DOF of the type within a field
  int64_t side_off = 0;       // first global side index of the type (side = off + e*nf + f)
  float* c2 = nullptr;        // [K]
  float* geo = nullptr;       // hex [K][24] trilinear coefficients; tet [K][12] G,J;
                              // pyramid [K][10][Np] G,J (component-major within an element:
                              // lanes on consecutive nodes read consecutive words); wedge [K][16]
                              // map coefficients x_r = a_r + s b_r, x_t = a_t + s b_t,
                              // x_s = c + r b_r + t b_t (a_r, b_r, a_t, b_t, c, 0)
  float* wpts = nullptr;      // wedge: cubature points, triangle (r, t) [nc / (N+1)][2], then s [N+1]
  float4* sgeo = nullptr;     // non-hex: [K*nf][nq] (n, w_q J^s [/sqrt J for the wedge])
  float* sisq = nullptr;      // wedge: [K*nf][nq] 1/sqrt(J) at face points
  float* ops = nullptr;       // volume operators (type-specific layout, see setup.cpp)
  float* Tt = nullptr;        // non-hex trace matrices [nf][8][Np][nq]
  float* L = nullptr;         // non-hex lift matrices [nf][8][nq][Np]
  // orientation-free operators of the warp-per-element kernels (kernels_gen2.cu)
  float4* sgeo2 = nullptr;    // [K*nf][nq]: triangle faces at canonical points, quads at local points
  float* sisq2 = nullptr;     // wedge: 1/sqrt(J) in the same order
  float* ops2 = nullptr;      // float operators (layout in setup.cpp: build_gen2_ops)
  int* iops2 = nullptr;       // integer tables (face-node gathers, lattice permutations)
  int nops2 = 0, niops2 = 0;  // sizes (elements)
};

// 1D TMA descriptor of a flat float array of n values, copied in boxes of `box` floats.
struct TmaArr {
  CUtensorMap map;
  const float* base = nullptr;
  int64_t n = 0;
  int box = 0;
  bool ok = false;
};
bool tma_map_1d(TmaArr& t, const float* base, int64_t n, int box);   // kernels.cu

// Tensor-core volume terms (precision 1 = BF16 x 3, 2 = FP16 x 3) of tets ([0]), pyramids ([1]) and
// wedges ([2]): rows of X (kx 16-bit values, hi and lo parts, scaled by a power of two per row; xis =
// 1 / scale), Y = B X in FP32 (nblk blocks of npp per row), B = the fixed block operator (FP32 copy
// and its scaled hi / lo parts; bis = 1 / its scale).  Output block b reads X columns
// [kb0[b], kb0[b] + kbn[b]) against B's rows [b npp, (b + 1) npp).  Tets and pyramids: a row per
// element, X = [W_r | W_s | W_t | p] (4 blocks of npk); wedges: a row per element and 1D level l,
// X = [y_p | y_s | y_u | y_v | y_w] (triangle-mode vectors).  Layouts in kernels_prec.cu.
struct PrecDev {
  unsigned short *xh = nullptr, *xl = nullptr, *bh = nullptr, *bl = nullptr;
  float* xis = nullptr;
  float* y = nullptr;
  float* b32 = nullptr;
  int npk = 0, npp = 0;
  float bis = 1.f;
  int nblk = 4, kx = 0;
  int kb0[8] = {0, 0, 0, 0, 0, 0, 0, 0}, kbn[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int vnp = 0;   // width of a block of Y as the warp kernel reads it (npp, or 2 npp when each of
                 // the four tet / pyramid blocks is computed in two halves: pyramids above 256 nodes)
};
__host__ __device__ inline int prec_slot(int t) { return t == DG_TET ? 0 : t == DG_PYR ? 1 : 2; }
// 2D TMA descriptors of X (hi, lo: boxes of 8 values x 128 rows) and B (hi, lo: 8 x npp)
struct PrecMaps {
  CUtensorMap xh, xl, bh, bl;
};
bool prec_maps(PrecMaps& M, const PrecDev& P, int64_t rows);   // kernels.cu

// A selection of elements per type (multi-rate level): list = NULL means 0..count-1.
struct Sel {
  const int* list[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t count[4] = {0, 0, 0, 0};
};

}  // namespace dgk

struct dg_mesh {
  int device = 0;
  cudaStream_t stream = nullptr;
  int N = 0, nq = 0;
  double tau_scale = 1.0, cfl = 0.5;
  int pyr_form = 0;
  int64_t K[4] = {0, 0, 0, 0};
  int64_t ndof = 0, nsides = 0;
  dgk::TypeDev td[4];
  int* side_nbr = nullptr;    // [nsides] neighbour's global side, -1 on a wall
  int* side_code = nullptr;   // [nsides] canonical face-frame code
  float* side_tau = nullptr;  // [nsides] tau_p = 1/{rho c}
  float* hexc = nullptr;      // hex constants: D1[n1*n1], Vm[n1], Vp[n1], w1[n1], r1[n1]
  int* hexperm = nullptr;     // [8][nq] local face point -> canonical index
  float* q = nullptr;         // [4][ndof] state
  float* res = nullptr;       // [4][ndof] LSRK residual
  float* trace = nullptr;     // [2 buffers][2 planes: p, u.n][nsides*nq]
  double* dacc = nullptr;     // energy accumulator
  double dt_min = 0.0;
  std::vector<double> dtK[4];
  std::vector<double> tet_mhat;  // host copy of the reference tet mass (energy)
  float* tet_mhat_dev = nullptr;
  float* tet_chol_dev = nullptr;   // R with M_hat = R^T R (upper triangular), energy
  // multi-rate (nlevels = 2): per-level element lists, RHS history, start-up flag
  int nlevels = 1;
  dgk::Sel all, lev[2];           // lev[0] = coarse (level 1), lev[1] = fine (level 2)
  int64_t level_count[2] = {0, 0};
  float* hist = nullptr;          // [3 slots][4][ndof]
  float* trace3 = nullptr;        // third trace buffer of the fused multi-rate schedule
  int cslot[3] = {0, 1, 2}, fslot[3] = {2, 0, 1};   // slots of r^n, r^{n-1}, r^{n-2} per level
  bool mr_started = false;
  // multi-rate LSRK(5,4) (integrator 1, mrlsrk.cu): S = fine elements and the coarse elements sharing
  // a face with one, T = S and the elements sharing a face with S; in_s[t][e] = 1 for elements of S;
  // mrl = 14 state-sized buffers allocated on first use
  int integrator = 0;
  dgk::Sel mr_s, mr_t, mr_tc;     // mr_tc: the coarse elements of T
  unsigned char* mr_in_s[4] = {nullptr, nullptr, nullptr, nullptr};
  // two levels: 1 for a coarse element with a fine face neighbour (only those elements' half-step
  // traces are read, by the fine substeps); counts per type
  unsigned char* mr_pred[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t mr_pred_count[4] = {0, 0, 0, 0};
  float* mrl = nullptr;
  bool hex_sem = false;           // SEM hexahedra (GLL nodes)
  bool tri_lat = true;            // tet / pyramid triangle faces exchange lattice values (gen2)
  bool wall_self = false;         // trace launches also write a wall side's own trace into its slot
  // element types of one stage / substep on their own streams (off with DG_TYPE_STREAMS=0, and
  // while per-type timing is on)
  bool type_streams = false;
  // kernel choices (dg_autotune): TMA staging of the fused N = 4 hex kernels, tensor-core tets
  bool use_hex_tma = true, use_tet_tc = true;
  // precision of the tet and pyramid volume products and the wedges' first contraction: 0 = FP32
  // (SIMT, or TF32 x 3 tensor-core tets for N <= 4), 1 = BF16 x 3, 2 = FP16 x 3 on the tensor cores
  // (kernels_prec.cu)
  int precision = 0;
  dgk::PrecDev prec[3];
  dgk::PrecMaps prec_maps[3];
  cudaStream_t tstream[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t tev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // adjoint (adjoint.cu): host data kept by the setup, device copies made on first use
  std::vector<float> face_w;      // [nsides][nq] w_q J^s at the canonical points (lattice faces: J^s)
  std::vector<double> face_mass;  // [nfn][nfn] face mass of the triangle lattice basis
  std::vector<double> tet_mhat_inv;
  float* face_w_dev = nullptr;
  float* face_mass_dev = nullptr;
  float* tet_minv_dev = nullptr;
  float* adj_buf = nullptr;       // scratch states of the reverse sweep
  size_t adj_states = 0;
  // point source and receivers in hexahedra (source.cu)
  std::vector<double> hex_coef;   // [K_hex][8][3] trilinear-map coefficients c0..c7 (x = c0 + c1 r + ...)
  std::vector<double> hex_r1, hex_w1;   // 1D nodes and weights of the hexahedron
  int64_t src_e = -1;             // hexahedron holding the source, -1 = none
  float* src_g = nullptr;         // [Np] M^{-1} phi(x_s)
  double src_amp = 0.0, src_f0 = 0.0, src_t0 = 0.0;
  float src_now = 0.f;            // amp ricker(t) for the next rhs / stage launch (0 = none)
  int nrec = 0;
  int* rec_e = nullptr;           // [nrec] hexahedron of each receiver
  float* rec_rows = nullptr;      // [nrec][Np] phi(x_r)
  int* derr = nullptr;            // device error word: bit 0 = a bounded device wait timed out
  dgk::TmaArr tma[5];             // q, res, hist, trace, trace3 (hex TMA staging)
  // host copy of the description the mesh was created from (batches merge meshes from it)
  struct HostDesc {
    std::vector<double> xyz;
    std::vector<int32_t> conn[4];
    std::vector<double> c2[4];
    dg_mesh_desc d{};
  } host;
  // per-element LSRK step (float, element order of each type) of a mesh that holds several
  // batched meshes, each stepped with its own dt; NULL = the scalar dt of the launch
  float* dte[4] = {nullptr, nullptr, nullptr, nullptr};
  // per-type kernel timing (dg_profile): event pairs recorded around each launch
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used[4];   // (start, stop) indices into ev_pool
  size_t ev_next = 0;
  int64_t launches[4] = {0, 0, 0, 0};
};

namespace dgk {
// Kernel launchers (kernels.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_trace(dg_mesh* m, const float* q, float* tout);
cudaError_t launch_rhs(dg_mesh* m, const float* q, const float* tin, float* rhs);
// (qout: the updated state, NULL = in place)
cudaError_t launch_stage(dg_mesh* m, float* q, float* res, const float* tin, float* tout, float a,
                         float b, float dt, float* qout = nullptr);
cudaError_t launch_energy(dg_mesh* m, const float* q, double* acc);
cudaError_t launch_trace_sel(dg_mesh* m, const float* q, float* tout, const Sel& sel);
cudaError_t launch_rhs_sel(dg_mesh* m, const float* q, const float* tin, float* rhs, const Sel& sel);
// Fused multi-rate AB3 step for the elements of sel (N <= 4): coarse elements write the traces of
// the half-step prediction to tout and of the new state to tout2; fine elements those of the new
// state to tout.  rhs -> hw, q += c0 rhs + c1 h1 + c2 h2, prediction q + p0 rhs + p1 h1 + p2 h2.
cudaError_t launch_mr(dg_mesh* m, bool coarse, const Sel& sel, float* q, const float* tin, float* tout,
                      float* tout2, float* hw, const float* h1, const float* h2, const float c[3],
                      const float p[3]);
cudaError_t launch_ab(dg_mesh* m, const Sel& sel, const float* qin, float* qout, const float* r0,
                      const float* r1, const float* r2, float h0, float h1, float h2);
// Contiguous device-to-device copies: n floats from src to dst per segment (batch gather / scatter).
struct Seg {
  const float* src;
  float* dst;
  int64_t n;
};
cudaError_t launch_seg_copy(const Seg* segs_dev, int nseg, cudaStream_t s);
// Hex constants (1D D, V^f, GL weights and nodes) of order N <= 4 into constant memory.
cudaError_t upload_hex_constants(int N, bool sem, const float* hc, int count);
struct Args;
// Tensor-core volume terms of type t (DG_TET / DG_PYR / DG_WEDGE) for the elements of A (precision
// > 0): pack X, Y = B X; sets A.vol, A.vol_np for the type's warp kernel (kernels_prec.cu).
cudaError_t launch_prec_volume(dg_mesh* m, int t, Args& A, cudaStream_t s);
// Scaled 16-bit hi / lo parts of the FP32 operator b into P.bh, P.bl (kernels_prec.cu).
cudaError_t prec_split_operator(PrecDev& P, const float* b, bool bf, cudaStream_t s);
}  // namespace dgk

// Message returned by dg_last_error() on this thread (api.cpp).
void dg_set_last_error(const std::string& msg);
// After a synchronisation: DG_ETIMEOUT (and the word cleared) if a bounded device wait timed out
// since the last report, DG_ECUDA if the word cannot be read, else DG_OK (api.cpp).
dg_status dg_device_flags(const dg_mesh* m);

// Carpenter & Kennedy (1994) LSRK(5,4) coefficients (api.cpp).
extern const double RK_A[5];
extern const double RK_B[5];
extern const double RK_C[5];   // stage times

// Point source and receivers (source.cu).  dg_source_at sets m->src_now = amp ricker(t) (0 without
// a source) for the next rhs / stage launch.
double dg_ricker(double t, double f0, double t0);
void dg_source_at(dg_mesh* m, double t);
// lam_p += the receivers' transpose of resid [nrec]
cudaError_t dg_receiver_inject(dg_mesh* m, const float* resid, float* lam);
// *g += coef rho_p . g_s over the source's hexahedron (device double g)
cudaError_t dg_source_amp_grad(dg_mesh* m, const float* rho, double coef, double* g);

// nsteps time steps of m on m->stream: LSRK(5,4), or multi-rate AB3 whose first call also runs the
// start-up (nsteps = 0 runs the start-up alone).  No synchronization (api.cpp).
cudaError_t dg_enqueue_steps(dg_mesh* m, int nsteps, double dt, double t0 = 0.0);
// nsteps coarse steps (2h) of the two-level multi-rate LSRK(5,4) on m->stream (mrlsrk.cu).
cudaError_t dg_mrlsrk_steps(dg_mesh* m, int nsteps, double h);
// Simulated time that dg_enqueue_steps(m, nsteps, dt) advances; fresh = the start-up runs too.
double dg_step_time(const dg_mesh* m, int nsteps, double dt, bool fresh);

// Reverse sweep of nsteps LSRK(5,4) steps of dt from the state m->q at time t0 (adjoint.cu): lam
// (device, [4][ndof]) holds dL/dq_n on entry and dL/dq_0 on return; resid (device [nsteps][nrec]
// or NULL) is the receiver forcing of the states after steps 1..nsteps; grad (device, one double
// per element in type order, or NULL) accumulates dL/dc^2, grad_amp (device double or NULL)
// dL/damp of the source.  Enqueued on m->stream; m->q is left unchanged.
cudaError_t dg_adjoint_run(dg_mesh* m, int nsteps, double dt, double t0, float* lam, const float* resid,
                           double* grad, double* grad_amp);

// Host setup (setup.cpp).
dg_status dg_setup(dg_mesh* m, const dg_mesh_desc* d, std::string& err);
void dg_free(dg_mesh* m);
// cudaMalloc whose block dg_free releases with the mesh's other buffers (NULL on failure).
void* dg_alloc_owned(dg_mesh* m, size_t bytes);
// Host setup without any device allocation or transfer (dg_host_check).
dg_status dg_setup_host_only(dg_mesh* m, const dg_mesh_desc* d, std::string& err, double ct[4]);
