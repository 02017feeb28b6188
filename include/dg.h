/*
 * dg.h - C ABI of the hybrid-mesh acoustic discontinuous Galerkin library (libdg).
 *
 * Semi-discrete system (arxiv 1507.02557, Sec. 2.2, Eq. skewform and the strong
 * form):  (1/kappa) p_t + div u = 0,  rho u_t + grad p = 0, with kappa = 1 and
 * rho = 1/c^2 per element, free-surface walls p = 0, upwind penalties
 * tau_p = 1/{rho c}, tau_u = {rho c} (times tau_scale).  Bases (Sec. 2.1):
 * GL-nodal hexahedra, LSC-DG modal wedges, semi-nodal rational pyramids,
 * nodal tetrahedra (equispaced lattice).  Time stepping: LSRK(5,4)
 * (Carpenter-Kennedy 2N-storage); time step of Eq. (dtK) with the computed
 * reference trace constants of Appendix B.
 *
 * State layout ("q"): float32 [4][ndof], fields p, u, v, w.  Within a field the
 * DOFs of all hexahedra come first, then wedges, pyramids, tetrahedra
 * (dg_layout gives the offsets); within a type, element-major with Np DOFs per
 * element:
 *   hex     node (i,j,k) at GL nodes (r_i,s_j,t_k), index i + (N+1)(j + (N+1)k)
 *   wedge   modal (i,j,k), index m + Ntri*j, m enumerating (i,k), i outer, k inner
 *           (P_i(a) P_j(s) ((1-c)/2)^i P_k^{(2i+1,0)}(t), orthonormal; LSC: / sqrt(J))
 *   pyramid semi-nodal (i,j,k), 0 <= i,j <= k <= N, k outer, then j, then i
 *   tet     nodal at r,s,t = -1 + 2(i,j,k)/N, i+j+k <= N, k outer, then j, then i
 *
 * Conventions
 *   - Every call returns a dg_status and never aborts or throws across the ABI.
 *   - Host arrays are borrowed for the duration of the call.  Device pointers
 *     are borrowed; the caller keeps them alive until the stream has finished.
 *   - Work is enqueued on the CUDA stream given to dg_mesh_create.  Inside a
 *     stage or substep the four element types' kernels run side by side on
 *     four streams the mesh owns, forked from and joined back into that stream
 *     with events, so the ordering seen on the given stream is unchanged (set
 *     DG_TYPE_STREAMS=0 in the environment at creation to keep them on the
 *     one stream; per-type timing with dg_profile does so while it is on).
 *     Only dg_mesh_create, dg_timestep, dg_energy and
 *     dg_get_state(on_device = 0) synchronise with the host.
 *   - Errors: DG_EINVAL bad argument; DG_ENOMEM device allocation failed;
 *     DG_ECUDA a CUDA call failed (dg_last_error() gives the message);
 *     DG_EMESH invalid mesh (J <= 0 at a quadrature point, a face shared by
 *     more than two elements); DG_ENOTSUP option not built.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh dg_mesh;  /* opaque; owns the device buffers it allocates */

typedef enum {
  DG_OK = 0,
  DG_EINVAL = -1,
  DG_ENOMEM = -2,
  DG_ECUDA = -3,
  DG_EMESH = -4,
  DG_ETIMEOUT = -5,
  DG_ENOTSUP = -6,
  DG_ENONFINITE = -7
} dg_status;

enum { DG_HEX = 0, DG_WEDGE = 1, DG_PYR = 2, DG_TET = 3 };

typedef struct {
  int64_t nverts;
  const double *xyz;       /* host, [nverts][3] vertex coordinates */
  int64_t nelem[4];        /* elements per type: hex, wedge, pyramid, tet */
  const int32_t *conn[4];  /* host, [nelem][8|6|5|4] vertex ids in the local order:
                              hex (r,s,t) = (+-1,+-1,+-1) lexicographic, r fastest;
                              wedge (r,t) = (-1,-1),(1,-1),(-1,1) at s=-1 then s=+1;
                              pyramid base (r,s) lexicographic at t=-1, apex (-1,-1,1);
                              tet (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1) */
  const double *c2[4];     /* host, [nelem] squared wave speed per element (> 0) */
  int N;                   /* polynomial order, 1..9 */
  int hex_basis;           /* 0 = GL nodes; 1 = SEM: GLL nodes and GLL points on every quad face */
  int pyr_form;            /* 0 = skew-symmetric, 1 = strong (identical results, Sec. 2.2) */
  double tau_scale;        /* 1 = upwind, 0 = central flux */
  int nlevels;             /* 1 = single-rate LSRK(5,4); 2 = two-level multi-rate AB3 */
  double cfl;              /* C of Eq. (dtK); <= 0 selects 0.5 */
  int precision;           /* volume products of tets and pyramids: 0 = FP32 (CUDA cores; tets at
                              N <= 4 on the tensor cores in TF32 x 3); 1 = BF16 x 3, 2 = FP16 x 3:
                              16-bit hi + lo split operands on the tensor cores, FP32 accumulation
                              (about 2^-17 / 2^-22 relative per product); hexahedra, the wedges'
                              second contraction and metric terms, and all face terms stay FP32.
                              Tets and pyramids: on meshes with the lattice face exchange (no wedge
                              triangle face against a tet or pyramid), any N.  Wedges: the
                              triangle-mode to cubature-point contraction at N >= 7.  The adjoint
                              refuses 1, 2 (DG_ENOTSUP) */
  int integrator;          /* nlevels = 2: 0 = multi-rate Adams-Bashforth 3 (default),
                              1 = multi-rate LSRK(5,4) (see dg_step) */
} dg_mesh_desc;

/* Build the mesh on the current CUDA device: face matching, geometric factors,
 * reference operators, local time steps (Eq. dtK).  stream: a cudaStream_t or
 * NULL for the default stream.  Synchronises.  Allocates the state q, the LSRK
 * residual and a face-trace exchange buffer, all zero-initialised. */
dg_status dg_mesh_create(const dg_mesh_desc *desc, void *stream, dg_mesh **out);
void dg_mesh_destroy(dg_mesh *mesh);

/* Run the host part of dg_mesh_create only (face matching, geometry checks,
 * reference operators, Eq. dtK, multi-rate levels) without touching any GPU.
 * Returns the global time step in *dt_min; if not NULL, trace_const[4] receives
 * the reference trace constants C_T(N) of hex, wedge, pyramid, tet (Appendix B)
 * and level_count[nlevels] the element count of each time-step level (coarse
 * first).  Same error codes as dg_mesh_create. */
dg_status dg_host_check(const dg_mesh_desc *desc, double *dt_min, double *trace_const,
                        int64_t *level_count);

/* DOF layout of one element type: offset of its first DOF within a field,
 * its element count and DOFs per element. */
dg_status dg_layout(const dg_mesh *mesh, int type, int64_t *offset, int64_t *nelem, int *Np);
dg_status dg_ndof(const dg_mesh *mesh, int64_t *ndof);
/* Elements of each type (counts[4]: hex, wedge, pyramid, tet) in time-step
 * level `level` (1 = coarsest .. nlevels = finest, Sec. 2.4).  level = 0 on a
 * multi-rate LSRK mesh (integrator 1): the elements of S, the fine elements and
 * the coarse elements sharing a face with one.  level = -1 on a two-level mesh: the
 * coarse elements sharing a face with a fine element (the only ones whose half-step
 * traces the fine substeps read, so the only ones that write them). */
dg_status dg_level_counts(const dg_mesh *mesh, int level, int64_t *counts);

/* Copy a state [4][ndof] into the mesh's state (and zero the LSRK residual).
 * q is a host pointer (on_device = 0) or a device pointer (on_device = 1). */
dg_status dg_set_state(dg_mesh *mesh, const float *q, int on_device);
/* Copy the mesh's state out; on_device = 0 synchronises. */
dg_status dg_get_state(const dg_mesh *mesh, float *q, int on_device);

/* rhs = M^{-1} A q for a device state q_dev [4][ndof] (Sec. 2.2-2.3); rhs_dev is
 * a device buffer of the same size.  Uses the mesh's trace buffer as scratch.
 * t is the time (unused: no source term). */
dg_status dg_rhs(dg_mesh *mesh, const float *q_dev, float *rhs_dev, double t);

/* Global time step dtau_min = min_K dtau_K of Eq. (dtK) (host, computed at
 * create).  level_count may be NULL; otherwise receives the element count of
 * each multi-rate level (nlevels entries). */
dg_status dg_timestep(const dg_mesh *mesh, double *dt_min, int64_t *level_count);

/* Advance the mesh's state (dt <= 0 uses dtau_min).  Asynchronous.
 *   nlevels = 1: nsteps LSRK(5,4) steps of size dt; *t_inout += nsteps*dt.
 *   nlevels = 2, integrator 0: nsteps coarse steps of the two-level multi-rate
 *     Adams-Bashforth-3 scheme (reading of Sec. 2.4): fine elements step dt twice,
 *     coarse elements step 2 dt once, coarse states at the half step are predicted
 *     from their AB3 history.  The first call after dg_set_state first runs the
 *     start-up (four LSRK(5,4) steps of size dt that record the rhs history);
 *     *t_inout += 4 dt (start-up) + nsteps * 2 dt.
 *   nlevels = 2, integrator 1: nsteps coarse steps of 2 dt of the two-level
 *     multi-rate LSRK(5,4) (a local time-stepping RK read for Sec. 2.4): the
 *     coarse region acts on the step through W(tau) = sum_j rho_{j+1} tau^{j+1}
 *     B (I - P) B^j y_n (rho: the LSRK(5,4) amplification coefficients, B the
 *     rhs operator, P the fine elements), the fine correction v' = B P (y + W + v)
 *     takes two LSRK(5,4) steps of dt, y += W(2 dt) + v.  Fourth order; one
 *     LSRK(5,4) step of 2 dt on an all-coarse mesh, two of dt on an all-fine one.
 *     No start-up; *t_inout += nsteps * 2 dt.  Allocates 14 state-sized buffers
 *     on first use (DG_ENOMEM if they do not fit). */
dg_status dg_step(dg_mesh *mesh, int nsteps, double dt, double *t_inout);

/* Direct access to the device state [4][ndof] owned by the mesh. */
dg_status dg_state_ptr(dg_mesh *mesh, float **q_dev);

/* E = 1/2 sum_K (p^T M_K p / kappa + rho u^T M_K u) in FP64 for a device state
 * (NULL = the mesh's state).  Synchronises. */
dg_status dg_energy(dg_mesh *mesh, const float *q_dev, double *E);

/* dg_energy for callers that cannot allocate device memory while they run:
 * real-time loops that cannot take the latency of cudaMalloc (which may
 * synchronise the device) and frameworks that have reserved all device memory
 * for their own pool.  No counterpart in the paper.  Equal to dg_energy within
 * FP32 rounding (the per-node terms are formed in FP64 here, in FP32 there;
 * the tests use 1e-6 relative); repeated calls on the same state return
 * bitwise-equal results (fixed summation order).  Allocates nothing: the
 * per-element partial sums live in a static device array of 2^20 + 1 doubles
 * (8 MiB) that every GPU loading libdg holds until exit.  Meshes with more
 * than 2^20 elements are rejected with DG_EINVAL.  The first call on a device
 * looks up that array's address (cudaGetSymbolAddress) with the mesh's device
 * current.  The array is shared by all calls and keeps the last call's
 * contents; calls that overlap on the GPU race on it.  Synchronises.  Errors
 * as dg_energy: DG_ETIMEOUT for a timed-out device wait, DG_ENONFINITE for a
 * non-finite energy, DG_ECUDA with dg_last_error() set. */
dg_status dg_energy_noalloc(dg_mesh *mesh, const float *q_dev, double *E);

/* Per-type kernel timing.  ms and launches (4 entries each, hex, wedge,
 * pyramid, tet; either may be NULL) receive the kernel time (CUDA events
 * recorded on the mesh's stream around each launch) and the launch count
 * accumulated since the previous dg_profile call (synchronises when either is
 * given); then the counters are reset and event recording is switched on
 * (enable = 1) or off (enable = 0).  Launch counts are kept even when off. */
dg_status dg_profile(dg_mesh *mesh, int enable, double *ms, int64_t *launches);

/* Self-test of the device watchdog.  Kernels that wait on the GPU (the
 * mbarrier waits of the TMA-staged hex kernel and of the tensor-core tet
 * kernel) bound every wait; a wait that runs out sets bit 0 of the mesh's
 * device error word, and the next synchronising call (dg_get_state to the host,
 * dg_energy) returns DG_ETIMEOUT and clears the word.  This call launches one
 * kernel whose bounded wait is on an mbarrier that no thread arrives on, so it
 * runs out after limit_cycles SM clocks (1 .. 2^32) and records the timeout the
 * same way; the call then synchronises and returns that status (DG_ETIMEOUT when
 * the watchdog works; the word is cleared).  No counterpart in the paper.
 * DG_EINVAL for a null mesh or a limit out of range. */
dg_status dg_watchdog_selftest(dg_mesh *mesh, int64_t limit_cycles);

/* Autotuner: picks, for this mesh, among the kernel choices the library has at
 * run time by timing nsteps (1..100) LSRK(5,4) steps of dt_min of a scratch
 * copy of the state on the mesh's stream, one choice after the other (the
 * others held; best of three runs, an alternative taken only when at least 2 %
 * faster): [0] TMA staging of the fused N = 4 hex kernels or cp.async
 * staging, [1] tensor-core tets (N <= 4) or the SIMT tet kernel, [2] the element
 * types of a stage on their own streams or on one.  The choices hold for all
 * later calls on the mesh (a batch graph bakes in those at its capture); the
 * results of the alternatives agree to FP32 rounding.  choice[3] (host, or
 * NULL) receives them (1 = the first alternative).  nsteps = 0 applies
 * choice[] as given instead (no timing, no synchronisation; choice[2] is set
 * to 0 where the mesh has no type streams).  Synchronises; allocates
 * one state copy for the call; the mesh's state is unchanged, its LSRK residual
 * and trace buffers are overwritten.  No counterpart in the paper (Sec. 4.3
 * notes the cost per degree of freedom changing with the number of elements). */
dg_status dg_autotune(dg_mesh *mesh, int nsteps, int *choice);

/* ---- batches: many meshes stepped together ---------------------------------
 * Sec. 4.3 (Figure perDofTimes) measures the time per degree of freedom rising
 * for small meshes, whose kernels cannot fill the GPU.  A batch steps several
 * meshes (any mix of N, element types, sizes and time-step levels) through one
 * CUDA graph in which each mesh is an independent branch, so the kernels of
 * different meshes run concurrently and a chunk of steps costs one graph launch.
 *
 * dg_batch_create: meshes[count] are borrowed and must outlive the batch; a mesh
 *   belongs to at most one batch; every mesh must be on the current device.
 *   Work is enqueued on cuda_stream (NULL = the legacy default stream is not
 *   capturable, so the batch then creates and owns a stream).  Allocates per-mesh
 *   branch streams and events.  DG_EINVAL on a NULL or repeated mesh or count < 1.
 * dg_batch_step: the same as dg_step(meshes[i], nsteps, dt[i], &t_inout[i]) for
 *   every i (dt NULL or dt[i] <= 0: that mesh's dt_min; t_inout NULL: not
 *   reported), with the same results bit for bit as, per mesh, one dg_step call
 *   of nsteps mod DG_BATCH_CHUNK steps followed by nsteps / DG_BATCH_CHUNK calls
 *   of DG_BATCH_CHUNK steps (the multi-rate history slots rotate with that
 *   period).  The batch stream first waits for each mesh's own stream, and
 *   each mesh's stream then waits for the batch, so per-mesh calls before and
 *   after stay ordered.  Steps: the multi-rate start-ups and nsteps mod
 *   DG_BATCH_CHUNK steps are enqueued directly, mesh after mesh; the rest are
 *   replays of a graph of DG_BATCH_CHUNK steps of every mesh.  The graph is
 *   captured on first use and cached (up to 4 graphs, keyed by the dt values and
 *   the meshes' history-slot phases; a mesh stepped on its own between batch
 *   calls may change its phase and cost one re-capture).  Asynchronous: errors
 *   of the kernels are reported by the next synchronising call on a mesh.
 *   Packing (default; environment DG_BATCH_PACK=0 at creation turns it off):
 *   single-rate meshes without a point source that share N, hex basis, pyramid
 *   form, tau_scale, precision, face exchange and run-time kernel choices (at
 *   creation) are merged into one combined mesh per such group, so each element
 *   type of a group costs one launch per stage; every element keeps its own
 *   mesh's step, so results are bitwise those of stepping the mesh alone.  Each
 *   dg_batch_step copies the members' states into the combined meshes and back
 *   (one gather and one scatter kernel per group).  Creating a batch with groups
 *   synchronises and allocates the combined meshes (about the members' own
 *   device memory again).  Other meshes are graph branches of their own.
 * dg_batch_set_packing: 1 = step the groups through their combined meshes,
 *   0 = every mesh on its own branch (drops the cached graphs; synchronises).
 * dg_batch_autotune: times nsteps (rounded up to a multiple of DG_BATCH_CHUNK,
 *   1..30) batch steps packed and unpacked (best of two graph replays each, after
 *   a capture), keeps the faster and returns it in *packed (may be NULL); the
 *   meshes' states are restored.  Synchronises; allocates one state copy per mesh
 *   for the call.
 * dg_batch_destroy: synchronises the batch stream and frees the batch's graphs,
 *   streams, events and combined meshes (not the meshes). */
#define DG_BATCH_CHUNK 3
typedef struct dg_batch dg_batch;
dg_status dg_batch_create(dg_mesh *const *meshes, int count, void *cuda_stream, dg_batch **out);
dg_status dg_batch_step(dg_batch *batch, int nsteps, const double *dt, double *t_inout);
/* Graph replays and captures since creation (for tests and measurements). */
dg_status dg_batch_stats(const dg_batch *batch, int64_t *replays, int64_t *captures);
dg_status dg_batch_set_packing(dg_batch *batch, int packed);
dg_status dg_batch_autotune(dg_batch *batch, int nsteps, int *packed);
void dg_batch_destroy(dg_batch *batch);

/* ---- point source and receivers (hexahedra) --------------------------------
 * The pressure equation (1/kappa) p_t + div u = f of Sec. 2.2 with the point
 * source f = amp ricker(t) delta(x - x_s), ricker(t) = (1 - 2 a) exp(-a),
 * a = pi^2 f0^2 (t - t0)^2; the paper's experiments have f = 0.  Its weak form
 * adds amp ricker(t) M_K^{-1} phi(x_s) to the p rhs of the hexahedron K that
 * holds x_s.  Receivers read p(x_r) = sum_n phi_n(x_r) p_n.  Points are located
 * by Newton's method on the trilinear maps; a point on a face shared by two
 * hexahedra belongs to the one of lower index; DG_EINVAL if no hexahedron holds
 * it.  Host arrays are borrowed for the call; both calls synchronise and
 * allocate device memory (kept until the mesh is destroyed).
 * dg_set_source: x[3], amp, f0 > 0, t0.  With a source, dg_step needs t_inout
 *   (its value is the start time; DG_EINVAL if NULL), adds the source at the
 *   stage times t + c_k dt, and is built for nlevels = 1 only (DG_ENOTSUP);
 *   dg_rhs adds it at t; batches refuse the mesh (DG_ENOTSUP).
 * dg_set_receivers: xyz[nrec][3] (nrec = 0 removes them).
 * dg_sample_receivers: out_dev[nrec] (device FP32) = p at the receivers of the
 *   device state q_dev (NULL = the mesh's state); asynchronous. */
dg_status dg_set_source(dg_mesh *mesh, const double *x, double amp, double f0, double t0);
dg_status dg_set_receivers(dg_mesh *mesh, int nrec, const double *xyz);
dg_status dg_sample_receivers(dg_mesh *mesh, const float *q_dev, float *out_dev);

/* Discrete adjoint of nsteps single-rate LSRK(5,4) steps of size dt (dt <= 0:
 * dt_min, as dg_step) started at time t0 from the mesh's current state q_0 (a
 * checkpoint).  No counterpart in the paper: the exact derivative of the
 * discrete map of Sec. 2.2-2.4 (the FP32 forward kernels, recomputed from q_0,
 * with the point source if one is set), for a loss L of the states q_1..q_n
 * after the steps.
 *   lambda_dev   device [4][ndof] FP32: dL/dq_n from what follows the window on
 *                entry (zeros if nothing), dL/dq_0 on return.
 *   resid_dev    device [nsteps][nrec] FP32 or NULL: receiver forcing; row j is
 *                dL/dd of the receiver samples of q_{j+1}, so for
 *                L = 1/2 sum (d - d_obs)^2 it is d - d_obs (DG_EINVAL without
 *                receivers).
 *   grad_c2_dev  device, one double per element in the type order of dg_layout
 *                (hexahedra, wedges, pyramids, tets; element order within a
 *                type), or NULL: dL/dc^2_K is ADDED to it (c^2 enters through
 *                1/rho = c^2 and through tau_p = 1/{rho c}, tau_u = {rho c} on
 *                the element's faces).  Contributions are summed with atomics:
 *                the last bits vary from run to run.
 *   grad_amp_dev device double or NULL: dL/damp of the point source is ADDED to
 *                it (DG_EINVAL without a source).
 * The transpose of the operator is applied as R^T = W F R F W^{-1} with
 * W = blockdiag(M, M/c^2) the energy weight and F = diag(1,-1,-1,-1), exact
 * for GL hexahedra and skew-form pyramids; DG_ENOTSUP for SEM hexahedra,
 * strong-form pyramids and nlevels = 2.  The mesh state is left unchanged; the
 * LSRK residual and trace buffers are overwritten.  Allocates nsteps + 9 state
 * copies of scratch on first use (kept until the mesh is destroyed or a larger
 * nsteps needs more) and synchronises on that first use only; otherwise
 * asynchronous on the mesh's stream.  Chain windows of steps by calling it per
 * window, last window first, after restoring each window's checkpoint with
 * dg_set_state. */
dg_status dg_adjoint_step(dg_mesh *mesh, int nsteps, double dt, double t0, float *lambda_dev,
                          const float *resid_dev, double *grad_c2_dev, double *grad_amp_dev);

const char *dg_status_string(dg_status s);
/* Message of the last DG_ECUDA / DG_EMESH / DG_EINVAL error on this thread. */
const char *dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
