// Host setup of a dg_mesh (FP64): face matching in canonical face frames,
// geometric factors, reference operators, local time steps (Eq. dtK), upload.
//
// Canonical face frame (shared by the two elements of a face):
//   triangle  corners ordered by increasing global vertex id G0 < G1 < G2, point
//             (xi,eta) of {xi,eta >= -1, xi+eta <= 0} at barycentric weights
//             (-(xi+eta)/2, (1+xi)/2, (1+eta)/2) on (G0,G1,G2);
//   quad      C00 = smallest-id corner, C10 = its edge neighbour of smaller id,
//             C01 = the other edge neighbour, C11 = opposite; bilinear blend.
// Face points: collapsed rule (N+1)^2 on triangles, GL (N+1)^2 on quads.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <stdexcept>

#include "internal.h"
#include "refelem.h"

using namespace dgref;

namespace {

struct SetupError : std::runtime_error {
  dg_status code;
  SetupError(dg_status c, const std::string& s) : std::runtime_error(s), code(c) {}
};

// dx_d/dr_a of the vertex map, F[3*d + a].
void map_jacobian(int t, const double* xv, const double* rst, double F[9]) {
  double r = rst[0], s = rst[1], u = rst[2];
  std::memset(F, 0, 9 * sizeof(double));
  if (t == HEX) {
    for (int v = 0; v < 8; ++v) {
      const double* c = vert_rst(HEX, v);
      double fr = 0.5 * (1 + c[0] * r), fs = 0.5 * (1 + c[1] * s), ft = 0.5 * (1 + c[2] * u);
      double g[3] = {0.5 * c[0] * fs * ft, fr * 0.5 * c[1] * ft, fr * fs * 0.5 * c[2]};
      for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a) F[3 * d + a] += xv[3 * v + d] * g[a];
    }
  } else if (t == TET) {
    for (int d = 0; d < 3; ++d)
      for (int a = 0; a < 3; ++a) F[3 * d + a] = 0.5 * (xv[3 * (a + 1) + d] - xv[d]);
  } else if (t == WEDGE) {
    double lam[3] = {-0.5 * (r + u), 0.5 * (1 + r), 0.5 * (1 + u)};
    double lr[3] = {-0.5, 0.5, 0.0}, lt[3] = {-0.5, 0.0, 0.5};
    double f0 = 0.5 * (1 - s), f1 = 0.5 * (1 + s);
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 3; ++v) {
        double lo = xv[3 * v + d], hi = xv[3 * (v + 3) + d];
        F[3 * d + 0] += lr[v] * (f0 * lo + f1 * hi);
        F[3 * d + 1] += lam[v] * 0.5 * (hi - lo);
        F[3 * d + 2] += lt[v] * (f0 * lo + f1 * hi);
      }
  } else {  // pyramid: x = (1-c)/2 B(a,b) + (1+c)/2 x_apex
    double h = 0.5 * (1 - u);
    double a = (1 + r) / h - 1, b = (1 + s) / h - 1;
    double Nab[4] = {0.25 * (1 - a) * (1 - b), 0.25 * (1 + a) * (1 - b), 0.25 * (1 - a) * (1 + b),
                     0.25 * (1 + a) * (1 + b)};
    double Na[4] = {-0.25 * (1 - b), 0.25 * (1 - b), -0.25 * (1 + b), 0.25 * (1 + b)};
    double Nb[4] = {-0.25 * (1 - a), -0.25 * (1 + a), 0.25 * (1 - a), 0.25 * (1 + a)};
    for (int d = 0; d < 3; ++d) {
      double B = 0, Ba = 0, Bb = 0;
      for (int v = 0; v < 4; ++v) {
        B += Nab[v] * xv[3 * v + d];
        Ba += Na[v] * xv[3 * v + d];
        Bb += Nb[v] * xv[3 * v + d];
      }
      F[3 * d + 0] = Ba;
      F[3 * d + 1] = Bb;
      F[3 * d + 2] = 0.5 * (1 + a) * Ba + 0.5 * (1 + b) * Bb + 0.5 * (xv[12 + d] - B);
    }
  }
}

double det3(const double F[9]) {
  return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
         F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// G[a][d] = d r_a / d x_d = inverse of F (F[d][a]).
double inverse_metric(const double F[9], double G[9]) {
  double J = det3(F);
  // columns of F: x_r, x_s, x_t; rows of G: (x_s x x_t)/J, (x_t x x_r)/J, (x_r x x_s)/J
  double c[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) c[a][d] = F[3 * d + a];
  auto cross = [](const double* p, const double* q, double* o) {
    o[0] = p[1] * q[2] - p[2] * q[1];
    o[1] = p[2] * q[0] - p[0] * q[2];
    o[2] = p[0] * q[1] - p[1] * q[0];
  };
  cross(c[1], c[2], G + 0);
  cross(c[2], c[0], G + 3);
  cross(c[0], c[1], G + 6);
  for (int i = 0; i < 9; ++i) G[i] /= J;
  return J;
}

// Reference gradient of J for the wedge map (second derivatives x_rs, x_ts are constant).
void wedge_grad_J(const double* xv, const double* rst, double gJ[3]) {
  double F[9];
  map_jacobian(WEDGE, xv, rst, F);
  double lr[3] = {-0.5, 0.5, 0.0}, lt[3] = {-0.5, 0.0, 0.5};
  double xrs[3] = {0, 0, 0}, xts[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 3; ++v) {
      double diff = 0.5 * (xv[3 * (v + 3) + d] - xv[3 * v + d]);
      xrs[d] += lr[v] * diff;
      xts[d] += lt[v] * diff;
    }
  auto detcols = [&](const double* c0, const double* c1, const double* c2) {
    double M[9];
    for (int d = 0; d < 3; ++d) {
      M[3 * d] = c0[d];
      M[3 * d + 1] = c1[d];
      M[3 * d + 2] = c2[d];
    }
    return det3(M);
  };
  double xr[3], xs[3], xt[3];
  for (int d = 0; d < 3; ++d) {
    xr[d] = F[3 * d];
    xs[d] = F[3 * d + 1];
    xt[d] = F[3 * d + 2];
  }
  gJ[0] = detcols(xr, xrs, xt);                       // d x_s/dr = x_rs
  gJ[1] = detcols(xrs, xs, xt) + detcols(xr, xs, xts); // d x_r/ds, d x_t/ds
  gJ[2] = detcols(xr, xts, xt);                       // d x_s/dt = x_ts
}

// Exact volume rule on a reference element (for reference mass matrices).
void volume_rule(int t, int q, std::vector<double>& P, std::vector<double>& W) {
  std::vector<double> x, wx, y, wy, z, wz;
  P.clear();
  W.clear();
  if (t == HEX) {
    gauss_jacobi(q, 0, 0, x, wx);
    for (int k = 0; k < q; ++k)
      for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) {
          P.insert(P.end(), {x[i], x[j], x[k]});
          W.push_back(wx[i] * wx[j] * wx[k]);
        }
  } else if (t == WEDGE) {
    std::vector<double> tp, tw;
    tri_rule(q - 1, tp, tw);
    gauss_jacobi(q, 0, 0, x, wx);
    for (int l = 0; l < q; ++l)
      for (size_t m = 0; m < tw.size(); ++m) {
        P.insert(P.end(), {tp[2 * m], x[l], tp[2 * m + 1]});
        W.push_back(tw[m] * wx[l]);
      }
  } else if (t == PYR) {
    gauss_jacobi(q, 0, 0, x, wx);
    gauss_jacobi(q, 2, 0, z, wz);
    for (int k = 0; k < q; ++k)
      for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) {
          double h = 0.5 * (1 - z[k]);
          P.insert(P.end(), {(1 + x[i]) * h - 1, (1 + x[j]) * h - 1, z[k]});
          W.push_back(wx[i] * wx[j] * wz[k] / 4.0);
        }
  } else {
    gauss_jacobi(q, 0, 0, x, wx);
    gauss_jacobi(q, 1, 0, y, wy);
    gauss_jacobi(q, 2, 0, z, wz);
    for (int k = 0; k < q; ++k)
      for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) {
          double r = 0.25 * (1 + x[i]) * (1 - y[j]) * (1 - z[k]) - 1;
          double s = 0.5 * (1 + y[j]) * (1 - z[k]) - 1;
          P.insert(P.end(), {r, s, z[k]});
          W.push_back(wx[i] * wy[j] * wz[k] / 8.0);
        }
  }
}

// Largest eigenvalue of the symmetric-definite pencil (A, B): Cholesky B = L L^T and
// cyclic Jacobi rotations on L^{-1} A L^{-T}.
double max_gen_eig(std::vector<double> A, std::vector<double> B, int n) {
  for (int j = 0; j < n; ++j) {  // Cholesky, lower
    double s = B[j * n + j];
    for (int k = 0; k < j; ++k) s -= B[j * n + k] * B[j * n + k];
    B[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double v = B[i * n + j];
      for (int k = 0; k < j; ++k) v -= B[i * n + k] * B[j * n + k];
      B[i * n + j] = v / B[j * n + j];
    }
  }
  // C = L^{-1} A L^{-T}: solve L X = A, then L C^T = X^T
  auto lsolve = [&](std::vector<double>& X) {
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < n; ++i) {
        double v = X[i * n + c];
        for (int k = 0; k < i; ++k) v -= B[i * n + k] * X[k * n + c];
        X[i * n + c] = v / B[i * n + i];
      }
  };
  lsolve(A);
  std::vector<double> T(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) T[i * n + j] = A[j * n + i];
  lsolve(T);
  std::vector<double>& C = T;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += C[p * n + q] * C[p * n + q];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = C[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double th = 0.5 * (C[q * n + q] - C[p * n + p]) / apq;
        double tt = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < n; ++k) {
          double akp = C[k * n + p], akq = C[k * n + q];
          C[k * n + p] = c * akp - s * akq;
          C[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = C[p * n + k], aqk = C[q * n + k];
          C[p * n + k] = c * apk - s * aqk;
          C[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  double mx = -1e300;
  for (int i = 0; i < n; ++i) mx = std::max(mx, C[i * n + i]);
  return mx;
}

// Reference trace constant C_T(N) (Appendix B), Euclidean face measure of the reference element;
// lobatto: SEM (GLL points on the quadrilateral faces, GLL-collocated hex mass), Table
// computedTraceSEM.
double trace_constant_eval(const Basis& B, bool lobatto) {
  int t = B.type, N = B.N, Np = B.Np;
  std::vector<double> P, W;
  volume_rule(t, N + 2, P, W);
  std::vector<double> M(Np * Np, 0.0), Ms(Np * Np, 0.0), phi(Np);
  for (size_t q = 0; q < W.size(); ++q) {
    B.eval(&P[3 * q], phi.data(), nullptr);
    for (int i = 0; i < Np; ++i)
      for (int j = 0; j < Np; ++j) M[i * Np + j] += W[q] * phi[i] * phi[j];
  }
  for (int f = 0; f < nfaces(t); ++f) {
    int nv = face_nverts(t, f);
    int key[4] = {0, 1, 2, 3};
    std::vector<double> pts, w;
    if (nv == 3) tri_rule(N, pts, w); else quad_rule(N, pts, w, lobatto);
    for (size_t q = 0; q < w.size(); ++q) {
      double rst[3], d1[3], d2[3];
      face_point(t, f, key, pts[2 * q], pts[2 * q + 1], rst, d1, d2);
      double cr[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2],
                      d1[0] * d2[1] - d1[1] * d2[0]};
      double ar = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      B.eval(rst, phi.data(), nullptr);
      for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) Ms[i * Np + j] += w[q] * ar * phi[i] * phi[j];
    }
  }
  return max_gen_eig(Ms, M, Np);
}

// C_T depends on the reference element alone: computed once per (type, N, node set) and process.
double trace_constant(const Basis& B, bool lobatto = false) {
  if (B.type == HEX) return lobatto ? 1.5 * B.N * (B.N + 1) : 1.5 * (B.N + 1) * (B.N + 2);
  static std::mutex mu;
  static std::map<std::array<int, 3>, double> cache;
  const std::array<int, 3> key{B.type, B.N, lobatto ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const double v = trace_constant_eval(B, lobatto);
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = v;
  return v;
}

// Canonical corner order (positions within the local corner list) of a face.
void canonical_key(int nv, const int64_t* gid, int key[4]) {
  if (nv == 3) {
    int o[3] = {0, 1, 2};
    std::sort(o, o + 3, [&](int x, int y) { return gid[x] < gid[y]; });
    key[0] = o[0]; key[1] = o[1]; key[2] = o[2]; key[3] = -1;
    return;
  }
  static const int cyc[4] = {0, 1, 3, 2};
  int p = 0;
  for (int m = 1; m < 4; ++m)
    if (gid[cyc[m]] < gid[cyc[p]]) p = m;
  int n1 = cyc[(p + 1) % 4], n2 = cyc[(p + 3) % 4];
  key[0] = cyc[p];
  key[1] = gid[n1] < gid[n2] ? n1 : n2;
  key[2] = gid[n1] < gid[n2] ? n2 : n1;
  key[3] = cyc[(p + 2) % 4];
}

int key_to_code(int nv, const int key[4]) {
  for (int c = 0; c < (nv == 3 ? 6 : 8); ++c) {
    int k2[4];
    face_code_key(nv, c, k2);
    bool ok = true;
    for (int m = 0; m < nv; ++m) ok &= (k2[m] == key[m]);
    if (ok) return c;
  }
  throw SetupError(DG_EMESH, "face orientation not recognised");
}

thread_local bool g_host_only = false;   // dg_host_check: run the host setup only

// Device bytes of the current setup call and an optional budget (environment DG_DEVICE_BYTES_LIMIT,
// read per dg_mesh_create): past it the setup fails with DG_ENOMEM before calling cudaMalloc, so
// out-of-memory handling can be exercised without exhausting a GPU.
thread_local size_t g_dev_bytes = 0, g_dev_limit = 0;
void* device_alloc(size_t bytes) {
  if (g_dev_limit && g_dev_bytes + bytes > g_dev_limit)
    throw SetupError(DG_ENOMEM, "device byte budget (DG_DEVICE_BYTES_LIMIT) exceeded");
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) throw SetupError(DG_ENOMEM, "cudaMalloc failed");
  g_dev_bytes += bytes;
  return p;
}

template <class T>
T* upload(const std::vector<T>& h, std::vector<void*>& owned) {
  if (h.empty() || g_host_only) return nullptr;
  void* p = device_alloc(h.size() * sizeof(T));
  owned.push_back(p);
  if (cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    throw SetupError(DG_ECUDA, "cudaMemcpy failed");
  return static_cast<T*>(p);
}

template <class T>
T* alloc_zero(size_t n, std::vector<void*>& owned) {
  void* p = nullptr;
  if (g_host_only) return nullptr;
  if (n == 0) n = 1;
  p = device_alloc(n * sizeof(T));
  owned.push_back(p);
  if (cudaMemset(p, 0, n * sizeof(T)) != cudaSuccess) throw SetupError(DG_ECUDA, "cudaMemset failed");
  return static_cast<T*>(p);
}

std::vector<void*>& owned_list(dg_mesh* m);


// ----------------------------------------------------------------------------- orientation-free face operators
// Triangle faces use the equispaced face lattice (l0,l1,l2), l0+l1+l2 = N, indexed
// by (l1,l2) with l2 outer, l1 inner.  A lattice node has barycentric weights l/N on
// the face's local corners; in the canonical frame its weights are l permuted by the
// face key, so the frame only permutes lattice nodes.  E[q][n] interpolates values at
// the canonical lattice to the canonical quadrature points (exact for P_N traces).
// Quadrilateral faces are handled at local GL points plus a permutation (hexperm).
int lattice_index(int N, int l1, int l2) {
  int idx = 0;
  for (int b = 0; b < l2; ++b) idx += N + 1 - b;
  return idx + l1;
}

void lattice_tables(int N, std::vector<int>& tperm, std::vector<int>& tinv, std::vector<double>& E,
                    const std::vector<double>& tpts) {
  const int nfn = (N + 1) * (N + 2) / 2, nq = (N + 1) * (N + 1);
  tperm.assign(6 * nfn, 0);
  tinv.assign(6 * nfn, 0);
  for (int c = 0; c < 6; ++c) {
    int key[4];
    face_code_key(3, c, key);
    for (int l2 = 0; l2 <= N; ++l2)
      for (int l1 = 0; l1 + l2 <= N; ++l1) {
        int l[3] = {N - l1 - l2, l1, l2};
        int m1 = l[key[1]], m2 = l[key[2]];
        int nl = lattice_index(N, l1, l2), nc = lattice_index(N, m1, m2);
        tperm[c * nfn + nl] = nc;
        tinv[c * nfn + nc] = nl;
      }
  }
  // Lagrange basis of the lattice via monomials in (lam1, lam2), evaluated at the face points
  std::vector<double> V(nfn * nfn);
  auto mono = [&](double a, double b, double* out) {
    int k = 0;
    for (int i = 0; i <= N; ++i)
      for (int j = 0; i + j <= N; ++j) out[k++] = std::pow(a, i) * std::pow(b, j);
  };
  for (int l2 = 0; l2 <= N; ++l2)
    for (int l1 = 0; l1 + l2 <= N; ++l1) mono((double)l1 / N, (double)l2 / N, &V[lattice_index(N, l1, l2) * nfn]);
  // invert V (rows = nodes, cols = monomials)
  std::vector<double> I(nfn * nfn, 0.0);
  for (int i = 0; i < nfn; ++i) I[i * nfn + i] = 1;
  for (int c = 0; c < nfn; ++c) {
    int p = c;
    for (int r = c + 1; r < nfn; ++r)
      if (std::fabs(V[r * nfn + c]) > std::fabs(V[p * nfn + c])) p = r;
    for (int k = 0; k < nfn; ++k) {
      std::swap(V[p * nfn + k], V[c * nfn + k]);
      std::swap(I[p * nfn + k], I[c * nfn + k]);
    }
    double dv = 1.0 / V[c * nfn + c];
    for (int k = 0; k < nfn; ++k) { V[c * nfn + k] *= dv; I[c * nfn + k] *= dv; }
    for (int r = 0; r < nfn; ++r) {
      if (r == c) continue;
      double f = V[r * nfn + c];
      for (int k = 0; k < nfn; ++k) { V[r * nfn + k] -= f * V[c * nfn + k]; I[r * nfn + k] -= f * I[c * nfn + k]; }
    }
  }
  // ell_n(x) = sum_k mono_k(x) I[k][n]   (I = V^{-1}: V[n][k] = mono_k(x_n))
  E.assign(nq * nfn, 0.0);
  std::vector<double> mv(nfn);
  for (int q = 0; q < nq; ++q) {
    mono(0.5 * (1 + tpts[2 * q]), 0.5 * (1 + tpts[2 * q + 1]), mv.data());
    for (int n = 0; n < nfn; ++n) {
      double v = 0;
      for (int k = 0; k < nfn; ++k) v += mv[k] * I[k * nfn + n];
      E[q * nfn + n] = v;
    }
  }
}

}  // namespace

// ----------------------------------------------------------------------------- registry of allocations
#include <mutex>
#include <unordered_map>
namespace {
std::mutex g_mu;
std::unordered_map<dg_mesh*, std::vector<void*>> g_owned;
std::vector<void*>& owned_list(dg_mesh* m) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_owned[m];
}
}  // namespace

dg_status dg_setup_host_only(dg_mesh* m, const dg_mesh_desc* d, std::string& err, double ct[4]) {
  g_host_only = true;
  dg_status st = dg_setup(m, d, err);
  g_host_only = false;
  if (st == DG_OK && ct) {
    for (int t = 0; t < 4; ++t) {
      Basis B;
      B.init(t, d->N, d->hex_basis == 1 && t == HEX);
      ct[t] = trace_constant(B, d->hex_basis == 1);
    }
  }
  dg_free(m);
  return st;
}

void* dg_alloc_owned(dg_mesh* m, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  owned_list(m).push_back(p);
  return p;
}

void dg_free(dg_mesh* m) {
  std::vector<void*> v;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_owned.find(m);
    if (it != g_owned.end()) {
      v.swap(it->second);
      g_owned.erase(it);
    }
  }
  for (void* p : v) cudaFree(p);
  if (m->adj_buf) cudaFree(m->adj_buf);
  m->adj_buf = nullptr;
}

dg_status dg_setup(dg_mesh* m, const dg_mesh_desc* d, std::string& err) {
  g_dev_bytes = 0;
  const char* lim = std::getenv("DG_DEVICE_BYTES_LIMIT");
  g_dev_limit = lim ? std::strtoull(lim, nullptr, 10) : 0;
  try {
    std::vector<void*>& owned = owned_list(m);
    const int N = d->N;
    m->N = N;
    const int n1 = N + 1, nq = n1 * n1;
    m->nq = nq;
    m->tau_scale = d->tau_scale;
    m->cfl = d->cfl > 0 ? d->cfl : 0.5;
    m->pyr_form = d->pyr_form;
    m->precision = d->precision;
    m->integrator = d->nlevels == 2 ? d->integrator : 0;
    const bool sem = d->hex_basis == 1;   // SEM hexahedra: GLL nodes, GLL points on quad faces
    m->hex_sem = sem;
    Basis B[4];
    for (int t = 0; t < 4; ++t) B[t].init(t, N, sem && t == HEX);
    m->hex_r1 = B[HEX].r1;
    m->hex_w1 = B[HEX].w1;
    m->hex_coef.assign((size_t)d->nelem[HEX] * 24, 0.0);
    const int nfc[4] = {6, 5, 5, 4};

    // --- offsets
    int64_t dof = 0, side = 0;
    for (int t = 0; t < 4; ++t) {
      m->K[t] = d->nelem[t];
      auto& td = m->td[t];
      td.K = (int)d->nelem[t];
      td.Np = B[t].Np;
      td.nf = nfc[t];
      td.dof_off = dof;
      td.side_off = side;
      dof += d->nelem[t] * B[t].Np;
      side += d->nelem[t] * nfc[t];
    }
    m->ndof = dof;
    m->nsides = side;

    // --- face matching by sorted vertex ids
    struct FaceKey {
      std::array<int64_t, 4> v;
      int64_t side;
    };
    std::vector<FaceKey> keys(side);
    std::vector<int> nbr(side, -1), code(side, 0);
    std::vector<float> tau(side, 0.f);
    std::vector<double> taud(side, 0.0);
    std::vector<std::array<int, 4>> skey(side);
    for (int t = 0; t < 4; ++t) {
      int nv = nverts(t);
      for (int64_t e = 0; e < d->nelem[t]; ++e) {
        const int32_t* cv = d->conn[t] + e * nv;
        for (int f = 0; f < nfc[t]; ++f) {
          int64_t s = m->td[t].side_off + e * nfc[t] + f;
          int fn = face_nverts(t, f);
          const int* fv = face_verts(t, f);
          int64_t gid[4] = {-1, -1, -1, -1};
          for (int c = 0; c < fn; ++c) {
            int32_t g = cv[fv[c]];
            if (g < 0 || g >= d->nverts) throw SetupError(DG_EINVAL, "vertex id out of range");
            gid[c] = g;
          }
          int key[4];
          canonical_key(fn, gid, key);
          code[s] = key_to_code(fn, key);
          for (int c = 0; c < 4; ++c) skey[s][c] = key[c];
          FaceKey fk;
          fk.v = {gid[0], gid[1], gid[2], gid[3]};
          std::sort(fk.v.begin(), fk.v.begin() + fn);
          fk.side = s;
          keys[s] = fk;
        }
      }
    }
    std::sort(keys.begin(), keys.end(), [](const FaceKey& a, const FaceKey& b) { return a.v < b.v; });
    for (size_t i = 0; i < keys.size();) {
      size_t j = i + 1;
      while (j < keys.size() && keys[j].v == keys[i].v) ++j;
      if (j - i > 2) throw SetupError(DG_EMESH, "face shared by more than two elements");
      if (j - i == 2) {
        nbr[keys[i].side] = (int)keys[i + 1].side;
        nbr[keys[i + 1].side] = (int)keys[i].side;
      }
      i = j;
    }
    // element of a side and its wave speed
    auto side_elem = [&](int64_t s, int& t, int64_t& e, int& f) {
      t = 3;
      while (t > 0 && s < m->td[t].side_off) --t;
      int64_t r = s - m->td[t].side_off;
      e = r / nfc[t];
      f = (int)(r % nfc[t]);
    };
    // triangle faces exchange lattice values (tet, pyramid) unless a wedge's triangle face meets
    // a tet or pyramid: the wedge's trace is not a polynomial there, so the whole mesh then keeps
    // the quadrature-point exchange of the older kernels for tets and pyramids
    m->tri_lat = true;
    for (int64_t s = 0; s < side; ++s) {
      int t, f, t2, f2;
      int64_t e, e2;
      if (nbr[s] < 0) continue;
      side_elem(s, t, e, f);
      side_elem(nbr[s], t2, e2, f2);
      if (face_nverts(t, f) == 3 && (t == WEDGE) != (t2 == WEDGE)) m->tri_lat = false;
    }
    for (int64_t s = 0; s < side; ++s) {
      int t, f, t2, f2;
      int64_t e, e2;
      side_elem(s, t, e, f);
      double c2m = d->c2[t][e];
      if (!(c2m > 0)) throw SetupError(DG_EINVAL, "c2 must be positive");
      double cm = std::sqrt(c2m), cp = cm;
      if (nbr[s] >= 0) {
        side_elem(nbr[s], t2, e2, f2);
        cp = std::sqrt(d->c2[t2][e2]);
      }
      taud[s] = 1.0 / (0.5 * (1.0 / cm + 1.0 / cp));  // 1/{rho c}, rho c = 1/c
      tau[s] = (float)taud[s];
    }

    // --- face rules in canonical coordinates
    std::vector<double> tpts, tw, qpts, qw;
    tri_rule(N, tpts, tw);
    quad_rule(N, qpts, qw, sem);

    // --- per-type geometry, operators and time-step data
    double CT[4];
    for (int t = 0; t < 4; ++t) CT[t] = trace_constant(B[t], sem);
    std::vector<double> jsmax[4], jinvmax[4], jsj[4], taup[4], tauu[4];
    for (int t = 0; t < 4; ++t) {
      int K = m->td[t].K;
      jsmax[t].assign(K, 0.0);
      jinvmax[t].assign(K, 0.0);
      jsj[t].assign(K, 0.0);
      taup[t].assign(K, 0.0);
      tauu[t].assign(K, 0.0);
    }
    int npmax = 0;   // basis values of the largest element (the hexahedron's (N+1)^3)
    for (int t = 0; t < 4; ++t) npmax = std::max(npmax, B[t].Np);
    std::vector<double> phi(npmax);
    m->face_w.assign((size_t)m->nsides * nq, 0.f);

    for (int t = 0; t < 4; ++t) {
      auto& td = m->td[t];
      const int K = td.K, Np = td.Np, nf = td.nf, nv = nverts(t);
      std::vector<float> c2f(K);
      for (int e = 0; e < K; ++e) c2f[e] = (float)d->c2[t][e];
      td.c2 = upload(c2f, owned);
      auto load_xv = [&](int64_t e, double* xv) {
        const int32_t* cv = d->conn[t] + e * nv;
        for (int v = 0; v < nv; ++v)
          for (int c = 0; c < 3; ++c) xv[3 * v + c] = d->xyz[3 * (int64_t)cv[v] + c];
      };
      // the element loops below run in parallel: each writes its own slices, errors are
      // collected and raised after the loop
      std::atomic<const char*> bad{nullptr};
      auto flag = [&](const char* msg) {
        const char* none = nullptr;
        bad.compare_exchange_strong(none, msg);
      };
      // volume geometry
      std::vector<double> wedge_pts, wedge_w;
      if (t == WEDGE) {
        std::vector<double> tp, tww, sx, sw;
        tri_rule(N, tp, tww);
        gauss_jacobi(n1, 0, 0, sx, sw);
        for (int l = 0; l < n1; ++l)
          for (size_t q = 0; q < tww.size(); ++q) {
            wedge_pts.insert(wedge_pts.end(), {tp[2 * q], sx[l], tp[2 * q + 1]});
            wedge_w.push_back(tww[q] * sw[l]);
          }
        td.nc = (int)wedge_w.size();
        std::vector<float> wp;   // triangle points (r, t), then the 1D points s
        for (double v : tp) wp.push_back((float)v);
        for (double v : sx) wp.push_back((float)v);
        td.wpts = upload(wp, owned);
      }
      const int gstride = t == HEX ? 24 : t == TET ? 12 : t == PYR ? 10 * Np : 16;
      std::vector<float> geo((size_t)K * gstride, 0.f);
#pragma omp parallel for schedule(dynamic, 256)
      for (int64_t e = 0; e < K; ++e) {
        double xv[24];
        load_xv(e, xv);
        float* ge = geo.data() + (size_t)e * gstride;
        double F[9], G[9];
        if (t == HEX) {
          // x = c0 + c1 r + c2 s + c3 t + c4 rs + c5 rt + c6 st + c7 rst (coefficients c1..c7)
          double cf[8][3] = {};
          for (int v = 0; v < 8; ++v) {
            const double* c = vert_rst(HEX, v);
            double mon[8] = {1, c[0], c[1], c[2], c[0] * c[1], c[0] * c[2], c[1] * c[2],
                             c[0] * c[1] * c[2]};
            for (int mm = 0; mm < 8; ++mm)
              for (int dd = 0; dd < 3; ++dd) cf[mm][dd] += 0.125 * mon[mm] * xv[3 * v + dd];
          }
          for (int mm = 1; mm < 8; ++mm)
            for (int dd = 0; dd < 3; ++dd) ge[3 * (mm - 1) + dd] = (float)cf[mm][dd];
          for (int mm = 0; mm < 8; ++mm)
            for (int dd = 0; dd < 3; ++dd) m->hex_coef[(size_t)e * 24 + 3 * mm + dd] = cf[mm][dd];
          double jmin = 1e300;
          for (int n = 0; n < Np; ++n) {
            map_jacobian(HEX, xv, &B[t].nodes[3 * n], F);
            double J = det3(F);
            jmin = std::min(jmin, J);
            jinvmax[t][e] = std::max(jinvmax[t][e], 1.0 / J);
          }
          if (!(jmin > 0)) flag("hexahedron with J <= 0");
        } else if (t == TET) {
          double rst0[3] = {-1, -1, -1};
          map_jacobian(TET, xv, rst0, F);
          double J = inverse_metric(F, G);
          if (!(J > 0)) flag("tetrahedron with J <= 0");
          for (int i = 0; i < 9; ++i) ge[i] = (float)G[i];
          ge[9] = (float)J;
          jinvmax[t][e] = 1.0 / J;
        } else if (t == PYR) {
          for (int n = 0; n < Np; ++n) {
            double a = B[t].lev_x[B[t].mk[n]][B[t].mi[n]], b = B[t].lev_x[B[t].mk[n]][B[t].mj[n]];
            double rst[3] = {0.5 * (a - 1), 0.5 * (b - 1), 0.0};
            map_jacobian(PYR, xv, rst, F);
            double J = inverse_metric(F, G);
            if (!(J > 0)) flag("pyramid with J <= 0");
            for (int i = 0; i < 9; ++i) ge[i * Np + n] = (float)G[i];   // [10][Np]: component-major
            ge[9 * Np + n] = (float)J;
            jinvmax[t][e] = std::max(jinvmax[t][e], 1.0 / J);
          }
        } else {  // wedge: J > 0 at every cubature point; the kernels rebuild the metric terms
          for (int q = 0; q < td.nc; ++q) {
            map_jacobian(WEDGE, xv, &wedge_pts[3 * q], F);
            double J = inverse_metric(F, G);
            if (!(J > 0)) flag("wedge with J <= 0");
          }
          // map coefficients: with lo / hi the bottom / top vertex of each triangle corner v,
          // x_r = sum_v lr_v (lo + hi) / 2 + s sum_v lr_v (hi - lo) / 2 (likewise x_t with lt) and
          // x_s = sum_v lam_v(r, t) (hi - lo) / 2, lam = (0, 1/2, 1/2) + r lr + t lt
          const double lr[3] = {-0.5, 0.5, 0.0}, lt[3] = {-0.5, 0.0, 0.5}, l0[3] = {0.0, 0.5, 0.5};
          for (int d = 0; d < 3; ++d) {
            double ar = 0, br = 0, at = 0, bt = 0, cs = 0;
            for (int v = 0; v < 3; ++v) {
              const double lo = xv[3 * v + d], hi = xv[3 * (v + 3) + d];
              ar += lr[v] * 0.5 * (lo + hi);
              br += lr[v] * 0.5 * (hi - lo);
              at += lt[v] * 0.5 * (lo + hi);
              bt += lt[v] * 0.5 * (hi - lo);
              cs += l0[v] * 0.5 * (hi - lo);
            }
            ge[d] = (float)ar;
            ge[3 + d] = (float)br;
            ge[6 + d] = (float)at;
            ge[9 + d] = (float)bt;
            ge[12 + d] = (float)cs;
          }
        }
      }
      if (bad.load()) throw SetupError(DG_EMESH, bad.load());
      td.geo = upload(geo, owned);

      // face geometry (non-hex: stored; all types: time-step data)
      const size_t nfq = (size_t)K * nf * nq;
      std::vector<float4> sgeo(t == HEX ? 0 : nfq), sgeo2(t == HEX ? 0 : nfq);
      std::vector<float> sisq(t == WEDGE ? nfq : 0), sisq2(t == WEDGE ? nfq : 0);
#pragma omp parallel for schedule(dynamic, 256)
      for (int64_t e = 0; e < K; ++e) {
        double xv[24];
        load_xv(e, xv);
        for (int f = 0; f < nf; ++f) {
          int64_t s = td.side_off + e * nf + f;
          int fnv = face_nverts(t, f);
          int key[4];
          for (int c = 0; c < 4; ++c) key[c] = skey[s][c];
          const std::vector<double>& pts = fnv == 3 ? tpts : qpts;
          const std::vector<double>& w = fnv == 3 ? tw : qw;
          const double* og = face_outward(t, f);
          taup[t][e] = std::max(taup[t][e], taud[s]);
          tauu[t][e] = std::max(tauu[t][e], 1.0 / taud[s]);
          double js0 = 0.0;
          for (int pass = 0; pass < (t == HEX ? 1 : 2); ++pass)
          for (int q = 0; q < nq; ++q) {
            double rst[3], d1[3], d2[3], F[9], G[9];
            // pass 0: canonical points; pass 1: the order of the orientation-free kernels
            // (canonical points on triangles, local points on quadrilaterals)
            static const int ident[4] = {0, 1, 2, 3};
            const int* kk = (pass == 1 && fnv == 4) ? ident : key;
            face_point(t, f, kk, pts[2 * q], pts[2 * q + 1], rst, d1, d2);
            map_jacobian(t, xv, rst, F);
            double J = inverse_metric(F, G);
            double x1[3], x2[3], nn[3];
            for (int dd = 0; dd < 3; ++dd) {
              x1[dd] = F[3 * dd] * d1[0] + F[3 * dd + 1] * d1[1] + F[3 * dd + 2] * d1[2];
              x2[dd] = F[3 * dd] * d2[0] + F[3 * dd + 1] * d2[1] + F[3 * dd + 2] * d2[2];
              nn[dd] = G[0 + dd] * og[0] + G[3 + dd] * og[1] + G[6 + dd] * og[2];
            }
            double cr[3] = {x1[1] * x2[2] - x1[2] * x2[1], x1[2] * x2[0] - x1[0] * x2[2],
                            x1[0] * x2[1] - x1[1] * x2[0]};
            double Js = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            double rc[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2],
                            d1[0] * d2[1] - d1[1] * d2[0]};
            double Jsref = std::sqrt(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]);
            double nl = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            if (pass == 0) {
              jsmax[t][e] = std::max(jsmax[t][e], Js / Jsref);
              jsj[t][e] = std::max(jsj[t][e], Js / Jsref / J);
              // face measure at the canonical points (adjoint): w J^s, or J^s alone on a face
              // whose traces are exchanged at the lattice (the face mass carries the weights)
              const bool lat = m->tri_lat && fnv == 3 && (t == TET || t == PYR);
              m->face_w[(size_t)s * nq + q] = (float)(lat ? Js : w[q] * Js);
            }
            if (!(J > 0)) flag("J <= 0 at a face point");
            if (t != HEX) {
              double wj = w[q] * Js;
              if (t == WEDGE) wj /= std::sqrt(J);
              if (pass == 1 && fnv == 3 && t != WEDGE) {
                // lattice exchange: the face is affine, n and J^s are constant over it; the
                // quadrature weights live in the face mass matrix folded into the lift
                wj = Js;
                if (q == 0) js0 = Js;
                else if (std::fabs(Js - js0) > 1e-9 * js0)
                  flag("triangle face of a tet or pyramid is not affine");
              }
              const size_t at = ((size_t)e * nf + f) * nq + q;
              float4 gv = make_float4((float)(nn[0] / nl), (float)(nn[1] / nl), (float)(nn[2] / nl), (float)wj);
              (pass == 0 ? sgeo : sgeo2)[at] = gv;
              if (t == WEDGE) (pass == 0 ? sisq : sisq2)[at] = (float)(1.0 / std::sqrt(J));
            }
          }
        }
      }
      if (bad.load()) throw SetupError(DG_EMESH, bad.load());
      if (t != HEX) {
        td.sgeo = upload(sgeo, owned);
        td.sgeo2 = upload(sgeo2, owned);
        if (t == WEDGE) {
          td.sisq = upload(sisq, owned);
          td.sisq2 = upload(sisq2, owned);
        }
      }

      // reference operators
      if (t == HEX) {
        std::vector<float> hc;
        std::vector<double> l(n1), dl(n1);
        for (int i = 0; i < n1; ++i) {
          lagrange(B[t].r1, B[t].r1[i], l.data(), dl.data());
          for (int mm = 0; mm < n1; ++mm) hc.push_back((float)dl[mm]);  // D1[i][m] = l_m'(r_i)
        }
        lagrange(B[t].r1, -1.0, l.data(), nullptr);
        for (int i = 0; i < n1; ++i) hc.push_back((float)l[i]);
        lagrange(B[t].r1, 1.0, l.data(), nullptr);
        for (int i = 0; i < n1; ++i) hc.push_back((float)l[i]);
        for (int i = 0; i < n1; ++i) hc.push_back((float)B[t].w1[i]);
        for (int i = 0; i < n1; ++i) hc.push_back((float)B[t].r1[i]);
        for (int i = 0; i < n1; ++i) hc.push_back((float)(1.0 / B[t].w1[i]));
        m->hexc = upload(hc, owned);
        if (!g_host_only && dgk::upload_hex_constants(N, sem, hc.data(), (int)hc.size()) != cudaSuccess)
          throw SetupError(DG_ECUDA, "constant upload failed");
        // local face point (iu + n1 iv) -> canonical index, per code
        std::vector<int> perm(dgk::NCODES * nq, 0);
        const double P[4][2] = {{-1, -1}, {1, -1}, {-1, 1}, {1, 1}};
        for (int c = 0; c < dgk::NCODES; ++c) {
          int key[4];
          face_code_key(4, c, key);
          for (int ib = 0; ib < n1; ++ib)
            for (int ia = 0; ia < n1; ++ia) {
              double al = B[t].r1[ia], be = B[t].r1[ib];
              double uv[2];
              for (int k2 = 0; k2 < 2; ++k2)
                uv[k2] = P[key[0]][k2] + 0.5 * (1 + al) * (P[key[1]][k2] - P[key[0]][k2]) +
                         0.5 * (1 + be) * (P[key[2]][k2] - P[key[0]][k2]);
              int iu = 0, iv = 0;
              for (int i = 0; i < n1; ++i) {
                if (std::fabs(B[t].r1[i] - uv[0]) < std::fabs(B[t].r1[iu] - uv[0])) iu = i;
                if (std::fabs(B[t].r1[i] - uv[1]) < std::fabs(B[t].r1[iv] - uv[1])) iv = i;
              }
              perm[c * nq + iu + n1 * iv] = ia + n1 * ib;
            }
        }
        m->hexperm = upload(perm, owned);
      } else {
        // trace (transposed) and lift matrices per (face, code)
        std::vector<float> Tt((size_t)nf * dgk::NCODES * Np * nq, 0.f), L((size_t)nf * dgk::NCODES * nq * Np, 0.f);
        std::vector<double> Minv;
        if (t == TET) {  // reference mass of the nodal basis and its inverse
          std::vector<double> P, W;
          volume_rule(TET, N + 2, P, W);
          std::vector<double> M(Np * Np, 0.0);
          for (size_t q = 0; q < W.size(); ++q) {
            B[t].eval(&P[3 * q], phi.data(), nullptr);
            for (int i = 0; i < Np; ++i)
              for (int j = 0; j < Np; ++j) M[i * Np + j] += W[q] * phi[i] * phi[j];
          }
          m->tet_mhat = M;
          Minv = M;
          // Gauss-Jordan inverse
          std::vector<double> I(Np * Np, 0.0);
          for (int i = 0; i < Np; ++i) I[i * Np + i] = 1;
          for (int c = 0; c < Np; ++c) {
            int p = c;
            for (int r = c + 1; r < Np; ++r)
              if (std::fabs(Minv[r * Np + c]) > std::fabs(Minv[p * Np + c])) p = r;
            for (int k = 0; k < Np; ++k) {
              std::swap(Minv[p * Np + k], Minv[c * Np + k]);
              std::swap(I[p * Np + k], I[c * Np + k]);
            }
            double dv = 1.0 / Minv[c * Np + c];
            for (int k = 0; k < Np; ++k) { Minv[c * Np + k] *= dv; I[c * Np + k] *= dv; }
            for (int r = 0; r < Np; ++r) {
              if (r == c) continue;
              double fct = Minv[r * Np + c];
              for (int k = 0; k < Np; ++k) { Minv[r * Np + k] -= fct * Minv[c * Np + k]; I[r * Np + k] -= fct * I[c * Np + k]; }
            }
          }
          Minv = I;
          m->tet_mhat_inv = Minv;
          std::vector<float> mh(M.begin(), M.end());
          m->tet_mhat_dev = upload(mh, owned);
          // Cholesky factor M = R^T R (R upper triangular): the energy kernel takes p^T M p = |R p|^2
          std::vector<double> R(Np * Np, 0.0);
          for (int i = 0; i < Np; ++i) {
            double d = M[i * Np + i];
            for (int k = 0; k < i; ++k) d -= R[k * Np + i] * R[k * Np + i];
            if (!(d > 0)) throw SetupError(DG_EINVAL, "tet reference mass not positive definite");
            R[i * Np + i] = std::sqrt(d);
            for (int j = i + 1; j < Np; ++j) {
              double v = M[i * Np + j];
              for (int k = 0; k < i; ++k) v -= R[k * Np + i] * R[k * Np + j];
              R[i * Np + j] = v / R[i * Np + i];
            }
          }
          std::vector<float> rf(R.begin(), R.end());
          m->tet_chol_dev = upload(rf, owned);
        }
        for (int f = 0; f < nf; ++f) {
          int fnv = face_nverts(t, f);
          const std::vector<double>& pts = fnv == 3 ? tpts : qpts;
          for (int c = 0; c < (fnv == 3 ? 6 : 8); ++c) {
            int key[4];
            face_code_key(fnv, c, key);
            std::vector<double> T(nq * Np);
            for (int q = 0; q < nq; ++q) {
              double rst[3], d1[3], d2[3];
              face_point(t, f, key, pts[2 * q], pts[2 * q + 1], rst, d1, d2);
              B[t].eval(rst, phi.data(), nullptr);
              for (int i = 0; i < Np; ++i) T[q * Np + i] = phi[i];
            }
            size_t base = ((size_t)f * dgk::NCODES + c) * nq * Np;
            for (int q = 0; q < nq; ++q)
              for (int i = 0; i < Np; ++i) {
                Tt[base + (size_t)i * nq + q] = (float)T[q * Np + i];
                double li = T[q * Np + i];
                if (t == TET) {
                  li = 0;
                  for (int j = 0; j < Np; ++j) li += Minv[i * Np + j] * T[q * Np + j];
                }
                L[base + (size_t)q * Np + i] = (float)li;
              }
          }
        }
        td.Tt = upload(Tt, owned);
        td.L = upload(L, owned);
        // volume operators
        std::vector<float> ops;
        std::vector<double> Mc, Cc;   // pyramid level-pair c-integrals (sum-factorised operators)
        if (t == TET) {
          // DT[a][m][n] = d l_m / d r_a (x_n)
          std::vector<double> g(3 * Np);
          std::vector<double> D(3 * Np * Np);
          for (int n = 0; n < Np; ++n) {
            B[t].eval(&B[t].nodes[3 * n], phi.data(), g.data());
            for (int a = 0; a < 3; ++a)
              for (int mm = 0; mm < Np; ++mm) D[(a * Np + mm) * Np + n] = g[a * Np + mm];
          }
          ops.assign(D.begin(), D.end());
        } else if (t == PYR) {
          // quadrature-free weak derivative operators (Sec. 2.3.4), factor (1+a)/2 at the test node
          const Basis& Bp = B[t];
          std::vector<double> c, wc;
          gauss_jacobi(2 * N + 4, 0, 0, c, wc);
          Mc.assign(n1 * n1, 0.0);
          Cc.assign(n1 * n1, 0.0);
          for (int n = 0; n <= N; ++n)
            for (int k = 0; k <= N; ++k) {
              double s1 = 0, s2 = 0;
              for (size_t q = 0; q < c.size(); ++q) {
                double h = 0.5 * (1 - c[q]);
                double Pk = jacobi(N - k, 2 * k + 3, 0, c[q]), dPk = jacobi_deriv(N - k, 2 * k + 3, 0, c[q]);
                double Pn = jacobi(N - n, 2 * n + 3, 0, c[q]);
                s1 += wc[q] * Pk * Pn * std::pow(h, 1 + k + n);
                double dk = dPk * std::pow(h, k) - (k > 0 ? 0.5 * k * std::pow(h, k - 1) * Pk : 0.0);
                s2 += wc[q] * dk * Pn * std::pow(h, 2 + n);
              }
              double nrm = std::sqrt(Bp.gam[n] * Bp.gam[k]);
              Mc[n * n1 + k] = s1 / nrm;
              Cc[n * n1 + k] = s2 / nrm;
            }
          std::vector<double> Dr(Np * Np), Ds(Np * Np), Dt(Np * Np);
          std::vector<double> la(n1), dla(n1), lb(n1), dlb(n1);
          for (int row = 0; row < Np; ++row) {
            int l = Bp.mi[row], mm = Bp.mj[row], n = Bp.mk[row];
            double al = Bp.lev_x[n][l], bm = Bp.lev_x[n][mm];
            for (int col = 0; col < Np; ++col) {
              int i = Bp.mi[col], j = Bp.mj[col], k = Bp.mk[col];
              lagrange(Bp.lev_x[k], al, la.data(), dla.data());
              lagrange(Bp.lev_x[k], bm, lb.data(), dlb.data());
              double fac = std::sqrt(Bp.lev_w[n][l] * Bp.lev_w[n][mm] / (Bp.lev_w[k][i] * Bp.lev_w[k][j]));
              double dr = fac * dla[i] * lb[j] * Mc[n * n1 + k];
              double ds = fac * la[i] * dlb[j] * Mc[n * n1 + k];
              double dc = fac * la[i] * lb[j] * Cc[n * n1 + k];
              Dr[row * Np + col] = dr;
              Ds[row * Np + col] = ds;
              Dt[row * Np + col] = 0.5 * (1 + al) * dr + 0.5 * (1 + bm) * ds + dc;
            }
          }
          // D[a][m][n] = D^a_{m n} (row m), then DT[a][m][n] = D^a_{n m}
          ops.resize(6 * Np * Np);
          const std::vector<double>* Ds3[3] = {&Dr, &Ds, &Dt};
          for (int a = 0; a < 3; ++a)
            for (int i = 0; i < Np; ++i)
              for (int j = 0; j < Np; ++j) {
                ops[(a * Np + i) * Np + j] = (float)(*Ds3[a])[i * Np + j];
                ops[3 * Np * Np + (a * Np + j) * Np + i] = (float)(*Ds3[a])[i * Np + j];
              }
        } else {  // wedge: V[nc][Np], Vg[3][nc][Np], VT[Np][nc], VgT[3][Np][nc], w[nc]
          int nc = td.nc;
          std::vector<double> g(3 * Np);
          ops.assign((size_t)8 * nc * Np + nc, 0.f);
          for (int q = 0; q < nc; ++q) {
            B[t].eval(&wedge_pts[3 * q], phi.data(), g.data());
            for (int i = 0; i < Np; ++i) {
              ops[(size_t)q * Np + i] = (float)phi[i];
              ops[(size_t)4 * nc * Np + (size_t)i * nc + q] = (float)phi[i];
              for (int a = 0; a < 3; ++a) {
                ops[(size_t)(1 + a) * nc * Np + (size_t)q * Np + i] = (float)g[a * Np + i];
                ops[(size_t)(5 + a) * nc * Np + (size_t)i * nc + q] = (float)g[a * Np + i];
              }
            }
            ops[(size_t)8 * nc * Np + q] = (float)wedge_w[q];
          }
        }
        td.ops = upload(ops, owned);

        // ---- orientation-free operators (kernels_gen2.cu); float layout:
        //  tet:   DV4[Np][Np] (D^r,D^s,D^t,0) | Lf[4][nfn][Np] = Mhat^{-1} face-node columns x Mf | E[nq][nfn]
        //  pyr:   DV4[Np][Np] | EF[4][nkl] | PF[4][nfn][nkl] | PF2[4][nfn][nkl] | LA[n1][nkl] | GC[n1] | E[nq][nfn]
        //         (nkl = (N+1)(N+2)/2 level-index pairs (k, l <= k))
        //  wedge: Vt4[nq][ntri] | V1[n1][n1] | D1[n1][n1] | w[nq][n1] | Vtl[2][nfn][ntri] | Ve[3][n1][ntri] |
        //         V1e[2][n1] | V1q[n1][n1] | E[nq][nfn]
        //  int layout: tperm[6][nfn] | tinv[6][nfn] | qperm[8][nq] | (tet) fnode[4][nfn]
        const int nfn = (N + 1) * (N + 2) / 2;
        std::vector<int> tperm, tinv;
        std::vector<double> E;
        lattice_tables(N, tperm, tinv, E, tpts);
        // face mass matrix of the lattice basis, Mf[m][n] = sum_q w_q l_m(x_q) l_n(x_q); it is
        // invariant under the six vertex permutations of the (symmetric) lattice
        std::vector<double> Mf(nfn * nfn, 0.0);
        for (int a = 0; a < nfn; ++a)
          for (int b2 = 0; b2 < nfn; ++b2)
            for (int q = 0; q < nq; ++q) Mf[a * nfn + b2] += tw[q] * E[q * nfn + a] * E[q * nfn + b2];
        m->face_mass = Mf;
        std::vector<float> o2;
        std::vector<int> i2(tperm.begin(), tperm.end());
        i2.insert(i2.end(), tinv.begin(), tinv.end());
        {
          // quad perm (same construction as the hexahedron's)
          const double P[4][2] = {{-1, -1}, {1, -1}, {-1, 1}, {1, 1}};
          std::vector<double> gx, gw;
          gauss_jacobi(n1, 0, 0, gx, gw);
          std::vector<int> qp(dgk::NCODES * nq, 0);
          for (int c = 0; c < dgk::NCODES; ++c) {
            int key[4];
            face_code_key(4, c, key);
            for (int ib = 0; ib < n1; ++ib)
              for (int ia = 0; ia < n1; ++ia) {
                double uv[2];
                for (int k2 = 0; k2 < 2; ++k2)
                  uv[k2] = P[key[0]][k2] + 0.5 * (1 + gx[ia]) * (P[key[1]][k2] - P[key[0]][k2]) +
                           0.5 * (1 + gx[ib]) * (P[key[2]][k2] - P[key[0]][k2]);
                int iu = 0, iv = 0;
                for (int i = 0; i < n1; ++i) {
                  if (std::fabs(gx[i] - uv[0]) < std::fabs(gx[iu] - uv[0])) iu = i;
                  if (std::fabs(gx[i] - uv[1]) < std::fabs(gx[iv] - uv[1])) iv = i;
                }
                qp[c * nq + iu + n1 * iv] = ia + n1 * ib;
              }
          }
          i2.insert(i2.end(), qp.begin(), qp.end());
        }
        auto lattice_rst = [&](int f, int l1, int l2, double rst[3]) {
          const int* fv = face_verts(t, f);
          const double l[3] = {(double)(N - l1 - l2) / N, (double)l1 / N, (double)l2 / N};
          for (int c = 0; c < 3; ++c)
            rst[c] = l[0] * vert_rst(t, fv[0])[c] + l[1] * vert_rst(t, fv[1])[c] + l[2] * vert_rst(t, fv[2])[c];
        };
        std::vector<double> gg(3 * Np);
        if (t == TET) {
          // DV4[n][m] = (D^r, D^s, D^t, 0)[n][m], row n = node / test function (ops holds DT[a][m][n])
          for (int n = 0; n < Np; ++n)
            for (int mm = 0; mm < Np; ++mm) {
              for (int a = 0; a < 3; ++a) o2.push_back(ops[(a * Np + mm) * Np + n]);
              o2.push_back(0.f);
            }
        }
        if (t == PYR) {
          // Sum-factorised volume operators (Sec. 2.3.4): the semi-nodal basis is a product of 1D
          // Lagrange factors per level, so with test level q, trial level k,
          //   D^r[(l,p,q),(i,j,k)] = E'qk[l][i] Eqk[p][j] cr[q][k],  D^s: E[l][i] E'[p][j] cr,
          //   D^t = (1+a_l)/2 D^r + (1+a_p)/2 D^s + E[l][i] E[p][j] cc[q][k],
          // Eqk[l][i] = sqrt(w^q_l / w^k_i) l^k_i(a^q_l), E' with the derivative of l^k_i (the GL rule
          // of level q integrates the a and b factors exactly), cr = Mc (nonzero for |q - k| <= 1),
          // cc = Cc (nonzero for k <= q + 1).  Layout: FE[n1][n1][n1][n1] (q, k, l, i) | FD (same) |
          // CR[n1][n1] | CC[n1][n1] | AH[n1][n1] = (1 + a^q_l)/2.
          const Basis& Bp = B[t];
          std::vector<float> fe((size_t)n1 * n1 * n1 * n1, 0.f), fd(fe.size(), 0.f), cr(n1 * n1, 0.f),
              cc(n1 * n1, 0.f), ah(n1 * n1, 0.f);
          std::vector<double> lk(n1), dlk(n1);
          for (int q = 0; q <= N; ++q) {
            for (int l = 0; l <= q; ++l) ah[q * n1 + l] = (float)(0.5 * (1 + Bp.lev_x[q][l]));
            for (int k = 0; k <= N; ++k) {
              if (std::abs(q - k) <= 1) cr[q * n1 + k] = (float)Mc[q * n1 + k];
              if (k <= q + 1) cc[q * n1 + k] = (float)Cc[q * n1 + k];
              for (int l = 0; l <= q; ++l) {
                lagrange(Bp.lev_x[k], Bp.lev_x[q][l], lk.data(), dlk.data());
                for (int i = 0; i <= k; ++i) {
                  const double f = std::sqrt(Bp.lev_w[q][l] / Bp.lev_w[k][i]);
                  fe[((size_t)(q * n1 + k) * n1 + l) * n1 + i] = (float)(f * lk[i]);
                  fd[((size_t)(q * n1 + k) * n1 + l) * n1 + i] = (float)(f * dlk[i]);
                }
              }
            }
          }
          o2.insert(o2.end(), fe.begin(), fe.end());
          o2.insert(o2.end(), fd.begin(), fd.end());
          o2.insert(o2.end(), cr.begin(), cr.end());
          o2.insert(o2.end(), cc.begin(), cc.end());
          o2.insert(o2.end(), ah.begin(), ah.end());
          // work items of the factorised products (ints after the face tables): PB[q][k] = first item
          // of level pair (q, k) (-1: no pair), then items (q, k, a, b) packed q | k << 4 | a << 8 |
          // b << 12 for the pairs with k <= q + 1, a < k + 1 (trial-level index), b < q + 1
          // (test-level index), a-major within a pair
          std::vector<int> pb(n1 * n1, -1), it;
          for (int q = 0; q <= N; ++q)
            for (int k = 0; k <= std::min(q + 1, N); ++k) {
              pb[q * n1 + k] = (int)it.size();
              for (int a = 0; a <= k; ++a)
                for (int b = 0; b <= q; ++b) it.push_back(q | (k << 4) | (a << 8) | (b << 12));
            }
          i2.insert(i2.end(), pb.begin(), pb.end());
          i2.insert(i2.end(), it.begin(), it.end());
        }
        if (t == TET) {
          std::vector<int> fnode(4 * nfn, -1);
          for (int f = 0; f < 4; ++f)
            for (int l2 = 0; l2 <= N; ++l2)
              for (int l1 = 0; l1 + l2 <= N; ++l1) {
                double rst[3];
                lattice_rst(f, l1, l2, rst);
                for (int n = 0; n < Np; ++n) {
                  const double* x = &B[t].nodes[3 * n];
                  if (std::fabs(x[0] - rst[0]) + std::fabs(x[1] - rst[1]) + std::fabs(x[2] - rst[2]) < 1e-9)
                    fnode[f * nfn + lattice_index(N, l1, l2)] = n;
                }
              }
          for (int v : fnode)
            if (v < 0) throw SetupError(DG_EINVAL, "tet face lattice not found among the nodes");
          // lift of lattice-point fluxes: Lf[f][n][i] = sum_m Mhat^{-1}[i][fnode[f][m]] Mf[m][n]
          for (int f = 0; f < 4; ++f)
            for (int n = 0; n < nfn; ++n)
              for (int i = 0; i < Np; ++i) {
                double v = 0.0;
                for (int mm = 0; mm < nfn; ++mm) v += Minv[i * Np + fnode[f * nfn + mm]] * Mf[mm * nfn + n];
                o2.push_back((float)v);
              }
          i2.insert(i2.end(), fnode.begin(), fnode.end());
        } else {
          if (t == WEDGE) {
            // tensor-product factors of the wedge basis and cubature (Sec. 2.3.3): phi_(mt,j) =
            // phi_tri_mt(r,t) phi_1D_j(s); points (qt, l).  Layout: Vt4[nqt][ntri] (phi, d/dr, d/dt, 0) |
            // V1[n1 (l)][n1 (j)] | D1[n1][n1] | w[nqt][n1] (w[qt] * w_l).
            const int ntri = Np / n1, nqt = nq;   // (N+1)(N+2)/2 triangle modes, (N+1)^2 triangle points
            std::vector<double> tp, tww, sx, sw;
            tri_rule(N, tp, tww);
            gauss_jacobi(n1, 0, 0, sx, sw);
            std::vector<double> Vt(nqt * ntri), Vtr(nqt * ntri), Vtt(nqt * ntri), V1(n1 * n1), D1(n1 * n1);
            // separable factors from the full basis: phi_(mt,0) = phi_tri_mt * phi_1D_0, phi_1D_0 = 1/sqrt(2)
            for (int qt = 0; qt < nqt; ++qt) {
              double rst[3] = {tp[2 * qt], 0.0, tp[2 * qt + 1]};
              B[t].eval(rst, phi.data(), gg.data());
              for (int mt = 0; mt < ntri; ++mt) {
                Vt[qt * ntri + mt] = phi[mt] * std::sqrt(2.0);
                Vtr[qt * ntri + mt] = gg[mt] * std::sqrt(2.0);
                Vtt[qt * ntri + mt] = gg[2 * Np + mt] * std::sqrt(2.0);
              }
            }
            for (int l = 0; l < n1; ++l)
              for (int j = 0; j < n1; ++j) {
                V1[l * n1 + j] = std::sqrt((2.0 * j + 1) / 2) * jacobi(j, 0, 0, sx[l]);
                D1[l * n1 + j] = std::sqrt((2.0 * j + 1) / 2) * jacobi_deriv(j, 0, 0, sx[l]);
              }
            // check the factorisation against the full basis at every cubature point
            for (int q = 0; q < td.nc; ++q) {
              const int qt = q % nqt, l = q / nqt;
              B[t].eval(&wedge_pts[3 * q], phi.data(), gg.data());
              for (int mm = 0; mm < Np; ++mm) {
                const int mt = mm % ntri, j = mm / ntri;
                const double ref[4] = {phi[mm], gg[mm], gg[Np + mm], gg[2 * Np + mm]};
                const double fac[4] = {Vt[qt * ntri + mt] * V1[l * n1 + j], Vtr[qt * ntri + mt] * V1[l * n1 + j],
                                       Vt[qt * ntri + mt] * D1[l * n1 + j], Vtt[qt * ntri + mt] * V1[l * n1 + j]};
                for (int c = 0; c < 4; ++c)
                  if (std::fabs(ref[c] - fac[c]) > 1e-10 * (1 + std::fabs(ref[c])))
                    throw SetupError(DG_EINVAL, "wedge basis does not factor");
              }
            }
            for (int qt = 0; qt < nqt; ++qt)
              for (int mt = 0; mt < ntri; ++mt) {
                o2.push_back((float)Vt[qt * ntri + mt]);
                o2.push_back((float)Vtr[qt * ntri + mt]);
                o2.push_back((float)Vtt[qt * ntri + mt]);
                o2.push_back(0.f);
              }
            for (double v : V1) o2.push_back((float)v);
            for (double v : D1) o2.push_back((float)v);
            for (int qt = 0; qt < nqt; ++qt)
              for (int l = 0; l < n1; ++l) o2.push_back((float)(tww[qt] * sw[l]));
          }
          // triangle-face lattice evaluations, then evaluations at the quad faces' local points
          std::vector<double> gx, gw;
          face_rule_1d(N, sem, gx, gw);
          if (t == WEDGE) {
            // factorised face evaluations of phi_(mt,j) = phi_tri_mt(r,t) phi_1D_j(s):
            //   Vtl[2][nfn][ntri]  phi_tri at the lattice of the triangle faces (s = -1, +1)
            //   Ve[3][n1][ntri]    phi_tri at the GL points along the edge of each quad face
            //                      (local u; local v runs along s)
            //   V1e[2][n1]         phi_1D_j(-1), phi_1D_j(+1)
            const int ntri = Np / n1;
            for (int f = 0; f < 2; ++f)
              for (int l2 = 0; l2 <= N; ++l2)
                for (int l1 = 0; l1 + l2 <= N; ++l1) {
                  double rst[3];
                  lattice_rst(f, l1, l2, rst);
                  const double rt[3] = {rst[0], 0.0, rst[2]};
                  B[t].eval(rt, phi.data(), nullptr);
                  for (int mt = 0; mt < ntri; ++mt) o2.push_back((float)(phi[mt] * std::sqrt(2.0)));
                }
            static const int ident4[4] = {0, 1, 2, 3};
            for (int f = 2; f < 5; ++f)
              for (int ia = 0; ia < n1; ++ia) {
                double rst[3], d1[3], d2[3];
                face_point(t, f, ident4, gx[ia], -1.0, rst, d1, d2);
                const double rt[3] = {rst[0], 0.0, rst[2]};
                B[t].eval(rt, phi.data(), nullptr);
                for (int mt = 0; mt < ntri; ++mt) o2.push_back((float)(phi[mt] * std::sqrt(2.0)));
              }
            for (int f = 0; f < 2; ++f)
              for (int j = 0; j < n1; ++j)
                o2.push_back((float)(std::sqrt((2.0 * j + 1) / 2) * jacobi(j, 0, 0, f == 0 ? -1.0 : 1.0)));
            //   V1q[n1][n1]        phi_1D_j at the quad faces' points along s (GL, or GLL with SEM)
            for (int l = 0; l < n1; ++l)
              for (int j = 0; j < n1; ++j) o2.push_back((float)(std::sqrt((2.0 * j + 1) / 2) * jacobi(j, 0, 0, gx[l])));
          }
          if (t == PYR) {
            // factorised face evaluations of the semi-nodal basis
            //   phi_kji = [l^k_i(a)/sqrt(w^k_i)] [l^k_j(b)/sqrt(w^k_j)] [h^k P^{(2k+3,0)}_{N-k}(t)/sqrt(gamma_k)]:
            // triangle face f = 1..4 fixes b = -1, a = +1, b = +1, a = -1; per (k, l), l <= k:
            //   EF[4][nkl]        the fixed coordinate's factor
            //   PF[4][nfn][nkl]   at lattice node x of the face: the free coordinate's factor times the t factor
            //   PF2[4][nfn][nkl]  = Mf PF (lift of lattice-point fluxes)
            // base (t = -1, h = 1, local GL points (a_p, b_q)):
            //   LA[n1][nkl]       l^k_l(x_p)/sqrt(w^k_l);   GC[n1]  P^{(2k+3,0)}_{N-k}(-1)/sqrt(gamma_k)
            const int nkl = n1 * (n1 + 1) / 2;
            std::vector<double> tmp(n1);
            auto lag = [&](int k, double x) {
              lagrange(B[t].lev_x[k], x, tmp.data(), nullptr);
              for (int l = 0; l <= k; ++l) tmp[l] /= std::sqrt(B[t].lev_w[k][l]);
            };
            const bool fixa[4] = {false, true, false, true};
            const double fixv[4] = {-1.0, 1.0, 1.0, -1.0};
            for (int ti = 0; ti < 4; ++ti)
              for (int k = 0; k <= N; ++k) {
                lag(k, fixv[ti]);
                for (int l = 0; l <= k; ++l) o2.push_back((float)tmp[l]);
              }
            std::vector<double> pf(4 * nfn * nkl);
            for (int ti = 0; ti < 4; ++ti)
              for (int l2 = 0; l2 <= N; ++l2)
                for (int l1 = 0; l1 + l2 <= N; ++l1) {
                  double rst[3];
                  lattice_rst(ti + 1, l1, l2, rst);
                  const double h = 0.5 * (1 - rst[2]);
                  const double a = h > 1e-14 ? (1 + rst[0]) / h - 1 : 0.0, b = h > 1e-14 ? (1 + rst[1]) / h - 1 : 0.0;
                  const int x = lattice_index(N, l1, l2);
                  for (int k = 0; k <= N; ++k) {
                    const double tk = std::pow(h, k) * jacobi(N - k, 2 * k + 3, 0, rst[2]) / std::sqrt(B[t].gam[k]);
                    lag(k, fixa[ti] ? b : a);
                    for (int l = 0; l <= k; ++l) pf[(ti * nfn + x) * nkl + k * (k + 1) / 2 + l] = tmp[l] * tk;
                  }
                }
            for (double v : pf) o2.push_back((float)v);
            for (int ti = 0; ti < 4; ++ti)
              for (int n = 0; n < nfn; ++n)
                for (int kl = 0; kl < nkl; ++kl) {
                  double v = 0.0;
                  for (int mm = 0; mm < nfn; ++mm) v += Mf[n * nfn + mm] * pf[(ti * nfn + mm) * nkl + kl];
                  o2.push_back((float)v);
                }
            for (int pp = 0; pp < n1; ++pp)
              for (int k = 0; k <= N; ++k) {
                lag(k, gx[pp]);
                for (int l = 0; l <= k; ++l) o2.push_back((float)tmp[l]);
              }
            for (int k = 0; k <= N; ++k) o2.push_back((float)(jacobi(N - k, 2 * k + 3, 0, -1.0) / std::sqrt(B[t].gam[k])));
          }
        }
        for (double v : E) o2.push_back((float)v);
        if (t != WEDGE) while (o2.size() % 4) o2.push_back(0.f);   // the kernels' size check (OPS_T)
        if (t == TET) {
          // the volume operator transposed (float4 rows), 16-byte aligned after the operators
          std::vector<float> dt4((size_t)Np * Np * 4);
          for (int n = 0; n < Np; ++n)
            for (int mm = 0; mm < Np; ++mm)
              for (int c = 0; c < 4; ++c) dt4[((size_t)mm * Np + n) * 4 + c] = o2[((size_t)n * Np + mm) * 4 + c];
          o2.insert(o2.end(), dt4.begin(), dt4.end());
        }
        td.ops2 = upload(o2, owned);
        td.iops2 = upload(i2, owned);
        td.nops2 = (int)o2.size();
        td.niops2 = (int)i2.size();
        // the operands of Y = B X in split 16-bit form, Y, and the TMA descriptors of X and B
        auto prec_buffers = [&](dgk::PrecDev& P, const std::vector<float>& b, int64_t rows) {
          P.b32 = upload(b, owned);
          P.bh = alloc_zero<unsigned short>(b.size(), owned);
          P.bl = alloc_zero<unsigned short>(b.size(), owned);
          P.xh = alloc_zero<unsigned short>((size_t)rows * P.kx, owned);
          P.xl = alloc_zero<unsigned short>((size_t)rows * P.kx, owned);
          P.xis = alloc_zero<float>((size_t)rows, owned);
          P.y = alloc_zero<float>((size_t)rows * P.nblk * P.npp, owned);
          if (dgk::prec_split_operator(P, P.b32, d->precision == 1, nullptr) != cudaSuccess ||
              !dgk::prec_maps(m->prec_maps[dgk::prec_slot(t)], P, rows))
            throw SetupError(DG_ECUDA, "tensor-core operands: operator split or TMA descriptors failed");
        };
        if (d->precision > 0 && (t == TET || t == PYR) && td.K > 0 && !g_host_only && Np <= 512) {
          // tensor-core volume products (kernels_prec.cu): the block operator B [4 npl][4 npk] from
          // D^a[x][y] = o2[(x Np + y) 4 + a]: block 0 (sum_a D^a W_a; pyramid (D^a)^T) reads the
          // three field columns of X, blocks 1..3 (D^a p) its p columns.  One MMA's N and one TMA
          // box hold at most 256 rows of B: above 256 nodes (pyramids at N = 8, 9) each block is
          // computed in two halves of npp rows (eight GEMM blocks, the same X columns per pair)
          dgk::PrecDev& P = m->prec[dgk::prec_slot(t)];
          const int halves = Np <= 256 ? 1 : 2;
          P.npk = (Np + 15) / 16 * 16;
          P.npp = halves == 1 ? P.npk : ((Np + 1) / 2 + 15) / 16 * 16;
          const int npk = P.npk, npl = halves * P.npp;   // npl: a block's width in Y
          P.vnp = npl;
          P.nblk = 4 * halves;
          P.kx = 4 * npk;
          for (int lb = 0; lb < 4; ++lb)
            for (int h = 0; h < halves; ++h) {
              P.kb0[lb * halves + h] = lb == 0 ? 0 : 3 * npk;
              P.kbn[lb * halves + h] = lb == 0 ? 3 * npk : npk;
            }
          std::vector<float> b((size_t)4 * npl * 4 * npk, 0.f);
          float bmax = 0.f;
          // D^a[x][y]: tets from DV4 (o2), pyramids from the dense host operators (ops: D[a][x][y])
          auto dop = [&](int a, int x, int y) -> float {
            return t == TET ? o2[((size_t)x * Np + y) * 4 + a] : ops[((size_t)a * Np + x) * Np + y];
          };
          for (int n = 0; n < Np; ++n)
            for (int mm = 0; mm < Np; ++mm)
              for (int a = 0; a < 3; ++a) {
                const float dnm = dop(a, n, mm), dmn = dop(a, mm, n);
                b[(size_t)n * 4 * npk + a * npk + mm] = t == TET ? dnm : dmn;
                b[(size_t)((1 + a) * npl + n) * 4 * npk + 3 * npk + mm] = dnm;
                bmax = std::max(bmax, std::fabs(dnm));
              }
          P.bis = bmax > 0.f ? std::ldexp(1.f, std::ilogb(bmax) - 14) : 1.f;   // operator scaled into [2^14, 2^15)
          const int64_t rows = (td.K + 127) / 128 * 128;
          prec_buffers(P, b, rows);
        } else if (d->precision > 0 && t == WEDGE && td.K > 0 && !g_host_only && N >= 7) {
          // wedges, N >= 7: the first contraction of the sum-factorised volume term (triangle
          // modes -> triangle cubature points) on the tensor cores (at N = 5 the X / Y round trip
          // through memory costs more than the FP32 contraction it replaces).  A row of X per
          // (element, 1D level l) holds five triangle-mode vectors [V1 p | D1 p | V1 u | V1 v | V1 w]
          // (npk columns each); B has seven blocks of npp cubature points: V, V_r, V_t against V1 p;
          // V against D1 p, V1 u, V1 v, V1 w, with V/V_r/V_t[qt][mt] = o2[(qt NT + mt) 4 + {0, 1, 2}]
          const int ntri = Np / n1, nqt = n1 * n1;
          dgk::PrecDev& P = m->prec[dgk::prec_slot(t)];
          P.npk = (ntri + 15) / 16 * 16;
          P.npp = (nqt + 15) / 16 * 16;
          const int npk = P.npk, npp = P.npp;
          P.vnp = npp;
          P.nblk = 7;
          P.kx = 5 * npk;
          const int xblk[7] = {0, 0, 0, 1, 2, 3, 4}, comp[7] = {0, 1, 2, 0, 0, 0, 0};
          std::vector<float> b((size_t)7 * npp * 5 * npk, 0.f);
          float bmax = 0.f;
          for (int bb = 0; bb < 7; ++bb) {
            P.kb0[bb] = xblk[bb] * npk;
            P.kbn[bb] = npk;
            for (int qt = 0; qt < nqt; ++qt)
              for (int mt = 0; mt < ntri; ++mt) {
                const float v = o2[((size_t)qt * ntri + mt) * 4 + comp[bb]];
                b[(size_t)(bb * npp + qt) * 5 * npk + xblk[bb] * npk + mt] = v;
                bmax = std::max(bmax, std::fabs(v));
              }
          }
          P.bis = bmax > 0.f ? std::ldexp(1.f, std::ilogb(bmax) - 14) : 1.f;
          const int64_t rows = (td.K * n1 + 127) / 128 * 128;
          prec_buffers(P, b, rows);
        }
      }
    }

    // --- local time steps (Eq. dtK)
    m->dt_min = 1e300;
    for (int t = 0; t < 4; ++t) {
      m->dtK[t].assign(m->td[t].K, 0.0);
      for (int e = 0; e < m->td[t].K; ++e) {
        double crk = std::max(taup[t][e], tauu[t][e] * d->c2[t][e]);
        double cj = t == WEDGE ? jsj[t][e] : jsmax[t][e] * jinvmax[t][e];
        double dte = m->cfl / (crk * CT[t] * cj);
        m->dtK[t][e] = dte;
        m->dt_min = std::min(m->dt_min, dte);
      }
    }

    // --- multi-rate levels (Sec. 2.4): level 1 = coarse, nlevels = fine; dtau_lev = 2^(nlevels-lev) dtau_min
    const int nlev = d->nlevels < 1 ? 1 : d->nlevels;
    m->nlevels = nlev;
    std::vector<std::vector<int>> level(4);
    for (int t = 0; t < 4; ++t) {
      level[t].assign(m->td[t].K, nlev);
      for (int e = 0; e < m->td[t].K; ++e)
        for (int L = 1; L <= nlev; ++L)
          if (std::ldexp(m->dt_min, nlev - L) <= m->dtK[t][e] * (1 + 1e-12)) {
            level[t][e] = L;
            break;
          }
    }
    for (bool changed = true; changed;) {   // neighbours differ by at most one level
      changed = false;
      for (int64_t s = 0; s < side; ++s) {
        if (nbr[s] < 0) continue;
        int t, f, t2, f2;
        int64_t e, e2;
        side_elem(s, t, e, f);
        side_elem(nbr[s], t2, e2, f2);
        if (level[t][e] < level[t2][e2] - 1) {
          level[t][e] = level[t2][e2] - 1;
          changed = true;
        }
      }
    }
    for (int t = 0; t < 4; ++t) {
      m->all.count[t] = m->td[t].K;
      m->all.list[t] = nullptr;
    }
    if (nlev == 2) {
      for (int L = 0; L < 2; ++L) {
        for (int t = 0; t < 4; ++t) {
          std::vector<int> lst;
          for (int e = 0; e < m->td[t].K; ++e)
            if (level[t][e] == L + 1) lst.push_back(e);
          m->lev[L].count[t] = (int64_t)lst.size();
          m->lev[L].list[t] = upload(lst, owned);
          m->level_count[L] += (int64_t)lst.size();
        }
      }
      m->hist = alloc_zero<float>(3 * 4 * (size_t)m->ndof, owned);
      m->trace3 = alloc_zero<float>(2 * (size_t)side * nq, owned);
      {   // coarse elements with a fine face neighbour: the readers of the half-step traces
        std::vector<std::vector<unsigned char>> pred(4);
        for (int t = 0; t < 4; ++t) pred[t].assign(m->td[t].K, 0);
        for (int64_t s2 = 0; s2 < side; ++s2) {
          if (nbr[s2] < 0) continue;
          int t, f, t2, f2;
          int64_t e, e2;
          side_elem(s2, t, e, f);
          side_elem(nbr[s2], t2, e2, f2);
          if (level[t][e] == 1 && level[t2][e2] == 2) pred[t][e] = 1;
        }
        for (int t = 0; t < 4; ++t) {
          m->mr_pred_count[t] = 0;
          for (unsigned char v : pred[t]) m->mr_pred_count[t] += v;
          m->mr_pred[t] = upload(pred[t], owned);
        }
      }
      if (d->integrator == 1) {
        // multi-rate LSRK element sets: S = fine + coarse next to fine, T = S + face neighbours of S
        std::vector<std::vector<unsigned char>> inS(4), inT(4);
        for (int t = 0; t < 4; ++t) {
          inS[t].assign(m->td[t].K, 0);
          for (int e = 0; e < m->td[t].K; ++e) inS[t][e] = level[t][e] == 2;
        }
        auto grow = [&](std::vector<std::vector<unsigned char>>& out, const std::vector<std::vector<unsigned char>>& in) {
          out = in;
          for (int64_t s2 = 0; s2 < side; ++s2) {
            if (nbr[s2] < 0) continue;
            int t, f, t2, f2;
            int64_t e, e2;
            side_elem(s2, t, e, f);
            side_elem(nbr[s2], t2, e2, f2);
            if (in[t2][e2]) out[t][e] = 1;
          }
        };
        std::vector<std::vector<unsigned char>> fineS = inS;
        grow(inS, fineS);
        grow(inT, inS);
        for (int t = 0; t < 4; ++t) {
          std::vector<int> ls, lt, ltc;
          for (int e = 0; e < m->td[t].K; ++e) {
            if (inS[t][e]) ls.push_back(e);
            if (inT[t][e]) lt.push_back(e);
            if (inT[t][e] && level[t][e] == 1) ltc.push_back(e);
          }
          m->mr_tc.count[t] = (int64_t)ltc.size();
          m->mr_tc.list[t] = upload(ltc, owned);
          m->mr_s.count[t] = (int64_t)ls.size();
          m->mr_s.list[t] = upload(ls, owned);
          m->mr_t.count[t] = (int64_t)lt.size();
          m->mr_t.list[t] = upload(lt, owned);
          m->mr_in_s[t] = upload(inS[t], owned);
        }
      }
    } else {
      m->level_count[0] = m->td[0].K + m->td[1].K + m->td[2].K + m->td[3].K;
    }

    // --- side arrays, state, traces
    m->side_nbr = upload(nbr, owned);
    m->side_code = upload(code, owned);
    m->side_tau = upload(tau, owned);
    m->q = alloc_zero<float>(4 * (size_t)m->ndof, owned);
    m->res = alloc_zero<float>(4 * (size_t)m->ndof, owned);
    m->trace = alloc_zero<float>(4 * (size_t)m->nsides * nq, owned);
    m->dacc = alloc_zero<double>(4, owned);
    m->derr = alloc_zero<int>(1, owned);
    if (!g_host_only) {   // TMA descriptors of the arrays the fused hex kernels stage
      dgk::tma_map_1d(m->tma[0], m->q, 4 * m->ndof, 128);
      dgk::tma_map_1d(m->tma[1], m->res, 4 * m->ndof, 128);
      if (m->hist) dgk::tma_map_1d(m->tma[2], m->hist, 12 * m->ndof, 128);
      dgk::tma_map_1d(m->tma[3], m->trace, 4 * m->nsides * nq, 160);
      if (m->trace3) dgk::tma_map_1d(m->tma[4], m->trace3, 2 * m->nsides * nq, 160);
    }
    if (!g_host_only && cudaDeviceSynchronize() != cudaSuccess) throw SetupError(DG_ECUDA, cudaGetErrorString(cudaGetLastError()));
    return DG_OK;
  } catch (const SetupError& e) {
    err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    err = e.what();
    return DG_EINVAL;
  }
}
