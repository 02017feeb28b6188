// Reference-element bases, rules and face frames (host, FP64).  See refelem.h.
#include "refelem.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace dgref {

// ----------------------------------------------------------------------------- 1D
double jacobi(int n, double a, double b, double x) {
  // Three-term recurrence of the standard Jacobi polynomials, P_n(1) = C(n+a, n).
  if (n == 0) return 1.0;
  double pm = 1.0, p = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int m = 2; m <= n; ++m) {
    double c = 2.0 * m + a + b;
    double A = 2.0 * m * (m + a + b) * (c - 2.0);
    double B = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
    double C = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c;
    double pn = (B * p - C * pm) / A;
    pm = p;
    p = pn;
  }
  return p;
}

double jacobi_deriv(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1.0) * jacobi(n - 1, a + 1.0, b + 1.0, x);
}

// Gauss-Jacobi nodes by Newton iteration with deflation of the roots already
// found, weights from the classical closed form.
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double r = -std::cos((2.0 * i + 1.0) * M_PI / (2.0 * n));
    if (i > 0) r = 0.5 * (r + x[i - 1]);
    for (int it = 0; it < 100; ++it) {
      double f = jacobi(n, a, b, r), df = jacobi_deriv(n, a, b, r);
      double s = 0.0;
      for (int j = 0; j < i; ++j) s += 1.0 / (r - x[j]);
      double dr = f / (df - f * s);
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    x[i] = r;
  }
  std::sort(x.begin(), x.end());
  double lg = std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) - std::lgamma(n + a + b + 1.0) -
              std::lgamma(n + 1.0);
  double c = std::exp(lg) * std::pow(2.0, a + b + 1.0);
  for (int i = 0; i < n; ++i) {
    double d = jacobi_deriv(n, a, b, x[i]);
    w[i] = c / ((1.0 - x[i] * x[i]) * d * d);
  }
}

void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  std::vector<double> xi, wi;
  if (n > 2) gauss_jacobi(n - 2, 1, 1, xi, wi);   // interior nodes: zeros of P'_{n-1}
  x[0] = -1.0;
  x[n - 1] = 1.0;
  for (int i = 1; i + 1 < n; ++i) x[i] = xi[i - 1];
  for (int i = 0; i < n; ++i) {
    const double p = jacobi(n - 1, 0, 0, x[i]);
    w[i] = 2.0 / (n * (n - 1.0) * p * p);
  }
}

void face_rule_1d(int N, bool lobatto, std::vector<double>& x, std::vector<double>& w) {
  if (lobatto) gauss_lobatto(N + 1, x, w);
  else gauss_jacobi(N + 1, 0, 0, x, w);
}

void lagrange(const std::vector<double>& nodes, double x, double* l, double* dl) {
  int n = (int)nodes.size();
  for (int i = 0; i < n; ++i) {
    double v = 1.0, d = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double fac = 1.0 / (nodes[i] - nodes[j]);
      d = d * (x - nodes[j]) * fac + v * fac;
      v *= (x - nodes[j]) * fac;
    }
    if (l) l[i] = v;
    if (dl) dl[i] = d;
  }
}

// ----------------------------------------------------------------------------- geometry tables
static const double HEXV[8][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1},
                                  {-1, -1, 1},  {1, -1, 1},  {-1, 1, 1},  {1, 1, 1}};
static const double WEDV[6][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, -1, 1},
                                  {-1, 1, -1},  {1, 1, -1},  {-1, 1, 1}};
static const double PYRV[5][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, 1}};
static const double TETV[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};

static const int HEXF[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
static const int WEDF[5][4] = {{0, 1, 2, -1}, {3, 4, 5, -1}, {0, 1, 3, 4}, {1, 2, 4, 5}, {0, 2, 3, 5}};
static const int PYRF[5][4] = {{0, 1, 2, 3}, {0, 1, 4, -1}, {1, 3, 4, -1}, {2, 3, 4, -1}, {0, 2, 4, -1}};
static const int TETF[4][4] = {{0, 1, 2, -1}, {0, 1, 3, -1}, {1, 2, 3, -1}, {0, 2, 3, -1}};

static const double HEXO[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
static const double WEDO[5][3] = {{0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {1, 0, 1}, {-1, 0, 0}};
static const double PYRO[5][3] = {{0, 0, -1}, {0, -1, 0}, {1, 0, 1}, {0, 1, 1}, {-1, 0, 0}};
static const double TETO[4][3] = {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}};

int nverts(int t) { return t == HEX ? 8 : t == WEDGE ? 6 : t == PYR ? 5 : 4; }
int nfaces(int t) { return t == HEX ? 6 : t == TET ? 4 : 5; }
const int* face_verts(int t, int f) {
  return t == HEX ? HEXF[f] : t == WEDGE ? WEDF[f] : t == PYR ? PYRF[f] : TETF[f];
}
int face_nverts(int t, int f) { return face_verts(t, f)[3] < 0 ? 3 : 4; }
const double* vert_rst(int t, int v) {
  return t == HEX ? HEXV[v] : t == WEDGE ? WEDV[v] : t == PYR ? PYRV[v] : TETV[v];
}
const double* face_outward(int t, int f) {
  return t == HEX ? HEXO[f] : t == WEDGE ? WEDO[f] : t == PYR ? PYRO[f] : TETO[f];
}
int num_nodes(int t, int N) {
  switch (t) {
    case HEX: return (N + 1) * (N + 1) * (N + 1);
    case WEDGE: return (N + 1) * (N + 1) * (N + 2) / 2;
    case PYR: return (N + 1) * (N + 2) * (2 * N + 3) / 6;
    default: return (N + 1) * (N + 2) * (N + 3) / 6;
  }
}

void face_code_key(int nv, int code, int key[4]) {
  if (nv == 3) {
    static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int m = 0; m < 3; ++m) key[m] = P[code][m];
    key[3] = -1;
    return;
  }
  // quad corners around the face: c00 -> c10 -> c11 -> c01 (lexicographic ids 0,1,3,2)
  static const int cyc[4] = {0, 1, 3, 2};
  int p = code >> 1, dir = (code & 1) ? 3 : 1;
  key[0] = cyc[p];
  key[1] = cyc[(p + dir) % 4];
  key[2] = cyc[(p + 4 - dir) % 4];
  key[3] = cyc[(p + 2) % 4];
}

// ----------------------------------------------------------------------------- face rules
void quad_rule(int N, std::vector<double>& pts, std::vector<double>& w, bool lobatto) {
  std::vector<double> x, wx;
  face_rule_1d(N, lobatto, x, wx);
  int n = N + 1;
  pts.resize(2 * n * n);
  w.resize(n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      pts[2 * (i + n * j)] = x[i];
      pts[2 * (i + n * j) + 1] = x[j];
      w[i + n * j] = wx[i] * wx[j];
    }
}

void tri_rule(int N, std::vector<double>& pts, std::vector<double>& w) {
  // collapsed rule: GL(N+1) in a, Gauss-Jacobi(1,0)(N+1) in b; xi = (1+a)(1-b)/2 - 1, eta = b
  std::vector<double> a, wa, b, wb;
  int n = N + 1;
  gauss_jacobi(n, 0, 0, a, wa);
  gauss_jacobi(n, 1, 0, b, wb);
  pts.resize(2 * n * n);
  w.resize(n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      pts[2 * (i + n * j)] = 0.5 * (1.0 + a[i]) * (1.0 - b[j]) - 1.0;
      pts[2 * (i + n * j) + 1] = b[j];
      w[i + n * j] = 0.5 * wa[i] * wb[j];
    }
}

void face_point(int t, int f, const int key[4], double u, double v, double rst[3], double d1[3],
                double d2[3]) {
  const int* fv = face_verts(t, f);
  if (face_nverts(t, f) == 3) {
    const double* R0 = vert_rst(t, fv[key[0]]);
    const double* R1 = vert_rst(t, fv[key[1]]);
    const double* R2 = vert_rst(t, fv[key[2]]);
    double m1 = 0.5 * (1 + u), m2 = 0.5 * (1 + v), m0 = 1.0 - m1 - m2;
    for (int c = 0; c < 3; ++c) {
      rst[c] = m0 * R0[c] + m1 * R1[c] + m2 * R2[c];
      d1[c] = 0.5 * (R1[c] - R0[c]);
      d2[c] = 0.5 * (R2[c] - R0[c]);
    }
  } else {
    const double* C[4];
    for (int m = 0; m < 4; ++m) C[m] = vert_rst(t, fv[key[m]]);
    double N0 = 0.25 * (1 - u) * (1 - v), N1 = 0.25 * (1 + u) * (1 - v);
    double N2 = 0.25 * (1 - u) * (1 + v), N3 = 0.25 * (1 + u) * (1 + v);
    for (int c = 0; c < 3; ++c) {
      rst[c] = N0 * C[0][c] + N1 * C[1][c] + N2 * C[2][c] + N3 * C[3][c];
      d1[c] = 0.25 * (-(1 - v) * C[0][c] + (1 - v) * C[1][c] - (1 + v) * C[2][c] + (1 + v) * C[3][c]);
      d2[c] = 0.25 * (-(1 - u) * C[0][c] - (1 + u) * C[1][c] + (1 - u) * C[2][c] + (1 + u) * C[3][c]);
    }
  }
}

// ----------------------------------------------------------------------------- bases
// Barycentric monomials lam1^a lam2^b lam3^c (a+b+c <= N) span P_N on the tet.
static void tet_monomials(int N, const double* rst, double* v, double* g) {
  double l[3] = {0.5 * (1 + rst[0]), 0.5 * (1 + rst[1]), 0.5 * (1 + rst[2])};
  int m = 0;
  for (int a = 0; a <= N; ++a)
    for (int b = 0; a + b <= N; ++b)
      for (int c = 0; a + b + c <= N; ++c) {
        double pa = std::pow(l[0], a), pb = std::pow(l[1], b), pc = std::pow(l[2], c);
        v[m] = pa * pb * pc;
        ++m;
      }
  if (g) {
    int Np = m;
    m = 0;
    for (int a = 0; a <= N; ++a)
      for (int b = 0; a + b <= N; ++b)
        for (int c = 0; a + b + c <= N; ++c) {
          double pa = std::pow(l[0], a), pb = std::pow(l[1], b), pc = std::pow(l[2], c);
          g[m] = a ? 0.5 * a * std::pow(l[0], a - 1) * pb * pc : 0.0;
          g[Np + m] = b ? 0.5 * b * pa * std::pow(l[1], b - 1) * pc : 0.0;
          g[2 * Np + m] = c ? 0.5 * c * pa * pb * std::pow(l[2], c - 1) : 0.0;
          ++m;
        }
  }
}

static void invert(std::vector<double>& A, int n) {
  // Gauss-Jordan elimination with partial pivoting, in place.
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (std::fabs(A[p * n + c]) < 1e-300) throw std::runtime_error("singular matrix");
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[p * n + k], A[c * n + k]);
        std::swap(I[p * n + k], I[c * n + k]);
      }
    double d = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] *= d;
      I[c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        I[r * n + k] -= f * I[c * n + k];
      }
    }
  }
  A.swap(I);
}

void Basis::init(int type_, int N_, bool lobatto) {
  type = type_;
  N = N_;
  Np = num_nodes(type, N);
  if (type == HEX) {
    face_rule_1d(N, lobatto, r1, w1);
    int n = N + 1;
    nodes.resize(3 * Np);
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = i + n * (j + n * k);
          nodes[3 * id] = r1[i];
          nodes[3 * id + 1] = r1[j];
          nodes[3 * id + 2] = r1[k];
        }
  } else if (type == TET) {
    nodes.clear();
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j + k <= N; ++j)
        for (int i = 0; i + j + k <= N; ++i) {
          nodes.push_back(-1.0 + 2.0 * i / N);
          nodes.push_back(-1.0 + 2.0 * j / N);
          nodes.push_back(-1.0 + 2.0 * k / N);
        }
    Vinv.assign(Np * Np, 0.0);
    std::vector<double> row(Np);
    for (int n = 0; n < Np; ++n) {
      tet_monomials(N, &nodes[3 * n], row.data(), nullptr);
      for (int m = 0; m < Np; ++m) Vinv[n * Np + m] = row[m];
    }
    invert(Vinv, Np);
  } else if (type == WEDGE) {
    mi.clear(); mj.clear(); mk.clear();
    for (int j = 0; j <= N; ++j)
      for (int i = 0; i <= N; ++i)
        for (int k = 0; i + k <= N; ++k) {
          mi.push_back(i); mj.push_back(j); mk.push_back(k);
        }
  } else {  // PYR
    lev_x.resize(N + 1);
    lev_w.resize(N + 1);
    for (int k = 0; k <= N; ++k) gauss_jacobi(k + 1, 0, 0, lev_x[k], lev_w[k]);
    mi.clear(); mj.clear(); mk.clear();
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= k; ++j)
        for (int i = 0; i <= k; ++i) {
          mi.push_back(i); mj.push_back(j); mk.push_back(k);
        }
    gam.resize(N + 1);
    for (int k = 0; k <= N; ++k) gam[k] = 2.0 / (2.0 * k + 3.0);  // int h^{2k+2} (P^{(2k+3,0)}_{N-k})^2
  }
}

// h^n P_n(x/h) and its partial derivatives by the homogenised Legendre recurrence
// (n+1) Q_{n+1} = (2n+1) x Q_n - n h^2 Q_{n-1}; regular at h = 0.
static void scaled_legendre(int n, double x, double h, double& Q, double& Qx, double& Qh) {
  double q0 = 1, q0x = 0, q0h = 0;
  if (n == 0) { Q = 1; Qx = 0; Qh = 0; return; }
  double q1 = x, q1x = 1, q1h = 0;
  for (int m = 1; m < n; ++m) {
    double q2 = ((2 * m + 1) * x * q1 - m * h * h * q0) / (m + 1);
    double q2x = ((2 * m + 1) * (q1 + x * q1x) - m * h * h * q0x) / (m + 1);
    double q2h = ((2 * m + 1) * x * q1h - m * (2 * h * q0 + h * h * q0h)) / (m + 1);
    q0 = q1; q0x = q1x; q0h = q1h;
    q1 = q2; q1x = q2x; q1h = q2h;
  }
  Q = q1; Qx = q1x; Qh = q1h;
}

void Basis::eval(const double* rst, double* phi, double* g) const {
  if (type == HEX) {
    int n = N + 1;
    std::vector<double> L(3 * n), dL(3 * n);
    for (int a = 0; a < 3; ++a) lagrange(r1, rst[a], &L[a * n], &dL[a * n]);
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = i + n * (j + n * k);
          phi[id] = L[i] * L[n + j] * L[2 * n + k];
          if (g) {
            g[id] = dL[i] * L[n + j] * L[2 * n + k];
            g[Np + id] = L[i] * dL[n + j] * L[2 * n + k];
            g[2 * Np + id] = L[i] * L[n + j] * dL[2 * n + k];
          }
        }
  } else if (type == TET) {
    std::vector<double> v(Np), gv(3 * Np);
    tet_monomials(N, rst, v.data(), g ? gv.data() : nullptr);
    for (int m = 0; m < Np; ++m) {
      double s = 0, s0 = 0, s1 = 0, s2 = 0;
      for (int j = 0; j < Np; ++j) {
        double c = Vinv[j * Np + m];
        s += v[j] * c;
        if (g) { s0 += gv[j] * c; s1 += gv[Np + j] * c; s2 += gv[2 * Np + j] * c; }
      }
      phi[m] = s;
      if (g) { g[m] = s0; g[Np + m] = s1; g[2 * Np + m] = s2; }
    }
  } else if (type == WEDGE) {
    // phi_ijk = h^i P_i(a) P_j(s) P_k^{(2i+1,0)}(t) / sqrt(4/((2i+1)(2j+1)(i+k+1))),
    // h = (1-t)/2, h*a = (1+r) - h.
    double r = rst[0], s = rst[1], t = rst[2];
    double h = 0.5 * (1 - t), x = (1 + r) - h;
    for (int m = 0; m < Np; ++m) {
      int i = mi[m], j = mj[m], k = mk[m];
      double Q, Qx, Qh;
      scaled_legendre(i, x, h, Q, Qx, Qh);
      double Pj = jacobi(j, 0, 0, s), dPj = jacobi_deriv(j, 0, 0, s);
      double Pk = jacobi(k, 2 * i + 1, 0, t), dPk = jacobi_deriv(k, 2 * i + 1, 0, t);
      double nrm = std::sqrt((2.0 * i + 1) * (2.0 * j + 1) * (i + k + 1) / 4.0);
      phi[m] = nrm * Q * Pj * Pk;
      if (g) {
        g[m] = nrm * Qx * Pj * Pk;
        g[Np + m] = nrm * Q * dPj * Pk;
        g[2 * Np + m] = nrm * ((0.5 * Qx - 0.5 * Qh) * Pj * Pk + Q * Pj * dPk);
      }
    }
  } else {  // PYR: l^k_i(a) l^k_j(b) h^k P^{(2k+3,0)}_{N-k}(c) / sqrt(w_i w_j gamma_k)
    // At the apex (h = 0) a and b are undefined but bounded inside the pyramid and every
    // level k >= 1 carries h^k -> 0; any bounded (a,b) gives the limit (values only).
    double t = rst[2], h = 0.5 * (1 - t);
    double a = h > 1e-14 ? (1 + rst[0]) / h - 1 : 0.0, b = h > 1e-14 ? (1 + rst[1]) / h - 1 : 0.0;
    std::vector<double> la(N + 1), dla(N + 1), lb(N + 1), dlb(N + 1);
    int kprev = -1;
    for (int m = 0; m < Np; ++m) {
      int i = mi[m], j = mj[m], k = mk[m];
      if (k != kprev) {
        lagrange(lev_x[k], a, la.data(), dla.data());
        lagrange(lev_x[k], b, lb.data(), dlb.data());
        kprev = k;
      }
      double P = jacobi(N - k, 2 * k + 3, 0, t), dP = jacobi_deriv(N - k, 2 * k + 3, 0, t);
      double nrm = 1.0 / std::sqrt(lev_w[k][i] * lev_w[k][j] * gam[k]);
      double hk = std::pow(h, k), hk1 = k > 0 ? std::pow(h, k - 1) : 0.0;
      phi[m] = nrm * la[i] * lb[j] * hk * P;
      if (g) {
        double gr = dla[i] * lb[j] * hk1 * P;                // d/dr = (1/h) d/da
        double gs = la[i] * dlb[j] * hk1 * P;
        double gc = la[i] * lb[j] * (hk * dP - 0.5 * k * hk1 * P);
        g[m] = nrm * gr;
        g[Np + m] = nrm * gs;
        g[2 * Np + m] = nrm * (0.5 * (1 + a) * gr + 0.5 * (1 + b) * gs + gc);
      }
    }
  }
}

}  // namespace dgref
