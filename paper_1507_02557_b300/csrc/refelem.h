// Reference-element data for the hybrid DG method, built on the host in FP64.
//
// Bases (Sec. 2.1 of arxiv 1507.02557):
//   hex      nodal Lagrange at tensor Gauss-Legendre nodes, or Gauss-Lobatto (SEM) (Sec. 2.1.1)
//   tet      nodal Lagrange at the equispaced lattice of the bi-unit tet (Sec. 2.1.2)
//   wedge    orthonormal modal basis, LSC-DG numerator (Sec. 2.1.3)
//   pyramid  semi-nodal orthogonal basis of the rational space B_N (Sec. 2.1.4)
// Face rules: tensor GL (or GLL with SEM hexahedra) (N+1)^2 on quadrilaterals; collapsed GL x Gauss-Jacobi(1,0)
// with (N+1)^2 points on triangles, given in a canonical face frame (see setup.cpp).
#pragma once
#include <vector>

namespace dgref {

enum { HEX = 0, WEDGE = 1, PYR = 2, TET = 3 };

// 1D rules and polynomials -------------------------------------------------
double jacobi(int n, double a, double b, double x);
double jacobi_deriv(int n, double a, double b, double x);
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
// n-point Gauss-Lobatto-Legendre rule: +-1 and the zeros of P'_{n-1}, w = 2 / (n (n-1) P_{n-1}(x)^2)
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w);
// the (N+1)-point quadrilateral-face rule in 1D: GL, or GLL with SEM hexahedra
void face_rule_1d(int N, bool lobatto, std::vector<double>& x, std::vector<double>& w);
void lagrange(const std::vector<double>& nodes, double x, double* l, double* dl);

// Reference element geometry --------------------------------------------------
int nverts(int type);
int nfaces(int type);
int face_nverts(int type, int f);
const int* face_verts(int type, int f);          // local vertex ids (tri c0,c1,c2; quad lexicographic)
const double* vert_rst(int type, int v);         // reference coordinates of local vertex v
const double* face_outward(int type, int f);     // reference gradient of an outward face function
int num_nodes(int type, int N);

// Canonical face codes: triangles 0..5 (permutations), quads 0..7 (dihedral keys).
// key[m] = local corner index of canonical corner m.
void face_code_key(int nv, int code, int key[4]);

// Basis evaluation at one reference point: values phi[Np], gradients g[3*Np] (d/dr, d/ds, d/dt).
// For the wedge this is the LSC numerator; for the pyramid the semi-nodal basis.
struct Basis {
  int type, N, Np;
  // hex / GL data
  std::vector<double> r1, w1;                    // 1D GL nodes and weights
  // tet data
  std::vector<double> nodes;                     // [Np*3] nodal points (hex, tet)
  std::vector<double> Vinv;                      // tet: inverse Vandermonde of the PKD basis [Np*Np]
  // pyramid data
  std::vector<std::vector<double>> lev_x, lev_w; // GL nodes/weights of each level k (k+1 points)
  std::vector<int> mi, mj, mk;                   // mode indices
  std::vector<double> gam;                       // pyramid c-normalisation per level
  void init(int type, int N, bool lobatto = false);   // lobatto: SEM hexahedron (GLL nodes)
  void eval(const double* rst, double* phi, double* g) const;
};

// Face cubature in canonical coordinates: pts[nq*2], w[nq] (tri: (xi,eta); quad: (alpha,beta)).
void tri_rule(int N, std::vector<double>& pts, std::vector<double>& w);
void quad_rule(int N, std::vector<double>& pts, std::vector<double>& w, bool lobatto = false);
// Reference point (rst) and tangents of canonical face point (u,v) for (type, face, key).
void face_point(int type, int f, const int key[4], double u, double v, double rst[3],
                double d1[3], double d2[3]);

}  // namespace dgref
