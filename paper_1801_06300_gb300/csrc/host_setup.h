// Host-side mesh, quadrature and basis preprocessing for the PCEXP library.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pcexp.h"

namespace pcexp {

// Gauss rules built by bisection + polynomial evaluation (long double).
struct Rule1D {
  std::vector<long double> x, w;  // on [0, 1]
};
Rule1D gauss_legendre_unit(int n);
// Gauss-Jacobi with weight (1 - x)^alpha on [-1, 1], mapped to [0, 1] with weight (1 - t)^alpha.
Rule1D gauss_jacobi_unit(int n, int alpha);

// Reference-triangle rule {xi, eta >= 0, xi + eta <= 1}: collapsed product
// rule (Gauss-Legendre x Gauss-Jacobi(1,0)), xi = a (1 - b), eta = b.
struct RuleTri {
  std::vector<long double> xi, eta, w;
};
RuleTri collapsed_triangle(int n);

// Reference-tetrahedron rule: collapsed product rule Gauss-Legendre x
// Gauss-Jacobi(1,0) x Gauss-Jacobi(2,0), xi = a (1-b)(1-c), eta = b (1-c), zeta = c.
struct RuleTet {
  std::vector<long double> xi, eta, zeta, w;
};
RuleTet collapsed_tetra(int n);

// Tetrahedra at p = 2 use fully symmetric rules of the collapsed rules' degree (5) with fewer
// points: Radon's 7-point rule on each face and a 14-point rule in the volume.
RuleTri radon_triangle();
// Empty on failure (the orbit parameters did not converge).
RuleTet symmetric_tetra14();

int n_basis(int dim, int p);

// Everything the device needs, built once on the host (D = dim, NF = D + 1 faces
// per element, NPERM = 2 or 6 face-vertex permutations).
struct Setup {
  int dim = 2, p = 0, nb = 0, nq = 0, nfq = 0, nv = 4;
  int64_t E = 0, F = 0, F_interior = 0;
  double volume = 0;
  // reference tables (row-major)
  std::vector<double> Bv;  // [nq][nb]              phi^_j at volume points
  std::vector<double> Dv;  // [D][nq][nb]           w_q d(phi^_j)/d xi_d
  std::vector<double> Wv;  // [nq]                  reference weights (sum 1/2 or 1/6)
  std::vector<double> Bf;  // [NF][NPERM][nfq][nb]  phi^_j at face points of local face f, vertices permuted
  std::vector<double> Wf;  // [nfq]                 face weights (sum 1 on edges, 1/2 on triangles)
  std::vector<double> Bc;  // [nb]                  phi^_j at the reference centroid
  std::vector<double> flam;  // [nfq][D]            face-rule barycentrics over a face's local vertices
  // per element
  std::vector<double> geo;     // [E][8 or 12]: A^-1 (D x D), sqrt(det A), h, 1 / sqrt(det A)
  std::vector<double> xqphys;  // [E][nq][D] physical volume points (projections, functionals)
  std::vector<int32_t> ef;     // [E][NF] face slot (face << 4) | (side << 3) | perm
  std::vector<double> Q;       // [E][nb][nb] paper <- internal
  // per face
  std::vector<int32_t> fel;   // [F][2] eL, eR (eR = -tag for boundary faces)
  std::vector<int32_t> floc;  // [F] fL | (fR << 8) | (permR << 16)
  std::vector<double> fgeo;   // [F][4] unit normal (D), measure factor
};

// Returns PCEXP_OK or an error code; msg receives a description on error.  elem_key
// (nullable, one per element) orders the elements for the choice of a face's L element (the
// lower key): a partition's submesh passes the global element indices, so that every face
// keeps the L element, and hence the quadrature points, it has in the whole mesh.
int build_setup(const pcexp_mesh& mesh, int p, Setup& s, std::string& msg, const int64_t* elem_key = nullptr);

}  // namespace pcexp
