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

int n_basis_2d(int p);

// Everything the device needs, built once on the host.
struct Setup {
  int dim = 2, p = 0, nb = 0, nq = 0, nfq = 0, nv = 4;
  int64_t E = 0, F = 0, F_interior = 0;
  double volume = 0;
  // reference tables (row-major)
  std::vector<double> Bv;  // [nq][nb]      phi^_j at volume points
  std::vector<double> Dv;  // [2][nq][nb]   w_q d(phi^_j)/d xi_d
  std::vector<double> Wv;  // [nq]          reference weights (sum 1/2)
  std::vector<double> Bf;  // [3][nfq][nb]  phi^_j at face points of local face f (L order)
  std::vector<double> Wf;  // [nfq]         edge weights on [0, 1]
  std::vector<double> Bc;  // [nb]          phi^_j at the reference centroid
  // per element
  std::vector<double> geo;     // [E][8]: Ainv00 Ainv01 Ainv10 Ainv11 sdet h 0 0
  std::vector<double> xqphys;  // [E][nq][2] physical volume points (host projections)
  std::vector<int32_t> ef;     // [E][3]  face*2 + side of local face f
  std::vector<double> Q;       // [E][nb][nb] paper <- internal
  // per face
  std::vector<int32_t> fel;   // [F][2] eL, eR (eR = -tag for boundary faces)
  std::vector<int32_t> floc;  // [F] fL | (fR << 8)
  std::vector<double> fgeo;   // [F][4] nx ny len 0
};

// Returns PCEXP_OK or an error code; msg receives a description on error.
int build_setup(const pcexp_mesh& mesh, int p, Setup& s, std::string& msg);

}  // namespace pcexp
