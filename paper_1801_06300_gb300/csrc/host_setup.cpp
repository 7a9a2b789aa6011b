// Host preprocessing: quadrature, reference basis, paper-basis transform,
// element geometry and the face list (Sec. 4.2-4.3 of the paper), for
// triangles (dim 2) and tetrahedra (dim 3).
//
// Quadrature (the paper does not fix it): p+1 Gauss points per direction.
// Edges: Gauss-Legendre.  Triangles (elements in 2D, faces in 3D): collapsed
// product rule Gauss-Legendre x Gauss-Jacobi(1,0), xi = a (1 - b), eta = b.
// Tetrahedra: Gauss-Legendre x Gauss-Jacobi(1,0) x Gauss-Jacobi(2,0),
// xi = a (1-b)(1-c), eta = b (1-c), zeta = c.  A simplex (v0, ..., vD) maps
// x = v0 + sum_k xi_k (v_k - v0).  Nodes are found here by bisection on sign
// changes of the three-term recurrence, weights from the closed Christoffel
// form.  Tetrahedra at p = 2 instead take fully symmetric rules of the same
// degree (5): 14 volume points (instead of 27) and Radon's 7 face points
// (instead of 9).
//
// Faces: local face f of an element is the face opposite vertex f, with
// vertices f+1, ..., f+D (mod D+1).  A face's points are the face rule on its
// L element (the lower element index) in that vertex order; the R element sees
// the same points through the permutation of its local face vertices that
// matches the L element's (on periodic master vertices).
#include "host_setup.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <unordered_map>

namespace pcexp {

namespace {

// P_n^{(a,b)}(x) by the three-term recurrence.
long double jacobi_p(int n, long double a, long double b, long double x) {
  if (n == 0) return 1.0L;
  long double p0 = 1.0L;
  long double p1 = (a + 1.0L) + (a + b + 2.0L) * (x - 1.0L) / 2.0L;
  for (int k = 2; k <= n; ++k) {
    long double c = 2.0L * k + a + b;
    long double a1 = 2.0L * k * (k + a + b) * (c - 2.0L);
    long double a2 = (c - 1.0L) * (c * (c - 2.0L) * x + a * a - b * b);
    long double a3 = 2.0L * (k + a - 1.0L) * (k + b - 1.0L) * c;
    long double p2 = (a2 * p1 - a3 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Gauss-Jacobi nodes/weights on [-1, 1] for (1 - x)^a (1 + x)^b.
void gauss_jacobi(int n, long double a, long double b, std::vector<long double>& x,
                  std::vector<long double>& w) {
  x.clear();
  w.clear();
  const int M = 20000;
  long double prev_x = -1.0L, prev_f = jacobi_p(n, a, b, -1.0L);
  for (int i = 1; i <= M; ++i) {
    long double xi = -std::cos(3.14159265358979323846264338327950288L * i / M);
    long double fi = jacobi_p(n, a, b, xi);
    if ((prev_f < 0) != (fi < 0) || fi == 0) {
      long double lo = prev_x, hi = xi, flo = prev_f;
      for (int it = 0; it < 200 && hi - lo > 0; ++it) {
        long double mid = 0.5L * (lo + hi);
        if (mid == lo || mid == hi) break;
        long double fm = jacobi_p(n, a, b, mid);
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      x.push_back(0.5L * (lo + hi));
    }
    prev_x = xi;
    prev_f = fi;
  }
  // Christoffel weights: Gamma(n+a+1) Gamma(n+b+1) / (Gamma(n+a+b+1) n!) 2^{a+b+1}
  //                      / ((1 - x^2) P_n'(x)^2), P_n' = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}.
  long double c = std::exp(std::lgamma((double)(n + a + 1)) + std::lgamma((double)(n + b + 1)) -
                           std::lgamma((double)(n + a + b + 1)) - std::lgamma((double)(n + 1))) *
                  std::pow(2.0L, a + b + 1.0L);
  for (long double xi : x) {
    long double dp = 0.5L * (n + a + b + 1.0L) * jacobi_p(n - 1, a + 1.0L, b + 1.0L, xi);
    w.push_back(c / ((1.0L - xi * xi) * dp * dp));
  }
}

struct Mono {
  int e[3];
};

// graded order: by total degree, then descending x-power, then descending y-power
std::vector<Mono> graded_exponents(int dim, int p) {
  std::vector<Mono> out;
  for (int deg = 0; deg <= p; ++deg)
    for (int px = deg; px >= 0; --px) {
      if (dim == 2) {
        out.push_back({{px, deg - px, 0}});
      } else {
        for (int py = deg - px; py >= 0; --py) out.push_back({{px, py, deg - px - py}});
      }
    }
  return out;
}

template <class R> R ipow(R x, int k) {
  R r = 1;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

// monomial k and its derivative along d at a point x (dim coordinates)
template <class R> R mono_val(const Mono& m, const R* x, int dim) {
  R r = 1;
  for (int d = 0; d < dim; ++d) r *= ipow(x[d], m.e[d]);
  return r;
}
template <class R> R mono_der(const Mono& m, int dd, const R* x, int dim) {
  if (m.e[dd] == 0) return R(0);
  R r = R(m.e[dd]) * ipow(x[dd], m.e[dd] - 1);
  for (int d = 0; d < dim; ++d)
    if (d != dd) r *= ipow(x[d], m.e[d]);
  return r;
}

struct Key {
  int64_t a, b, c;
  bool operator==(const Key& o) const { return a == o.a && b == o.b && c == o.c; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)k.a * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k.b + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)k.c + 0x85157AF5ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};
Key sorted_key(int64_t* v, int n) {
  std::sort(v, v + n);
  return Key{v[0], v[1], n > 2 ? v[2] : -1};
}

}  // namespace

Rule1D gauss_legendre_unit(int n) {
  std::vector<long double> x, w;
  gauss_jacobi(n, 0.0L, 0.0L, x, w);
  // exact symmetry: x_{n-1-i} = -x_i
  for (int i = 0; i < n / 2; ++i) {
    long double xs = 0.5L * (x[n - 1 - i] - x[i]);
    long double ws = 0.5L * (w[i] + w[n - 1 - i]);
    x[i] = -xs;
    x[n - 1 - i] = xs;
    w[i] = w[n - 1 - i] = ws;
  }
  if (n % 2) x[n / 2] = 0.0L;
  Rule1D r;
  for (int i = 0; i < n; ++i) {
    r.x.push_back(0.5L * (x[i] + 1.0L));
    r.w.push_back(0.5L * w[i]);
  }
  return r;
}

Rule1D gauss_jacobi_unit(int n, int alpha) {
  std::vector<long double> x, w;
  gauss_jacobi(n, (long double)alpha, 0.0L, x, w);
  Rule1D r;
  long double sc = std::pow(2.0L, (long double)(alpha + 1));
  for (int i = 0; i < n; ++i) {
    r.x.push_back(0.5L * (x[i] + 1.0L));
    r.w.push_back(w[i] / sc);
  }
  return r;
}

RuleTri collapsed_triangle(int n) {
  Rule1D a = gauss_legendre_unit(n), b = gauss_jacobi_unit(n, 1);
  RuleTri t;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      t.xi.push_back(a.x[i] * (1.0L - b.x[j]));
      t.eta.push_back(b.x[j]);
      t.w.push_back(a.w[i] * b.w[j]);
    }
  return t;
}

int n_basis(int dim, int p) { return dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6; }

RuleTet collapsed_tetra(int n) {
  Rule1D a = gauss_legendre_unit(n), b = gauss_jacobi_unit(n, 1), c = gauss_jacobi_unit(n, 2);
  RuleTet t;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        t.xi.push_back(a.x[i] * (1.0L - b.x[j]) * (1.0L - c.x[k]));
        t.eta.push_back(b.x[j] * (1.0L - c.x[k]));
        t.zeta.push_back(c.x[k]);
        t.w.push_back(a.w[i] * b.w[j] * c.w[k]);
      }
  return t;
}

// Radon's rule of degree 5 on the reference triangle (area 1/2), in closed form: the centroid
// with weight 9/40 of the area, and the two orbits (a, a, 1 - 2a) of the barycentric
// coordinates, a = (6 -+ sqrt 15)/21, with weights (155 -+ sqrt 15)/1200 of the area.
RuleTri radon_triangle() {
  RuleTri t;
  auto add = [&](long double l1, long double l2, long double w) {
    t.xi.push_back(l1);
    t.eta.push_back(l2);
    t.w.push_back(w);
  };
  add(1.0L / 3.0L, 1.0L / 3.0L, 9.0L / 80.0L);
  const long double r = std::sqrt(15.0L);
  for (int s = -1; s <= 1; s += 2) {
    const long double a = (6.0L + s * r) / 21.0L, w = (155.0L + s * r) / 2400.0L;
    add(a, a, w);
    add(a, 1.0L - 2.0L * a, w);
    add(1.0L - 2.0L * a, a, w);
  }
  return t;
}

// Fully symmetric 14-point rule of degree 5 on the reference tetrahedron (volume 1/6): two
// orbits of four points, barycentric coordinates (a, a, a, 1 - 3a), and one orbit of six,
// (b, b, 1/2 - b, 1/2 - b), each orbit with one weight.  The six parameters
// x = (a1, w1, a2, w2, b, w3) make every monomial xi^i eta^j zeta^k of degree <= 5 integrate to
// i! j! k! / (i + j + k + 3)!: 56 consistent equations, solved by Gauss-Newton (normal
// equations, Gaussian elimination) in long double from a rough starting point.
RuleTet symmetric_tetra14() {
  // each point: coordinates c0 + x[par] * dir (reference coordinates xi, eta, zeta), weight x[wi]
  struct Pt {
    int par, wi;
    long double c0[3], dir[3];
  };
  std::vector<Pt> pts;
  for (int o = 0; o < 2; ++o) {  // (a, a, a, 1 - 3a): lam_0 = 1 - 3a, or one of lam_1..3 is
    pts.push_back({2 * o, 2 * o + 1, {0, 0, 0}, {1, 1, 1}});
    for (int k = 0; k < 3; ++k) {
      Pt q{2 * o, 2 * o + 1, {0, 0, 0}, {1, 1, 1}};
      q.c0[k] = 1.0L;
      q.dir[k] = -3.0L;
      pts.push_back(q);
    }
  }
  // (b, b, 1/2 - b, 1/2 - b): of lam_1..3, the ones equal to b are those of the pair holding b
  // that lie among them (lam_0 = b for the pairs {0, k}, lam_0 = 1/2 - b otherwise)
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) {
      Pt q{4, 5, {0.5L, 0.5L, 0.5L}, {-1, -1, -1}};
      for (int k = 1; k <= 3; ++k)
        if (k == i || k == j) {
          q.c0[k - 1] = 0.0L;
          q.dir[k - 1] = 1.0L;
        }
      pts.push_back(q);
    }
  std::vector<std::array<int, 3>> mono;
  for (int i = 0; i <= 5; ++i)
    for (int j = 0; i + j <= 5; ++j)
      for (int k = 0; i + j + k <= 5; ++k) mono.push_back({i, j, k});
  auto fact = [](int n) {
    long double f = 1.0L;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
  };
  auto ipow = [](long double v, int e) {
    long double r = 1.0L;
    for (int i = 0; i < e; ++i) r *= v;
    return r;
  };
  long double x[6] = {0.1L, 0.01L, 0.3L, 0.02L, 0.05L, 0.007L};
  const int M = (int)mono.size();
  long double rlast = 1.0L;
  for (int it = 0; it < 100; ++it) {
    long double JtJ[6][7] = {};
    long double rmax = 0.0L;
    for (int m = 0; m < M; ++m) {
      const int* e = mono[m].data();
      long double r = -fact(e[0]) * fact(e[1]) * fact(e[2]) / fact(e[0] + e[1] + e[2] + 3);
      long double J[6] = {};
      for (const Pt& q : pts) {
        long double c[3], f = 1.0L, df = 0.0L;
        for (int d = 0; d < 3; ++d) c[d] = q.c0[d] + x[q.par] * q.dir[d];
        for (int d = 0; d < 3; ++d) f *= ipow(c[d], e[d]);
        for (int d = 0; d < 3; ++d) {
          if (e[d] == 0 || q.dir[d] == 0.0L) continue;
          long double g = e[d] * ipow(c[d], e[d] - 1) * q.dir[d];
          for (int d2 = 0; d2 < 3; ++d2)
            if (d2 != d) g *= ipow(c[d2], e[d2]);
          df += g;
        }
        r += x[q.wi] * f;
        J[q.wi] += f;
        J[q.par] += x[q.wi] * df;
      }
      rmax = std::max(rmax, std::fabs(r));
      for (int a = 0; a < 6; ++a) {
        for (int b = 0; b < 6; ++b) JtJ[a][b] += J[a] * J[b];
        JtJ[a][6] -= J[a] * r;
      }
    }
    rlast = rmax;
    if (rmax < 1e-18L) break;
    // Gaussian elimination with partial pivoting on [JtJ | -Jt r]
    for (int c = 0; c < 6; ++c) {
      int piv = c;
      for (int rr = c + 1; rr < 6; ++rr)
        if (std::fabs(JtJ[rr][c]) > std::fabs(JtJ[piv][c])) piv = rr;
      if (JtJ[piv][c] == 0.0L) return RuleTet{};
      for (int k = 0; k < 7; ++k) std::swap(JtJ[c][k], JtJ[piv][k]);
      for (int rr = c + 1; rr < 6; ++rr) {
        const long double f = JtJ[rr][c] / JtJ[c][c];
        for (int k = c; k < 7; ++k) JtJ[rr][k] -= f * JtJ[c][k];
      }
    }
    long double dx[6];
    for (int c = 5; c >= 0; --c) {
      long double s = JtJ[c][6];
      for (int k = c + 1; k < 6; ++k) s -= JtJ[c][k] * dx[k];
      dx[c] = s / JtJ[c][c];
    }
    long double step = 0.0L;
    for (int a = 0; a < 6; ++a) {
      x[a] += dx[a];
      step = std::max(step, std::fabs(dx[a]));
    }
    if (step < 1e-19L) break;
  }
  RuleTet t;
  if (!(rlast < 1e-15L)) return t;
  for (const Pt& q : pts) {
    t.xi.push_back(q.c0[0] + x[q.par] * q.dir[0]);
    t.eta.push_back(q.c0[1] + x[q.par] * q.dir[1]);
    t.zeta.push_back(q.c0[2] + x[q.par] * q.dir[2]);
    t.w.push_back(x[q.wi]);
  }
  return t;
}

int build_setup(const pcexp_mesh& mesh, int p, Setup& s, std::string& msg, const int64_t* elem_key) {
  const int D = mesh.dim;
  if (D != 2 && D != 3) {
    msg = "mesh dimension must be 2 (triangles) or 3 (tetrahedra)";
    return PCEXP_ERR_UNSUPPORTED;
  }
  if (p < 0 || p > 3) {
    msg = "order p must be 0..3";
    return PCEXP_ERR_INVALID_ARG;
  }
  if (D == 3 && p > 2) {
    msg = "tetrahedra are supported up to p = 2";
    return PCEXP_ERR_UNSUPPORTED;
  }
  if (mesh.n_elem <= 0 || mesh.n_vert <= 0 || !mesh.coords || !mesh.elem_vert) {
    msg = "empty mesh";
    return PCEXP_ERR_INVALID_ARG;
  }
  const int NF = D + 1, NPERM = D == 2 ? 2 : 6, GEO = D == 2 ? 8 : 12;
  const int n1 = p + 1, nb = n_basis(D, p);
  s.dim = D;
  s.nv = D + 2;
  s.p = p;
  s.nb = nb;
  const bool sym = D == 3 && p == 2;  // symmetric rules (14 volume, 7 face points)
  s.nq = D == 2 ? n1 * n1 : sym ? 14 : n1 * n1 * n1;
  s.nfq = D == 2 ? n1 : sym ? 7 : n1 * n1;
  s.E = mesh.n_elem;
  const int64_t E = s.E;
  const int nq = s.nq, nfq = s.nfq;

  // ---- reference rules (long double, once)
  std::vector<std::array<long double, 3>> xr(nq);
  std::vector<long double> wr(nq);
  if (D == 2) {
    RuleTri tri = collapsed_triangle(n1);
    for (int q = 0; q < nq; ++q) {
      xr[q] = {tri.xi[q], tri.eta[q], 0.0L};
      wr[q] = tri.w[q];
    }
  } else {
    RuleTet tet = sym ? symmetric_tetra14() : collapsed_tetra(n1);
    if ((int)tet.w.size() != nq) {
      msg = "volume quadrature rule construction failed";
      return PCEXP_ERR_INVALID_ARG;
    }
    for (int q = 0; q < nq; ++q) {
      xr[q] = {tet.xi[q], tet.eta[q], tet.zeta[q]};
      wr[q] = tet.w[q];
    }
  }
  // face rule as barycentrics over the face's D vertices, weights summing to 1 (2D) or 1/2 (3D)
  std::vector<std::array<long double, 3>> lam(nfq);
  std::vector<long double> wf(nfq);
  if (D == 2) {
    Rule1D edge = gauss_legendre_unit(n1);
    for (int q = 0; q < nfq; ++q) {
      lam[q] = {1.0L - edge.x[q], edge.x[q], 0.0L};
      wf[q] = edge.w[q];
    }
  } else {
    RuleTri tri = sym ? radon_triangle() : collapsed_triangle(n1);
    for (int q = 0; q < nfq; ++q) {
      lam[q] = {1.0L - tri.xi[q] - tri.eta[q], tri.xi[q], tri.eta[q]};
      wf[q] = tri.w[q];
    }
  }
  s.flam.assign((size_t)nfq * D, 0.0);
  for (int q = 0; q < nfq; ++q)
    for (int k = 0; k < D; ++k) s.flam[(size_t)q * D + k] = (double)lam[q][k];

  // ---- reference orthonormal basis: MGS of monomials about the reference centroid
  const std::vector<Mono> ex = graded_exponents(D, p);
  const long double cen = 1.0L / (D + 1);
  std::vector<long double> Cr(nb * nb, 0.0L);  // phi^_i = sum_k Cr[i][k] mono_k(xi - cen)
  {
    std::vector<long double> vals(nb * nq), psi(nb * nq);
    for (int k = 0; k < nb; ++k)
      for (int q = 0; q < nq; ++q) {
        long double y[3] = {xr[q][0] - cen, xr[q][1] - cen, xr[q][2] - cen};
        vals[k * nq + q] = mono_val(ex[k], y, D);
      }
    for (int i = 0; i < nb; ++i) {
      std::vector<long double> c(nb, 0.0L), v(vals.begin() + i * nq, vals.begin() + (i + 1) * nq);
      c[i] = 1.0L;
      for (int j = 0; j < i; ++j) {
        long double d = 0;
        for (int q = 0; q < nq; ++q) d += wr[q] * v[q] * psi[j * nq + q];
        for (int q = 0; q < nq; ++q) v[q] -= d * psi[j * nq + q];
        for (int k = 0; k < nb; ++k) c[k] -= d * Cr[j * nb + k];
      }
      long double nr = 0;
      for (int q = 0; q < nq; ++q) nr += wr[q] * v[q] * v[q];
      nr = std::sqrt(nr);
      for (int q = 0; q < nq; ++q) psi[i * nq + q] = v[q] / nr;
      for (int k = 0; k < nb; ++k) Cr[i * nb + k] = c[k] / nr;
    }
  }
  auto phi = [&](int i, const long double* x) {
    long double y[3] = {x[0] - cen, x[1] - cen, D == 3 ? x[2] - cen : 0.0L};
    long double r = 0;
    for (int k = 0; k <= i; ++k) r += Cr[i * nb + k] * mono_val(ex[k], y, D);
    return r;
  };
  auto dphi = [&](int i, int d, const long double* x) {
    long double y[3] = {x[0] - cen, x[1] - cen, D == 3 ? x[2] - cen : 0.0L};
    long double r = 0;
    for (int k = 0; k <= i; ++k) r += Cr[i * nb + k] * mono_der(ex[k], d, y, D);
    return r;
  };
  s.Bv.assign(nq * nb, 0);
  s.Dv.assign(D * nq * nb, 0);
  s.Wv.assign(nq, 0);
  for (int q = 0; q < nq; ++q) {
    s.Wv[q] = (double)wr[q];
    for (int j = 0; j < nb; ++j) {
      s.Bv[q * nb + j] = (double)phi(j, xr[q].data());
      for (int d = 0; d < D; ++d) s.Dv[(d * nq + q) * nb + j] = (double)(wr[q] * dphi(j, d, xr[q].data()));
    }
  }
  // reference vertices, local face vertices and face-vertex permutations
  long double VR[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  auto fv = [&](int f, int k) { return (f + 1 + k) % (D + 1); };
  static const int PERM2[2][3] = {{0, 1, 2}, {1, 0, 2}};
  static const int PERM3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  auto perm = [&](int pi, int k) { return D == 2 ? PERM2[pi][k] : PERM3[pi][k]; };
  s.Bf.assign((size_t)NF * NPERM * nfq * nb, 0);
  s.Wf.assign(nfq, 0);
  for (int q = 0; q < nfq; ++q) s.Wf[q] = (double)wf[q];
  for (int f = 0; f < NF; ++f)
    for (int pi = 0; pi < NPERM; ++pi)
      for (int q = 0; q < nfq; ++q) {
        long double x[3] = {0, 0, 0};
        for (int k = 0; k < D; ++k)
          for (int d = 0; d < 3; ++d) x[d] += lam[q][k] * VR[fv(f, perm(pi, k))][d];
        for (int j = 0; j < nb; ++j) s.Bf[(((size_t)f * NPERM + pi) * nfq + q) * nb + j] = (double)phi(j, x);
      }
  s.Bc.assign(nb, 0);
  {
    long double x[3] = {cen, cen, D == 3 ? cen : 0.0L};
    for (int j = 0; j < nb; ++j) s.Bc[j] = (double)phi(j, x);
  }

  // ---- element geometry and the paper-basis transform Q_e (Eq. basis, Algorithm 1).
  // Per element in double on offsets from v0 (edge vectors are exact), so the
  // centroid-scaled monomials keep full relative precision far from the origin.
  const double* X = mesh.coords;
  const int32_t* EV = mesh.elem_vert;
  s.geo.assign((size_t)E * GEO, 0.0);
  s.xqphys.assign((size_t)E * nq * D, 0.0);
  s.Q.assign((size_t)E * nb * nb, 0.0);
  s.volume = 0;
  const double fact = D == 2 ? 2.0 : 6.0;
  std::vector<double> rq(nq * 3), pw(nq), psi(nb * nq), vv(nq);
  for (int64_t e = 0; e < E; ++e) {
    int32_t v[4];
    for (int k = 0; k <= D; ++k) {
      v[k] = EV[(D + 1) * e + k];
      if (v[k] < 0 || v[k] >= mesh.n_vert) {
        msg = "element vertex out of range";
        return PCEXP_ERR_MESH;
      }
    }
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // columns: v_k - v0
    for (int k = 0; k < D; ++k)
      for (int d = 0; d < D; ++d) A[d][k] = X[D * v[k + 1] + d] - X[D * v[0] + d];
    double det, Ai[3][3];
    if (D == 2) {
      det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
      Ai[0][0] = A[1][1] / det;
      Ai[0][1] = -A[0][1] / det;
      Ai[1][0] = -A[1][0] / det;
      Ai[1][1] = A[0][0] / det;
    } else {
      const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1], c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2],
                   c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
      det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
      Ai[0][0] = c00 / det;
      Ai[1][0] = c01 / det;
      Ai[2][0] = c02 / det;
      Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
      Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
      Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
      Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
      Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
      Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    }
    if (!(det > 0)) {
      msg = "inverted or degenerate element " + std::to_string(e);
      return PCEXP_ERR_MESH;
    }
    // boundary measure |dE|
    double bnd = 0;
    for (int f = 0; f < NF; ++f) {
      double P[3][3];
      for (int k = 0; k < D; ++k)
        for (int d = 0; d < D; ++d) P[k][d] = X[D * v[fv(f, k)] + d];
      if (D == 2) {
        bnd += std::hypot(P[1][0] - P[0][0], P[1][1] - P[0][1]);
      } else {
        const double a[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
        const double b[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
        const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
        bnd += 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
      }
    }
    double* g = &s.geo[(size_t)GEO * e];
    for (int r = 0; r < D; ++r)
      for (int c = 0; c < D; ++c) g[r * D + c] = Ai[r][c];
    const double sdet = std::sqrt(det);
    g[D * D] = sdet;
    g[D * D + 1] = 2.0 * D * (det / fact) / bnd;  // h = 2 d |E| / |dE|
    g[D * D + 2] = 1.0 / sdet;                     // so the kernels multiply instead of dividing
    s.volume += det / fact;
    // quadrature points as offsets from v0, weights, centroid offset and half-extents
    double rc[3] = {0, 0, 0}, area = 0;
    for (int q = 0; q < nq; ++q) {
      for (int d = 0; d < D; ++d) {
        double a = 0;
        for (int k = 0; k < D; ++k) a += A[d][k] * (double)xr[q][k];
        rq[q * 3 + d] = a;
        s.xqphys[((size_t)e * nq + q) * D + d] = X[D * v[0] + d] + a;
      }
      pw[q] = (double)wr[q] * det;
      for (int d = 0; d < D; ++d) rc[d] += pw[q] * rq[q * 3 + d];
      area += pw[q];
    }
    double Lh[3];
    for (int d = 0; d < D; ++d) {
      rc[d] /= area;
      double mn = 0, mx = 0;  // offsets of the vertices from v0 (v0 itself at 0)
      for (int k = 0; k < D; ++k) {
        mn = std::min(mn, A[d][k]);
        mx = std::max(mx, A[d][k]);
      }
      Lh[d] = 0.5 * (mx - mn);
    }
    // paper basis values at the points by MGS (psi_i <- chi_i; psi_i -= <psi_i,psi_j> psi_j; normalise)
    for (int i = 0; i < nb; ++i) {
      for (int q = 0; q < nq; ++q) {
        double y[3];
        for (int d = 0; d < D; ++d) y[d] = (rq[q * 3 + d] - rc[d]) / Lh[d];
        vv[q] = mono_val(ex[i], y, D);
      }
      for (int j = 0; j < i; ++j) {
        double d = 0;
        for (int q = 0; q < nq; ++q) d += pw[q] * vv[q] * psi[j * nq + q];
        for (int q = 0; q < nq; ++q) vv[q] -= d * psi[j * nq + q];
      }
      double nr = 0;
      for (int q = 0; q < nq; ++q) nr += pw[q] * vv[q] * vv[q];
      nr = std::sqrt(nr);
      for (int q = 0; q < nq; ++q) psi[i * nq + q] = vv[q] / nr;
    }
    // Q[i][j] = <psi_i, phi_j>_E, phi_j = phi^_j / sqrt(det)
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double acc = 0;
        for (int q = 0; q < nq; ++q) acc += pw[q] * psi[i * nq + q] * s.Bv[q * nb + j];
        s.Q[((size_t)e * nb + i) * nb + j] = acc / sdet;
      }
  }

  // ---- faces: match element faces on periodic master vertices
  auto master = [&](int32_t vtx) -> int64_t { return mesh.vert_master ? mesh.vert_master[vtx] : vtx; };
  std::unordered_map<Key, int64_t, KeyHash> first;  // face -> e*NF+f of its first occurrence
  first.reserve((size_t)E * NF);
  std::unordered_map<Key, int32_t, KeyHash> btag;
  for (int64_t i = 0; i < mesh.n_bface; ++i) {
    int64_t vs[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) vs[k] = mesh.bface_vert[(size_t)D * i + k];
    int32_t t = mesh.bface_tag ? mesh.bface_tag[i] : 0;
    if (t != PCEXP_BC_SLIP_WALL && t != PCEXP_BC_FARFIELD && t != PCEXP_BC_SYMMETRY) {
      msg = "unknown boundary tag";
      return PCEXP_ERR_MESH;
    }
    btag[sorted_key(vs, D)] = t;
  }
  std::vector<int64_t> partner((size_t)E * NF, -1);
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < NF; ++f) {
      int64_t vs[3] = {0, 0, 0};
      for (int k = 0; k < D; ++k) vs[k] = master(EV[(D + 1) * e + fv(f, k)]);
      const Key key = sorted_key(vs, D);
      auto it = first.find(key);
      if (it == first.end()) {
        first.emplace(key, e * NF + f);
      } else {
        if (it->second < 0) {
          msg = "face shared by more than two elements";
          return PCEXP_ERR_MESH;
        }
        partner[it->second] = e * NF + f;
        partner[e * NF + f] = it->second;
        it->second = -1;
      }
    }
  s.ef.assign((size_t)E * NF, -1);
  s.fel.clear();
  s.floc.clear();
  s.fgeo.clear();
  int64_t F = 0;
  // interior faces first, in order of their L element
  // elements in increasing key order (their index without keys): the element of a face met
  // first is its L element, whose face points the face uses
  std::vector<int64_t> order((size_t)E);
  for (int64_t e = 0; e < E; ++e) order[(size_t)e] = e;
  if (elem_key)
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return elem_key[a] < elem_key[b]; });
  for (int pass = 0; pass < 2; ++pass)
    for (int64_t oe = 0; oe < E; ++oe)
      for (int f = 0; f < NF; ++f) {
        const int64_t e = order[(size_t)oe];
        const int64_t id = e * NF + f;
        if (s.ef[id] >= 0) continue;
        const int64_t pr = partner[id];
        if ((pass == 0) != (pr >= 0)) continue;
        if (F >= (int64_t(1) << 27)) {
          msg = "too many faces";
          return PCEXP_ERR_UNSUPPORTED;
        }
        int32_t lv[3];
        for (int k = 0; k < D; ++k) lv[k] = EV[(D + 1) * e + fv(f, k)];
        double nrm[3] = {0, 0, 0}, meas;
        if (D == 2) {
          const double tx = X[2 * lv[1]] - X[2 * lv[0]], ty = X[2 * lv[1] + 1] - X[2 * lv[0] + 1];
          const double len = std::hypot(tx, ty);
          nrm[0] = ty / len;
          nrm[1] = -tx / len;
          meas = len;
        } else {
          double a[3], b[3], o[3];
          for (int d = 0; d < 3; ++d) {
            a[d] = X[3 * lv[1] + d] - X[3 * lv[0] + d];
            b[d] = X[3 * lv[2] + d] - X[3 * lv[0] + d];
            o[d] = X[3 * lv[0] + d] - X[3 * EV[4 * e + f] + d];  // from the opposite vertex
          }
          double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
          const double cn = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
          const double sg = (c[0] * o[0] + c[1] * o[1] + c[2] * o[2]) < 0 ? -1.0 : 1.0;
          for (int d = 0; d < 3; ++d) nrm[d] = sg * c[d] / cn;
          meas = cn;  // twice the face area: the face weights sum to 1/2
        }
        int32_t eR, fR = 0, pR = 0;
        if (pr >= 0) {
          eR = (int32_t)(pr / NF);
          fR = (int)(pr % NF);
          int pi_of[3] = {-1, -1, -1};
          for (int k = 0; k < D; ++k)
            for (int j = 0; j < D; ++j)
              if (master(EV[(D + 1) * (int64_t)eR + fv(fR, j)]) == master(lv[k])) pi_of[k] = j;
          pR = -1;
          for (int pi = 0; pi < NPERM; ++pi) {
            bool ok = true;
            for (int k = 0; k < D; ++k) ok = ok && perm(pi, k) == pi_of[k];
            if (ok) pR = pi;
          }
          if (pR < 0 || (D == 2 && pR != 1)) {
            msg = D == 2 ? "neighbouring elements traverse a shared edge in the same sense"
                         : "shared face vertices do not match";
            return PCEXP_ERR_MESH;
          }
          s.ef[pr] = (int32_t)((F << 4) | (1 << 3) | pR);
        } else {
          int64_t vs[3] = {0, 0, 0};
          for (int k = 0; k < D; ++k) vs[k] = lv[k];
          auto it = btag.find(sorted_key(vs, D));
          if (it == btag.end()) {
            msg = "boundary face of element " + std::to_string(e) + " has no tag";
            return PCEXP_ERR_MESH;
          }
          eR = -it->second;
        }
        s.ef[id] = (int32_t)(F << 4);
        s.fel.push_back((int32_t)e);
        s.fel.push_back(eR);
        s.floc.push_back(f | (fR << 8) | (pR << 16));
        for (int d = 0; d < 3; ++d)
          if (d < D) s.fgeo.push_back(nrm[d]);
        s.fgeo.push_back(meas);
        if (D == 2) s.fgeo.push_back(0.0);
        ++F;
      }
  s.F = F;
  s.F_interior = 0;
  for (int64_t i = 0; i < F; ++i)
    if (s.fel[2 * i + 1] >= 0) ++s.F_interior;
  return PCEXP_OK;
}

}  // namespace pcexp
