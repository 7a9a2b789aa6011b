// Host preprocessing: quadrature, reference basis, paper-basis transform,
// element geometry and the face list (Sec. 4.2-4.3 of the paper).
//
// Quadrature (the paper does not fix it; same reading as the documented
// rules): Gauss-Legendre with p+1 points on edges; on triangles the collapsed
// product rule Gauss-Legendre x Gauss-Jacobi(1,0) with p+1 points per
// direction, mapped to the physical triangle (v0, v1, v2) by
// x = v0 + xi (v1 - v0) + eta (v2 - v0), xi = a (1 - b), eta = b.
// Nodes are found here by bisection on sign changes of the three-term
// recurrence, weights from the closed Christoffel form.
#include "host_setup.h"

#include <algorithm>
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

struct Poly2 {
  int ex, ey;
};

std::vector<Poly2> graded_exponents(int p) {
  std::vector<Poly2> e;
  for (int deg = 0; deg <= p; ++deg)
    for (int px = deg; px >= 0; --px) e.push_back({px, deg - px});
  return e;
}

long double ipow(long double x, int k) {
  long double r = 1.0L;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
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

int n_basis_2d(int p) { return (p + 1) * (p + 2) / 2; }

int build_setup(const pcexp_mesh& mesh, int p, Setup& s, std::string& msg) {
  if (mesh.dim != 2) {
    msg = "only triangle meshes (dim = 2) are supported";
    return PCEXP_ERR_UNSUPPORTED;
  }
  if (p < 0 || p > 3) {
    msg = "order p must be 0..3";
    return PCEXP_ERR_INVALID_ARG;
  }
  if (mesh.n_elem <= 0 || mesh.n_vert <= 0 || !mesh.coords || !mesh.elem_vert) {
    msg = "empty mesh";
    return PCEXP_ERR_INVALID_ARG;
  }
  const int nb = n_basis_2d(p), n1 = p + 1;
  s.p = p;
  s.nb = nb;
  s.nq = n1 * n1;
  s.nfq = n1;
  s.E = mesh.n_elem;
  const int64_t E = s.E;
  const int nq = s.nq, nfq = s.nfq;

  // ---- reference rule and reference orthonormal basis (MGS of monomials in (xi-1/3, eta-1/3))
  RuleTri tri = collapsed_triangle(n1);
  Rule1D edge = gauss_legendre_unit(n1);
  std::vector<Poly2> ex = graded_exponents(p);
  auto mono = [&](int k, long double xi, long double eta) {
    return ipow(xi - 1.0L / 3, ex[k].ex) * ipow(eta - 1.0L / 3, ex[k].ey);
  };
  auto dmono = [&](int k, int d, long double xi, long double eta) -> long double {
    if (d == 0)
      return ex[k].ex ? ex[k].ex * ipow(xi - 1.0L / 3, ex[k].ex - 1) * ipow(eta - 1.0L / 3, ex[k].ey) : 0.0L;
    return ex[k].ey ? ex[k].ey * ipow(xi - 1.0L / 3, ex[k].ex) * ipow(eta - 1.0L / 3, ex[k].ey - 1) : 0.0L;
  };
  std::vector<long double> Cr(nb * nb, 0.0L);  // phi^_i = sum_k Cr[i][k] mono_k
  {
    std::vector<long double> vals(nb * nq), psi(nb * nq);
    for (int k = 0; k < nb; ++k)
      for (int q = 0; q < nq; ++q) vals[k * nq + q] = mono(k, tri.xi[q], tri.eta[q]);
    for (int i = 0; i < nb; ++i) {
      std::vector<long double> c(nb, 0.0L), v(vals.begin() + i * nq, vals.begin() + (i + 1) * nq);
      c[i] = 1.0L;
      for (int j = 0; j < i; ++j) {
        long double d = 0;
        for (int q = 0; q < nq; ++q) d += tri.w[q] * v[q] * psi[j * nq + q];
        for (int q = 0; q < nq; ++q) v[q] -= d * psi[j * nq + q];
        for (int k = 0; k < nb; ++k) c[k] -= d * Cr[j * nb + k];
      }
      long double nr = 0;
      for (int q = 0; q < nq; ++q) nr += tri.w[q] * v[q] * v[q];
      nr = std::sqrt(nr);
      for (int q = 0; q < nq; ++q) psi[i * nq + q] = v[q] / nr;
      for (int k = 0; k < nb; ++k) Cr[i * nb + k] = c[k] / nr;
    }
  }
  auto phi = [&](int i, long double xi, long double eta) {
    long double r = 0;
    for (int k = 0; k <= i; ++k) r += Cr[i * nb + k] * mono(k, xi, eta);
    return r;
  };
  auto dphi = [&](int i, int d, long double xi, long double eta) {
    long double r = 0;
    for (int k = 0; k <= i; ++k) r += Cr[i * nb + k] * dmono(k, d, xi, eta);
    return r;
  };
  s.Bv.assign(nq * nb, 0);
  s.Dv.assign(2 * nq * nb, 0);
  s.Wv.assign(nq, 0);
  for (int q = 0; q < nq; ++q) {
    s.Wv[q] = (double)tri.w[q];
    for (int j = 0; j < nb; ++j) {
      s.Bv[q * nb + j] = (double)phi(j, tri.xi[q], tri.eta[q]);
      for (int d = 0; d < 2; ++d)
        s.Dv[(d * nq + q) * nb + j] = (double)(tri.w[q] * dphi(j, d, tri.xi[q], tri.eta[q]));
    }
  }
  const long double VX[3] = {0, 1, 0}, VY[3] = {0, 0, 1};
  s.Bf.assign(3 * nfq * nb, 0);
  s.Wf.assign(nfq, 0);
  for (int q = 0; q < nfq; ++q) s.Wf[q] = (double)edge.w[q];
  for (int f = 0; f < 3; ++f) {
    int a = (f + 1) % 3, b = (f + 2) % 3;
    for (int q = 0; q < nfq; ++q) {
      long double t = edge.x[q];
      long double xi = VX[a] + t * (VX[b] - VX[a]), eta = VY[a] + t * (VY[b] - VY[a]);
      for (int j = 0; j < nb; ++j) s.Bf[(f * nfq + q) * nb + j] = (double)phi(j, xi, eta);
    }
  }
  s.Bc.assign(nb, 0);
  for (int j = 0; j < nb; ++j) s.Bc[j] = (double)phi(j, 1.0L / 3, 1.0L / 3);

  // ---- element geometry and the paper-basis transform Q_e (Eq. basis, Algorithm 1)
  const double* X = mesh.coords;
  const int32_t* EV = mesh.elem_vert;
  s.geo.assign(E * 8, 0.0);
  s.xqphys.assign(E * nq * 2, 0.0);
  s.Q.assign(E * nb * nb, 0.0);
  s.volume = 0;
  for (int64_t e = 0; e < E; ++e) {
    int32_t v[3] = {EV[3 * e], EV[3 * e + 1], EV[3 * e + 2]};
    for (int k = 0; k < 3; ++k)
      if (v[k] < 0 || v[k] >= mesh.n_vert) {
        msg = "element vertex out of range";
        return PCEXP_ERR_MESH;
      }
    long double x0 = X[2 * v[0]], y0 = X[2 * v[0] + 1];
    long double x1 = X[2 * v[1]], y1 = X[2 * v[1] + 1];
    long double x2 = X[2 * v[2]], y2 = X[2 * v[2] + 1];
    long double A00 = x1 - x0, A01 = x2 - x0, A10 = y1 - y0, A11 = y2 - y0;
    long double det = A00 * A11 - A01 * A10;
    if (!(det > 0)) {
      msg = "inverted or degenerate element " + std::to_string(e);
      return PCEXP_ERR_MESH;
    }
    long double perim = std::hypot((double)(x1 - x0), (double)(y1 - y0)) +
                        std::hypot((double)(x2 - x1), (double)(y2 - y1)) +
                        std::hypot((double)(x0 - x2), (double)(y0 - y2));
    double* g = &s.geo[8 * e];
    g[0] = (double)(A11 / det);
    g[1] = (double)(-A01 / det);
    g[2] = (double)(-A10 / det);
    g[3] = (double)(A00 / det);
    long double sdet = std::sqrt(det);
    g[4] = (double)sdet;
    g[5] = (double)(2.0L * det / perim);  // h = 2 d |E| / |dE| with |E| = det / 2, d = 2
    s.volume += (double)(0.5L * det);
    // physical quadrature points
    std::vector<long double> px(nq), py(nq), pw(nq);
    long double xc = 0, yc = 0, area = 0;
    for (int q = 0; q < nq; ++q) {
      px[q] = x0 + tri.xi[q] * A00 + tri.eta[q] * A01;
      py[q] = y0 + tri.xi[q] * A10 + tri.eta[q] * A11;
      pw[q] = tri.w[q] * det;
      xc += pw[q] * px[q];
      yc += pw[q] * py[q];
      area += pw[q];
      s.xqphys[(e * nq + q) * 2] = (double)px[q];
      s.xqphys[(e * nq + q) * 2 + 1] = (double)py[q];
    }
    xc /= area;
    yc /= area;
    long double Lx = 0.5L * (std::max({x0, x1, x2}) - std::min({x0, x1, x2}));
    long double Ly = 0.5L * (std::max({y0, y1, y2}) - std::min({y0, y1, y2}));
    // paper basis values at the points by MGS (psi_i <- chi_i; psi_i -= <psi_i,psi_j> psi_j; normalise)
    std::vector<long double> psi(nb * nq);
    for (int i = 0; i < nb; ++i) {
      std::vector<long double> vv(nq);
      for (int q = 0; q < nq; ++q)
        vv[q] = ipow((px[q] - xc) / Lx, ex[i].ex) * ipow((py[q] - yc) / Ly, ex[i].ey);
      for (int j = 0; j < i; ++j) {
        long double d = 0;
        for (int q = 0; q < nq; ++q) d += pw[q] * vv[q] * psi[j * nq + q];
        for (int q = 0; q < nq; ++q) vv[q] -= d * psi[j * nq + q];
      }
      long double nr = 0;
      for (int q = 0; q < nq; ++q) nr += pw[q] * vv[q] * vv[q];
      nr = std::sqrt(nr);
      for (int q = 0; q < nq; ++q) psi[i * nq + q] = vv[q] / nr;
    }
    // Q[i][j] = <psi_i, phi_j>_E, phi_j = phi^_j / sqrt(det)
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        long double acc = 0;
        for (int q = 0; q < nq; ++q) acc += pw[q] * psi[i * nq + q] * (long double)s.Bv[q * nb + j];
        s.Q[(e * nb + i) * nb + j] = (double)(acc / sdet);
      }
  }

  // ---- faces: match edges on periodic master vertices
  auto master = [&](int32_t v) -> int64_t { return mesh.vert_master ? mesh.vert_master[v] : v; };
  auto key2 = [](int64_t a, int64_t b) -> uint64_t {
    if (a > b) std::swap(a, b);
    return ((uint64_t)a << 32) | (uint64_t)b;
  };
  std::unordered_map<uint64_t, int64_t> first;  // edge -> e*3+f of its first occurrence
  first.reserve(E * 3);
  std::unordered_map<uint64_t, int32_t> btag;
  for (int64_t i = 0; i < mesh.n_bface; ++i) {
    int32_t a = mesh.bface_vert[2 * i], b = mesh.bface_vert[2 * i + 1];
    int32_t t = mesh.bface_tag ? mesh.bface_tag[i] : 0;
    if (t != PCEXP_BC_SLIP_WALL && t != PCEXP_BC_FARFIELD) {
      msg = "unknown boundary tag";
      return PCEXP_ERR_MESH;
    }
    btag[key2(a, b)] = t;
  }
  std::vector<int64_t> partner(E * 3, -1);
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 3; ++f) {
      int32_t a = EV[3 * e + (f + 1) % 3], b = EV[3 * e + (f + 2) % 3];
      uint64_t k = key2(master(a), master(b));
      auto it = first.find(k);
      if (it == first.end()) {
        first.emplace(k, e * 3 + f);
      } else {
        if (it->second < 0) {
          msg = "edge shared by more than two elements";
          return PCEXP_ERR_MESH;
        }
        partner[it->second] = e * 3 + f;
        partner[e * 3 + f] = it->second;
        it->second = -1;
      }
    }
  s.ef.assign(E * 3, -1);
  s.fel.clear();
  s.floc.clear();
  s.fgeo.clear();
  int64_t F = 0;
  // interior faces first, in order of their L element
  for (int pass = 0; pass < 2; ++pass)
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 3; ++f) {
        int64_t id = e * 3 + f;
        if (s.ef[id] >= 0) continue;
        int64_t pr = partner[id];
        if ((pass == 0) != (pr >= 0)) continue;
        int32_t a = EV[3 * e + (f + 1) % 3], b = EV[3 * e + (f + 2) % 3];
        double ax = X[2 * a], ay = X[2 * a + 1], bx = X[2 * b], by = X[2 * b + 1];
        double tx = bx - ax, ty = by - ay, len = std::hypot(tx, ty);
        int32_t eR, fR = 0;
        if (pr >= 0) {
          eR = (int32_t)(pr / 3);
          fR = (int)(pr % 3);
          int32_t aR = EV[3 * eR + (fR + 1) % 3], bR = EV[3 * eR + (fR + 2) % 3];
          if (master(aR) != master(b) || master(bR) != master(a)) {
            msg = "neighbouring elements traverse a shared edge in the same sense";
            return PCEXP_ERR_MESH;
          }
          s.ef[pr] = (int32_t)(F * 2 + 1);
        } else {
          auto it = btag.find(key2(a, b));
          if (it == btag.end()) {
            msg = "boundary edge " + std::to_string(a) + "-" + std::to_string(b) + " has no tag";
            return PCEXP_ERR_MESH;
          }
          eR = -it->second;
        }
        s.ef[id] = (int32_t)(F * 2);
        s.fel.push_back((int32_t)e);
        s.fel.push_back(eR);
        s.floc.push_back(f | (fR << 8));
        s.fgeo.push_back(ty / len);
        s.fgeo.push_back(-tx / len);
        s.fgeo.push_back(len);
        s.fgeo.push_back(0.0);
        ++F;
      }
  s.F = F;
  s.F_interior = 0;
  for (int64_t i = 0; i < F; ++i)
    if (s.fel[2 * i + 1] >= 0) ++s.F_interior;
  return PCEXP_OK;
}

}  // namespace pcexp
