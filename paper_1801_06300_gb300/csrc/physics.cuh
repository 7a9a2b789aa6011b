// Euler physics for the DG kernels (Sec. 4.1, 4.4 of the paper), written once
// over a scalar type S that is either a real type (the residual) or Tangent<T>
// (value + directional derivative: the tangent-linear J v kernel).
//
// Riemann flux: Roe's solver with square-root-density averages and no entropy
// fix, F~ = 1/2 (F_n(U_L) + F_n(U_R)) - 1/2 sum_k |lambda_k| alpha_k r_k.
// Ghost states: slip wall mirrors the normal velocity; the far field uses the
// one-dimensional Riemann invariants R+- = q_n +- 2 c / (gamma - 1), with R+
// from the interior unless its normal Mach number is <= -1, R- from the free
// stream unless it is >= 1, entropy and tangential velocity from the interior
// when the boundary normal velocity is >= 0, else from the free stream.
#pragma once
#include <cuda_runtime.h>

#define PCEXP_DEV __device__ __forceinline__

namespace pcexp {

// ---------------------------------------------------------------- tangent scalar
template <class T>
struct Tangent {
  T v, d;  // value and derivative along the direction
};

template <class T> PCEXP_DEV T val(T x) { return x; }
template <class T> PCEXP_DEV T val(Tangent<T> x) { return x.v; }

template <class T> PCEXP_DEV Tangent<T> operator+(Tangent<T> a, Tangent<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> PCEXP_DEV Tangent<T> operator-(Tangent<T> a, Tangent<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> PCEXP_DEV Tangent<T> operator-(Tangent<T> a) { return {-a.v, -a.d}; }
template <class T> PCEXP_DEV Tangent<T> operator*(Tangent<T> a, Tangent<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> PCEXP_DEV Tangent<T> operator/(Tangent<T> a, Tangent<T> b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> PCEXP_DEV Tangent<T> operator+(Tangent<T> a, T b) { return {a.v + b, a.d}; }
template <class T> PCEXP_DEV Tangent<T> operator+(T a, Tangent<T> b) { return {a + b.v, b.d}; }
template <class T> PCEXP_DEV Tangent<T> operator-(Tangent<T> a, T b) { return {a.v - b, a.d}; }
template <class T> PCEXP_DEV Tangent<T> operator-(T a, Tangent<T> b) { return {a - b.v, -b.d}; }
template <class T> PCEXP_DEV Tangent<T> operator*(Tangent<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> PCEXP_DEV Tangent<T> operator*(T a, Tangent<T> b) { return {a * b.v, a * b.d}; }
template <class T> PCEXP_DEV Tangent<T> operator/(Tangent<T> a, T b) { return {a.v / b, a.d / b}; }
template <class T> PCEXP_DEV Tangent<T> operator/(T a, Tangent<T> b) {
  T q = a / b.v;
  return {q, -q * b.d / b.v};
}

PCEXP_DEV double sqrt_s(double x) { return sqrt(x); }
PCEXP_DEV float sqrt_s(float x) { return sqrtf(x); }
template <class T> PCEXP_DEV Tangent<T> sqrt_s(Tangent<T> x) {
  T s = sqrt_s(x.v);
  return {s, x.d / (T(2) * s)};
}
// |x| with derivative sign(x) * dx, sign(0) = 0
PCEXP_DEV double abs_s(double x) { return fabs(x); }
PCEXP_DEV float abs_s(float x) { return fabsf(x); }
template <class T> PCEXP_DEV Tangent<T> abs_s(Tangent<T> x) {
  T sg = x.v > T(0) ? T(1) : (x.v < T(0) ? T(-1) : T(0));
  return {sg * x.v, sg * x.d};
}
PCEXP_DEV double pow_s(double x, double e) { return pow(x, e); }
PCEXP_DEV float pow_s(float x, float e) { return powf(x, e); }
template <class T> PCEXP_DEV Tangent<T> pow_s(Tangent<T> x, T e) {
  T pv = pow_s(x.v, e);
  return {pv, e * pv / x.v * x.d};
}
template <class S> PCEXP_DEV S select_s(bool c, S a, S b) { return c ? a : b; }


// ------------------------------------------------- multi-direction tangent (Jacobians)
// Jet<T, N>: value and its derivatives along N directions; evaluating a flux on
// Jets seeded with unit directions gives N columns of its exact Jacobian.
template <class T, int N>
struct Jet {
  T v;
  T d[N];
};
template <class T, int N> PCEXP_DEV T val(const Jet<T, N>& x) { return x.v; }
#define PCEXP_JET_BIN(OP, DEXPR)                                                        \
  template <class T, int N>                                                             \
  PCEXP_DEV Jet<T, N> operator OP(const Jet<T, N>& a, const Jet<T, N>& b) {             \
    Jet<T, N> r;                                                                        \
    r.v = a.v OP b.v;                                                                   \
    _Pragma("unroll") for (int k = 0; k < N; ++k) r.d[k] = DEXPR;                       \
    return r;                                                                           \
  }
PCEXP_JET_BIN(+, a.d[k] + b.d[k])
PCEXP_JET_BIN(-, a.d[k] - b.d[k])
PCEXP_JET_BIN(*, a.d[k] * b.v + a.v * b.d[k])
#undef PCEXP_JET_BIN
template <class T, int N> PCEXP_DEV Jet<T, N> operator/(const Jet<T, N>& a, const Jet<T, N>& b) {
  Jet<T, N> r;
  r.v = a.v / b.v;
  const T ib = T(1) / b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <class T, int N> PCEXP_DEV Jet<T, N> operator-(const Jet<T, N>& a) {
  Jet<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <class T, int N> PCEXP_DEV Jet<T, N> operator+(const Jet<T, N>& a, T b) { Jet<T, N> r = a; r.v += b; return r; }
template <class T, int N> PCEXP_DEV Jet<T, N> operator+(T a, const Jet<T, N>& b) { Jet<T, N> r = b; r.v += a; return r; }
template <class T, int N> PCEXP_DEV Jet<T, N> operator-(const Jet<T, N>& a, T b) { Jet<T, N> r = a; r.v -= b; return r; }
template <class T, int N> PCEXP_DEV Jet<T, N> operator-(T a, const Jet<T, N>& b) {
  Jet<T, N> r;
  r.v = a - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -b.d[k];
  return r;
}
template <class T, int N> PCEXP_DEV Jet<T, N> operator*(const Jet<T, N>& a, T b) {
  Jet<T, N> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
  return r;
}
template <class T, int N> PCEXP_DEV Jet<T, N> operator*(T a, const Jet<T, N>& b) { return b * a; }
template <class T, int N> PCEXP_DEV Jet<T, N> operator/(const Jet<T, N>& a, T b) { return a * (T(1) / b); }
template <class T, int N> PCEXP_DEV Jet<T, N> operator/(T a, const Jet<T, N>& b) {
  Jet<T, N> r;
  r.v = a / b.v;
  const T f = -r.v / b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = f * b.d[k];
  return r;
}
template <class T, int N> PCEXP_DEV Jet<T, N> sqrt_s(const Jet<T, N>& x) {
  Jet<T, N> r;
  r.v = sqrt_s(x.v);
  const T f = T(0.5) / r.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = f * x.d[k];
  return r;
}
template <class T, int N> PCEXP_DEV Jet<T, N> abs_s(const Jet<T, N>& x) {
  const T sg = x.v > T(0) ? T(1) : (x.v < T(0) ? T(-1) : T(0));
  Jet<T, N> r;
  r.v = sg * x.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = sg * x.d[k];
  return r;
}
template <class T, int N> PCEXP_DEV Jet<T, N> pow_s(const Jet<T, N>& x, T e) {
  Jet<T, N> r;
  r.v = pow_s(x.v, e);
  const T f = e * r.v / x.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = f * x.d[k];
  return r;
}
template <class S, class T> struct Lift {
  PCEXP_DEV static S of(T x) { return S(x); }
};
template <class T> struct Lift<Tangent<T>, T> {
  PCEXP_DEV static Tangent<T> of(T x) { return {x, T(0)}; }
};
template <class T, int N> struct Lift<Jet<T, N>, T> {
  PCEXP_DEV static Jet<T, N> of(T x) {
    Jet<T, N> r;
    r.v = x;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = T(0);
    return r;
  }
};

// ------------------------------------------------------- hyper-dual (second order)
// HD4<T>: value v, partials d[c] along 4 seeded directions, the directional
// derivative t along one more direction, and the partials dt[c] of t.  Running a
// flux on HD4 gives d/dU_c (dF/dU . t): the second-order term needed by the adjoint of
// a Jacobian-vector product with respect to the linearisation state.
template <class T>
struct HD4 {
  T v;
  T d[4];
  T t;
  T dt[4];
};
template <class T> PCEXP_DEV T val(const HD4<T>& x) { return x.v; }
template <class T> PCEXP_DEV HD4<T> operator+(const HD4<T>& a, const HD4<T>& b) {
  HD4<T> r;
  r.v = a.v + b.v;
  r.t = a.t + b.t;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    r.d[c] = a.d[c] + b.d[c];
    r.dt[c] = a.dt[c] + b.dt[c];
  }
  return r;
}
template <class T> PCEXP_DEV HD4<T> operator-(const HD4<T>& a) {
  HD4<T> r;
  r.v = -a.v;
  r.t = -a.t;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    r.d[c] = -a.d[c];
    r.dt[c] = -a.dt[c];
  }
  return r;
}
template <class T> PCEXP_DEV HD4<T> operator-(const HD4<T>& a, const HD4<T>& b) { return a + (-b); }
template <class T> PCEXP_DEV HD4<T> operator*(const HD4<T>& a, const HD4<T>& b) {
  HD4<T> r;
  r.v = a.v * b.v;
  r.t = a.t * b.v + a.v * b.t;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    r.d[c] = a.d[c] * b.v + a.v * b.d[c];
    r.dt[c] = a.dt[c] * b.v + a.t * b.d[c] + a.d[c] * b.t + a.v * b.dt[c];
  }
  return r;
}
template <class T> PCEXP_DEV HD4<T> operator*(const HD4<T>& a, T b) {
  HD4<T> r;
  r.v = a.v * b;
  r.t = a.t * b;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    r.d[c] = a.d[c] * b;
    r.dt[c] = a.dt[c] * b;
  }
  return r;
}
template <class T> PCEXP_DEV HD4<T> operator*(T a, const HD4<T>& b) { return b * a; }
template <class T> PCEXP_DEV HD4<T> operator+(const HD4<T>& a, T b) { HD4<T> r = a; r.v += b; return r; }
template <class T> PCEXP_DEV HD4<T> operator+(T a, const HD4<T>& b) { HD4<T> r = b; r.v += a; return r; }
template <class T> PCEXP_DEV HD4<T> operator-(const HD4<T>& a, T b) { HD4<T> r = a; r.v -= b; return r; }
template <class T> PCEXP_DEV HD4<T> operator-(T a, const HD4<T>& b) { return (-b) + a; }
// f(a) from f, f', f'' at a.v
template <class T> PCEXP_DEV HD4<T> hd_apply(const HD4<T>& a, T f0, T f1, T f2) {
  HD4<T> r;
  r.v = f0;
  r.t = f1 * a.t;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    r.d[c] = f1 * a.d[c];
    r.dt[c] = f1 * a.dt[c] + f2 * a.d[c] * a.t;
  }
  return r;
}
template <class T> PCEXP_DEV HD4<T> hd_inv(const HD4<T>& a) {
  const T i = T(1) / a.v;
  return hd_apply(a, i, -i * i, T(2) * i * i * i);
}
template <class T> PCEXP_DEV HD4<T> operator/(const HD4<T>& a, const HD4<T>& b) { return a * hd_inv(b); }
template <class T> PCEXP_DEV HD4<T> operator/(const HD4<T>& a, T b) { return a * (T(1) / b); }
template <class T> PCEXP_DEV HD4<T> operator/(T a, const HD4<T>& b) { return hd_inv(b) * a; }
template <class T> PCEXP_DEV HD4<T> sqrt_s(const HD4<T>& a) {
  const T s = sqrt_s(a.v);
  return hd_apply(a, s, T(0.5) / s, T(-0.25) / (s * a.v));
}
template <class T> PCEXP_DEV HD4<T> abs_s(const HD4<T>& a) {
  const T sg = a.v > T(0) ? T(1) : (a.v < T(0) ? T(-1) : T(0));
  return hd_apply(a, sg * a.v, sg, T(0));
}
template <class T> PCEXP_DEV HD4<T> pow_s(const HD4<T>& a, T e) {
  const T p = pow_s(a.v, e);
  return hd_apply(a, p, e * p / a.v, e * (e - T(1)) * p / (a.v * a.v));
}
template <class T> struct Lift<HD4<T>, T> {
  PCEXP_DEV static HD4<T> of(T x) {
    HD4<T> r;
    r.v = x;
    r.t = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) r.d[c] = r.dt[c] = T(0);
    return r;
  }
};

// ---------------------------------------------------------------- free stream
template <class T>
struct Free {
  T gamma, rho, u, v, p;
};

// ---------------------------------------------------------------- fluxes (2D, 4 variables)
// Physical fluxes along x and y of U = (rho, rho u, rho v, rho E).
template <class S, class T>
PCEXP_DEV void euler_flux(const S U[4], T g, S Fx[4], S Fy[4]) {
  S ir = T(1) / U[0];
  S u = U[1] * ir, v = U[2] * ir;
  S p = (g - T(1)) * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
  S e = U[3] + p;
  Fx[0] = U[1];
  Fx[1] = U[1] * u + p;
  Fx[2] = U[2] * u;
  Fx[3] = e * u;
  Fy[0] = U[2];
  Fy[1] = U[1] * v;
  Fy[2] = U[2] * v + p;
  Fy[3] = e * v;
}

// Roe flux F~(U_L, U_R) . n
template <class S, class T>
PCEXP_DEV void roe_flux(const S L[4], const S R[4], T nx, T ny, T g, S F[4]) {
  const T gm = g - T(1);
  S rL = L[0], irL = T(1) / rL, uL = L[1] * irL, vL = L[2] * irL;
  S pL = gm * (L[3] - T(0.5) * (L[1] * uL + L[2] * vL));
  S rR = R[0], irR = T(1) / rR, uR = R[1] * irR, vR = R[2] * irR;
  S pR = gm * (R[3] - T(0.5) * (R[1] * uR + R[2] * vR));
  S qL = uL * nx + vL * ny, qR = uR * nx + vR * ny;
  S HL = (L[3] + pL) * irL, HR = (R[3] + pR) * irR;
  // central part
  S c0 = rL * qL + rR * qR;
  S c1 = L[1] * qL + R[1] * qR + (pL + pR) * nx;
  S c2 = L[2] * qL + R[2] * qR + (pL + pR) * ny;
  S c3 = (L[3] + pL) * qL + (R[3] + pR) * qR;
  // Roe averages
  S sL = sqrt_s(rL), sR = sqrt_s(rR), is = T(1) / (sL + sR);
  S rh = sL * sR;
  S uh = (sL * uL + sR * uR) * is, vh = (sL * vL + sR * vR) * is;
  S Hh = (sL * HL + sR * HR) * is;
  S q2 = uh * uh + vh * vh;
  S cc = gm * (Hh - T(0.5) * q2);
  S c = sqrt_s(cc);
  S qh = uh * nx + vh * ny;
  // jumps and wave strengths
  S dp = pR - pL, dr = rR - rL, du = uR - uL, dv = vR - vL;
  S dq = du * nx + dv * ny;
  S l1 = abs_s(qh - c), l2 = abs_s(qh), l4 = abs_s(qh + c);
  S i2c = T(0.5) / cc;
  S a1 = (dp - rh * c * dq) * i2c;
  S a4 = (dp + rh * c * dq) * i2c;
  S a2 = dr - dp / cc;
  S t1 = l1 * a1, t4 = l4 * a4, t2 = l2 * a2, ts = l2 * rh;
  S d0 = t1 + t2 + t4;
  S d1 = t1 * (uh - c * nx) + t2 * uh + ts * (du - dq * nx) + t4 * (uh + c * nx);
  S d2 = t1 * (vh - c * ny) + t2 * vh + ts * (dv - dq * ny) + t4 * (vh + c * ny);
  S d3 = t1 * (Hh - c * qh) + t2 * (T(0.5) * q2) + ts * (uh * du + vh * dv - qh * dq) + t4 * (Hh + c * qh);
  F[0] = T(0.5) * (c0 - d0);
  F[1] = T(0.5) * (c1 - d1);
  F[2] = T(0.5) * (c2 - d2);
  F[3] = T(0.5) * (c3 - d3);
}

template <class S, class T>
PCEXP_DEV void ghost_slip_wall(const S U[4], T nx, T ny, S G[4]) {
  S ir = T(1) / U[0];
  S qn = (U[1] * nx + U[2] * ny) * ir;  // normal velocity
  G[0] = U[0];
  G[1] = U[1] - T(2) * U[0] * qn * nx;
  G[2] = U[2] - T(2) * U[0] * qn * ny;
  G[3] = U[3];
}

template <class S, class T>
PCEXP_DEV void ghost_farfield(const S U[4], T nx, T ny, const Free<T>& fs, S G[4]) {
  const T g = fs.gamma, gm = g - T(1);
  S ir = T(1) / U[0];
  S u = U[1] * ir, v = U[2] * ir;
  S p = gm * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
  S c = sqrt_s(g * p * ir);
  S qn = u * nx + v * ny;
  T cinf = sqrt_s(g * fs.p / fs.rho);
  T qinf = fs.u * nx + fs.v * ny;
  T mn = val(qn) / val(c);
  S rp = select_s(mn > T(-1), qn + T(2) * c / gm, Lift<S, T>::of(qinf + T(2) * cinf / gm));
  S rm = select_s(mn < T(1), Lift<S, T>::of(qinf - T(2) * cinf / gm), qn - T(2) * c / gm);
  S qb = T(0.5) * (rp + rm);
  S cb = T(0.25) * gm * (rp - rm);
  bool out = val(qb) >= T(0);
  S s_in = p / pow_s(U[0], g);
  T s_inf = fs.p / pow_s(fs.rho, g);
  S sb = select_s(out, s_in, Lift<S, T>::of(s_inf));
  S ut = select_s(out, u - qn * nx, Lift<S, T>::of(fs.u - qinf * nx));
  S vt = select_s(out, v - qn * ny, Lift<S, T>::of(fs.v - qinf * ny));
  S ub = ut + qb * nx, vb = vt + qb * ny;
  S rb = pow_s(cb * cb / (g * sb), T(1) / gm);
  S pb = rb * cb * cb / g;
  G[0] = rb;
  G[1] = rb * ub;
  G[2] = rb * vb;
  G[3] = pb / gm + T(0.5) * rb * (ub * ub + vb * vb);
}

}  // namespace pcexp
