// Euler physics for the DG kernels (Sec. 4.1, 4.4 of the paper), written once
// over the dimension D (2 or 3; D + 2 conservative variables) and over a scalar
// type S that is a real type (the residual), Tangent<T> (value + directional
// derivative: J v), Jet<T, N> (point Jacobians) or HD<T, N> (second order).
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
PCEXP_DEV double exp_s(double x) { return exp(x); }
template <class T, int N> PCEXP_DEV Jet<T, N> exp_s(const Jet<T, N>& x) {
  Jet<T, N> r;
  r.v = exp(x.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = r.v * x.d[k];
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
// HD<T, N>: value v, partials d[c] along N seeded directions, the directional
// derivative t along one more direction, and the partials dt[c] of t.  Running a
// flux on HD gives d/dU_c (dF/dU . t): the second-order term needed by the adjoint of
// a Jacobian-vector product with respect to the linearisation state.
template <class T, int N>
struct HD {
  T v;
  T d[N];
  T t;
  T dt[N];
};
template <class T, int N> PCEXP_DEV T val(const HD<T, N>& x) { return x.v; }
template <class T, int N> PCEXP_DEV HD<T, N> operator+(const HD<T, N>& a, const HD<T, N>& b) {
  HD<T, N> r;
  r.v = a.v + b.v;
  r.t = a.t + b.t;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    r.d[c] = a.d[c] + b.d[c];
    r.dt[c] = a.dt[c] + b.dt[c];
  }
  return r;
}
template <class T, int N> PCEXP_DEV HD<T, N> operator-(const HD<T, N>& a) {
  HD<T, N> r;
  r.v = -a.v;
  r.t = -a.t;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    r.d[c] = -a.d[c];
    r.dt[c] = -a.dt[c];
  }
  return r;
}
template <class T, int N> PCEXP_DEV HD<T, N> operator-(const HD<T, N>& a, const HD<T, N>& b) { return a + (-b); }
template <class T, int N> PCEXP_DEV HD<T, N> operator*(const HD<T, N>& a, const HD<T, N>& b) {
  HD<T, N> r;
  r.v = a.v * b.v;
  r.t = a.t * b.v + a.v * b.t;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    r.d[c] = a.d[c] * b.v + a.v * b.d[c];
    r.dt[c] = a.dt[c] * b.v + a.t * b.d[c] + a.d[c] * b.t + a.v * b.dt[c];
  }
  return r;
}
template <class T, int N> PCEXP_DEV HD<T, N> operator*(const HD<T, N>& a, T b) {
  HD<T, N> r;
  r.v = a.v * b;
  r.t = a.t * b;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    r.d[c] = a.d[c] * b;
    r.dt[c] = a.dt[c] * b;
  }
  return r;
}
template <class T, int N> PCEXP_DEV HD<T, N> operator*(T a, const HD<T, N>& b) { return b * a; }
template <class T, int N> PCEXP_DEV HD<T, N> operator+(const HD<T, N>& a, T b) { HD<T, N> r = a; r.v += b; return r; }
template <class T, int N> PCEXP_DEV HD<T, N> operator+(T a, const HD<T, N>& b) { HD<T, N> r = b; r.v += a; return r; }
template <class T, int N> PCEXP_DEV HD<T, N> operator-(const HD<T, N>& a, T b) { HD<T, N> r = a; r.v -= b; return r; }
template <class T, int N> PCEXP_DEV HD<T, N> operator-(T a, const HD<T, N>& b) { return (-b) + a; }
// f(a) from f, f', f'' at a.v
template <class T, int N> PCEXP_DEV HD<T, N> hd_apply(const HD<T, N>& a, T f0, T f1, T f2) {
  HD<T, N> r;
  r.v = f0;
  r.t = f1 * a.t;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    r.d[c] = f1 * a.d[c];
    r.dt[c] = f1 * a.dt[c] + f2 * a.d[c] * a.t;
  }
  return r;
}
template <class T, int N> PCEXP_DEV HD<T, N> hd_inv(const HD<T, N>& a) {
  const T i = T(1) / a.v;
  return hd_apply(a, i, -i * i, T(2) * i * i * i);
}
template <class T, int N> PCEXP_DEV HD<T, N> operator/(const HD<T, N>& a, const HD<T, N>& b) { return a * hd_inv(b); }
template <class T, int N> PCEXP_DEV HD<T, N> operator/(const HD<T, N>& a, T b) { return a * (T(1) / b); }
template <class T, int N> PCEXP_DEV HD<T, N> operator/(T a, const HD<T, N>& b) { return hd_inv(b) * a; }
template <class T, int N> PCEXP_DEV HD<T, N> sqrt_s(const HD<T, N>& a) {
  const T s = sqrt_s(a.v);
  return hd_apply(a, s, T(0.5) / s, T(-0.25) / (s * a.v));
}
template <class T, int N> PCEXP_DEV HD<T, N> abs_s(const HD<T, N>& a) {
  const T sg = a.v > T(0) ? T(1) : (a.v < T(0) ? T(-1) : T(0));
  return hd_apply(a, sg * a.v, sg, T(0));
}
template <class T, int N> PCEXP_DEV HD<T, N> pow_s(const HD<T, N>& a, T e) {
  const T p = pow_s(a.v, e);
  return hd_apply(a, p, e * p / a.v, e * (e - T(1)) * p / (a.v * a.v));
}
template <class T, int N> struct Lift<HD<T, N>, T> {
  PCEXP_DEV static HD<T, N> of(T x) {
    HD<T, N> r;
    r.v = x;
    r.t = T(0);
#pragma unroll
    for (int c = 0; c < N; ++c) r.d[c] = r.dt[c] = T(0);
    return r;
  }
};

// ---------------------------------------------------------------- free stream
// vel holds the free-stream velocity in x, y (and z in 3D; zero in the x-y-plane cases)
template <class T>
struct Free {
  T gamma, rho, p;
  T vel[3];
};

// ------------------------------------------------------ fluxes (D dimensions, D+2 variables)
// Physical fluxes F[d] along the Cartesian axes of U = (rho, rho v_1..rho v_D, rho E).
template <int D, class S, class T>
PCEXP_DEV void euler_flux(const S (&U)[D + 2], T g, S (&F)[D][D + 2]) {
  constexpr int NV = D + 2;
  const S ir = T(1) / U[0];
  S vel[D];
#pragma unroll
  for (int d = 0; d < D; ++d) vel[d] = U[1 + d] * ir;
  S ke = U[1] * vel[0];
#pragma unroll
  for (int d = 1; d < D; ++d) ke = ke + U[1 + d] * vel[d];
  const S p = (g - T(1)) * (U[NV - 1] - T(0.5) * ke);
  const S e = U[NV - 1] + p;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    F[d][0] = U[1 + d];
#pragma unroll
    for (int k = 0; k < D; ++k) F[d][1 + k] = (k == d) ? U[1 + k] * vel[d] + p : U[1 + k] * vel[d];
    F[d][NV - 1] = e * vel[d];
  }
}

template <int D, class S, class T>
PCEXP_DEV S dot_n(const S (&a)[D], const T (&n)[D]) {
  S r = a[0] * n[0];
#pragma unroll
  for (int d = 1; d < D; ++d) r = r + a[d] * n[d];
  return r;
}

// Roe flux F~(U_L, U_R) . n.  vrn = v_r . n, the normal velocity of a rotating frame at the
// face point (Sec. 4.1): F . n = F_abs . n - vrn U and the waves' speeds are shifted by -vrn
// (vrn = 0: the fixed frame, the same operations as without it).
template <int D, class S, class T>
PCEXP_DEV void roe_flux(const S (&L)[D + 2], const S (&R)[D + 2], const T (&n)[D], T g, S (&F)[D + 2],
                        T vrn = T(0)) {
  constexpr int NV = D + 2;
  const T gm = g - T(1);
  S rL = L[0], irL = T(1) / rL, rR = R[0], irR = T(1) / rR;
  S vL[D], vR[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    vL[d] = L[1 + d] * irL;
    vR[d] = R[1 + d] * irR;
  }
  S keL = L[1] * vL[0], keR = R[1] * vR[0];
#pragma unroll
  for (int d = 1; d < D; ++d) {
    keL = keL + L[1 + d] * vL[d];
    keR = keR + R[1 + d] * vR[d];
  }
  S pL = gm * (L[NV - 1] - T(0.5) * keL);
  S pR = gm * (R[NV - 1] - T(0.5) * keR);
  S qL = dot_n<D>(vL, n), qR = dot_n<D>(vR, n);
  S HL = (L[NV - 1] + pL) * irL, HR = (R[NV - 1] + pR) * irR;
  // central part
  S c[NV];
  c[0] = rL * qL + rR * qR;
#pragma unroll
  for (int d = 0; d < D; ++d) c[1 + d] = L[1 + d] * qL + R[1 + d] * qR + (pL + pR) * n[d];
  c[NV - 1] = (L[NV - 1] + pL) * qL + (R[NV - 1] + pR) * qR;
  // Roe averages
  S sL = sqrt_s(rL), sR = sqrt_s(rR), is = T(1) / (sL + sR);
  S rh = sL * sR;
  S vh[D];
#pragma unroll
  for (int d = 0; d < D; ++d) vh[d] = (sL * vL[d] + sR * vR[d]) * is;
  S Hh = (sL * HL + sR * HR) * is;
  S q2 = vh[0] * vh[0];
#pragma unroll
  for (int d = 1; d < D; ++d) q2 = q2 + vh[d] * vh[d];
  S cc = gm * (Hh - T(0.5) * q2);
  S cs = sqrt_s(cc);
  S qh = dot_n<D>(vh, n);
  // jumps and wave strengths
  S dp = pR - pL, dr = rR - rL;
  S dv[D];
#pragma unroll
  for (int d = 0; d < D; ++d) dv[d] = vR[d] - vL[d];
  S dq = dot_n<D>(dv, n);
  const S qs = vrn != T(0) ? qh - vrn : qh;  // wave speeds relative to the frame
  S l1 = abs_s(qs - cs), l2 = abs_s(qs), l4 = abs_s(qs + cs);
  S i2c = T(0.5) / cc;
  S a1 = (dp - rh * cs * dq) * i2c;
  S a4 = (dp + rh * cs * dq) * i2c;
  S a2 = dr - dp / cc;
  S t1 = l1 * a1, t4 = l4 * a4, t2 = l2 * a2, ts = l2 * rh;
  S dd[NV];
  dd[0] = t1 + t2 + t4;
  S vdv = vh[0] * dv[0];
#pragma unroll
  for (int d = 1; d < D; ++d) vdv = vdv + vh[d] * dv[d];
#pragma unroll
  for (int d = 0; d < D; ++d)
    dd[1 + d] = t1 * (vh[d] - cs * n[d]) + t2 * vh[d] + ts * (dv[d] - dq * n[d]) + t4 * (vh[d] + cs * n[d]);
  dd[NV - 1] = t1 * (Hh - cs * qh) + t2 * (T(0.5) * q2) + ts * (vdv - qh * dq) + t4 * (Hh + cs * qh);
  if (vrn != T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = c[v] - vrn * (L[v] + R[v]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = T(0.5) * (c[v] - dd[v]);
}

// Slip wall and symmetry plane: the velocity relative to the wall (which moves with a
// rotating frame: vrn = v_r . n) has its normal component mirrored; density and pressure are
// kept.  v_g = v - 2 q n with q = v . n - vrn, so |v_g|^2 = |v|^2 - 4 q vrn and the ghost's
// total energy is rho E - 2 rho q vrn (unchanged in a fixed frame).
template <int D, class S, class T>
PCEXP_DEV void ghost_slip_wall(const S (&U)[D + 2], const T (&n)[D], S (&G)[D + 2], T vrn = T(0)) {
  constexpr int NV = D + 2;
  const S ir = T(1) / U[0];
  S m[D];
#pragma unroll
  for (int d = 0; d < D; ++d) m[d] = U[1 + d];
  S qn = dot_n<D>(m, n) * ir;  // normal velocity
  if (vrn != T(0)) qn = qn - vrn;
  G[0] = U[0];
#pragma unroll
  for (int d = 0; d < D; ++d) G[1 + d] = U[1 + d] - T(2) * U[0] * qn * n[d];
  G[NV - 1] = U[NV - 1];
  if (vrn != T(0)) G[NV - 1] = G[NV - 1] - T(2) * vrn * (U[0] * qn);
}

template <int D, class S, class T>
PCEXP_DEV void ghost_farfield(const S (&U)[D + 2], const T (&n)[D], const Free<T>& fs, S (&G)[D + 2]) {
  constexpr int NV = D + 2;
  const T g = fs.gamma, gm = g - T(1);
  const S ir = T(1) / U[0];
  S vel[D];
#pragma unroll
  for (int d = 0; d < D; ++d) vel[d] = U[1 + d] * ir;
  S ke = U[1] * vel[0];
#pragma unroll
  for (int d = 1; d < D; ++d) ke = ke + U[1 + d] * vel[d];
  const S p = gm * (U[NV - 1] - T(0.5) * ke);
  const S c = sqrt_s(g * p * ir);
  const S qn = dot_n<D>(vel, n);
  const T cinf = sqrt_s(g * fs.p / fs.rho);
  T qinf = fs.vel[0] * n[0];
#pragma unroll
  for (int d = 1; d < D; ++d) qinf += fs.vel[d] * n[d];
  const T mn = val(qn) / val(c);
  const S rp = select_s(mn > T(-1), qn + T(2) * c / gm, Lift<S, T>::of(qinf + T(2) * cinf / gm));
  const S rm = select_s(mn < T(1), Lift<S, T>::of(qinf - T(2) * cinf / gm), qn - T(2) * c / gm);
  const S qb = T(0.5) * (rp + rm);
  const S cb = T(0.25) * gm * (rp - rm);
  const bool out = val(qb) >= T(0);
  const S s_in = p / pow_s(U[0], g);
  const T s_inf = fs.p / pow_s(fs.rho, g);
  const S sb = select_s(out, s_in, Lift<S, T>::of(s_inf));
  const S rb = pow_s(cb * cb / (g * sb), T(1) / gm);
  const S pb = rb * cb * cb / g;
  S kb = Lift<S, T>::of(T(0));
  G[0] = rb;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const S vt = select_s(out, vel[d] - qn * n[d], Lift<S, T>::of(fs.vel[d] - qinf * n[d]));
    const S vb = vt + qb * n[d];
    G[1 + d] = rb * vb;
    kb = kb + vb * vb;
  }
  G[NV - 1] = pb / gm + T(0.5) * rb * kb;
}

// The far-field ghost state of ghost_farfield with the free-stream velocity as a scalar of
// type S, for derivatives with respect to the free stream (the Mach number and the flow
// angle enter the scheme only through this velocity).  Same arithmetic, operation by
// operation, as ghost_farfield.
template <int D, class S, class T>
PCEXP_DEV void ghost_farfield_v(const S (&U)[D + 2], const T (&n)[D], T g, T rho_inf, T p_inf, const S (&vinf)[3],
                                S (&G)[D + 2]) {
  constexpr int NV = D + 2;
  const T gm = g - T(1);
  const S ir = T(1) / U[0];
  S vel[D];
#pragma unroll
  for (int d = 0; d < D; ++d) vel[d] = U[1 + d] * ir;
  S ke = U[1] * vel[0];
#pragma unroll
  for (int d = 1; d < D; ++d) ke = ke + U[1 + d] * vel[d];
  const S p = gm * (U[NV - 1] - T(0.5) * ke);
  const S c = sqrt_s(g * p * ir);
  const S qn = dot_n<D>(vel, n);
  const T cinf = sqrt_s(g * p_inf / rho_inf);
  S qinf = vinf[0] * n[0];
#pragma unroll
  for (int d = 1; d < D; ++d) qinf = qinf + vinf[d] * n[d];
  const T mn = val(qn) / val(c);
  const S rp = select_s(mn > T(-1), qn + T(2) * c / gm, qinf + T(2) * cinf / gm);
  const S rm = select_s(mn < T(1), qinf - T(2) * cinf / gm, qn - T(2) * c / gm);
  const S qb = T(0.5) * (rp + rm);
  const S cb = T(0.25) * gm * (rp - rm);
  const bool out = val(qb) >= T(0);
  const S s_in = p / pow_s(U[0], g);
  const T s_inf = p_inf / pow_s(rho_inf, g);
  const S sb = select_s(out, s_in, Lift<S, T>::of(s_inf));
  const S rb = pow_s(cb * cb / (g * sb), T(1) / gm);
  const S pb = rb * cb * cb / g;
  S kb = Lift<S, T>::of(T(0));
  G[0] = rb;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const S vt = select_s(out, vel[d] - qn * n[d], vinf[d] - qinf * n[d]);
    const S vb = vt + qb * n[d];
    G[1 + d] = rb * vb;
    kb = kb + vb * vb;
  }
  G[NV - 1] = pb / gm + T(0.5) * rb * kb;
}

}  // namespace pcexp
