// DG operator kernels: the residual R(u) of Eq. euler3 (Sec. 4.2) and its
// tangent-linear J(u) v (the exact Jacobian of Eq. jac1 / jac2, applied
// matrix-free), plus the element time-step rule of Eq. x3d.
//
// Basis: a reference-triangle orthonormal basis phi^_j mapped affinely and
// scaled by |det A_e|^-1/2, so it is orthonormal on every element (the mass
// matrix is the identity, as with the paper's basis).  With x = v0 + A xi:
//   U(x_q)        = |det A|^-1/2 sum_j phi^_j(xi_q) u_j
//   volume term   = |det A|^1/2 sum_q w_q sum_d' d phi^_i/d xi_d'(xi_q) Fhat_d'
//                   with Fhat_d' = sum_d (A^-1)_{d' d} F_d(U(x_q))
//   face term     = -|det A|^-1/2 sum_q w_q |e| phi^_i(x_q) F~_n(x_q)
// Two launches per operator: a face kernel (one thread per face point)
// writes |e| w_q F~_n into the face-flux buffer G; an element kernel (a tile
// of elements per block, staged in shared memory) adds the volume term and
// lifts the face fluxes of its three edges.  Every face flux is computed once
// and every output is written once, in a fixed order (deterministic).
#include <cfloat>

#include "kernels.h"

namespace pcexp {

template <int P> struct Ord {
  static constexpr int NB = (P + 1) * (P + 2) / 2;
  static constexpr int NQ = (P + 1) * (P + 1);
  static constexpr int NFQ = P + 1;
  static constexpr int ET = (256 / NQ) > 128 ? 128 : (256 / NQ);  // elements per block
};

template <class S> struct PartOf;
template <> struct PartOf<double> { PCEXP_DEV static double get(double x) { return x; } };
template <> struct PartOf<float> { PCEXP_DEV static float get(float x) { return x; } };
template <class T> struct PartOf<Tangent<T>> { PCEXP_DEV static T get(Tangent<T> x) { return x.d; } };

// ------------------------------------------------------------------ face kernel
template <class T, int P, bool TAN>
__global__ void __launch_bounds__(256) face_kernel(DGData<T> d, const T* __restrict__ u,
                                                   const T* __restrict__ du, T* __restrict__ G,
                                                   const int* __restrict__ skip) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NFQ = O::NFQ;
  using S = typename std::conditional<TAN, Tangent<T>, T>::type;
  __shared__ T sBf[3 * NFQ * NB];
  __shared__ T sWf[NFQ];
  if (skip && *skip) return;
  for (int i = threadIdx.x; i < 3 * NFQ * NB; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < NFQ; i += blockDim.x) sWf[i] = d.Wf[i];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.F * NFQ) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = loc >> 8;
  const T nx = d.fgeo[4 * f], ny = d.fgeo[4 * f + 1], len = d.fgeo[4 * f + 2];
  S UL[4], UR[4];
  {
    const T isd = T(1) / d.geo[8 * (int64_t)eL + 4];
    const T* ue = u + (int64_t)eL * 4 * NB;
    const T* be = sBf + (fL * NFQ + q) * NB;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0, b = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        a += be[j] * ue[v * NB + j];
        if constexpr (TAN) b += be[j] * du[(int64_t)eL * 4 * NB + v * NB + j];
      }
      if constexpr (TAN) UL[v] = S{a * isd, b * isd};
      else UL[v] = a * isd;
    }
  }
  if (eR >= 0) {
    const T isd = T(1) / d.geo[8 * (int64_t)eR + 4];
    const T* ue = u + (int64_t)eR * 4 * NB;
    const T* be = sBf + (fR * NFQ + (NFQ - 1 - q)) * NB;  // R traverses the edge backwards
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0, b = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        a += be[j] * ue[v * NB + j];
        if constexpr (TAN) b += be[j] * du[(int64_t)eR * 4 * NB + v * NB + j];
      }
      if constexpr (TAN) UR[v] = S{a * isd, b * isd};
      else UR[v] = a * isd;
    }
  } else if (-eR == PCEXP_BC_SLIP_WALL) {
    ghost_slip_wall<S, T>(UL, nx, ny, UR);
  } else {
    ghost_farfield<S, T>(UL, nx, ny, d.fs, UR);
  }
  S Fn[4];
  roe_flux<S, T>(UL, UR, nx, ny, d.fs.gamma, Fn);
  const T wl = len * sWf[q];
  T* g = G + idx * 4;
#pragma unroll
  for (int v = 0; v < 4; ++v) g[v] = wl * PartOf<S>::get(Fn[v]);
}

// --------------------------------------------------------------- element kernel
template <class T, int P, bool TAN>
__global__ void __launch_bounds__(256) elem_kernel(DGData<T> d, const T* __restrict__ u,
                                                   const T* __restrict__ du, const T* __restrict__ G,
                                                   T* __restrict__ out, const T* __restrict__ escale,
                                                   const int* __restrict__ skip, const double* __restrict__ oscale) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NQ = O::NQ, NFQ = O::NFQ, ET = O::ET, NVB = 4 * NB;
  using S = typename std::conditional<TAN, Tangent<T>, T>::type;
  __shared__ T sBv[NQ * NB];
  __shared__ T sDv[2 * NQ * NB];
  __shared__ T sBf[3 * NFQ * NB];
  __shared__ T su[ET * NVB];
  __shared__ T sdu[TAN ? ET * NVB : 1];
  __shared__ T sF[ET * NQ * 8];
  __shared__ T sgeo[ET * 8];
  if (skip && *skip) return;
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)((d.E - e0) < ET ? (d.E - e0) : ET);
  for (int i = threadIdx.x; i < NQ * NB; i += blockDim.x) sBv[i] = d.Bv[i];
  for (int i = threadIdx.x; i < 2 * NQ * NB; i += blockDim.x) sDv[i] = d.Dv[i];
  for (int i = threadIdx.x; i < 3 * NFQ * NB; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < ne * NVB; i += blockDim.x) {
    su[i] = u[e0 * NVB + i];
    if constexpr (TAN) sdu[i] = du[e0 * NVB + i];
  }
  for (int i = threadIdx.x; i < ne * 8; i += blockDim.x) sgeo[i] = d.geo[e0 * 8 + i];
  __syncthreads();
  const T g = d.fs.gamma;
  const T osc = oscale ? (T)*oscale : T(1);
  // phase 1: flux at each volume point, mapped to reference directions
  for (int it = threadIdx.x; it < ne * NQ; it += blockDim.x) {
    const int el = it / NQ, q = it - el * NQ;
    const T* ge = sgeo + el * 8;
    const T isd = T(1) / ge[4];
    S U[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0, b = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        a += sBv[q * NB + j] * su[el * NVB + v * NB + j];
        if constexpr (TAN) b += sBv[q * NB + j] * sdu[el * NVB + v * NB + j];
      }
      if constexpr (TAN) U[v] = S{a * isd, b * isd};
      else U[v] = a * isd;
    }
    S Fx[4], Fy[4];
    euler_flux<S, T>(U, g, Fx, Fy);
    T* fo = sF + (el * NQ + q) * 8;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const T fx = PartOf<S>::get(Fx[v]), fy = PartOf<S>::get(Fy[v]);
      fo[v] = ge[0] * fx + ge[1] * fy;
      fo[4 + v] = ge[2] * fx + ge[3] * fy;
    }
  }
  __syncthreads();
  // phase 2: test against grad phi, lift the three face fluxes
  for (int it = threadIdx.x; it < ne * NVB; it += blockDim.x) {
    const int el = it / NVB, r = it - el * NVB;
    const int v = r / NB, i = r - v * NB;
    const T sd = sgeo[el * 8 + 4];
    T acc = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      acc += sDv[q * NB + i] * sF[(el * NQ + q) * 8 + v] + sDv[(NQ + q) * NB + i] * sF[(el * NQ + q) * 8 + 4 + v];
    acc *= sd;
    const int64_t e = e0 + el;
    T lift = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int fs = d.ef[3 * e + k];
      const int64_t face = fs >> 1;
      const T* gf = G + face * NFQ * 4;
      if (fs & 1) {
#pragma unroll
        for (int q = 0; q < NFQ; ++q) lift += sBf[(k * NFQ + (NFQ - 1 - q)) * NB + i] * gf[q * 4 + v];
      } else {
#pragma unroll
        for (int q = 0; q < NFQ; ++q) lift -= sBf[(k * NFQ + q) * NB + i] * gf[q * 4 + v];
      }
    }
    acc = (acc + lift / sd) * osc;
    if (escale) acc *= escale[e];
    out[e0 * NVB + it] = acc;
  }
}

template <class T, int P>
static cudaError_t dg_op_p(const DGData<T>& d, const T* u, const T* du, T* out, T* G, const T* escale,
                           const int* skip, const double* oscale, cudaStream_t st, const cudaEvent_t* ev) {
  using O = Ord<P>;
  const int64_t nfp = d.F * O::NFQ;
  if (ev) cudaEventRecord(ev[0], st);
  if (nfp > 0) {
    const int64_t nb = (nfp + 255) / 256;
    if (du) face_kernel<T, P, true><<<(unsigned)nb, 256, 0, st>>>(d, u, du, G, skip);
    else face_kernel<T, P, false><<<(unsigned)nb, 256, 0, st>>>(d, u, du, G, skip);
  }
  if (ev) cudaEventRecord(ev[1], st);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  if (du) elem_kernel<T, P, true><<<(unsigned)eb, 256, 0, st>>>(d, u, du, G, out, escale, skip, oscale);
  else elem_kernel<T, P, false><<<(unsigned)eb, 256, 0, st>>>(d, u, du, G, out, escale, skip, oscale);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_dg_operator(const DGData<T>& d, const T* u, const T* du, T* out, T* G, const T* escale,
                               const int* skip, cudaStream_t st, const cudaEvent_t* ev, const double* oscale) {
  switch (d.p) {
    case 0: return dg_op_p<T, 0>(d, u, du, out, G, escale, skip, oscale, st, ev);
    case 1: return dg_op_p<T, 1>(d, u, du, out, G, escale, skip, oscale, st, ev);
    case 2: return dg_op_p<T, 2>(d, u, du, out, G, escale, skip, oscale, st, ev);
    case 3: return dg_op_p<T, 3>(d, u, du, out, G, escale, skip, oscale, st, ev);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------- point Jacobians (linearisation)
// The exact Jacobian of the scheme (Eq. jac1, jac2) is assembled point by point: the
// volume flux Jacobians dF_d/dU and the Riemann-flux Jacobians dF~/dU_L, dF~/dU_R are
// evaluated exactly by running the flux code on Jet<T,4> numbers seeded with unit
// directions (the paper obtains the Riemann-flux Jacobians by AD as well).  Every J v
// of a PCEXP step is taken at u_n, so the Jacobians are built once per step and each
// of the 2m+1 products reduces to traces, 4x4 mat-vecs and the test/lift contractions.
template <class T, int P>
__global__ void __launch_bounds__(256) linearize_vol_kernel(DGData<T> d, const T* __restrict__ u,
                                                            T* __restrict__ Avol) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NQ = O::NQ;
  using J4 = Jet<T, 4>;
  const int64_t n = d.E * NQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t e = idx / NQ;
  const int q = (int)(idx - e * NQ);
  const T* ge = d.geo + 8 * e;
  const T isd = T(1) / ge[4];
  J4 U[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    T a = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) a += d.Bv[q * NB + j] * u[e * 4 * NB + v * NB + j];
    U[v].v = a * isd;
#pragma unroll
    for (int c = 0; c < 4; ++c) U[v].d[c] = (v == c) ? T(1) : T(0);
  }
  J4 Fx[4], Fy[4];
  euler_flux<J4, T>(U, d.fs.gamma, Fx, Fy);
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Avol[(int64_t)(0 * 16 + v * 4 + c) * n + idx] = ge[0] * Fx[v].d[c] + ge[1] * Fy[v].d[c];
      Avol[(int64_t)(1 * 16 + v * 4 + c) * n + idx] = ge[2] * Fx[v].d[c] + ge[3] * Fy[v].d[c];
    }
}

template <class T, int P>
__global__ void __launch_bounds__(128) linearize_face_kernel(DGData<T> d, const T* __restrict__ u,
                                                             T* __restrict__ Bface) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NFQ = O::NFQ;
  using J4 = Jet<T, 4>;
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = loc >> 8;
  const T nx = d.fgeo[4 * f], ny = d.fgeo[4 * f + 1], len = d.fgeo[4 * f + 2];
  const T wq = len * d.Wf[q];
  T uL[4], uR[4];
  const T isdL = T(1) / d.geo[8 * (int64_t)eL + 4];
  T isdR = T(0);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    T a = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) a += d.Bf[(fL * NFQ + q) * NB + j] * u[(int64_t)eL * 4 * NB + v * NB + j];
    uL[v] = a * isdL;
  }
  if (eR >= 0) {
    isdR = T(1) / d.geo[8 * (int64_t)eR + 4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j)
        a += d.Bf[(fR * NFQ + (NFQ - 1 - q)) * NB + j] * u[(int64_t)eR * 4 * NB + v * NB + j];
      uR[v] = a * isdR;
    }
  }
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    J4 L[4], R[4], F[4];
    if (side == 1 && eR < 0) {
#pragma unroll
      for (int k = 0; k < 16; ++k) Bface[(int64_t)(16 + k) * n + idx] = T(0);
      break;
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      L[v].v = uL[v];
#pragma unroll
      for (int c = 0; c < 4; ++c) L[v].d[c] = (side == 0 && v == c) ? T(1) : T(0);
    }
    if (eR >= 0) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        R[v].v = uR[v];
#pragma unroll
        for (int c = 0; c < 4; ++c) R[v].d[c] = (side == 1 && v == c) ? T(1) : T(0);
      }
    } else if (-eR == PCEXP_BC_SLIP_WALL) {
      ghost_slip_wall<J4, T>(L, nx, ny, R);
    } else {
      ghost_farfield<J4, T>(L, nx, ny, d.fs, R);
    }
    roe_flux<J4, T>(L, R, nx, ny, d.fs.gamma, F);
    const T sc = wq * (side == 0 ? isdL : isdR);
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int c = 0; c < 4; ++c) Bface[(int64_t)(side * 16 + v * 4 + c) * n + idx] = sc * F[v].d[c];
  }
}

template <class T, int P>
__global__ void __launch_bounds__(256) face_apply_kernel(DGData<T> d, const T* __restrict__ Bface,
                                                         const T* __restrict__ dv, T* __restrict__ G,
                                                         const int* __restrict__ skip) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NFQ = O::NFQ;
  __shared__ T sBf[3 * NFQ * NB];
  if (skip && *skip) return;
  for (int i = threadIdx.x; i < 3 * NFQ * NB; i += blockDim.x) sBf[i] = d.Bf[i];
  __syncthreads();
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = loc >> 8;
  T B[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) B[k] = (k < 16 || eR >= 0) ? Bface[(int64_t)k * n + idx] : T(0);
  T tL[4], tR[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    T a = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) a += sBf[(fL * NFQ + q) * NB + j] * dv[(int64_t)eL * 4 * NB + v * NB + j];
    tL[v] = a;
  }
  if (eR >= 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j)
        a += sBf[(fR * NFQ + (NFQ - 1 - q)) * NB + j] * dv[(int64_t)eR * 4 * NB + v * NB + j];
      tR[v] = a;
    }
  }
  T* g = G + idx * 4;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    T a = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) a += B[v * 4 + c] * tL[c];
    if (eR >= 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) a += B[16 + v * 4 + c] * tR[c];
    }
    g[v] = a;
  }
}

template <class T, int P>
__global__ void __launch_bounds__(256) elem_apply_kernel(DGData<T> d, const T* __restrict__ Avol,
                                                         const T* __restrict__ dv, const T* __restrict__ G,
                                                         T* __restrict__ out, const T* __restrict__ escale,
                                                         const int* __restrict__ skip,
                                                         const double* __restrict__ oscale) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NQ = O::NQ, NFQ = O::NFQ, ET = O::ET, NVB = 4 * NB;
  __shared__ T sBv[NQ * NB];
  __shared__ T sDv[2 * NQ * NB];
  __shared__ T sBf[3 * NFQ * NB];
  __shared__ T sdu[ET * NVB];
  __shared__ T sF[ET * NQ * 8];
  __shared__ T ssd[ET];
  static_assert(ET * NQ <= 256, "one volume point per thread");
  if (skip && *skip) return;
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)((d.E - e0) < ET ? (d.E - e0) : ET);
  const int64_t n = d.E * NQ;
  // issue this thread's point-Jacobian loads first, so they are in flight while the
  // block stages its tile of dv in shared memory
  const int el1 = threadIdx.x / NQ, q1 = threadIdx.x - (threadIdx.x / NQ) * NQ;
  const bool has_pt = threadIdx.x < ne * NQ;
  const int64_t pidx = (e0 + el1) * NQ + q1;
  T A[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) A[k] = has_pt ? Avol[(int64_t)k * n + pidx] : T(0);
  for (int i = threadIdx.x; i < NQ * NB; i += blockDim.x) sBv[i] = d.Bv[i];
  for (int i = threadIdx.x; i < 2 * NQ * NB; i += blockDim.x) sDv[i] = d.Dv[i];
  for (int i = threadIdx.x; i < 3 * NFQ * NB; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < ne * NVB; i += blockDim.x) sdu[i] = dv[e0 * NVB + i];
  for (int i = threadIdx.x; i < ne; i += blockDim.x) ssd[i] = d.geo[(e0 + i) * 8 + 4];
  __syncthreads();
  const T osc = oscale ? (T)*oscale : T(1);
  // phase 1: trace of dv at this thread's volume point, times the mapped flux Jacobians
  if (has_pt) {
    T t[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) a += sBv[q1 * NB + j] * sdu[el1 * NVB + v * NB + j];
      t[v] = a;
    }
    T* fo = sF + (el1 * NQ + q1) * 8;
#pragma unroll
    for (int dd = 0; dd < 2; ++dd)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        T a = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) a += A[dd * 16 + v * 4 + c] * t[c];
        fo[dd * 4 + v] = a;
      }
  }
  __syncthreads();
  // phase 2: test against grad phi (the sqrt(det) factors cancel), lift the face terms
  for (int it = threadIdx.x; it < ne * NVB; it += blockDim.x) {
    const int el = it / NVB, r = it - el * NVB;
    const int v = r / NB, i = r - v * NB;
    T acc = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      acc += sDv[q * NB + i] * sF[(el * NQ + q) * 8 + v] + sDv[(NQ + q) * NB + i] * sF[(el * NQ + q) * 8 + 4 + v];
    const int64_t e = e0 + el;
    T lift = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int fs = d.ef[3 * e + k];
      const int64_t face = fs >> 1;
      const T* gf = G + face * NFQ * 4;
      if (fs & 1) {
#pragma unroll
        for (int q = 0; q < NFQ; ++q) lift += sBf[(k * NFQ + (NFQ - 1 - q)) * NB + i] * gf[q * 4 + v];
      } else {
#pragma unroll
        for (int q = 0; q < NFQ; ++q) lift -= sBf[(k * NFQ + q) * NB + i] * gf[q * 4 + v];
      }
    }
    acc = (acc + lift / ssd[el]) * osc;
    if (escale) acc *= escale[e];
    out[e0 * NVB + it] = acc;
  }
}

template <class T, int P>
static cudaError_t linearize_p(const DGData<T>& d, const T* u, LinData<T> lin, cudaStream_t st) {
  using O = Ord<P>;
  const int64_t nv = d.E * O::NQ, nf = d.F * O::NFQ;
  linearize_vol_kernel<T, P><<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(d, u, lin.Avol);
  if (nf > 0) linearize_face_kernel<T, P><<<(unsigned)((nf + 127) / 128), 128, 0, st>>>(d, u, lin.Bface);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_linearize(const DGData<T>& d, const T* u, LinData<T> lin, cudaStream_t st) {
  switch (d.p) {
    case 0: return linearize_p<T, 0>(d, u, lin, st);
    case 1: return linearize_p<T, 1>(d, u, lin, st);
    case 2: return linearize_p<T, 2>(d, u, lin, st);
    case 3: return linearize_p<T, 3>(d, u, lin, st);
  }
  return cudaErrorInvalidValue;
}

template <class T, int P>
static cudaError_t jac_apply_p(const DGData<T>& d, LinData<T> lin, const T* dv, T* out, T* G, const T* escale,
                               const int* skip, const double* oscale, cudaStream_t st, const cudaEvent_t* ev) {
  using O = Ord<P>;
  const int64_t nf = d.F * O::NFQ;
  if (ev) cudaEventRecord(ev[0], st);
  if (nf > 0) face_apply_kernel<T, P><<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(d, lin.Bface, dv, G, skip);
  if (ev) cudaEventRecord(ev[1], st);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  elem_apply_kernel<T, P><<<(unsigned)eb, 256, 0, st>>>(d, lin.Avol, dv, G, out, escale, skip, oscale);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_jac_apply(const DGData<T>& d, LinData<T> lin, const T* dv, T* out, T* G, const T* escale,
                             const int* skip, const double* oscale, cudaStream_t st, const cudaEvent_t* ev) {
  switch (d.p) {
    case 0: return jac_apply_p<T, 0>(d, lin, dv, out, G, escale, skip, oscale, st, ev);
    case 1: return jac_apply_p<T, 1>(d, lin, dv, out, G, escale, skip, oscale, st, ev);
    case 2: return jac_apply_p<T, 2>(d, lin, dv, out, G, escale, skip, oscale, st, ev);
    case 3: return jac_apply_p<T, 3>(d, lin, dv, out, G, escale, skip, oscale, st, ev);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------- adjoint J^T w
// Transpose of the point-Jacobian J v (same linearisation state).  With the output
// factors of J v folded into w (w~ = osc * escale_e * w), the face kernel forms the
// adjoint of the lifted face flux at every face point,
//   Gbar = -(1/sd_L) sum_i Bf_L[i] w~_L[i] + (1/sd_R) sum_i Bf_R[i] w~_R[i],
// and stores B_L^T Gbar and B_R^T Gbar; the element kernel applies the transposed
// volume Jacobians to the transposed test of w~ and gathers the transposed traces
// of its three faces.  Deterministic (no atomics).
template <class T, int P>
__global__ void __launch_bounds__(256) face_adjoint_kernel(DGData<T> d, const T* __restrict__ Bface,
                                                           const T* __restrict__ w, T* __restrict__ GT,
                                                           const T* __restrict__ escale, T osc) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NFQ = O::NFQ;
  __shared__ T sBf[3 * NFQ * NB];
  for (int i = threadIdx.x; i < 3 * NFQ * NB; i += blockDim.x) sBf[i] = d.Bf[i];
  __syncthreads();
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = loc >> 8;
  T gb[4];
  {
    const T sc = -osc * (escale ? escale[eL] : T(1)) / d.geo[8 * (int64_t)eL + 4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0;
#pragma unroll
      for (int i = 0; i < NB; ++i) a += sBf[(fL * NFQ + q) * NB + i] * w[(int64_t)eL * 4 * NB + v * NB + i];
      gb[v] = sc * a;
    }
  }
  if (eR >= 0) {
    const T sc = osc * (escale ? escale[eR] : T(1)) / d.geo[8 * (int64_t)eR + 4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T a = 0;
#pragma unroll
      for (int i = 0; i < NB; ++i)
        a += sBf[(fR * NFQ + (NFQ - 1 - q)) * NB + i] * w[(int64_t)eR * 4 * NB + v * NB + i];
      gb[v] += sc * a;
    }
  }
  T* o = GT + idx * 8;
#pragma unroll
  for (int side = 0; side < 2; ++side)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T a = 0;
      if (side == 0 || eR >= 0) {
#pragma unroll
        for (int v = 0; v < 4; ++v) a += Bface[(int64_t)(side * 16 + v * 4 + c) * n + idx] * gb[v];
      }
      o[side * 4 + c] = a;
    }
}

template <class T, int P>
__global__ void __launch_bounds__(256) elem_adjoint_kernel(DGData<T> d, const T* __restrict__ Avol,
                                                           const T* __restrict__ w, const T* __restrict__ GT,
                                                           T* __restrict__ out, const T* __restrict__ escale,
                                                           T osc) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NQ = O::NQ, NFQ = O::NFQ, ET = O::ET, NVB = 4 * NB;
  __shared__ T sBv[NQ * NB];
  __shared__ T sDv[2 * NQ * NB];
  __shared__ T sBf[3 * NFQ * NB];
  __shared__ T sw[ET * NVB];
  __shared__ T sU[ET * NQ * 4];
  static_assert(ET * NQ <= 256, "one volume point per thread");
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)((d.E - e0) < ET ? (d.E - e0) : ET);
  const int64_t n = d.E * NQ;
  for (int i = threadIdx.x; i < NQ * NB; i += blockDim.x) sBv[i] = d.Bv[i];
  for (int i = threadIdx.x; i < 2 * NQ * NB; i += blockDim.x) sDv[i] = d.Dv[i];
  for (int i = threadIdx.x; i < 3 * NFQ * NB; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < ne * NVB; i += blockDim.x)
    sw[i] = w[e0 * NVB + i] * osc * (escale ? escale[e0 + i / NVB] : T(1));
  __syncthreads();
  // phase 1: transposed test, then transposed volume Jacobians, at this thread's point
  const int el1 = threadIdx.x / NQ, q1 = threadIdx.x - (threadIdx.x / NQ) * NQ;
  if (threadIdx.x < ne * NQ) {
    const int64_t pidx = (e0 + el1) * NQ + q1;
    T fb[8];
#pragma unroll
    for (int dd = 0; dd < 2; ++dd)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        T a = 0;
#pragma unroll
        for (int i = 0; i < NB; ++i) a += sDv[(dd * NQ + q1) * NB + i] * sw[el1 * NVB + v * NB + i];
        fb[dd * 4 + v] = a;
      }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T a = 0;
#pragma unroll
      for (int dd = 0; dd < 2; ++dd)
#pragma unroll
        for (int v = 0; v < 4; ++v) a += Avol[(int64_t)(dd * 16 + v * 4 + c) * n + pidx] * fb[dd * 4 + v];
      sU[(el1 * NQ + q1) * 4 + c] = a;
    }
  }
  __syncthreads();
  // phase 2: transposed volume traces plus the transposed face traces of the 3 faces
  for (int it = threadIdx.x; it < ne * NVB; it += blockDim.x) {
    const int el = it / NVB, r = it - el * NVB;
    const int c = r / NB, j = r - c * NB;
    T acc = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc += sBv[q * NB + j] * sU[(el * NQ + q) * 4 + c];
    const int64_t e = e0 + el;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int fs = d.ef[3 * e + k];
      const int64_t face = fs >> 1;
      const int side = fs & 1;
      const T* gt = GT + face * NFQ * 8 + side * 4 + c;
#pragma unroll
      for (int q = 0; q < NFQ; ++q) {
        const int qq = side ? (NFQ - 1 - q) : q;
        acc += sBf[(k * NFQ + qq) * NB + j] * gt[q * 8];
      }
    }
    out[e0 * NVB + it] = acc;
  }
}

template <class T, int P>
static cudaError_t jac_adjoint_p(const DGData<T>& d, LinData<T> lin, const T* w, T* out, T* GT, const T* escale,
                                 T osc, cudaStream_t st) {
  using O = Ord<P>;
  const int64_t nf = d.F * O::NFQ;
  if (nf > 0) face_adjoint_kernel<T, P><<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(d, lin.Bface, w, GT, escale, osc);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  elem_adjoint_kernel<T, P><<<(unsigned)eb, 256, 0, st>>>(d, lin.Avol, w, GT, out, escale, osc);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_jac_adjoint(const DGData<T>& d, LinData<T> lin, const T* w, T* out, T* GT, const T* escale, T osc,
                               cudaStream_t st) {
  switch (d.p) {
    case 0: return jac_adjoint_p<T, 0>(d, lin, w, out, GT, escale, osc, st);
    case 1: return jac_adjoint_p<T, 1>(d, lin, w, out, GT, escale, osc, st);
    case 2: return jac_adjoint_p<T, 2>(d, lin, w, out, GT, escale, osc, st);
    case 3: return jac_adjoint_p<T, 3>(d, lin, w, out, GT, escale, osc, st);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------- second-order adjoint (d(J(u) v)/du)^T w
// S(u) = w~^T J(u) v is differentiated with respect to the linearisation state u:
// every flux is evaluated on hyper-dual numbers (value, 4 seeded partials, the
// directional derivative along the traces of v, its 4 partials), contracted with the
// transposed test (volume) or transposed lift (faces) of w~ and mapped back through the
// transposed traces.  Same output factors and scratch layout as the adjoint kernels.
template <class T, int P>
__global__ void __launch_bounds__(128) face_hess_kernel(DGData<T> d, const T* __restrict__ u,
                                                        const T* __restrict__ v, const T* __restrict__ w,
                                                        T* __restrict__ GT, const T* __restrict__ escale, T osc) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NFQ = O::NFQ;
  using H = HD4<T>;
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = loc >> 8;
  const T nx = d.fgeo[4 * f], ny = d.fgeo[4 * f + 1], len = d.fgeo[4 * f + 2];
  const T wq = len * d.Wf[q];
  const T sdL = d.geo[8 * (int64_t)eL + 4];
  const T sdR = eR >= 0 ? d.geo[8 * (int64_t)eR + 4] : T(1);
  const T* bL = d.Bf + (fL * NFQ + q) * NB;
  const T* bR = d.Bf + (fR * NFQ + (NFQ - 1 - q)) * NB;
  T uL[4], tL[4], uR[4], tR[4], gb[4];
  const T scL = -osc * (escale ? escale[eL] : T(1)) / sdL;
  const T scR = osc * (eR >= 0 && escale ? escale[eR] : T(1)) / sdR;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    T a = 0, b = 0, g = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int64_t o = (int64_t)eL * 4 * NB + c * NB + j;
      a += bL[j] * u[o];
      b += bL[j] * v[o];
      g += bL[j] * w[o];
    }
    uL[c] = a / sdL;
    tL[c] = b / sdL;
    gb[c] = scL * g;
    uR[c] = tR[c] = T(0);
  }
  if (eR >= 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T a = 0, b = 0, g = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int64_t o = (int64_t)eR * 4 * NB + c * NB + j;
        a += bR[j] * u[o];
        b += bR[j] * v[o];
        g += bR[j] * w[o];
      }
      uR[c] = a / sdR;
      tR[c] = b / sdR;
      gb[c] += scR * g;
    }
  }
  T* o = GT + idx * 8;
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    if (side == 1 && eR < 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) o[4 + c] = T(0);
      break;
    }
    H L[4], R[4], F[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      L[c].v = uL[c];
      L[c].t = tL[c];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        L[c].d[k] = (side == 0 && k == c) ? T(1) : T(0);
        L[c].dt[k] = T(0);
      }
    }
    if (eR >= 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        R[c].v = uR[c];
        R[c].t = tR[c];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          R[c].d[k] = (side == 1 && k == c) ? T(1) : T(0);
          R[c].dt[k] = T(0);
        }
      }
    } else if (-eR == PCEXP_BC_SLIP_WALL) {
      ghost_slip_wall<H, T>(L, nx, ny, R);
    } else {
      ghost_farfield<H, T>(L, nx, ny, d.fs, R);
    }
    roe_flux<H, T>(L, R, nx, ny, d.fs.gamma, F);
    const T sc = wq / (side == 0 ? sdL : sdR);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T a = 0;
#pragma unroll
      for (int vv = 0; vv < 4; ++vv) a += gb[vv] * F[vv].dt[c];
      o[side * 4 + c] = sc * a;
    }
  }
}

template <class T, int P>
__global__ void __launch_bounds__(256) elem_hess_kernel(DGData<T> d, const T* __restrict__ u, const T* __restrict__ v,
                                                        const T* __restrict__ w, const T* __restrict__ GT,
                                                        T* __restrict__ out, const T* __restrict__ escale, T osc) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NQ = O::NQ, NFQ = O::NFQ, ET = O::ET, NVB = 4 * NB;
  using H = HD4<T>;
  __shared__ T sBv[NQ * NB];
  __shared__ T sDv[2 * NQ * NB];
  __shared__ T sBf[3 * NFQ * NB];
  __shared__ T su[ET * NVB];
  __shared__ T sv[ET * NVB];
  __shared__ T sw[ET * NVB];
  __shared__ T sU[ET * NQ * 4];
  __shared__ T sgeo[ET * 8];
  static_assert(ET * NQ <= 256, "one volume point per thread");
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)((d.E - e0) < ET ? (d.E - e0) : ET);
  for (int i = threadIdx.x; i < NQ * NB; i += blockDim.x) sBv[i] = d.Bv[i];
  for (int i = threadIdx.x; i < 2 * NQ * NB; i += blockDim.x) sDv[i] = d.Dv[i];
  for (int i = threadIdx.x; i < 3 * NFQ * NB; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < ne * NVB; i += blockDim.x) {
    su[i] = u[e0 * NVB + i];
    sv[i] = v[e0 * NVB + i];
    sw[i] = w[e0 * NVB + i] * osc * (escale ? escale[e0 + i / NVB] : T(1));
  }
  for (int i = threadIdx.x; i < ne * 8; i += blockDim.x) sgeo[i] = d.geo[e0 * 8 + i];
  __syncthreads();
  const int el1 = threadIdx.x / NQ, q1 = threadIdx.x - (threadIdx.x / NQ) * NQ;
  if (threadIdx.x < ne * NQ) {
    const T* ge = sgeo + el1 * 8;
    const T sd = ge[4];
    H U[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T a = 0, b = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        a += sBv[q1 * NB + j] * su[el1 * NVB + c * NB + j];
        b += sBv[q1 * NB + j] * sv[el1 * NVB + c * NB + j];
      }
      U[c].v = a / sd;
      U[c].t = b;  // the sqrt(det) factors of trace and test cancel
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        U[c].d[k] = (k == c) ? T(1) : T(0);
        U[c].dt[k] = T(0);
      }
    }
    H Fx[4], Fy[4];
    euler_flux<H, T>(U, d.fs.gamma, Fx, Fy);
    T fb[8];
#pragma unroll
    for (int dd = 0; dd < 2; ++dd)
#pragma unroll
      for (int vv = 0; vv < 4; ++vv) {
        T a = 0;
#pragma unroll
        for (int i = 0; i < NB; ++i) a += sDv[(dd * NQ + q1) * NB + i] * sw[el1 * NVB + vv * NB + i];
        fb[dd * 4 + vv] = a;
      }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      T a = 0;
#pragma unroll
      for (int vv = 0; vv < 4; ++vv) {
        const T f0 = ge[0] * Fx[vv].dt[c] + ge[1] * Fy[vv].dt[c];
        const T f1 = ge[2] * Fx[vv].dt[c] + ge[3] * Fy[vv].dt[c];
        a += fb[vv] * f0 + fb[4 + vv] * f1;
      }
      sU[(el1 * NQ + q1) * 4 + c] = a / sd;
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < ne * NVB; it += blockDim.x) {
    const int el = it / NVB, r = it - el * NVB;
    const int c = r / NB, j = r - c * NB;
    T acc = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc += sBv[q * NB + j] * sU[(el * NQ + q) * 4 + c];
    const int64_t e = e0 + el;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int fs = d.ef[3 * e + k];
      const int64_t face = fs >> 1;
      const int side = fs & 1;
      const T* gt = GT + face * NFQ * 8 + side * 4 + c;
#pragma unroll
      for (int q = 0; q < NFQ; ++q) {
        const int qq = side ? (NFQ - 1 - q) : q;
        acc += sBf[(k * NFQ + qq) * NB + j] * gt[q * 8];
      }
    }
    out[e0 * NVB + it] = acc;
  }
}

template <class T, int P>
static cudaError_t jvp_state_adjoint_p(const DGData<T>& d, const T* u, const T* v, const T* w, T* out, T* GT,
                                       const T* escale, T osc, cudaStream_t st) {
  using O = Ord<P>;
  const int64_t nf = d.F * O::NFQ;
  if (nf > 0) face_hess_kernel<T, P><<<(unsigned)((nf + 127) / 128), 128, 0, st>>>(d, u, v, w, GT, escale, osc);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  elem_hess_kernel<T, P><<<(unsigned)eb, 256, 0, st>>>(d, u, v, w, GT, out, escale, osc);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_jvp_state_adjoint(const DGData<T>& d, const T* u, const T* v, const T* w, T* out, T* GT,
                                     const T* escale, T osc, cudaStream_t st) {
  switch (d.p) {
    case 0: return jvp_state_adjoint_p<T, 0>(d, u, v, w, out, GT, escale, osc, st);
    case 1: return jvp_state_adjoint_p<T, 1>(d, u, v, w, out, GT, escale, osc, st);
    case 2: return jvp_state_adjoint_p<T, 2>(d, u, v, w, out, GT, escale, osc, st);
    case 3: return jvp_state_adjoint_p<T, 3>(d, u, v, w, out, GT, escale, osc, st);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ output functional
// Pressure force on the slip walls along the unit direction (ax, ay):
//   J = sum_{wall faces} sum_q |e| w_q p(U_L(x_q)) (n . a),  p = (gamma-1)(E - |m|^2 / (2 rho)),
// with its gradient dJ/du (trace transpose of dp/dU); value by a fixed-order reduction.
template <class T, int P>
__global__ void __launch_bounds__(256) wall_force_kernel(DGData<T> d, int64_t f0, const T* __restrict__ u, double ax,
                                                         double ay, double* __restrict__ grad, double* __restrict__ value,
                                                         double* __restrict__ partials, unsigned* counter) {
  using O = Ord<P>;
  constexpr int NB = O::NB, NFQ = O::NFQ;
  __shared__ double red[8];
  __shared__ bool last;
  double acc = 0;
  const T gm = d.fs.gamma - T(1);
  for (int64_t f = f0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < d.F; f += (int64_t)gridDim.x * blockDim.x) {
    if (-d.fel[2 * f + 1] != PCEXP_BC_SLIP_WALL) continue;
    const int e = d.fel[2 * f];
    const int fl = d.floc[f] & 0xff;
    const double nx = (double)d.fgeo[4 * f], ny = (double)d.fgeo[4 * f + 1], len = (double)d.fgeo[4 * f + 2];
    const double na = nx * ax + ny * ay;
    const double isd = 1.0 / (double)d.geo[8 * (int64_t)e + 4];
    double g[4 * NB];
    for (int k = 0; k < 4 * NB; ++k) g[k] = 0.0;
    for (int q = 0; q < NFQ; ++q) {
      const T* b = d.Bf + (fl * NFQ + q) * NB;
      double U[4];
      for (int c = 0; c < 4; ++c) {
        double a = 0;
        for (int j = 0; j < NB; ++j) a += (double)b[j] * (double)u[(int64_t)e * 4 * NB + c * NB + j];
        U[c] = a * isd;
      }
      const double ux = U[1] / U[0], uy = U[2] / U[0];
      const double p = (double)gm * (U[3] - 0.5 * U[0] * (ux * ux + uy * uy));
      const double wq = len * (double)d.Wf[q] * na;
      acc += wq * p;
      const double dp[4] = {(double)gm * 0.5 * (ux * ux + uy * uy), -(double)gm * ux, -(double)gm * uy, (double)gm};
      for (int c = 0; c < 4; ++c)
        for (int j = 0; j < NB; ++j) g[c * NB + j] += wq * dp[c] * (double)b[j] * isd;
    }
    // at most two wall faces per element on the supported meshes; a + b is exact in either order
    if (grad)
      for (int k = 0; k < 4 * NB; ++k) atomicAdd(grad + (int64_t)e * 4 * NB + k, g[k]);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
    partials[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    double b = 0;
    for (unsigned i = 0; i < gridDim.x; ++i) b += __ldcg(partials + i);
    *value = b;
    *counter = 0;
  }
}

template <class T>
cudaError_t launch_wall_force(const DGData<T>& d, int64_t f0, const T* u, double ax, double ay, double* grad,
                              double* value, double* partials, unsigned* counter, cudaStream_t st) {
  const int64_t nb = d.F - f0;
  unsigned g = (unsigned)((nb + 255) / 256);
  if (g < 1) g = 1;
  if (g > RED_BLOCKS) g = RED_BLOCKS;
  switch (d.p) {
    case 0: wall_force_kernel<T, 0><<<g, 256, 0, st>>>(d, f0, u, ax, ay, grad, value, partials, counter); break;
    case 1: wall_force_kernel<T, 1><<<g, 256, 0, st>>>(d, f0, u, ax, ay, grad, value, partials, counter); break;
    case 2: wall_force_kernel<T, 2><<<g, 256, 0, st>>>(d, f0, u, ax, ay, grad, value, partials, counter); break;
    case 3: wall_force_kernel<T, 3><<<g, 256, 0, st>>>(d, f0, u, ax, ay, grad, value, partials, counter); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ time step
// dt_e = CFL h_e / ((2p+1)(|v| + c)) with v, c at the element centroid (Eq. x3d).
template <class T, int P>
__global__ void __launch_bounds__(256) local_dt_kernel(DGData<T> d, const T* __restrict__ u,
                                                       const double* cfl_dev, double cfl_host,
                                                       T* __restrict__ dte, double* __restrict__ dtmin,
                                                       double* __restrict__ partials,
                                                       unsigned* __restrict__ counter) {
  constexpr int NB = Ord<P>::NB;
  __shared__ double red[8];
  __shared__ bool last;
  const double cfl = cfl_dev ? *cfl_dev : cfl_host;
  double mn = DBL_MAX;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.E; e += (int64_t)gridDim.x * blockDim.x) {
    const T isd = T(1) / d.geo[8 * e + 4];
    double U[4];
    for (int v = 0; v < 4; ++v) {
      T a = 0;
      for (int j = 0; j < NB; ++j) a += d.Bc[j] * u[e * 4 * NB + v * NB + j];
      U[v] = (double)(a * isd);
    }
    const double gam = (double)d.fs.gamma;
    const double ux = U[1] / U[0], uy = U[2] / U[0];
    const double p = (gam - 1.0) * (U[3] - 0.5 * U[0] * (ux * ux + uy * uy));
    const double c = sqrt(gam * p / U[0]);
    const double h = (double)d.geo[8 * e + 5];
    const double dt = cfl * h / ((2 * d.p + 1) * (sqrt(ux * ux + uy * uy) + c));
    if (dte) dte[e] = (T)dt;
    mn = fmin(mn, dt);
  }
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmin(b, red[w]);
    partials[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    double b = DBL_MAX;
    for (unsigned i = 0; i < gridDim.x; ++i) b = fmin(b, __ldcg(partials + i));
    *dtmin = b;
    *counter = 0;
  }
}

template <class T>
cudaError_t launch_local_dt(const DGData<T>& d, const T* u, const double* cfl_dev, double cfl, T* dte,
                            double* dtmin, double* partials, unsigned* counter, cudaStream_t st) {
  int64_t nb = (d.E + 255) / 256;
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  switch (d.p) {
    case 0: local_dt_kernel<T, 0><<<(unsigned)nb, 256, 0, st>>>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter); break;
    case 1: local_dt_kernel<T, 1><<<(unsigned)nb, 256, 0, st>>>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter); break;
    case 2: local_dt_kernel<T, 2><<<(unsigned)nb, 256, 0, st>>>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter); break;
    case 3: local_dt_kernel<T, 3><<<(unsigned)nb, 256, 0, st>>>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ basis conversion
template <class T>
__global__ void paper_to_internal_kernel(const double* __restrict__ src, T* __restrict__ dst,
                                         const double* __restrict__ Q, int64_t E, int nb, int nv) {
  const int64_t n = E * nv * nb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / (nv * nb);
    const int r = (int)(idx - e * nv * nb), v = r / nb, j = r - v * nb;
    const double* q = Q + e * nb * nb;
    const double* s = src + e * nv * nb + v * nb;
    double a = 0;
    for (int i = 0; i < nb; ++i) a += q[i * nb + j] * s[i];
    dst[idx] = (T)a;
  }
}

template <class T>
__global__ void internal_to_paper_kernel(const T* __restrict__ src, double* __restrict__ dst,
                                         const double* __restrict__ Q, int64_t E, int nb, int nv) {
  const int64_t n = E * nv * nb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / (nv * nb);
    const int r = (int)(idx - e * nv * nb), v = r / nb, i = r - v * nb;
    const double* q = Q + e * nb * nb + i * nb;
    const T* s = src + e * nv * nb + v * nb;
    double a = 0;
    for (int j = 0; j < nb; ++j) a += q[j] * (double)s[j];
    dst[idx] = a;
  }
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

template <class T>
cudaError_t launch_paper_to_internal(const double* src, T* dst, const double* Q, int64_t E, int nb, int nv, cudaStream_t st) {
  paper_to_internal_kernel<T><<<grid_for(E * nb * nv), 256, 0, st>>>(src, dst, Q, E, nb, nv);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_internal_to_paper(const T* src, double* dst, const double* Q, int64_t E, int nb, int nv, cudaStream_t st) {
  internal_to_paper_kernel<T><<<grid_for(E * nb * nv), 256, 0, st>>>(src, dst, Q, E, nb, nv);
  return cudaGetLastError();
}

template <class T>
__global__ void scale_elements_kernel(T* __restrict__ x, const T* __restrict__ s, int64_t E, int nvb) {
  const int64_t n = E * nvb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x)
    x[idx] *= s[idx / nvb];
}
template <class T>
cudaError_t launch_scale_elements(T* x, const T* s, int64_t E, int nvb, cudaStream_t st) {
  scale_elements_kernel<T><<<grid_for(E * nvb), 256, 0, st>>>(x, s, E, nvb);
  return cudaGetLastError();
}

// Density residual norm of Eq. cfl with the orthonormal basis:
// (1/|Omega|) sqrt(sum_e sum_i (R[e][0][i] / s_e)^2); then CFL(n) of Eq. cfl.
template <class T>
__global__ void __launch_bounds__(256) density_norm_kernel(const T* __restrict__ R, const T* __restrict__ s,
                                                           int64_t E, int nb, int nv, double volume,
                                                           StepState* ss, double* __restrict__ partials,
                                                           int ramp_n, int p, double cfl_max) {
  __shared__ double red[8];
  __shared__ bool last;
  double acc = 0;
  const int64_t n = E * nb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / nb;
    const int i = (int)(idx - e * nb);
    double r = (double)R[e * nv * nb + i];
    if (s) r /= (double)s[e];
    acc += r * r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
    partials[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(&ss->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    double b = 0;
    for (unsigned i = 0; i < gridDim.x; ++i) b += __ldcg(partials + i);
    const double rn = sqrt(b) / volume;
    ss->res_norm = rn;
    if (!isfinite(rn)) ss->err = 1;
    if (ramp_n > 0) {
      const double a = rn > 0 ? 1.0 / (rn * rn * rn) : DBL_MAX;
      const double b2 = 1.0 + (double)(ramp_n - 1) / (2 * p + 1);
      ss->cfl = fmin(cfl_max, fmax(a, b2));
    }
    ss->counter = 0;
  }
}

template <class T>
cudaError_t launch_density_norm(const T* R, const T* s, int64_t E, int nb, int nv, double volume, StepState* ss,
                                double* partials, int ramp_n, int p, double cfl_max, cudaStream_t st) {
  int64_t b = (E * nb + 255) / 256;
  if (b > RED_BLOCKS) b = RED_BLOCKS;
  density_norm_kernel<T><<<(unsigned)(b < 1 ? 1 : b), 256, 0, st>>>(R, s, E, nb, nv, volume, ss, partials, ramp_n, p, cfl_max);
  return cudaGetLastError();
}

#define PCEXP_INST(T)                                                                                         \
  template cudaError_t launch_wall_force<T>(const DGData<T>&, int64_t, const T*, double, double, double*, double*, \
                                            double*, unsigned*, cudaStream_t);                                \
  template cudaError_t launch_jvp_state_adjoint<T>(const DGData<T>&, const T*, const T*, const T*, T*, T*,        \
                                                   const T*, T, cudaStream_t);                                \
  template cudaError_t launch_jac_adjoint<T>(const DGData<T>&, LinData<T>, const T*, T*, T*, const T*, T,        \
                                             cudaStream_t);                                                   \
  template cudaError_t launch_linearize<T>(const DGData<T>&, const T*, LinData<T>, cudaStream_t);               \
  template cudaError_t launch_jac_apply<T>(const DGData<T>&, LinData<T>, const T*, T*, T*, const T*, const int*, \
                                           const double*, cudaStream_t, const cudaEvent_t*);                  \
  template cudaError_t launch_dg_operator<T>(const DGData<T>&, const T*, const T*, T*, T*, const T*, const int*, \
                                             cudaStream_t, const cudaEvent_t*, const double*);                \
  template cudaError_t launch_local_dt<T>(const DGData<T>&, const T*, const double*, double, T*, double*,      \
                                          double*, unsigned*, cudaStream_t);                                   \
  template cudaError_t launch_paper_to_internal<T>(const double*, T*, const double*, int64_t, int, int,        \
                                                   cudaStream_t);                                              \
  template cudaError_t launch_internal_to_paper<T>(const T*, double*, const double*, int64_t, int, int,        \
                                                   cudaStream_t);                                              \
  template cudaError_t launch_scale_elements<T>(T*, const T*, int64_t, int, cudaStream_t);                     \
  template cudaError_t launch_density_norm<T>(const T*, const T*, int64_t, int, int, double, StepState*,       \
                                              double*, int, int, double, cudaStream_t);
PCEXP_INST(double)
PCEXP_INST(float)

}  // namespace pcexp
