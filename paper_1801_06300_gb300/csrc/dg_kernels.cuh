// DG operator kernels on triangles (D = 2) and tetrahedra (D = 3): the residual
// R(u) of Eq. euler3 (Sec. 4.2), its tangent-linear J(u) v (the exact Jacobian of
// Eq. jac1 / jac2, applied matrix-free), the transpose and second-order adjoints,
// the output functionals and the element time-step rule of Eq. x3d.  Each
// dimension is instantiated in its own translation unit (dg2d.cu, dg3d.cu).
//
// Basis: a reference-simplex orthonormal basis phi^_j mapped affinely and scaled
// by |det A_e|^-1/2, so it is orthonormal on every element (the mass matrix is the
// identity, as with the paper's basis).  With x = v0 + A xi:
//   U(x_q)        = |det A|^-1/2 sum_j phi^_j(xi_q) u_j
//   volume term   = |det A|^1/2 sum_q w_q sum_d' d phi^_i/d xi_d'(xi_q) Fhat_d'
//                   with Fhat_d' = sum_d (A^-1)_{d' d} F_d(U(x_q))
//   face term     = -|det A|^-1/2 sum_q w_q |f| phi^_i(x_q) F~_n(x_q)
// Two launches per operator: a face kernel (one thread per face point) writes
// |f| w_q F~_n into the face-flux buffer G; an element kernel (a tile of elements
// per block, staged in shared memory) adds the volume term and lifts the face
// fluxes of its D+1 faces.  Every face flux is computed once and every output is
// written once, in a fixed order (deterministic).
//
// Face points are those of the face's L element (its local face-vertex order).
// The trace tables Bf[face][perm][q][j] hold phi^_j at face point q of local face
// `face` when the element's face vertices are the L element's permuted by `perm`
// (perm 0 = identity; in 2D perm 1 reverses the edge).  An element's face slot
// ef = (face index << 4) | (side << 3) | perm.
#pragma once
#include <cfloat>
#include <type_traits>

#include "kernels.h"

namespace pcexp {

template <int D, int P> struct Ord {
  static constexpr int NV = D + 2;
  static constexpr int NB = D == 2 ? (P + 1) * (P + 2) / 2 : (P + 1) * (P + 2) * (P + 3) / 6;
  // volume and face points: collapsed rules with p + 1 points per direction, except
  // tetrahedra at p = 2 (the symmetric 14-point volume and 7-point face rules)
  static constexpr int NQ = D == 2 ? (P + 1) * (P + 1) : P == 2 ? 14 : (P + 1) * (P + 1) * (P + 1);
  static constexpr int NFQ = D == 2 ? P + 1 : P == 2 ? 7 : (P + 1) * (P + 1);
  static constexpr int NF = D + 1;                  // faces per element
  static constexpr int NPERM = D == 2 ? 2 : 6;      // vertex permutations of a face
  static constexpr int GEO = D == 2 ? 8 : 12;       // geometry record: A^-1 (D x D), sqrt|det|, h, 1/sqrt|det|
  static constexpr int SD = D * D;       // sqrt|det A|
  static constexpr int HE = D * D + 1;   // h
  static constexpr int ISD = D * D + 2;  // 1 / sqrt|det A| (multiplications instead of FP64 divisions)
  static constexpr int NVB = NV * NB;
  // elements per block (tetrahedra: at most 16, which keeps the FP64 tile within 48 KB)
  static constexpr int ET0 = (256 / NQ) > 128 ? 128 : (256 / NQ);
  static constexpr int ET = (D == 3 && ET0 > 16) ? 16 : ET0;
  static constexpr int NJV = D * NV * NV;           // volume point-Jacobian entries
  static constexpr int NJF = 2 * NV * NV;           // face point-Jacobian entries
  static constexpr int NBF = NF * NPERM * NFQ * NB;  // trace-table entries
  static constexpr bool SMEM_BF = D == 2;            // stage the trace tables in shared memory
};

template <class S> struct PartOf;
template <> struct PartOf<double> { PCEXP_DEV static double get(double x) { return x; } };
template <> struct PartOf<float> { PCEXP_DEV static float get(float x) { return x; } };
template <class T> struct PartOf<Tangent<T>> { PCEXP_DEV static T get(Tangent<T> x) { return x.d; } };

// table read: shared memory, or global memory through the read-only cache
template <bool SMEM, class T> PCEXP_DEV T tab(const T* p) {
  if constexpr (SMEM) return *p;
  else return __ldg(p);
}

// slip wall or symmetry plane: both take the slip-wall ghost state
PCEXP_DEV bool mirror_bc(int eR) { return -eR == PCEXP_BC_SLIP_WALL || -eR == PCEXP_BC_SYMMETRY; }

// Source term of a rotating frame on the orthonormal basis: S = -omega x m is linear in U, so
// int_E phi_i S(U_h) dx = -(omega x m_i) coefficient-wise (m_i the momentum coefficients of
// test function i).  Returns component k (0..D-1) given the D momentum coefficients m.
template <class T, int D>
PCEXP_DEV T rot_source(const T* om, const T (&m)[D], int k) {
  const T mx = m[0], my = m[1], mz = D == 3 ? m[D - 1] : T(0);
  const T c = k == 0 ? om[1] * mz - om[2] * my : (k == 1 ? om[2] * mx - om[0] * mz : om[0] * my - om[1] * mx);
  return -c;
}

template <class O> PCEXP_DEV int slot_face(int fs) { return fs >> 4; }
PCEXP_DEV int slot_side(int fs) { return (fs >> 3) & 1; }
PCEXP_DEV int slot_perm(int fs) { return fs & 7; }

// ------------------------------------------------------------------ face kernel
template <class T, int D, int P, bool TAN>
__global__ void __launch_bounds__(256) face_kernel(DGData<T> d, const T* __restrict__ u,
                                                   const T* __restrict__ du, T* __restrict__ G,
                                                   const int* __restrict__ skip) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, GEO = O::GEO;
  constexpr bool SM = O::SMEM_BF;
  using S = typename std::conditional<TAN, Tangent<T>, T>::type;
  __shared__ T sBf[SM ? O::NBF : 1];
  __shared__ T sWf[NFQ];
  if (skip && *skip) return;
  if constexpr (SM)
    for (int i = threadIdx.x; i < O::NBF; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < NFQ; i += blockDim.x) sWf[i] = d.Wf[i];
  __syncthreads();
  const T* Bf = SM ? sBf : d.Bf;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.F * NFQ) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = (loc >> 8) & 0xff, pR = loc >> 16;
  T n[D];
#pragma unroll
  for (int k = 0; k < D; ++k) n[k] = d.fgeo[4 * f + k];
  const T meas = d.fgeo[4 * f + D];
  S UL[NV], UR[NV];
  {
    const T isd = d.geo[GEO * (int64_t)eL + O::ISD];
    const T* ue = u + (int64_t)eL * NV * NB;
    const T* be = Bf + ((fL * NPERM) * NFQ + q) * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0, b = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const T bj = tab<SM>(be + j);
        a += bj * ue[v * NB + j];
        if constexpr (TAN) b += bj * du[(int64_t)eL * NV * NB + v * NB + j];
      }
      if constexpr (TAN) UL[v] = S{a * isd, b * isd};
      else UL[v] = a * isd;
    }
  }
  if (eR >= 0) {
    const T isd = d.geo[GEO * (int64_t)eR + O::ISD];
    const T* ue = u + (int64_t)eR * NV * NB;
    const T* be = Bf + ((fR * NPERM + pR) * NFQ + q) * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0, b = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const T bj = tab<SM>(be + j);
        a += bj * ue[v * NB + j];
        if constexpr (TAN) b += bj * du[(int64_t)eR * NV * NB + v * NB + j];
      }
      if constexpr (TAN) UR[v] = S{a * isd, b * isd};
      else UR[v] = a * isd;
    }
  } else if (mirror_bc(eR)) {
    ghost_slip_wall<D, S, T>(UL, n, UR, d.rot ? d.vrn[idx] : T(0));
  } else {
    ghost_farfield<D, S, T>(UL, n, d.fs, UR);
  }
  S Fn[NV];
  roe_flux<D, S, T>(UL, UR, n, d.fs.gamma, Fn, d.rot ? d.vrn[idx] : T(0));
  const T wl = meas * sWf[q];
  T* g = G + idx * NV;
#pragma unroll
  for (int v = 0; v < NV; ++v) g[v] = wl * PartOf<S>::get(Fn[v]);
}

// Rows of the element kernel's tables and coefficient tiles are padded to whole 16-byte
// vectors so that a row is read with 16-byte loads.
template <class T> constexpr int VECW = 16 / (int)sizeof(T);
template <class T, int N> constexpr int PADV = (N + VECW<T> - 1) / VECW<T> * VECW<T>;

// r[0..N) = p[0..N) from a 16-byte-aligned row (shared memory, or global through the
// read-only cache), N a multiple of VECW<T>
template <class T, int N, bool GLOBAL = false>
PCEXP_DEV void load_row(const T* p, T (&r)[N]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
      const float4 a = GLOBAL ? __ldg(reinterpret_cast<const float4*>(p) + k) : reinterpret_cast<const float4*>(p)[k];
      r[4 * k] = a.x;
      r[4 * k + 1] = a.y;
      r[4 * k + 2] = a.z;
      r[4 * k + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const double2 a = GLOBAL ? __ldg(reinterpret_cast<const double2*>(p) + k) : reinterpret_cast<const double2*>(p)[k];
      r[2 * k] = a.x;
      r[2 * k + 1] = a.y;
    }
  }
}

// c[0..N) = p[0..N), coefficients of one variable of an element (read-only in the kernel):
// 8-byte loads of FP32 pairs when N is even (rows then start on 8-byte boundaries)
template <class T, int N>
PCEXP_DEV void load_coeffs(const T* __restrict__ p, T (&c)[N]) {
  if constexpr (sizeof(T) == 4 && N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const float2 a = __ldg(reinterpret_cast<const float2*>(p) + k);
      c[2 * k] = a.x;
      c[2 * k + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) c[k] = __ldg(p + k);
  }
}

// lift of the D+1 face fluxes onto test function i of variable v of element e
template <class T, int D, int P, bool SM>
PCEXP_DEV T lift_faces(const DGData<T>& d, const T* Bf, const T* __restrict__ G, int64_t e, int v, int i) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, NF = O::NF;
  T lift = 0;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int fs = d.ef[NF * e + k];
    const T* gf = G + (int64_t)slot_face<O>(fs) * NFQ * NV;
    const T* tb = Bf + ((k * NPERM + slot_perm(fs)) * NFQ) * NB + i;
    T a = 0;
#pragma unroll
    for (int q = 0; q < NFQ; ++q) a += tab<SM>(tb + q * NB) * gf[q * NV + v];
    lift = slot_side(fs) ? lift + a : lift - a;
  }
  return lift;
}

// --------------------------------------------------------------- element kernel
// Phase 1: one thread per volume point forms the trace (and tangent) of u, the Euler flux
// and its mapping to reference directions.  Phase 2: a group of S lanes owns one (element,
// variable) pair and accumulates all nb test functions at once over a strided share of the
// (point, direction) sum and of the element's faces (the lift pre-scaled by 1/|det A| so it
// shares the accumulator); a shuffle tree combines the S shares.  Every operand row is read
// with 16-byte loads and serves all nb accumulators.  (Staging the block's face fluxes and
// the 3D trace tables in shared memory was measured slower on GB300: the larger footprint
// costs more occupancy than the L1 traffic it saves.)
template <class T, int D, int P, bool TAN>
__global__ void __launch_bounds__(256) elem_kernel(DGData<T> d, const T* __restrict__ u,
                                                   const T* __restrict__ du, const T* __restrict__ G,
                                                   T* __restrict__ out, const T* __restrict__ escale,
                                                   const int* __restrict__ skip, const double* __restrict__ oscale) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, NFQ = O::NFQ, ET = O::ET, NVB = O::NVB, NV = O::NV, GEO = O::GEO;
  constexpr int DV = D * NV, NF = O::NF, NPERM = O::NPERM;
  constexpr int NBP = PADV<T, NB>;
  constexpr bool SM = O::SMEM_BF;
  constexpr int NPAIR = ET * NV;
  constexpr int S = (NPAIR * 8 <= 256) ? 8 : (NPAIR * 4 <= 256) ? 4 : (NPAIR * 2 <= 256) ? 2 : 1;
  constexpr int ROUNDS = (NPAIR * S + 255) / 256;
  using Sc = typename std::conditional<TAN, Tangent<T>, T>::type;
  __shared__ __align__(16) T sBv[NQ * NBP];
  __shared__ __align__(16) T sDv[D * NQ * NBP];
  __shared__ __align__(16) T sBf[SM ? NF * NPERM * NFQ * NBP : 1];
  __shared__ __align__(16) T su[ET * NV * NBP];
  __shared__ __align__(16) T sdu[TAN ? ET * NV * NBP : 1];
  __shared__ T sF[ET * NQ * DV];
  __shared__ T sgeo[ET * GEO];
  if (skip && *skip) return;
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)((d.E - e0) < ET ? (d.E - e0) : ET);
  for (int i = threadIdx.x; i < NQ * NBP; i += blockDim.x) {
    const int r = i / NBP, j = i - r * NBP;
    sBv[i] = j < NB ? d.Bv[r * NB + j] : T(0);
  }
  for (int i = threadIdx.x; i < D * NQ * NBP; i += blockDim.x) {
    const int r = i / NBP, j = i - r * NBP;
    sDv[i] = j < NB ? d.Dv[r * NB + j] : T(0);
  }
  if constexpr (SM)
    for (int i = threadIdx.x; i < NF * NPERM * NFQ * NBP; i += blockDim.x) sBf[i] = d.BfP[i];
  for (int i = threadIdx.x; i < ne * NV * NBP; i += blockDim.x) {
    const int r = i / NBP, j = i - r * NBP;
    su[i] = j < NB ? u[e0 * NVB + r * NB + j] : T(0);
    if constexpr (TAN) sdu[i] = j < NB ? du[e0 * NVB + r * NB + j] : T(0);
  }
  for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) sgeo[i] = d.geo[e0 * GEO + i];
  __syncthreads();
  const T g = d.fs.gamma;
  const T osc = oscale ? (T)*oscale : T(1);
  // phase 1: flux at each volume point, mapped to reference directions
  for (int it = threadIdx.x; it < ne * NQ; it += blockDim.x) {
    const int el = it / NQ, q = it - el * NQ;
    const T* ge = sgeo + el * GEO;
    const T isd = ge[O::ISD];
    T b[NBP];
    load_row<T, NBP>(sBv + q * NBP, b);
    Sc U[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T c[NBP];
      load_row<T, NBP>(su + (el * NV + v) * NBP, c);
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) a = fma(b[j], c[j], a);
      if constexpr (TAN) {
        load_row<T, NBP>(sdu + (el * NV + v) * NBP, c);
        T t = 0;
#pragma unroll
        for (int j = 0; j < NB; ++j) t = fma(b[j], c[j], t);
        U[v] = Sc{a * isd, t * isd};
      } else {
        U[v] = a * isd;
      }
    }
    Sc F[D][NV];
    euler_flux<D, Sc, T>(U, g, F);
    if (d.rot) {  // rotating frame: F - U v_r^T at the point
      const T* vr = d.vrq + ((e0 + el) * NQ + q) * D;
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) F[k][v] = F[k][v] - U[v] * vr[k];
    }
    T* fo = sF + (el * NQ + q) * DV;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T fk[D];
#pragma unroll
      for (int k = 0; k < D; ++k) fk[k] = PartOf<Sc>::get(F[k][v]);
#pragma unroll
      for (int dd = 0; dd < D; ++dd) {
        T a = ge[dd * D] * fk[0];
#pragma unroll
        for (int k = 1; k < D; ++k) a += ge[dd * D + k] * fk[k];
        fo[dd * NV + v] = a;
      }
    }
  }
  __syncthreads();
  const T* Bf = SM ? sBf : d.BfP;
  // phase 2: S lanes per (element, variable): test against grad phi and lift the faces
  const int ls = threadIdx.x % S;
#pragma unroll 1
  for (int round = 0; round < ROUNDS; ++round) {
    const int pr = round * (256 / S) + (int)threadIdx.x / S;
    const bool act = pr < ne * NV;
    const int prc = act ? pr : 0;
    const int el = prc / NV, v = prc - (prc / NV) * NV;
    T acc[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] = T(0);
    for (int k = ls; k < NQ * D; k += S) {
      const int q = k / D, dd = k - (k / D) * D;
      const T f = sF[(el * NQ + q) * DV + dd * NV + v];
      T row[NBP];
      load_row<T, NBP>(sDv + (dd * NQ + q) * NBP, row);
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[i] = fma(row[i], f, acc[i]);
    }
    const int64_t e = e0 + el;
    const T isd = sgeo[el * GEO + O::ISD];
    const T rdet = isd * isd;  // the lift carries 1/sqrt|det|, the volume term sqrt|det|
    for (int kf = ls; kf < NF; kf += S) {
      const int fs = d.ef[NF * e + kf];
      const T* gf = G + (int64_t)slot_face<O>(fs) * NFQ * NV;
      const T* tb = Bf + ((kf * NPERM + slot_perm(fs)) * NFQ) * NBP;
      const T sg = slot_side(fs) ? rdet : -rdet;
#pragma unroll
      for (int q = 0; q < NFQ; ++q) {
        const T gq = sg * gf[q * NV + v];
        T row[NBP];
        load_row<T, NBP, !SM>(tb + q * NBP, row);
#pragma unroll
        for (int i = 0; i < NB; ++i) acc[i] = fma(row[i], gq, acc[i]);
      }
    }
#pragma unroll
    for (int off = S / 2; off >= 1; off /= 2)
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
    if (act) {
      const T es = escale ? escale[e] : T(1);
      const T sc = sgeo[el * GEO + O::SD] * osc * es;
      const bool src = d.rot && v >= 1 && v <= D;
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i % S == ls) {
          T o = acc[i] * sc;
          if (src) {  // the rotating frame's source, on the coefficients of u (R) or du (J v)
            const T* xr = (TAN ? sdu : su) + el * NV * NBP + i;
            T m[D];
#pragma unroll
            for (int k = 0; k < D; ++k) m[k] = xr[(1 + k) * NBP];
            o += rot_source<T, D>(d.om, m, v - 1) * osc * es;
          }
          out[e * NVB + v * NB + i] = o;
        }
    }
  }
}

template <class T, int D, int P>
cudaError_t dg_op_p(const DGData<T>& d, const T* u, const T* du, T* out, T* G, const T* escale, const int* skip,
                    const double* oscale, cudaStream_t st, const cudaEvent_t* ev) {
  using O = Ord<D, P>;
  const int64_t nfp = d.F * O::NFQ;
  if (ev) cudaEventRecord(ev[0], st);
  if (nfp > 0) {
    const int64_t nb = (nfp + 255) / 256;
    if (du) face_kernel<T, D, P, true><<<(unsigned)nb, 256, 0, st>>>(d, u, du, G, skip);
    else face_kernel<T, D, P, false><<<(unsigned)nb, 256, 0, st>>>(d, u, du, G, skip);
  }
  if (ev) cudaEventRecord(ev[1], st);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  if (du) elem_kernel<T, D, P, true><<<(unsigned)eb, 256, 0, st>>>(d, u, du, G, out, escale, skip, oscale);
  else elem_kernel<T, D, P, false><<<(unsigned)eb, 256, 0, st>>>(d, u, du, G, out, escale, skip, oscale);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

// ------------------------------------- FP32 volume J v by flux tangents, one element per lane
// The reference tables [Bv (nq x nb) | Dv (D x nq x nb)] of one (D, p) in constant memory.
// They depend on the reference simplex alone, so every context of that order uploads the
// same bytes (tan_tables_p); the kernel below reads them at warp-uniform addresses, which
// the constant cache serves as broadcasts outside the load/store pipe.
template <int D, int P> __constant__ float c_tan[(D + 1) * Ord<D, P>::NQ * Ord<D, P>::NB];

// ---------------------------------- the same J v volume part as a pipelined persistent kernel
// cp.async copies (global -> shared, no register staging), 4 or 16 bytes
PCEXP_DEV void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
PCEXP_DEV void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
PCEXP_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
PCEXP_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory words of one stage of elem_tan_pipe_kernel<D, P>: u, u' rows, face fluxes,
// geometry records and face slots of 32 elements.
template <int D, int P> struct TanPipe {
  using O = Ord<D, P>;
  static constexpr int NBP = PADV<float, O::NB>;
  static constexpr int UR0 = 2 * O::NV * NBP;
  static constexpr int UROW = UR0 + (36 - UR0 % 32) % 32;
  static constexpr int GREC = O::NF * O::NFQ * O::NV;
  static constexpr int GROW = GREC | 1;
  static constexpr int PST = O::NVB | 1;
  static constexpr int SU = 32 * UROW, SG = 32 * GROW, SGEO = 32 * O::GEO, SEF = 32 * O::NF;
  // warps per block: with two 41 KB stages two blocks fit an SM (P2); six warps each keep the
  // registers of 2 x 192 threads within the SM's file and split the 14 points 3/3/2/2/2/2
  static constexpr int WARPS = D == 3 ? 6 : O::NF;
  static constexpr int PART = WARPS * 32 * PST;
  // the partial sums reuse the consumed rows and face fluxes (not the geometry records)
  static constexpr int SROWS = ((SU + SG > PART ? SU + SG : PART) + 3) / 4 * 4;
  static constexpr int STAGE = SROWS + SGEO + SEF;  // words (SGEO and SU keep 16-byte alignment)
  static_assert(SU % 4 == 0, "16-byte alignment of the face fluxes");
  static constexpr size_t BYTES = 2 * (size_t)STAGE * 4;
};

// Persistent element kernel of the FP32 J v on tetrahedra: a block of six warps loops over
// tiles of 32 elements (one element per lane; the warps split the volume points and the
// faces, so every reference-table index is warp-uniform and the tables are read from constant
// memory).  While tile t is computed, tile t + gridDim.x is copied into the other
// shared-memory stage by cp.async: its u, u' rows and geometry records at the start of the
// tile, its face fluxes (gathered through its face slots, which are loaded into a register at
// the start and are needed only then) after the volume loop.  The staging latency is hidden
// behind a tile of compute.
template <int D, int P>
__global__ void __launch_bounds__(32 * TanPipe<D, P>::WARPS, 2) elem_tan_pipe_kernel(DGData<float> d, const float* __restrict__ u,
                                                                     const float* __restrict__ du,
                                                                     const float* __restrict__ G, float* __restrict__ out,
                                                                     const float* __restrict__ escale,
                                                                     const int* __restrict__ skip,
                                                                     const double* __restrict__ oscale, int64_t ntiles) {
  using O = Ord<D, P>;
  using L = TanPipe<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, NFQ = O::NFQ, NV = O::NV, NF = O::NF, NPERM = O::NPERM, GEO = O::GEO;
  constexpr int NVB = O::NVB, QW = L::WARPS, NT = 32 * QW;
  static_assert(NT >= 32 * NF, "one thread per (element, face) slot of a tile");
  constexpr int NBP = L::NBP, UROW = L::UROW, GROW = L::GROW, PST = L::PST;
  static_assert(!O::SMEM_BF, "tetrahedra read the trace tables through the read-only cache");
  extern __shared__ __align__(16) float dsm[];
  if (skip && *skip) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  const float g = d.fs.gamma;
  const float osc = oscale ? (float)*oscale : 1.f;

  // copies of tile tt into stage S: u, u' rows (4-byte copies into padded rows), geometry
  // records (16-byte copies); the face fluxes follow once the face slots are known
  auto stage_rows = [&](int64_t tt, float* S) {
    const int64_t e0 = tt * 32;
    const int ne = (int)((d.E - e0) < 32 ? (d.E - e0) : 32);
    float* su = S;
    float* sgeo = S + L::SROWS;
    for (int i = tid; i < ne * NVB; i += NT) {
      const int el = i / NVB, r = i - el * NVB, v = r / NB, j = r - v * NB;
      cp_async4(su + el * UROW + v * NBP + j, u + e0 * NVB + i);
      cp_async4(su + el * UROW + (NV + v) * NBP + j, du + e0 * NVB + i);
    }
    for (int i = tid; i < ne * (GEO / 4); i += NT) cp_async16(sgeo + 4 * i, d.geo + e0 * GEO + 4 * i);
  };
  auto stage_faces = [&](int64_t tt, float* S, int fs) {
    const int64_t e0 = tt * 32;
    const int ne = (int)((d.E - e0) < 32 ? (d.E - e0) : 32);
    if (tid < ne * NF) {
      int* sef = reinterpret_cast<int*>(S + L::SROWS + L::SGEO);
      sef[tid] = fs;
      const int el = tid / NF, kf = tid - el * NF;
      float* dst = S + L::SU + el * GROW + kf * NFQ * NV;
      const float* src = G + (int64_t)slot_face<O>(fs) * NFQ * NV;
#pragma unroll 5
      for (int k = 0; k < NFQ * NV; ++k) cp_async4(dst + k, src + k);
    }
  };

  // prologue: tile t into stage 0
  {
    stage_rows(t, dsm);
    const int64_t e0 = t * 32;
    const int ne = (int)((d.E - e0) < 32 ? (d.E - e0) : 32);
    const int fs = tid < ne * NF ? d.ef[e0 * NF + tid] : 0;
    stage_faces(t, dsm, fs);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
  }
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    float* S = dsm + (it & 1) * L::STAGE;
    float* N = dsm + ((it & 1) ^ 1) * L::STAGE;
    const int64_t e0 = t * 32;
    const int ne = (int)((d.E - e0) < 32 ? (d.E - e0) : 32);
    const int64_t tn = t + gridDim.x;
    const bool has_next = tn < ntiles;
    int fs_next = 0;
    if (has_next) {
      stage_rows(tn, N);
      const int64_t en0 = tn * 32;
      const int nen = (int)((d.E - en0) < 32 ? (d.E - en0) : 32);
      if (tid < nen * NF) fs_next = d.ef[en0 * NF + tid];
    }
    const float* su = S;
    const float* sg = S + L::SU;
    const float* sgeo = S + L::SROWS;
    const int* sef = reinterpret_cast<const int*>(S + L::SROWS + L::SGEO);
    const int el = lane < ne ? lane : 0;  // lanes past the last element repeat element 0; discarded
    const float* ge = sgeo + el * GEO;
    float Ai[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) Ai[k] = ge[k];
    const float isd = ge[O::ISD];
    float acc[NV][NB];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[v][i] = 0.f;
    const float* ur = su + el * UROW;
    // flux tangent at volume point q mapped to reference directions, tested (accumulated)
    auto point = [&](int q, const Tangent<float>(&U)[NV]) {
      Tangent<float> F[D][NV];
      euler_flux<D, Tangent<float>, float>(U, g, F);
      const float* dq = c_tan<D, P> + NQ * NB + q * NB;
#pragma unroll
      for (int dd = 0; dd < D; ++dd) {
        float fh[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float a = Ai[dd * D] * F[0][v].d;
#pragma unroll
          for (int k = 1; k < D; ++k) a += Ai[dd * D + k] * F[k][v].d;
          fh[v] = a;
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const float tq = dq[dd * NQ * NB + i];
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v][i] = fmaf(tq, fh[v], acc[v][i]);
        }
      }
    };
    // two of the warp's points per pass: each u, u' row read from shared memory serves both
    // traces (the rows are the kernel's main shared-memory traffic)
#pragma unroll 1
    for (int q0 = w; q0 < NQ; q0 += 2 * QW) {
      const int q1 = q0 + QW;
      const bool two = q1 < NQ;  // warp-uniform
      const float* b0 = c_tan<D, P> + q0 * NB;
      const float* b1 = c_tan<D, P> + (two ? q1 : q0) * NB;
      Tangent<float> U0[NV], U1[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float c[NBP];
        load_row<float, NBP>(ur + v * NBP, c);
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          a0 = fmaf(b0[j], c[j], a0);
          a1 = fmaf(b1[j], c[j], a1);
        }
        load_row<float, NBP>(ur + (NV + v) * NBP, c);
        float t0 = 0.f, t1 = 0.f;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          t0 = fmaf(b0[j], c[j], t0);
          t1 = fmaf(b1[j], c[j], t1);
        }
        U0[v] = Tangent<float>{a0 * isd, t0 * isd};
        U1[v] = Tangent<float>{a1 * isd, t1 * isd};
        asm volatile("" ::: "memory");  // one variable's rows in flight at a time (registers)
      }
      point(q0, U0);
      if (two) point(q1, U1);
    }
    // the next tile's face fluxes, now that its face slots have arrived
    if (has_next) stage_faces(tn, N, fs_next);
    cp_async_commit();
    // faces: lift of the staged face fluxes, pre-scaled by 1/|det A| to share the accumulators;
    // faces 0..NF-2 go whole to the last warps (warp QW - 1 - kf, which have fewer volume
    // points); the points of face NF-1 are split between warps 0 and 1, so that no warp waits
    // at the tile's barriers for one that has a whole face more
    // (with 14 points, 3/3/2/2/2/2 over six warps, the four warps of two points take one whole
    // face each instead)
    static_assert(QW - (NF - 1) >= 2, "two warps share the last face");
    constexpr bool FACE_PER_LIGHT_WARP = QW - NQ % QW == NF;
    const float rdet = isd * isd;
    int kf = -1, qa = 0, qb = NFQ;
    if constexpr (FACE_PER_LIGHT_WARP) {
      if (w >= QW - NF) kf = QW - 1 - w;
    } else {
      if (w >= QW - (NF - 1)) {
        kf = QW - 1 - w;
      } else if (w < 2) {
        kf = NF - 1;
        qa = w == 0 ? 0 : (NFQ + 1) / 2;
        qb = w == 0 ? (NFQ + 1) / 2 : NFQ;
      }
    }
    if (kf >= 0) {  // warp-uniform
      const int fs = sef[el * NF + kf];
      const float sgn = slot_side(fs) ? rdet : -rdet;
      const float* tb = d.BfP + ((kf * NPERM + slot_perm(fs)) * NFQ) * NBP;
      const float* gr = sg + el * GROW + kf * NFQ * NV;
#pragma unroll
      for (int q = 0; q < NFQ; ++q) {
        if (q < qa || q >= qb) continue;  // warp-uniform
        float row[NBP];
        load_row<float, NBP, true>(tb + q * NBP, row);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float gq = sgn * gr[q * NV + v];
#pragma unroll
          for (int i = 0; i < NB; ++i) acc[v][i] = fmaf(row[i], gq, acc[v][i]);
        }
      }
    }
    __syncthreads();  // the stage is consumed; the partial sums reuse it
    float* part = S;
    float* pr = part + (w * 32 + lane) * PST;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int i = 0; i < NB; ++i) pr[v * NB + i] = acc[v][i];
    __syncthreads();
    for (int o = tid; o < ne * NVB; o += NT) {
      const int el2 = o / NVB, r = o - el2 * NVB;
      float s = part[el2 * PST + r];
#pragma unroll
      for (int ww = 1; ww < QW; ++ww) s += part[(ww * 32 + el2) * PST + r];
      float sc = sgeo[el2 * GEO + O::SD] * osc;
      if (escale) sc *= escale[e0 + el2];
      out[e0 * NVB + o] = s * sc;
    }
    cp_async_wait_all();
    __syncthreads();  // next stage landed; this stage's partial sums are read
  }
}

template <int D, int P>
cudaError_t tan_tables_p(const DGData<float>& d, cudaStream_t st) {
  using O = Ord<D, P>;
  cudaError_t e = cudaSuccess;
  if constexpr (D == 3) {
    e = cudaFuncSetAttribute(elem_tan_pipe_kernel<D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TanPipe<D, P>::BYTES);
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpyToSymbolAsync(c_tan<D, P>, d.Bv, sizeof(float) * (D + 1) * O::NQ * O::NB, 0,
                                 cudaMemcpyDeviceToDevice, st);
}

// ------------------------------------------------------- point Jacobians (linearisation)
// The exact Jacobian of the scheme (Eq. jac1, jac2) is assembled point by point: the
// volume flux Jacobians dF_d/dU and the Riemann-flux Jacobians dF~/dU_L, dF~/dU_R are
// evaluated exactly by running the flux code on Jet<T, D+2> numbers seeded with unit
// directions (the paper obtains the Riemann-flux Jacobians by AD as well).  Every J v
// of a PCEXP step is taken at u_n, so the Jacobians are built once per step and each
// of the 2m+1 products reduces to traces, small mat-vecs and the test/lift contractions.
template <class T, int D, int P>
__global__ void __launch_bounds__(256) linearize_vol_kernel(DGData<T> d, const T* __restrict__ u,
                                                            T* __restrict__ Avol) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, NV = O::NV, GEO = O::GEO;
  using J = Jet<T, NV>;
  const int64_t n = d.E * NQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t e = idx / NQ;
  const int q = (int)(idx - e * NQ);
  const T* ge = d.geo + GEO * e;
  const T isd = ge[O::ISD];
  J U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) a += __ldg(d.Bv + q * NB + j) * u[e * NV * NB + v * NB + j];
    U[v].v = a * isd;
#pragma unroll
    for (int c = 0; c < NV; ++c) U[v].d[c] = (v == c) ? T(1) : T(0);
  }
  J F[D][NV];
  euler_flux<D, J, T>(U, d.fs.gamma, F);
  if (d.rot) {
    const T* vr = d.vrq + idx * D;
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) F[k][v] = F[k][v] - U[v] * vr[k];
  }
#pragma unroll
  for (int dd = 0; dd < D; ++dd)
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        T a = ge[dd * D] * F[0][v].d[c];
#pragma unroll
        for (int k = 1; k < D; ++k) a += ge[dd * D + k] * F[k][v].d[c];
        Avol[(int64_t)(dd * NV * NV + v * NV + c) * n + idx] = a;
      }
}

template <class T, int D, int P>
__global__ void __launch_bounds__(128) linearize_face_kernel(DGData<T> d, const T* __restrict__ u,
                                                             T* __restrict__ Bface) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, GEO = O::GEO, NN = NV * NV;
  using J = Jet<T, NV>;
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = (loc >> 8) & 0xff, pR = loc >> 16;
  T nr[D];
#pragma unroll
  for (int k = 0; k < D; ++k) nr[k] = d.fgeo[4 * f + k];
  const T wq = d.fgeo[4 * f + D] * d.Wf[q];
  T uL[NV], uR[NV];
  const T isdL = d.geo[GEO * (int64_t)eL + O::ISD];
  T isdR = T(0);
  {
    const T* be = d.Bf + ((fL * NPERM) * NFQ + q) * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) a += __ldg(be + j) * u[(int64_t)eL * NV * NB + v * NB + j];
      uL[v] = a * isdL;
    }
  }
  if (eR >= 0) {
    isdR = d.geo[GEO * (int64_t)eR + O::ISD];
    const T* be = d.Bf + ((fR * NPERM + pR) * NFQ + q) * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) a += __ldg(be + j) * u[(int64_t)eR * NV * NB + v * NB + j];
      uR[v] = a * isdR;
    }
  }
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    J L[NV], R[NV], F[NV];
    if (side == 1 && eR < 0) {
#pragma unroll
      for (int k = 0; k < NN; ++k) Bface[bface_at<T, 2 * NN>(NN + k, idx, n)] = T(0);
      break;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      L[v].v = uL[v];
#pragma unroll
      for (int c = 0; c < NV; ++c) L[v].d[c] = (side == 0 && v == c) ? T(1) : T(0);
    }
    if (eR >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R[v].v = uR[v];
#pragma unroll
        for (int c = 0; c < NV; ++c) R[v].d[c] = (side == 1 && v == c) ? T(1) : T(0);
      }
    } else if (mirror_bc(eR)) {
      ghost_slip_wall<D, J, T>(L, nr, R, d.rot ? d.vrn[idx] : T(0));
    } else {
      ghost_farfield<D, J, T>(L, nr, d.fs, R);
    }
    roe_flux<D, J, T>(L, R, nr, d.fs.gamma, F, d.rot ? d.vrn[idx] : T(0));
    const T sc = wq * (side == 0 ? isdL : isdR);
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int c = 0; c < NV; ++c) Bface[bface_at<T, 2 * NN>(side * NN + v * NV + c, idx, n)] = sc * F[v].d[c];
  }
}

template <class T, int D, int P>
__global__ void __launch_bounds__(256) face_apply_kernel(DGData<T> d, const T* __restrict__ Bface,
                                                         const T* __restrict__ dv, T* __restrict__ G,
                                                         const int* __restrict__ skip) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, NN = NV * NV;
  constexpr bool SM = O::SMEM_BF;
  __shared__ T sBf[SM ? O::NBF : 1];
  if (skip && *skip) return;
  if constexpr (SM)
    for (int i = threadIdx.x; i < O::NBF; i += blockDim.x) sBf[i] = d.Bf[i];
  __syncthreads();
  const T* Bf = SM ? sBf : d.Bf;
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = (loc >> 8) & 0xff, pR = loc >> 16;
  // the point's block in 16-byte vectors (bface_at); chunks wholly on the R side are not
  // loaded on boundary faces (the linearisation stores zeros there)
  T B[O::NJF];
  {
    constexpr int VEC = 16 / (int)sizeof(T), NCH = O::NJF / VEC, R = O::NJF % VEC;
    const bool two = eR >= 0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (c * VEC < NN || two) {
        T x[VEC];
        load_row<T, VEC, true>(Bface + ((int64_t)c * n + idx) * VEC, x);
#pragma unroll
        for (int i = 0; i < VEC; ++i) B[c * VEC + i] = x[i];
      } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) B[c * VEC + i] = T(0);
      }
    }
    if constexpr (R > 0) {
      static_assert(R == 2 && sizeof(T) == 4, "the remainder of a point's block is one float pair");
      const float2 x = two ? __ldg(reinterpret_cast<const float2*>(Bface + (int64_t)NCH * VEC * n + idx * R))
                           : make_float2(0.f, 0.f);
      B[NCH * VEC] = x.x;
      B[NCH * VEC + 1] = x.y;
    }
  }
  // traces of dv at the point from each side: the table row (shared memory in 2D; in 3D the
  // padded copy, 16-byte loads) and the element's rows of dv (8-byte loads when nb is even:
  // the kernel is bound by its load instructions as much as by its bytes)
  constexpr int NBP = PADV<T, NB>;
  auto trace = [&](int64_t e, int fl, int pm, T(&t)[NV]) {
    T b[NBP];
    if constexpr (SM) {
      const T* be = Bf + ((fl * NPERM + pm) * NFQ + q) * NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) b[j] = be[j];
    } else {
      load_row<T, NBP, true>(d.BfP + ((fl * NPERM + pm) * NFQ + q) * NBP, b);
    }
    const T* ve = dv + e * NV * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T c[NB];
      load_coeffs<T, NB>(ve + v * NB, c);
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) a += b[j] * c[j];
      t[v] = a;
    }
  };
  T tL[NV], tR[NV];
  trace(eL, fL, 0, tL);
  if (eR >= 0) trace(eR, fR, pR, tR);
  T* g = G + idx * NV;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = 0;
#pragma unroll
    for (int c = 0; c < NV; ++c) a += B[v * NV + c] * tL[c];
    if (eR >= 0) {
#pragma unroll
      for (int c = 0; c < NV; ++c) a += B[NN + v * NV + c] * tR[c];
    }
    g[v] = a;
  }
}

template <class T, int D, int P>
__global__ void __launch_bounds__(256) elem_apply_kernel(DGData<T> d, const T* __restrict__ Avol,
                                                         const T* __restrict__ dv, const T* __restrict__ G,
                                                         T* __restrict__ out, const T* __restrict__ escale,
                                                         const int* __restrict__ skip,
                                                         const double* __restrict__ oscale) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, ET = O::ET, NVB = O::NVB, NV = O::NV, GEO = O::GEO, DV = D * NV;
  constexpr int NN = NV * NV;
  constexpr int NPRE = D == 2 ? O::NJV : NN;  // point-Jacobian entries loaded before the staging
  constexpr bool SM = O::SMEM_BF;
  __shared__ T sBv[NQ * NB];
  __shared__ T sDv[D * NQ * NB];
  __shared__ T sBf[SM ? O::NBF : 1];
  __shared__ T sdu[ET * NVB];
  __shared__ T sF[ET * NQ * DV];
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
  T A[NPRE];
#pragma unroll
  for (int k = 0; k < NPRE; ++k) A[k] = has_pt ? Avol[(int64_t)k * n + pidx] : T(0);
  for (int i = threadIdx.x; i < NQ * NB; i += blockDim.x) sBv[i] = d.Bv[i];
  for (int i = threadIdx.x; i < D * NQ * NB; i += blockDim.x) sDv[i] = d.Dv[i];
  if constexpr (SM)
    for (int i = threadIdx.x; i < O::NBF; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < ne * NVB; i += blockDim.x) sdu[i] = dv[e0 * NVB + i];
  for (int i = threadIdx.x; i < ne; i += blockDim.x) ssd[i] = d.geo[(e0 + i) * GEO + O::ISD];
  __syncthreads();
  const T osc = oscale ? (T)*oscale : T(1);
  // phase 1: trace of dv at this thread's volume point, times the mapped flux Jacobians
  if (has_pt) {
    T t[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) a += sBv[q1 * NB + j] * sdu[el1 * NVB + v * NB + j];
      t[v] = a;
    }
    T* fo = sF + (el1 * NQ + q1) * DV;
#pragma unroll
    for (int dd = 0; dd < D; ++dd)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T a = 0;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const int k = dd * NN + v * NV + c;
          const T akc = k < NPRE ? A[k < NPRE ? k : 0] : Avol[(int64_t)k * n + pidx];
          a += akc * t[c];
        }
        fo[dd * NV + v] = a;
      }
  }
  __syncthreads();
  const T* Bf = SM ? sBf : d.Bf;
  // phase 2: test against grad phi (the sqrt(det) factors cancel), lift the face terms
  for (int it = threadIdx.x; it < ne * NVB; it += blockDim.x) {
    const int el = it / NVB, r = it - el * NVB;
    const int v = r / NB, i = r - v * NB;
    T acc = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int dd = 0; dd < D; ++dd) acc += sDv[(dd * NQ + q) * NB + i] * sF[(el * NQ + q) * DV + dd * NV + v];
    const int64_t e = e0 + el;
    const T lift = lift_faces<T, D, P, SM>(d, Bf, G, e, v, i);
    acc = acc + lift * ssd[el];
    if (d.rot && v >= 1 && v <= D) {  // the rotating frame's source on the coefficients of dv
      T m[D];
#pragma unroll
      for (int k = 0; k < D; ++k) m[k] = sdu[el * NVB + (1 + k) * NB + i];
      acc += rot_source<T, D>(d.om, m, v - 1);
    }
    acc *= osc;
    if (escale) acc *= escale[e];
    out[e0 * NVB + it] = acc;
  }
}

template <class T, int D, int P>
cudaError_t linearize_p(const DGData<T>& d, const T* u, LinData<T> lin, bool faces_only, cudaStream_t st) {
  using O = Ord<D, P>;
  const int64_t nv = d.E * O::NQ, nf = d.F * O::NFQ;
  if (!faces_only) linearize_vol_kernel<T, D, P><<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(d, u, lin.Avol);
  if (nf > 0) linearize_face_kernel<T, D, P><<<(unsigned)((nf + 127) / 128), 128, 0, st>>>(d, u, lin.Bface);
  return cudaGetLastError();
}

// J v from the face point Jacobians and either the volume point Jacobians (u_elem null)
// or the volume flux tangents recomputed at u_elem (the elements then read u and dv
// instead of D nv^2 values per volume point).
//
// face_tan: the face part recomputes the Riemann-flux tangent at every face point from the
// traces of u_elem and dv (face_kernel<TAN>) instead of applying the stored face point
// Jacobians (it then reads u_n and dv instead of 2 nv^2 values per face point).
template <class T, int D, int P>
cudaError_t jac_apply_p(const DGData<T>& d, LinData<T> lin, const T* u_elem, const T* dv, T* out, T* G,
                        const T* escale, const int* skip, const double* oscale, cudaStream_t st,
                        const cudaEvent_t* ev, bool face_tan) {
  using O = Ord<D, P>;
  const int64_t nf = d.F * O::NFQ;
  if (ev) cudaEventRecord(ev[0], st);
  if (nf > 0) {
    if (face_tan && u_elem)
      face_kernel<T, D, P, true><<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(d, u_elem, dv, G, skip);
    else
      face_apply_kernel<T, D, P><<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(d, lin.Bface, dv, G, skip);
  }
  if (ev) cudaEventRecord(ev[1], st);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  if (u_elem) {
    if constexpr (std::is_same<T, float>::value && D == 3) {
      if (d.rot) {  // the frame terms live in the tile kernel
        elem_kernel<T, D, P, true><<<(unsigned)eb, 256, 0, st>>>(d, u_elem, dv, G, out, escale, skip, oscale);
      } else if (d.E > 0) {
        // persistent: two blocks per SM (two 42 KB stages each), tiles of 32 elements
        static int nsm = 0;
        if (!nsm) {
          int dev = 0;
          cudaGetDevice(&dev);
          if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 152;
        }
        const int64_t ntiles = (d.E + 31) / 32;
        const int64_t grid = ntiles < 2 * (int64_t)nsm ? ntiles : 2 * (int64_t)nsm;
        elem_tan_pipe_kernel<D, P><<<(unsigned)grid, 32 * TanPipe<D, P>::WARPS, TanPipe<D, P>::BYTES, st>>>(
            d, u_elem, dv, G, out, escale, skip, oscale, ntiles);
      }
    } else {
      elem_kernel<T, D, P, true><<<(unsigned)eb, 256, 0, st>>>(d, u_elem, dv, G, out, escale, skip, oscale);
    }
  } else {
    elem_apply_kernel<T, D, P><<<(unsigned)eb, 256, 0, st>>>(d, lin.Avol, dv, G, out, escale, skip, oscale);
  }
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

// ------------------------------------------------------------- adjoint J^T w
// Transpose of the point-Jacobian J v (same linearisation state).  With the output
// factors of J v folded into w (w~ = osc * escale_e * w), the face kernel forms the
// adjoint of the lifted face flux at every face point,
//   Gbar = -(1/sd_L) sum_i Bf_L[i] w~_L[i] + (1/sd_R) sum_i Bf_R[i] w~_R[i],
// and stores B_L^T Gbar and B_R^T Gbar; the element kernel applies the transposed
// volume Jacobians to the transposed test of w~ and gathers the transposed traces
// of its faces.  Deterministic (no atomics).
template <class T, int D, int P>
__global__ void __launch_bounds__(256) face_adjoint_kernel(DGData<T> d, const T* __restrict__ Bface,
                                                           const T* __restrict__ w, T* __restrict__ GT,
                                                           const T* __restrict__ escale, T osc) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, GEO = O::GEO, NN = NV * NV;
  constexpr bool SM = O::SMEM_BF;
  __shared__ T sBf[SM ? O::NBF : 1];
  if constexpr (SM)
    for (int i = threadIdx.x; i < O::NBF; i += blockDim.x) sBf[i] = d.Bf[i];
  __syncthreads();
  const T* Bf = SM ? sBf : d.Bf;
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = (loc >> 8) & 0xff, pR = loc >> 16;
  T gb[NV];
  {
    const T sc = -osc * (escale ? escale[eL] : T(1)) * d.geo[GEO * (int64_t)eL + O::ISD];
    const T* be = Bf + ((fL * NPERM) * NFQ + q) * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0;
#pragma unroll
      for (int i = 0; i < NB; ++i) a += tab<SM>(be + i) * w[(int64_t)eL * NV * NB + v * NB + i];
      gb[v] = sc * a;
    }
  }
  if (eR >= 0) {
    const T sc = osc * (escale ? escale[eR] : T(1)) * d.geo[GEO * (int64_t)eR + O::ISD];
    const T* be = Bf + ((fR * NPERM + pR) * NFQ + q) * NB;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0;
#pragma unroll
      for (int i = 0; i < NB; ++i) a += tab<SM>(be + i) * w[(int64_t)eR * NV * NB + v * NB + i];
      gb[v] += sc * a;
    }
  }
  T* o = GT + idx * 2 * NV;
#pragma unroll
  for (int side = 0; side < 2; ++side)
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      T a = 0;
      if (side == 0 || eR >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) a += Bface[bface_at<T, 2 * NN>(side * NN + v * NV + c, idx, n)] * gb[v];
      }
      o[side * NV + c] = a;
    }
}

// transposed face traces of the D+1 faces for coefficient j of variable c of element e
template <class T, int D, int P, bool SM>
PCEXP_DEV T gather_faces_T(const DGData<T>& d, const T* Bf, const T* __restrict__ GT, int64_t e, int c, int j) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, NF = O::NF;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int fs = d.ef[NF * e + k];
    const T* gt = GT + (int64_t)slot_face<O>(fs) * NFQ * 2 * NV + slot_side(fs) * NV + c;
    const T* tb = Bf + ((k * NPERM + slot_perm(fs)) * NFQ) * NB + j;
#pragma unroll
    for (int q = 0; q < NFQ; ++q) acc += tab<SM>(tb + q * NB) * gt[q * 2 * NV];
  }
  return acc;
}

template <class T, int D, int P>
__global__ void __launch_bounds__(256) elem_adjoint_kernel(DGData<T> d, const T* __restrict__ Avol,
                                                           const T* __restrict__ w, const T* __restrict__ GT,
                                                           T* __restrict__ out, const T* __restrict__ escale,
                                                           T osc) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, ET = O::ET, NVB = O::NVB, NV = O::NV, NN = NV * NV;
  constexpr bool SM = O::SMEM_BF;
  __shared__ T sBv[NQ * NB];
  __shared__ T sDv[D * NQ * NB];
  __shared__ T sBf[SM ? O::NBF : 1];
  __shared__ T sw[ET * NVB];
  __shared__ T sU[ET * NQ * NV];
  static_assert(ET * NQ <= 256, "one volume point per thread");
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)((d.E - e0) < ET ? (d.E - e0) : ET);
  const int64_t n = d.E * NQ;
  for (int i = threadIdx.x; i < NQ * NB; i += blockDim.x) sBv[i] = d.Bv[i];
  for (int i = threadIdx.x; i < D * NQ * NB; i += blockDim.x) sDv[i] = d.Dv[i];
  if constexpr (SM)
    for (int i = threadIdx.x; i < O::NBF; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < ne * NVB; i += blockDim.x)
    sw[i] = w[e0 * NVB + i] * osc * (escale ? escale[e0 + i / NVB] : T(1));
  __syncthreads();
  // phase 1: transposed test, then transposed volume Jacobians, at this thread's point
  const int el1 = threadIdx.x / NQ, q1 = threadIdx.x - (threadIdx.x / NQ) * NQ;
  if (threadIdx.x < ne * NQ) {
    const int64_t pidx = (e0 + el1) * NQ + q1;
    T fb[D * NV];
#pragma unroll
    for (int dd = 0; dd < D; ++dd)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T a = 0;
#pragma unroll
        for (int i = 0; i < NB; ++i) a += sDv[(dd * NQ + q1) * NB + i] * sw[el1 * NVB + v * NB + i];
        fb[dd * NV + v] = a;
      }
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      T a = 0;
#pragma unroll
      for (int dd = 0; dd < D; ++dd)
#pragma unroll
        for (int v = 0; v < NV; ++v) a += Avol[(int64_t)(dd * NN + v * NV + c) * n + pidx] * fb[dd * NV + v];
      sU[(el1 * NQ + q1) * NV + c] = a;
    }
  }
  __syncthreads();
  const T* Bf = SM ? sBf : d.Bf;
  // phase 2: transposed volume traces plus the transposed face traces
  for (int it = threadIdx.x; it < ne * NVB; it += blockDim.x) {
    const int el = it / NVB, r = it - el * NVB;
    const int c = r / NB, j = r - c * NB;
    T acc = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc += sBv[q * NB + j] * sU[(el * NQ + q) * NV + c];
    acc += gather_faces_T<T, D, P, SM>(d, Bf, GT, e0 + el, c, j);
    if (d.rot && c >= 1 && c <= D) {  // transpose of the source -omega x: +omega x w~ (antisymmetric)
      T m[D];
#pragma unroll
      for (int k = 0; k < D; ++k) m[k] = sw[el * NVB + (1 + k) * NB + j];
      acc -= rot_source<T, D>(d.om, m, c - 1);
    }
    out[e0 * NVB + it] = acc;
  }
}

template <class T, int D, int P>
cudaError_t jac_adjoint_p(const DGData<T>& d, LinData<T> lin, const T* w, T* out, T* GT, const T* escale, T osc,
                          cudaStream_t st) {
  using O = Ord<D, P>;
  const int64_t nf = d.F * O::NFQ;
  if (nf > 0) face_adjoint_kernel<T, D, P><<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(d, lin.Bface, w, GT, escale, osc);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  elem_adjoint_kernel<T, D, P><<<(unsigned)eb, 256, 0, st>>>(d, lin.Avol, w, GT, out, escale, osc);
  return cudaGetLastError();
}

// ------------------------------------------- second-order adjoint (d(J(u) v)/du)^T w
// S(u) = w~^T J(u) v is differentiated with respect to the linearisation state u:
// every flux is evaluated on hyper-dual numbers (value, D+2 seeded partials, the
// directional derivative along the traces of v, its partials), contracted with the
// transposed test (volume) or transposed lift (faces) of w~ and mapped back through the
// transposed traces.  Same output factors and scratch layout as the adjoint kernels.
template <class T, int D, int P>
__global__ void __launch_bounds__(128) face_hess_kernel(DGData<T> d, const T* __restrict__ u,
                                                        const T* __restrict__ v, const T* __restrict__ w,
                                                        T* __restrict__ GT, const T* __restrict__ escale, T osc) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, GEO = O::GEO;
  using H = HD<T, NV>;
  const int64_t n = d.F * NFQ;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int64_t f = idx / NFQ;
  const int q = (int)(idx - f * NFQ);
  const int eL = d.fel[2 * f], eR = d.fel[2 * f + 1];
  const int loc = d.floc[f];
  const int fL = loc & 0xff, fR = (loc >> 8) & 0xff, pR = loc >> 16;
  T nr[D];
#pragma unroll
  for (int k = 0; k < D; ++k) nr[k] = d.fgeo[4 * f + k];
  const T wq = d.fgeo[4 * f + D] * d.Wf[q];
  const T sdL = d.geo[GEO * (int64_t)eL + O::SD];
  const T sdR = eR >= 0 ? d.geo[GEO * (int64_t)eR + O::SD] : T(1);
  const T* bL = d.Bf + ((fL * NPERM) * NFQ + q) * NB;
  const T* bR = d.Bf + ((fR * NPERM + (eR >= 0 ? pR : 0)) * NFQ + q) * NB;
  T uL[NV], tL[NV], uR[NV], tR[NV], gb[NV];
  const T scL = -osc * (escale ? escale[eL] : T(1)) / sdL;
  const T scR = osc * (eR >= 0 && escale ? escale[eR] : T(1)) / sdR;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    T a = 0, b = 0, g = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int64_t o = (int64_t)eL * NV * NB + c * NB + j;
      const T bj = __ldg(bL + j);
      a += bj * u[o];
      b += bj * v[o];
      g += bj * w[o];
    }
    uL[c] = a / sdL;
    tL[c] = b / sdL;
    gb[c] = scL * g;
    uR[c] = tR[c] = T(0);
  }
  if (eR >= 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      T a = 0, b = 0, g = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int64_t o = (int64_t)eR * NV * NB + c * NB + j;
        const T bj = __ldg(bR + j);
        a += bj * u[o];
        b += bj * v[o];
        g += bj * w[o];
      }
      uR[c] = a / sdR;
      tR[c] = b / sdR;
      gb[c] += scR * g;
    }
  }
  T* o = GT + idx * 2 * NV;
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    if (side == 1 && eR < 0) {
#pragma unroll
      for (int c = 0; c < NV; ++c) o[NV + c] = T(0);
      break;
    }
    H L[NV], R[NV], F[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      L[c].v = uL[c];
      L[c].t = tL[c];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        L[c].d[k] = (side == 0 && k == c) ? T(1) : T(0);
        L[c].dt[k] = T(0);
      }
    }
    if (eR >= 0) {
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        R[c].v = uR[c];
        R[c].t = tR[c];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          R[c].d[k] = (side == 1 && k == c) ? T(1) : T(0);
          R[c].dt[k] = T(0);
        }
      }
    } else if (mirror_bc(eR)) {
      ghost_slip_wall<D, H, T>(L, nr, R);
    } else {
      ghost_farfield<D, H, T>(L, nr, d.fs, R);
    }
    roe_flux<D, H, T>(L, R, nr, d.fs.gamma, F);
    const T sc = wq / (side == 0 ? sdL : sdR);
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      T a = 0;
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) a += gb[vv] * F[vv].dt[c];
      o[side * NV + c] = sc * a;
    }
  }
}

template <class T, int D, int P>
__global__ void __launch_bounds__(256) elem_hess_kernel(DGData<T> d, const T* __restrict__ u, const T* __restrict__ v,
                                                        const T* __restrict__ w, const T* __restrict__ GT,
                                                        T* __restrict__ out, const T* __restrict__ escale, T osc) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, ET = O::ET, NVB = O::NVB, NV = O::NV, GEO = O::GEO;
  constexpr bool SM = O::SMEM_BF;
  using H = HD<T, NV>;
  __shared__ T sBv[NQ * NB];
  __shared__ T sDv[D * NQ * NB];
  __shared__ T sBf[SM ? O::NBF : 1];
  __shared__ T su[ET * NVB];
  __shared__ T sv[ET * NVB];
  __shared__ T sw[ET * NVB];
  __shared__ T sU[ET * NQ * NV];
  __shared__ T sgeo[ET * GEO];
  static_assert(ET * NQ <= 256, "one volume point per thread");
  const int64_t e0 = (int64_t)blockIdx.x * ET;
  const int ne = (int)((d.E - e0) < ET ? (d.E - e0) : ET);
  for (int i = threadIdx.x; i < NQ * NB; i += blockDim.x) sBv[i] = d.Bv[i];
  for (int i = threadIdx.x; i < D * NQ * NB; i += blockDim.x) sDv[i] = d.Dv[i];
  if constexpr (SM)
    for (int i = threadIdx.x; i < O::NBF; i += blockDim.x) sBf[i] = d.Bf[i];
  for (int i = threadIdx.x; i < ne * NVB; i += blockDim.x) {
    su[i] = u[e0 * NVB + i];
    sv[i] = v[e0 * NVB + i];
    sw[i] = w[e0 * NVB + i] * osc * (escale ? escale[e0 + i / NVB] : T(1));
  }
  for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) sgeo[i] = d.geo[e0 * GEO + i];
  __syncthreads();
  const int el1 = threadIdx.x / NQ, q1 = threadIdx.x - (threadIdx.x / NQ) * NQ;
  if (threadIdx.x < ne * NQ) {
    const T* ge = sgeo + el1 * GEO;
    const T sd = ge[O::SD];
    H U[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      T a = 0, b = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        a += sBv[q1 * NB + j] * su[el1 * NVB + c * NB + j];
        b += sBv[q1 * NB + j] * sv[el1 * NVB + c * NB + j];
      }
      U[c].v = a / sd;
      U[c].t = b;  // the sqrt(det) factors of trace and test cancel
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        U[c].d[k] = (k == c) ? T(1) : T(0);
        U[c].dt[k] = T(0);
      }
    }
    H F[D][NV];
    euler_flux<D, H, T>(U, d.fs.gamma, F);
    T fb[D * NV];
#pragma unroll
    for (int dd = 0; dd < D; ++dd)
#pragma unroll
      for (int vv = 0; vv < NV; ++vv) {
        T a = 0;
#pragma unroll
        for (int i = 0; i < NB; ++i) a += sDv[(dd * NQ + q1) * NB + i] * sw[el1 * NVB + vv * NB + i];
        fb[dd * NV + vv] = a;
      }
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      T a = 0;
#pragma unroll
      for (int vv = 0; vv < NV; ++vv)
#pragma unroll
        for (int dd = 0; dd < D; ++dd) {
          T fm = ge[dd * D] * F[0][vv].dt[c];
#pragma unroll
          for (int k = 1; k < D; ++k) fm += ge[dd * D + k] * F[k][vv].dt[c];
          a += fb[dd * NV + vv] * fm;
        }
      sU[(el1 * NQ + q1) * NV + c] = a / sd;
    }
  }
  __syncthreads();
  const T* Bf = SM ? sBf : d.Bf;
  for (int it = threadIdx.x; it < ne * NVB; it += blockDim.x) {
    const int el = it / NVB, r = it - el * NVB;
    const int c = r / NB, j = r - c * NB;
    T acc = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc += sBv[q * NB + j] * sU[(el * NQ + q) * NV + c];
    acc += gather_faces_T<T, D, P, SM>(d, Bf, GT, e0 + el, c, j);
    out[e0 * NVB + it] = acc;
  }
}

template <class T, int D, int P>
cudaError_t jvp_state_adjoint_p(const DGData<T>& d, const T* u, const T* v, const T* w, T* out, T* GT,
                                const T* escale, T osc, cudaStream_t st) {
  using O = Ord<D, P>;
  const int64_t nf = d.F * O::NFQ;
  if (nf > 0) face_hess_kernel<T, D, P><<<(unsigned)((nf + 127) / 128), 128, 0, st>>>(d, u, v, w, GT, escale, osc);
  const int64_t eb = (d.E + O::ET - 1) / O::ET;
  elem_hess_kernel<T, D, P><<<(unsigned)eb, 256, 0, st>>>(d, u, v, w, GT, out, escale, osc);
  return cudaGetLastError();
}

// ------------------------------------------- adjoint with respect to the free stream
// theta = (Mach number, flow angle in degrees) enters the operator only through the
// free-stream velocity of the far-field ghost state.  For the far-field faces (indices >= f0)
// this kernel adds to acc[0..1]
//   order 1:  sum_q sum_v gbar_q[v] dF~_v/dtheta_k                       ((dR/dtheta)^T w)
//   order 2:  sum_q sum_v gbar_q[v] d/dtheta_k (dF~_v/dU_L . t_L)          ((d(J t)/dtheta)^T w)
// with gbar_q[v] = -osc |f| w_q / sqrt|det A_L| sum_i phi_i(x_q) w[e_L][v][i] (the transposed lift
// of w, the face term of R at the L element) and t_L the trace of t.  Jet numbers seeded on
// the velocity give the first derivatives, hyper-dual numbers (velocity seeds, tangent t_L)
// the mixed second ones.  dvel = {dvel/dMach (D), dvel/dalpha (D)}.  osc_dev (nullable)
// multiplies osc.  Fixed-order sum: per-block partials, the last block adds them to acc.
template <class T, int D, int P, int ORDER>
__global__ void __launch_bounds__(128) param_adjoint_kernel(DGData<T> d, int64_t f0, const T* __restrict__ u,
                                                            const T* __restrict__ t, const T* __restrict__ w,
                                                            double osc, const double* __restrict__ osc_dev,
                                                            double dvm0, double dvm1, double dva0, double dva1,
                                                            double* __restrict__ acc, double* __restrict__ partials,
                                                            unsigned* counter) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, GEO = O::GEO;
  __shared__ double red[2][4];
  __shared__ bool last;
  double a0 = 0.0, a1 = 0.0;
  const double os = osc * (osc_dev ? *osc_dev : 1.0);
  const int64_t n = (d.F - f0) * NFQ;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = f0 + idx / NFQ;
    const int q = (int)(idx % NFQ);
    if (-d.fel[2 * f + 1] != PCEXP_BC_FARFIELD) continue;
    const int eL = d.fel[2 * f];
    const int fL = d.floc[f] & 0xff;
    T nr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) nr[k] = d.fgeo[4 * f + k];
    const T isd = d.geo[GEO * (int64_t)eL + O::ISD];
    const T* be = d.Bf + ((fL * NPERM) * NFQ + q) * NB;
    const T wl = d.fgeo[4 * f + D] * d.Wf[q];
    T uL[NV], tL[NV], gb[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T a = 0, b = 0, c = 0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const T bj = __ldg(be + j);
        const int64_t o = (int64_t)eL * NV * NB + v * NB + j;
        a += bj * u[o];
        if (ORDER == 2) b += bj * t[o];
        c += bj * w[o];
      }
      uL[v] = a * isd;
      tL[v] = b * isd;
      gb[v] = (T)(-os) * wl * isd * c;
    }
    const double dm[3] = {dvm0, dvm1, 0.0}, da[3] = {dva0, dva1, 0.0};
    if constexpr (ORDER == 1) {
      using J = Jet<T, 2>;
      J L[NV], R[NV], F[NV], vi[3];
#pragma unroll
      for (int v = 0; v < NV; ++v) L[v] = Lift<J, T>::of(uL[v]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        vi[k].v = d.fs.vel[k];
        vi[k].d[0] = (T)dm[k];
        vi[k].d[1] = (T)da[k];
      }
      ghost_farfield_v<D, J, T>(L, nr, d.fs.gamma, d.fs.rho, d.fs.p, vi, R);
      roe_flux<D, J, T>(L, R, nr, d.fs.gamma, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        a0 += (double)gb[v] * (double)F[v].d[0];
        a1 += (double)gb[v] * (double)F[v].d[1];
      }
    } else {
      using H = HD<T, 2>;
      H L[NV], R[NV], F[NV], vi[3];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        L[v] = Lift<H, T>::of(uL[v]);
        L[v].t = tL[v];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        vi[k] = Lift<H, T>::of(d.fs.vel[k]);
        vi[k].d[0] = (T)dm[k];
        vi[k].d[1] = (T)da[k];
      }
      ghost_farfield_v<D, H, T>(L, nr, d.fs.gamma, d.fs.rho, d.fs.p, vi, R);
      roe_flux<D, H, T>(L, R, nr, d.fs.gamma, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        a0 += (double)gb[v] * (double)F[v].dt[0];
        a1 += (double)gb[v] * (double)F[v].dt[1];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a0;
    red[1][threadIdx.x >> 5] = a1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = 0, b1 = 0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
      b0 += red[0][ww];
      b1 += red[1][ww];
    }
    partials[2 * blockIdx.x] = b0;
    partials[2 * blockIdx.x + 1] = b1;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    double b0 = 0, b1 = 0;
    for (unsigned i = 0; i < gridDim.x; ++i) {
      b0 += __ldcg(partials + 2 * i);
      b1 += __ldcg(partials + 2 * i + 1);
    }
    acc[0] += b0;
    acc[1] += b1;
    *counter = 0;
  }
}

template <class T, int D, int P>
cudaError_t param_adjoint_p(const DGData<T>& d, int64_t f0, int order, const T* u, const T* t, const T* w, double osc,
                            const double* osc_dev, const double* dvel, double* acc, double* partials,
                            unsigned* counter, cudaStream_t st) {
  const int64_t n = (d.F - f0) * Ord<D, P>::NFQ;
  if (n <= 0) return cudaSuccess;
  int64_t g = (n + 127) / 128;
  if (g > RED_BLOCKS) g = RED_BLOCKS;
  if (order == 1)
    param_adjoint_kernel<T, D, P, 1><<<(unsigned)g, 128, 0, st>>>(d, f0, u, t, w, osc, osc_dev, dvel[0], dvel[1],
                                                                   dvel[2], dvel[3], acc, partials, counter);
  else
    param_adjoint_kernel<T, D, P, 2><<<(unsigned)g, 128, 0, st>>>(d, f0, u, t, w, osc, osc_dev, dvel[0], dvel[1],
                                                                   dvel[2], dvel[3], acc, partials, counter);
  return cudaGetLastError();
}

// ------------------------------------------------------------ output functionals
// fixed-order sum of one double per thread into *value (last-block reduction)
PCEXP_DEV void block_sum_last(double acc, double* value, double* partials, unsigned* counter, bool sqrt_out) {
  __shared__ double red[8];
  __shared__ bool last;
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
    *value = sqrt_out ? sqrt(b) : b;
    *counter = 0;
  }
}

// Pressure force on the slip walls along the unit direction a:
//   J = sum_{wall faces} sum_q |f| w_q p(U_L(x_q)) (n . a),  p = (gamma-1)(E - |m|^2 / (2 rho)),
// with its gradient dJ/du (trace transpose of dp/dU); value by a fixed-order reduction.
template <class T, int D, int P>
__global__ void __launch_bounds__(256) wall_force_kernel(DGData<T> d, int64_t f0, const T* __restrict__ u, double ax,
                                                         double ay, double az, double* __restrict__ grad,
                                                         double* __restrict__ value, double* __restrict__ partials,
                                                         unsigned* counter) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NFQ = O::NFQ, NV = O::NV, NPERM = O::NPERM, GEO = O::GEO;
  const double a3[3] = {ax, ay, az};
  double acc = 0;
  const T gm = d.fs.gamma - T(1);
  for (int64_t f = f0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < d.F; f += (int64_t)gridDim.x * blockDim.x) {
    if (-d.fel[2 * f + 1] != PCEXP_BC_SLIP_WALL) continue;
    const int e = d.fel[2 * f];
    const int fl = d.floc[f] & 0xff;
    double na = 0;
    for (int k = 0; k < D; ++k) na += (double)d.fgeo[4 * f + k] * a3[k];
    const double meas = (double)d.fgeo[4 * f + D];
    const double isd = (double)d.geo[GEO * (int64_t)e + O::ISD];
    double g[NV * NB];
    for (int k = 0; k < NV * NB; ++k) g[k] = 0.0;
    for (int q = 0; q < NFQ; ++q) {
      const T* b = d.Bf + ((fl * NPERM) * NFQ + q) * NB;
      double U[NV];
      for (int c = 0; c < NV; ++c) {
        double a = 0;
        for (int j = 0; j < NB; ++j) a += (double)b[j] * (double)u[(int64_t)e * NV * NB + c * NB + j];
        U[c] = a * isd;
      }
      double vel[D], v2 = 0;
      for (int k = 0; k < D; ++k) {
        vel[k] = U[1 + k] / U[0];
        v2 += vel[k] * vel[k];
      }
      const double p = (double)gm * (U[NV - 1] - 0.5 * U[0] * v2);
      const double wq = meas * (double)d.Wf[q] * na;
      acc += wq * p;
      double dp[NV];
      dp[0] = (double)gm * 0.5 * v2;
      for (int k = 0; k < D; ++k) dp[1 + k] = -(double)gm * vel[k];
      dp[NV - 1] = (double)gm;
      for (int c = 0; c < NV; ++c)
        for (int j = 0; j < NB; ++j) g[c * NB + j] += wq * dp[c] * (double)b[j] * isd;
    }
    // on the 2D walls at most two wall faces meet in one element, and a + b is the same
    // in either order; elements with three or more wall faces sum in arrival order
    if (grad)
      for (int k = 0; k < NV * NB; ++k) atomicAdd(grad + (int64_t)e * NV * NB + k, g[k]);
  }
  block_sum_last(acc, value, partials, counter, false);
}

// Vortex-error functional J = ||U_h - U_exact||_L2 (all conservative variables) with the
// exact state of the translated isentropic vortex at the volume points, and the
// unnormalised gradient sum_q w_q (U_h - U_ex)_v dU_h/du_{e,v,j} (scaled by 1/J afterwards).
// prm: eps, x_c, y_c, period (<= 0: none), t.  The field lies in the x-y plane.
template <class T, int D, int P>
__global__ void __launch_bounds__(256) vortex_error_kernel(DGData<T> d, const T* __restrict__ u,
                                                           const double* __restrict__ xq, double eps, double xc,
                                                           double yc, double period, double t,
                                                           double* __restrict__ grad, double* __restrict__ value,
                                                           double* __restrict__ partials, unsigned* counter) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, NV = O::NV, GEO = O::GEO;
  double acc = 0;
  const double g = (double)d.fs.gamma, rinf = (double)d.fs.rho, pinf = (double)d.fs.p;
  const double u0 = (double)d.fs.vel[0], v0 = (double)d.fs.vel[1];
  const double Tinf = pinf / rinf, pi = 3.141592653589793238462643383279502884;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.E; e += (int64_t)gridDim.x * blockDim.x) {
    const double sd = (double)d.geo[GEO * e + O::SD];
    double ge[NV * NB];
    for (int k = 0; k < NV * NB; ++k) ge[k] = 0.0;
    for (int q = 0; q < NQ; ++q) {
      double dx = xq[(e * NQ + q) * D] - (xc + u0 * t), dy = xq[(e * NQ + q) * D + 1] - (yc + v0 * t);
      if (period > 0) {
        dx -= period * nearbyint(dx / period);
        dy -= period * nearbyint(dy / period);
      }
      const double r2 = dx * dx + dy * dy;
      const double fe = eps / (2 * pi) * exp(0.5 * (1 - r2));
      const double uu = u0 - fe * dy, vv = v0 + fe * dx;
      const double Tv = Tinf - (g - 1) * eps * eps / (8 * g * pi * pi) * exp(1 - r2);
      const double rho = rinf * pow(Tv / Tinf, 1.0 / (g - 1));
      const double p = rho * Tv;
      double Ue[NV];
      Ue[0] = rho;
      Ue[1] = rho * uu;
      Ue[2] = rho * vv;
      if (D == 3) Ue[3] = 0.0;
      Ue[NV - 1] = p / (g - 1) + 0.5 * rho * (uu * uu + vv * vv);
      const double wq = (double)d.Wv[q] * sd * sd;  // |det A| w^_q
      for (int c = 0; c < NV; ++c) {
        double a = 0;
        for (int j = 0; j < NB; ++j) a += (double)d.Bv[q * NB + j] * (double)u[e * NV * NB + c * NB + j];
        const double diff = a / sd - Ue[c];
        acc += wq * diff * diff;
        for (int j = 0; j < NB; ++j) ge[c * NB + j] += wq * diff * (double)d.Bv[q * NB + j] / sd;
      }
    }
    if (grad)
      for (int k = 0; k < NV * NB; ++k) grad[e * NV * NB + k] = ge[k];
  }
  block_sum_last(acc, value, partials, counter, true);
}

// Partials of the vortex-error functional with respect to theta = (Mach, alpha in degrees,
// eps) at a fixed state: out[0] = sum w_q |U_h - U_ex|^2 (= J^2), out[1 + k] = sum w_q
// (U_h - U_ex) . dU_ex/dtheta_k, so dJ/dtheta_k = -out[1 + k] / J.  The exact state is
// evaluated on Jet numbers seeded with the free-stream velocity derivatives (dvel: d/dMach
// x, y, then d/dalpha x, y) and with eps.  Fixed-order last-block sums.
template <class T, int D, int P>
__global__ void __launch_bounds__(256) vortex_param_grad_kernel(DGData<T> d, const T* __restrict__ u,
                                                                const double* __restrict__ xq, double eps, double xc,
                                                                double yc, double period, double t, double dvm0,
                                                                double dvm1, double dva0, double dva1,
                                                                double* __restrict__ out, double* __restrict__ partials,
                                                                unsigned* counter) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NQ = O::NQ, NV = O::NV, GEO = O::GEO;
  using J = Jet<double, 3>;
  __shared__ double red[4][8];
  __shared__ bool last;
  double acc[4] = {0, 0, 0, 0};
  const double g = (double)d.fs.gamma, rinf = (double)d.fs.rho, pinf = (double)d.fs.p;
  const double Tinf = pinf / rinf, pi = 3.141592653589793238462643383279502884;
  J u0, v0, ep;
  u0.v = (double)d.fs.vel[0];
  u0.d[0] = dvm0;
  u0.d[1] = dva0;
  u0.d[2] = 0.0;
  v0.v = (double)d.fs.vel[1];
  v0.d[0] = dvm1;
  v0.d[1] = dva1;
  v0.d[2] = 0.0;
  ep.v = eps;
  ep.d[0] = ep.d[1] = 0.0;
  ep.d[2] = 1.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.E; e += (int64_t)gridDim.x * blockDim.x) {
    const double sd = (double)d.geo[GEO * e + O::SD];
    for (int q = 0; q < NQ; ++q) {
      J dx = (xq[(e * NQ + q) * D] - xc) - u0 * t;
      J dy = (xq[(e * NQ + q) * D + 1] - yc) - v0 * t;
      if (period > 0) {
        dx = dx - period * nearbyint(dx.v / period);
        dy = dy - period * nearbyint(dy.v / period);
      }
      const J r2 = dx * dx + dy * dy;
      const J fe = ep * (1.0 / (2 * pi)) * exp_s(0.5 * (1.0 - r2));
      const J uu = u0 - fe * dy, vv = v0 + fe * dx;
      const J Tv = Tinf - ((g - 1) / (8 * g * pi * pi)) * (ep * ep) * exp_s(1.0 - r2);
      const J rho = rinf * pow_s(Tv * (1.0 / Tinf), 1.0 / (g - 1));
      const J p = rho * Tv;
      J Ue[NV];
      Ue[0] = rho;
      Ue[1] = rho * uu;
      Ue[2] = rho * vv;
      if (D == 3) Ue[3] = Lift<J, double>::of(0.0);
      Ue[NV - 1] = p * (1.0 / (g - 1)) + 0.5 * rho * (uu * uu + vv * vv);
      const double wq = (double)d.Wv[q] * sd * sd;
      for (int c = 0; c < NV; ++c) {
        double a = 0;
        for (int j = 0; j < NB; ++j) a += (double)d.Bv[q * NB + j] * (double)u[e * NV * NB + c * NB + j];
        const double diff = a / sd - Ue[c].v;
        acc[0] += wq * diff * diff;
        for (int k = 0; k < 3; ++k) acc[1 + k] += wq * diff * Ue[c].d[k];
      }
    }
  }
  for (int k = 0; k < 4; ++k) {
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double b = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[k][w];
      partials[4 * blockIdx.x + k] = b;
    }
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double b = 0;
      for (unsigned i = 0; i < gridDim.x; ++i) b += __ldcg(partials + 4 * i + k);
      out[k] = b;
    }
    *counter = 0;
  }
}

template <class T, int D, int P>
cudaError_t vortex_param_grad_p(const DGData<T>& d, const T* u, const double* xq, const double* prm, const double* dvel,
                                double* out, double* partials, unsigned* counter, cudaStream_t st) {
  int64_t nb = (d.E + 255) / 256;
  if (nb > RED_BLOCKS / 2) nb = RED_BLOCKS / 2;
  vortex_param_grad_kernel<T, D, P><<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, st>>>(
      d, u, xq, prm[0], prm[1], prm[2], prm[3], prm[4], dvel[0], dvel[1], dvel[2], dvel[3], out, partials, counter);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ time step
// dt_e = CFL h_e / ((2p+1)(|v| + c)) with v, c at the element centroid (Eq. x3d).
template <class T, int D, int P>
__global__ void __launch_bounds__(256) local_dt_kernel(DGData<T> d, const T* __restrict__ u,
                                                       const double* cfl_dev, double cfl_host,
                                                       T* __restrict__ dte, double* __restrict__ dtmin,
                                                       double* __restrict__ partials,
                                                       unsigned* __restrict__ counter) {
  using O = Ord<D, P>;
  constexpr int NB = O::NB, NV = O::NV, GEO = O::GEO;
  __shared__ double red[8];
  __shared__ bool last;
  const double cfl = cfl_dev ? *cfl_dev : cfl_host;
  double mn = DBL_MAX;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.E_loc; e += (int64_t)gridDim.x * blockDim.x) {
    const T isd = d.geo[GEO * e + O::ISD];
    double U[NV];
    for (int v = 0; v < NV; ++v) {
      T a = 0;
      for (int j = 0; j < NB; ++j) a += d.Bc[j] * u[e * NV * NB + v * NB + j];
      U[v] = (double)(a * isd);
    }
    const double gam = (double)d.fs.gamma;
    double v2 = 0;
    for (int k = 0; k < D; ++k) v2 += (U[1 + k] / U[0]) * (U[1 + k] / U[0]);
    const double p = (gam - 1.0) * (U[NV - 1] - 0.5 * U[0] * v2);
    const double c = sqrt(gam * p / U[0]);
    if (d.rot) {  // the velocity relative to the rotating frame carries the waves
      v2 = 0;
      for (int k = 0; k < D; ++k) {
        const double vk = U[1 + k] / U[0] - (double)d.vrc[e * D + k];
        v2 += vk * vk;
      }
    }
    const double h = (double)d.geo[GEO * e + O::HE];
    const double dt = cfl * h / ((2 * d.p + 1) * (sqrt(v2) + c));
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

// ------------------------------------------------------------------ launchers
// The launchers below dispatch on p for one dimension D; orders above PMAX<D> are
// rejected when a context is created.
template <int D> constexpr int PMAX = D == 2 ? 3 : 2;

#define PCEXP_PSWITCH(D, CALL)                       \
  switch (d.p) {                                     \
    case 0: { constexpr int P_ = 0; return CALL; }   \
    case 1: { constexpr int P_ = 1; return CALL; }   \
    case 2: { constexpr int P_ = 2; return CALL; }   \
    case 3: {                                        \
      if constexpr (PMAX<D> >= 3) {                  \
        constexpr int P_ = PMAX<D> >= 3 ? 3 : 0;     \
        return CALL;                                 \
      }                                              \
      break;                                         \
    }                                                \
  }                                                  \
  return cudaErrorInvalidValue;

template <class T, int D>
cudaError_t launch_dg_operator_d(const DGData<T>& d, const T* u, const T* du, T* out, T* G, const T* escale,
                                 const int* skip, cudaStream_t st, const cudaEvent_t* ev, const double* oscale) {
  PCEXP_PSWITCH(D, (dg_op_p<T, D, P_>(d, u, du, out, G, escale, skip, oscale, st, ev)))
}
template <class T, int D>
cudaError_t launch_linearize_d(const DGData<T>& d, const T* u, LinData<T> lin, bool faces_only, cudaStream_t st) {
  PCEXP_PSWITCH(D, (linearize_p<T, D, P_>(d, u, lin, faces_only, st)))
}
template <class T, int D>
cudaError_t launch_jac_apply_d(const DGData<T>& d, LinData<T> lin, const T* u_elem, const T* dv, T* out, T* G,
                               const T* escale, const int* skip, const double* oscale, cudaStream_t st,
                               const cudaEvent_t* ev, bool face_tan) {
  PCEXP_PSWITCH(D, (jac_apply_p<T, D, P_>(d, lin, u_elem, dv, out, G, escale, skip, oscale, st, ev, face_tan)))
}
template <int D>
cudaError_t launch_tan_tables_d(const DGData<float>& d, cudaStream_t st) {
  PCEXP_PSWITCH(D, (tan_tables_p<D, P_>(d, st)))
}
template <class T, int D>
cudaError_t launch_jac_adjoint_d(const DGData<T>& d, LinData<T> lin, const T* w, T* out, T* GT, const T* escale,
                                 T osc, cudaStream_t st) {
  PCEXP_PSWITCH(D, (jac_adjoint_p<T, D, P_>(d, lin, w, out, GT, escale, osc, st)))
}
template <class T, int D>
cudaError_t launch_jvp_state_adjoint_d(const DGData<T>& d, const T* u, const T* v, const T* w, T* out, T* GT,
                                       const T* escale, T osc, cudaStream_t st) {
  PCEXP_PSWITCH(D, (jvp_state_adjoint_p<T, D, P_>(d, u, v, w, out, GT, escale, osc, st)))
}

template <class T, int D>
cudaError_t launch_param_adjoint_d(const DGData<T>& d, int64_t f0, int order, const T* u, const T* t, const T* w,
                                   double osc, const double* osc_dev, const double* dvel, double* acc,
                                   double* partials, unsigned* counter, cudaStream_t st) {
  PCEXP_PSWITCH(D, (param_adjoint_p<T, D, P_>(d, f0, order, u, t, w, osc, osc_dev, dvel, acc, partials, counter, st)))
}

template <class T, int D, int P>
cudaError_t wall_force_p(const DGData<T>& d, int64_t f0, const T* u, double ax, double ay, double az, double* grad,
                         double* value, double* partials, unsigned* counter, cudaStream_t st) {
  const int64_t nb = d.F - f0;
  unsigned g = (unsigned)((nb + 255) / 256);
  if (g < 1) g = 1;
  if (g > RED_BLOCKS) g = RED_BLOCKS;
  wall_force_kernel<T, D, P><<<g, 256, 0, st>>>(d, f0, u, ax, ay, az, grad, value, partials, counter);
  return cudaGetLastError();
}
template <class T, int D>
cudaError_t launch_wall_force_d(const DGData<T>& d, int64_t f0, const T* u, double ax, double ay, double az,
                                double* grad, double* value, double* partials, unsigned* counter, cudaStream_t st) {
  PCEXP_PSWITCH(D, (wall_force_p<T, D, P_>(d, f0, u, ax, ay, az, grad, value, partials, counter, st)))
}

template <class T, int D, int P>
cudaError_t vortex_error_p(const DGData<T>& d, const T* u, const double* xq, const double* prm, double* grad,
                           double* value, double* partials, unsigned* counter, cudaStream_t st) {
  int64_t nb = (d.E + 255) / 256;
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  vortex_error_kernel<T, D, P><<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, st>>>(
      d, u, xq, prm[0], prm[1], prm[2], prm[3], prm[4], grad, value, partials, counter);
  return cudaGetLastError();
}
template <class T, int D>
cudaError_t launch_vortex_error_d(const DGData<T>& d, const T* u, const double* xq, const double* prm, double* grad,
                                  double* value, double* partials, unsigned* counter, cudaStream_t st) {
  PCEXP_PSWITCH(D, (vortex_error_p<T, D, P_>(d, u, xq, prm, grad, value, partials, counter, st)))
}

template <class T, int D>
cudaError_t launch_vortex_param_grad_d(const DGData<T>& d, const T* u, const double* xq, const double* prm,
                                       const double* dvel, double* out, double* partials, unsigned* counter,
                                       cudaStream_t st) {
  PCEXP_PSWITCH(D, (vortex_param_grad_p<T, D, P_>(d, u, xq, prm, dvel, out, partials, counter, st)))
}

template <class T, int D, int P>
cudaError_t local_dt_p(const DGData<T>& d, const T* u, const double* cfl_dev, double cfl, T* dte, double* dtmin,
                       double* partials, unsigned* counter, cudaStream_t st) {
  int64_t nb = (d.E + 255) / 256;
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  local_dt_kernel<T, D, P><<<(unsigned)nb, 256, 0, st>>>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter);
  return cudaGetLastError();
}
template <class T, int D>
cudaError_t launch_local_dt_d(const DGData<T>& d, const T* u, const double* cfl_dev, double cfl, T* dte,
                              double* dtmin, double* partials, unsigned* counter, cudaStream_t st) {
  PCEXP_PSWITCH(D, (local_dt_p<T, D, P_>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter, st)))
}

#undef PCEXP_PSWITCH

#define PCEXP_INST_D(T, D)                                                                                         \
  template cudaError_t launch_dg_operator_d<T, D>(const DGData<T>&, const T*, const T*, T*, T*, const T*,           \
                                                  const int*, cudaStream_t, const cudaEvent_t*, const double*);    \
  template cudaError_t launch_linearize_d<T, D>(const DGData<T>&, const T*, LinData<T>, bool, cudaStream_t);       \
  template cudaError_t launch_jac_apply_d<T, D>(const DGData<T>&, LinData<T>, const T*, const T*, T*, T*,          \
                                                const T*, const int*, const double*, cudaStream_t,                 \
                                                const cudaEvent_t*, bool);                                         \
  template cudaError_t launch_jac_adjoint_d<T, D>(const DGData<T>&, LinData<T>, const T*, T*, T*, const T*, T,     \
                                                  cudaStream_t);                                                   \
  template cudaError_t launch_jvp_state_adjoint_d<T, D>(const DGData<T>&, const T*, const T*, const T*, T*, T*,    \
                                                        const T*, T, cudaStream_t);                                \
  template cudaError_t launch_wall_force_d<T, D>(const DGData<T>&, int64_t, const T*, double, double, double,      \
                                                 double*, double*, double*, unsigned*, cudaStream_t);              \
  template cudaError_t launch_vortex_error_d<T, D>(const DGData<T>&, const T*, const double*, const double*,       \
                                                   double*, double*, double*, unsigned*, cudaStream_t);            \
  template cudaError_t launch_local_dt_d<T, D>(const DGData<T>&, const T*, const double*, double, T*, double*,     \
                                               double*, unsigned*, cudaStream_t);                                  \
  template cudaError_t launch_vortex_param_grad_d<T, D>(const DGData<T>&, const T*, const double*, const double*,   \
                                                        const double*, double*, double*, unsigned*, cudaStream_t); \
  template cudaError_t launch_param_adjoint_d<T, D>(const DGData<T>&, int64_t, int, const T*, const T*, const T*,  \
                                                    double, const double*, const double*, double*, double*,        \
                                                    unsigned*, cudaStream_t);

}  // namespace pcexp
