// Krylov kernels: Arnoldi with classical Gram-Schmidt run twice (CGS2) over
// the tall-skinny basis, the FP64 phi-function of the small Hessenberg
// matrix, and the fused PCEXP update (Sec. 2.2 of the paper, Eq. vm-vm2,
// final; Eq. s9, s10).
//
// Basis storage: V[i] holds an unnormalised vector z_i and KState.s[i] its
// scale, v_i = s_i z_i, so normalisation costs no extra pass.  One Arnoldi
// column j runs as
//   w   = s_j J z_j = J v_j          (DG tangent-linear kernel, scale on its output)
//   P   : h_i  = s_i <z_i, w>,  ||w||                          (read V_j, w)
//   UP  : w   -= sum_i s_i^2 <z_i,w> z_i; h2_i = s_i <z_i, w>  (read V_j, w; write w)
//   UN  : z_{j+1} = w - sum_i s_i^2 <z_i,w> z_i; h_{j+1,j} = ||z_{j+1}||, s_{j+1} = 1/h_{j+1,j}
// so every stored z_i has the size of ||J|| (no growth like ||J||^i, which would
// overflow FP32 storage).  The selective form (FP32-mixed default) runs a column as
//   P, U1: z_{j+1} = w - sum_i s_i^2 <z_i,w> z_i, ||z_{j+1}||       (read V_j, w; write z_{j+1})
// and keeps that first update when ||z_{j+1}|| >= ||w|| / sqrt(2); otherwise the second
// pass follows, P2 (h2 = V_j^T z_{j+1}) and UN in place on z_{j+1}.  The second pass's
// launches leave at once in the columns that keep their first update.
// Each streaming kernel writes per-block partial sums; the last block to
// finish (atomic ticket) reduces them in a fixed order and applies the scalar
// update, so results are deterministic and no extra launch is needed.
// Partial products are accumulated in FP64 (FP64 form) or in compensated FP32
// pairs converted to FP64 once per warp (FP32-mixed form).
#include <cooperative_groups.h>
#include <cfloat>

#include "kernels.h"

namespace pcexp {

// Elements per thread per row-loop iteration: one 16-byte load (double2 / float4).
template <class T> struct VecN {
  static constexpr int N = 16 / sizeof(T);
};

template <class T, int VN>
PCEXP_DEV void load_vec(const T* p, T (&x)[VN]) {
  if constexpr (sizeof(T) == 8) {
    double2 a = *reinterpret_cast<const double2*>(p);
    x[0] = a.x;
    x[1] = a.y;
  } else {
    float4 a = *reinterpret_cast<const float4*>(p);
    x[0] = a.x;
    x[1] = a.y;
    x[2] = a.z;
    x[3] = a.w;
  }
}
template <class T, int VN>
PCEXP_DEV void store_vec(T* p, const T (&x)[VN]) {
  if constexpr (sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
}

// Dot-product accumulator.  FP64 form: a double.  FP32-mixed form: an unevaluated
// float pair hi + lo updated with Knuth's TwoSum, so per-thread sums and the warp
// shuffle tree run on the FP32 pipe (GB300 has 1/62 the FP64 rate) while keeping
// about twice FP32 precision; each warp converts to FP64 once per column.
// Both are 8 bytes, so block partial sums are stored in the same FP64-sized slots; the
// float pair stays a pair through the block and grid reductions and is converted to
// FP64 once per column (each FP64 warp instruction costs tens of cycles here).
template <class T> struct Acc;
template <> struct Acc<double> {
  double s;
  PCEXP_DEV void zero() { s = 0.0; }
  PCEXP_DEV void add(double x) { s += x; }
  PCEXP_DEV void add_acc(const Acc& o) { s += o.s; }
  PCEXP_DEV void add_partner(int o) { s += __shfl_xor_sync(0xffffffffu, s, o); }
  PCEXP_DEV void shfl_from(const Acc& src, int o) { s = __shfl_xor_sync(0xffffffffu, src.s, o); }
  PCEXP_DEV double value() const { return s; }
};
template <> struct Acc<float> {
  float hi, lo;
  PCEXP_DEV void zero() { hi = lo = 0.f; }
  PCEXP_DEV void add(float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
  }
  PCEXP_DEV void add_acc(const Acc& o) {
    add(o.hi);
    lo += o.lo;
  }
  PCEXP_DEV void add_partner(int o) {
    Acc p;
    p.shfl_from(*this, o);
    add_acc(p);
  }
  PCEXP_DEV void shfl_from(const Acc& src, int o) {
    hi = __shfl_xor_sync(0xffffffffu, src.hi, o);
    lo = __shfl_xor_sync(0xffffffffu, src.lo, o);
  }
  PCEXP_DEV double value() const { return (double)hi + (double)lo; }
};
static_assert(sizeof(Acc<float>) == 8 && sizeof(Acc<double>) == 8, "partials are 8-byte slots");

// sum_v a[v] * b[v] in T (FMA chain over one 16-byte chunk)
template <class T, int VN>
PCEXP_DEV T dot_vec(const T (&a)[VN], const T (&b)[VN]) {
  T s = 0;
#pragma unroll
  for (int v = 0; v < VN; ++v) s = fma(a[v], b[v], s);
  return s;
}

// acc += <a, b> over one chunk.  FP64: FMAs straight into the accumulator (one FP64
// instruction per element; the FP64 pipe bounds these passes).  FP32: the chunk's FMA chain,
// then one compensated addition.
template <class T, int VN>
PCEXP_DEV void acc_dot(Acc<T>& acc, const T (&a)[VN], const T (&b)[VN]) {
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int v = 0; v < VN; ++v) acc.s = fma(a[v], b[v], acc.s);
  } else {
    acc.add(dot_vec<T, VN>(a, b));
  }
}

// Selective re-orthogonalisation (Daniel, Gragg, Kaufman & Stewart 1976): the first pass
// is kept alone when ||w_1|| >= ||w|| / sqrt(2), i.e. when it cancelled less than that.
constexpr double DGKS_KAPPA = 0.70710678118654752440;

// Stage logic of the last block: per-column entries in parallel, scalars on thread 0.
//   PROJ      h = V^T w: column j of H (and of H1), update coefficients, ||w||
//   UPD_PROJ  h2 = V^T w_1 after the update: added to column j, new coefficients
//   PROJ2     the same for the selective form's separate second projection
//   UPD1      the selective form's first update w_1 = w - V h alone, with ||w_1||: keep it as
//             z_{j+1} (skip2) when it cancelled less than DGKS_KAPPA, else leave the column
//             to PROJ2 + UPD_NORM
//   UPD_NORM  z_{j+1} = w_1 - V h2, h_{j+1,j} = ||z_{j+1}||, breakdown test
PCEXP_DEV void cgs_finalize(int mode, int j, const double* dots, KState* ks, double eta) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  if (mode == CGS_PROJ || mode == CGS_UPD_PROJ || mode == CGS_PROJ2) {
    // w = J v_j is already normalised by s_j (applied by the J v kernel)
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      const double si = ks->s[i];
      const double h = si * dots[i];
      if (!isfinite(h)) bad = 1;
      if (mode == CGS_PROJ) {
        ks->H[i * MMAX + j] = h;
        ks->H1[i * MMAX + j] = h;
      } else {
        ks->H[i * MMAX + j] += h;
      }
      ks->coef[i] = si * h;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (mode == CGS_PROJ) ks->wnorm0 = sqrt(dots[j + 1]);
      if (bad) {
        ks->err = 1;
        ks->done = 1;
      }
    }
    return;
  }
  if (threadIdx.x != 0) return;
  if (mode == CGS_NORM) {
    const double beta = sqrt(dots[0]);
    ks->beta = beta;
    ks->k = 0;
    if (!isfinite(beta)) {
      ks->err = 1;
      ks->done = 1;
    } else if (beta == 0.0) {
      ks->done = 1;
    } else {
      ks->s[0] = 1.0 / beta;
      ks->done = 0;
    }
    return;
  }
  if (mode == CGS_UPD1) {
    // a non-finite or zero norm takes the second pass, whose norm test reports it; a kept
    // first pass has ||w_1|| >= ||w|| / sqrt(2) > eta ||w||, so it needs no breakdown test
    const double n1 = sqrt(dots[0]);
    const bool keep1 = isfinite(n1) && n1 > 0.0 && n1 >= DGKS_KAPPA * ks->wnorm0;
    ks->skip2 = keep1 ? 1 : 0;
    if (keep1) {
      ks->H[(j + 1) * MMAX + j] = n1;
      ks->k = j + 1;
      ks->s[j + 1] = 1.0 / n1;
    }
    return;
  }
  // CGS_UPD_NORM
  const double hn = sqrt(dots[0]);
  ks->pass2 |= 1u << j;
  ks->H[(j + 1) * MMAX + j] = hn;
  ks->k = j + 1;
  if (!isfinite(hn)) {
    ks->err = 1;
    ks->done = 1;
  } else if (hn == 0.0 || hn <= eta * ks->wnorm0) {
    ks->done = 1;  // happy breakdown: K_{j+1} is invariant
  } else {
    ks->s[j + 1] = 1.0 / hn;
  }
}

// The passes that belong to a column's second Gram-Schmidt pass leave at once when the
// selective form kept the first pass.
PCEXP_DEV bool cgs_skipped(int fmode, const KState* ks) {
  return (fmode == CGS_PROJ2 || fmode == CGS_UPD_NORM) && ks->skip2;
}

// Warp reduction of NC accumulators at once (NC a power of two <= 32): plain
// butterfly levels until NC values remain per lane pair group, then transpose levels
// in which each lane keeps half of its columns and receives the partner's other half.
// Afterwards lane l holds the warp sum of column (l mod NC): NC - 1 + (5 - log2 NC) NC
// additions per lane instead of 5 NC.  Fixed order, so deterministic.
template <class T, int NC, int L, int O>
PCEXP_DEV void transpose_level(Acc<T> (&a)[NC], int lane) {
  if constexpr (L >= 2) {
    const bool upper = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < L / 2; ++i) {
      Acc<T> send = upper ? a[i] : a[i + L / 2];
      Acc<T> keep = upper ? a[i + L / 2] : a[i];
      Acc<T> recv;
      recv.shfl_from(send, O);
      keep.add_acc(recv);
      a[i] = keep;
    }
    transpose_level<T, NC, L / 2, O / 2>(a, lane);
  }
}

template <class T, int NC>
PCEXP_DEV Acc<T> warp_reduce_columns(Acc<T> (&a)[NC], int lane) {
  constexpr int LOGNC = NC >= 32 ? 5 : NC >= 16 ? 4 : NC >= 8 ? 3 : NC >= 4 ? 2 : NC >= 2 ? 1 : 0;
  static_assert((1 << LOGNC) == NC, "NC must be a power of two <= 32");
#pragma unroll
  for (int o = 16; o >= NC; o >>= 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c].add_partner(o);
  }
  transpose_level<T, NC, NC, NC / 2>(a, lane);
  return a[0];
}

// Row Gram-Schmidt pass (NORM, PROJ, UPD_PROJ, UPD_NORM): every thread owns whole 16-byte
// chunks of rows and accumulates all columns for them; the launch bounds hold it at 128
// registers so that two blocks share an SM.
// MODE is how the pass streams; fmode (CgsMode) what its last block does with the sums.  In
// the selective form the second pass's UPD_NORM runs in place (w == out == z_{j+1}, each
// element read and then written by the same thread), so w and out are not restrict-qualified.
template <class T, int NC, int MODE>
__global__ void __launch_bounds__(256, 2) cgs_kernel(const T* __restrict__ Z, int64_t ldz, int64_t Kp, int j,
                                                  T* w, T* out, KState* ks,
                                                  double* __restrict__ partials, double eta, int fmode) {
  constexpr int VN = VecN<T>::N;
  constexpr int NACC = (MODE == CGS_PROJ) ? NC + 1 : (MODE == CGS_UPD_PROJ ? NC : 1);
  __shared__ T scoef[NC > 0 ? NC : 1];
  __shared__ Acc<T> red[8][NACC];
  __shared__ bool last;
  if (ks->done) return;  // breakdown reached earlier: uniform early exit
  if (cgs_skipped(fmode, ks)) return;
  const int nc = (MODE == CGS_NORM) ? 0 : j + 1;
  if (MODE == CGS_UPD_PROJ || MODE == CGS_UPD_NORM)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) scoef[c] = (T)ks->coef[c];
  __syncthreads();
  Acc<T> acc[NACC];
#pragma unroll
  for (int c = 0; c < NACC; ++c) acc[c].zero();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * VN;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r < Kp; r += stride) {
    T x[VN];
    load_vec<T, VN>(w + r, x);
    if constexpr (MODE == CGS_NORM) {
      acc_dot<T, VN>(acc[0], x, x);
    } else if constexpr (MODE == CGS_PROJ) {
      // columns in groups of 8: a group's loads are issued together (the column index
      // clamped to the last one, so no load waits behind a branch) before its FMAs
      constexpr int G = NC < 8 ? NC : 8;
#pragma unroll
      for (int c0 = 0; c0 < NC; c0 += G) {
        if (c0 < nc) {
          T z[G][VN];
#pragma unroll
          for (int g = 0; g < G; ++g) load_vec<T, VN>(Z + (int64_t)(c0 + g < nc ? c0 + g : nc - 1) * ldz + r, z[g]);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (c0 + g < nc) acc_dot<T, VN>(acc[c0 + g], z[g], x);
        }
      }
      acc_dot<T, VN>(acc[NC], x, x);
    } else {
      // update pass in the same column groups; the projection pass of UPD_PROJ below
      // re-reads each group's chunks
      constexpr int G = NC < 8 ? NC : 8;
#pragma unroll
      for (int c0 = 0; c0 < NC; c0 += G) {
        if (c0 < nc) {
          T z[G][VN];
#pragma unroll
          for (int g = 0; g < G; ++g) load_vec<T, VN>(Z + (int64_t)(c0 + g < nc ? c0 + g : nc - 1) * ldz + r, z[g]);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (c0 + g < nc)
#pragma unroll
              for (int v = 0; v < VN; ++v) x[v] = fma(-scoef[c0 + g], z[g][v], x[v]);
        }
      }
      if constexpr (MODE == CGS_UPD_PROJ) {
        store_vec<T, VN>(w + r, x);
        // reload the chunks rather than keep all of them live across the store (255 -> 128
        // registers, two blocks per SM instead of one; the reloads hit L1/L2)
        asm volatile("" ::: "memory");
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += G) {
          if (c0 < nc) {
            T z[G][VN];
#pragma unroll
            for (int g = 0; g < G; ++g) load_vec<T, VN>(Z + (int64_t)(c0 + g < nc ? c0 + g : nc - 1) * ldz + r, z[g]);
#pragma unroll
            for (int g = 0; g < G; ++g)
              if (c0 + g < nc) acc_dot<T, VN>(acc[c0 + g], z[g], x);
          }
        }
      } else {
        store_vec<T, VN>(out + r, x);
        acc_dot<T, VN>(acc[0], x, x);
      }
    }
  }
  // block reduction in the accumulator type (fixed order): warp tree, then over warps
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (MODE == CGS_NORM || MODE == CGS_UPD_NORM) {
    for (int o = 16; o > 0; o >>= 1) acc[0].add_partner(o);
    if (lane == 0) red[wid][0] = acc[0];
  } else {
    Acc<T> cols[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) cols[c] = acc[c];
    const Acc<T> mine = warp_reduce_columns<T, NC>(cols, lane);
    if (lane < NC) red[wid][lane] = mine;
    if constexpr (MODE == CGS_PROJ) {
      for (int o = 16; o > 0; o >>= 1) acc[NC].add_partner(o);
      if (lane == 0) red[wid][NC] = acc[NC];
    }
  }
  __syncthreads();
  const int nred = (MODE == CGS_PROJ) ? nc + 1 : (MODE == CGS_UPD_PROJ ? nc : 1);
  Acc<T>* P = reinterpret_cast<Acc<T>*>(partials);
  for (int c = threadIdx.x; c < nred; c += blockDim.x) {
    const int cc = (MODE == CGS_PROJ && c == nc) ? NC : c;
    Acc<T> a = red[0][cc];
    for (int q = 1; q < nw; ++q) a.add_acc(red[q][cc]);
    P[(int64_t)c * gridDim.x + blockIdx.x] = a;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ks->counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double dots[MMAX + 2];
  // every lane issues all its partial loads before summing them (fixed order per lane,
  // fixed shuffle tree), so the serial tail of the last block is one L2 round trip
  constexpr int PER_LANE = (RED_BLOCKS + 31) / 32;
  for (int c = wid; c < nred; c += nw) {
    const unsigned long long* pc = reinterpret_cast<const unsigned long long*>(P + (int64_t)c * gridDim.x);
    unsigned long long pv[PER_LANE];
#pragma unroll
    for (int t = 0; t < PER_LANE; ++t) {
      const unsigned b = lane + 32u * t;
      pv[t] = b < gridDim.x ? __ldcg(pc + b) : 0ull;
    }
    Acc<T> a;
    a.zero();
#pragma unroll
    for (int t = 0; t < PER_LANE; ++t) a.add_acc(*reinterpret_cast<const Acc<T>*>(&pv[t]));
    for (int o = 16; o > 0; o >>= 1) a.add_partner(o);
    if (lane == 0) dots[c] = a.value();
  }
  __syncthreads();
  if (ks->group) {  // partitioned: the sums over all partitions are finalised afterwards
    for (int c = threadIdx.x; c < nred; c += blockDim.x) ks->gsum[c] = dots[c];
    if (threadIdx.x == 0) ks->counter = 0;
    return;
  }
  cgs_finalize(fmode, j, dots, ks, eta);
  if (threadIdx.x == 0) ks->counter = 0;
}

// Per-block sums red[0..nred) -> partials; the last block to finish (atomic ticket) reduces
// them in a fixed order and finalises the column.  Every thread of the block calls this.
template <class T>
PCEXP_DEV void cgs_grid_tail(const Acc<T>* red, int nred, int mode, int j, KState* ks, double* partials,
                             double eta) {
  __shared__ bool last;
  __shared__ double dots[MMAX + 2];
  Acc<T>* P = reinterpret_cast<Acc<T>*>(partials);
  for (int c = threadIdx.x; c < nred; c += blockDim.x) P[(int64_t)c * gridDim.x + blockIdx.x] = red[c];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ks->counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int PER_LANE = (RED_BLOCKS + 31) / 32;
  for (int c = wid; c < nred; c += nw) {
    const unsigned long long* pc = reinterpret_cast<const unsigned long long*>(P + (int64_t)c * gridDim.x);
    unsigned long long pv[PER_LANE];
#pragma unroll
    for (int t = 0; t < PER_LANE; ++t) {
      const unsigned b = lane + 32u * t;
      pv[t] = b < gridDim.x ? __ldcg(pc + b) : 0ull;
    }
    Acc<T> a;
    a.zero();
#pragma unroll
    for (int t = 0; t < PER_LANE; ++t) a.add_acc(*reinterpret_cast<const Acc<T>*>(&pv[t]));
    for (int o = 16; o > 0; o >>= 1) a.add_partner(o);
    if (lane == 0) dots[c] = a.value();
  }
  __syncthreads();
  if (ks->group) {
    for (int c = threadIdx.x; c < nred; c += blockDim.x) ks->gsum[c] = dots[c];
    if (threadIdx.x == 0) ks->counter = 0;
    return;
  }
  cgs_finalize(mode, j, dots, ks, eta);
  if (threadIdx.x == 0) ks->counter = 0;
}

// Column-split Gram-Schmidt pass (PROJ, UPD_PROJ, UPD_NORM).  The 8 warps of a block walk
// the same tiles of 32 x VN rows; warp w owns the columns c = w, w + 8, ... (NCW of them),
// so a thread holds NCW accumulators instead of one per column and many blocks fit per SM
// (more loads in flight).  Update modes: each warp forms its partial sum of coef_c z_c,
// the partials meet in shared memory, warp 0 subtracts them in a fixed warp order, stores
// the updated tile and publishes it, and each warp projects it on its own columns with
// the chunks still in registers (two block barriers per tile).
constexpr int CGS_WARPS = 8;

// 16-byte asynchronous copy global -> shared (bypassing L1), and its group fences
PCEXP_DEV void cgs_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
PCEXP_DEV void cgs_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
PCEXP_DEV void cgs_cp_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
PCEXP_DEV void cgs_cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class T, int NCW, int MODE>
__global__ void __launch_bounds__(256) cgs_cs_kernel(const T* __restrict__ Z, int64_t ldz, int64_t Kp, int j,
                                                     T* __restrict__ w, T* __restrict__ out, KState* ks,
                                                     double* __restrict__ partials, double eta, int fmode) {
  constexpr int VN = VecN<T>::N, TR = 32 * VN;
  __shared__ T scoef[CGS_WARPS * NCW];
  __shared__ T part[(MODE == CGS_PROJ) ? 1 : CGS_WARPS * TR];
  __shared__ T xs[(MODE == CGS_UPD_PROJ) ? TR : 1];
  __shared__ Acc<T> red[CGS_WARPS * NCW + 1];
  if (ks->done) return;  // breakdown reached earlier: uniform early exit
  if (cgs_skipped(fmode, ks)) return;
  const int nc = j + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = threadIdx.x; c < CGS_WARPS * NCW; c += blockDim.x) scoef[c] = c < nc ? (T)ks->coef[c] : T(0);
  __syncthreads();
  Acc<T> acc[NCW + 1];
#pragma unroll
  for (int k = 0; k <= NCW; ++k) acc[k].zero();
  const int64_t ntile = (Kp + TR - 1) / TR;
  // FP32 update-and-projection pass: each thread copies its own chunks of the block's next
  // tile into its own shared-memory slots with cp.async while it works on the current tile
  // (two stages), so the next tile's loads are in flight across this tile's two block
  // barriers without holding registers; no other thread reads a thread's slots, so the copies
  // need no barrier of their own.  (C5: 29.5 -> 26.4 ms per step; the projection pass, which
  // has no barriers, measured slower staged: 24.6 against 22.3 ms.)
  constexpr bool STAGED = MODE == CGS_UPD_PROJ && sizeof(T) == 4;
  constexpr int SLOTS = NCW + 1;  // the thread's column chunks, then its chunk of w
  __shared__ __align__(16) T stg[STAGED ? 2 * CGS_WARPS * SLOTS * TR : 1];
  auto slot = [&](int buf, int k) { return stg + ((buf * CGS_WARPS + wid) * SLOTS + k) * TR + lane * VN; };
  auto issue = [&](int64_t t, int buf) {
    const int64_t r = t * TR + lane * VN;
    if (r >= Kp) return;
#pragma unroll
    for (int k = 0; k < NCW; ++k)
      if (wid + CGS_WARPS * k < nc) cgs_cp16(slot(buf, k), Z + (wid + CGS_WARPS * k) * ldz + r);
    if (MODE == CGS_PROJ || wid == 0) cgs_cp16(slot(buf, NCW), w + r);
  };
  if constexpr (STAGED) {
    if ((int64_t)blockIdx.x < ntile) issue(blockIdx.x, 0);
    cgs_cp_commit();
  }
  int it = 0;
  for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x, ++it) {
    const int64_t r = t * TR + lane * VN;
    const bool valid = r < Kp;
    if constexpr (STAGED) {
      if (t + gridDim.x < ntile) issue(t + gridDim.x, (it & 1) ^ 1);
      cgs_cp_commit();
      cgs_cp_wait_prev();  // this tile's copies (all but the group just committed) have landed
    }
    T z[NCW][VN];
#pragma unroll
    for (int k = 0; k < NCW; ++k) {
      const int c = wid + CGS_WARPS * k;
      if (valid && c < nc) {
        if constexpr (STAGED) {
#pragma unroll
          for (int v = 0; v < VN; ++v) z[k][v] = slot(it & 1, k)[v];
        } else {
          load_vec<T, VN>(Z + c * ldz + r, z[k]);
        }
      } else {
#pragma unroll
        for (int v = 0; v < VN; ++v) z[k][v] = T(0);
      }
    }
    // every warp needs the tile of w for the projection; in the update modes only warp 0
    // (which applies the update), loading it here so the load overlaps the column loads
    T x[VN];
    if (valid && (MODE == CGS_PROJ || wid == 0)) {
      if constexpr (STAGED) {
#pragma unroll
        for (int v = 0; v < VN; ++v) x[v] = slot(it & 1, NCW)[v];
      } else {
        load_vec<T, VN>(w + r, x);
      }
    } else {
#pragma unroll
      for (int v = 0; v < VN; ++v) x[v] = T(0);
    }
    if constexpr (MODE == CGS_PROJ) {
#pragma unroll
      for (int k = 0; k < NCW; ++k) acc_dot<T, VN>(acc[k], z[k], x);
      if (wid == 0) acc_dot<T, VN>(acc[NCW], x, x);
    } else {
      T p[VN];
#pragma unroll
      for (int v = 0; v < VN; ++v) p[v] = T(0);
#pragma unroll
      for (int k = 0; k < NCW; ++k) {
        const T cf = scoef[wid + CGS_WARPS * k];
#pragma unroll
        for (int v = 0; v < VN; ++v) p[v] = fma(cf, z[k][v], p[v]);
      }
#pragma unroll
      for (int v = 0; v < VN; ++v) part[wid * TR + lane * VN + v] = p[v];
      __syncthreads();
      // warp 0 forms the updated tile once (fixed warp order), stores it and publishes it
      if (wid == 0) {
#pragma unroll
        for (int q = 0; q < CGS_WARPS; ++q)
#pragma unroll
          for (int v = 0; v < VN; ++v) x[v] -= part[q * TR + lane * VN + v];
        if (valid) store_vec<T, VN>((MODE == CGS_UPD_PROJ ? w : out) + r, x);
        if constexpr (MODE == CGS_UPD_PROJ) {
#pragma unroll
          for (int v = 0; v < VN; ++v) xs[lane * VN + v] = x[v];
        } else {
          acc_dot<T, VN>(acc[NCW], x, x);
        }
      }
      __syncthreads();
      if constexpr (MODE == CGS_UPD_PROJ) {
        T xn[VN];
#pragma unroll
        for (int v = 0; v < VN; ++v) xn[v] = xs[lane * VN + v];
#pragma unroll
        for (int k = 0; k < NCW; ++k) acc_dot<T, VN>(acc[k], z[k], xn);
      }
    }
  }
  if constexpr (STAGED) cgs_cp_wait_all();  // no copy outlives the block
  // warp sums of the owned columns (fixed shuffle tree); each column has one owner warp
  if constexpr (MODE != CGS_UPD_NORM) {
#pragma unroll
    for (int k = 0; k < NCW; ++k) {
      for (int o = 16; o > 0; o >>= 1) acc[k].add_partner(o);
      if (lane == 0) red[wid + CGS_WARPS * k] = acc[k];
    }
  }
  if (MODE != CGS_UPD_PROJ && wid == 0) {
    for (int o = 16; o > 0; o >>= 1) acc[NCW].add_partner(o);
    if (lane == 0) red[MODE == CGS_PROJ ? CGS_WARPS * NCW : 0] = acc[NCW];
  }
  __syncthreads();
  // partial-sum slots: PROJ columns 0..nc-1 and the norm at nc; UPD_PROJ columns; UPD_NORM the norm
  __shared__ Acc<T> ordered[MMAX + 1];
  const int nred = (MODE == CGS_PROJ) ? nc + 1 : (MODE == CGS_UPD_PROJ ? nc : 1);
  for (int c = threadIdx.x; c < nred; c += blockDim.x)
    ordered[c] = (MODE == CGS_PROJ && c == nc) ? red[CGS_WARPS * NCW] : red[c];
  __syncthreads();
  cgs_grid_tail<T>(ordered, nred, fmode, j, ks, partials, eta);
}

template <class KernelT>
static unsigned wave_grid(KernelT kernel, int64_t chunks) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0);
  if (occ < 1) occ = 1;
  int64_t g = (int64_t)sms * occ;
  const int64_t need = (chunks + 255) / 256;
  if (g > need) g = need;
  if (g > RED_BLOCKS) g = RED_BLOCKS;
  return (unsigned)(g < 1 ? 1 : g);
}

template <class T, int NC, int MODE>
static void cgs_launch(const T* Z, int64_t ldz, int64_t Kp, int j, T* w, T* out, KState* ks, double* partials,
                       double eta, int fmode, cudaStream_t st) {
  static unsigned grid_cache = 0;
  static int64_t kp_cache = -1;
  if (kp_cache != Kp) {
    grid_cache = wave_grid(cgs_kernel<T, NC, MODE>, Kp / VecN<T>::N);
    kp_cache = Kp;
  }
  cgs_kernel<T, NC, MODE><<<grid_cache, 256, 0, st>>>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode);
}

template <class T, int NCW, int MODE>
static void cgs_cs_launch(const T* Z, int64_t ldz, int64_t Kp, int j, T* w, T* out, KState* ks, double* partials,
                          double eta, int fmode, cudaStream_t st) {
  static unsigned grid_cache = 0;
  static int64_t kp_cache = -1;
  if (kp_cache != Kp) {
    grid_cache = wave_grid(cgs_cs_kernel<T, NCW, MODE>, (Kp + 32 * VecN<T>::N - 1) / (32 * VecN<T>::N) * 256);
    kp_cache = Kp;
  }
  cgs_cs_kernel<T, NCW, MODE><<<grid_cache, 256, 0, st>>>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode);
}

// Which layout serves a precision and pass: the column-split kernel (column capacity
// 8 x NCW, NCW = 1, 2, 4) or the row kernel (every thread accumulates all columns of its
// rows).  Measured on GB300 (C2 and the 48^3 tetrahedra): the FP32 projections gain from
// the column split (fewer registers, more loads in flight); the FP64 passes are bound by
// the FP64 pipe and the update-and-norm pass keeps one accumulator, so the row kernel's
// single barrier-free sweep is faster for those.
template <class T, int MODE> struct CgsColumnSplit {
  static constexpr bool value = sizeof(T) == 4 && MODE != CGS_UPD_NORM;
};

template <class T, int MODE>
static void cgs_dispatch(int nc, const T* Z, int64_t ldz, int64_t Kp, int j, T* w, T* out, KState* ks,
                         double* partials, double eta, int fmode, cudaStream_t st) {
  if constexpr (CgsColumnSplit<T, MODE>::value) {
    if (nc <= CGS_WARPS) cgs_cs_launch<T, 1, MODE>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode, st);
    else if (nc <= 2 * CGS_WARPS) cgs_cs_launch<T, 2, MODE>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode, st);
    else cgs_cs_launch<T, 4, MODE>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode, st);
  } else {
    if (nc <= 4) cgs_launch<T, 4, MODE>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode, st);
    else if (nc <= 8) cgs_launch<T, 8, MODE>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode, st);
    else if (nc <= 16) cgs_launch<T, 16, MODE>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode, st);
    else cgs_launch<T, 32, MODE>(Z, ldz, Kp, j, w, out, ks, partials, eta, fmode, st);
  }
}

template <class T>
cudaError_t launch_cgs(int mode, const T* Z, int64_t ldz, int64_t Kp, int j, T* w, T* out, KState* ks,
                       double* partials, double eta, cudaStream_t st) {
  const int nc = j + 1;
  if (nc > MMAX) return cudaErrorInvalidValue;
  switch (mode) {
    case CGS_NORM: cgs_launch<T, 0, CGS_NORM>(Z, ldz, Kp, j, w, out, ks, partials, eta, mode, st); break;
    case CGS_PROJ:
    case CGS_PROJ2: cgs_dispatch<T, CGS_PROJ>(nc, Z, ldz, Kp, j, w, out, ks, partials, eta, mode, st); break;
    case CGS_UPD_PROJ: cgs_dispatch<T, CGS_UPD_PROJ>(nc, Z, ldz, Kp, j, w, out, ks, partials, eta, mode, st); break;
    case CGS_UPD_NORM:
    case CGS_UPD1: cgs_dispatch<T, CGS_UPD_NORM>(nc, Z, ldz, Kp, j, w, out, ks, partials, eta, mode, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------ Gram-Schmidt of a partitioned run
__global__ void __launch_bounds__(256) cgs_group_finalize_kernel(int mode, int j, KState* ks, double eta) {
  __shared__ double dots[MMAX + 2];
  if (ks->done) return;  // the pass did not run (uniform)
  if (cgs_skipped(mode, ks)) return;  // the pass did not run (uniform)
  for (int c = threadIdx.x; c < MMAX + 2; c += blockDim.x) dots[c] = ks->gtot[c];
  __syncthreads();
  cgs_finalize(mode, j, dots, ks, eta);
}
cudaError_t launch_cgs_group_finalize(int mode, int j, KState* ks, double eta, cudaStream_t st) {
  cgs_group_finalize_kernel<<<1, 256, 0, st>>>(mode, j, ks, eta);
  return cudaGetLastError();
}

__global__ void group_reduce_kernel(PartPtrs slots, int nparts, int n, double* out, int op) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = reinterpret_cast<const double*>(slots.p[0])[i];
    for (int q = 1; q < nparts; ++q) {
      const double b = reinterpret_cast<const double*>(slots.p[q])[i];
      a = op == 1 ? fmin(a, b) : a + b;
    }
    out[i] = a;
  }
}
cudaError_t launch_group_reduce(PartPtrs slots, int nparts, int n, double* out, int op, cudaStream_t st) {
  group_reduce_kernel<<<1, 64, 0, st>>>(slots, nparts, n, out, op);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ phi kernel
// exp(A) by scaling and squaring with the [8/8] diagonal Pade approximant
//   r(X) = N(X) / N(-X),  N(X) = sum_j c_j X^j,  c_j = (16-j)! 8! / (16! j! (8-j)!),
// applied to X = A / 2^s with ||X||_1 <= 1 (the Pade error is far below FP64 rounding).
// For phi: A = [[dt H_k, e_1, 0], [0, 0, 1], [0, 0, 0]]; column k of exp(A) holds
// phi_1(dt H) e_1 and column k+1 holds phi_2(dt H) e_1.
//
// FP64 issues at a few instructions per clock per SM on this GPU, so one CTA would
// spend ~10 us per (m+2)^3 product.  The kernels run as a cluster of PHI_CTAS CTAs:
// every CTA keeps a full copy of the matrices in shared memory (5 buffers), computes
// its share of the rows of each product and writes them into every CTA of the cluster
// (distributed shared memory), then the cluster barrier publishes them.  The Pade solve
// factors the denominator redundantly in each CTA and splits the right-hand-side columns.
constexpr int PN = MMAX + 2;      // phi: (m+2) x (m+2)
constexpr int PN2 = 2 * PN;       // phi adjoint: block-triangular 2 (m+2) x 2 (m+2)
constexpr int PHI_CTAS = 8;

namespace cg = cooperative_groups;

// C = A B for rows i = rank, rank + PHI_CTAS, ... ; results broadcast to all CTAs.
template <int LD>
__device__ void mat_mul_cluster(cg::cluster_group& cl, const double* A, const double* B, double* C, int n) {
  const int rank = (int)cl.block_rank();
  const int nrow = (n - rank + PHI_CTAS - 1) / PHI_CTAS;
  for (int t = threadIdx.x; t < nrow * n; t += blockDim.x) {
    const int i = rank + (t / n) * PHI_CTAS, jj = t % n;
    double a = 0;
    for (int l = 0; l < n; ++l) a = fma(A[i * LD + l], B[l * LD + jj], a);
#pragma unroll
    for (int r = 0; r < PHI_CTAS; ++r) cl.map_shared_rank(C, r)[i * LD + jj] = a;
  }
  cl.sync();
}

// exp of the n x n matrix held (identically) in buffer A of every CTA of the cluster.
// sm holds 5 LD x LD buffers; returns the buffer with the result (same in all CTAs),
// or nullptr if the input is not finite.  Must be called by all threads of all CTAs.
template <int LD>
__device__ double* expm_cluster(cg::cluster_group& cl, double* sm, int n) {
  double* A = sm;
  double* B2 = A + LD * LD;
  double* B4 = B2 + LD * LD;
  double* B6 = B4 + LD * LD;
  double* Vb = B6 + LD * LD;
  __shared__ int s_sq;
  __shared__ int piv_row;
  __shared__ float colsum[LD];
  const int rank = (int)cl.block_rank();
  // ||A||_1 from parallel column sums in FP32 (it only selects s; the same arithmetic in
  // every CTA gives the same s)
  for (int jj = threadIdx.x; jj < n; jj += blockDim.x) {
    float c = 0.f;
    for (int i = 0; i < n; ++i) c += fabsf((float)A[i * LD + jj]);
    colsum[jj] = c;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    float m = 0.f;
    for (int jj = threadIdx.x; jj < n; jj += 32) m = fmaxf(m, colsum[jj]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      int s = 0;
      if (m > 1.0f) s = (int)ceilf(log2f(m)) + 1;  // +1 covers the FP32 estimate
      if (!(m <= 3.0e38f) || s > 1000) s = -1;     // NaN or overflow
      s_sq = s;
    }
  }
  __syncthreads();
  const int sq = s_sq;
  if (sq < 0) return nullptr;  // uniform across the cluster (same data, same arithmetic)
  const double sc = ldexp(1.0, -sq);
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[(t / n) * LD + t % n] *= sc;
  // every CTA must have finished writing its own A before remote products land
  cl.sync();
  double c[9];
  c[0] = 1.0;
  for (int jj = 1; jj <= 8; ++jj) c[jj] = c[jj - 1] * (double)(8 - jj + 1) / (double)(jj * (16 - jj + 1));
  mat_mul_cluster<LD>(cl, A, A, B2, n);
  mat_mul_cluster<LD>(cl, B2, B2, B4, n);
  mat_mul_cluster<LD>(cl, B4, B2, B6, n);
  // V = c0 I + c2 B2 + c4 B4 + c6 B6 (Vb);  W = c1 I + c3 B2 + c5 B4 + c7 B6 (into B6)
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, jj = t - i * n, o = i * LD + jj;
    const double id = (i == jj) ? 1.0 : 0.0;
    const double b2 = B2[o], b4 = B4[o], b6 = B6[o];
    Vb[o] = c[0] * id + c[2] * b2 + c[4] * b4 + c[6] * b6;
    B6[o] = c[1] * id + c[3] * b2 + c[5] * b4 + c[7] * b6;
  }
  cl.sync();  // B2 is overwritten remotely next
  mat_mul_cluster<LD>(cl, B4, B4, B2, n);  // B8
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int o = (t / n) * LD + t % n;
    Vb[o] += c[8] * B2[o];
  }
  cl.sync();  // B4 is overwritten remotely next
  mat_mul_cluster<LD>(cl, A, B6, B4, n);  // U = X W
  // N = V + U (Vb), D = V - U (B2)
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int o = (t / n) * LD + t % n;
    const double V = Vb[o], U = B4[o];
    Vb[o] = V + U;
    B2[o] = V - U;
  }
  __syncthreads();
  // solve D X = N: LU with partial pivoting repeated in every CTA (identical); this CTA
  // keeps the right-hand-side columns jj = rank, rank + PHI_CTAS, ...
  double* Dm = B2;
  double* Nm = Vb;
  const int ncol = (n - rank + PHI_CTAS - 1) / PHI_CTAS;
  for (int col = 0; col < n; ++col) {
    if (threadIdx.x < 32) {
      // partial pivoting by warp argmax on the bit patterns of |x|
      unsigned long long best = 0ull;
      int bi = col;
      for (int i = col + threadIdx.x; i < n; i += 32) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(Dm[i * LD + col]) & 0x7fffffffffffffffull;
        if (key > best || i == col) {
          best = key;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) piv_row = bi;
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != col) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double a = Dm[col * LD + t];
        Dm[col * LD + t] = Dm[pr * LD + t];
        Dm[pr * LD + t] = a;
      }
      for (int t = threadIdx.x; t < ncol; t += blockDim.x) {
        const int jj = rank + t * PHI_CTAS;
        double b = Nm[col * LD + jj];
        Nm[col * LD + jj] = Nm[pr * LD + jj];
        Nm[pr * LD + jj] = b;
      }
      __syncthreads();
    }
    const double piv = Dm[col * LD + col];
    const int nr = n - col - 1, w = (n - col - 1) + ncol;
    for (int t = threadIdx.x; t < nr * w; t += blockDim.x) {
      const int i = col + 1 + t / w, q = t % w;
      const double f = Dm[i * LD + col] / piv;
      if (q < n - col - 1) {
        const int jj = col + 1 + q;
        Dm[i * LD + jj] -= f * Dm[col * LD + jj];
      } else {
        const int jj = rank + (q - (n - col - 1)) * PHI_CTAS;
        Nm[i * LD + jj] -= f * Nm[col * LD + jj];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr; t += blockDim.x) Dm[(col + 1 + t) * LD + col] = 0.0;
    __syncthreads();
  }
  for (int col = n - 1; col >= 0; --col) {
    const double piv = Dm[col * LD + col];
    for (int t = threadIdx.x; t < ncol; t += blockDim.x) Nm[col * LD + rank + t * PHI_CTAS] /= piv;
    __syncthreads();
    for (int t = threadIdx.x; t < col * ncol; t += blockDim.x) {
      const int i = t / ncol, jj = rank + (t % ncol) * PHI_CTAS;
      Nm[i * LD + jj] -= Dm[i * LD + col] * Nm[col * LD + jj];
    }
    __syncthreads();
  }
  // publish this CTA's solution columns once every CTA has finished its own solve
  cl.sync();
  for (int t = threadIdx.x; t < n * ncol; t += blockDim.x) {
    const int i = t / ncol, jj = rank + (t % ncol) * PHI_CTAS;
    const double v = Nm[i * LD + jj];
#pragma unroll
    for (int r = 0; r < PHI_CTAS; ++r)
      if (r != rank) cl.map_shared_rank(Nm, r)[i * LD + jj] = v;
  }
  cl.sync();
  // squaring (X in Vb, B4 as the other buffer)
  double* X = Vb;
  double* Y = B4;
  for (int it = 0; it < sq; ++it) {
    mat_mul_cluster<LD>(cl, X, X, Y, n);
    double* t = X;
    X = Y;
    Y = t;
  }
  return X;
}

// which = 1: the update coefficients use phi_1(dt H) e_1 (Eq. s8, s9, s10); which = 2: they use
// phi_2(dt H) e_1 (the ETD2 term of Eq. s7), times dt / *dt_prev when dt_prev is given.
//
// Every evaluation also forms the relative a-posteriori error estimate of the Krylov phi_1
// product (Saad 1992, the leading term of the error of Eq. final),
//   est = dt h_{k+1,k} |e_k^T phi_2(dt H_k) e_1| / ||phi_1(dt H_k) e_1||,
// from the phi_2 column of the same exponential.  check_tol > 0 is a checkpoint of the
// adaptive dimension: only est is formed, and ks->done is raised when est <= check_tol.
__global__ void __cluster_dims__(PHI_CTAS, 1, 1) __launch_bounds__(256)
    phi_kernel(KState* ks, const double* dt_dev, double dt_host, double factor, StepState* ss, int stage, int which,
               const double* dt_prev, double check_tol) {
  extern __shared__ double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int k = ks->k;
  const double dt = dt_dev ? *dt_dev : dt_host;
  if (check_tol > 0.0 && (k == 0 || ks->err || ks->done)) return;  // uniform across the cluster
  if (k == 0 || ks->err) {  // uniform across the cluster: no shared-memory traffic happens
    if (rank == 0 && threadIdx.x == 0) {
      for (int i = 0; i <= MMAX; ++i) ks->acoef[i] = 0.0;
      if (ss) {
        ss->k[stage] = 0;
        ss->beta[stage] = ks->beta;
        ss->pass2[stage] = ks->pass2;
        if (ks->err) ss->err = ks->err;
      }
    }
    return;
  }
  const int n = k + 2;
  double* A = sm;
  for (int t = threadIdx.x; t < PN * PN; t += blockDim.x) A[t] = 0.0;
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, jj = t - i * k;
    A[i * PN + jj] = dt * ks->H[i * MMAX + jj];
  }
  if (threadIdx.x == 0) {
    A[0 * PN + k] = 1.0;
    A[k * PN + k + 1] = 1.0;
  }
  __syncthreads();
  const double* X = expm_cluster<PN>(cl, sm, n);
  if (rank == 0 && threadIdx.x == 0) {
    if (!X) {
      ks->err = 1;
      if (ss) ss->err = 1;
      return;
    }
    double n1 = 0.0;
    for (int i = 0; i < k; ++i) n1 += X[i * PN + k] * X[i * PN + k];
    const double est = dt * fabs(ks->H[k * MMAX + k - 1]) * fabs(X[(k - 1) * PN + k + 1]) / sqrt(n1);
    ks->err_est = est;
    if (check_tol > 0.0) {
      if (est <= check_tol) ks->done = 1;  // the estimate may be NaN: then the process goes on
      return;
    }
    const double beta = ks->beta;
    const double f = dt_prev ? factor * dt / *dt_prev : factor;
    bool ok = true;
    for (int i = 0; i < k; ++i) {
      const double y1 = X[i * PN + k], y2 = X[i * PN + k + 1];
      ks->y[i] = y1;
      ks->y2[i] = y2;
      ks->acoef[i] = f * dt * beta * (which == 2 ? y2 : y1) * ks->s[i];
      ok = ok && isfinite(ks->acoef[i]);
    }
    for (int i = k; i <= MMAX; ++i) ks->acoef[i] = 0.0;
    if (!ok) ks->err = 1;
    if (ss) {
      ss->k[stage] = k;
      ss->beta[stage] = beta;
      ss->kerr[stage] = est;
      ss->pass2[stage] = ks->pass2;
      if (!ok) ss->err = 1;
    }
  }
}

// Adjoint of y = phi_1(dt H) e_1 (the first k entries of column k of exp(A)):
//   Hbar = dt [L_exp(A^T, Xbar)]_{0:k,0:k},  Xbar = ybar in rows 0..k-1 of column k,
// where L_exp(M, E), the Frechet derivative of exp, is the top-right block of
// exp([[M, E], [0, M]]) (block-triangular identity; Najfeld & Havel 1995).
__global__ void __cluster_dims__(PHI_CTAS, 1, 1) __launch_bounds__(256)
    phi_adjoint_kernel(const double* __restrict__ H, int k, int ldh, double dt, const double* __restrict__ ybar,
                       double* __restrict__ Hbar, int* __restrict__ err) {
  extern __shared__ double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int n0 = k + 2, n = 2 * n0;
  double* M = sm;
  for (int t = threadIdx.x; t < PN2 * PN2; t += blockDim.x) M[t] = 0.0;
  __syncthreads();
  // M = [[A^T, Xbar], [0, A^T]] with A = [[dt H, e_1, 0], [0, 0, 1], [0, 0, 0]]
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, jj = t - i * k;
    const double a = dt * H[jj * ldh + i];  // (A^T)_{ij} = A_{ji}
    M[i * PN2 + jj] = a;
    M[(n0 + i) * PN2 + n0 + jj] = a;
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) M[t * PN2 + n0 + k] = ybar[t];
  if (threadIdx.x == 0) {
    M[k * PN2 + 0] = 1.0;  // (A^T)_{k,0} = A_{0,k} = 1
    M[(k + 1) * PN2 + k] = 1.0;
    M[(n0 + k) * PN2 + n0 + 0] = 1.0;
    M[(n0 + k + 1) * PN2 + n0 + k] = 1.0;
  }
  __syncthreads();
  const double* X = expm_cluster<PN2>(cl, sm, n);
  if (rank == 0) {
    if (!X) {
      if (threadIdx.x == 0) *err = 1;
      return;
    }
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
      const int i = t / k, jj = t - i * k;
      Hbar[i * ldh + jj] = dt * X[i * PN2 + n0 + jj];
    }
  }
}

static cudaError_t phi_smem_attr(size_t smem) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(phi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

cudaError_t launch_phi(KState* ks, const double* dt_dev, double dt, double factor, StepState* ss, int stage,
                       cudaStream_t st, int which, const double* dt_prev) {
  const size_t smem = 5 * PN * PN * sizeof(double);
  cudaError_t e = phi_smem_attr(smem);
  if (e != cudaSuccess) return e;
  phi_kernel<<<PHI_CTAS, 256, smem, st>>>(ks, dt_dev, dt, factor, ss, stage, which, dt_prev, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_phi_check(KState* ks, const double* dt_dev, double tol, cudaStream_t st) {
  const size_t smem = 5 * PN * PN * sizeof(double);
  cudaError_t e = phi_smem_attr(smem);
  if (e != cudaSuccess) return e;
  phi_kernel<<<PHI_CTAS, 256, smem, st>>>(ks, dt_dev, 1.0, 1.0, nullptr, 0, 1, nullptr, tol);
  return cudaGetLastError();
}

cudaError_t launch_phi_adjoint(const double* H, int k, int ldh, double dt, const double* ybar, double* Hbar, int* err,
                               cudaStream_t st) {
  if (k < 1 || k > MMAX) return cudaErrorInvalidValue;
  const size_t smem = 5 * PN2 * PN2 * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(phi_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  phi_adjoint_kernel<<<PHI_CTAS, 256, smem, st>>>(H, k, ldh, dt, ybar, Hbar, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ axpy
template <class T>
__global__ void __launch_bounds__(256) krylov_axpy_kernel(const double* __restrict__ base64, double* __restrict__ out64,
                                                          T* __restrict__ shadow, T* __restrict__ delta,
                                                          const T* __restrict__ Z, int64_t ldz, int64_t Kp,
                                                          const KState* ks) {
  __shared__ T sc[MMAX];
  const int k = ks->k;
  for (int i = threadIdx.x; i < MMAX; i += blockDim.x) sc[i] = (T)ks->acoef[i];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += stride) {
    T a = 0;
    for (int i = 0; i < k; ++i) a = fma(sc[i], Z[i * ldz + r], a);
    const double o = base64[r] + (double)a;
    out64[r] = o;
    if (delta) delta[r] = a;
    if (shadow && (void*)shadow != (void*)out64) shadow[r] = (T)o;
  }
}

template <class T>
cudaError_t launch_krylov_axpy(const double* base64, double* out64, T* shadow, T* delta, const T* Z, int64_t ldz,
                               int64_t Kp, const KState* ks, cudaStream_t st) {
  int64_t g = (Kp + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  krylov_axpy_kernel<T><<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(base64, out64, shadow, delta, Z, ldz, Kp, ks);
  return cudaGetLastError();
}

template <class T>
__global__ void combine_kernel(T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ c, int64_t n) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    a[r] = b[r] - a[r] - c[r];
}
template <class T>
cudaError_t launch_combine_corrector(T* a, const T* b, const T* c, int64_t Kp, cudaStream_t st) {
  int64_t g = (Kp + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  combine_kernel<T><<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(a, b, c, Kp);
  return cudaGetLastError();
}

// out = x - y - z (z nullable)
template <class T>
__global__ void lincomb3_kernel(T* __restrict__ out, const T* __restrict__ x, const T* __restrict__ y,
                                const T* __restrict__ z, int64_t n) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    out[r] = z ? x[r] - y[r] - z[r] : x[r] - y[r];
}
template <class T>
cudaError_t launch_lincomb3(T* out, const T* x, const T* y, const T* z, int64_t Kp, cudaStream_t st) {
  int64_t g = (Kp + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  lincomb3_kernel<T><<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(out, x, y, z, Kp);
  return cudaGetLastError();
}

template <class Tin, class Tout>
__global__ void cast_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, int64_t n) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    y[r] = (Tout)x[r];
}
template <class Tin, class Tout>
cudaError_t launch_cast(const Tin* x, Tout* y, int64_t n, cudaStream_t st) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  cast_kernel<Tin, Tout><<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

__global__ void reset_kstate_kernel(KState* ks) {
  if (threadIdx.x == 0) {
    ks->k = 0;
    ks->done = 0;
    ks->err = 0;
    ks->counter = 0;
    ks->beta = 0;
    ks->err_est = 0;
    ks->skip2 = 0;
    ks->pass2 = 0u;
  }
  for (int i = threadIdx.x; i < (MMAX + 1) * MMAX; i += blockDim.x) ks->H[i] = 0.0;
}
cudaError_t launch_reset_kstate(KState* ks, cudaStream_t st) {
  reset_kstate_kernel<<<1, 256, 0, st>>>(ks);
  return cudaGetLastError();
}

__global__ void set_dt_kernel(StepState* ss, double dt) { ss->dt = dt; }
__global__ void set_cfl_kernel(StepState* ss, double cfl) { ss->cfl = cfl; }
cudaError_t launch_set_cfl(StepState* ss, double cfl, cudaStream_t st) {
  set_cfl_kernel<<<1, 1, 0, st>>>(ss, cfl);
  return cudaGetLastError();
}
__global__ void keep_dt_kernel(StepState* ss) { ss->dt_prev = ss->dt; }
__global__ void cap_cfl_kernel(StepState* ss, double cap) { ss->cfl = fmin(ss->cfl, cap); }
cudaError_t launch_cap_cfl(StepState* ss, double cap, cudaStream_t st) {
  cap_cfl_kernel<<<1, 1, 0, st>>>(ss, cap);
  return cudaGetLastError();
}
cudaError_t launch_keep_dt(StepState* ss, cudaStream_t st) {
  keep_dt_kernel<<<1, 1, 0, st>>>(ss);
  return cudaGetLastError();
}
__global__ void set_param_kernel(double* p, double v) { *p = v; }
__global__ void copy_dt_kernel(StepState* ss, const double* p) { ss->dt = *p; }
cudaError_t launch_set_param(double* param, double v, cudaStream_t st) {
  set_param_kernel<<<1, 1, 0, st>>>(param, v);
  return cudaGetLastError();
}
cudaError_t launch_copy_dt(StepState* ss, const double* param, cudaStream_t st) {
  copy_dt_kernel<<<1, 1, 0, st>>>(ss, param);
  return cudaGetLastError();
}
cudaError_t launch_set_dt(StepState* ss, double dt, cudaStream_t st) {
  set_dt_kernel<<<1, 1, 0, st>>>(ss, dt);
  return cudaGetLastError();
}

template cudaError_t launch_cgs<double>(int, const double*, int64_t, int64_t, int, double*, double*, KState*, double*,
                                        double, cudaStream_t);
template cudaError_t launch_cgs<float>(int, const float*, int64_t, int64_t, int, float*, float*, KState*, double*,
                                       double, cudaStream_t);
template cudaError_t launch_krylov_axpy<double>(const double*, double*, double*, double*, const double*, int64_t,
                                                int64_t, const KState*, cudaStream_t);
template cudaError_t launch_krylov_axpy<float>(const double*, double*, float*, float*, const float*, int64_t,
                                               int64_t, const KState*, cudaStream_t);
template cudaError_t launch_lincomb3<double>(double*, const double*, const double*, const double*, int64_t,
                                             cudaStream_t);
template cudaError_t launch_lincomb3<float>(float*, const float*, const float*, const float*, int64_t, cudaStream_t);
template cudaError_t launch_combine_corrector<double>(double*, const double*, const double*, int64_t, cudaStream_t);
template cudaError_t launch_combine_corrector<float>(float*, const float*, const float*, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace pcexp
