// Reverse of the Krylov stage of a PCEXP step as computed (FP64): the adjoint of
//   u_out = u_base + factor dt beta V_k y,  y = phi_1(dt H_k) e_1,
// through the CGS2 Arnoldi process that built V and H (Eq. vm-vm2, final, s9/s10).
//
// Forward column j (v_i = s_i z_i, z_{j+1} stored unnormalised):
//   w0 = J v_j;  h1 = V_j^T w0;  w1 = w0 - V_j h1;  h2 = V_j^T w1;  w2 = w1 - V_j h2;
//   eta = ||w2||;  v_{j+1} = w2 / eta;  H[:, j] = h1 + h2;  H[j+1, j] = eta.
// Reverse column j (bars are adjoints; Hbar from the phi adjoint, Vbar accumulated):
//   w2bar = vbar_{j+1} / eta + (etabar - (v_{j+1} . vbar_{j+1}) / eta) v_{j+1}
//   h2bar = Hbar[:, j] - V_j^T w2bar;   w1bar = w2bar + V_j h2bar
//   h1bar = Hbar[:, j] - V_j^T w1bar;   w0bar = w1bar + V_j h1bar
//   Vbar_j += w1 h2bar^T - w2bar h2^T + w0 h1bar^T - w1bar h1^T
//   vbar_j += J^T w0bar;   ubar_lin += (d(J v_j)/du)^T w0bar
// w1 and w0 are recomputed from V, h1 and h2.  Reductions use the same fixed-order
// last-block scheme as the forward kernels (deterministic).
#include <cfloat>

#include "kernels.h"

namespace pcexp {

namespace {

constexpr int AB = 304;  // blocks of the adjoint streaming kernels (2 x 152 SMs)

PCEXP_DEV double warp_sum(double a) {
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

// Block reduction of NACC per-thread sums into partials[c * gridDim + block]; returns
// true in the one block that finishes last, after it has reduced every column into
// as->dots (fixed order).
template <int NACC>
__device__ bool reduce_last(double (&acc)[NACC], int nred, double* partials, AdjState* as) {
  __shared__ double red[8][NACC];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NACC; ++c) {
    const double a = warp_sum(acc[c]);
    if (lane == 0) red[wid][c] = a;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nred; c += blockDim.x) {
    double a = 0;
    for (int q = 0; q < 8; ++q) a += red[q][c];
    partials[(int64_t)c * gridDim.x + blockIdx.x] = a;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&as->counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // a partition of a partitioned run leaves its sums for the sum over the partitions, and the
  // reduction is finished afterwards (launch_adj_finish)
  double* dst = as->group ? as->gsum : as->dots;
  for (int c = wid; c < nred; c += 8) {
    double a = 0;
    for (unsigned b = lane; b < gridDim.x; b += 32) a += __ldcg(partials + (int64_t)c * gridDim.x + b);
    a = warp_sum(a);
    if (lane == 0) dst[c] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) as->counter = 0;
  return !as->group;
}

// The finishing steps of the reductions, from the summed as->dots (called by the last block of
// the reduction, or by the finishing kernel of a partitioned run)
PCEXP_DEV void finish_alpha(int j, const KState* ks, AdjState* as) {
  if (threadIdx.x == 0) as->alpha = ks->s[j + 1] * as->dots[0];
}
PCEXP_DEV void finish_upd(int mode, int j, const KState* ks, AdjState* as) {
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double hb = as->Hbar[i * MMAX + j] - ks->s[i] * as->dots[i];
    if (mode == 0) {
      as->hb2[i] = hb;
      as->cb2[i] = hb * ks->s[i];
    } else {
      as->hb1[i] = hb;
      as->cb1[i] = hb * ks->s[i];
    }
  }
}
PCEXP_DEV void finish_ybar(int k, double fdt, const KState* ks, AdjState* as) {
  if (threadIdx.x != 0) return;
  double bb = 0;
  for (int i = 0; i < k; ++i) {
    const double yb = fdt * ks->beta * ks->s[i] * as->dots[i];
    as->ybar[i] = yb;
    bb += ks->y[i] * yb;
  }
  as->betabar = bb / ks->beta;
  for (int i = 0; i < MMAX * (MMAX + 1); ++i) as->Hbar[i] = 0.0;
}
PCEXP_DEV void finish_b0(AdjState* as) {
  if (threadIdx.x == 0) as->alpha = as->dots[0];
}

// w1 = z_{j+1} + sum_i h2_i s_i z_i,  w0 = w1 + sum_i h1_i s_i z_i
__global__ void __launch_bounds__(256) recompute_kernel(const double* __restrict__ Z, int64_t ldz, int64_t Kp, int j,
                                                        const KState* ks, double* __restrict__ w1,
                                                        double* __restrict__ w0) {
  __shared__ double c1[MMAX + 1], c0[MMAX + 1];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double h1 = ks->H1[i * MMAX + j];
    c1[i] = (ks->H[i * MMAX + j] - h1) * ks->s[i];
    c0[i] = h1 * ks->s[i];
  }
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x) {
    double a = Z[(int64_t)(j + 1) * ldz + r], b = 0;
    for (int i = 0; i <= j; ++i) {
      const double z = Z[(int64_t)i * ldz + r];
      a = fma(c1[i], z, a);
      b = fma(c0[i], z, b);
    }
    w1[r] = a;
    w0[r] = a + b;
  }
}

// ALPHA: alpha = s_{j+1} (z_{j+1} . vbar_{j+1})
__global__ void __launch_bounds__(256) alpha_kernel(const double* __restrict__ Z, int64_t ldz,
                                                    const double* __restrict__ Vb, int64_t Kp, int j, const KState* ks,
                                                    AdjState* as, double* __restrict__ partials) {
  double acc[1] = {0.0};
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma(Z[(int64_t)(j + 1) * ldz + r], Vb[(int64_t)(j + 1) * ldz + r], acc[0]);
  if (reduce_last<1>(acc, 1, partials, as)) finish_alpha(j, ks, as);
}

// mode 0 (W2): wb = vbar_{j+1}/eta + (etabar - alpha/eta) s_{j+1} z_{j+1}   (zero when last)
// mode 1 (W1): wb = win + sum_i cb2_i z_i
// then dots_i = z_i . wb (i <= j) and hbar = Hbar[i][j] - s_i dots_i, cb = hbar s_i
template <int NC>
__global__ void __launch_bounds__(256) upd_proj_kernel(int mode, const double* __restrict__ Z, int64_t ldz,
                                                       const double* __restrict__ Vb, const double* __restrict__ win,
                                                       double* __restrict__ wb, int64_t Kp, int j, int last_col,
                                                       const KState* ks, AdjState* as, double* __restrict__ partials) {
  __shared__ double cc[MMAX + 1];
  __shared__ double ca, cbz;
  const int nc = j + 1;
  if (mode == 1)
    for (int i = threadIdx.x; i < nc; i += blockDim.x) cc[i] = as->cb2[i];
  if (threadIdx.x == 0) {
    if (mode == 0 && !last_col) {
      const double eta = ks->H[(j + 1) * MMAX + j];
      const double etab = as->Hbar[(j + 1) * MMAX + j];
      ca = 1.0 / eta;
      cbz = (etab - as->alpha / eta) * ks->s[j + 1];
    } else {
      ca = 0.0;
      cbz = 0.0;
    }
  }
  __syncthreads();
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x) {
    double x;
    if (mode == 0) {
      x = (last_col ? 0.0 : ca * Vb[(int64_t)(j + 1) * ldz + r] + cbz * Z[(int64_t)(j + 1) * ldz + r]);
    } else {
      x = win[r];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < nc) x = fma(cc[c], Z[(int64_t)c * ldz + r], x);
    }
    wb[r] = x;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < nc) acc[c] = fma(Z[(int64_t)c * ldz + r], x, acc[c]);
  }
  if (reduce_last<NC>(acc, nc, partials, as)) finish_upd(mode, j, ks, as);
}

// Vbar_i += w1 hb2_i - wb2 h2_i + w0 hb1_i - wb1 h1_i (i <= j);  wb0 = wb1 + sum_i cb1_i z_i
__global__ void __launch_bounds__(256) rank_kernel(const double* __restrict__ Z, int64_t ldz, double* __restrict__ Vb,
                                                   const double* __restrict__ w1, const double* __restrict__ w0,
                                                   const double* __restrict__ wb2, const double* __restrict__ wb1,
                                                   double* __restrict__ wb0, int64_t Kp, int j, const KState* ks,
                                                   const AdjState* as) {
  __shared__ double a1[MMAX + 1], a2[MMAX + 1], a3[MMAX + 1], a4[MMAX + 1], cb1[MMAX + 1];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double h1 = ks->H1[i * MMAX + j];
    a1[i] = as->hb2[i];
    a2[i] = ks->H[i * MMAX + j] - h1;  // h2
    a3[i] = as->hb1[i];
    a4[i] = h1;
    cb1[i] = as->cb1[i];
  }
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x) {
    const double x1 = w1[r], x0 = w0[r], y2 = wb2[r], y1 = wb1[r];
    double o = y1;
    for (int i = 0; i <= j; ++i) {
      double* vb = Vb + (int64_t)i * ldz + r;
      *vb += x1 * a1[i] - y2 * a2[i] + x0 * a3[i] - y1 * a4[i];
      o = fma(cb1[i], Z[(int64_t)i * ldz + r], o);
    }
    wb0[r] = o;
  }
}

// y += (*a) x (a from device) or y += a_host x
__global__ void axpy_kernel(double* __restrict__ y, const double* __restrict__ x, const double* a_dev, double a_host,
                            int64_t n) {
  const double a = a_dev ? *a_dev * a_host : a_host;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    y[r] = fma(a, x[r], y[r]);
}

// Seeding from the adjoint ubar of u_out = u_base + factor dt beta sum_i y_i s_i z_i:
// ybar_i = factor dt beta s_i (z_i . ubar),  betabar = sum_i y_i ybar_i / beta
template <int NC>
__global__ void __launch_bounds__(256) ybar_kernel(const double* __restrict__ Z, int64_t ldz,
                                                   const double* __restrict__ ubar, int64_t Kp, int k, double fdt,
                                                   const KState* ks, AdjState* as, double* __restrict__ partials) {
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x) {
    const double x = ubar[r];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < k) acc[c] = fma(Z[(int64_t)c * ldz + r], x, acc[c]);
  }
  if (reduce_last<NC>(acc, k, partials, as)) finish_ybar(k, fdt, ks, as);
}

// Vbar_i = factor dt beta y_i ubar for i < k, zero for k <= i <= m
__global__ void vbar_init_kernel(double* __restrict__ Vb, int64_t ldz, const double* __restrict__ ubar, int64_t Kp,
                                 int k, int m, double fdt, const KState* ks) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x) {
    const double x = ubar[r];
    for (int i = 0; i <= m; ++i) Vb[(int64_t)i * ldz + r] = i < k ? fdt * ks->beta * ks->y[i] * x : 0.0;
  }
}

// bbar = (vbar_0 - v_0 (v_0 . vbar_0)) / beta + betabar v_0, with v_0 = s_0 z_0, beta = 1/s_0
__global__ void __launch_bounds__(256) b0dot_kernel(const double* __restrict__ Z, const double* __restrict__ Vb,
                                                    int64_t Kp, AdjState* as, double* __restrict__ partials) {
  double acc[1] = {0.0};
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma(Z[r], Vb[r], acc[0]);
  if (reduce_last<1>(acc, 1, partials, as)) finish_b0(as);
}

__global__ void finish_kernel(int kind, int mode, int j, int k, double fdt, const KState* ks, AdjState* as) {
  switch (kind) {
    case ADJ_YBAR: finish_ybar(k, fdt, ks, as); break;
    case ADJ_ALPHA: finish_alpha(j, ks, as); break;
    case ADJ_B0: finish_b0(as); break;
    default: finish_upd(mode, j, ks, as); break;
  }
}
__global__ void bbar_kernel(const double* __restrict__ Z, const double* __restrict__ Vb, double* __restrict__ bbar,
                            int64_t Kp, const KState* ks, const AdjState* as) {
  const double s0 = ks->s[0];
  const double cz = (as->betabar - s0 * s0 * as->alpha) * s0;  // alpha = z_0 . vbar_0
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < Kp; r += (int64_t)gridDim.x * blockDim.x)
    bbar[r] = s0 * Vb[r] + cz * Z[r];
}

template <int NC>
void launch_upd(int mode, const double* Z, int64_t ldz, const double* Vb, const double* win, double* wb, int64_t Kp,
                int j, int last_col, const KState* ks, AdjState* as, double* partials, cudaStream_t st) {
  upd_proj_kernel<NC><<<AB, 256, 0, st>>>(mode, Z, ldz, Vb, win, wb, Kp, j, last_col, ks, as, partials);
}

}  // namespace

cudaError_t launch_adj_ybar(const double* Z, int64_t ldz, const double* ubar, int64_t Kp, int k, double fdt,
                            const KState* ks, AdjState* as, double* partials, cudaStream_t st) {
  if (k < 1 || k > MMAX) return cudaErrorInvalidValue;
  if (k <= 8) ybar_kernel<8><<<AB, 256, 0, st>>>(Z, ldz, ubar, Kp, k, fdt, ks, as, partials);
  else if (k <= 16) ybar_kernel<16><<<AB, 256, 0, st>>>(Z, ldz, ubar, Kp, k, fdt, ks, as, partials);
  else ybar_kernel<32><<<AB, 256, 0, st>>>(Z, ldz, ubar, Kp, k, fdt, ks, as, partials);
  return cudaGetLastError();
}

cudaError_t launch_adj_vbar_init(double* Vb, int64_t ldz, const double* ubar, int64_t Kp, int k, int m, double fdt,
                                 const KState* ks, cudaStream_t st) {
  vbar_init_kernel<<<AB, 256, 0, st>>>(Vb, ldz, ubar, Kp, k, m, fdt, ks);
  return cudaGetLastError();
}

cudaError_t launch_adj_recompute(const double* Z, int64_t ldz, int64_t Kp, int j, const KState* ks, double* w1,
                                 double* w0, cudaStream_t st) {
  if (j + 1 > MMAX) return cudaErrorInvalidValue;
  recompute_kernel<<<AB, 256, 0, st>>>(Z, ldz, Kp, j, ks, w1, w0);
  return cudaGetLastError();
}

cudaError_t launch_adj_alpha(const double* Z, int64_t ldz, const double* Vb, int64_t Kp, int j, const KState* ks,
                             AdjState* as, double* partials, cudaStream_t st) {
  alpha_kernel<<<AB, 256, 0, st>>>(Z, ldz, Vb, Kp, j, ks, as, partials);
  return cudaGetLastError();
}

cudaError_t launch_adj_upd(int mode, const double* Z, int64_t ldz, const double* Vb, const double* win, double* wb,
                           int64_t Kp, int j, int last_col, const KState* ks, AdjState* as, double* partials,
                           cudaStream_t st) {
  const int nc = j + 1;
  if (nc > MMAX) return cudaErrorInvalidValue;
  if (nc <= 8) launch_upd<8>(mode, Z, ldz, Vb, win, wb, Kp, j, last_col, ks, as, partials, st);
  else if (nc <= 16) launch_upd<16>(mode, Z, ldz, Vb, win, wb, Kp, j, last_col, ks, as, partials, st);
  else launch_upd<32>(mode, Z, ldz, Vb, win, wb, Kp, j, last_col, ks, as, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_adj_rank(const double* Z, int64_t ldz, double* Vb, const double* w1, const double* w0,
                            const double* wb2, const double* wb1, double* wb0, int64_t Kp, int j, const KState* ks,
                            const AdjState* as, cudaStream_t st) {
  rank_kernel<<<AB, 256, 0, st>>>(Z, ldz, Vb, w1, w0, wb2, wb1, wb0, Kp, j, ks, as);
  return cudaGetLastError();
}

cudaError_t launch_adj_b0dot(const double* Z, const double* Vb, int64_t Kp, AdjState* as, double* partials,
                             cudaStream_t st) {
  b0dot_kernel<<<AB, 256, 0, st>>>(Z, Vb, Kp, as, partials);
  return cudaGetLastError();
}

cudaError_t launch_adj_bbar_from(const double* Z, const double* Vb, double* bbar, int64_t Kp, const KState* ks,
                                 const AdjState* as, cudaStream_t st) {
  bbar_kernel<<<AB, 256, 0, st>>>(Z, Vb, bbar, Kp, ks, as);
  return cudaGetLastError();
}

cudaError_t launch_adj_finish(int kind, int mode, int j, int k, double fdt, const KState* ks, AdjState* as,
                              cudaStream_t st) {
  finish_kernel<<<1, 256, 0, st>>>(kind, mode, j, k, fdt, ks, as);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* y, const double* x, const double* a_dev, double a_host, int64_t n, cudaStream_t st) {
  axpy_kernel<<<AB, 256, 0, st>>>(y, x, a_dev, a_host, n);
  return cudaGetLastError();
}

}  // namespace pcexp
