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
// overflow FP32 storage).
// Each streaming kernel writes per-block partial sums; the last block to
// finish (atomic ticket) reduces them in a fixed order and applies the scalar
// update, so results are deterministic and no extra launch is needed.
// Partial products are accumulated in FP64 (FP64 form) or in FP32 over 8
// elements and then in FP64 (FP32-mixed form).
#include <cfloat>

#include "kernels.h"

namespace pcexp {

// Elements per thread per row-loop iteration: 16-byte (double2) loads in FP64;
// in FP32 two float4 loads for the read-only reductions and one float4 where the
// kernel also keeps every basis element in registers (update + projection).
template <class T, int MODE> struct VecN {
  static constexpr int N = sizeof(T) == 8 ? 2 : ((MODE == CGS_PROJ || MODE == CGS_NORM) ? 8 : 4);
};

template <class T, int VN>
PCEXP_DEV void load_vec(const T* p, T (&x)[VN], bool stream) {
  if constexpr (sizeof(T) == 8) {
    static_assert(VN == 2, "FP64 uses double2");
    double2 a = stream ? __ldcs(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
    x[0] = a.x;
    x[1] = a.y;
  } else {
#pragma unroll
    for (int h = 0; h < VN / 4; ++h) {
      float4 a = stream ? __ldcs(reinterpret_cast<const float4*>(p) + h) : reinterpret_cast<const float4*>(p)[h];
      x[4 * h + 0] = a.x;
      x[4 * h + 1] = a.y;
      x[4 * h + 2] = a.z;
      x[4 * h + 3] = a.w;
    }
  }
}
template <class T, int VN>
PCEXP_DEV void store_vec(T* p, const T (&x)[VN]) {
  if constexpr (sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  } else {
#pragma unroll
    for (int h = 0; h < VN / 4; ++h)
      reinterpret_cast<float4*>(p)[h] = make_float4(x[4 * h], x[4 * h + 1], x[4 * h + 2], x[4 * h + 3]);
  }
}

// sum_v a[v] * b[v] in T (FP32 partial over VN elements in the mixed form), returned in FP64
template <class T, int VN>
PCEXP_DEV double dot_vec(const T (&a)[VN], const T (&b)[VN]) {
  T s = 0;
#pragma unroll
  for (int v = 0; v < VN; ++v) s = fma(a[v], b[v], s);
  return (double)s;
}

// Scalar stage logic run by one thread of the last block.
PCEXP_DEV void cgs_finalize(int mode, int j, const double* dots, KState* ks, double eta) {
  if (mode == CGS_NORM) {
    const double b2 = dots[0];
    const double beta = sqrt(b2);
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
  // w = J v_j is already normalised by s_j (applied by the J v kernel)
  if (mode == CGS_PROJ || mode == CGS_UPD_PROJ) {
    bool ok = true;
    for (int i = 0; i <= j; ++i) {
      const double si = ks->s[i];
      const double h = si * dots[i];
      ok = ok && isfinite(h);
      if (mode == CGS_PROJ) ks->H[i * MMAX + j] = h;
      else ks->H[i * MMAX + j] += h;
      ks->coef[i] = si * si * dots[i];
    }
    if (mode == CGS_PROJ) ks->wnorm0 = sqrt(dots[j + 1]);
    if (!ok) {
      ks->err = 1;
      ks->done = 1;
    }
    return;
  }
  // CGS_UPD_NORM
  const double nn = sqrt(dots[0]);
  const double hn = nn;
  ks->H[(j + 1) * MMAX + j] = hn;
  ks->k = j + 1;
  if (!isfinite(hn)) {
    ks->err = 1;
    ks->done = 1;
  } else if (nn == 0.0 || hn <= eta * ks->wnorm0) {
    ks->done = 1;  // happy breakdown: K_{j+1} is invariant
  } else {
    ks->s[j + 1] = 1.0 / nn;
  }
}

template <class T, int NC, int MODE>
__global__ void __launch_bounds__(256) cgs_kernel(const T* __restrict__ Z, int64_t ldz, int64_t Kp, int j,
                                                  T* __restrict__ w, T* __restrict__ out, KState* ks,
                                                  double* __restrict__ partials, double eta) {
  constexpr int VN = VecN<T, MODE>::N;
  constexpr int NACC = (MODE == CGS_PROJ) ? NC + 1 : (MODE == CGS_UPD_PROJ ? NC : 1);
  __shared__ T scoef[NC > 0 ? NC : 1];
  __shared__ double red[8][NACC];
  __shared__ bool last;
  if (ks->done) return;  // breakdown reached earlier: uniform early exit
  const int nc = (MODE == CGS_NORM) ? 0 : j + 1;
  if (MODE == CGS_UPD_PROJ || MODE == CGS_UPD_NORM)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) scoef[c] = (T)ks->coef[c];
  __syncthreads();
  double acc[NACC];
#pragma unroll
  for (int c = 0; c < NACC; ++c) acc[c] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * VN;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r < Kp; r += stride) {
    T x[VN];
    load_vec<T, VN>(w + r, x, false);
    if constexpr (MODE == CGS_NORM) {
      acc[0] += dot_vec<T, VN>(x, x);
    } else if constexpr (MODE == CGS_PROJ) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < nc) {
          T z[VN];
          load_vec<T, VN>(Z + c * ldz + r, z, true);
          acc[c] += dot_vec<T, VN>(z, x);
        }
      }
      acc[NC] += dot_vec<T, VN>(x, x);
    } else {
      T zc[NC][VN];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < nc) {
          load_vec<T, VN>(Z + c * ldz + r, zc[c], true);
#pragma unroll
          for (int v = 0; v < VN; ++v) x[v] = fma(-scoef[c], zc[c][v], x[v]);
        }
      }
      if constexpr (MODE == CGS_UPD_PROJ) {
        store_vec<T, VN>(w + r, x);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < nc) acc[c] += dot_vec<T, VN>(zc[c], x);
      } else {
        store_vec<T, VN>(out + r, x);
        acc[0] += dot_vec<T, VN>(x, x);
      }
    }
  }
  // block reduction (fixed order)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NACC; ++c) {
    double a = acc[c];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[wid][c] = a;
  }
  __syncthreads();
  const int nred = (MODE == CGS_PROJ) ? nc + 1 : (MODE == CGS_UPD_PROJ ? nc : 1);
  for (int c = threadIdx.x; c < nred; c += blockDim.x) {
    double a = 0;
    for (int q = 0; q < nw; ++q) a += red[q][(MODE == CGS_PROJ && c == nc) ? NC : c];
    partials[(int64_t)c * gridDim.x + blockIdx.x] = a;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ks->counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double dots[MMAX + 2];
  for (int c = wid; c < nred; c += nw) {
    double a = 0;
    for (unsigned b = lane; b < gridDim.x; b += 32) a += __ldcg(partials + (int64_t)c * gridDim.x + b);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) dots[c] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cgs_finalize(MODE, j, dots, ks, eta);
    ks->counter = 0;
  }
}

template <class T, int MODE>
static void cgs_dispatch(int nc, const T* Z, int64_t ldz, int64_t Kp, int j, T* w, T* out, KState* ks,
                         double* partials, double eta, unsigned grid, cudaStream_t st) {
  if (nc <= 4) cgs_kernel<T, 4, MODE><<<grid, 256, 0, st>>>(Z, ldz, Kp, j, w, out, ks, partials, eta);
  else if (nc <= 8) cgs_kernel<T, 8, MODE><<<grid, 256, 0, st>>>(Z, ldz, Kp, j, w, out, ks, partials, eta);
  else if (nc <= 16) cgs_kernel<T, 16, MODE><<<grid, 256, 0, st>>>(Z, ldz, Kp, j, w, out, ks, partials, eta);
  else cgs_kernel<T, 32, MODE><<<grid, 256, 0, st>>>(Z, ldz, Kp, j, w, out, ks, partials, eta);
}

template <class T>
cudaError_t launch_cgs(int mode, const T* Z, int64_t ldz, int64_t Kp, int j, T* w, T* out, KState* ks,
                       double* partials, double eta, cudaStream_t st) {
  const int64_t per = 256LL * 2;
  int64_t g = (Kp + per - 1) / per;
  if (g > RED_BLOCKS) g = RED_BLOCKS;
  if (g < 1) g = 1;
  const unsigned grid = (unsigned)g;
  const int nc = j + 1;
  if (nc > MMAX) return cudaErrorInvalidValue;
  switch (mode) {
    case CGS_NORM: cgs_kernel<T, 0, CGS_NORM><<<grid, 256, 0, st>>>(Z, ldz, Kp, j, w, out, ks, partials, eta); break;
    case CGS_PROJ: cgs_dispatch<T, CGS_PROJ>(nc, Z, ldz, Kp, j, w, out, ks, partials, eta, grid, st); break;
    case CGS_UPD_PROJ: cgs_dispatch<T, CGS_UPD_PROJ>(nc, Z, ldz, Kp, j, w, out, ks, partials, eta, grid, st); break;
    case CGS_UPD_NORM: cgs_dispatch<T, CGS_UPD_NORM>(nc, Z, ldz, Kp, j, w, out, ks, partials, eta, grid, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ phi kernel
// exp of the augmented matrix A = [[dt H_k, e_1, 0], [0, 0, 1], [0, 0, 0]] by
// scaling and squaring with the [8/8] diagonal Pade approximant
//   r(X) = N(X) / N(-X),  N(X) = sum_j c_j X^j,  c_j = (16-j)! 8! / (16! j! (8-j)!),
// applied to X = A / 2^s with ||X||_1 <= 1, where the Pade error is far below
// FP64 rounding.  Column k of exp(A) holds phi_1(dt H) e_1, column k+1 phi_2(dt H) e_1.
constexpr int PN = MMAX + 2;

__device__ void mat_mul(const double* A, const double* B, double* C, int n) {
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, jj = t - i * n;
    double a = 0;
    for (int l = 0; l < n; ++l) a = fma(A[i * PN + l], B[l * PN + jj], a);
    C[i * PN + jj] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(512) phi_kernel(KState* ks, const double* dt_dev, double dt_host,
                                                  double factor, StepState* ss, int stage) {
  extern __shared__ double sm[];
  double* A = sm;             // X, later the result
  double* B2 = A + PN * PN;
  double* B4 = B2 + PN * PN;
  double* B6 = B4 + PN * PN;
  double* Nm = B6 + PN * PN;  // V + U
  double* Dm = Nm + PN * PN;  // V - U
  double* Tm = Dm + PN * PN;
  __shared__ int s_sq;
  __shared__ int piv_row;
  const int k = ks->k;
  const double dt = dt_dev ? *dt_dev : dt_host;
  if (k == 0 || ks->err) {
    if (threadIdx.x == 0) {
      for (int i = 0; i <= MMAX; ++i) ks->acoef[i] = 0.0;
      if (ss) {
        ss->k[stage] = 0;
        ss->beta[stage] = ks->beta;
        if (ks->err) ss->err = 1;
      }
    }
    return;
  }
  const int n = k + 2;
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
  if (threadIdx.x == 0) {
    double nrm = 0;
    for (int jj = 0; jj < n; ++jj) {
      double c = 0;
      for (int i = 0; i < n; ++i) c += fabs(A[i * PN + jj]);
      nrm = fmax(nrm, c);
    }
    int s = 0;
    if (nrm > 1.0) s = (int)ceil(log2(nrm));
    if (!isfinite(nrm) || s > 1000) s = -1;
    s_sq = s;
  }
  __syncthreads();
  if (s_sq < 0) {
    if (threadIdx.x == 0) {
      ks->err = 1;
      if (ss) ss->err = 1;
    }
    return;
  }
  const double sc = ldexp(1.0, -s_sq);
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, jj = t - i * n;
    A[i * PN + jj] *= sc;
  }
  __syncthreads();
  // Pade [8/8] coefficients
  double c[9];
  c[0] = 1.0;
  for (int jj = 1; jj <= 8; ++jj) c[jj] = c[jj - 1] * (double)(8 - jj + 1) / (double)(jj * (16 - jj + 1));
  mat_mul(A, A, B2, n);
  mat_mul(B2, B2, B4, n);
  mat_mul(B4, B2, B6, n);
  // B8 into Tm
  mat_mul(B4, B4, Tm, n);
  // V = c0 I + c2 B2 + c4 B4 + c6 B6 + c8 B8 -> Dm ; W = c1 I + c3 B2 + c5 B4 + c7 B6 -> Nm
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, jj = t - i * n;
    const int o = i * PN + jj;
    const double id = (i == jj) ? 1.0 : 0.0;
    Dm[o] = c[0] * id + c[2] * B2[o] + c[4] * B4[o] + c[6] * B6[o] + c[8] * Tm[o];
    Nm[o] = c[1] * id + c[3] * B2[o] + c[5] * B4[o] + c[7] * B6[o];
  }
  __syncthreads();
  mat_mul(A, Nm, Tm, n);  // U = X W
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, jj = t - i * n;
    const int o = i * PN + jj;
    const double V = Dm[o], U = Tm[o];
    Nm[o] = V + U;
    Dm[o] = V - U;
  }
  __syncthreads();
  // solve Dm X = Nm (Gaussian elimination, partial pivoting); X overwrites Nm
  for (int col = 0; col < n; ++col) {
    if (threadIdx.x == 0) {
      int pr = col;
      double best = fabs(Dm[col * PN + col]);
      for (int i = col + 1; i < n; ++i) {
        const double v = fabs(Dm[i * PN + col]);
        if (v > best) {
          best = v;
          pr = i;
        }
      }
      piv_row = pr;
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != col) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double a = Dm[col * PN + t];
        Dm[col * PN + t] = Dm[pr * PN + t];
        Dm[pr * PN + t] = a;
        double b = Nm[col * PN + t];
        Nm[col * PN + t] = Nm[pr * PN + t];
        Nm[pr * PN + t] = b;
      }
      __syncthreads();
    }
    const double piv = Dm[col * PN + col];
    for (int t = threadIdx.x; t < (n - col - 1) * n; t += blockDim.x) {
      const int i = col + 1 + t / n, jj = t % n;
      const double f = Dm[i * PN + col] / piv;
      Nm[i * PN + jj] -= f * Nm[col * PN + jj];
      if (jj > col) Dm[i * PN + jj] -= f * Dm[col * PN + jj];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n - col - 1; t += blockDim.x) Dm[(col + 1 + t) * PN + col] = 0.0;
    __syncthreads();
  }
  for (int col = n - 1; col >= 0; --col) {
    const double piv = Dm[col * PN + col];
    for (int t = threadIdx.x; t < n; t += blockDim.x) Nm[col * PN + t] /= piv;
    __syncthreads();
    for (int t = threadIdx.x; t < col * n; t += blockDim.x) {
      const int i = t / n, jj = t % n;
      Nm[i * PN + jj] -= Dm[i * PN + col] * Nm[col * PN + jj];
    }
    __syncthreads();
  }
  // squaring
  double* X = Nm;
  double* Y = Tm;
  for (int it = 0; it < s_sq; ++it) {
    mat_mul(X, X, Y, n);
    double* t = X;
    X = Y;
    Y = t;
  }
  if (threadIdx.x == 0) {
    const double beta = ks->beta;
    bool ok = true;
    for (int i = 0; i < k; ++i) {
      const double y1 = X[i * PN + k], y2 = X[i * PN + k + 1];
      ks->y[i] = y1;
      ks->y2[i] = y2;
      ks->acoef[i] = factor * dt * beta * y1 * ks->s[i];
      ok = ok && isfinite(ks->acoef[i]);
    }
    for (int i = k; i <= MMAX; ++i) ks->acoef[i] = 0.0;
    if (!ok) ks->err = 1;
    if (ss) {
      ss->k[stage] = k;
      ss->beta[stage] = beta;
      if (!ok) ss->err = 1;
    }
  }
}

cudaError_t launch_phi(KState* ks, const double* dt_dev, double dt, double factor, StepState* ss, int stage,
                       cudaStream_t st) {
  const size_t smem = 7 * PN * PN * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(phi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  phi_kernel<<<1, 512, smem, st>>>(ks, dt_dev, dt, factor, ss, stage);
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
  }
  for (int i = threadIdx.x; i < (MMAX + 1) * MMAX; i += blockDim.x) ks->H[i] = 0.0;
}
cudaError_t launch_reset_kstate(KState* ks, cudaStream_t st) {
  reset_kstate_kernel<<<1, 256, 0, st>>>(ks);
  return cudaGetLastError();
}

__global__ void set_dt_kernel(StepState* ss, double dt) { ss->dt = dt; }
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
template cudaError_t launch_combine_corrector<double>(double*, const double*, const double*, int64_t, cudaStream_t);
template cudaError_t launch_combine_corrector<float>(float*, const float*, const float*, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace pcexp
