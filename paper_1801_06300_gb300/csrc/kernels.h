// Launchers of the device kernels (host-callable), shared by the C API.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pcexp.h"
#include "physics.cuh"

namespace pcexp {

constexpr int MMAX = 32;        // largest Krylov dimension
constexpr int RED_BLOCKS = 608;  // blocks of the streaming reductions (4 x 152 SMs)
constexpr int VPAD = 64;        // vector length padding (elements)

// Device-resident Arnoldi state.  V holds unnormalised vectors z_i with
// v_i = s_i z_i; the Hessenberg matrix is row-major with leading dimension MMAX.
struct KState {
  double H[(MMAX + 1) * MMAX];
  double H1[(MMAX + 1) * MMAX];  // first Gram-Schmidt pass alone (the adjoint needs both passes)
  double s[MMAX + 1];
  double coef[MMAX + 1];   // Gram-Schmidt update coefficients in units of z_i
  double acoef[MMAX + 1];  // axpy coefficients (factor * beta * y_i * s_i)
  double y[MMAX];          // phi_1(dt H_k) e_1
  double y2[MMAX];         // phi_2(dt H_k) e_1
  double beta;
  double wnorm0;
  double err_est;          // relative a-posteriori error estimate of the last phi evaluation
  double gsum[MMAX + 2];   // partitioned runs: this partition's sums of the last Gram-Schmidt pass
  double gtot[MMAX + 2];   // partitioned runs: the sums over all partitions
  int k;
  int done;
  int err;
  unsigned counter;
  int group;               // partitioned run: the passes leave their sums in gsum, unfinalised
  int skip2;               // selective form: the current column keeps its first pass
  unsigned pass2;          // bit j: column j ran the second pass
};

// Device-resident scalars of the reverse Krylov stage.
struct AdjState {
  double hb1[MMAX + 1], hb2[MMAX + 1], cb1[MMAX + 1], cb2[MMAX + 1];
  double dots[MMAX + 2];
  double ybar[MMAX];
  double Hbar[(MMAX + 1) * MMAX];  // row-major, leading dimension MMAX
  double alpha, betabar;
  double gsum[MMAX + 2];  // partitioned runs: this partition's sums of the last reduction
  unsigned counter;
  int err;
  int group;              // partitioned run: reductions leave their sums in gsum, unfinished
};

// Device-resident per-step scalars.
struct StepState {
  double dt;        // global dt (or 1 for local pseudo-steps)
  double cfl;       // CFL number in use
  double res_norm;  // density residual norm (Eq. cfl)
  double beta[2];
  int k[2];
  int err;
  unsigned counter;
  double dtmin_scratch;
  double dt_prev;  // dt of the previous ETD2 step (its divided difference of N)
  double kerr[2];  // Krylov error estimates of the two stages
  unsigned pass2[2];  // columns of each stage that ran the second Gram-Schmidt pass (bit j)
};

// Mesh/geometry/tables on the device, for one scalar type.  D = dim, NV = D + 2,
// NF = D + 1 faces per element, NPERM = 2 (2D) or 6 (3D) face-vertex permutations.
template <class T>
struct DGData {
  const T* geo;          // [E][GEO]: A^-1 (D x D row-major), sqrt|det A|, h, 1/sqrt|det A|; GEO = 8 or 12
  const int32_t* ef;     // [E][NF]: face slot (face << 4) | (side << 3) | perm
  const int32_t* fel;    // [F][2]: e_L, e_R (e_R = -tag on boundary faces)
  const int32_t* floc;   // [F]: f_L | f_R << 8 | perm_R << 16
  const T* fgeo;         // [F][4]: unit normal (D), measure factor |f| with sum_q Wf = 1 (2D) or 1/2 (3D)
  const T* Bv;           // [nq][nb]
  const T* Dv;           // [D][nq][nb]
  const T* Bf;           // [NF][NPERM][nfq][nb]
  const T* Wf;           // [nfq]
  const T* Bc;           // [nb]
  const T* Wv;           // [nq] reference volume weights
  const T* BfP;          // [NF][NPERM][nfq][nbp]: Bf with rows padded to whole 16-byte vectors
  // rotating frame (rot != 0): v_r = omega x x at the volume points [E][nq][D], v_r . n at the
  // face points [F][nfq] (the L element's), v_r at the element centroids [E][D]; null otherwise
  const T* vrq;
  const T* vrn;
  const T* vrc;
  T om[3];
  int rot;
  int64_t E, F;
  int64_t E_loc;         // elements owned by this partition (E without partitions; ghosts follow)
  Free<T> fs;
  int p;
  int dim;
};

// Point Jacobians of the DG operator at a linearisation state u, NV = D + 2.
//   Avol [D NV NV][E*nq]:  k = d'*NV*NV + v*NV + c: sum_d (A^-1)_{d'd} dF_d[v]/dU[c] at volume points
//                          (structure of arrays: entry k of every point is contiguous)
//   Bface, NJF = 2 NV NV entries per face point: k = s*NV*NV + v*NV + c: |f| w_q / sqrt(det_s)
//                          dF~[v]/dU_s[c], s = L (0), R (1), the ghost-state chain rule folded into
//                          s = L on boundary faces; in 16-byte chunks of VEC = 16 / sizeof(T)
//                          entries, [NJF / VEC][F*nfq][VEC], the NJF % VEC left over in
//                          [F*nfq][NJF % VEC] after them (bface_at), so a point's block loads as
//                          16-byte vectors
// Index of entry k of face point idx (of n) in Bface.
template <class T, int NJF>
__host__ __device__ __forceinline__ int64_t bface_at(int k, int64_t idx, int64_t n) {
  constexpr int VEC = 16 / (int)sizeof(T), NCH = NJF / VEC, R = NJF % VEC;
  return k < NCH * VEC ? ((int64_t)(k / VEC) * n + idx) * VEC + k % VEC
                       : (int64_t)NCH * VEC * n + idx * R + (k - NCH * VEC);
}

template <class T>
struct LinData {
  T* Avol;
  T* Bface;
};

// ---- DG operator (dg_kernels.cuh, instantiated per dimension in dg2d.cu / dg3d.cu)
template <class T, int D>
cudaError_t launch_dg_operator_d(const DGData<T>& d, const T* u, const T* du, T* out, T* G, const T* escale,
                                 const int* skip, cudaStream_t st, const cudaEvent_t* ev, const double* oscale);
template <class T, int D>
cudaError_t launch_linearize_d(const DGData<T>& d, const T* u, LinData<T> lin, bool faces_only, cudaStream_t st);
template <class T, int D>
cudaError_t launch_jac_apply_d(const DGData<T>& d, LinData<T> lin, const T* u_elem, const T* dv, T* out, T* G,
                               const T* escale, const int* skip, const double* oscale, cudaStream_t st,
                               const cudaEvent_t* ev, bool face_tan);
template <int D>
cudaError_t launch_tan_tables_d(const DGData<float>& d, cudaStream_t st);
template <class T, int D>
cudaError_t launch_jac_adjoint_d(const DGData<T>& d, LinData<T> lin, const T* w, T* out, T* GT, const T* escale,
                                 T osc, cudaStream_t st);
template <class T, int D>
cudaError_t launch_jvp_state_adjoint_d(const DGData<T>& d, const T* u, const T* v, const T* w, T* out, T* GT,
                                       const T* escale, T osc, cudaStream_t st);
template <class T, int D>
cudaError_t launch_wall_force_d(const DGData<T>& d, int64_t f0, const T* u, double ax, double ay, double az,
                                double* grad, double* value, double* partials, unsigned* counter, cudaStream_t st);
template <class T, int D>
cudaError_t launch_vortex_error_d(const DGData<T>& d, const T* u, const double* xq, const double* prm, double* grad,
                                  double* value, double* partials, unsigned* counter, cudaStream_t st);
template <class T, int D>
cudaError_t launch_param_adjoint_d(const DGData<T>& d, int64_t f0, int order, const T* u, const T* t, const T* w,
                                   double osc, const double* osc_dev, const double* dvel, double* acc,
                                   double* partials, unsigned* counter, cudaStream_t st);
template <class T, int D>
cudaError_t launch_vortex_param_grad_d(const DGData<T>& d, const T* u, const double* xq, const double* prm,
                                       const double* dvel, double* out, double* partials, unsigned* counter,
                                       cudaStream_t st);
template <class T, int D>
cudaError_t launch_local_dt_d(const DGData<T>& d, const T* u, const double* cfl_dev, double cfl, T* dte,
                              double* dtmin, double* partials, unsigned* counter, cudaStream_t st);

// out = R(u)  or  out = J(u) du  (du != nullptr); G is face-flux scratch [F][nfq][NV].
// escale (nullable): per-element output factor.  skip (nullable): device flag, nonzero = no-op.
// ev (nullable): three events recorded before the face kernel, between the
// two kernels and after the element kernel.  oscale (nullable, device): one
// more scalar factor on the output (the Krylov basis scale s_j).
template <class T>
cudaError_t launch_dg_operator(const DGData<T>& d, const T* u, const T* du, T* out, T* G,
                               const T* escale, const int* skip, cudaStream_t st,
                               const cudaEvent_t* ev = nullptr, const double* oscale = nullptr) {
  return d.dim == 3 ? launch_dg_operator_d<T, 3>(d, u, du, out, G, escale, skip, st, ev, oscale)
                    : launch_dg_operator_d<T, 2>(d, u, du, out, G, escale, skip, st, ev, oscale);
}
// Evaluate the point Jacobians at u (once per linearisation state): faces and volume, or
// the face blocks only (faces_only, when the volume part of J v recomputes flux tangents).
template <class T>
cudaError_t launch_linearize(const DGData<T>& d, const T* u, LinData<T> lin, cudaStream_t st,
                             bool faces_only = false) {
  return d.dim == 3 ? launch_linearize_d<T, 3>(d, u, lin, faces_only, st)
                    : launch_linearize_d<T, 2>(d, u, lin, faces_only, st);
}
// out = J(u) dv: the face part from the face point Jacobians, or (face_tan, with u_elem) from
// Riemann-flux tangents recomputed at u_elem; the volume part from the volume point
// Jacobians (u_elem null) or the flux tangents at u_elem (same ev / escale / skip / oscale
// conventions as the operator).
template <class T>
cudaError_t launch_jac_apply(const DGData<T>& d, LinData<T> lin, const T* dv, T* out, T* G, const T* escale,
                             const int* skip, const double* oscale, cudaStream_t st, const cudaEvent_t* ev,
                             const T* u_elem = nullptr, bool face_tan = false) {
  return d.dim == 3 ? launch_jac_apply_d<T, 3>(d, lin, u_elem, dv, out, G, escale, skip, oscale, st, ev, face_tan)
                    : launch_jac_apply_d<T, 2>(d, lin, u_elem, dv, out, G, escale, skip, oscale, st, ev, face_tan);
}
// Upload the reference tables [Bv | Dv] of the context's (D, p) to the constant-memory copy
// read by the FP32 flux-tangent J v on tetrahedra (device-to-device, on st; same bytes for
// every context of that order).  Triangles use the tile kernel, which reads the tables from
// global memory.
inline cudaError_t launch_tan_tables(const DGData<float>& d, cudaStream_t st) {
  return d.dim == 3 ? launch_tan_tables_d<3>(d, st) : cudaSuccess;
}
// out = (osc * diag(escale) * J(u))^T w from the point Jacobians; GT is scratch [F][nfq][2 NV].
template <class T>
cudaError_t launch_jac_adjoint(const DGData<T>& d, LinData<T> lin, const T* w, T* out, T* GT, const T* escale, T osc,
                               cudaStream_t st) {
  return d.dim == 3 ? launch_jac_adjoint_d<T, 3>(d, lin, w, out, GT, escale, osc, st)
                    : launch_jac_adjoint_d<T, 2>(d, lin, w, out, GT, escale, osc, st);
}
// out = (d/du [ (osc diag(escale) J(u) v)^T w ])^T, the second-order adjoint; GT scratch [F][nfq][2 NV].
template <class T>
cudaError_t launch_jvp_state_adjoint(const DGData<T>& d, const T* u, const T* v, const T* w, T* out, T* GT,
                                     const T* escale, T osc, cudaStream_t st) {
  return d.dim == 3 ? launch_jvp_state_adjoint_d<T, 3>(d, u, v, w, out, GT, escale, osc, st)
                    : launch_jvp_state_adjoint_d<T, 2>(d, u, v, w, out, GT, escale, osc, st);
}
// Pressure force on the slip walls along (ax, ay, az) -> *value, gradient added into grad
// (nullable); boundary faces are those with index >= f0.
template <class T>
cudaError_t launch_wall_force(const DGData<T>& d, int64_t f0, const T* u, double ax, double ay, double az,
                              double* grad, double* value, double* partials, unsigned* counter, cudaStream_t st) {
  return d.dim == 3 ? launch_wall_force_d<T, 3>(d, f0, u, ax, ay, az, grad, value, partials, counter, st)
                    : launch_wall_force_d<T, 2>(d, f0, u, ax, ay, az, grad, value, partials, counter, st);
}
// ||U_h - U_vortex||_L2 -> *value and its unnormalised gradient (times J) -> grad (nullable);
// xq: physical volume points [E][nq][D] (FP64); prm (host): eps, x_c, y_c, period, t.
template <class T>
cudaError_t launch_vortex_error(const DGData<T>& d, const T* u, const double* xq, const double* prm, double* grad,
                                double* value, double* partials, unsigned* counter, cudaStream_t st) {
  return d.dim == 3 ? launch_vortex_error_d<T, 3>(d, u, xq, prm, grad, value, partials, counter, st)
                    : launch_vortex_error_d<T, 2>(d, u, xq, prm, grad, value, partials, counter, st);
}
// dt_e = cfl h_e / ((2p+1)(|v_c| + c_c)) -> dte[E]; min over e -> *dtmin (last-block reduction).
template <class T>
cudaError_t launch_local_dt(const DGData<T>& d, const T* u, const double* cfl_dev, double cfl,
                            T* dte, double* dtmin, double* partials, unsigned* counter, cudaStream_t st) {
  return d.dim == 3 ? launch_local_dt_d<T, 3>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter, st)
                    : launch_local_dt_d<T, 2>(d, u, cfl_dev, cfl, dte, dtmin, partials, counter, st);
}
// acc[0..1] += adjoint with respect to (Mach, alpha in degrees) of the far-field faces (index >= f0):
// order 1: (dR(u)/dtheta)^T w; order 2: (d(J(u) t)/dtheta)^T w; both times osc (and *osc_dev).
// dvel: d(free-stream velocity)/dMach (x, y), then d/dalpha (x, y).
template <class T>
cudaError_t launch_param_adjoint(const DGData<T>& d, int64_t f0, int order, const T* u, const T* t, const T* w,
                                 double osc, const double* osc_dev, const double* dvel, double* acc, double* partials,
                                 unsigned* counter, cudaStream_t st) {
  return d.dim == 3 ? launch_param_adjoint_d<T, 3>(d, f0, order, u, t, w, osc, osc_dev, dvel, acc, partials, counter, st)
                    : launch_param_adjoint_d<T, 2>(d, f0, order, u, t, w, osc, osc_dev, dvel, acc, partials, counter, st);
}
// out[0] = sum w |U_h - U_ex|^2, out[1..3] = sum w (U_h - U_ex) . dU_ex/d(Mach, alpha, eps) for the
// vortex-error functional (prm: eps, x_c, y_c, period, t; dvel as for launch_param_adjoint)
template <class T>
cudaError_t launch_vortex_param_grad(const DGData<T>& d, const T* u, const double* xq, const double* prm,
                                     const double* dvel, double* out, double* partials, unsigned* counter,
                                     cudaStream_t st) {
  return d.dim == 3 ? launch_vortex_param_grad_d<T, 3>(d, u, xq, prm, dvel, out, partials, counter, st)
                    : launch_vortex_param_grad_d<T, 2>(d, u, xq, prm, dvel, out, partials, counter, st);
}
// ---- dimension-free kernels (dg_common.cu)
// basis conversions at the interface (Q_e: paper <- internal)
template <class T>
cudaError_t launch_paper_to_internal(const double* src, T* dst, const double* Q, int64_t E, int nb, int nv, cudaStream_t st);
template <class T>
cudaError_t launch_internal_to_paper(const T* src, double* dst, const double* Q, int64_t E, int nb, int nv, cudaStream_t st);
// x[e][:] *= s[e] (block of nvb entries per element)
template <class T>
cudaError_t launch_scale_elements(T* x, const T* s, int64_t E, int nvb, cudaStream_t st);
// x *= s (s a device scalar, n entries)
cudaError_t launch_scale_by_inverse(double* x, const double* s, int64_t n, cudaStream_t st);
// FP64 FMA rate of the current device (TFLOP/s) from DFMA chains on every SM
cudaError_t measure_fp64_fma_rate(double* tflops);
cudaError_t measure_fp32_fma_rate(double* tflops);
// sum_e sum_q w^_q |det A_e| (s/s0)^2 of the FP64 state u (Eq. entropy_error) -> *value
cudaError_t launch_entropy_sum(const double* u, const double* Bv, const double* Wv, const double* sd, int64_t E, int nb,
                               int nq, int nv, double gamma, double s0, double* value, double* partials,
                               unsigned* counter, cudaStream_t st);
// density residual norm sqrt(sum (R[e][0][i] / s[e])^2) / volume -> ss->res_norm, then the CFL ramp
template <class T>
cudaError_t launch_density_norm(const T* R, const T* s, int64_t E, int nb, int nv, double volume,
                                StepState* ss, double* partials, int ramp_n, int p, double cfl_max,
                                cudaStream_t st);

// ---- Krylov (krylov_kernels.cu)
// Gram-Schmidt passes.  UPD1 streams like UPD_NORM (update and norm) and PROJ2 like PROJ;
// they differ in what the last block does with the sums (cgs_finalize).
enum CgsMode { CGS_PROJ = 0, CGS_UPD_PROJ = 1, CGS_UPD_NORM = 2, CGS_NORM = 3, CGS_UPD1 = 4, CGS_PROJ2 = 5 };
template <class T>
cudaError_t launch_cgs(int mode, const T* Z, int64_t ldz, int64_t Kp, int j, T* w, T* out,
                       KState* ks, double* partials, double eta, cudaStream_t st);
// phi_1/phi_2 of dt H_k (dt from *dt_dev when non-null, else dt) -> ks->y, ks->y2,
// ks->acoef = factor * dt * beta * y_i * s_i (which = 1) or factor * dt * beta * y2_i * s_i (which = 2),
// times dt / *dt_prev when dt_prev is non-null; records k and beta into ss->k[stage], ss->beta[stage].
cudaError_t launch_phi(KState* ks, const double* dt_dev, double dt, double factor, StepState* ss,
                       int stage, cudaStream_t st, int which = 1, const double* dt_prev = nullptr);
// Checkpoint of the adaptive Krylov dimension: the error estimate of phi_1(dt H_k) e_1 at the
// current dimension k -> ks->err_est, and ks->done = 1 (the remaining columns are skipped)
// when it is <= tol.  No update coefficients are written.
cudaError_t launch_phi_check(KState* ks, const double* dt_dev, double tol, cudaStream_t st);
// Hbar = (d y / d H)^T ybar for y = phi_1(dt H) e_1 (H, Hbar: k x k row-major, leading dim ldh; device)
cudaError_t launch_phi_adjoint(const double* H, int k, int ldh, double dt, const double* ybar, double* Hbar, int* err,
                               cudaStream_t st);
// out64 = base64 + sum_i acoef_i z_i; delta = sum_i acoef_i z_i; shadow = (T) out64
template <class T>
cudaError_t launch_krylov_axpy(const double* base64, double* out64, T* shadow, T* delta, const T* Z,
                               int64_t ldz, int64_t Kp, const KState* ks, cudaStream_t st);
// a = b - a - c  (corrector input N_* - N_n = R(u_*) - R_n - J_n delta)
template <class T>
cudaError_t launch_combine_corrector(T* a, const T* b, const T* c, int64_t Kp, cudaStream_t st);
template <class Tin, class Tout>
cudaError_t launch_cast(const Tin* x, Tout* y, int64_t n, cudaStream_t st);
// out = x - y - z (z nullable)
template <class T>
cudaError_t launch_lincomb3(T* out, const T* x, const T* y, const T* z, int64_t Kp, cudaStream_t st);
// ss->dt_prev = ss->dt
cudaError_t launch_keep_dt(StepState* ss, cudaStream_t st);
// ---- partitioned runs (several contexts, one per partition)
constexpr int MAX_PARTS = 16;
struct PartPtrs {
  const void* p[MAX_PARTS];
};
// Gram-Schmidt pass of a partition: apply the pass's scalar step (breakdown test, H entries,
// scales) to the partition-summed ks->gtot (mode, column j as for launch_cgs)
cudaError_t launch_cgs_group_finalize(int mode, int j, KState* ks, double eta, cudaStream_t st);
// out[i] = sum over q < nparts of slots.p[q][i] (doubles, i < n), in partition order; op 1: min
cudaError_t launch_group_reduce(PartPtrs slots, int nparts, int n, double* out, int op, cudaStream_t st);
// ghost rows of a partition's vector x (element rows n_local .. n_local + n_ghost): row g from
// element src_elem[g] of partition src_part[g]'s copy srcs.p[src_part[g]] (nvb entries per row)
template <class T>
cudaError_t launch_gather_ghosts(T* x, PartPtrs srcs, const int32_t* src_part, const int32_t* src_elem,
                                 int64_t n_local, int64_t n_ghost, int nvb, cudaStream_t st);
// x[from, to) = 0
template <class T>
cudaError_t launch_zero_range(T* x, int64_t from, int64_t to, cudaStream_t st);
// ss->cfl = min(ss->cfl, cap) (the Krylov-error cap of the steady march)
cudaError_t launch_cap_cfl(StepState* ss, double cap, cudaStream_t st);
cudaError_t launch_reset_kstate(KState* ks, cudaStream_t st);
// ---- reverse Krylov stage (adjoint.cu, FP64)
// Reverse of the Krylov stage, step by step.  Each reduction (ybar, alpha, upd, b0dot) leaves
// its sums in as->dots and finishes in its last block; in a partitioned run (as->group) it
// leaves them in as->gsum instead, and launch_adj_finish(kind, ...) finishes from as->dots once
// they are summed over the partitions.
enum AdjReduction { ADJ_YBAR = 0, ADJ_ALPHA = 1, ADJ_UPD0 = 2, ADJ_UPD1 = 3, ADJ_B0 = 4 };
cudaError_t launch_adj_ybar(const double* Z, int64_t ldz, const double* ubar, int64_t Kp, int k, double fdt,
                            const KState* ks, AdjState* as, double* partials, cudaStream_t st);
cudaError_t launch_adj_vbar_init(double* Vb, int64_t ldz, const double* ubar, int64_t Kp, int k, int m, double fdt,
                                 const KState* ks, cudaStream_t st);
cudaError_t launch_adj_recompute(const double* Z, int64_t ldz, int64_t Kp, int j, const KState* ks, double* w1,
                                 double* w0, cudaStream_t st);
cudaError_t launch_adj_alpha(const double* Z, int64_t ldz, const double* Vb, int64_t Kp, int j, const KState* ks,
                             AdjState* as, double* partials, cudaStream_t st);
cudaError_t launch_adj_upd(int mode, const double* Z, int64_t ldz, const double* Vb, const double* win, double* wb,
                           int64_t Kp, int j, int last_col, const KState* ks, AdjState* as, double* partials,
                           cudaStream_t st);
cudaError_t launch_adj_rank(const double* Z, int64_t ldz, double* Vb, const double* w1, const double* w0,
                            const double* wb2, const double* wb1, double* wb0, int64_t Kp, int j, const KState* ks,
                            const AdjState* as, cudaStream_t st);
cudaError_t launch_adj_b0dot(const double* Z, const double* Vb, int64_t Kp, AdjState* as, double* partials,
                             cudaStream_t st);
cudaError_t launch_adj_bbar_from(const double* Z, const double* Vb, double* bbar, int64_t Kp, const KState* ks,
                                 const AdjState* as, cudaStream_t st);
cudaError_t launch_adj_finish(int kind, int mode, int j, int k, double fdt, const KState* ks, AdjState* as,
                              cudaStream_t st);
cudaError_t launch_axpy(double* y, const double* x, const double* a_dev, double a_host, int64_t n, cudaStream_t st);
cudaError_t launch_set_dt(StepState* ss, double dt, cudaStream_t st);
cudaError_t launch_set_cfl(StepState* ss, double cfl, cudaStream_t st);
cudaError_t launch_set_param(double* param, double v, cudaStream_t st);
cudaError_t launch_copy_dt(StepState* ss, const double* param, cudaStream_t st);

}  // namespace pcexp
