/*
 * pcexp.h -- C interface of the GB300 library for the Krylov step of the
 * predictor-corrector exponential (PCEXP) scheme on the DG discretisation of
 * the Euler equations (Li, Luo, Wang & Ju, "An Exponential Time-Integrator
 * Scheme for Steady and Unsteady Inviscid Flows").
 *
 * The problem statement follows the paper: a mesh, a DG order p and a state
 * u (Sec. 4.2, Eq. uexp), a time step dt and a Krylov dimension m give the
 * state at t + dt (Sec. 2.1, Eq. s9/s10); steady runs march to a residual
 * drop with the CFL ramp of Eq. cfl (Sec. 5.2).
 *
 * Conventions shared by every call
 *   - Every function returns PCEXP_OK (0) or a negative PCEXP_ERR_* code and
 *     never aborts the process; pcexp_status_string() names a code.
 *   - State-shaped arrays hold K = n_elem * n_var * n_basis doubles laid out
 *     [element][variable][basis function]; variables are (rho, rho u, rho v,
 *     rho E).  With basis_io == PCEXP_BASIS_PAPER the coefficients are those
 *     of the paper's element basis (Eq. basis: scaled Cartesian monomials
 *     about the centroid, orthonormalised by modified Gram-Schmidt,
 *     Algorithm 1); with PCEXP_BASIS_INTERNAL they are those of the library's
 *     own orthonormal basis (a reference-triangle orthonormal basis scaled by
 *     |det A_e|^-1/2).  Both bases are orthonormal, so norms and inner
 *     products agree in either.
 *   - on_device != 0: pointers are device pointers read/written on the
 *     context's stream; otherwise host pointers, copied synchronously.
 *   - The caller owns every pointer it passes; nothing is retained after a
 *     call returns.  The library owns its internal device buffers and frees
 *     them in pcexp_destroy().
 *   - One context per stream; a context is not thread-safe.
 *   - Krylov breakdown is not an error: it is reported in pcexp_step_info.
 */
#ifndef PCEXP_H
#define PCEXP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PCEXP_OK 0
#define PCEXP_ERR_INVALID_ARG (-1) /* bad pointer, size, order or option */
#define PCEXP_ERR_MESH (-2)        /* unmatched / non-conforming / inverted mesh */
#define PCEXP_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define PCEXP_ERR_OOM (-4)         /* device allocation failed */
#define PCEXP_ERR_NONFINITE (-5)   /* a norm, beta or h_{j+1,j} was NaN/Inf */
#define PCEXP_ERR_TIMEOUT (-6)     /* a partition of a group missed a rendezvous (failed or stalled) */
#define PCEXP_ERR_UNSUPPORTED (-7) /* valid request this build does not cover */

/* ---- boundary tags (Sec. 4.4, Sec. 5.2) ---- */
#define PCEXP_BC_SLIP_WALL 1 /* ghost state mirrors the normal velocity (relative to the frame) */
#define PCEXP_BC_FARFIELD 2  /* characteristic (Riemann-invariant) ghost state */
#define PCEXP_BC_SYMMETRY 3  /* symmetry plane (Sec. 5.2, sphere case): the slip-wall ghost state of
                                inviscid flow; not part of the wall-force functionals */

/* ---- options ---- */
#define PCEXP_FP64 0       /* every vector, flux and reduction in FP64 */
#define PCEXP_FP32_MIXED 1 /* R, J v and the Krylov basis in FP32; reductions,
                              Hessenberg, phi and the master state in FP64 */
#define PCEXP_BASIS_PAPER 0
#define PCEXP_BASIS_INTERNAL 1

/* Re-orthogonalisation of the Arnoldi process (Sec. 2.2, Eq. vm-vm2; the paper names the
 * classical Arnoldi process and no Gram-Schmidt variant).  Every column j first projects
 * w = J v_j on v_1..v_j and subtracts (one classical Gram-Schmidt pass, w_1 = w - V h).
 * ALWAYS: a second pass projects and subtracts again (CGS2).  SELECTIVE: the second pass
 * runs only when the first cancelled much of w, ||w_1|| < ||w|| / sqrt(2) (the criterion of
 * Daniel, Gragg, Kaufman and Stewart, 1976); otherwise v_{j+1} = w_1 / ||w_1|| and column j
 * of H is the first pass's.  The decision is taken on the device per column, from the FP64
 * sums.  AUTO (0): ALWAYS for PCEXP_FP64 contexts (the form whose reverse step replays both
 * passes) and SELECTIVE for PCEXP_FP32_MIXED, where the basis is stored in FP32 and a second
 * pass after a first without cancellation changes it by FP32 rounding only.  SELECTIVE is
 * not offered for PCEXP_FP64 contexts (UNSUPPORTED). */
#define PCEXP_REORTH_AUTO 0
#define PCEXP_REORTH_ALWAYS 1
#define PCEXP_REORTH_SELECTIVE 2

#define PCEXP_SCHEME_PCEXP 0 /* Eq. s9 + s10 */
#define PCEXP_SCHEME_EXP1 1  /* Eq. s9 alone (first stage) */
#define PCEXP_SCHEME_ETD2 2  /* Eq. s7: ETD1 + dt (dt/dt_{n-1}) phi_2(dt J_n)(N_n - N_{n-1}), history in
                                the context; the first step after a state change is ETD1 (Eq. s8) */

#define PCEXP_DT_GIVEN 0      /* global dt passed by the caller */
#define PCEXP_DT_GLOBAL_CFL 1 /* dt = min_e dt_e(CFL), Eq. x3d */
#define PCEXP_DT_LOCAL_CFL 2  /* local steps: du/dtau = D R(u), D = diag(dt_e(CFL)),
                                 unit pseudo-step (reading for steady runs) */

#define PCEXP_PROJ_FREESTREAM 0 /* params: none */
#define PCEXP_PROJ_VORTEX 1     /* params: eps, xc, yc, period (0 = none) [, core radius R (default
                                   1; distances in units of R)]; in 3D the planar vortex, uniform
                                   in z, zero z-velocity */
#define PCEXP_PROJ_BLOBS 2      /* params: radius, then n x (x, y, a_rho, a_p) */

#define PCEXP_MAX_KRYLOV 32 /* largest supported m (the paper uses m = 30) */

/* Mesh of positively oriented triangles (dim = 2, orders p = 0..3) or tetrahedra
 * (dim = 3, p = 0..2; higher orders return PCEXP_ERR_UNSUPPORTED).
 * coords [n_vert][dim]; elem_vert [n_elem][dim+1]; vert_master [n_vert] maps
 * each vertex to its periodic master (NULL: no periodic identification);
 * bface_vert [n_bface][dim] + bface_tag [n_bface] list the tagged boundary
 * faces (edges in 2D, triangles in 3D).  Faces are matched on master vertices;
 * a face with no partner and no tag, or shared by more than two elements, is a
 * PCEXP_ERR_MESH.  A face's quadrature points are those of its L element (the
 * lower element index) in that element's local face-vertex order.  Quadrature (the
 * paper leaves it open): Gauss rules with p + 1 points per direction (collapsed on
 * triangles and tetrahedra), except tetrahedra at p = 2, which take fully symmetric
 * rules of the same degree 5 with 14 volume and 7 face points. */
typedef struct pcexp_mesh {
  int32_t dim;
  int64_t n_vert;
  const double* coords;
  int64_t n_elem;
  const int32_t* elem_vert;
  const int32_t* vert_master;
  int64_t n_bface;
  const int32_t* bface_vert;
  const int32_t* bface_tag;
} pcexp_mesh;

/* Free stream (nondimensional): gamma (7/5 in the paper, Sec. 4.1), Mach
 * number, flow angle in degrees, density and pressure; and the angular velocity omega
 * of a rotating frame of reference (Sec. 4.1, Eq. euler; zero: a fixed frame).  With
 * omega != 0 the flux is F_abs - U v_r^T, v_r = omega x x, the source -rho omega x v is
 * added, the Roe waves move with the frame and the slip wall mirrors the velocity relative
 * to it; the mesh must have no periodic identification and no far-field faces, and in 2D
 * only omega[2] may be nonzero (otherwise PCEXP_ERR_INVALID_ARG).  The steps' local time
 * steps use the velocity relative to the frame at the centroid.  The adjoint entry points
 * (pcexp_step_backward, pcexp_jvp_state_adjoint) return PCEXP_ERR_UNSUPPORTED in a
 * rotating frame. */
typedef struct pcexp_physics {
  double gamma;
  double mach;
  double alpha_deg;
  double rho_inf;
  double p_inf;
  double omega[3];
} pcexp_physics;

typedef struct pcexp_options {
  int32_t precision;    /* PCEXP_FP64 | PCEXP_FP32_MIXED */
  int32_t m_max;        /* Krylov storage, 1..PCEXP_MAX_KRYLOV */
  double breakdown_eta; /* happy breakdown when h_{j+1,j} <= eta ||J v_j||; <=0: default
                           (1e-12 FP64, 1e-6 FP32-mixed) */
  int32_t basis_io;     /* PCEXP_BASIS_PAPER | PCEXP_BASIS_INTERNAL */
  double krylov_tol;    /* Krylov tolerance (Sec. 5 uses 1e-5); <= 0: fixed dimension m.  > 0: in
                           every step stage the Arnoldi process ends at the first k = 5, 10, ...
                           (k < m) whose relative error estimate (below) is <= krylov_tol, and the
                           steady march caps its CFL from the first stage's estimate:
                           cap = CFL_used * clamp(0.8 (tol / est)^(1/2), 1/4, 2) */
  int32_t reorth;       /* PCEXP_REORTH_AUTO | PCEXP_REORTH_ALWAYS | PCEXP_REORTH_SELECTIVE */
} pcexp_options;

typedef struct pcexp_step_info {
  int32_t krylov_dim[2]; /* Arnoldi dimension reached in each stage (0 if skipped) */
  double beta[2];        /* ||R_n|| and ||N_* - N_n|| */
  double dt;             /* dt used (1 for local pseudo-steps) */
  double res_norm;       /* density residual norm of Eq. cfl at u_n */
  double krylov_err[2];  /* relative a-posteriori error estimate of each stage's phi product
                            (Saad 1992, cited in Sec. 2.2): dt h_{k+1,k} |e_k^T phi_2(dt H_k) e_1|
                            / ||phi_1(dt H_k) e_1|| at the dimension k used */
  uint32_t reorth_cols[2]; /* bit j set: Arnoldi column j of the stage ran the second
                              Gram-Schmidt pass (all columns under PCEXP_REORTH_ALWAYS) */
} pcexp_step_info;

typedef struct pcexp_steady_info {
  int32_t iterations;
  double res_first; /* ||R(rho_1)|| */
  double res_last;  /* ||R(rho_n)|| at exit */
  int32_t converged;
} pcexp_steady_info;

typedef struct pcexp_ctx pcexp_ctx;

/* Builds faces, geometry, quadrature, bases and device buffers for order p
 * (0..3).  cuda_stream is a cudaStream_t (NULL: the legacy default stream).
 * Errors: INVALID_ARG, MESH, CUDA, OOM.  On error *out is NULL. */
int pcexp_create(pcexp_ctx** out, const pcexp_mesh* mesh, int p,
                 const pcexp_physics* phys, const pcexp_options* opt, void* cuda_stream);

/* Frees every device buffer of the context.  NULL is a no-op. */
int pcexp_destroy(pcexp_ctx* ctx);

/* Sizes: number of elements, basis functions per variable, variables and
 * K = n_elem * n_var * n_basis.  Any output pointer may be NULL. */
int pcexp_sizes(const pcexp_ctx* ctx, int64_t* n_elem, int32_t* n_basis,
                int32_t* n_var, int64_t* K);

/* Sets / reads the master state u (K doubles). */
int pcexp_set_state(pcexp_ctx* ctx, const double* U, int on_device);
int pcexp_get_state(pcexp_ctx* ctx, double* U, int on_device);

/* L2 projection of an analytic state (PCEXP_PROJ_*) onto the DG space,
 * written into the master state.  params as listed at PCEXP_PROJ_*. */
int pcexp_project_state(pcexp_ctx* ctx, int kind, const double* params, int n_params);

/* R(U) of Eq. euler3 (Sec. 4.2): volume term, Roe flux on interior and
 * periodic faces, Roe flux against the ghost state on boundary faces. */
int pcexp_residual(pcexp_ctx* ctx, const double* U, double* R, int on_device);

/* J(U) v, the exact directional derivative of R at U (Eq. jac1, jac2),
 * matrix-free by a tangent-linear kernel. */
int pcexp_jvp(pcexp_ctx* ctx, const double* U, const double* v, double* Jv, int on_device);

/* J(U)^T w, the adjoint of pcexp_jvp (transpose of the exact Jacobian of
 * Eq. jac1, jac2), from the same point Jacobians, in the same basis as U. */
int pcexp_vjp(pcexp_ctx* ctx, const double* U, const double* w, double* JTw, int on_device);

/* (d/dU [w^T J(U) v])^T: the adjoint, with respect to the linearisation state U,
 * of the Jacobian-vector product (second derivatives of R; J_n = J(u_n) depends
 * on u_n, Eq. s9/s10).  FP64 contexts only (PCEXP_ERR_UNSUPPORTED otherwise). */
int pcexp_jvp_state_adjoint(pcexp_ctx* ctx, const double* U, const double* v, const double* w,
                            double* out, int on_device);

/* Time-step sizes of Eq. x3d at the master state: local != 0 writes n_elem
 * values dt_e, otherwise one value min_e dt_e. */
int pcexp_compute_dt(pcexp_ctx* ctx, double cfl, int local, double* dt, int on_device);

/* Arnoldi process (Eq. vm-vm2) for J(U) started from b: V [m+1][K] (column j
 * = v_{j+1}, same basis as U), H [(m+1) * m] row-major Hessenberg H~_m,
 * *k = dimension reached (< m on happy breakdown), *beta = ||b||.  Classical
 * Gram-Schmidt with the context's re-orthogonalisation (PCEXP_REORTH_*: two passes, or the
 * second pass only where the first cancelled).  V may be NULL. */
int pcexp_arnoldi(pcexp_ctx* ctx, const double* U, const double* b, int m,
                  double* V, double* H, int* k, double* beta, int on_device);

/* phi_1(dt H) e_1 and phi_2(dt H) e_1 (Eq. Phi1, Phi2, final) for the k x k
 * matrix H (row-major, leading dimension ldh; host arrays), evaluated on the
 * device in FP64 from the exponential of the augmented matrix
 * [[dt H, e_1, 0], [0, 0, 1], [0, 0, 0]] by scaling and squaring with a
 * diagonal Pade approximant.  phi2 may be NULL.  k <= PCEXP_MAX_KRYLOV. */
int pcexp_phi(pcexp_ctx* ctx, const double* H, int k, int ldh, double dt,
              double* phi1, double* phi2);

/* Adjoint of pcexp_phi: Hbar = (d y / d H)^T ybar for y = phi_1(dt H) e_1
 * (k x k, row-major with leading dimension ldh; host arrays).  Computed on the
 * device in FP64 as dt times the leading block of the Frechet derivative
 * L_exp(A^T, Ybar), the top-right block of exp([[A^T, Ybar], [0, A^T]]). */
int pcexp_phi_adjoint(pcexp_ctx* ctx, const double* H, int k, int ldh, double dt,
                      const double* ybar, double* Hbar);

/* Reverse of one PCEXP step (Eq. s9, s10) exactly as computed with the global
 * time step dt and Krylov dimension m: given the state U = u_n (the checkpoint)
 * and ubar_next, the adjoint of u_{n+1}, writes ubar = (du_{n+1}/du_n)^T
 * ubar_next and, when theta_bar (host, 2 doubles) is not NULL, the adjoint of the
 * free-stream parameters theta = (Mach number, flow angle in degrees) of the step,
 * theta_bar = (du_{n+1}/dtheta)^T ubar_next (theta enters through the far-field ghost
 * state of every R and J v of the step; the mixed second derivatives of J_n are
 * included).  The step is recomputed from u_n; dt is held constant.  Covers the
 * adjoint of R, of J_n (including its dependence on u_n), of the CGS2 Arnoldi
 * processes, of phi and of both updates.  FP64 contexts only
 * (PCEXP_ERR_UNSUPPORTED otherwise).  The first call allocates the reverse work
 * space (about 2 (m_max + 1) + 16 state vectors). */
int pcexp_step_backward(pcexp_ctx* ctx, const double* U, double dt, int m,
                        const double* ubar_next, double* ubar, double* theta_bar, int on_device);

/* Adjoint of pcexp_project_state: theta_bar = (d u_0 / d theta)^T ubar0 for the projected
 * state u_0 of kind (PCEXP_PROJ_*) and params, with theta = (Mach, alpha in degrees) and,
 * for PCEXP_PROJ_VORTEX, the vortex strength eps as a third entry (theta_bar holds 2 or 3
 * doubles, host).  ubar0 has K entries in the context's basis (host or device).  The
 * derivative of the pointwise state is exact (forward-mode dual numbers through the same
 * state formulas) and is projected with the volume rule; host computation.  FP64 contexts.
 * Errors: INVALID_ARG, UNSUPPORTED (FP32-mixed), CUDA. */
int pcexp_project_state_adjoint(pcexp_ctx* ctx, int kind, const double* params, int n_params,
                                const double* ubar0, double* theta_bar, int on_device);

/* One PCEXP (Eq. s9, s10), EXP1 (Eq. s9) or ETD2 (Eq. s7) step on the master state
 * with Krylov dimension m (<= m_max).  dt_mode PCEXP_DT_*: dt_or_cfl is dt for
 * PCEXP_DT_GIVEN, else the CFL number.  info may be NULL; when given, the
 * call synchronises the stream to fill it.
 * ETD2 keeps u_n, R(u_n) and dt of its last step in the context (the first ETD2 step
 * allocates 3 state vectors for them) and forms N_n - N_{n-1} = R_n - R_{n-1} -
 * J_n (u_n - u_{n-1}) with one J v; its second Krylov stage takes phi_2.  Setting or
 * projecting the state, another scheme or a steady march clears the history, and the next
 * ETD2 step is then ETD1 (krylov_dim[1] = 0).  ETD2 with PCEXP_DT_LOCAL_CFL is INVALID_ARG. */
int pcexp_step(pcexp_ctx* ctx, int scheme, int dt_mode, double dt_or_cfl, int m,
               pcexp_step_info* info);

/* Steady march with local pseudo-steps and the CFL ramp of Eq. cfl until
 * ||R(rho_n)|| <= 10^-decades ||R(rho_1)|| or max_iter iterations. */
int pcexp_march_steady(pcexp_ctx* ctx, int scheme, double cfl_max, double decades,
                       int max_iter, int m, pcexp_steady_info* info);

/* Output functionals of a state U (not part of the paper's scheme; they seed
 * adjoint runs):
 *  - PCEXP_FUNC_WALL_FX / _FY / _FZ (FZ on tetrahedra only): the pressure force on
 *    the slip walls, J = sum over wall faces and their Gauss points of
 *    |f| w_q p(U) (n . a), a the unit axis, n the outward normal of the fluid element;
 *  - PCEXP_FUNC_VORTEX_L2: the L2 error against the translated isentropic vortex,
 *    J = (sum_e sum_q w_q |U_h(x_q) - U_exact(x_q)|^2)^(1/2) over all conservative
 *    variables at the volume points; params = {eps, x_c, y_c, period (<= 0: none), t}
 *    (the vortex of PCEXP_PROJ_VORTEX advected by the free stream for time t).
 * grad (nullable) receives dJ/dU in the basis of U; it is computed on the device and
 * for the vortex error divided by J (J > 0 assumed).  The wall-force gradient on an
 * element with three or more wall faces sums its contributions in arrival order.
 * pcexp_functional covers the kinds without parameters.  FP64 contexts only;
 * INVALID_ARG for an unknown kind or missing parameters, UNSUPPORTED for FP32. */
#define PCEXP_FUNC_WALL_FX 0
#define PCEXP_FUNC_WALL_FY 1
#define PCEXP_FUNC_VORTEX_L2 2
#define PCEXP_FUNC_WALL_FZ 3
int pcexp_functional(pcexp_ctx* ctx, int kind, const double* U, double* value, double* grad, int on_device);
int pcexp_functional_params(pcexp_ctx* ctx, int kind, const double* params, int n_params, const double* U,
                            double* value, double* grad, int on_device);
/* Partial derivatives of an output functional with respect to its parameters at a fixed
 * state U: dJ[0..2] = dJ/d(Mach, alpha in degrees, eps).  The wall forces depend on U alone
 * (all zero); the vortex error depends on the exact translated vortex, whose mean velocity
 * is the free stream's (Mach, alpha) and whose strength is eps:
 * dJ/dtheta = -(1/J) sum w_q (U_h - U_ex) . dU_ex/dtheta, on the device (dual numbers through
 * the exact state).  Same parameters as pcexp_functional_params.  FP64 contexts. */
int pcexp_functional_param_grad(pcexp_ctx* ctx, int kind, const double* params, int n_params, const double* U,
                                double* dJ, int on_device);

/* Replaces the free stream (Mach number, angle, density, pressure, gamma) used
 * by the far-field boundary condition; the mesh and state are kept.  omega must equal
 * the context's (INVALID_ARG otherwise): the frame's arrays are built at creation. */
int pcexp_set_physics(pcexp_ctx* ctx, const pcexp_physics* phys);

/* Diagnostics of the master state (Sec. 5):
 *  - kind 0: density residual norm of Eq. cfl, (1/|Omega|) ||R(rho)||, |Omega| = sum_e |E|;
 *  - kind 1: entropy error of Eq. entropy_error (Sec. 5.1),
 *    sqrt((1/|Omega|) int (s/s0)^2 dx - 1) with s = p / rho^gamma and s0 = p_inf / rho_inf^gamma,
 *    integrated by the volume rule in FP64 on the FP64 master state (either precision form);
 *    a negative radicand (rounding of a free stream) gives 0.
 * Synchronises the stream.  Errors: INVALID_ARG (kind), NONFINITE, CUDA, OOM (the first
 * kind-1 call allocates the FP64 volume tables, nq (nb + 1) + n_elem doubles). */
int pcexp_output(pcexp_ctx* ctx, int kind, double* value);

/* ---- kernel-class timing (diagnostic) ----
 * With profiling enabled every kernel launch of the context is bracketed by
 * CUDA events on the context's stream.  pcexp_profile_read synchronises the
 * stream and returns, for one kernel class, the number of launches and their
 * summed device time (ms) since profiling was enabled. */
#define PCEXP_KC_RESIDUAL_FACE 0 /* face Riemann-flux kernel of R(u) */
#define PCEXP_KC_RESIDUAL_ELEM 1 /* element volume + lift kernel of R(u) */
#define PCEXP_KC_JVP_FACE 2      /* face kernel of J v (point-Jacobian or tangent form) */
#define PCEXP_KC_JVP_ELEM 3      /* element kernel of J v */
#define PCEXP_KC_CGS_NORM 4      /* ||b|| of the Krylov start vector */
#define PCEXP_KC_CGS_PROJ 5      /* h = V^T w, ||w|| */
#define PCEXP_KC_CGS_UPD_PROJ 6  /* w -= V h; h2 = V^T w */
#define PCEXP_KC_CGS_UPD_NORM 7  /* v_{j+1} = w - V h2; ||v_{j+1}|| (selective form: only where
                                    the first pass cancelled; the other launches leave at once) */
#define PCEXP_KC_PHI 8           /* phi of the Hessenberg matrix */
#define PCEXP_KC_AXPY 9          /* u + sum_i c_i v_i */
#define PCEXP_KC_DT 10           /* element time steps */
#define PCEXP_KC_OTHER 11        /* small bookkeeping kernels */
#define PCEXP_KC_LINEARIZE 12    /* point Jacobians at u_n (once per step) */
#define PCEXP_KC_CGS_UPD1 13     /* selective form: w_1 = w - V h; ||w_1|| and the decision */
#define PCEXP_KC_CGS_PROJ2 14    /* selective form: h2 = V^T w_1 where the first pass cancelled */
#define PCEXP_KC_COUNT 15
int pcexp_profile_enable(pcexp_ctx* ctx, int enable);
int pcexp_profile_read(pcexp_ctx* ctx, int kernel_class, int64_t* launches, double* ms);

/* R(U) exactly as pcexp_residual computes it, for callers that cannot allocate device
 * memory when they need R(U): hosts whose own pool or caching allocator owns all device
 * memory, hosts with a fixed memory budget reserved at start-up, and real-time loops that
 * may not call cudaMalloc/cudaFree (which can synchronise the device) after set-up.  The
 * paper has no counterpart; this is an interface variant.
 * U and R are device pointers to K doubles in the library's INTERNAL basis (whatever
 * basis_io the context uses); the context must be FP64.  The call only enqueues the two DG
 * kernels on the context's stream and returns; it calls no cudaMalloc/cudaFree or other
 * allocating routine.  Its face-flux scratch is a fixed 8 MiB device array inside the
 * library (held by every GPU that loads the library until the process exits): meshes with
 * faces x face quadrature points x (dim + 2) > 2^20 doubles get PCEXP_ERR_INVALID_ARG
 * (face points: p + 1 on edges, (p + 1)^2 on triangular faces, 7 at p = 2).  The first call on a
 * device makes that device current and looks up the array's device address; make that
 * first call before any stream capture.  All calls share the array, which keeps the last
 * call's face fluxes: calls whose kernels overlap on the GPU race; calls on one stream are
 * ordered.  Errors (with pcexp_last_error text): INVALID_ARG, UNSUPPORTED (FP32-mixed
 * context), CUDA. */
int pcexp_residual_noalloc(pcexp_ctx* ctx, const double* U, double* R);

/* Measurement aid (the paper has no counterpart): the FP64 fused multiply-add rate of
 * the current device in TFLOP/s, from independent DFMA chains on every SM timed with CUDA
 * events (best of three launches after a warm-up; a few milliseconds).  It is the roof of
 * the FP64 form's compute-bound kernels.  Allocates and frees one small device buffer and
 * a private stream.  Errors: INVALID_ARG, CUDA. */
int pcexp_fp64_fma_rate(double* tflops);

/* The same for FP32 fused multiply-adds (the roof of the FP32-mixed form's arithmetic-bound
 * kernels, e.g. the element J v on tetrahedra).  Errors: INVALID_ARG, CUDA. */
int pcexp_fp32_fma_rate(double* tflops);

/* Waits for all work queued on the context's stream. */
int pcexp_synchronize(pcexp_ctx* ctx);

/* ---- partitioned runs (an element decomposition; the paper runs on one processor)
 *
 * The operator of Sec. 4.3 (Eq. euler3) couples an element only to the elements across its
 * faces.  A partition therefore computes its own elements' rows of R(u) and J v (Sec. 4.4)
 * from its own elements and a one-element halo (the other partitions' elements that share a
 * face with one of its own), and the rest of the Krylov step (Sec. 2.2, Eq. s9/s10: the
 * Gram-Schmidt inner products and norms of the Arnoldi process, the axpys) is arithmetic on
 * its own rows plus sums over partitions.  A group holds one context per partition, each on
 * its own device (or all on one) and stream.  In a step, each operator pass first gathers
 * the halo rows of its input vector from the owning partitions' device buffers (peer reads),
 * each Gram-Schmidt pass sums its (j + 2) partial sums over the partitions in partition
 * order (every partition obtains the same Hessenberg matrix, bit for bit), and the global
 * dt of PCEXP_DT_GLOBAL_CFL is the minimum over partitions.  The results equal those of one
 * context on the whole mesh up to the summation order of the inner products.  A group call
 * drives each partition from a host thread of its own; the partitions meet at host
 * rendezvous points, the ordering between their streams is by CUDA events, and no kernel
 * waits on another.  A group is not thread-safe; one group call at a time.
 *
 * Global state-shaped arrays are host arrays of the whole mesh (layout and basis as for one
 * context).  After a failed group call the state is undefined until the next set/project. */
typedef struct pcexp_group pcexp_group;

/* part[e] in [0, n_parts) for every element (n_parts <= 16, n_elem >= n_parts): recursive
 * coordinate bisection of the element centroids (each set of elements going to n parts is
 * split at the floor(n/2)/n quantile along its axis of largest extent; ties by element
 * index).  Host only.  Errors: INVALID_ARG. */
int pcexp_partition(const pcexp_mesh* mesh, int n_parts, int32_t* part);

/* The elements partition k computes with: *n_owned of its own (ascending element index),
 * then its halo (ascending), *n_total in all; elems (NULL: sizes only) receives them and must
 * hold n_elem entries.  Host only.  Errors: INVALID_ARG, MESH. */
int pcexp_partition_halo(const pcexp_mesh* mesh, const int32_t* part, int n_parts, int k,
                         int64_t* n_owned, int64_t* n_total, int64_t* elems);

/* Creates a group of n_parts contexts (1..16), partition k on device devices[k] (NULL: all
 * on the current device), each with the submesh of its own and halo elements: a face keeps
 * the quadrature points of the whole mesh's L element; halo faces with no partner in the
 * submesh get the symmetry-plane ghost state, whose halo rows are discarded.  Devices of
 * different partitions must allow peer access (else UNSUPPORTED).  The state starts at the
 * free stream.  Errors: INVALID_ARG (bad option, index out of range, empty partition),
 * MESH, CUDA, OOM, UNSUPPORTED. */
int pcexp_group_create(pcexp_group** out, const pcexp_mesh* mesh, const int32_t* part, int n_parts,
                       const int32_t* devices, int p, const pcexp_physics* phys,
                       const pcexp_options* opt);
int pcexp_group_destroy(pcexp_group* group);

/* Own and halo element counts of partition k. */
int pcexp_group_sizes(const pcexp_group* group, int k, int64_t* n_owned, int64_t* n_halo);

/* State of the whole mesh (host, K doubles), scattered to / gathered from the partitions. */
int pcexp_group_set_state(pcexp_group* group, const double* U);
int pcexp_group_get_state(pcexp_group* group, double* U);
int pcexp_group_project_state(pcexp_group* group, int kind, const double* params, int n_params);

/* R(U) and J(U) v of the whole mesh (host arrays).  Each partition receives only its own rows
 * of U and v; the halo rows come from the exchange of the operator pass, as in a step. */
int pcexp_group_residual(pcexp_group* group, const double* U, double* R);
int pcexp_group_jvp(pcexp_group* group, const double* U, const double* v, double* Jv);

/* The adjoint operator passes of the reverse step on the whole mesh (host arrays): J(U)^T w as
 * pcexp_vjp, and (d(J(U) v)/dU)^T w as pcexp_jvp_state_adjoint (FP64 groups; UNSUPPORTED in
 * FP32-mixed groups and rotating frames).  Each partition receives only its own rows; the halo
 * rows of U, v and w come from the exchange (an own element's transposed face terms need w on
 * the neighbouring halo element), and each partition returns its own rows. */
int pcexp_group_vjp(pcexp_group* group, const double* U, const double* w, double* JTw);
int pcexp_group_jvp_state_adjoint(pcexp_group* group, const double* U, const double* v,
                                  const double* w, double* out);

/* pcexp_step_backward on the whole mesh (host arrays; FP64, fixed frame): the forward step is
 * recomputed partitioned from U, and its reverse runs partitioned too.  Every reduction of the
 * reverse Gram-Schmidt is summed over the partitions (partition order) before its finishing
 * step, the adjoint operator passes exchange their inputs' halo rows, and theta_bar (NULL:
 * not returned) is the sum of the partitions' sums over their own elements.  Errors: those of
 * pcexp_step_backward, TIMEOUT. */
int pcexp_group_step_backward(pcexp_group* group, const double* U, double dt, int m,
                              const double* ubar_next, double* ubar, double* theta_bar);

/* Arnoldi process of pcexp_arnoldi (J at U, start vector b; host arrays) with the partitioned
 * Gram-Schmidt sums: H [(m+1) x m] row-major, *k, *beta as for pcexp_arnoldi.  The call
 * checks that every partition holds the same H (else CUDA). */
int pcexp_group_arnoldi(pcexp_group* group, const double* U, const double* b, int m, double* H,
                        int* k, double* beta);

/* One step of pcexp_step on the group's state (schemes, dt modes and their rules as there;
 * the global dt of GLOBAL_CFL is the minimum over all partitions' elements, LOCAL_CFL scales
 * each partition's own rows by its own elements' steps).  info as for pcexp_step, res_norm
 * over the whole mesh.  Steps run eagerly (no CUDA graph).  Errors: those of pcexp_step,
 * TIMEOUT (a partition missed a rendezvous for 120 s: it failed or stalled). */
int pcexp_group_step(pcexp_group* group, int scheme, int dt_mode, double dt_or_cfl, int m,
                     pcexp_step_info* info);

/* pcexp_march_steady on the group's state (Sec. 5.2, Eq. cfl): each iteration's density
 * residual norm is summed over the partitions on the host (partition order) before the stop
 * test and the CFL ramp, so every partition takes the same decisions; the Krylov-error cap
 * (krylov_tol of the options) uses the estimate every partition shares.  info as for
 * pcexp_march_steady.  Errors: those of pcexp_march_steady, TIMEOUT. */
int pcexp_group_march_steady(pcexp_group* group, int scheme, double cfl_max, double decades,
                             int max_iter, int m, pcexp_steady_info* info);

/* Static description of a status code. */
const char* pcexp_status_string(int status);

/* Human-readable detail of the last error raised on the calling thread
 * (empty string if none).  Valid until the next call on that thread. */
const char* pcexp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PCEXP_H */
