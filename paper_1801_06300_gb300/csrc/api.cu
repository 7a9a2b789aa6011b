// The C interface of include/pcexp.h: context set-up, basis conversion at the
// boundary, and the launch sequence of one PCEXP / EXP1 step (Eq. s9, s10).
//
// A step never waits for the host: the time step, beta, the Hessenberg matrix,
// the breakdown flag and the Krylov dimension stay in device memory, and the
// kernels after a happy breakdown exit at once.  Only pcexp_step with a
// non-NULL info, the steady march (one 8-byte residual read per iteration)
// and host-pointer transfers synchronise.
#include <algorithm>
#include <array>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "host_setup.h"
#include "kernels.h"
#include "partition.h"

using namespace pcexp;

struct pcexp_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  bool fp32 = false;
  int dim = 2, p = 0, nb = 0, nq = 0, nfq = 0, nv = 4;
  int64_t E = 0, F = 0, K = 0, Kp = 0;
  int m_max = 0;
  double eta = 0;
  double ktol = 0;  // Krylov tolerance of the adaptive dimension (<= 0: fixed dimension)
  bool selective = false;  // Arnoldi: second Gram-Schmidt pass only after a cancelling first pass
  int basis_io = PCEXP_BASIS_PAPER;
  double volume = 0;
  pcexp_physics phys{};
  Setup host;
  // device data
  double* Q = nullptr;
  int32_t *ef = nullptr, *fel = nullptr, *floc = nullptr;
  void *geo = nullptr, *fgeo = nullptr, *tabs = nullptr;
  double* U64[2] = {nullptr, nullptr};
  void* S32[2] = {nullptr, nullptr};  // FP32 shadows (mixed form only)
  void *V = nullptr, *w = nullptr, *tmp = nullptr, *delta = nullptr, *G = nullptr, *dte = nullptr;
  double *io64a = nullptr, *io64b = nullptr;
  void *Avol = nullptr, *Bface = nullptr;  // point Jacobians at the linearisation state
  const void* lin_state = nullptr;         // state the last linearize() recorded
  bool jv_tangent = false;                 // volume part of J v by flux tangents (FP32-mixed)
  bool face_tangent = false;               // face part of J v by Riemann-flux tangents (no face blocks)
  void* GT = nullptr;                      // adjoint face scratch [F][nfq][2 nv]
  double* xq = nullptr;                    // physical volume points [E][nq][dim] (first vortex functional)
  double* diag = nullptr;                  // FP64 [Bv (nq nb) | Wv (nq) | sqrt|det A| (E)] (first entropy output)
  double* pgrad = nullptr;                 // 4 doubles: sums of the functional-parameter gradient
  // rotating frame: v_r at volume points, v_r . n at face points, v_r at centroids (precision of
  // the DG kernels); allocated when omega != 0
  void *vrq = nullptr, *vrn = nullptr, *vrc = nullptr;
  bool rot = false;
  // ETD2 history (first ETD2 step): u_{n-1}, R_{n-1}, and R_n of the step in progress
  void *h_u = nullptr, *h_R = nullptr, *h_Rc = nullptr;
  bool etd2_prev = false;  // the history holds the previous ETD2 step of the current state
  // reverse-step work space (FP64 contexts, allocated by the first backward call)
  double *b_un = nullptr, *b_us = nullptr, *b_dl = nullptr, *b_V1 = nullptr, *b_Vb = nullptr;
  double *b_w1 = nullptr, *b_w0 = nullptr, *b_wb2 = nullptr, *b_wb1 = nullptr, *b_wb0 = nullptr;
  double *b_t1 = nullptr, *b_t2 = nullptr, *b_ubn = nullptr, *b_ubs = nullptr, *b_db = nullptr, *b_bb = nullptr,
         *b_rb = nullptr, *b_gin = nullptr;
  double* b_small = nullptr;  // 2 MMAX^2 doubles: H and Hbar of pcexp_phi_adjoint
  double* b_theta = nullptr;  // adjoint of (Mach, alpha in degrees) of the reverse step (2 doubles)
  KState* b_ks1 = nullptr;
  AdjState* b_as = nullptr;
  KState* ks = nullptr;
  StepState* ss = nullptr;
  double* partials = nullptr;
  int cur = 0;
  std::vector<void*> allocs;
  // CUDA graphs of whole steps, keyed by (scheme, dt mode, m, state slot)
  struct StepGraph {
    int scheme, dt_mode, m, cur, cur_after;
    cudaGraphExec_t exec;
  };
  std::vector<StepGraph> graphs;
  std::vector<int> seen_keys;
  double* param = nullptr;  // dt or CFL of the step being replayed (device)
  cudaStream_t cap_st = nullptr;  // private stream for capture (the caller's may be the legacy stream)
  // kernel-class timing
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_rec;  // (class, start, end) triples of indices into ev_pool
  double prof_ms[PCEXP_KC_COUNT] = {};
  int64_t prof_n[PCEXP_KC_COUNT] = {};
  // partition of a group (pcexp_group_create): the first n_local elements are its own, the
  // n_ghost after them its halo, whose rows are gathered from the owning partitions
  pcexp_group* grp = nullptr;
  int part = -1;
  int64_t n_local = 0, n_ghost = 0;
  int32_t *g_src_part = nullptr, *g_src_elem = nullptr;  // [n_ghost] owning partition, its local index
};

// A partitioned run: one context per partition, each on its own device and stream, driven by
// one host thread per partition during a group call.  The partitions meet in rounds: each
// publishes a device pointer and records an event, all meet at a host barrier, each makes its
// stream wait for the others' events and enqueues the work that reads their data, records a
// second event, meets them again and waits for theirs.  So the data a round reads is complete
// before it is read and is not overwritten before every partition has read it, with no device-side
// wait between kernels.
struct pcexp_group {
  int n = 0;
  std::vector<pcexp_ctx*> ctx;
  std::vector<int> dev;
  std::vector<cudaStream_t> st;
  std::vector<std::vector<int64_t>> elems;  // per partition: global element of each local element
  std::vector<double> own_volume;           // per partition: measure of its own elements
  int64_t E = 0;
  int nb = 0, nv = 0;
  double volume = 0;
  int fp32 = 0;
  // rendezvous
  std::mutex mu;
  std::condition_variable cv;
  int arrived = 0;
  uint64_t gen = 0;
  bool abort = false;
  std::vector<const void*> pub;
  std::vector<double> hostval;  // per partition: a host scalar being summed (steady march)
  std::vector<cudaEvent_t> ev_ready, ev_done;
  std::vector<std::string> errs;
};

namespace {

thread_local std::string g_last_error;

#define PCEXP_CK(...)                                                       \
  do {                                                                      \
    cudaError_t _e = (__VA_ARGS__);                                         \
    if (_e != cudaSuccess) {                                                \
      g_last_error = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e); \
      return _e == cudaErrorMemoryAllocation ? PCEXP_ERR_OOM : PCEXP_ERR_CUDA; \
    }                                                                       \
  } while (0)

template <class T>
int dalloc(pcexp_ctx* c, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 16);
  if (e != cudaSuccess) {
    g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return PCEXP_ERR_OOM;
  }
  c->allocs.push_back(q);
  e = cudaMemsetAsync(q, 0, n * sizeof(T) + 16, c->st);
  if (e != cudaSuccess) return PCEXP_ERR_CUDA;
  *p = reinterpret_cast<T*>(q);
  return PCEXP_OK;
}

#define PCEXP_TRY(...)      \
  do {                      \
    int _r = (__VA_ARGS__); \
    if (_r != PCEXP_OK) return _r; \
  } while (0)

template <class T>
int upload(pcexp_ctx* c, void** dst, const std::vector<double>& src) {
  T* d = nullptr;
  PCEXP_TRY(dalloc(c, &d, src.size() ? src.size() : 1));
  std::vector<T> tmp(src.begin(), src.end());
  if (!tmp.empty()) PCEXP_CK(cudaMemcpyAsync(d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  *dst = d;
  return PCEXP_OK;
}

template <class T>
DGData<T> dgdata(const pcexp_ctx* c) {
  DGData<T> d;
  const T* tabs = reinterpret_cast<const T*>(c->tabs);
  const int nb = c->nb, nq = c->nq, nfq = c->nfq;
  d.geo = reinterpret_cast<const T*>(c->geo);
  d.ef = c->ef;
  d.fel = c->fel;
  d.floc = c->floc;
  d.fgeo = reinterpret_cast<const T*>(c->fgeo);
  const int D = c->dim, NF = D + 1, NPERM = D == 2 ? 2 : 6;
  d.Bv = tabs;
  d.Dv = d.Bv + nq * nb;
  d.Bf = d.Dv + D * nq * nb;
  d.Wf = d.Bf + NF * NPERM * nfq * nb;
  d.Bc = d.Wf + nfq;
  d.Wv = d.Bc + nb;
  {
    // padded trace tables: after Wv, at the next 16-byte boundary (as laid out in create_impl)
    const size_t vec = 16 / sizeof(T), off = (size_t)((d.Wv + nq) - tabs);
    d.BfP = tabs + (off + vec - 1) / vec * vec;
  }
  d.E = c->E;
  d.E_loc = c->grp ? c->n_local : c->E;
  d.F = c->F;
  const double a = c->phys.alpha_deg * M_PI / 180.0;
  const double cinf = std::sqrt(c->phys.gamma * c->phys.p_inf / c->phys.rho_inf);
  d.fs.gamma = (T)c->phys.gamma;
  d.fs.rho = (T)c->phys.rho_inf;
  d.fs.p = (T)c->phys.p_inf;
  d.fs.vel[0] = (T)(c->phys.mach * cinf * std::cos(a));
  d.fs.vel[1] = (T)(c->phys.mach * cinf * std::sin(a));
  d.fs.vel[2] = T(0);
  d.p = c->p;
  d.dim = D;
  d.rot = c->rot ? 1 : 0;
  d.vrq = reinterpret_cast<const T*>(c->vrq);
  d.vrn = reinterpret_cast<const T*>(c->vrn);
  d.vrc = reinterpret_cast<const T*>(c->vrc);
  for (int k = 0; k < 3; ++k) d.om[k] = (T)c->phys.omega[k];
  return d;
}

// ---- kernel-class timing: events bracket each launch when profiling is on
int prof_flush(pcexp_ctx* c) {
  if (c->ev_rec.empty()) {
    c->ev_used = 0;
    return PCEXP_OK;
  }
  PCEXP_CK(cudaStreamSynchronize(c->st));
  for (size_t i = 0; i + 2 < c->ev_rec.size(); i += 3) {
    float ms = 0;
    PCEXP_CK(cudaEventElapsedTime(&ms, c->ev_pool[c->ev_rec[i + 1]], c->ev_pool[c->ev_rec[i + 2]]));
    c->prof_ms[c->ev_rec[i]] += ms;
    c->prof_n[c->ev_rec[i]] += 1;
  }
  c->ev_rec.clear();
  c->ev_used = 0;
  return PCEXP_OK;
}

cudaEvent_t* prof_events(pcexp_ctx* c, int n) {
  if (!c->prof) return nullptr;
  if (c->ev_used + n > c->ev_pool.size()) {
    if (c->ev_pool.size() >= 16384) {
      if (prof_flush(c) != PCEXP_OK) return nullptr;
    } else {
      size_t add = c->ev_pool.size() ? c->ev_pool.size() : 1024;
      for (size_t i = 0; i < add; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
      }
    }
  }
  cudaEvent_t* e = &c->ev_pool[c->ev_used];
  c->ev_used += n;
  return e;
}

void prof_note(pcexp_ctx* c, int cls, cudaEvent_t* e0, int offset) {
  if (!e0) return;
  const int i0 = (int)(e0 - c->ev_pool.data()) + offset;
  c->ev_rec.push_back(cls);
  c->ev_rec.push_back(i0);
  c->ev_rec.push_back(i0 + 1);
}

// one timed launch of kernel class cls
#define PCEXP_LAUNCH(c, cls, ...)                                  \
  do {                                                             \
    cudaEvent_t* _ev = prof_events(c, 2);                          \
    if (_ev) cudaEventRecord(_ev[0], (c)->st);                     \
    cudaError_t _e = (__VA_ARGS__);                                \
    if (_ev) {                                                     \
      cudaEventRecord(_ev[1], (c)->st);                            \
      prof_note(c, cls, _ev, 0);                                   \
    }                                                              \
    if (_e != cudaSuccess) {                                       \
      g_last_error = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e); \
      return PCEXP_ERR_CUDA;                                       \
    }                                                              \
  } while (0)

// ---- partitioned runs (pcexp_group): rendezvous, halo exchange, split reductions
constexpr int GROUP_WAIT_S = 120;  // a partition not at a rendezvous by then has failed

int group_barrier(pcexp_group* g) {
  std::unique_lock<std::mutex> lk(g->mu);
  if (g->abort) {
    g_last_error = "another partition of the group failed";
    return PCEXP_ERR_TIMEOUT;
  }
  const uint64_t my = g->gen;
  if (++g->arrived == g->n) {
    g->arrived = 0;
    ++g->gen;
    g->cv.notify_all();
    return PCEXP_OK;
  }
  const auto until = std::chrono::steady_clock::now() + std::chrono::seconds(GROUP_WAIT_S);
  while (g->gen == my && !g->abort)
    if (g->cv.wait_until(lk, until) == std::cv_status::timeout && g->gen == my) {
      g->abort = true;
      g->cv.notify_all();
      g_last_error = "partition rendezvous timed out";
      return PCEXP_ERR_TIMEOUT;
    }
  if (g->gen == my) {
    g_last_error = "another partition of the group failed";
    return PCEXP_ERR_TIMEOUT;
  }
  return PCEXP_OK;
}

// One round: publish `mine`, then consume(pointers of all partitions) on every partition's
// stream once every partition's work so far is complete; later work on any stream starts after
// every partition's consume.
template <class F>
int group_round(pcexp_ctx* c, const void* mine, F&& consume) {
  pcexp_group* g = c->grp;
  const int me = c->part;
  g->pub[me] = mine;
  PCEXP_CK(cudaEventRecord(g->ev_ready[me], c->st));
  PCEXP_TRY(group_barrier(g));
  PartPtrs pp{};
  for (int q = 0; q < g->n; ++q) {
    pp.p[q] = g->pub[q];
    if (q != me) PCEXP_CK(cudaStreamWaitEvent(c->st, g->ev_ready[q], 0));
  }
  PCEXP_TRY(consume(pp));
  PCEXP_CK(cudaEventRecord(g->ev_done[me], c->st));
  PCEXP_TRY(group_barrier(g));
  for (int q = 0; q < g->n; ++q)
    if (q != me) PCEXP_CK(cudaStreamWaitEvent(c->st, g->ev_done[q], 0));
  return PCEXP_OK;
}

// Halo rows of x (a state-shaped vector of the partition) <- the owners' rows of the same vector.
template <class T>
int group_exchange(pcexp_ctx* c, const T* x) {
  if (!c->grp) return PCEXP_OK;
  T* xm = const_cast<T*>(x);  // the context's own buffer; only its halo rows are written
  return group_round(c, x, [&](const PartPtrs& pp) -> int {
    PCEXP_CK(launch_gather_ghosts<T>(xm, pp, c->g_src_part, c->g_src_elem, c->n_local, c->n_ghost,
                                     c->nv * c->nb, c->st));
    return PCEXP_OK;
  });
}

// Halo rows of x <- 0: operator outputs and Krylov vectors carry zero halo rows, so that the
// inner products over all local rows are sums over the own elements.
template <class T>
int group_zero_halo(pcexp_ctx* c, T* x) {
  if (!c->grp) return PCEXP_OK;
  const int64_t nvb = (int64_t)c->nv * c->nb;
  PCEXP_CK(launch_zero_range<T>(x, c->n_local * nvb, (c->n_local + c->n_ghost) * nvb, c->st));
  return PCEXP_OK;
}

template <class T> double* dev_field(T* base, size_t off) {
  return reinterpret_cast<double*>(reinterpret_cast<char*>(base) + off);
}

// A Gram-Schmidt pass of a partitioned run left this partition's sums in ks->gsum: sum them
// over the partitions (partition order, the same on every partition) and finalise the column.
int group_cgs(pcexp_ctx* c, int mode, int j) {
  if (!c->grp) return PCEXP_OK;
  return group_round(c, dev_field(c->ks, offsetof(KState, gsum)), [&](const PartPtrs& pp) -> int {
    PCEXP_CK(launch_group_reduce(pp, c->grp->n, MMAX + 2, dev_field(c->ks, offsetof(KState, gtot)), 0, c->st));
    PCEXP_CK(launch_cgs_group_finalize(mode, j, c->ks, c->eta, c->st));
    return PCEXP_OK;
  });
}

// Sum over the partitions of a host scalar, in partition order (the same on every partition).
int group_host_sum(pcexp_ctx* c, double x, double* sum) {
  pcexp_group* g = c->grp;
  g->hostval[(size_t)c->part] = x;
  PCEXP_TRY(group_barrier(g));
  double s = 0;
  for (int q = 0; q < g->n; ++q) s += g->hostval[(size_t)q];
  PCEXP_TRY(group_barrier(g));  // no partition writes its next value before all have read
  *sum = s;
  return PCEXP_OK;
}

// ss->dt <- the minimum over the partitions of their ss->dtmin_scratch (Eq. x3d over all elements)
int group_min_dt(pcexp_ctx* c) {
  return group_round(c, dev_field(c->ss, offsetof(StepState, dtmin_scratch)), [&](const PartPtrs& pp) -> int {
    PCEXP_CK(launch_group_reduce(pp, c->grp->n, 1, dev_field(c->ss, offsetof(StepState, dt)), 1, c->st));
    return PCEXP_OK;
  });
}

// the two kernels of one DG operator application (face, element)
template <class T>
int dg_apply(pcexp_ctx* c, const DGData<T>& d, const T* u, const T* du, T* out, const T* escale, const int* skip,
             const double* oscale = nullptr) {
  PCEXP_TRY(group_exchange<T>(c, u));
  if (du) PCEXP_TRY(group_exchange<T>(c, du));
  cudaEvent_t* ev = prof_events(c, 3);
  cudaError_t e = launch_dg_operator<T>(d, u, du, out, reinterpret_cast<T*>(c->G), escale, skip, c->st, ev, oscale);
  if (ev) {
    prof_note(c, du ? PCEXP_KC_JVP_FACE : PCEXP_KC_RESIDUAL_FACE, ev, 0);
    prof_note(c, du ? PCEXP_KC_JVP_ELEM : PCEXP_KC_RESIDUAL_ELEM, ev, 1);
  }
  if (e != cudaSuccess) {
    g_last_error = std::string("DG operator launch: ") + cudaGetErrorString(e);
    return PCEXP_ERR_CUDA;
  }
  return group_zero_halo<T>(c, out);
}

template <class T> LinData<T> lindata(pcexp_ctx* c) {
  return LinData<T>{reinterpret_cast<T*>(c->Avol), reinterpret_cast<T*>(c->Bface)};
}

// Linearise the operator at u for the J v products that follow.  FP64 contexts build the
// face and volume point Jacobians once; FP32-mixed contexts build the face blocks only and
// recompute the volume flux tangents at u in every J v (reading u and dv instead of
// D nv^2 values per volume point).  blocks = true builds both (the transpose needs them).
template <class T>
int linearize(pcexp_ctx* c, const DGData<T>& d, const T* u, bool blocks = false) {
  c->lin_state = u;
  if (c->face_tangent && !blocks) return PCEXP_OK;  // every J v recomputes its tangents at u
  const bool faces_only = c->jv_tangent && !blocks;
  PCEXP_LAUNCH(c, PCEXP_KC_LINEARIZE, launch_linearize<T>(d, u, lindata<T>(c), c->st, faces_only));
  return PCEXP_OK;
}

// J(u_lin) dv (two kernels: face, element)
template <class T>
int jac_apply(pcexp_ctx* c, const DGData<T>& d, const T* dv, T* out, const T* escale, const int* skip,
              const double* oscale) {
  PCEXP_TRY(group_exchange<T>(c, dv));
  cudaEvent_t* ev = prof_events(c, 3);
  const T* u_elem = c->jv_tangent ? reinterpret_cast<const T*>(c->lin_state) : nullptr;
  cudaError_t e = launch_jac_apply<T>(d, lindata<T>(c), dv, out, reinterpret_cast<T*>(c->G), escale, skip, oscale,
                                      c->st, ev, u_elem, c->face_tangent);
  if (ev) {
    prof_note(c, PCEXP_KC_JVP_FACE, ev, 0);
    prof_note(c, PCEXP_KC_JVP_ELEM, ev, 1);
  }
  if (e != cudaSuccess) {
    g_last_error = std::string("Jacobian apply launch: ") + cudaGetErrorString(e);
    return PCEXP_ERR_CUDA;
  }
  if (c->grp) {
    // a Krylov vector gets its zero halo rows back (the Gram-Schmidt sums run over all rows)
    const T* V = reinterpret_cast<const T*>(c->V);
    if (dv >= V && dv < V + (int64_t)(c->m_max + 1) * c->Kp) PCEXP_TRY(group_zero_halo<T>(c, const_cast<T*>(dv)));
  }
  return group_zero_halo<T>(c, out);
}

template <class T> T* Vcol(pcexp_ctx* c, int j) { return reinterpret_cast<T*>(c->V) + (int64_t)j * c->Kp; }
template <class T> T* shadow(pcexp_ctx* c, int i) {
  return c->fp32 ? reinterpret_cast<T*>(c->S32[i]) : reinterpret_cast<T*>(c->U64[i]);
}

// Input state-shaped double array (host or device) -> internal basis in T (dst, device).
template <class T>
int import_vec(pcexp_ctx* c, const double* src, int on_device, T* dst) {
  const double* s = src;
  if (!on_device) {
    PCEXP_CK(cudaMemcpyAsync(c->io64a, src, c->K * sizeof(double), cudaMemcpyHostToDevice, c->st));
    s = c->io64a;
  }
  if (c->basis_io == PCEXP_BASIS_PAPER) PCEXP_CK(launch_paper_to_internal<T>(s, dst, c->Q, c->E, c->nb, c->nv, c->st));
  else PCEXP_CK(launch_cast<double, T>(s, dst, c->K, c->st));
  return PCEXP_OK;
}

template <class T>
int export_vec(pcexp_ctx* c, const T* src, double* dst, int on_device) {
  double* d = on_device ? dst : c->io64b;
  if (c->basis_io == PCEXP_BASIS_PAPER) PCEXP_CK(launch_internal_to_paper<T>(src, d, c->Q, c->E, c->nb, c->nv, c->st));
  else PCEXP_CK(launch_cast<T, double>(src, d, c->K, c->st));
  if (!on_device) {
    PCEXP_CK(cudaMemcpyAsync(dst, c->io64b, c->K * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PCEXP_CK(cudaStreamSynchronize(c->st));
  }
  return PCEXP_OK;
}

template <class T>
int refresh_shadow(pcexp_ctx* c, int i) {
  if (c->fp32) PCEXP_CK(launch_cast<double, float>(c->U64[i], reinterpret_cast<float*>(c->S32[i]), c->Kp, c->st));
  return PCEXP_OK;
}

// Columns between checkpoints of the adaptive Krylov dimension.
constexpr int KRYLOV_CHECK = 5;

// Arnoldi on J (times escale) started from V[0]; m columns at most.  J is the
// operator linearised by the last linearize() call.  With a Krylov tolerance and the
// step's dt on the device (dt_dev), every KRYLOV_CHECK-th column k < m is a checkpoint: the
// process ends at k when the error estimate of phi_1(dt H_k) e_1 is within the tolerance.
template <class T>
int arnoldi(pcexp_ctx* c, const T* escale, int m, const double* dt_dev = nullptr) {
  const DGData<T> d = dgdata<T>(c);
  T* w = reinterpret_cast<T*>(c->w);
  T* G = reinterpret_cast<T*>(c->G);
  T* V = reinterpret_cast<T*>(c->V);
  (void)G;
  PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_reset_kstate(c->ks, c->st));
  PCEXP_LAUNCH(c, PCEXP_KC_CGS_NORM, launch_cgs<T>(CGS_NORM, V, c->Kp, c->Kp, 0, V, nullptr, c->ks, c->partials, c->eta, c->st));
  PCEXP_TRY(group_cgs(c, CGS_NORM, 0));
  for (int j = 0; j < m; ++j) {
    // w = J v_j = s_j J z_j: the basis scale is applied to the output, so every
    // stored vector stays of the size of ||J|| (no growth like ||J||^j)
    PCEXP_TRY(jac_apply<T>(c, d, Vcol<T>(c, j), w, escale, &c->ks->done, &c->ks->s[j]));
    PCEXP_LAUNCH(c, PCEXP_KC_CGS_PROJ, launch_cgs<T>(CGS_PROJ, V, c->Kp, c->Kp, j, w, nullptr, c->ks, c->partials, c->eta, c->st));
    PCEXP_TRY(group_cgs(c, CGS_PROJ, j));
    if (c->selective) {
      // the first update alone, w_1 = w - V h straight into z_{j+1}, with ||w_1||; where it
      // cancelled, the second projection and update follow (in place on z_{j+1}), otherwise
      // those two passes leave at once
      T* z1 = Vcol<T>(c, j + 1);
      PCEXP_LAUNCH(c, PCEXP_KC_CGS_UPD1, launch_cgs<T>(CGS_UPD1, V, c->Kp, c->Kp, j, w, z1, c->ks, c->partials, c->eta, c->st));
      PCEXP_TRY(group_cgs(c, CGS_UPD1, j));
      PCEXP_LAUNCH(c, PCEXP_KC_CGS_PROJ2, launch_cgs<T>(CGS_PROJ2, V, c->Kp, c->Kp, j, z1, nullptr, c->ks, c->partials, c->eta, c->st));
      PCEXP_TRY(group_cgs(c, CGS_PROJ2, j));
      PCEXP_LAUNCH(c, PCEXP_KC_CGS_UPD_NORM, launch_cgs<T>(CGS_UPD_NORM, V, c->Kp, c->Kp, j, z1, z1, c->ks, c->partials, c->eta, c->st));
      PCEXP_TRY(group_cgs(c, CGS_UPD_NORM, j));
    } else {
      PCEXP_LAUNCH(c, PCEXP_KC_CGS_UPD_PROJ, launch_cgs<T>(CGS_UPD_PROJ, V, c->Kp, c->Kp, j, w, nullptr, c->ks, c->partials, c->eta, c->st));
      PCEXP_TRY(group_cgs(c, CGS_UPD_PROJ, j));
      PCEXP_LAUNCH(c, PCEXP_KC_CGS_UPD_NORM, launch_cgs<T>(CGS_UPD_NORM, V, c->Kp, c->Kp, j, w, Vcol<T>(c, j + 1), c->ks, c->partials, c->eta, c->st));
      PCEXP_TRY(group_cgs(c, CGS_UPD_NORM, j));
    }
    if (c->ktol > 0 && dt_dev && (j + 1) % KRYLOV_CHECK == 0 && j + 1 < m)
      PCEXP_LAUNCH(c, PCEXP_KC_PHI, launch_phi_check(c->ks, dt_dev, c->ktol, c->st));
  }
  return PCEXP_OK;
}

// Stages of Eq. s9 (and s10) once V[0] holds R_n (scaled by escale when given)
// and ss->dt holds dt.  u_n = U64[cur]; the new state ends in U64[cur] (PCEXP)
// or U64[1-cur] (EXP1; cur flips).
template <class T>
int krylov_stages(pcexp_ctx* c, int scheme, const T* escale, int m) {
  const DGData<T> d = dgdata<T>(c);
  const int a = c->cur, b = 1 - c->cur;
  T* S0 = shadow<T>(c, a);
  T* S1 = shadow<T>(c, b);
  T* V = reinterpret_cast<T*>(c->V);
  T* G = reinterpret_cast<T*>(c->G);
  T* w = reinterpret_cast<T*>(c->w);
  T* tmp = reinterpret_cast<T*>(c->tmp);
  T* delta = reinterpret_cast<T*>(c->delta);
  // J_n: point Jacobians at u_n, shared by all 2m+1 products of the step
  PCEXP_TRY(linearize<T>(c, d, S0));
  // predictor: u_* = u_n + dt phi_1(dt J_n) R_n
  PCEXP_TRY(arnoldi<T>(c, escale, m, &c->ss->dt));
  PCEXP_LAUNCH(c, PCEXP_KC_PHI, launch_phi(c->ks, &c->ss->dt, 0.0, 1.0, c->ss, 0, c->st));
  PCEXP_LAUNCH(c, PCEXP_KC_AXPY, launch_krylov_axpy<T>(c->U64[a], c->U64[b], S1, delta, V, c->Kp, c->Kp, c->ks, c->st));
  if (scheme == PCEXP_SCHEME_EXP1) {
    c->cur = b;
    return PCEXP_OK;
  }
  // corrector input N_* - N_n = R(u_*) - R_n - J_n (u_* - u_n)
  (void)G;
  PCEXP_TRY(dg_apply<T>(c, d, S1, nullptr, w, escale, nullptr));
  PCEXP_TRY(jac_apply<T>(c, d, delta, tmp, escale, nullptr, nullptr));
  PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_combine_corrector<T>(V, w, tmp, c->Kp, c->st));
  // corrector: u_{n+1} = u_* + dt/2 phi_1(dt J_n) (N_* - N_n)
  PCEXP_TRY(arnoldi<T>(c, escale, m, &c->ss->dt));
  PCEXP_LAUNCH(c, PCEXP_KC_PHI, launch_phi(c->ks, &c->ss->dt, 0.0, 0.5, c->ss, 1, c->st));
  PCEXP_LAUNCH(c, PCEXP_KC_AXPY, launch_krylov_axpy<T>(c->U64[b], c->U64[a], S0, nullptr, V, c->Kp, c->Kp, c->ks, c->st));
  return PCEXP_OK;
}

// ETD2 (Eq. s7) once V[0] holds R_n and ss->dt holds dt:
//   u_{n+1} = u_n + dt phi_1(dt J_n) R_n + dt (dt / dt_{n-1}) phi_2(dt J_n) (N_n - N_{n-1}),
//   N_n - N_{n-1} = R_n - R_{n-1} - J_n (u_n - u_{n-1})  (N(u) = R(u) - J_n u, Eq. starteq2).
// Without history (the first step after a state change) it is ETD1 (Eq. s8).  The new state
// ends in U64[1 - cur]; u_n, R_n and dt become the history of the next step.
template <class T>
int etd2_stages(pcexp_ctx* c, int m) {
  const DGData<T> d = dgdata<T>(c);
  const int a = c->cur, b = 1 - c->cur;
  T* S0 = shadow<T>(c, a);
  T* S1 = shadow<T>(c, b);
  T* V = reinterpret_cast<T*>(c->V);
  T* tmp = reinterpret_cast<T*>(c->tmp);
  T* delta = reinterpret_cast<T*>(c->delta);
  T* hu = reinterpret_cast<T*>(c->h_u);
  T* hR = reinterpret_cast<T*>(c->h_R);
  T* hRc = reinterpret_cast<T*>(c->h_Rc);
  const size_t vb = (size_t)c->Kp * sizeof(T);
  PCEXP_CK(cudaMemcpyAsync(hRc, V, vb, cudaMemcpyDeviceToDevice, c->st));  // R_n
  PCEXP_TRY(linearize<T>(c, d, S0));
  // ETD1 part: u_n + dt phi_1(dt J_n) R_n
  PCEXP_TRY(arnoldi<T>(c, nullptr, m, &c->ss->dt));
  PCEXP_LAUNCH(c, PCEXP_KC_PHI, launch_phi(c->ks, &c->ss->dt, 0.0, 1.0, c->ss, 0, c->st));
  PCEXP_LAUNCH(c, PCEXP_KC_AXPY, launch_krylov_axpy<T>(c->U64[a], c->U64[b], S1, nullptr, V, c->Kp, c->Kp, c->ks, c->st));
  if (c->etd2_prev) {
    // N_n - N_{n-1}, then + dt (dt / dt_{n-1}) phi_2(dt J_n) (N_n - N_{n-1})
    PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_lincomb3<T>(delta, S0, hu, nullptr, c->Kp, c->st));
    PCEXP_TRY(jac_apply<T>(c, d, delta, tmp, nullptr, nullptr, nullptr));
    PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_lincomb3<T>(V, hRc, hR, tmp, c->Kp, c->st));
    PCEXP_TRY(arnoldi<T>(c, nullptr, m, &c->ss->dt));
    PCEXP_LAUNCH(c, PCEXP_KC_PHI, launch_phi(c->ks, &c->ss->dt, 0.0, 1.0, c->ss, 1, c->st, 2, &c->ss->dt_prev));
    PCEXP_LAUNCH(c, PCEXP_KC_AXPY,
                 launch_krylov_axpy<T>(c->U64[b], c->U64[b], S1, nullptr, V, c->Kp, c->Kp, c->ks, c->st));
  }
  PCEXP_CK(cudaMemcpyAsync(hu, S0, vb, cudaMemcpyDeviceToDevice, c->st));
  PCEXP_CK(cudaMemcpyAsync(hR, hRc, vb, cudaMemcpyDeviceToDevice, c->st));
  PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_keep_dt(c->ss, c->st));
  c->etd2_prev = true;
  c->cur = b;
  return PCEXP_OK;
}

// The launch sequence of one step; reads dt (or the CFL number) from c->param so
// that it can be captured once into a CUDA graph and replayed.
template <class T>
int enqueue_step(pcexp_ctx* c, int scheme, int dt_mode, int m) {
  const DGData<T> d = dgdata<T>(c);
  T* S0 = shadow<T>(c, c->cur);
  T* V = reinterpret_cast<T*>(c->V);
  T* dte = reinterpret_cast<T*>(c->dte);
  const T* escale = nullptr;
  PCEXP_CK(cudaMemsetAsync(&c->ss->err, 0, sizeof(int), c->st));
  if (dt_mode == PCEXP_DT_GIVEN) {
    PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_copy_dt(c->ss, c->param, c->st));
  } else if (c->grp) {
    // the own elements' steps; the global one is their minimum over the partitions (the halo
    // elements' local steps are not formed: their rows of every scaled vector are zero)
    PCEXP_LAUNCH(c, PCEXP_KC_DT, launch_local_dt<T>(d, S0, c->param, 0.0, dte, &c->ss->dtmin_scratch, c->partials, &c->ss->counter, c->st));
    if (dt_mode == PCEXP_DT_LOCAL_CFL) {
      escale = dte;
      PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_set_dt(c->ss, 1.0, c->st));
    } else {
      PCEXP_TRY(group_min_dt(c));
    }
  } else {
    PCEXP_LAUNCH(c, PCEXP_KC_DT, launch_local_dt<T>(d, S0, c->param, 0.0, dte, &c->ss->dt, c->partials, &c->ss->counter, c->st));
    if (dt_mode == PCEXP_DT_LOCAL_CFL) {
      escale = dte;
      PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_set_dt(c->ss, 1.0, c->st));
    }
  }
  PCEXP_TRY(dg_apply<T>(c, d, S0, nullptr, V, nullptr, nullptr));
  PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_density_norm<T>(V, nullptr, c->E, c->nb, c->nv, c->volume, c->ss, c->partials, 0, c->p, 0.0, c->st));
  if (escale) PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_scale_elements<T>(V, escale, c->E, c->nv * c->nb, c->st));
  if (scheme == PCEXP_SCHEME_ETD2) return etd2_stages<T>(c, m);
  c->etd2_prev = false;
  return krylov_stages<T>(c, scheme, escale, m);
}

template <class T>
int step_impl(pcexp_ctx* c, int scheme, int dt_mode, double dt_or_cfl, int m, pcexp_step_info* info) {
  const bool etd1_start = scheme == PCEXP_SCHEME_ETD2 && !c->etd2_prev;
  if (scheme == PCEXP_SCHEME_ETD2 && !c->h_u) {
    const size_t es = c->fp32 ? sizeof(float) : sizeof(double), n = (size_t)c->Kp * es / sizeof(double);
    double *a = nullptr, *b = nullptr, *r = nullptr;
    PCEXP_TRY(dalloc(c, &a, n));
    PCEXP_TRY(dalloc(c, &b, n));
    PCEXP_TRY(dalloc(c, &r, n));
    c->h_u = a;
    c->h_R = b;
    c->h_Rc = r;
  }
  PCEXP_CK(launch_set_param(c->param, dt_or_cfl, c->st));
  // an ETD2 step without history (ETD1) runs eagerly: its graph would differ from the others;
  // so do the steps of a partition (their rounds synchronise with the other partitions' host
  // threads)
  if (c->prof || etd1_start || c->grp) {
    PCEXP_TRY(enqueue_step<T>(c, scheme, dt_mode, m));
  } else {
    // the first step of a configuration runs eagerly (it also initialises lazily
    // cached launch parameters); the second is captured into a graph, later ones replay it
    const int key = ((scheme * 4 + dt_mode) * 64 + m) * 2 + c->cur;
    pcexp_ctx::StepGraph* g = nullptr;
    for (auto& e : c->graphs)
      if (e.scheme == scheme && e.dt_mode == dt_mode && e.m == m && e.cur == c->cur) g = &e;
    if (g) {
      PCEXP_CK(cudaGraphLaunch(g->exec, c->st));
      c->cur = g->cur_after;
    } else if (std::find(c->seen_keys.begin(), c->seen_keys.end(), key) == c->seen_keys.end()) {
      c->seen_keys.push_back(key);
      PCEXP_TRY(enqueue_step<T>(c, scheme, dt_mode, m));
    } else {
      const int cur0 = c->cur;
      if (!c->cap_st) PCEXP_CK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
      // capture on the private stream (nothing runs during capture), replay on the caller's
      cudaStream_t user_st = c->st;
      c->st = c->cap_st;
      cudaError_t eb = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
      if (eb != cudaSuccess) {
        c->st = user_st;
        g_last_error = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(eb);
        return PCEXP_ERR_CUDA;
      }
      const int r = enqueue_step<T>(c, scheme, dt_mode, m);
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(c->st, &graph);
      c->st = user_st;
      if (r != PCEXP_OK || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        c->cur = cur0;
        g_last_error = "step capture failed: " + std::string(cudaGetErrorString(ee)) + "; " + g_last_error;
        return r != PCEXP_OK ? r : PCEXP_ERR_CUDA;
      }
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        c->cur = cur0;
        g_last_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
        return PCEXP_ERR_CUDA;
      }
      c->graphs.push_back({scheme, dt_mode, m, cur0, c->cur, exec});
      PCEXP_CK(cudaGraphLaunch(exec, c->st));
    }
  }
  if (scheme != PCEXP_SCHEME_ETD2) c->etd2_prev = false;  // also after a replayed graph
  if (info) {
    StepState h;
    PCEXP_CK(cudaMemcpyAsync(&h, c->ss, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    PCEXP_CK(cudaStreamSynchronize(c->st));
    const bool one_stage = scheme == PCEXP_SCHEME_EXP1 || etd1_start;
    info->krylov_dim[0] = h.k[0];
    info->krylov_dim[1] = one_stage ? 0 : h.k[1];
    info->beta[0] = h.beta[0];
    info->beta[1] = one_stage ? 0.0 : h.beta[1];
    info->dt = h.dt;
    info->res_norm = h.res_norm;
    info->krylov_err[0] = h.kerr[0];
    info->krylov_err[1] = one_stage ? 0.0 : h.kerr[1];
    info->reorth_cols[0] = h.pass2[0];
    info->reorth_cols[1] = one_stage ? 0u : h.pass2[1];
    if (h.err) {
      g_last_error = "non-finite norm, beta or Hessenberg entry";
      return PCEXP_ERR_NONFINITE;
    }
  }
  return PCEXP_OK;
}

template <class T>
int march_impl(pcexp_ctx* c, int scheme, double cfl_max, double decades, int max_iter, int m,
               pcexp_steady_info* info) {
  const DGData<T> d = dgdata<T>(c);
  T* V = reinterpret_cast<T*>(c->V);
  T* G = reinterpret_cast<T*>(c->G);
  T* dte = reinterpret_cast<T*>(c->dte);
  double r1 = -1, rn = -1;
  int n = 1;
  bool conv = false;
  c->etd2_prev = false;
  // Krylov-error cap on the CFL (adaptive dimension only): after each iteration the cap
  // becomes CFL_used * clamp(0.8 (tol / est)^(1/2), 1/4, 2) from the first stage's estimate
  double cap = cfl_max, cfl_used = 0;
  for (; n <= max_iter + 1; ++n) {
    T* S0 = shadow<T>(c, c->cur);
    PCEXP_CK(cudaMemsetAsync(&c->ss->err, 0, sizeof(int), c->st));
    (void)G;
    PCEXP_TRY(dg_apply<T>(c, d, S0, nullptr, V, nullptr, nullptr));
    PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_density_norm<T>(V, nullptr, c->E, c->nb, c->nv, c->volume, c->ss, c->partials, n, c->p, cfl_max, c->st));
    StepState h;
    PCEXP_CK(cudaMemcpyAsync(&h, c->ss, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    PCEXP_CK(cudaStreamSynchronize(c->st));
    rn = h.res_norm;
    if (c->grp) {
      // the norm over the whole mesh from the partitions' sums of squares (each partition's norm
      // is over its own rows, divided by its submesh's measure), and the ramp of Eq. cfl from it
      const double a = rn * c->volume;
      double s2 = 0;
      PCEXP_TRY(group_host_sum(c, a * a, &s2));
      rn = std::sqrt(s2) / c->grp->volume;
      const double ra = rn > 0 ? 1.0 / (rn * rn * rn) : DBL_MAX;
      const double rb = 1.0 + (double)(n - 1) / (2 * c->p + 1);
      h.cfl = std::fmin(cfl_max, std::fmax(ra, rb));
      PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_set_cfl(c->ss, h.cfl, c->st));
    }
    if (!std::isfinite(rn)) {
      g_last_error = "non-finite residual norm";
      return PCEXP_ERR_NONFINITE;
    }
    if (r1 < 0) r1 = rn;
    if (rn <= r1 * std::pow(10.0, -decades)) {
      conv = true;
      break;
    }
    if (n > max_iter) break;
    if (c->ktol > 0) {
      if (n > 1) {
        const double est = h.kerr[0];
        const double f = !(est > 0) ? 2.0 : std::min(2.0, std::max(0.25, 0.8 * std::sqrt(c->ktol / est)));
        cap = std::min(cfl_max, cfl_used * f);
      }
      cfl_used = std::min(h.cfl, cap);
      PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_cap_cfl(c->ss, cap, c->st));
    }
    PCEXP_LAUNCH(c, PCEXP_KC_DT, launch_local_dt<T>(d, S0, &c->ss->cfl, 0.0, dte, &c->ss->dtmin_scratch, c->partials, &c->ss->counter, c->st));
    PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_set_dt(c->ss, 1.0, c->st));
    PCEXP_LAUNCH(c, PCEXP_KC_OTHER, launch_scale_elements<T>(V, dte, c->E, c->nv * c->nb, c->st));
    PCEXP_TRY(krylov_stages<T>(c, scheme, dte, m));
  }
  if (info) {
    info->iterations = n - 1;
    info->res_first = r1;
    info->res_last = rn;
    info->converged = conv ? 1 : 0;
  }
  return PCEXP_OK;
}

__global__ void scale_vec_kernel(double* x, const KState* ks, int col, int64_t n) {
  const double s = ks->s[col];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] *= s;
}

template <class T>
int arnoldi_abi(pcexp_ctx* c, const double* U, const double* b, int m, double* Vout, double* H, int* k, double* beta,
                int on_device) {
  T* lin = reinterpret_cast<T*>(c->delta);
  PCEXP_TRY(import_vec<T>(c, U, on_device, lin));
  PCEXP_TRY(import_vec<T>(c, b, on_device, Vcol<T>(c, 0)));
  PCEXP_TRY(linearize<T>(c, dgdata<T>(c), lin));
  PCEXP_TRY(arnoldi<T>(c, nullptr, m, &c->ss->dt));
  KState hk;
  PCEXP_CK(cudaMemcpyAsync(&hk, c->ks, sizeof(hk), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  if (hk.err) {
    g_last_error = "non-finite Arnoldi quantity";
    return PCEXP_ERR_NONFINITE;
  }
  const int kk = hk.k;
  if (k) *k = kk;
  if (beta) *beta = hk.beta;
  if (H) {
    for (int i = 0; i <= m; ++i)
      for (int j = 0; j < m; ++j) H[i * m + j] = (i <= kk && j < kk) ? hk.H[i * MMAX + j] : 0.0;
  }
  if (Vout) {
    const int ncol = hk.done ? kk : kk + 1;
    for (int j = 0; j <= m; ++j) {
      double* dst = Vout + (int64_t)j * c->K;
      if (j < ncol && hk.beta > 0) {
        double* dd = on_device ? dst : c->io64b;
        if (c->basis_io == PCEXP_BASIS_PAPER)
          PCEXP_CK(launch_internal_to_paper<T>(Vcol<T>(c, j), dd, c->Q, c->E, c->nb, c->nv, c->st));
        else PCEXP_CK(launch_cast<T, double>(Vcol<T>(c, j), dd, c->K, c->st));
        scale_vec_kernel<<<152 * 4, 256, 0, c->st>>>(dd, c->ks, j, c->K);
        PCEXP_CK(cudaGetLastError());
        if (!on_device) {
          PCEXP_CK(cudaMemcpyAsync(dst, dd, c->K * sizeof(double), cudaMemcpyDeviceToHost, c->st));
          PCEXP_CK(cudaStreamSynchronize(c->st));
        }
      } else if (on_device) {
        PCEXP_CK(cudaMemsetAsync(dst, 0, c->K * sizeof(double), c->st));
      } else {
        std::memset(dst, 0, c->K * sizeof(double));
      }
    }
    PCEXP_CK(cudaStreamSynchronize(c->st));
  }
  return PCEXP_OK;
}

// Host L2 projection of an analytic state onto the internal basis:
// u_j = sqrt(det) sum_q w^_q U(x_q) phi^_j(xi_q).  The vortex and the blobs lie in
// the x-y plane (z-velocity zero in 3D).
int project_host(pcexp_ctx* c, int kind, const double* prm, int np, std::vector<double>& u) {
  const Setup& s = c->host;
  const int D = c->dim, NV = c->nv, GEO = D == 2 ? 8 : 12;
  const double g = c->phys.gamma;
  const double a = c->phys.alpha_deg * M_PI / 180.0;
  const double cinf = std::sqrt(g * c->phys.p_inf / c->phys.rho_inf);
  const double u0 = c->phys.mach * cinf * std::cos(a), v0 = c->phys.mach * cinf * std::sin(a);
  const double rinf = c->phys.rho_inf, pinf = c->phys.p_inf;
  if (kind == PCEXP_PROJ_VORTEX && (np < 4 || (np >= 5 && !(prm[4] > 0)))) return PCEXP_ERR_INVALID_ARG;
  if (kind == PCEXP_PROJ_BLOBS && (np < 1 || (np - 1) % 4)) return PCEXP_ERR_INVALID_ARG;
  if (kind < 0 || kind > 2) return PCEXP_ERR_INVALID_ARG;
  u.assign(c->E * c->nv * c->nb, 0.0);
  for (int64_t e = 0; e < c->E; ++e) {
    const double sd = s.geo[GEO * e + D * D];
    for (int q = 0; q < c->nq; ++q) {
      const double x = s.xqphys[(e * c->nq + q) * D], y = s.xqphys[(e * c->nq + q) * D + 1];
      double rho = rinf, uu = u0, vv = v0, p = pinf;
      if (kind == PCEXP_PROJ_VORTEX) {
        const double eps = prm[0], period = prm[3], rad = np >= 5 ? prm[4] : 1.0;
        double dx = x - prm[1], dy = y - prm[2];
        if (period > 0) {
          dx -= period * std::nearbyint(dx / period);
          dy -= period * std::nearbyint(dy / period);
        }
        dx /= rad;
        dy /= rad;
        const double r2 = dx * dx + dy * dy;
        const double f = eps / (2 * M_PI) * std::exp(0.5 * (1 - r2));
        uu = u0 - f * dy;
        vv = v0 + f * dx;
        const double Tinf = pinf / rinf;
        const double T = Tinf - (g - 1) * eps * eps / (8 * g * M_PI * M_PI) * std::exp(1 - r2);
        rho = rinf * std::pow(T / Tinf, 1.0 / (g - 1));
        p = rho * T;
      } else if (kind == PCEXP_PROJ_BLOBS) {
        const double R = prm[0];
        for (int b = 0; b < (np - 1) / 4; ++b) {
          const double* bb = prm + 1 + 4 * b;
          const double wgt = std::exp(-((x - bb[0]) * (x - bb[0]) + (y - bb[1]) * (y - bb[1])) / (R * R));
          rho += bb[2] * wgt;
          p += bb[3] * wgt;
        }
      }
      double U[5] = {rho, rho * uu, rho * vv, 0.0, 0.0};
      U[NV - 1] = p / (g - 1) + 0.5 * rho * (uu * uu + vv * vv);
      for (int v = 0; v < NV; ++v)
        for (int j = 0; j < c->nb; ++j)
          u[(e * c->nv + v) * c->nb + j] += sd * s.Wv[q] * U[v] * s.Bv[q * c->nb + j];
    }
  }
  return PCEXP_OK;
}

// Forward-mode number with three derivative directions (Mach, alpha in degrees, eps) for the
// exact derivative of the projected analytic states (host).
struct Dual3 {
  double v, d[3];
};
Dual3 dc(double x) { return {x, {0.0, 0.0, 0.0}}; }
Dual3 operator+(Dual3 a, Dual3 b) { return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}}; }
Dual3 operator-(Dual3 a, Dual3 b) { return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}}; }
Dual3 operator*(Dual3 a, Dual3 b) {
  return {a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]}};
}
Dual3 operator*(double a, Dual3 b) { return {a * b.v, {a * b.d[0], a * b.d[1], a * b.d[2]}}; }
Dual3 dpow(Dual3 x, double e) {
  const double pv = std::pow(x.v, e), f = e * pv / x.v;
  return {pv, {f * x.d[0], f * x.d[1], f * x.d[2]}};
}

// theta_bar = (du_0/dtheta)^T ubar for the states of project_host, theta = (Mach, alpha in
// degrees, eps): the pointwise state formulas of project_host on Dual3 numbers, projected with
// the same volume rule; ubar in the internal basis.
int project_adjoint_host(pcexp_ctx* c, int kind, const double* prm, int np, const std::vector<double>& ubar,
                         double tb[3]) {
  const Setup& s = c->host;
  const int D = c->dim, NV = c->nv;
  const double g = c->phys.gamma;
  const double cinf = std::sqrt(g * c->phys.p_inf / c->phys.rho_inf);
  const Dual3 mach{c->phys.mach, {1.0, 0.0, 0.0}};
  const Dual3 alpha{c->phys.alpha_deg * M_PI / 180.0, {0.0, M_PI / 180.0, 0.0}};
  const Dual3 ca{std::cos(alpha.v), {0.0, -std::sin(alpha.v) * alpha.d[1], 0.0}};
  const Dual3 sa{std::sin(alpha.v), {0.0, std::cos(alpha.v) * alpha.d[1], 0.0}};
  const Dual3 u0 = cinf * (mach * ca), v0 = cinf * (mach * sa);
  const double rinf = c->phys.rho_inf, pinf = c->phys.p_inf;
  if (kind == PCEXP_PROJ_VORTEX && (np < 4 || (np >= 5 && !(prm[4] > 0)))) return PCEXP_ERR_INVALID_ARG;
  if (kind == PCEXP_PROJ_BLOBS && (np < 1 || (np - 1) % 4)) return PCEXP_ERR_INVALID_ARG;
  if (kind < 0 || kind > 2) return PCEXP_ERR_INVALID_ARG;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t e = 0; e < c->E; ++e) {
    const double sd = s.geo[(D == 2 ? 8 : 12) * e + D * D];
    for (int q = 0; q < c->nq; ++q) {
      const double x = s.xqphys[(e * c->nq + q) * D], y = s.xqphys[(e * c->nq + q) * D + 1];
      Dual3 rho = dc(rinf), uu = u0, vv = v0, p = dc(pinf);
      if (kind == PCEXP_PROJ_VORTEX) {
        const Dual3 eps{prm[0], {0.0, 0.0, 1.0}};
        const double period = prm[3], rad = np >= 5 ? prm[4] : 1.0;
        double dx = x - prm[1], dy = y - prm[2];
        if (period > 0) {
          dx -= period * std::nearbyint(dx / period);
          dy -= period * std::nearbyint(dy / period);
        }
        dx /= rad;
        dy /= rad;
        const double r2 = dx * dx + dy * dy;
        const Dual3 f = (std::exp(0.5 * (1 - r2)) / (2 * M_PI)) * eps;
        uu = u0 - dy * f;
        vv = v0 + dx * f;
        const double Tinf = pinf / rinf;
        const Dual3 T = dc(Tinf) - ((g - 1) / (8 * g * M_PI * M_PI) * std::exp(1 - r2)) * (eps * eps);
        rho = rinf * dpow((1.0 / Tinf) * T, 1.0 / (g - 1));
        p = rho * T;
      } else if (kind == PCEXP_PROJ_BLOBS) {
        const double R = prm[0];
        double r = rinf, pp = pinf;
        for (int b = 0; b < (np - 1) / 4; ++b) {
          const double* bb = prm + 1 + 4 * b;
          const double wgt = std::exp(-((x - bb[0]) * (x - bb[0]) + (y - bb[1]) * (y - bb[1])) / (R * R));
          r += bb[2] * wgt;
          pp += bb[3] * wgt;
        }
        rho = dc(r);
        p = dc(pp);
      }
      Dual3 U[5] = {rho, rho * uu, rho * vv, dc(0.0), dc(0.0)};
      U[NV - 1] = (1.0 / (g - 1)) * p + 0.5 * (rho * (uu * uu + vv * vv));
      for (int v = 0; v < NV; ++v)
        for (int j = 0; j < c->nb; ++j) {
          const double w = sd * s.Wv[q] * s.Bv[q * c->nb + j] * ubar[(e * c->nv + v) * c->nb + j];
          for (int k = 0; k < 3; ++k) acc[k] += w * U[v].d[k];
        }
    }
  }
  for (int k = 0; k < 3; ++k) tb[k] = acc[k];
  return PCEXP_OK;
}

// Checks omega against the mesh (no periodic faces, no far-field faces, rotation about z in
// 2D) and uploads the frame arrays: v_r = omega x x at the volume points, v_r . n at the face
// points of each face (its L element's points, the face rule over its local vertices), v_r at
// the element centroids.
int setup_rotation(pcexp_ctx* c, const pcexp_mesh* mesh) {
  const double* om = c->phys.omega;
  c->rot = om[0] != 0.0 || om[1] != 0.0 || om[2] != 0.0;
  if (!c->rot) return PCEXP_OK;
  const Setup& s = c->host;
  const int D = c->dim;
  if (D == 2 && (om[0] != 0.0 || om[1] != 0.0)) {
    g_last_error = "in 2D the frame rotates about z: omega = (0, 0, omega_z)";
    return PCEXP_ERR_INVALID_ARG;
  }
  if (!mesh || !mesh->coords) {
    g_last_error = "the rotating frame is set up when the context is created";
    return PCEXP_ERR_INVALID_ARG;
  }
  if (mesh->vert_master)
    for (int64_t v = 0; v < mesh->n_vert; ++v)
      if (mesh->vert_master[v] != v) {
        g_last_error = "a rotating frame needs a mesh without periodic faces (v_r depends on position)";
        return PCEXP_ERR_INVALID_ARG;
      }
  for (int64_t f = 0; f < s.F; ++f)
    if (s.fel[2 * f + 1] == -PCEXP_BC_FARFIELD) {
      g_last_error = "far-field faces are not defined in a rotating frame";
      return PCEXP_ERR_INVALID_ARG;
    }
  auto vr_at = [&](const double* x, double* out) {  // omega x x (x-y components in 2D)
    const double X[3] = {x[0], x[1], D == 3 ? x[2] : 0.0};
    const double r[3] = {om[1] * X[2] - om[2] * X[1], om[2] * X[0] - om[0] * X[2], om[0] * X[1] - om[1] * X[0]};
    for (int k = 0; k < D; ++k) out[k] = r[k];
  };
  std::vector<double> vq((size_t)c->E * c->nq * D), vn((size_t)(s.F > 0 ? s.F : 1) * c->nfq, 0.0),
      vc((size_t)c->E * D);
  for (int64_t i = 0; i < c->E * c->nq; ++i) vr_at(&s.xqphys[(size_t)i * D], &vq[(size_t)i * D]);
  const int NF = D + 1;
  for (int64_t e = 0; e < c->E; ++e) {
    double x[3] = {0, 0, 0};
    for (int k = 0; k <= D; ++k)
      for (int d = 0; d < D; ++d) x[d] += mesh->coords[(size_t)D * mesh->elem_vert[(size_t)(D + 1) * e + k] + d];
    for (int d = 0; d < D; ++d) x[d] /= (D + 1);
    vr_at(x, &vc[(size_t)e * D]);
  }
  for (int64_t f = 0; f < s.F; ++f) {
    const int64_t eL = s.fel[2 * f];
    const int fL = s.floc[f] & 0xff;
    for (int q = 0; q < c->nfq; ++q) {
      double x[3] = {0, 0, 0}, v[3];
      for (int k = 0; k < D; ++k) {
        const int32_t vtx = mesh->elem_vert[(size_t)(D + 1) * eL + (fL + 1 + k) % NF];
        for (int d = 0; d < D; ++d) x[d] += s.flam[(size_t)q * D + k] * mesh->coords[(size_t)D * vtx + d];
      }
      vr_at(x, v);
      double a = 0;
      for (int d = 0; d < D; ++d) a += v[d] * s.fgeo[4 * f + d];
      vn[(size_t)f * c->nfq + q] = a;
    }
  }
  if (c->fp32) {
    PCEXP_TRY(upload<float>(c, &c->vrq, vq));
    PCEXP_TRY(upload<float>(c, &c->vrn, vn));
    PCEXP_TRY(upload<float>(c, &c->vrc, vc));
  } else {
    PCEXP_TRY(upload<double>(c, &c->vrq, vq));
    PCEXP_TRY(upload<double>(c, &c->vrn, vn));
    PCEXP_TRY(upload<double>(c, &c->vrc, vc));
  }
  return PCEXP_OK;
}

int UNSUPPORTED_ROTATING(const char* what) {
  g_last_error = std::string(what) + " is not provided in a rotating frame";
  return PCEXP_ERR_UNSUPPORTED;
}

int UNSUPPORTED_FP32_HESS(pcexp_ctx*) {
  g_last_error = "the second-order adjoint is provided for the FP64 form";
  return PCEXP_ERR_UNSUPPORTED;
}

// The re-orthogonalisation option: FP64 contexts keep both Gram-Schmidt passes (their
// reverse step replays the two-pass process as computed).
int check_reorth(const pcexp_options* opt) {
  if (opt->reorth != PCEXP_REORTH_AUTO && opt->reorth != PCEXP_REORTH_ALWAYS &&
      opt->reorth != PCEXP_REORTH_SELECTIVE) {
    g_last_error = "reorth: PCEXP_REORTH_AUTO, PCEXP_REORTH_ALWAYS or PCEXP_REORTH_SELECTIVE";
    return PCEXP_ERR_INVALID_ARG;
  }
  if (opt->reorth == PCEXP_REORTH_SELECTIVE && opt->precision == PCEXP_FP64) {
    g_last_error = "selective re-orthogonalisation is provided for the FP32-mixed form";
    return PCEXP_ERR_UNSUPPORTED;
  }
  return PCEXP_OK;
}

int check_ctx(const pcexp_ctx* c) {
  if (!c) {
    g_last_error = "null context";
    return PCEXP_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) {
    g_last_error = cudaGetErrorString(e);
    return PCEXP_ERR_CUDA;
  }
  return PCEXP_OK;
}

int create_impl(pcexp_ctx* c, const pcexp_mesh* mesh, int p, const pcexp_physics* phys, const pcexp_options* opt,
                const int64_t* elem_key = nullptr) {
  std::string msg;
  int r = build_setup(*mesh, p, c->host, msg, elem_key);
  if (r != PCEXP_OK) {
    g_last_error = msg;
    return r;
  }
  const Setup& s = c->host;
  c->dim = s.dim;
  c->nv = s.nv;
  c->p = p;
  c->nb = s.nb;
  c->nq = s.nq;
  c->nfq = s.nfq;
  c->E = s.E;
  c->F = s.F;
  c->K = c->E * c->nv * c->nb;
  c->Kp = (c->K + VPAD - 1) / VPAD * VPAD;
  c->volume = s.volume;
  c->phys = *phys;
  c->fp32 = opt->precision == PCEXP_FP32_MIXED;
  c->jv_tangent = c->fp32;
  // the face part of J v applies the stored face point Jacobians: recomputing the Roe-flux
  // tangents per face point in every J v measured slower on GB300 (48^3 tetrahedra, P2:
  // 37.6 against 33.9 + 2.0 ms per step with the blocks and their linearisation)
  c->face_tangent = false;
  c->m_max = opt->m_max;
  c->eta = opt->breakdown_eta > 0 ? opt->breakdown_eta : (c->fp32 ? 1e-6 : 1e-12);
  c->ktol = opt->krylov_tol > 0 ? opt->krylov_tol : 0.0;
  c->selective = opt->reorth == PCEXP_REORTH_SELECTIVE || (opt->reorth == PCEXP_REORTH_AUTO && c->fp32);
  c->basis_io = opt->basis_io;
  // tables
  std::vector<double> tabs;
  tabs.insert(tabs.end(), s.Bv.begin(), s.Bv.end());
  tabs.insert(tabs.end(), s.Dv.begin(), s.Dv.end());
  tabs.insert(tabs.end(), s.Bf.begin(), s.Bf.end());
  tabs.insert(tabs.end(), s.Wf.begin(), s.Wf.end());
  tabs.insert(tabs.end(), s.Bc.begin(), s.Bc.end());
  tabs.insert(tabs.end(), s.Wv.begin(), s.Wv.end());
  {
    // the trace tables again with each row padded to whole 16-byte vectors (4 floats or
    // 2 doubles), the padded block itself starting on a 16-byte boundary
    const size_t vec = c->fp32 ? 4 : 2, nbp = (s.nb + vec - 1) / vec * vec;
    while (tabs.size() % vec) tabs.push_back(0.0);
    const size_t rows = s.Bf.size() / s.nb;
    for (size_t r = 0; r < rows; ++r)
      for (size_t j = 0; j < nbp; ++j) tabs.push_back(j < (size_t)s.nb ? s.Bf[r * s.nb + j] : 0.0);
  }
  const size_t es = c->fp32 ? sizeof(float) : sizeof(double);
  if (c->fp32) {
    PCEXP_TRY(upload<float>(c, &c->tabs, tabs));
    PCEXP_TRY(upload<float>(c, &c->geo, s.geo));
    PCEXP_TRY(upload<float>(c, &c->fgeo, s.fgeo));
    if (c->jv_tangent) PCEXP_CK(launch_tan_tables(dgdata<float>(c), c->st));
  } else {
    PCEXP_TRY(upload<double>(c, &c->tabs, tabs));
    PCEXP_TRY(upload<double>(c, &c->geo, s.geo));
    PCEXP_TRY(upload<double>(c, &c->fgeo, s.fgeo));
  }
  void* q = nullptr;
  PCEXP_TRY(upload<double>(c, &q, s.Q));
  c->Q = reinterpret_cast<double*>(q);
  PCEXP_TRY(dalloc(c, &c->ef, s.ef.size()));
  PCEXP_TRY(dalloc(c, &c->fel, s.fel.size() + 2));
  PCEXP_TRY(dalloc(c, &c->floc, s.floc.size() + 1));
  PCEXP_CK(cudaMemcpyAsync(c->ef, s.ef.data(), s.ef.size() * 4, cudaMemcpyHostToDevice, c->st));
  if (s.F) {
    PCEXP_CK(cudaMemcpyAsync(c->fel, s.fel.data(), s.fel.size() * 4, cudaMemcpyHostToDevice, c->st));
    PCEXP_CK(cudaMemcpyAsync(c->floc, s.floc.data(), s.floc.size() * 4, cudaMemcpyHostToDevice, c->st));
  }
  // state and work vectors
  const int64_t Kp = c->Kp;
  for (int i = 0; i < 2; ++i) PCEXP_TRY(dalloc(c, &c->U64[i], Kp));
  auto valloc = [&](void** p, size_t n) -> int {
    if (c->fp32) {
      float* f = nullptr;
      int rr = dalloc(c, &f, n);
      *p = f;
      return rr;
    }
    double* d = nullptr;
    int rr = dalloc(c, &d, n);
    *p = d;
    return rr;
  };
  if (c->fp32)
    for (int i = 0; i < 2; ++i) PCEXP_TRY(valloc(&c->S32[i], Kp));
  PCEXP_TRY(valloc(&c->V, (size_t)(c->m_max + 1) * Kp));
  PCEXP_TRY(valloc(&c->w, Kp));
  PCEXP_TRY(valloc(&c->tmp, Kp));
  PCEXP_TRY(valloc(&c->delta, Kp));
  const size_t nfp = (size_t)(c->F > 0 ? c->F : 1) * c->nfq, nv = (size_t)c->nv;
  PCEXP_TRY(valloc(&c->G, nfp * nv));
  PCEXP_TRY(valloc(&c->dte, c->E));
  PCEXP_TRY(valloc(&c->Avol, (size_t)c->dim * nv * nv * c->E * c->nq));
  PCEXP_TRY(valloc(&c->GT, 2 * nv * nfp));
  PCEXP_TRY(valloc(&c->Bface, 2 * nv * nv * nfp));
  PCEXP_TRY(dalloc(c, &c->io64a, Kp));
  PCEXP_TRY(dalloc(c, &c->io64b, Kp));
  PCEXP_TRY(dalloc(c, &c->ks, 1));
  PCEXP_TRY(dalloc(c, &c->ss, 1));
  PCEXP_TRY(dalloc(c, &c->partials, (size_t)RED_BLOCKS * (MMAX + 2)));
  PCEXP_TRY(dalloc(c, &c->param, 1));
  (void)es;
  PCEXP_CK(cudaStreamSynchronize(c->st));
  PCEXP_TRY(setup_rotation(c, mesh));
  // free-stream initial state
  std::vector<double> u;
  PCEXP_TRY(project_host(c, PCEXP_PROJ_FREESTREAM, nullptr, 0, u));
  PCEXP_CK(cudaMemcpyAsync(c->U64[0], u.data(), u.size() * 8, cudaMemcpyHostToDevice, c->st));
  PCEXP_TRY(refresh_shadow<double>(c, 0));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

template <class T>
int vjp_impl(pcexp_ctx* c, const double* U, const double* w, double* JTw, int on_device) {
  T* a = reinterpret_cast<T*>(c->tmp);
  T* b = reinterpret_cast<T*>(c->delta);
  T* o = reinterpret_cast<T*>(c->w);
  const DGData<T> d = dgdata<T>(c);
  PCEXP_TRY(import_vec<T>(c, U, on_device, a));
  PCEXP_TRY(import_vec<T>(c, w, on_device, b));
  PCEXP_TRY(linearize<T>(c, d, a, true));
  PCEXP_CK(launch_jac_adjoint<T>(d, lindata<T>(c), b, o, reinterpret_cast<T*>(c->GT), nullptr, T(1), c->st));
  PCEXP_TRY(export_vec<T>(c, o, JTw, on_device));
  if (on_device) PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}


// ------------------------------------------------------------------ reverse step
int alloc_backward(pcexp_ctx* c) {
  if (c->b_un) return PCEXP_OK;
  const size_t Kp = (size_t)c->Kp, Vn = (size_t)(c->m_max + 1) * Kp;
  double** vecs[] = {&c->b_un, &c->b_us, &c->b_dl, &c->b_w1, &c->b_w0, &c->b_wb2, &c->b_wb1, &c->b_wb0,
                     &c->b_t1, &c->b_t2, &c->b_ubn, &c->b_ubs, &c->b_db, &c->b_bb, &c->b_rb, &c->b_gin};
  for (double** v : vecs) PCEXP_TRY(dalloc(c, v, Kp));
  PCEXP_TRY(dalloc(c, &c->b_V1, Vn));
  PCEXP_TRY(dalloc(c, &c->b_Vb, Vn));
  PCEXP_TRY(dalloc(c, &c->b_small, (size_t)2 * MMAX * MMAX));
  PCEXP_TRY(dalloc(c, &c->b_theta, 2));
  PCEXP_TRY(dalloc(c, &c->b_ks1, 1));
  PCEXP_TRY(dalloc(c, &c->b_as, 1));
  if (c->grp) {  // partition of a group: the reverse reductions are summed over the partitions
    const int one = 1;
    PCEXP_CK(cudaMemcpyAsync(reinterpret_cast<char*>(c->b_as) + offsetof(AdjState, group), &one, sizeof(int),
                             cudaMemcpyHostToDevice, c->st));
  }
  PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

// d(free-stream velocity)/d(Mach) and d/d(alpha in degrees), x and y components: the velocity
// Ma c_inf (cos alpha, sin alpha) is the only place the two parameters enter the operator.
void freestream_velocity_derivatives(const pcexp_physics& ph, double dvel[4]) {
  const double a = ph.alpha_deg * M_PI / 180.0, cinf = std::sqrt(ph.gamma * ph.p_inf / ph.rho_inf);
  dvel[0] = cinf * std::cos(a);
  dvel[1] = cinf * std::sin(a);
  dvel[2] = -ph.mach * cinf * std::sin(a) * M_PI / 180.0;
  dvel[3] = ph.mach * cinf * std::cos(a) * M_PI / 180.0;
}

// theta_bar += (d(...)/dtheta)^T w for the reverse step: order 1 with u (R(u)), order 2 with
// u and t (J(u) t), scaled by osc (and *osc_dev)
int param_adjoint(pcexp_ctx* c, const DGData<double>& d, int order, const double* u, const double* t, const double* w,
                  double osc, const double* osc_dev) {
  double dvel[4];
  freestream_velocity_derivatives(c->phys, dvel);
  PCEXP_CK(launch_param_adjoint<double>(d, c->host.F_interior, order, u, t, w, osc, osc_dev, dvel, c->b_theta,
                                        c->partials, &c->b_as->counter, c->st));
  return PCEXP_OK;
}

// A reduction of the reverse Krylov stage in a partitioned run: the partitions' sums (left in
// b_as->gsum) summed in partition order into b_as->dots, then the reduction's finishing step.
int adj_round(pcexp_ctx* c, int kind, int mode, int j, int k, double fdt, const KState* ks) {
  if (!c->grp) return PCEXP_OK;
  AdjState* as = c->b_as;
  return group_round(c, dev_field(as, offsetof(AdjState, gsum)), [&](const PartPtrs& pp) -> int {
    PCEXP_CK(launch_group_reduce(pp, c->grp->n, MMAX + 2, dev_field(as, offsetof(AdjState, dots)), 0, c->st));
    PCEXP_CK(launch_adj_finish(kind, mode, j, k, fdt, ks, as, c->st));
    return PCEXP_OK;
  });
}

// Seeding of a stage's reverse from the adjoint ubar of u_out = u_base + fdt beta V_k y
int adj_seed(pcexp_ctx* c, const double* Z, const double* ubar, int k, int m, double fdt, const KState* ks) {
  PCEXP_CK(launch_adj_ybar(Z, c->Kp, ubar, c->Kp, k, fdt, ks, c->b_as, c->partials, c->st));
  PCEXP_TRY(adj_round(c, ADJ_YBAR, 0, 0, k, fdt, ks));
  PCEXP_CK(launch_adj_vbar_init(c->b_Vb, c->Kp, ubar, c->Kp, k, m, fdt, ks, c->st));
  return PCEXP_OK;
}

// Reverse of Gram-Schmidt column j (its w0 bar ends in b_wb0)
int adj_column(pcexp_ctx* c, const double* Z, int j, bool last_col, const KState* ks) {
  const int64_t Kp = c->Kp;
  PCEXP_CK(launch_adj_recompute(Z, Kp, Kp, j, ks, c->b_w1, c->b_w0, c->st));
  if (!last_col) {
    PCEXP_CK(launch_adj_alpha(Z, Kp, c->b_Vb, Kp, j, ks, c->b_as, c->partials, c->st));
    PCEXP_TRY(adj_round(c, ADJ_ALPHA, 0, j, 0, 0.0, ks));
  }
  for (int mode = 0; mode < 2; ++mode) {
    PCEXP_CK(launch_adj_upd(mode, Z, Kp, c->b_Vb, mode == 0 ? nullptr : c->b_wb2, mode == 0 ? c->b_wb2 : c->b_wb1,
                            Kp, j, last_col ? 1 : 0, ks, c->b_as, c->partials, c->st));
    PCEXP_TRY(adj_round(c, mode == 0 ? ADJ_UPD0 : ADJ_UPD1, mode, j, 0, 0.0, ks));
  }
  PCEXP_CK(launch_adj_rank(Z, Kp, c->b_Vb, c->b_w1, c->b_w0, c->b_wb2, c->b_wb1, c->b_wb0, Kp, j, ks, c->b_as,
                           c->st));
  return PCEXP_OK;
}

// out = J_n^T w (w's halo rows from the owners in a partitioned run; own rows of out kept)
int adj_jt(pcexp_ctx* c, const DGData<double>& d, double* w, double* out) {
  PCEXP_TRY(group_exchange<double>(c, w));
  PCEXP_CK(launch_jac_adjoint<double>(d, lindata<double>(c), w, out, reinterpret_cast<double*>(c->GT), nullptr, 1.0,
                                      c->st));
  return group_zero_halo<double>(c, out);
}

// out = (d(J(u) v)/du)^T w at u = b_un (v's and w's halo rows from the owners; v's restored to
// zero when it is a Krylov vector)
int adj_hess(pcexp_ctx* c, const DGData<double>& d, double* v, bool v_krylov, double* w, double* out) {
  PCEXP_TRY(group_exchange<double>(c, v));
  PCEXP_TRY(group_exchange<double>(c, w));
  PCEXP_CK(launch_jvp_state_adjoint<double>(d, c->b_un, v, w, out, reinterpret_cast<double*>(c->GT), nullptr, 1.0,
                                            c->st));
  if (v_krylov) PCEXP_TRY(group_zero_halo<double>(c, v));
  return group_zero_halo<double>(c, out);
}

// Reverse of one Arnoldi + phi + update stage; Vb holds the seeded basis adjoints.
// Accumulates the second-order terms into b_ubn and leaves the start-vector adjoint in b_bb.
// In a partitioned run every vector here keeps zero halo rows except while an adjoint operator
// pass reads them (the parameter adjoint then counts each boundary face in its own partition).
int reverse_krylov(pcexp_ctx* c, const DGData<double>& d, double* Z, const KState* ks, int k) {
  const int64_t Kp = c->Kp;
  for (int j = k - 1; j >= 0; --j) {
    PCEXP_TRY(adj_column(c, Z, j, j == k - 1, ks));
    // w0 = J_n v_j: vbar_j += J_n^T w0bar;  ubar_n += (d(J(u) v_j)/du)^T w0bar, v_j = s_j z_j
    PCEXP_TRY(adj_jt(c, d, c->b_wb0, c->b_t1));
    PCEXP_CK(launch_axpy(c->b_Vb + (int64_t)j * Kp, c->b_t1, nullptr, 1.0, Kp, c->st));
    PCEXP_TRY(adj_hess(c, d, Z + (int64_t)j * Kp, true, c->b_wb0, c->b_t2));
    PCEXP_CK(launch_axpy(c->b_ubn, c->b_t2, &ks->s[j], 1.0, Kp, c->st));
    PCEXP_TRY(group_zero_halo<double>(c, c->b_wb0));
    // theta_bar += s_j (d(J(u_n; theta) z_j)/dtheta)^T w0bar
    PCEXP_TRY(param_adjoint(c, d, 2, c->b_un, Z + (int64_t)j * Kp, c->b_wb0, 1.0, &ks->s[j]));
  }
  PCEXP_CK(launch_adj_b0dot(Z, c->b_Vb, Kp, c->b_as, c->partials, c->st));
  PCEXP_TRY(adj_round(c, ADJ_B0, 0, 0, 0, 0.0, ks));
  PCEXP_CK(launch_adj_bbar_from(Z, c->b_Vb, c->b_bb, Kp, ks, c->b_as, c->st));
  return PCEXP_OK;
}

int step_backward_impl(pcexp_ctx* c, const double* U, double dt, int m, const double* ubar_next, double* ubar,
                       double* theta_bar, int on_device) {
  PCEXP_TRY(alloc_backward(c));
  const DGData<double> d = dgdata<double>(c);
  const int64_t Kp = c->Kp;
  double* V = reinterpret_cast<double*>(c->V);
  double* w = reinterpret_cast<double*>(c->w);
  double* tmp = reinterpret_cast<double*>(c->tmp);
  const size_t vbytes = (size_t)Kp * sizeof(double);
  const bool prof = c->prof;
  c->prof = false;
  PCEXP_TRY(import_vec<double>(c, U, on_device, c->b_un));
  PCEXP_TRY(import_vec<double>(c, ubar_next, on_device, c->b_gin));
  // ---- forward recompute of the step from the checkpoint u_n (Eq. s9, s10)
  PCEXP_CK(cudaMemsetAsync(&c->ss->err, 0, sizeof(int), c->st));
  PCEXP_CK(launch_set_dt(c->ss, dt, c->st));
  PCEXP_TRY(dg_apply<double>(c, d, c->b_un, nullptr, V, nullptr, nullptr));
  PCEXP_TRY(linearize<double>(c, d, c->b_un));
  PCEXP_TRY(arnoldi<double>(c, nullptr, m));
  PCEXP_CK(cudaMemcpyAsync(c->b_ks1, c->ks, sizeof(KState), cudaMemcpyDeviceToDevice, c->st));
  PCEXP_CK(cudaMemcpyAsync(c->b_V1, V, (size_t)(m + 1) * vbytes, cudaMemcpyDeviceToDevice, c->st));
  PCEXP_CK(launch_phi(c->b_ks1, &c->ss->dt, 0.0, 1.0, c->ss, 0, c->st));
  PCEXP_CK(launch_krylov_axpy<double>(c->b_un, c->b_us, c->b_us, c->b_dl, c->b_V1, Kp, Kp, c->b_ks1, c->st));
  PCEXP_TRY(dg_apply<double>(c, d, c->b_us, nullptr, w, nullptr, nullptr));
  PCEXP_TRY(jac_apply<double>(c, d, c->b_dl, tmp, nullptr, nullptr, nullptr));
  PCEXP_CK(launch_combine_corrector<double>(V, w, tmp, Kp, c->st));
  PCEXP_TRY(arnoldi<double>(c, nullptr, m));
  PCEXP_CK(launch_phi(c->ks, &c->ss->dt, 0.0, 0.5, c->ss, 1, c->st));
  KState h1, h2;
  PCEXP_CK(cudaMemcpyAsync(&h1, c->b_ks1, sizeof(KState), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaMemcpyAsync(&h2, c->ks, sizeof(KState), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  if (h1.err || h2.err) {
    c->prof = prof;
    g_last_error = "non-finite quantity in the recomputed step";
    return PCEXP_ERR_NONFINITE;
  }
  const int k1 = h1.k, k2 = h2.k;
  // ---- reverse
  PCEXP_CK(cudaMemsetAsync(c->b_theta, 0, 2 * sizeof(double), c->st));
  PCEXP_CK(cudaMemsetAsync(c->b_ubn, 0, vbytes, c->st));
  PCEXP_CK(cudaMemsetAsync(c->b_rb, 0, vbytes, c->st));
  PCEXP_CK(cudaMemsetAsync(c->b_db, 0, vbytes, c->st));
  PCEXP_CK(cudaMemcpyAsync(c->b_ubs, c->b_gin, vbytes, cudaMemcpyDeviceToDevice, c->st));
  if (k2 > 0) {
    // u_{n+1} = u_* + dt/2 beta_2 V_2 y_2
    PCEXP_TRY(adj_seed(c, V, c->b_gin, k2, m, 0.5 * dt, c->ks));
    PCEXP_CK(launch_phi_adjoint(c->ks->H, k2, MMAX, dt, c->b_as->ybar, c->b_as->Hbar, &c->b_as->err, c->st));
    PCEXP_TRY(reverse_krylov(c, d, V, c->ks, k2));
    // N_* - N_n = R(u_*) - R_n - J_n delta, with bbar_2 = b_bb
    PCEXP_TRY(adj_jt(c, d, c->b_bb, c->b_t1));
    PCEXP_CK(launch_axpy(c->b_db, c->b_t1, nullptr, -1.0, Kp, c->st));
    PCEXP_TRY(adj_hess(c, d, c->b_dl, false, c->b_bb, c->b_t2));
    PCEXP_CK(launch_axpy(c->b_ubn, c->b_t2, nullptr, -1.0, Kp, c->st));
    PCEXP_TRY(group_zero_halo<double>(c, c->b_bb));
    PCEXP_CK(launch_axpy(c->b_rb, c->b_bb, nullptr, -1.0, Kp, c->st));
    // theta_bar -= (d(J(u_n; theta) delta)/dtheta)^T bbar_2;  += (dR(u_*; theta)/dtheta)^T bbar_2
    PCEXP_TRY(param_adjoint(c, d, 2, c->b_un, c->b_dl, c->b_bb, -1.0, nullptr));
    PCEXP_TRY(param_adjoint(c, d, 1, c->b_us, nullptr, c->b_bb, 1.0, nullptr));
    PCEXP_TRY(linearize<double>(c, d, c->b_us));
    PCEXP_TRY(adj_jt(c, d, c->b_bb, c->b_t1));
    PCEXP_CK(launch_axpy(c->b_ubs, c->b_t1, nullptr, 1.0, Kp, c->st));
    PCEXP_TRY(linearize<double>(c, d, c->b_un));
  }
  // u_* = u_n + delta
  PCEXP_CK(launch_axpy(c->b_ubn, c->b_ubs, nullptr, 1.0, Kp, c->st));
  PCEXP_CK(launch_axpy(c->b_db, c->b_ubs, nullptr, 1.0, Kp, c->st));
  if (k1 > 0) {
    // delta = dt beta_1 V_1 y_1
    PCEXP_TRY(adj_seed(c, c->b_V1, c->b_db, k1, m, dt, c->b_ks1));
    PCEXP_CK(launch_phi_adjoint(c->b_ks1->H, k1, MMAX, dt, c->b_as->ybar, c->b_as->Hbar, &c->b_as->err, c->st));
    PCEXP_TRY(reverse_krylov(c, d, c->b_V1, c->b_ks1, k1));
    PCEXP_CK(launch_axpy(c->b_rb, c->b_bb, nullptr, 1.0, Kp, c->st));
  }
  // R_n = R(u_n)
  PCEXP_TRY(adj_jt(c, d, c->b_rb, c->b_t1));
  PCEXP_CK(launch_axpy(c->b_ubn, c->b_t1, nullptr, 1.0, Kp, c->st));
  PCEXP_TRY(group_zero_halo<double>(c, c->b_rb));
  PCEXP_TRY(param_adjoint(c, d, 1, c->b_un, nullptr, c->b_rb, 1.0, nullptr));
  c->prof = prof;
  PCEXP_TRY(export_vec<double>(c, c->b_ubn, ubar, on_device));
  int aerr = 0;
  double th[2] = {0.0, 0.0};
  PCEXP_CK(cudaMemcpyAsync(&aerr, &c->b_as->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaMemcpyAsync(th, c->b_theta, sizeof(th), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  if (theta_bar) {
    theta_bar[0] = th[0];
    theta_bar[1] = th[1];
  }
  if (aerr) {
    g_last_error = "non-finite phi adjoint";
    return PCEXP_ERR_NONFINITE;
  }
  return PCEXP_OK;
}

int phi_adjoint_abi(pcexp_ctx* c, const double* H, int k, int ldh, double dt, const double* ybar, double* Hbar) {
  PCEXP_TRY(alloc_backward(c));
  AdjState* as = c->b_as;
  double* dH = c->b_small;  // k*k entries, leading dimension k
  double* dHb = c->b_small + MMAX * MMAX;
  PCEXP_CK(cudaMemsetAsync(&as->err, 0, sizeof(int), c->st));
  std::vector<double> Hk((size_t)k * k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Hk[(size_t)i * k + j] = H[(size_t)i * ldh + j];
  PCEXP_CK(cudaMemcpyAsync(dH, Hk.data(), Hk.size() * 8, cudaMemcpyHostToDevice, c->st));
  PCEXP_CK(cudaMemcpyAsync(as->ybar, ybar, (size_t)k * 8, cudaMemcpyHostToDevice, c->st));
  PCEXP_CK(launch_phi_adjoint(dH, k, k, dt, as->ybar, dHb, &as->err, c->st));
  std::vector<double> out((size_t)k * k);
  int err = 0;
  PCEXP_CK(cudaMemcpyAsync(out.data(), dHb, out.size() * 8, cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaMemcpyAsync(&err, &as->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  if (err) return PCEXP_ERR_NONFINITE;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Hbar[(size_t)i * ldh + j] = out[(size_t)i * k + j];
  return PCEXP_OK;
}
}  // namespace

namespace pcexp {
// Sets the calling thread's pcexp_last_error() text (for entry points outside this file).
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

// Read-only view of a context for pcexp_residual_noalloc (noalloc.cu); makes the
// context's device current.
int ctx_noalloc_view(pcexp_ctx* c, DGData<double>* d, cudaStream_t* st, int* nfq, int* fp32, int* device) {
  int r = check_ctx(c);
  if (r != PCEXP_OK) return r;
  *d = dgdata<double>(c);
  *st = c->st;
  *nfq = c->nfq;
  *fp32 = c->fp32 ? 1 : 0;
  *device = c->device;
  return PCEXP_OK;
}
}  // namespace pcexp

extern "C" {

int pcexp_create(pcexp_ctx** out, const pcexp_mesh* mesh, int p, const pcexp_physics* phys,
                 const pcexp_options* opt, void* cuda_stream) {
  if (!out) return PCEXP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !phys || !opt) return PCEXP_ERR_INVALID_ARG;
  if (opt->m_max < 1 || opt->m_max > PCEXP_MAX_KRYLOV) return PCEXP_ERR_INVALID_ARG;
  if (opt->precision != PCEXP_FP64 && opt->precision != PCEXP_FP32_MIXED) return PCEXP_ERR_INVALID_ARG;
  if (opt->basis_io != PCEXP_BASIS_PAPER && opt->basis_io != PCEXP_BASIS_INTERNAL) return PCEXP_ERR_INVALID_ARG;
  if (!(phys->gamma > 1.0) || !(phys->rho_inf > 0) || !(phys->p_inf > 0)) return PCEXP_ERR_INVALID_ARG;
  PCEXP_TRY(check_reorth(opt));
  pcexp_ctx* c = new pcexp_ctx();
  cudaGetDevice(&c->device);
  c->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int r = create_impl(c, mesh, p, phys, opt);
  if (r != PCEXP_OK) {
    std::string keep = g_last_error;
    pcexp_destroy(c);
    g_last_error = keep;
    return r;
  }
  *out = c;
  return PCEXP_OK;
}

int pcexp_destroy(pcexp_ctx* c) {
  if (!c) return PCEXP_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->st);
  for (void* p : c->allocs) cudaFree(p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  delete c;
  return PCEXP_OK;
}

int pcexp_sizes(const pcexp_ctx* c, int64_t* n_elem, int32_t* n_basis, int32_t* n_var, int64_t* K) {
  if (!c) return PCEXP_ERR_INVALID_ARG;
  if (n_elem) *n_elem = c->E;
  if (n_basis) *n_basis = c->nb;
  if (n_var) *n_var = c->nv;
  if (K) *K = c->K;
  return PCEXP_OK;
}

int pcexp_set_state(pcexp_ctx* c, const double* U, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U) return PCEXP_ERR_INVALID_ARG;
  PCEXP_TRY(import_vec<double>(c, U, on_device, c->U64[c->cur]));
  PCEXP_TRY(refresh_shadow<double>(c, c->cur));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  c->etd2_prev = false;
  return PCEXP_OK;
}

int pcexp_get_state(pcexp_ctx* c, double* U, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U) return PCEXP_ERR_INVALID_ARG;
  return export_vec<double>(c, c->U64[c->cur], U, on_device);
}

int pcexp_project_state(pcexp_ctx* c, int kind, const double* params, int n_params) {
  PCEXP_TRY(check_ctx(c));
  if (n_params > 0 && !params) return PCEXP_ERR_INVALID_ARG;
  std::vector<double> u;
  PCEXP_TRY(project_host(c, kind, params, n_params, u));
  PCEXP_CK(cudaMemcpyAsync(c->U64[c->cur], u.data(), u.size() * 8, cudaMemcpyHostToDevice, c->st));
  PCEXP_TRY(refresh_shadow<double>(c, c->cur));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  c->etd2_prev = false;
  return PCEXP_OK;
}

int pcexp_residual(pcexp_ctx* c, const double* U, double* R, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !R) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) {
    float* in = reinterpret_cast<float*>(c->tmp);
    float* out = reinterpret_cast<float*>(c->w);
    PCEXP_TRY(import_vec<float>(c, U, on_device, in));
    PCEXP_CK(launch_dg_operator<float>(dgdata<float>(c), in, nullptr, out, reinterpret_cast<float*>(c->G), nullptr, nullptr, c->st));
    PCEXP_TRY(export_vec<float>(c, out, R, on_device));
  } else {
    double* in = reinterpret_cast<double*>(c->tmp);
    double* out = reinterpret_cast<double*>(c->w);
    PCEXP_TRY(import_vec<double>(c, U, on_device, in));
    PCEXP_CK(launch_dg_operator<double>(dgdata<double>(c), in, nullptr, out, reinterpret_cast<double*>(c->G), nullptr, nullptr, c->st));
    PCEXP_TRY(export_vec<double>(c, out, R, on_device));
  }
  if (on_device) PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

int pcexp_jvp(pcexp_ctx* c, const double* U, const double* v, double* Jv, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !v || !Jv) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) {
    float* a = reinterpret_cast<float*>(c->tmp);
    float* b = reinterpret_cast<float*>(c->delta);
    float* o = reinterpret_cast<float*>(c->w);
    PCEXP_TRY(import_vec<float>(c, U, on_device, a));
    PCEXP_TRY(import_vec<float>(c, v, on_device, b));
    PCEXP_CK(launch_dg_operator<float>(dgdata<float>(c), a, b, o, reinterpret_cast<float*>(c->G), nullptr, nullptr, c->st));
    PCEXP_TRY(export_vec<float>(c, o, Jv, on_device));
  } else {
    double* a = reinterpret_cast<double*>(c->tmp);
    double* b = reinterpret_cast<double*>(c->delta);
    double* o = reinterpret_cast<double*>(c->w);
    PCEXP_TRY(import_vec<double>(c, U, on_device, a));
    PCEXP_TRY(import_vec<double>(c, v, on_device, b));
    PCEXP_CK(launch_dg_operator<double>(dgdata<double>(c), a, b, o, reinterpret_cast<double*>(c->G), nullptr, nullptr, c->st));
    PCEXP_TRY(export_vec<double>(c, o, Jv, on_device));
  }
  if (on_device) PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

int pcexp_jvp_state_adjoint(pcexp_ctx* c, const double* U, const double* v, const double* w, double* out,
                            int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !v || !w || !out) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) return UNSUPPORTED_FP32_HESS(c);
  if (c->rot) return UNSUPPORTED_ROTATING("the second-order adjoint");
  double* a = reinterpret_cast<double*>(c->tmp);
  double* b = reinterpret_cast<double*>(c->delta);
  double* ww = reinterpret_cast<double*>(c->V);  // V[0] as scratch
  double* o = reinterpret_cast<double*>(c->w);
  PCEXP_TRY(import_vec<double>(c, U, on_device, a));
  PCEXP_TRY(import_vec<double>(c, v, on_device, b));
  PCEXP_TRY(import_vec<double>(c, w, on_device, ww));
  PCEXP_CK(launch_jvp_state_adjoint<double>(dgdata<double>(c), a, b, ww, o, reinterpret_cast<double*>(c->GT), nullptr,
                                            1.0, c->st));
  PCEXP_TRY(export_vec<double>(c, o, out, on_device));
  if (on_device) PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

int pcexp_functional_params(pcexp_ctx* c, int kind, const double* params, int n_params, const double* U,
                            double* value, double* grad, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !value) return PCEXP_ERR_INVALID_ARG;
  if (kind != PCEXP_FUNC_WALL_FX && kind != PCEXP_FUNC_WALL_FY && kind != PCEXP_FUNC_WALL_FZ &&
      kind != PCEXP_FUNC_VORTEX_L2)
    return PCEXP_ERR_INVALID_ARG;
  if (kind == PCEXP_FUNC_WALL_FZ && c->dim != 3) return PCEXP_ERR_INVALID_ARG;
  if (kind == PCEXP_FUNC_VORTEX_L2 && (!params || n_params < 5)) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) {
    g_last_error = "output functionals are provided for the FP64 form";
    return PCEXP_ERR_UNSUPPORTED;
  }
  double* a = reinterpret_cast<double*>(c->tmp);
  double* g = reinterpret_cast<double*>(c->w);
  const DGData<double> d = dgdata<double>(c);
  PCEXP_TRY(import_vec<double>(c, U, on_device, a));
  if (kind == PCEXP_FUNC_VORTEX_L2) {
    if (!c->xq) {
      PCEXP_TRY(dalloc(c, &c->xq, c->host.xqphys.size()));
      PCEXP_CK(cudaMemcpyAsync(c->xq, c->host.xqphys.data(), c->host.xqphys.size() * sizeof(double),
                               cudaMemcpyHostToDevice, c->st));
    }
    PCEXP_CK(launch_vortex_error<double>(d, a, c->xq, params, grad ? g : nullptr, &c->ss->dtmin_scratch,
                                         c->partials, &c->ss->counter, c->st));
    if (grad) PCEXP_CK(launch_scale_by_inverse(g, &c->ss->dtmin_scratch, c->Kp, c->st));
  } else {
    PCEXP_CK(cudaMemsetAsync(g, 0, (size_t)c->Kp * sizeof(double), c->st));
    const double ax = kind == PCEXP_FUNC_WALL_FX ? 1.0 : 0.0, ay = kind == PCEXP_FUNC_WALL_FY ? 1.0 : 0.0;
    const double az = kind == PCEXP_FUNC_WALL_FZ ? 1.0 : 0.0;
    PCEXP_CK(launch_wall_force<double>(d, c->host.F_interior, a, ax, ay, az, g, &c->ss->dtmin_scratch, c->partials,
                                       &c->ss->counter, c->st));
  }
  PCEXP_CK(cudaMemcpyAsync(value, &c->ss->dtmin_scratch, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if (grad) PCEXP_TRY(export_vec<double>(c, g, grad, on_device));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

int pcexp_functional_param_grad(pcexp_ctx* c, int kind, const double* params, int n_params, const double* U,
                                double* dJ, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !dJ) return PCEXP_ERR_INVALID_ARG;
  if (kind != PCEXP_FUNC_WALL_FX && kind != PCEXP_FUNC_WALL_FY && kind != PCEXP_FUNC_WALL_FZ &&
      kind != PCEXP_FUNC_VORTEX_L2)
    return PCEXP_ERR_INVALID_ARG;
  if (kind == PCEXP_FUNC_VORTEX_L2 && (!params || n_params < 5)) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) {
    g_last_error = "output functionals are provided for the FP64 form";
    return PCEXP_ERR_UNSUPPORTED;
  }
  dJ[0] = dJ[1] = dJ[2] = 0.0;
  if (kind != PCEXP_FUNC_VORTEX_L2) return PCEXP_OK;  // the wall forces depend on U alone
  double* a = reinterpret_cast<double*>(c->tmp);
  const DGData<double> d = dgdata<double>(c);
  PCEXP_TRY(import_vec<double>(c, U, on_device, a));
  if (!c->xq) {
    PCEXP_TRY(dalloc(c, &c->xq, c->host.xqphys.size()));
    PCEXP_CK(cudaMemcpyAsync(c->xq, c->host.xqphys.data(), c->host.xqphys.size() * sizeof(double),
                             cudaMemcpyHostToDevice, c->st));
  }
  if (!c->pgrad) PCEXP_TRY(dalloc(c, &c->pgrad, 4));
  double dvel[4];
  freestream_velocity_derivatives(c->phys, dvel);
  PCEXP_CK(launch_vortex_param_grad<double>(d, a, c->xq, params, dvel, c->pgrad, c->partials, &c->ss->counter, c->st));
  double out[4];
  PCEXP_CK(cudaMemcpyAsync(out, c->pgrad, sizeof(out), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  const double J = std::sqrt(out[0]);
  if (!(J > 0)) {
    g_last_error = "the vortex error is zero: its gradient is not defined";
    return PCEXP_ERR_NONFINITE;
  }
  for (int k = 0; k < 3; ++k) dJ[k] = -out[1 + k] / J;
  return PCEXP_OK;
}

int pcexp_project_state_adjoint(pcexp_ctx* c, int kind, const double* params, int n_params, const double* ubar0,
                                double* theta_bar, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!ubar0 || !theta_bar || (n_params > 0 && !params)) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) {
    g_last_error = "the projection adjoint is provided for the FP64 form";
    return PCEXP_ERR_UNSUPPORTED;
  }
  double* a = reinterpret_cast<double*>(c->tmp);
  PCEXP_TRY(import_vec<double>(c, ubar0, on_device, a));
  std::vector<double> ub((size_t)c->K);
  PCEXP_CK(cudaMemcpyAsync(ub.data(), a, c->K * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  double tb[3];
  PCEXP_TRY(project_adjoint_host(c, kind, params, n_params, ub, tb));
  theta_bar[0] = tb[0];
  theta_bar[1] = tb[1];
  if (kind == PCEXP_PROJ_VORTEX) theta_bar[2] = tb[2];
  return PCEXP_OK;
}

int pcexp_functional(pcexp_ctx* c, int kind, const double* U, double* value, double* grad, int on_device) {
  if (kind == PCEXP_FUNC_VORTEX_L2) return PCEXP_ERR_INVALID_ARG;  // needs its parameters
  return pcexp_functional_params(c, kind, nullptr, 0, U, value, grad, on_device);
}

int pcexp_set_physics(pcexp_ctx* c, const pcexp_physics* phys) {
  PCEXP_TRY(check_ctx(c));
  if (!phys || !(phys->gamma > 1.0) || !(phys->rho_inf > 0) || !(phys->p_inf > 0)) return PCEXP_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k)
    if (phys->omega[k] != c->phys.omega[k]) {
      g_last_error = "omega is fixed when the context is created (its frame arrays depend on the mesh)";
      return PCEXP_ERR_INVALID_ARG;
    }
  PCEXP_CK(cudaStreamSynchronize(c->st));
  c->phys = *phys;
  // captured steps hold the old free stream in their kernel arguments
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  c->seen_keys.clear();
  return PCEXP_OK;
}

int pcexp_step_backward(pcexp_ctx* c, const double* U, double dt, int m, const double* ubar_next, double* ubar,
                        double* theta_bar, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !ubar_next || !ubar || m < 1 || m > c->m_max || !(dt > 0) || !std::isfinite(dt))
    return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) {
    g_last_error = "the reverse step is provided for the FP64 form";
    return PCEXP_ERR_UNSUPPORTED;
  }
  if (c->rot) return UNSUPPORTED_ROTATING("the reverse step");
  return step_backward_impl(c, U, dt, m, ubar_next, ubar, theta_bar, on_device);
}

int pcexp_phi_adjoint(pcexp_ctx* c, const double* H, int k, int ldh, double dt, const double* ybar, double* Hbar) {
  PCEXP_TRY(check_ctx(c));
  if (!H || !ybar || !Hbar || k < 1 || k > PCEXP_MAX_KRYLOV || ldh < k) return PCEXP_ERR_INVALID_ARG;
  return phi_adjoint_abi(c, H, k, ldh, dt, ybar, Hbar);
}

int pcexp_vjp(pcexp_ctx* c, const double* U, const double* w, double* JTw, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !w || !JTw) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) return vjp_impl<float>(c, U, w, JTw, on_device);
  return vjp_impl<double>(c, U, w, JTw, on_device);
}

int pcexp_compute_dt(pcexp_ctx* c, double cfl, int local, double* dt, int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!dt || !(cfl > 0)) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) {
    float* dte = reinterpret_cast<float*>(c->dte);
    PCEXP_CK(launch_local_dt<float>(dgdata<float>(c), shadow<float>(c, c->cur), nullptr, cfl, dte, &c->ss->dtmin_scratch,
                                     c->partials, &c->ss->counter, c->st));
    if (local) PCEXP_CK(launch_cast<float, double>(dte, c->io64b, c->E, c->st));
  } else {
    double* dte = reinterpret_cast<double*>(c->dte);
    PCEXP_CK(launch_local_dt<double>(dgdata<double>(c), shadow<double>(c, c->cur), nullptr, cfl, dte, &c->ss->dtmin_scratch,
                                      c->partials, &c->ss->counter, c->st));
    if (local) PCEXP_CK(cudaMemcpyAsync(c->io64b, dte, c->E * 8, cudaMemcpyDeviceToDevice, c->st));
  }
  const double* src = local ? c->io64b : &c->ss->dtmin_scratch;
  const size_t n = local ? (size_t)c->E : 1;
  PCEXP_CK(cudaMemcpyAsync(dt, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

int pcexp_arnoldi(pcexp_ctx* c, const double* U, const double* b, int m, double* V, double* H, int* k, double* beta,
                  int on_device) {
  PCEXP_TRY(check_ctx(c));
  if (!U || !b || m < 1 || m > c->m_max) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) return arnoldi_abi<float>(c, U, b, m, V, H, k, beta, on_device);
  return arnoldi_abi<double>(c, U, b, m, V, H, k, beta, on_device);
}

int pcexp_phi(pcexp_ctx* c, const double* H, int k, int ldh, double dt, double* phi1, double* phi2) {
  PCEXP_TRY(check_ctx(c));
  if (!H || !phi1 || k < 1 || k > PCEXP_MAX_KRYLOV || ldh < k) return PCEXP_ERR_INVALID_ARG;
  KState hk;
  std::memset(&hk, 0, sizeof(hk));
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) hk.H[i * MMAX + j] = H[i * ldh + j];
  for (int i = 0; i <= MMAX; ++i) hk.s[i] = 1.0;
  hk.k = k;
  hk.beta = 1.0;
  PCEXP_CK(cudaMemcpyAsync(c->ks, &hk, sizeof(hk), cudaMemcpyHostToDevice, c->st));
  PCEXP_CK(launch_phi(c->ks, nullptr, dt, 1.0, nullptr, 0, c->st));
  PCEXP_CK(cudaMemcpyAsync(&hk, c->ks, sizeof(hk), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  if (hk.err) return PCEXP_ERR_NONFINITE;
  for (int i = 0; i < k; ++i) {
    phi1[i] = hk.y[i];
    if (phi2) phi2[i] = hk.y2[i];
  }
  return PCEXP_OK;
}

int pcexp_step(pcexp_ctx* c, int scheme, int dt_mode, double dt_or_cfl, int m, pcexp_step_info* info) {
  PCEXP_TRY(check_ctx(c));
  if (scheme != PCEXP_SCHEME_PCEXP && scheme != PCEXP_SCHEME_EXP1 && scheme != PCEXP_SCHEME_ETD2)
    return PCEXP_ERR_INVALID_ARG;
  if (dt_mode < PCEXP_DT_GIVEN || dt_mode > PCEXP_DT_LOCAL_CFL) return PCEXP_ERR_INVALID_ARG;
  if (scheme == PCEXP_SCHEME_ETD2 && dt_mode == PCEXP_DT_LOCAL_CFL) {
    g_last_error = "ETD2 is a time-accurate scheme: give dt or a global CFL number";
    return PCEXP_ERR_INVALID_ARG;
  }
  if (m < 1 || m > c->m_max || !(dt_or_cfl > 0) || !std::isfinite(dt_or_cfl)) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) return step_impl<float>(c, scheme, dt_mode, dt_or_cfl, m, info);
  return step_impl<double>(c, scheme, dt_mode, dt_or_cfl, m, info);
}

int pcexp_march_steady(pcexp_ctx* c, int scheme, double cfl_max, double decades, int max_iter, int m,
                       pcexp_steady_info* info) {
  PCEXP_TRY(check_ctx(c));
  if (scheme != PCEXP_SCHEME_PCEXP && scheme != PCEXP_SCHEME_EXP1) return PCEXP_ERR_INVALID_ARG;
  if (m < 1 || m > c->m_max || !(cfl_max > 0) || !(decades > 0) || max_iter < 0) return PCEXP_ERR_INVALID_ARG;
  if (c->fp32) return march_impl<float>(c, scheme, cfl_max, decades, max_iter, m, info);
  return march_impl<double>(c, scheme, cfl_max, decades, max_iter, m, info);
}

int pcexp_output(pcexp_ctx* c, int kind, double* value) {
  PCEXP_TRY(check_ctx(c));
  if (!value) return PCEXP_ERR_INVALID_ARG;
  if (kind != 0 && kind != 1) return PCEXP_ERR_INVALID_ARG;
  if (kind == 1) {
    // entropy error of Eq. entropy_error on the FP64 master state with FP64 tables (an FP32
    // evaluation would lose the small radicand of a near-isentropic flow to rounding)
    const Setup& s = c->host;
    const int GEO = c->dim == 2 ? 8 : 12;
    if (!c->diag) {
      std::vector<double> t(s.Bv);
      t.insert(t.end(), s.Wv.begin(), s.Wv.end());
      for (int64_t e = 0; e < c->E; ++e) t.push_back(s.geo[GEO * e + c->dim * c->dim]);
      PCEXP_TRY(dalloc(c, &c->diag, t.size()));
      PCEXP_CK(cudaMemcpyAsync(c->diag, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    }
    const double g = c->phys.gamma;
    const double s0 = c->phys.p_inf / std::pow(c->phys.rho_inf, g);
    const double* Bv = c->diag;
    const double* Wv = Bv + (size_t)c->nq * c->nb;
    const double* sd = Wv + c->nq;
    PCEXP_CK(launch_entropy_sum(c->U64[c->cur], Bv, Wv, sd, c->E, c->nb, c->nq, c->nv, g, s0,
                                &c->ss->dtmin_scratch, c->partials, &c->ss->counter, c->st));
    double sum = 0;
    PCEXP_CK(cudaMemcpyAsync(&sum, &c->ss->dtmin_scratch, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    PCEXP_CK(cudaStreamSynchronize(c->st));
    if (!std::isfinite(sum)) {
      g_last_error = "non-finite entropy integral";
      return PCEXP_ERR_NONFINITE;
    }
    *value = std::sqrt(std::max(sum / c->volume - 1.0, 0.0));
    return PCEXP_OK;
  }
  if (c->fp32) {
    float* V = reinterpret_cast<float*>(c->V);
    PCEXP_CK(launch_dg_operator<float>(dgdata<float>(c), shadow<float>(c, c->cur), nullptr, V, reinterpret_cast<float*>(c->G),
                                        nullptr, nullptr, c->st));
    PCEXP_CK(launch_density_norm<float>(V, nullptr, c->E, c->nb, c->nv, c->volume, c->ss, c->partials, 0, c->p, 0.0, c->st));
  } else {
    double* V = reinterpret_cast<double*>(c->V);
    PCEXP_CK(launch_dg_operator<double>(dgdata<double>(c), shadow<double>(c, c->cur), nullptr, V, reinterpret_cast<double*>(c->G),
                                         nullptr, nullptr, c->st));
    PCEXP_CK(launch_density_norm<double>(V, nullptr, c->E, c->nb, c->nv, c->volume, c->ss, c->partials, 0, c->p, 0.0, c->st));
  }
  StepState h;
  PCEXP_CK(cudaMemcpyAsync(&h, c->ss, sizeof(h), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  *value = h.res_norm;
  return PCEXP_OK;
}

int pcexp_profile_enable(pcexp_ctx* c, int enable) {
  PCEXP_TRY(check_ctx(c));
  PCEXP_TRY(prof_flush(c));
  for (int i = 0; i < PCEXP_KC_COUNT; ++i) {
    c->prof_ms[i] = 0;
    c->prof_n[i] = 0;
  }
  c->prof = enable != 0;
  return PCEXP_OK;
}

int pcexp_profile_read(pcexp_ctx* c, int kernel_class, int64_t* launches, double* ms) {
  PCEXP_TRY(check_ctx(c));
  if (kernel_class < 0 || kernel_class >= PCEXP_KC_COUNT) return PCEXP_ERR_INVALID_ARG;
  PCEXP_TRY(prof_flush(c));
  if (launches) *launches = c->prof_n[kernel_class];
  if (ms) *ms = c->prof_ms[kernel_class];
  return PCEXP_OK;
}

int pcexp_synchronize(pcexp_ctx* c) {
  PCEXP_TRY(check_ctx(c));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

int pcexp_fp64_fma_rate(double* tflops) {
  if (!tflops) return PCEXP_ERR_INVALID_ARG;
  PCEXP_CK(measure_fp64_fma_rate(tflops));
  return PCEXP_OK;
}

int pcexp_fp32_fma_rate(double* tflops) {
  if (!tflops) return PCEXP_ERR_INVALID_ARG;
  PCEXP_CK(measure_fp32_fma_rate(tflops));
  return PCEXP_OK;
}

const char* pcexp_last_error(void) { return g_last_error.c_str(); }

const char* pcexp_status_string(int status) {
  switch (status) {
    case PCEXP_OK: return "ok";
    case PCEXP_ERR_INVALID_ARG: return "invalid argument";
    case PCEXP_ERR_MESH: return "invalid mesh";
    case PCEXP_ERR_CUDA: return "CUDA error";
    case PCEXP_ERR_OOM: return "out of device memory";
    case PCEXP_ERR_NONFINITE: return "non-finite value";
    case PCEXP_ERR_TIMEOUT: return "wait timed out (partition rendezvous)";
    case PCEXP_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

}  // extern "C"

// ================================================================ partitioned runs
namespace {

int check_opts(const pcexp_physics* phys, const pcexp_options* opt) {
  if (opt->m_max < 1 || opt->m_max > PCEXP_MAX_KRYLOV) return PCEXP_ERR_INVALID_ARG;
  if (opt->precision != PCEXP_FP64 && opt->precision != PCEXP_FP32_MIXED) return PCEXP_ERR_INVALID_ARG;
  if (opt->basis_io != PCEXP_BASIS_PAPER && opt->basis_io != PCEXP_BASIS_INTERNAL) return PCEXP_ERR_INVALID_ARG;
  if (!(phys->gamma > 1.0) || !(phys->rho_inf > 0) || !(phys->p_inf > 0)) return PCEXP_ERR_INVALID_ARG;
  return check_reorth(opt);
}

// Runs fn(k) for every partition, each on a host thread of its own with its device current.
// The first failure that is not another partition's failure seen at a rendezvous is reported.
template <class F>
int group_run(pcexp_group* g, F&& fn) {
  {
    std::lock_guard<std::mutex> lk(g->mu);
    g->abort = false;
    g->arrived = 0;
  }
  std::vector<int> rc((size_t)g->n, PCEXP_OK);
  std::vector<std::string> err((size_t)g->n);
  auto body = [&](int k) {
    if (cudaSetDevice(g->dev[(size_t)k]) != cudaSuccess) {
      rc[(size_t)k] = PCEXP_ERR_CUDA;
      err[(size_t)k] = "cudaSetDevice failed";
    } else {
      rc[(size_t)k] = fn(k);
      if (rc[(size_t)k] != PCEXP_OK) err[(size_t)k] = g_last_error;
    }
    if (rc[(size_t)k] != PCEXP_OK) {
      std::lock_guard<std::mutex> lk(g->mu);
      g->abort = true;
      g->cv.notify_all();
    }
  };
  if (g->n == 1) {
    body(0);
  } else {
    std::vector<std::thread> th;
    for (int k = 0; k < g->n; ++k) th.emplace_back(body, k);
    for (auto& t : th) t.join();
  }
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 0; k < g->n; ++k)
      if (rc[(size_t)k] != PCEXP_OK && (pass == 1 || rc[(size_t)k] != PCEXP_ERR_TIMEOUT)) {
        g_last_error = "partition " + std::to_string(k) + ": " + err[(size_t)k];
        return rc[(size_t)k];
      }
  return PCEXP_OK;
}

// restores the calling thread's current device when a group call returns (the per-partition
// calls it makes switch to each partition's device)
struct DeviceGuard {
  int dev = 0;
  DeviceGuard() { cudaGetDevice(&dev); }
  ~DeviceGuard() { cudaSetDevice(dev); }
};

int check_group(pcexp_group* g) {
  if (!g) {
    g_last_error = "null group";
    return PCEXP_ERR_INVALID_ARG;
  }
  return PCEXP_OK;
}

// local vector of partition k (its elements' rows of a global state-shaped host array); halo rows
// are left zero when `halo` is false
void gather_local(const pcexp_group* g, int k, const double* U, std::vector<double>& loc, bool halo) {
  const int64_t nvb = (int64_t)g->nv * g->nb;
  const auto& el = g->elems[(size_t)k];
  const int64_t n = halo ? (int64_t)el.size() : g->ctx[(size_t)k]->n_local;
  loc.assign(el.size() * (size_t)nvb, 0.0);
  for (int64_t e = 0; e < n; ++e) std::memcpy(&loc[(size_t)(e * nvb)], U + el[(size_t)e] * nvb, (size_t)nvb * 8);
}

void scatter_owned(const pcexp_group* g, int k, const std::vector<double>& loc, double* U) {
  const int64_t nvb = (int64_t)g->nv * g->nb;
  const auto& el = g->elems[(size_t)k];
  for (int64_t e = 0; e < g->ctx[(size_t)k]->n_local; ++e)
    std::memcpy(U + el[(size_t)e] * nvb, &loc[(size_t)(e * nvb)], (size_t)nvb * 8);
}

// R (and J v with v) of a partition whose inputs carry only their own rows: the halo rows come
// from the exchange of the operator passes
template <class T>
int group_operator_part(pcexp_ctx* c, const std::vector<double>& u, const std::vector<double>* v, std::vector<double>& out) {
  const DGData<T> d = dgdata<T>(c);
  T* a = reinterpret_cast<T*>(c->tmp);
  T* b = reinterpret_cast<T*>(c->delta);
  T* o = reinterpret_cast<T*>(c->w);
  PCEXP_TRY(import_vec<T>(c, u.data(), 0, a));
  if (!v) {
    PCEXP_TRY(dg_apply<T>(c, d, a, nullptr, o, nullptr, nullptr));
  } else {
    PCEXP_TRY(import_vec<T>(c, v->data(), 0, b));
    PCEXP_TRY(group_exchange<T>(c, a));
    PCEXP_TRY(linearize<T>(c, d, a));
    PCEXP_TRY(jac_apply<T>(c, d, b, o, nullptr, nullptr, nullptr));
  }
  out.assign((size_t)c->K, 0.0);
  return export_vec<T>(c, o, out.data(), 0);
}

// J(U)^T w (adj = 1) or (d(J(U) v)/dU)^T w (adj = 2) of a partition whose inputs carry only
// their own rows: the halo rows of U, v and w come from the exchange (the transposed face terms
// of an own element need w on the neighbouring halo element), the output keeps its own rows
template <class T>
int group_adjoint_part(pcexp_ctx* c, int adj, const std::vector<double>& u, const std::vector<double>* v,
                       const std::vector<double>& w, std::vector<double>& out) {
  const DGData<T> d = dgdata<T>(c);
  T* a = reinterpret_cast<T*>(c->tmp);
  T* b = reinterpret_cast<T*>(c->delta);
  T* ww = reinterpret_cast<T*>(c->V);  // V[0] as scratch
  T* o = reinterpret_cast<T*>(c->w);
  PCEXP_TRY(import_vec<T>(c, u.data(), 0, a));
  PCEXP_TRY(import_vec<T>(c, w.data(), 0, ww));
  PCEXP_TRY(group_exchange<T>(c, a));
  PCEXP_TRY(group_exchange<T>(c, ww));
  if (adj == 1) {
    PCEXP_TRY(linearize<T>(c, d, a, true));
    PCEXP_CK(launch_jac_adjoint<T>(d, lindata<T>(c), ww, o, reinterpret_cast<T*>(c->GT), nullptr, T(1), c->st));
  } else {
    if constexpr (std::is_same<T, double>::value) {
      PCEXP_TRY(import_vec<T>(c, v->data(), 0, b));
      PCEXP_TRY(group_exchange<T>(c, b));
      PCEXP_CK(launch_jvp_state_adjoint<double>(d, a, b, ww, o, reinterpret_cast<double*>(c->GT), nullptr, 1.0, c->st));
    } else {
      return UNSUPPORTED_FP32_HESS(c);
    }
  }
  PCEXP_TRY(group_zero_halo<T>(c, o));
  out.assign((size_t)c->K, 0.0);
  return export_vec<T>(c, o, out.data(), 0);
}

template <class T>
int group_arnoldi_part(pcexp_ctx* c, const std::vector<double>& u, const std::vector<double>& b, int m, KState* hk) {
  const DGData<T> d = dgdata<T>(c);
  T* lin = reinterpret_cast<T*>(c->delta);
  PCEXP_TRY(import_vec<T>(c, u.data(), 0, lin));
  PCEXP_TRY(import_vec<T>(c, b.data(), 0, Vcol<T>(c, 0)));
  PCEXP_TRY(group_exchange<T>(c, lin));
  PCEXP_TRY(linearize<T>(c, d, lin));
  PCEXP_TRY(arnoldi<T>(c, nullptr, m, nullptr));
  PCEXP_CK(cudaMemcpyAsync(hk, c->ks, sizeof(KState), cudaMemcpyDeviceToHost, c->st));
  PCEXP_CK(cudaStreamSynchronize(c->st));
  return PCEXP_OK;
}

}  // namespace

extern "C" {

int pcexp_partition(const pcexp_mesh* mesh, int n_parts, int32_t* part) {
  if (!mesh || !part || n_parts < 1 || n_parts > MAX_PARTS || mesh->n_elem < n_parts ||
      (mesh->dim != 2 && mesh->dim != 3)) {
    g_last_error = "invalid partition request";
    return PCEXP_ERR_INVALID_ARG;
  }
  rcb_partition(*mesh, n_parts, part);
  return PCEXP_OK;
}

int pcexp_partition_halo(const pcexp_mesh* mesh, const int32_t* part, int n_parts, int k, int64_t* n_owned,
                         int64_t* n_total, int64_t* elems) {
  if (!mesh || !part || n_parts < 1 || k < 0 || k >= n_parts || !n_owned || !n_total) return PCEXP_ERR_INVALID_ARG;
  for (int64_t e = 0; e < mesh->n_elem; ++e)
    if (part[e] < 0 || part[e] >= n_parts) {
      g_last_error = "partition index out of range";
      return PCEXP_ERR_INVALID_ARG;
    }
  std::vector<int64_t> nbr;
  std::string msg;
  int r = face_neighbours(*mesh, nbr, msg);
  if (r != PCEXP_OK) {
    g_last_error = msg;
    return r;
  }
  Halo h;
  build_halo(*mesh, nbr, part, k, h);
  *n_owned = h.n_owned;
  *n_total = (int64_t)h.elems.size();
  if (elems) std::memcpy(elems, h.elems.data(), h.elems.size() * sizeof(int64_t));
  return PCEXP_OK;
}

int pcexp_group_destroy(pcexp_group* g) {
  if (!g) return PCEXP_OK;
  for (int k = 0; k < g->n; ++k) {
    cudaSetDevice(g->dev[(size_t)k]);
    if (k < (int)g->ctx.size() && g->ctx[(size_t)k]) pcexp_destroy(g->ctx[(size_t)k]);
    if (k < (int)g->ev_ready.size() && g->ev_ready[(size_t)k]) cudaEventDestroy(g->ev_ready[(size_t)k]);
    if (k < (int)g->ev_done.size() && g->ev_done[(size_t)k]) cudaEventDestroy(g->ev_done[(size_t)k]);
    if (k < (int)g->st.size() && g->st[(size_t)k]) cudaStreamDestroy(g->st[(size_t)k]);
  }
  delete g;
  return PCEXP_OK;
}

int pcexp_group_create(pcexp_group** out, const pcexp_mesh* mesh, const int32_t* part, int n_parts,
                       const int32_t* devices, int p, const pcexp_physics* phys, const pcexp_options* opt) {
  if (!out) return PCEXP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !part || !phys || !opt || n_parts < 1 || n_parts > MAX_PARTS) return PCEXP_ERR_INVALID_ARG;
  PCEXP_TRY(check_opts(phys, opt));
  std::vector<int64_t> count((size_t)n_parts, 0);
  for (int64_t e = 0; e < mesh->n_elem; ++e) {
    if (part[e] < 0 || part[e] >= n_parts) {
      g_last_error = "partition index out of range";
      return PCEXP_ERR_INVALID_ARG;
    }
    ++count[(size_t)part[e]];
  }
  for (int64_t c : count)
    if (c == 0) {
      g_last_error = "empty partition";
      return PCEXP_ERR_INVALID_ARG;
    }
  int dev0 = 0;
  cudaGetDevice(&dev0);
  std::vector<int64_t> nbr;
  std::string msg;
  int r = face_neighbours(*mesh, nbr, msg);
  if (r != PCEXP_OK) {
    g_last_error = msg;
    return r;
  }
  pcexp_group* g = new pcexp_group();
  g->n = n_parts;
  g->E = mesh->n_elem;
  g->ctx.assign((size_t)n_parts, nullptr);
  g->st.assign((size_t)n_parts, nullptr);
  g->ev_ready.assign((size_t)n_parts, nullptr);
  g->ev_done.assign((size_t)n_parts, nullptr);
  g->pub.assign((size_t)n_parts, nullptr);
  g->hostval.assign((size_t)n_parts, 0.0);
  g->elems.resize((size_t)n_parts);
  g->own_volume.assign((size_t)n_parts, 0.0);
  g->fp32 = opt->precision == PCEXP_FP32_MIXED;
  for (int k = 0; k < n_parts; ++k) g->dev.push_back(devices ? devices[k] : dev0);
  auto fail = [&](int code) {
    const std::string keep = g_last_error;
    pcexp_group_destroy(g);
    cudaSetDevice(dev0);
    g_last_error = keep;
    return code;
  };
  std::vector<int64_t> n_owned((size_t)n_parts);
  for (int k = 0; k < n_parts; ++k) {
    Halo h;
    build_halo(*mesh, nbr, part, k, h);
    Submesh sm;
    if ((r = build_submesh(*mesh, h, sm, msg)) != PCEXP_OK) {
      g_last_error = msg;
      return fail(r);
    }
    if (cudaSetDevice(g->dev[(size_t)k]) != cudaSuccess ||
        cudaStreamCreateWithFlags(&g->st[(size_t)k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_ready[(size_t)k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_done[(size_t)k], cudaEventDisableTiming) != cudaSuccess) {
      g_last_error = "stream or event creation failed on the partition's device";
      return fail(PCEXP_ERR_CUDA);
    }
    pcexp_ctx* c = new pcexp_ctx();
    g->ctx[(size_t)k] = c;
    c->device = g->dev[(size_t)k];
    c->st = g->st[(size_t)k];
    const pcexp_mesh mv = sm.view();
    if ((r = create_impl(c, &mv, p, phys, opt, h.elems.data())) != PCEXP_OK) return fail(r);
    c->grp = g;
    c->part = k;
    c->n_local = h.n_owned;
    c->n_ghost = (int64_t)h.elems.size() - h.n_owned;
    // own measure: sqrt|det A| is entry D^2 of an element's geometry row; |E| = |det A| / D!
    const int D = c->dim, G = D == 2 ? 8 : 12;
    for (int64_t e = 0; e < h.n_owned; ++e) {
      const double sd = c->host.geo[(size_t)(e * G + D * D)];
      g->own_volume[(size_t)k] += sd * sd / (D == 2 ? 2.0 : 6.0);
    }
    g->nb = c->nb;
    g->nv = c->nv;
    n_owned[(size_t)k] = h.n_owned;
    g->elems[(size_t)k] = std::move(h.elems);
  }
  for (double v : g->own_volume) g->volume += v;
  // halo maps: owning partition and its local index of every halo element
  for (int k = 0; k < n_parts; ++k) {
    pcexp_ctx* c = g->ctx[(size_t)k];
    cudaSetDevice(c->device);
    const auto& el = g->elems[(size_t)k];
    std::vector<int32_t> sp((size_t)c->n_ghost + 1, 0), se((size_t)c->n_ghost + 1, 0);
    for (int64_t i = 0; i < c->n_ghost; ++i) {
      const int64_t ge = el[(size_t)(c->n_local + i)];
      const int q = part[ge];
      const auto& eq = g->elems[(size_t)q];
      const auto it = std::lower_bound(eq.begin(), eq.begin() + n_owned[(size_t)q], ge);
      sp[(size_t)i] = q;
      se[(size_t)i] = (int32_t)(it - eq.begin());
    }
    if (dalloc(c, &c->g_src_part, sp.size()) != PCEXP_OK || dalloc(c, &c->g_src_elem, se.size()) != PCEXP_OK)
      return fail(PCEXP_ERR_OOM);
    const int group_flag = 1;
    if (cudaMemcpyAsync(c->g_src_part, sp.data(), sp.size() * 4, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->g_src_elem, se.data(), se.size() * 4, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(reinterpret_cast<char*>(c->ks) + offsetof(KState, group), &group_flag, sizeof(int),
                        cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
      g_last_error = "upload of the halo maps failed";
      return fail(PCEXP_ERR_CUDA);
    }
    // the halo gather reads the other partitions' buffers directly
    for (int q = 0; q < n_parts; ++q) {
      const int dq = g->dev[(size_t)q];
      if (dq == c->device) continue;
      int can = 0;
      cudaDeviceCanAccessPeer(&can, c->device, dq);
      if (!can) {
        g_last_error = "partitions on devices without peer access";
        return fail(PCEXP_ERR_UNSUPPORTED);
      }
      const cudaError_t pe = cudaDeviceEnablePeerAccess(dq, 0);
      if (pe != cudaSuccess && pe != cudaErrorPeerAccessAlreadyEnabled) {
        g_last_error = std::string("cudaDeviceEnablePeerAccess: ") + cudaGetErrorString(pe);
        return fail(PCEXP_ERR_CUDA);
      }
      cudaGetLastError();  // clear an already-enabled status
    }
  }
  cudaSetDevice(dev0);
  *out = g;
  return PCEXP_OK;
}

int pcexp_group_sizes(const pcexp_group* g, int k, int64_t* n_owned, int64_t* n_halo) {
  if (!g || k < 0 || k >= g->n) return PCEXP_ERR_INVALID_ARG;
  if (n_owned) *n_owned = g->ctx[(size_t)k]->n_local;
  if (n_halo) *n_halo = g->ctx[(size_t)k]->n_ghost;
  return PCEXP_OK;
}

int pcexp_group_set_state(pcexp_group* g, const double* U) {
  PCEXP_TRY(check_group(g));
  if (!U) return PCEXP_ERR_INVALID_ARG;
  DeviceGuard keep;
  std::vector<double> loc;
  for (int k = 0; k < g->n; ++k) {
    gather_local(g, k, U, loc, true);
    const int r = pcexp_set_state(g->ctx[(size_t)k], loc.data(), 0);
    if (r != PCEXP_OK) return r;
  }
  return PCEXP_OK;
}

int pcexp_group_get_state(pcexp_group* g, double* U) {
  PCEXP_TRY(check_group(g));
  if (!U) return PCEXP_ERR_INVALID_ARG;
  DeviceGuard keep;
  std::vector<double> loc;
  for (int k = 0; k < g->n; ++k) {
    loc.assign((size_t)g->ctx[(size_t)k]->K, 0.0);
    const int r = pcexp_get_state(g->ctx[(size_t)k], loc.data(), 0);
    if (r != PCEXP_OK) return r;
    scatter_owned(g, k, loc, U);
  }
  return PCEXP_OK;
}

int pcexp_group_project_state(pcexp_group* g, int kind, const double* params, int n_params) {
  PCEXP_TRY(check_group(g));
  DeviceGuard keep;
  for (int k = 0; k < g->n; ++k) {
    const int r = pcexp_project_state(g->ctx[(size_t)k], kind, params, n_params);
    if (r != PCEXP_OK) return r;
  }
  return PCEXP_OK;
}

static int group_operator(pcexp_group* g, const double* U, const double* v, double* out) {
  PCEXP_TRY(check_group(g));
  if (!U || !out) return PCEXP_ERR_INVALID_ARG;
  std::vector<std::vector<double>> res((size_t)g->n);
  PCEXP_TRY(group_run(g, [&](int k) -> int {
    pcexp_ctx* c = g->ctx[(size_t)k];
    std::vector<double> u, dv;
    gather_local(g, k, U, u, false);
    if (v) gather_local(g, k, v, dv, false);
    return c->fp32 ? group_operator_part<float>(c, u, v ? &dv : nullptr, res[(size_t)k])
                   : group_operator_part<double>(c, u, v ? &dv : nullptr, res[(size_t)k]);
  }));
  for (int k = 0; k < g->n; ++k) scatter_owned(g, k, res[(size_t)k], out);
  return PCEXP_OK;
}

int pcexp_group_residual(pcexp_group* g, const double* U, double* R) { return group_operator(g, U, nullptr, R); }

static int group_adjoint(pcexp_group* g, int adj, const double* U, const double* v, const double* w, double* out) {
  PCEXP_TRY(check_group(g));
  if (!U || !w || !out || (adj == 2 && !v)) return PCEXP_ERR_INVALID_ARG;
  if (adj == 2 && g->fp32) {
    g_last_error = "the second-order adjoint is provided for the FP64 form";
    return PCEXP_ERR_UNSUPPORTED;
  }
  if (adj == 2 && g->ctx[0]->rot) {
    g_last_error = "the second-order adjoint is not provided in a rotating frame";
    return PCEXP_ERR_UNSUPPORTED;
  }
  std::vector<std::vector<double>> res((size_t)g->n);
  PCEXP_TRY(group_run(g, [&](int k) -> int {
    pcexp_ctx* c = g->ctx[(size_t)k];
    std::vector<double> uu, vv, wl;
    gather_local(g, k, U, uu, false);
    gather_local(g, k, w, wl, false);
    if (v) gather_local(g, k, v, vv, false);
    return c->fp32 ? group_adjoint_part<float>(c, adj, uu, v ? &vv : nullptr, wl, res[(size_t)k])
                   : group_adjoint_part<double>(c, adj, uu, v ? &vv : nullptr, wl, res[(size_t)k]);
  }));
  for (int k = 0; k < g->n; ++k) scatter_owned(g, k, res[(size_t)k], out);
  return PCEXP_OK;
}

int pcexp_group_vjp(pcexp_group* g, const double* U, const double* w, double* JTw) {
  return group_adjoint(g, 1, U, nullptr, w, JTw);
}

int pcexp_group_jvp_state_adjoint(pcexp_group* g, const double* U, const double* v, const double* w, double* out) {
  return group_adjoint(g, 2, U, v, w, out);
}

int pcexp_group_jvp(pcexp_group* g, const double* U, const double* v, double* Jv) {
  if (!v) return PCEXP_ERR_INVALID_ARG;
  return group_operator(g, U, v, Jv);
}

int pcexp_group_arnoldi(pcexp_group* g, const double* U, const double* b, int m, double* H, int* k, double* beta) {
  PCEXP_TRY(check_group(g));
  if (!U || !b || m < 1 || m > g->ctx[0]->m_max) return PCEXP_ERR_INVALID_ARG;
  std::vector<KState> hk((size_t)g->n);
  PCEXP_TRY(group_run(g, [&](int q) -> int {
    pcexp_ctx* c = g->ctx[(size_t)q];
    std::vector<double> u, bb;
    gather_local(g, q, U, u, false);
    gather_local(g, q, b, bb, false);
    return c->fp32 ? group_arnoldi_part<float>(c, u, bb, m, &hk[(size_t)q])
                   : group_arnoldi_part<double>(c, u, bb, m, &hk[(size_t)q]);
  }));
  for (int q = 1; q < g->n; ++q)
    if (hk[(size_t)q].k != hk[0].k ||
        std::memcmp(hk[(size_t)q].H, hk[0].H, sizeof(double) * (MMAX + 1) * MMAX) != 0) {
      g_last_error = "partitions disagree on the Hessenberg matrix";
      return PCEXP_ERR_CUDA;
    }
  if (hk[0].err) {
    g_last_error = "non-finite Arnoldi quantity";
    return PCEXP_ERR_NONFINITE;
  }
  const int kk = hk[0].k;
  if (k) *k = kk;
  if (beta) *beta = hk[0].beta;
  if (H)
    for (int i = 0; i <= m; ++i)
      for (int j = 0; j < m; ++j) H[i * m + j] = (i <= kk && j < kk) ? hk[0].H[i * MMAX + j] : 0.0;
  return PCEXP_OK;
}

int pcexp_group_step_backward(pcexp_group* g, const double* U, double dt, int m, const double* ubar_next,
                              double* ubar, double* theta_bar) {
  PCEXP_TRY(check_group(g));
  if (!U || !ubar_next || !ubar || m < 1 || m > g->ctx[0]->m_max || !(dt > 0) || !std::isfinite(dt))
    return PCEXP_ERR_INVALID_ARG;
  if (g->fp32) {
    g_last_error = "the reverse step is provided for the FP64 form";
    return PCEXP_ERR_UNSUPPORTED;
  }
  if (g->ctx[0]->rot) {
    g_last_error = "the reverse step is not provided in a rotating frame";
    return PCEXP_ERR_UNSUPPORTED;
  }
  std::vector<std::vector<double>> res((size_t)g->n);
  std::vector<std::array<double, 2>> th((size_t)g->n, std::array<double, 2>{0.0, 0.0});
  PCEXP_TRY(group_run(g, [&](int k) -> int {
    pcexp_ctx* c = g->ctx[(size_t)k];
    std::vector<double> u, ub;
    gather_local(g, k, U, u, false);
    gather_local(g, k, ubar_next, ub, false);
    res[(size_t)k].assign((size_t)c->K, 0.0);
    return step_backward_impl(c, u.data(), dt, m, ub.data(), res[(size_t)k].data(), th[(size_t)k].data(), 0);
  }));
  for (int k = 0; k < g->n; ++k) scatter_owned(g, k, res[(size_t)k], ubar);
  if (theta_bar) {  // each partition's sums cover the boundary faces of its own elements
    theta_bar[0] = theta_bar[1] = 0.0;
    for (int k = 0; k < g->n; ++k) {
      theta_bar[0] += th[(size_t)k][0];
      theta_bar[1] += th[(size_t)k][1];
    }
  }
  return PCEXP_OK;
}

int pcexp_group_march_steady(pcexp_group* g, int scheme, double cfl_max, double decades, int max_iter, int m,
                             pcexp_steady_info* info) {
  PCEXP_TRY(check_group(g));
  if (scheme != PCEXP_SCHEME_PCEXP && scheme != PCEXP_SCHEME_EXP1) return PCEXP_ERR_INVALID_ARG;
  if (m < 1 || m > g->ctx[0]->m_max || !(cfl_max > 0) || !(decades > 0) || max_iter < 0) return PCEXP_ERR_INVALID_ARG;
  std::vector<pcexp_steady_info> inf((size_t)g->n);
  PCEXP_TRY(group_run(g, [&](int k) -> int {
    pcexp_ctx* c = g->ctx[(size_t)k];
    return c->fp32 ? march_impl<float>(c, scheme, cfl_max, decades, max_iter, m, &inf[(size_t)k])
                   : march_impl<double>(c, scheme, cfl_max, decades, max_iter, m, &inf[(size_t)k]);
  }));
  if (info) *info = inf[0];  // every partition took the same decisions from the same norms
  return PCEXP_OK;
}

int pcexp_group_step(pcexp_group* g, int scheme, int dt_mode, double dt_or_cfl, int m, pcexp_step_info* info) {
  PCEXP_TRY(check_group(g));
  if (scheme != PCEXP_SCHEME_PCEXP && scheme != PCEXP_SCHEME_EXP1 && scheme != PCEXP_SCHEME_ETD2)
    return PCEXP_ERR_INVALID_ARG;
  if (dt_mode < PCEXP_DT_GIVEN || dt_mode > PCEXP_DT_LOCAL_CFL) return PCEXP_ERR_INVALID_ARG;
  if (scheme == PCEXP_SCHEME_ETD2 && dt_mode == PCEXP_DT_LOCAL_CFL) {
    g_last_error = "ETD2 is a time-accurate scheme: give dt or a global CFL number";
    return PCEXP_ERR_INVALID_ARG;
  }
  if (m < 1 || m > g->ctx[0]->m_max || !(dt_or_cfl > 0)) return PCEXP_ERR_INVALID_ARG;
  std::vector<pcexp_step_info> inf((size_t)g->n);
  PCEXP_TRY(group_run(g, [&](int k) -> int {
    pcexp_ctx* c = g->ctx[(size_t)k];
    return c->fp32 ? step_impl<float>(c, scheme, dt_mode, dt_or_cfl, m, &inf[(size_t)k])
                   : step_impl<double>(c, scheme, dt_mode, dt_or_cfl, m, &inf[(size_t)k]);
  }));
  if (info) {
    *info = inf[0];
    // each partition's norm is (its sum of squares)^(1/2) / its measure (own and halo elements)
    double s2 = 0;
    for (int k = 0; k < g->n; ++k) {
      const double a = inf[(size_t)k].res_norm * g->ctx[(size_t)k]->volume;
      s2 += a * a;
    }
    info->res_norm = std::sqrt(s2) / g->volume;
  }
  return PCEXP_OK;
}

}  // extern "C"
