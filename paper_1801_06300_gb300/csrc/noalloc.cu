// pcexp_residual_noalloc: R(U) without any device allocation.
//
// Some callers cannot allocate device memory at the time they need R(U): code
// running inside CUDA stream capture (where cudaMalloc is not allowed), hosts
// with a pre-reserved memory budget or a custom allocator that must not be
// bypassed, and real-time loops that forbid allocator calls after set-up.  For
// them this entry point keeps the one scratch buffer the DG operator needs --
// the face-flux buffer written by the face kernel and read by the element
// kernel -- in a fixed file-scope device array instead of a context buffer.
//
// Limits and sharing:
//   * the array holds NOALLOC_FACE_FLUX_DOUBLES doubles (8 MiB); meshes whose
//     face-flux buffer (faces x (p+1) points x 4 variables) is larger are
//     rejected with PCEXP_ERR_INVALID_ARG;
//   * every GPU that loads the library holds the array until the process exits;
//   * all calls share it: calls whose kernels overlap on the GPU (different
//     streams, or different contexts without ordering) race on it.  Calls on
//     one stream are ordered and safe.  The face kernel writes every entry the
//     element kernel reads, so nothing needs clearing between calls.
#include <mutex>

#include "kernels.h"

namespace pcexp {
// host access to the context internals (api.cu)
int ctx_noalloc_view(pcexp_ctx* c, DGData<double>* d, cudaStream_t* st, int* nfq, int* fp32, int* device);
}  // namespace pcexp

namespace {

constexpr long long NOALLOC_FACE_FLUX_DOUBLES = 1LL << 20;  // 8 MiB
static __device__ __align__(256) double g_noalloc_face_flux[NOALLOC_FACE_FLUX_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch[MAX_DEVICES] = {};  // device address of the array, per device

// Host code must not pass &g_noalloc_face_flux to a kernel (that names a
// host-side stand-in): the device address is looked up once per device with
// that device current.
int scratch_address(int device, double** out) {
  if (device < 0 || device >= MAX_DEVICES) return PCEXP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[device]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_face_flux);
    if (e != cudaSuccess || !p) return PCEXP_ERR_CUDA;
    g_scratch[device] = p;
  }
  *out = g_scratch[device];
  return PCEXP_OK;
}

}  // namespace

extern "C" int pcexp_residual_noalloc(pcexp_ctx* ctx, const double* U, double* R) {
  using namespace pcexp;
  if (!ctx || !U || !R) return PCEXP_ERR_INVALID_ARG;
  DGData<double> d;
  cudaStream_t st = nullptr;
  int nfq = 0, fp32 = 0, device = 0;
  int r = ctx_noalloc_view(ctx, &d, &st, &nfq, &fp32, &device);
  if (r != PCEXP_OK) return r;
  if (fp32) return PCEXP_ERR_UNSUPPORTED;
  if (d.F * nfq * (d.dim + 2) > NOALLOC_FACE_FLUX_DOUBLES) return PCEXP_ERR_INVALID_ARG;
  double* G = nullptr;
  r = scratch_address(device, &G);
  if (r != PCEXP_OK) return r;
  cudaError_t e = launch_dg_operator<double>(d, U, nullptr, R, G, nullptr, nullptr, st);
  return e == cudaSuccess ? PCEXP_OK : PCEXP_ERR_CUDA;
}
