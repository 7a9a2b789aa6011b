// pcexp_residual_noalloc: R(U) without any device allocation.
//
// Some callers cannot allocate device memory at the time they need R(U): hosts that
// hand all device memory to their own pool or caching allocator and forbid other
// allocations, hosts with a fixed memory budget reserved at start-up, and real-time loops
// that may not call cudaMalloc/cudaFree (which can synchronise the device) once set up.
// For them this entry point keeps the one scratch buffer the DG operator needs -- the
// face-flux buffer written by the face kernel and read by the element kernel -- in a fixed
// file-scope device array instead of a context buffer.
//
// Limits and sharing:
//   * the array holds NOALLOC_FACE_FLUX_DOUBLES = 2^20 doubles (8 MiB); meshes whose
//     face-flux buffer (faces x face quadrature points x (dim + 2) variables) is larger
//     are rejected with PCEXP_ERR_INVALID_ARG;
//   * every GPU that loads the library holds the array until the process exits;
//   * all calls share it: calls whose kernels overlap on the GPU (different streams, or
//     different contexts without ordering) race on it.  Calls on one stream are ordered
//     and safe.  The face kernel writes every entry the element kernel reads, so nothing
//     needs clearing between calls, and the last call's contents stay in the array.
#include <mutex>
#include <string>

#include "kernels.h"

namespace pcexp {
// host access to the context internals (api.cu): makes the context's device current
int ctx_noalloc_view(pcexp_ctx* c, DGData<double>* d, cudaStream_t* st, int* nfq, int* fp32, int* device);
void set_last_error(const char* msg);
}  // namespace pcexp

namespace {

constexpr long long NOALLOC_FACE_FLUX_DOUBLES = 1LL << 20;  // 8 MiB
static __device__ __align__(256) double g_noalloc_face_flux[NOALLOC_FACE_FLUX_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch[MAX_DEVICES] = {};  // device address of the array, per device

// Host code must not pass &g_noalloc_face_flux to a kernel (in host code that names a
// host-side stand-in, not device memory).  The device address is looked up once per
// device, with that device made current here, and cached.
int scratch_address(int device, double** out) {
  if (device < 0 || device >= MAX_DEVICES) {
    pcexp::set_last_error("pcexp_residual_noalloc: device index beyond the 64 the library tracks");
    return PCEXP_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[device]) {
    cudaError_t e = cudaSetDevice(device);
    double* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_face_flux);
    if (e != cudaSuccess || !p) {
      const std::string m = std::string("pcexp_residual_noalloc: cudaGetSymbolAddress of the scratch array: ") +
                            cudaGetErrorString(e);
      pcexp::set_last_error(m.c_str());
      return PCEXP_ERR_CUDA;
    }
    g_scratch[device] = p;
  }
  *out = g_scratch[device];
  return PCEXP_OK;
}

}  // namespace

extern "C" int pcexp_residual_noalloc(pcexp_ctx* ctx, const double* U, double* R) {
  using namespace pcexp;
  if (!ctx || !U || !R) {
    set_last_error("pcexp_residual_noalloc: null context, input or output pointer");
    return PCEXP_ERR_INVALID_ARG;
  }
  DGData<double> d;
  cudaStream_t st = nullptr;
  int nfq = 0, fp32 = 0, device = 0;
  int r = ctx_noalloc_view(ctx, &d, &st, &nfq, &fp32, &device);
  if (r != PCEXP_OK) return r;
  if (fp32) {
    set_last_error("pcexp_residual_noalloc: the context is FP32-mixed; this entry point covers FP64 contexts");
    return PCEXP_ERR_UNSUPPORTED;
  }
  const long long need = (long long)d.F * nfq * (d.dim + 2);
  if (need > NOALLOC_FACE_FLUX_DOUBLES) {
    const std::string m = "pcexp_residual_noalloc: face-flux scratch too small: need " + std::to_string(need) +
                          " doubles, have " + std::to_string(NOALLOC_FACE_FLUX_DOUBLES);
    set_last_error(m.c_str());
    return PCEXP_ERR_INVALID_ARG;
  }
  double* G = nullptr;
  r = scratch_address(device, &G);
  if (r != PCEXP_OK) return r;
  cudaError_t e = launch_dg_operator<double>(d, U, nullptr, R, G, nullptr, nullptr, st);
  if (e != cudaSuccess) {
    const std::string m = std::string("pcexp_residual_noalloc: DG operator launch: ") + cudaGetErrorString(e);
    set_last_error(m.c_str());
    return PCEXP_ERR_CUDA;
  }
  return PCEXP_OK;
}
