// chi0_invert_eps_noalloc: the Dyson inversion without any device allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's caching allocator that must account for
// every byte it hands out), or a service that must keep a fixed device-memory
// footprint once it has started, so that a later allocation can neither fail
// nor push another tenant of the GPU out of memory.  This entry point runs the
// same blocked Gauss-Jordan kernels as chi0_invert_eps, one frequency after
// another, with all of their scratch (the row/column panels, the pivot-block
// inverse, the Coulomb factors and the error flag) in one file-scope device
// array whose size is fixed at build time.  Every GPU that loads the library
// holds that array until the process exits.  The first call on a device
// looks up the array's device address (cudaGetSymbolAddress, once per
// device, with that device current); make that first call before any stream
// capture begins.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/chi0.h"
#include "internal.cuh"

namespace {

constexpr int kNoallocMaxNg = 2048;  // largest N_G this entry point accepts
constexpr int kPanelW = 32;          // pivot-block width of the Gauss-Jordan kernels

// layout of the scratch array (bytes)
constexpr size_t kColBytes = (size_t)kNoallocMaxNg * kPanelW * sizeof(double2);
constexpr size_t kRowBytes = (size_t)kPanelW * kNoallocMaxNg * sizeof(double2);
constexpr size_t kPivBytes = (size_t)kPanelW * kPanelW * sizeof(double2);
constexpr size_t kVBytes = (size_t)kNoallocMaxNg * sizeof(double);
constexpr size_t kErrBytes = 256;
constexpr size_t kOffCol = 0;
constexpr size_t kOffRow = kOffCol + kColBytes;
constexpr size_t kOffPiv = kOffRow + kRowBytes;
constexpr size_t kOffV = kOffPiv + kPivBytes;
constexpr size_t kOffErr = kOffV + kVBytes;
constexpr size_t kScratchBytes = kOffErr + kErrBytes;  // ~2.1 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per
// device, with that device current).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" chi0_status chi0_invert_eps_noalloc(const void* chi0, const double* v_sqrt, int ng,
                                               int nw, void* out, void* cuda_stream) {
  if (!chi0 || !v_sqrt || !out) return CHI0_EINVAL;
  if (ng < 1 || nw < 1) return CHI0_EINVAL;
  if (ng > kNoallocMaxNg) return CHI0_EUNSUPPORTED;  // scratch holds panels for N_G <= 2048
  for (int i = 0; i < ng; ++i)
    if (!(std::isfinite(v_sqrt[i]) && v_sqrt[i] > 0.0)) return CHI0_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  double2* colp = reinterpret_cast<double2*>(b + kOffCol);
  double2* rowp = reinterpret_cast<double2*>(b + kOffRow);
  double2* pinv = reinterpret_cast<double2*>(b + kOffPiv);
  double* vs = reinterpret_cast<double*>(b + kOffV);
  int* err = reinterpret_cast<int*>(b + kOffErr);
  // the array keeps the previous call's contents: clear the error flag
  if (cudaMemsetAsync(err, 0, 2 * sizeof(int), st) != cudaSuccess ||
      cudaMemcpyAsync(vs, v_sqrt, (size_t)ng * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  const size_t n2 = (size_t)ng * ng;
  for (int iw = 0; iw < nw; ++iw) {
    const double2* c = static_cast<const double2*>(chi0) + iw * n2;
    double2* o = static_cast<double2*>(out) + iw * n2;
    if (chi0::launch_dyson(c, vs, ng, 1, o, colp, rowp, pinv, err, st) != cudaSuccess) {
      cudaGetLastError();
      return CHI0_ECUDA;
    }
  }
  int h[2] = {0, 0};
  if (cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  return h[0] ? CHI0_ENOTPD : CHI0_OK;
}
