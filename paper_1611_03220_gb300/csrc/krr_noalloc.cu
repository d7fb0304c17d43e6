// Kernel-matrix product that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need the product:
// code running while a stream is being captured into a CUDA graph (a
// cudaMalloc there breaks the capture), code inside a framework whose
// caching allocator already holds the GPU's memory (a raw cudaMalloc can
// fail although the framework's pool has room), and latency-critical loops
// that must not take the implicit device synchronisation an allocation or
// free may cause.  For them this file offers the FP64 product
// Q = K(Xr, Xc) V + shift V with its split-column partial sums in a fixed,
// file-scope device array instead of handle workspace.
//
// The array (NOALLOC_SCRATCH_DOUBLES doubles, 8 MiB) exists on every GPU that
// loads this library until the process exits.  Every call shares it and it
// keeps the last call's contents; nothing in it needs to start at zero
// because each call writes every partial it later reads.  Calls whose
// kernels overlap on the GPU (different streams, or different host threads)
// race on the array.
#include <cmath>
#include <mutex>

#include "krr_internal.cuh"

namespace krr {
namespace {

constexpr size_t NOALLOC_SCRATCH_DOUBLES = size_t(1) << 20;

__device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = reinterpret_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace krr

extern "C" krr_status krr_kernel_matvec_fp64_noalloc(const float* Xr, int nr, int ldxr,
                                                     const float* Xc, int nc, int ldxc, int d,
                                                     double sigma, double shift, const double* V,
                                                     int k, int ldv, double* Q, int ldq,
                                                     void* stream) {
  using namespace krr;
  if (!Xr || !Xc || !V || !Q) return KRR_EINVAL;
  if (nr <= 0 || nc <= 0 || d <= 0 || k < 1 || k > KRR_MAX_RHS) return KRR_EINVAL;
  if (ldxr < d || ldxc < d || ldv < k || ldq < k) return KRR_EINVAL;
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return KRR_EINVAL;
  if (shift != 0.0 && nr != nc) return KRR_EINVAL;
  if ((size_t)nr * (size_t)k > NOALLOC_SCRATCH_DOUBLES) return KRR_EINVAL;
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return KRR_ECUDA;
  }
  try {
    launch_mv_fp64_capped(reinterpret_cast<cudaStream_t>(stream), Xr, nr, ldxr, Xc, nc, ldxc, d,
                          sigma, shift, V, k, ldv, Q, ldq, scratch, NOALLOC_SCRATCH_DOUBLES);
  } catch (const Error& e) {
    return e.st;
  }
  return KRR_OK;
}
