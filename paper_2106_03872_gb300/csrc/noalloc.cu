// ks_overlap_noalloc: the overlap matrix A^H B of two device blocks without any device
// allocation, for callers that must not call cudaMalloc.
//
// The split-K partial sums of the overlap GEMM need scratch memory.  Inside a ks_grid that
// scratch is allocated once by ks_grid_create; here it is a fixed array in this file, so the
// call needs no handle and allocates nothing.  The array holds 262,144 complex128 values
// (4 MiB) and every GPU that loads this library keeps it until the process exits.
#include <mutex>

#include "kernels.h"

namespace {

constexpr size_t kOverlapScratchElems = 262144;   // double2 elements = 4 MiB

}  // namespace

// Shared by every call on a device; each call overwrites the partials it reads.
static __device__ __align__(256) double2 ks_overlap_scratch[kOverlapScratchElems];

namespace {

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (with
// that device current) and cached.
void* scratch_on_current_device() {
  int dev = 0;
  KS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) ks::fail(KS_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, ks_overlap_scratch);
    if (e != cudaSuccess) ks::fail_cuda(e, "cudaGetSymbolAddress(ks_overlap_scratch)", __FILE__, __LINE__);
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" ks_status ks_overlap_noalloc(const void* a_dev, const void* b_dev, int m, int n, int nG, int fp64,
                                        void* out_dev, void* stream) {
  try {
    if (!a_dev || !b_dev || !out_dev) ks::fail(KS_ERR_ARG, "ks_overlap_noalloc: NULL device pointer");
    if (m < 1 || n < 1 || nG < 1) ks::fail(KS_ERR_ARG, "ks_overlap_noalloc: m=%d n=%d nG=%d must be >= 1", m, n, nG);
    if ((size_t)m * (size_t)n > kOverlapScratchElems)
      ks::fail(KS_ERR_ARG, "ks_overlap_noalloc: m*n = %zu exceeds the scratch maximum of %zu (4 MiB)",
               (size_t)m * (size_t)n, kOverlapScratchElems);
    double2* part = static_cast<double2*>(scratch_on_current_device());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double2* out = static_cast<double2*>(out_dev);
    if (fp64)
      ks::gemm_cn<double>(static_cast<const double2*>(a_dev), nG, static_cast<const double2*>(b_dev), nG, m, n, nG,
                          part, kOverlapScratchElems, out, s);
    else
      ks::gemm_cn<float>(static_cast<const float2*>(a_dev), nG, static_cast<const float2*>(b_dev), nG, m, n, nG,
                         part, kOverlapScratchElems, out, s);
    return KS_OK;
  } catch (const ks::Error& e) {
    return e.st;
  } catch (...) {
    ks::set_last_error("ks_overlap_noalloc: unexpected internal error");
    return KS_ERR_CUDA;
  }
}
