// ks_overlap_noalloc: the overlap matrix A^H B of two device blocks without any device
// allocation, for callers that must not call cudaMalloc.
//
// The split-K partial sums of the overlap GEMM need scratch memory.  Inside a ks_grid that
// scratch is allocated once by ks_grid_create; here it is a fixed array in this file, so the
// call needs no handle and allocates nothing.  The array holds 262,144 complex128 values
// (4 MiB) and every GPU that loads this library keeps it until the process exits.
#include <cuda.h>   // driver types only: the two driver calls below are looked up at run time

#include <mutex>

#include "kernels.h"

namespace {

constexpr size_t kOverlapScratchElems = 262144;   // double2 elements = 4 MiB

}  // namespace

// Shared by every call on a device; each call overwrites the partials it reads.
static __device__ __align__(256) double2 ks_overlap_scratch[kOverlapScratchElems];

namespace {

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 256;
struct ScratchEntry {
  void* addr = nullptr;
  unsigned long long ctx_id = 0;   // the context the address belongs to (0: none yet)
};
ScratchEntry g_scratch[kMaxDevices];

// Identifier of the calling thread's current context (unique for the life of the process), or 0
// when no context is current yet.  The driver's entry points are obtained through the runtime, so
// the library needs no link against the driver library.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    KS_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
    KS_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      ks::fail(KS_ERR_CUDA, "ks_overlap_noalloc: the driver lacks cuCtxGetCurrent / cuCtxGetId");
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current device's current context.  In host code
// the array's name is only a host-side stand-in, so the address is looked up with that device
// current (cudaGetSymbolAddress) and cached together with the context's identifier; a new
// context (after cudaDeviceReset, for example) holds a new copy of the array, and its address is
// looked up again.
void* scratch_on_current_device() {
  int dev = 0;
  KS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) ks::fail(KS_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchEntry& e = g_scratch[dev];
  const unsigned long long id = current_context_id();
  if (e.addr && id != 0 && id == e.ctx_id) return e.addr;
  void* p = nullptr;
  const cudaError_t err = cudaGetSymbolAddress(&p, ks_overlap_scratch);   // binds the context if needed
  if (err != cudaSuccess) ks::fail_cuda(err, "cudaGetSymbolAddress(ks_overlap_scratch)", __FILE__, __LINE__);
  e.addr = p;
  e.ctx_id = current_context_id();
  return p;
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
