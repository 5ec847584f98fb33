// frx_ozaki_gemm_static: the Ozaki-scheme product of frx_ozaki_gemm for callers that
// cannot allocate device memory.
//
// Some callers have no way to call cudaMalloc: a plugin running inside a host
// framework that has already reserved the whole device memory for its own caching
// allocator (a new cudaMalloc fails or fragments that pool), or code that is handed
// only a stream and no allocator.  This entry point takes its scratch from a fixed
// array in device memory that is part of this library (file-scope, see below), so it
// performs no allocation of its own.
#include "frx_internal.cuh"

namespace {

// Largest problem the fixed scratch holds: m, n, k <= 512 and slices <= 8.
constexpr int64_t kStaticMaxDim = 512;
constexpr int kStaticMaxSlices = 8;
constexpr size_t kStaticScratchBytes = (size_t)24 * 1024 * 1024 + (size_t)64 * 1024;

// The scratch itself.  Its bytes are reserved on a device when this file's module is
// loaded there: under CUDA's default lazy module loading that is the first call of
// frx_ozaki_gemm_static on the device (CUDA_MODULE_LOADING=EAGER moves it to the
// library's load), and it stays reserved until the process exits.  In host code
// `g_static_scratch` names a host-side stand-in, not device memory; the device address
// comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the scratch on the current device.  Looked up on every call: the
// lookup is a host-side query that enqueues no work, and it stays right after a
// cudaDeviceReset, which reloads the module at another address.
int scratch_on_current_device(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return FRX_E_CUDA;
  *out = p;
  return FRX_OK;
}

}  // namespace

extern "C" {

int frx_ozaki_gemm_static(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                          double* C_lo, int64_t m, int64_t n, int64_t k, int slices, int mode, void* stream) {
  if (m > kStaticMaxDim || n > kStaticMaxDim || k > kStaticMaxDim || slices > kStaticMaxSlices)
    return FRX_E_UNSUPPORTED;
  size_t need = frx_ozaki_gemm_workspace_bytes(m, n, k, slices);
  if (need == 0) return FRX_E_ARG;
  if (need > kStaticScratchBytes) return FRX_E_UNSUPPORTED;
  void* scratch = nullptr;
  int st = scratch_on_current_device(&scratch);
  if (st != FRX_OK) return st;
  return frx_ozaki_gemm(A, lda, B, ldb, C, ldc, C_lo, m, n, k, slices, mode, scratch, kStaticScratchBytes,
                        stream);
}

}  // extern "C"
