// mpcgemm_noalloc: the complex GEMM for callers that cannot allocate device
// memory.  Its scratch space is a file-scope device array of fixed size
// (MPC_NOALLOC_SCRATCH_BYTES) instead of a caller-provided workspace.
//
// The array belongs to this translation unit's device module (which has no
// kernels), so it is reserved on a device when that module is loaded there:
// under CUDA's default lazy module loading, when this entry point (or its
// status reader) first looks the array up on that device; under eager loading
// (CUDA_MODULE_LOADING=EAGER), on every device the process initialises, whether
// or not it calls this entry point.  It stays reserved until the process exits.
// Host code cannot pass `g_noalloc_scratch` to a kernel (in host code the name
// is a host-side shadow, not a device address); the device address is looked
// up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "common.cuh"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[MPC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
int scratch_for_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return MPC_ECUDA - (int)e;
  if (dev < 0 || dev >= kMaxDevices) return MPC_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return MPC_ECUDA - (int)(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return MPC_OK;
}

}  // namespace

extern "C" int mpcgemm_noalloc(int64_t m, int64_t n, int64_t k, int32_t p_bits, const mpc_mat *A, const mpc_mat *B,
                               mpc_mat *C, int method, int algo, void *stream) {
  mpc_plan plan;
  int rc = mpcgemm_plan(m, n, k, p_bits, method, algo, nullptr, &plan);
  if (rc != MPC_OK) return rc;
  if (plan.ws_bytes > (uint64_t)MPC_NOALLOC_SCRATCH_BYTES) return MPC_ENOSPC;   // problem too large
  void *scratch = nullptr;
  rc = scratch_for_current_device(&scratch);
  if (rc != MPC_OK) return rc;
  return mpcgemm_ex(m, n, k, p_bits, A, B, C, method, algo, nullptr, scratch, (size_t)MPC_NOALLOC_SCRATCH_BYTES,
                    stream);
}

extern "C" int mpcgemm_noalloc_read_status(mpc_status *status, void *stream) {
  if (!status) return MPC_EINVAL;
  void *scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);   // a lookup, no allocation
  if (rc != MPC_OK) return rc;
  // the status block sits at the start of the array (offset 0 of every plan)
  return mpcgemm_read_status(scratch, (size_t)MPC_NOALLOC_SCRATCH_BYTES, status, stream);
}
