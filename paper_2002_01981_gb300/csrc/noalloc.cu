// ifcm_fit_noalloc: one IFCM run whose scratch is held by the library itself.
//
// Some callers cannot allocate device memory at the point where they want a
// segmentation: code recording a CUDA graph under global capture mode (where
// cudaMalloc is not permitted), plugins of a host framework that hands them
// only the device pointers of their inputs and outputs and owns every other
// allocation, or latency-bound loops that must not take the allocator's
// implicit synchronisation.  ifcm_fit asks them for a workspace; this entry
// point needs none.  Its scratch is the fixed device array below.  The CUDA
// runtime places it in a GPU's memory when it loads this library's module on
// that GPU -- with lazy module loading, at the first call there -- and it
// stays until the process exits.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "launch.h"

namespace pifcm {
void set_error_message(const char* fmt, ...);
}

// 64 MiB of scratch: room for an ifcm_fit workspace of up to 64 MiB, e.g. a
// volume of about 1.36 million voxels (111^3) at c = 4 (the uniform start and
// two membership buffers of c planes, plus the per-tile partial sums).
static constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of the array is not a device address).
ifcm_status scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    pifcm::set_error_message("cudaGetDevice: %s", cudaGetErrorString(e));
    return IFCM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    pifcm::set_error_message("device %d beyond the %d devices this entry point tracks", dev,
                             kMaxDevices);
    return IFCM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      pifcm::set_error_message("cudaGetSymbolAddress(scratch) on device %d: %s", dev,
                               cudaGetErrorString(e));
      return IFCM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return IFCM_OK;
}

}  // namespace

extern "C" ifcm_status ifcm_fit_noalloc(const float* x, ifcm_shape shape, const ifcm_params* p,
                                        const double* lam_xi, const float* u_init,
                                        const double* c_init, float* u_out, double* c_out,
                                        double* J_out, int32_t* iters_out, void* stream) {
  const size_t need = ifcm_fit_workspace_bytes(shape, p);
  if (need == 0)   // invalid parameters: let ifcm_fit name the problem
    return ifcm_fit(x, shape, p, lam_xi, u_init, c_init, u_out, c_out, J_out, iters_out,
                    nullptr, 0, stream);
  if (need > kNoAllocScratchBytes) {
    pifcm::set_error_message(
        "ifcm_fit_noalloc: this volume needs %zu bytes of scratch but the library's static "
        "scratch holds %zu bytes (64 MiB); use ifcm_fit with a caller workspace",
        need, kNoAllocScratchBytes);
    return IFCM_ERR_NOMEM;
  }
  void* scratch = nullptr;
  const ifcm_status s = scratch_on_current_device(&scratch);
  if (s != IFCM_OK) return s;
  // ifcm_fit clears the status word and the update counter and rewrites every
  // other scratch region before reading it, so stale contents left by an
  // earlier call are harmless.
  return ifcm_fit(x, shape, p, lam_xi, u_init, c_init, u_out, c_out, J_out, iters_out, scratch,
                  kNoAllocScratchBytes, stream);
}

// The device status word of the last ifcm_fit_noalloc call on the current
// device (it sits at the start of the static scratch, as in any workspace).
extern "C" ifcm_status ifcm_fit_noalloc_status(void* stream) {
  void* scratch = nullptr;
  const ifcm_status s = scratch_on_current_device(&scratch);
  if (s != IFCM_OK) return s;
  return ifcm_device_status(scratch, stream);
}
