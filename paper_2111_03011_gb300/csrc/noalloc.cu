// Squared norm of a head tensor for callers that cannot allocate device memory.
//
// tn_head_norm keeps its per-group partial sums in scratch that the head
// allocates with cudaMalloc.  Some callers cannot allocate: code embedded in
// another framework that owns every byte of device memory through its own
// allocator, or a latency-critical loop where cudaMalloc (which may
// synchronise the device) is forbidden.  This file gives them the same
// reduction with its scratch in a fixed file-scope device array instead.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"
#include "tn_gb300.h"

namespace tn {
void set_last_error(const std::string& msg);
}

namespace {

// Per-group partial sums; every GPU that loads the library holds this array
// (1 MiB) until the process exits.
constexpr int64_t kMaxGroups = TN_NOALLOC_MAX_GROUPS;
static __device__ __align__(256) double g_group_sums[kMaxGroups];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {nullptr};

int fail(int code, const std::string& msg) {
  tn::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int tn_head_norm_noalloc(const void* head_c128, int64_t n_groups, int n_open, double* norm_out,
                                    void* stream) {
  if (!head_c128 || !norm_out) return fail(TN_ERR_INVALID, "head or norm_out is NULL");
  if (n_groups < 1 || n_groups > kMaxGroups)
    return fail(TN_ERR_INVALID, "n_groups must be in [1, " + std::to_string(kMaxGroups) + "] for the fixed scratch");
  if (n_open < 0 || n_open > 30) return fail(TN_ERR_INVALID, "n_open must be in [0, 30]");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(TN_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  // Host code sees only a stand-in for the array: its device address is
  // looked up with the device current.  Outside a stream capture it is looked
  // up again on every call (cheap, and it allocates nothing), so an address
  // made stale by cudaDeviceReset (which reloads the module) is never used;
  // inside a capture the address cached by an earlier call is used.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
  if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_group_sums);
      if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_dev_ptr[dev] = (double*)p;
    } else if (!g_dev_ptr[dev]) {
      return fail(TN_ERR_INVALID, "the first call on a device must come before any stream capture");
    }
    scratch = g_dev_ptr[dev];
  }
  // every entry read by the sum is first written by the per-group pass, so
  // nothing left by an earlier call needs clearing
  e = tn::launch_group_norms((const double2*)head_c128, n_groups, n_open, scratch, norm_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("norm launch: ") + cudaGetErrorString(e));
  return TN_OK;
}
