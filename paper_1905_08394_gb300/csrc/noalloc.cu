// Allocation-free amplitude entry point.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool, plug-ins loaded into a host that owns every
// allocation, or tools that must not grow device memory after start-up.  For
// them peps_amplitudes_noalloc runs the same device path as
// peps_amplitudes_device, but its workspace is the file-scope device array
// below instead of caller memory.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// Cost: every GPU that loads this library holds the array (64 MiB) until the
// process exits.  Workloads whose workspace would exceed it are rejected.
#include <cuda_runtime.h>

#include <mutex>

#include "common.h"

namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;  // 64 MiB

// The scratch.  In host code this name is only a stand-in for the device
// array: its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (set-up once per
// device, with that device current).
int scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return peps::internal_fail(PEPS_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return peps::internal_fail(PEPS_EUNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return peps::internal_fail(PEPS_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                                 cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PEPS_OK;
}

}  // namespace

extern "C" int peps_amplitudes_noalloc(peps_ctx *ctx, const uint64_t *d_bitstrings, int64_t n,
                                       peps_c128 *d_out, const peps_opts *opts, void *stream) {
  if (!ctx) return peps::internal_fail(PEPS_EINVAL, "peps_amplitudes_noalloc: NULL context");
  peps_opts o{};
  if (opts) o = *opts;
  if (o.flags & PEPS_FLAG_TIMING)
    return peps::internal_fail(PEPS_EINVAL,
                               "peps_amplitudes_noalloc: PEPS_FLAG_TIMING is not available here "
                               "(it creates CUDA events)");
  // A CUDA graph would be captured and instantiated anew on every call (the
  // plan is rebuilt each time), which allocates and gains nothing.
  if (o.flags & PEPS_FLAG_GRAPH)
    return peps::internal_fail(PEPS_EINVAL,
                               "peps_amplitudes_noalloc: PEPS_FLAG_GRAPH is not available here "
                               "(it creates a capture stream and instantiates a graph)");
  size_t need = 0;
  int rc = peps_workspace_bytes(ctx, n, &o, &need);
  if (rc) return rc;
  if (need > kNoAllocBytes)
    return peps::internal_fail(PEPS_ENOMEM,
                               "peps_amplitudes_noalloc: this call needs %zu bytes of workspace; the "
                               "static scratch holds %zu (use peps_amplitudes_device with caller memory)",
                               need, kNoAllocBytes);
  void *ws = nullptr;
  rc = scratch_address(&ws);
  if (rc) return rc;
  // The scratch is shared by every context and keeps the previous call's
  // contents: drop this context's cached tables and site tensors so that the
  // call rebuilds them (status words, records and accumulators are cleared by
  // every call of the device path).  The new tables are uploaded on `stream`,
  // behind the kernels of earlier calls enqueued there, which may still read
  // the old ones.
  peps::internal_forget_workspace(ctx);
  o.flags |= PEPS_FLAG_REBUILD;
  return peps_amplitudes_device(ctx, d_bitstrings, n, d_out, &o, ws, kNoAllocBytes, stream);
}
