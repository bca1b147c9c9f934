// dgx_rhs_noalloc: the residual for callers that cannot allocate device memory.
//
// Some programs that call this library may not allocate device memory while
// they run: a host whose whole device memory budget is reserved once at start
// up (real-time or embedded deployments), or a plugin environment that hands
// the library nothing but its input and output buffers.  Such callers cannot
// obtain the scratch workspace that dgx_rhs needs.  This entry point takes the
// scratch from a fixed array that lives inside the library instead; it calls
// no cudaMalloc, cudaFree or other allocating routine.  (The handle itself is
// still built by dgx_create / dgx_set_mesh_*, which allocate their small
// tables once at set-up.)
//
// The array is a file-scope static device variable of DGX_NOALLOC_SCRATCH_BYTES
// (64 MiB): every GPU on which the library's device code is loaded holds it
// until the process exits.  In host code its name is only a host-side handle
// for the symbol, not a device address, so the first call on each device asks
// the runtime for the array's device address (cudaGetSymbolAddress, with that
// device current) and caches it; make that first call before any stream
// capture.  All calls on a device share the one array: calls whose kernels can
// overlap on the GPU (two streams, or two handles on the same device) race on
// it and must be serialised by the caller.  The array keeps the previous
// call's contents; nothing in it needs to start at zero because the residual
// writes every scratch value before reading it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dgx.h"

static __device__ __align__(256) unsigned char dgx_noalloc_scratch[DGX_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex scratch_mutex;
void* scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
dgx_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DGX_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return DGX_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(scratch_mutex);
  if (!scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, dgx_noalloc_scratch) != cudaSuccess || !p) return DGX_ECUDA;
    scratch_addr[dev] = p;
  }
  *out = scratch_addr[dev];
  return DGX_OK;
}
}  // namespace

extern "C" dgx_status dgx_rhs_noalloc(dgx_handle* h, const void* U, void* dUdt, void* stream) {
  if (!h || !U || !dUdt || U == dUdt) return DGX_EINVAL;
  const size_t need = dgx_workspace_bytes(h, DGX_OP_RHS);
  if (need == 0) return DGX_ESTATE;
  if (need > (size_t)DGX_NOALLOC_SCRATCH_BYTES) return DGX_EINVAL;  // mesh too large for the fixed scratch
  void* scratch = nullptr;
  const dgx_status st = scratch_for_current_device(&scratch);
  if (st != DGX_OK) return st;
  return dgx_rhs(h, U, dUdt, scratch, stream);
}
