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
// (64 MiB).  Under CUDA's lazy module loading (the default) the module that
// holds it, and with it the 64 MiB, is created on a device the first time this
// entry point runs there; from then on that device holds it until the process
// exits.  In host code the array's name is only a host-side handle for the
// symbol, not a device address, so the first call on each device asks the
// runtime for the array's device address (cudaGetSymbolAddress, with that
// device current) and caches it together with the identity of the device's
// current context; a later call in a new context (after cudaDeviceReset, say)
// looks the address up again.  Make the first call on each device as a
// warm-up: before reserving the rest of device memory and before any stream
// capture.  The handle's device must be current (else DGX_EINVAL).  All calls
// on a device share the one array: calls whose kernels can overlap on the GPU
// (two streams, or two handles on the same device) race on it and must be
// serialised by the caller.  The array keeps the previous call's contents;
// nothing in it needs to start at zero because the residual writes every
// scratch value before reading it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dgx.h"

extern "C" int dgx_internal_handle_device(const dgx_handle* h);

static __device__ __align__(256) unsigned char dgx_noalloc_scratch[DGX_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex scratch_mutex;
struct Entry {
  void* addr = nullptr;
  unsigned long long ctx = 0;  // id of the context the address belongs to
};
Entry scratch_cache[kMaxDevices];

// Driver entry points for the identity of the current context, resolved once
// through the runtime (no link-time dependency on the driver library).
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = (CtxGetCurrentFn)f1;
      get_id = (CtxGetIdFn)f2;
    }
    resolved = true;
  }
  void* ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// Device address of the scratch array on device dev (which is current).
dgx_status scratch_for_device(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return DGX_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(scratch_mutex);
  unsigned long long ctx = 0;
  const bool known_ctx = current_context_id(&ctx);
  Entry& e = scratch_cache[dev];
  if (!e.addr || !known_ctx || e.ctx != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, dgx_noalloc_scratch) != cudaSuccess || !p) {
      e = Entry{};
      return DGX_ECUDA;
    }
    e.addr = p;
    e.ctx = known_ctx ? ctx : 0;
  }
  *out = e.addr;
  return DGX_OK;
}
}  // namespace

extern "C" dgx_status dgx_rhs_noalloc(dgx_handle* h, const void* U, void* dUdt, void* stream) {
  if (!h || !U || !dUdt || U == dUdt) return DGX_EINVAL;
  const size_t need = dgx_workspace_bytes(h, DGX_OP_RHS);
  if (need == 0) return DGX_ESTATE;
  if (need > (size_t)DGX_NOALLOC_SCRATCH_BYTES) return DGX_EINVAL;  // mesh too large for the fixed scratch
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return DGX_ECUDA;
  if (cur != dgx_internal_handle_device(h)) return DGX_EINVAL;  // the handle's device must be current
  void* scratch = nullptr;
  const dgx_status st = scratch_for_device(cur, &scratch);
  if (st != DGX_OK) return st;
  return dgx_rhs(h, U, dUdt, scratch, stream);
}
