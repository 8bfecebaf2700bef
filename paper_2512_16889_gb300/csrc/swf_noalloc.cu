// Right-hand-side evaluation for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc (or anything that does): host applications that hand
// out all device memory themselves from a pool of their own, and latency-critical loops that
// cannot absorb the device-wide synchronisation that cudaFree brings.  For them,
// swf_rhs_noalloc performs the same evaluation as swf_rhs_dev but takes its workspace from one
// file-scope device array of fixed size instead of a context.
//
// The array lives in every GPU that loads this library until the process exits.  All calls
// on a device share it and it keeps the last call's contents: nothing in it has to start at
// zero (every byte a call reads was written earlier in the same call), but two calls that
// overlap on the GPU (different streams, or different host threads) race on it.
#include <cuda.h>

#include <mutex>

#include "swf_internal.h"

namespace {

// Largest grid the scratch holds: 4 components x 65536 points in complex128, plus tables.
constexpr size_t kMaxSites = 65536;
constexpr size_t kScratchBytes = (size_t)4 * kMaxSites * 16 + ((size_t)128 << 10);

static __device__ __align__(256) unsigned char g_rhs_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// The array's device address is a property of the CUDA context that loaded the module: after
// the device's primary context is reset and created again it can change.  The cache therefore
// remembers the unique id of the context it was looked up in (cuCtxGetId) and looks again when
// the current context's id differs.  Without the driver entry points (a driver older than
// CUDA 12.0) every call looks the address up.
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
};
std::mutex g_mu;
ScratchSlot g_slot[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_entry_once;

void load_entry_points() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  bool failed = false;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_current = (CtxGetCurrentFn)fn;
  else
    failed = true;
  fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_id = (CtxGetIdFn)fn;
  else
    failed = true;
  if (failed) cudaGetLastError();  // a missing entry point is not an error of a later call
}

// Id of the current context, or 0 when it cannot be read.
unsigned long long current_ctx_id() {
  std::call_once(g_entry_once, load_entry_points);
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return 0;
  if (g_ctx_get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current device's context.  In host code the
// array's name is only a host-side stand-in, so kernels must be given this address.
swf_status scratch_address(int device, void** out) {
  // 0 when no context is current yet (the lookup below creates the device's primary context)
  const unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchSlot& slot = g_slot[device];
  if (id == 0 || slot.ptr == nullptr || slot.ctx_id != id) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess) return swf::cuda_status(e, "cudaGetSymbolAddress(rhs scratch)");
    slot.ptr = p;
    slot.ctx_id = id != 0 ? id : current_ctx_id();
  }
  *out = slot.ptr;
  return SWF_OK;
}

}  // namespace

extern "C" swf_status swf_rhs_noalloc(const swf_instance* inst, int bg, swf_precision prec, double t,
                                      const void* psi_dev, void* out_dev, void* stream) {
  using namespace swf;
  swf_status s = validate_instances(1, inst, prec);
  if (s != SWF_OK) return s;
  if (bg != 0 && bg != 1) { set_error("bg must be 0 (U) or 1 (V)"); return SWF_EINVAL; }
  if (!psi_dev || !out_dev || psi_dev == out_dev) {
    set_error("psi_dev/out_dev must be distinct device pointers");
    return SWF_EINVAL;
  }
  if (!std::isfinite(t)) { set_error("t must be finite"); return SWF_EINVAL; }
  const GridDesc g = make_grid(inst->grid);
  const size_t need = rhs_scratch_bytes(g, prec);
  if ((size_t)g.N > kMaxSites || need > kScratchBytes) {
    set_error("swf_rhs_noalloc: grid of " + std::to_string(g.N) + " points exceeds the fixed scratch (at most " +
              std::to_string(kMaxSites) + " points)");
    return SWF_EINVAL;
  }
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (device < 0 || device >= kMaxDevices) { set_error("device index out of range"); return SWF_EINVAL; }
  void* scratch = nullptr;
  if ((s = scratch_address(device, &scratch)) != SWF_OK) return s;
  const FieldDesc fd = make_field_desc(*inst, bg);
  return rhs_eval_scratch(g, fd, prec, t, psi_dev, out_dev, scratch, (cudaStream_t)stream);
}
