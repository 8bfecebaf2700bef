// Right-hand-side evaluation for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc (or anything that does): code running while a stream
// is being captured into a CUDA graph, where an allocation is not captured and cudaFree
// synchronises the whole device; latency-critical loops that cannot afford that
// synchronisation; and host applications that hand out all device memory themselves.  For
// them, swf_rhs_noalloc performs the same evaluation as swf_rhs_dev but takes its workspace
// from one file-scope device array of fixed size instead of a context.
//
// The array lives in every GPU that loads this library until the process exits.  All calls
// on a device share it and it keeps the last call's contents: nothing in it has to start at
// zero (every byte a call reads was written earlier in the same call), but two calls that
// overlap on the GPU (different streams, or different host threads) race on it.
#include <mutex>

#include "swf_internal.h"

namespace {

// Largest grid the scratch holds: 4 components x 65536 points in complex128, plus tables.
constexpr size_t kMaxSites = 65536;
constexpr size_t kScratchBytes = (size_t)4 * kMaxSites * 16 + ((size_t)128 << 10);

static __device__ __align__(256) unsigned char g_rhs_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.  In
// host code the array's name is only a host-side stand-in, so kernels must get this address.
swf_status scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess) return swf::cuda_status(e, "cudaGetSymbolAddress(rhs scratch)");
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
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
