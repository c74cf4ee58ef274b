// adg_step_noalloc: global time steps that allocate no device memory.
//
// Who needs it: code that is not allowed to call cudaMalloc while it steps,
// e.g. a plug-in whose host application owns and budgets all device memory,
// or a caller whose framework forbids raw device allocations at that point.
// Such a caller keeps its dofs in memory it already owns and passes them in;
// the only extra device memory the step needs - the time-integrated face
// traces that the local kernel writes and the neighbour kernel reads - lives
// in the fixed-size array below instead of being allocated.
//
// The array is a file-scope static __device__ object of kScratchBytes; every
// GPU that loads this library holds it until the process exits.  Its device
// address is looked up once per device, on the first call made with that
// device current (that first call should therefore come before any stream
// capture).  All calls share the array and it keeps whatever the last call
// left there; every trace is written before it is read, so nothing has to be
// cleared, but calls whose work overlaps on the GPU (different streams, or
// different contexts at the same time) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "adg_internal.hpp"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB of face traces
static __device__ __align__(256) unsigned char g_trace_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

}  // namespace

extern "C" int adg_step_noalloc(adg_ctx* ctx, void* d_Q, int n_steps, void* stream) {
  if (!ctx || !d_Q || n_steps < 0) return ADG_E_INVALID;
  adg::Ctx& c = ctx->c;
  if (!c.inited) {
    c.last_error = "call adg_init first";
    return ADG_E_STATE;
  }
  if (c.ncl != 1 || c.S != 1 || !c.gfaces.empty() || c.n_fault_faces) {
    c.last_error = "adg_step_noalloc needs a global-time-stepping context (one cluster), ensemble 1, "
                   "and no gravitational or fault faces";
    return ADG_E_INVALID;
  }
  const size_t need = (size_t)c.nt * 4 * adg::face_stride(c.N) * (c.fp64 ? 8 : 4);
  if (need > kScratchBytes) {
    c.last_error = "adg_step_noalloc: the face traces of this mesh need " + std::to_string(need) +
                   " bytes of scratch; the fixed maximum is " + std::to_string(kScratchBytes) + " bytes";
    return ADG_E_INVALID;
  }
  int dev = -1;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess || dev != c.cfg.device || dev < 0 || dev >= kMaxDevices) {
    c.last_error = "adg_step_noalloc: make the context's device current before the call";
    return ADG_E_INVALID;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      ce = cudaGetSymbolAddress(&p, g_trace_scratch);
      if (ce != cudaSuccess || !p) {
        c.last_error = std::string("adg_step_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce);
        return ADG_E_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  // NULL is CUDA's default stream (the legacy one), as for any CUDA call: a
  // caller that wrote d_Q there, torch's default stream included, is ordered
  // before these kernels
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamLegacy;
  adg::StepArgs a = c.base_args();
  a.Q = d_Q;
  a.trace = scratch;
  adg::Seg sg{};  // the whole mesh, one global step of dt_min
  sg.v_begin = 0;
  sg.n = c.nt;
  sg.dt = c.dtmin;
  double fa = 0.0, fb = c.dtmin, fac = 1.0;
  for (int k = 0; k <= c.N; ++k) {
    fac *= (k + 1);
    sg.tcoef[k] = (fb - fa) / fac;
    fb *= c.dtmin;
  }
  const adg::Segs g = adg::make_segs(&sg, 1, 1);
  for (int i = 0; i < n_steps; ++i) {
    int rc = adg::launch_local(c.fp64, c.N, a, g, st);
    if (!rc) rc = adg::launch_neighbour(c.fp64, c.N, a, g, st);
    if (rc) {
      c.last_error = std::string("adg_step_noalloc: launch failed: ") + cudaGetErrorString((cudaError_t)rc);
      return ADG_E_CUDA;
    }
  }
  c.last_error.clear();
  return ADG_OK;
}
