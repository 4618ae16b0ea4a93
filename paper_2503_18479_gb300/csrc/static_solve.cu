// static_solve.cu -- mts_solve_static: the port solve, objective and loss gradient without
// any caller-provided or library-allocated scratch buffer.
//
// Some callers cannot allocate device memory at the moment they want to solve: code that
// runs inside another framework's allocator-free region (a real-time control loop on the
// scanner host, a plugin whose host application owns every device allocation, a process
// that has pinned its memory budget up front). This entry point serves them: the per-call
// working state that mts_solve keeps in the caller's tape lives here in one file-scope
// device array of fixed size, reserved when the library's device code is loaded and held
// by every GPU that loads it until the process exits.
//
// The host never touches the array by name (in host code the name is only a stand-in for
// the device symbol): its device address is looked up with cudaGetSymbolAddress, with the
// device current, and passed to the kernels.
#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace mts {

// Shared per-process scratch of every mts_solve_static call on this device.
static __device__ __align__(256) unsigned char g_static_scratch[MTS_STATIC_SCRATCH_BYTES];

namespace {
// Device address of the scratch array in the current context. Looked up on every call
// (a table lookup once the module is loaded) rather than cached, so that a context that was
// destroyed and re-created (cudaDeviceReset, a host framework resetting the device) never
// leaves a stale address behind. The first lookup in a context loads the module, which is
// why the first call on a device must come before any stream capture.
mts_status static_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || p == nullptr) return MTS_ECUDA;
  *out = p;
  return MTS_OK;
}
}  // namespace

}  // namespace mts

using namespace mts;

extern "C" mts_status mts_solve_static(const mts_problem* pb, mts_precision prec,
                                       const void* basis, const mts_eval* ev, double* I_out,
                                       double* loss_out, double* dloss_dC_out,
                                       mts_stream stream) {
  // the same argument rules as mts_solve, checked before anything else happens
  size_t need = mts_tape_bytes(pb, ev ? ev->n_cfg : -1, prec);
  if (need == 0) return MTS_EINVAL;
  if (need > (size_t)MTS_STATIC_SCRATCH_BYTES) return MTS_EWORKSPACE;
  if ((loss_out || dloss_dC_out) && !ev->target) return MTS_EINVAL;
  void* scratch = nullptr;
  mts_status s = static_scratch(&scratch);
  if (s != MTS_OK) return s;
  // mts_solve clears the words that must start at zero and writes every other region it
  // reads later in the same call, so the previous call's contents are never used.
  s = mts_solve(pb, prec, basis, ev, I_out, loss_out, scratch, (size_t)MTS_STATIC_SCRATCH_BYTES,
                stream);
  if (s != MTS_OK || !dloss_dC_out) return s;
  // dloss/dC = the tape's reduced gradient (grad_loss = 1 for every configuration)
  TapeLayout tl = tape_layout(pb, ev->n_cfg, prec);
  cudaError_t e = cudaMemcpyAsync(dloss_dC_out, static_cast<char*>(scratch) + tl.dldc,
                                  sizeof(double) * (size_t)ev->n_cfg * pb->n_ports,
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? MTS_OK : MTS_ECUDA;
}

extern "C" mts_status mts_solve_static_status(const mts_problem* pb, int64_t n_cfg,
                                              mts_precision prec, int64_t* n_bad,
                                              mts_stream stream) {
  // the per-system status words of the last mts_solve_static call live in the static
  // array at the tape offsets of (pb, n_cfg, prec); mts_tape_status counts them
  size_t need = mts_tape_bytes(pb, n_cfg, prec);
  if (need == 0) return MTS_EINVAL;
  if (need > (size_t)MTS_STATIC_SCRATCH_BYTES) return MTS_EWORKSPACE;
  void* scratch = nullptr;
  mts_status s = static_scratch(&scratch);
  if (s != MTS_OK) return s;
  return mts_tape_status(pb, n_cfg, prec, scratch, n_bad, stream);
}
