// Host-side helpers shared by the single-environment and batched entry points.
#pragma once

#include <cuda_runtime.h>

#include "flock.h"

// NVTX push/pop, defined in flock_nvtx.cu: the NVTX header includes the
// system's fcntl.h, whose `struct flock` would clash with namespace flock.
extern "C" __attribute__((visibility("hidden"))) void flock_nvtx_push(const char *name);
extern "C" __attribute__((visibility("hidden"))) void flock_nvtx_pop(void);

namespace flock {

// NVTX range over a scope (header-only NVTX 3: without a profiler attached a
// range costs a few nanoseconds and needs no library).  Entry points and
// the launches of each phase are named "flock:<what>", so a timeline shows
// where a step's host time goes and which call enqueued which kernels.
struct NvtxRange {
  explicit NvtxRange(const char *name) { flock_nvtx_push(name); }
  ~NvtxRange() { flock_nvtx_pop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Inst;

// Validates params and fills the derived constants and cell geometry of one
// instance (stencil 1: 3 x 3 cells of width >= d_v; 2: 5 x 5 of >= d_v / 2).
int derive(const flock_params &p, int stencil, Inst &I, flock_derived *D);
// Resolves the launch shape (0 fields = library choice) for n agents.
int choose_tuning(const Inst &I, int n, const flock_tuning *req, flock_tuning &t);
// Tile counts and shared-memory staging capacity.
void set_tiles(Inst &I, int n, const flock_tuning &t);
// Records a CUDA error for flock_last_cuda_error and returns FLOCK_ECUDA.
int cuda_fail(cudaError_t e, const char *what);
// Raises the dynamic shared-memory limit of the neighbour kernels (once).
cudaError_t set_kernel_attrs();

// Launch with programmatic stream serialization (pdl = true): the kernel's
// blocks may be scheduled while the previous kernel in the stream finishes,
// hiding the launch gap; every kernel launched this way waits in pdl_wait()
// before it reads what the previous one wrote.
template <typename... KArgs, typename... Args>
static cudaError_t launch(bool pdl, void (*k)(KArgs...), int grid, int block, size_t smem,
                          cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, ((KArgs)args)...);
}

}  // namespace flock
