// Host-side helpers shared by the single-environment and batched entry points.
#pragma once

#include <cuda_runtime.h>

#include "flock.h"

namespace flock {

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

}  // namespace flock
