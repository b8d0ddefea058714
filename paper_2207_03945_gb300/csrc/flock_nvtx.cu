// NVTX ranges of the library's entry points and phases (see NvtxRange in
// flock_host.h).  A translation unit of its own: the NVTX 3 header includes
// the system's fcntl.h, whose `struct flock` clashes with namespace flock.
// NVTX 3 is header-only: without a profiler attached, a push or pop is a
// call through an empty function table.
#include <nvtx3/nvToolsExt.h>

#define FLOCK_HIDDEN __attribute__((visibility("hidden")))

extern "C" FLOCK_HIDDEN void flock_nvtx_push(const char *name) { nvtxRangePushA(name); }
extern "C" FLOCK_HIDDEN void flock_nvtx_pop(void) { nvtxRangePop(); }
