// Batched flock step: many independent instances of the environment of arXiv
// 2207.03945 (Section 4.1) advanced by one persistent cooperative kernel (or,
// mode 3, that kernel for the binning and a second persistent launch for the
// neighbour scan).
//
// The kernel runs the four phases of a step over flattened work lists that
// span all active instances, separated by grid barriers:
//   A  agents  -> apply actions, bin into the instance's cell list
//   B  cells   -> exclusive scan, 1024-cell tiles (one global scan: instance
//                 k's cells and agents are contiguous ranges, in the same order)
//   C  agents  -> counting-sort scatter into cell order
//   D  chunks  -> 32 consecutive sorted agents of one instance per warp,
//                 taken from a shared ticket; neighbour scan (direct form)
// Descriptors and outputs live in device memory read by the kernel, so one
// captured graph serves every step and every change of the active set.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "flock_device.cuh"
#include "flock_host.h"

namespace flock {

constexpr int kBatchBlock = 256;
constexpr int kCtrBarCount = 0, kCtrBarGen = 1, kCtrTicket = 2, kCtrExit = 3, kCtrAbort = 4;

// Device-resident arguments of the batched kernel.
struct BatchDev {
  int n_inst, n_total, c_total, n_scan_tiles;
  int n_chunks, pad0, pad1, pad2;
  Bufs B;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier with a bounded wait.  Returns false (and latches
// FLOCK_ERR_TIMEOUT) when the wait gives up; the caller then leaves.
__device__ bool grid_barrier(unsigned *ctr, unsigned *err, unsigned spin_limit, int *flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire(&ctr[kCtrBarGen]);
    __threadfence();
    const unsigned arrived = atomicAdd(&ctr[kCtrBarCount], 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(&ctr[kCtrBarCount], 0u);
      __threadfence();
      st_release(&ctr[kCtrBarGen], gen + 1u);
    } else {
      ok = 0;
      for (unsigned it = 0; it < spin_limit; ++it) {
        if (ld_acquire(&ctr[kCtrBarGen]) != gen) {
          ok = 1;
          break;
        }
        __nanosleep(64);
      }
      if (!ok) {
        atomicOr(err, FLOCK_ERR_TIMEOUT);
        atomicExch(&ctr[kCtrAbort], 1u);
      }
    }
    // a block that gave up, or that sees that another one did, stops
    if (ok && ld_acquire(&ctr[kCtrAbort])) ok = 0;
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

// Largest k with pre[k] <= x, for pre[0] = 0 <= x < pre[n].
__device__ __forceinline__ int find_inst(const int *pre, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(pre + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The same search by the 32 lanes of a warp together (x the same in every
// lane, n >= 1): each round the lanes load 32 evenly spaced entries of the
// range still open, and the last lane whose entry is <= x narrows it to its
// stretch, so that 1,024 instances take two dependent loads instead of ten.
// pre is nondecreasing and pre[0] = 0 <= x, so lane 0 always qualifies.
__device__ __forceinline__ int warp_find_inst(const int *pre, int n, int x) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = n;  // the answer is in [lo, hi); pre[lo] <= x
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const int idx = lo + lane * step;
    const bool ok = idx < hi && __ldg(pre + idx) <= x;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    lo += (31 - __clz(m)) * step;
    hi = min(lo + step, hi);
  }
  return lo;
}

// Instance of each thread's agent f for a block whose agents start at f0:
// the first warp searches f0's instance and the block shares it; each
// thread then walks forward from there (a block's agents span few
// instances).  pre[n] is the total.  Blocks of at least 32 threads.
__device__ __forceinline__ int block_inst(const int *pre, int n, int f0, int f, int *sh) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int k = warp_find_inst(pre, n, f0);
    if (threadIdx.x == 0) *sh = k;
  }
  __syncthreads();
  int k = *sh;
  while (k + 1 < n && __ldg(pre + k + 1) <= f) ++k;
  return k;
}

// SPLIT: phases A-C only; the neighbour scan runs as the next launch
// (k_batch_neigh), where it has the registers of a kernel of its own.
template <int H, int V, bool SPLIT>
__global__ void __launch_bounds__(kBatchBlock, SPLIT ? 6 : 1) k_batch_step(const BatchDev *__restrict__ d, Inst *insts,
                                                          const int *__restrict__ apre,
                                                          const int *__restrict__ cpre,
                                                          unsigned *ctr, unsigned spin_limit) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int flag;
  __shared__ int wsum[33];
  const BatchDev D = *d;
  Bufs B = D.B;
  unsigned err = 0;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstride = gridDim.x * blockDim.x;

  // ---- phase A: apply actions and bin (Section 4.1: act, then observe) ----
  for (int f = gtid; f < D.n_total; f += gstride) {
    const int k = find_inst(apre, D.n_inst, f);
    const Inst &I = insts[k];
    phaseA_agent(I, f - I.agent_base, B.actions + I.agent_base, nullptr, I.reset, B.counts,
                 B.cellrank, err);
  }
  if (!grid_barrier(ctr, B.err, spin_limit, &flag)) goto done;

  // ---- phase B: scan of the cell counts ----
  for (int t = blockIdx.x; t < D.n_scan_tiles; t += gridDim.x)
    phaseB_tile(t, B, reinterpret_cast<int *>(smem));
  if (!grid_barrier(ctr, B.err, spin_limit, &flag)) goto done;

  // ---- phase C: scatter into cell order, cell starts ----
  {
    int *tp = reinterpret_cast<int *>(smem);
    tile_prefix(B, tp, wsum);
    for (int f = gtid; f < D.n_total; f += gstride) {
      const int k = find_inst(apre, D.n_inst, f);
      const Inst &I = insts[k];
      phaseC_agent(f, I.state + (f - I.agent_base), B, tp);
    }
    for (int c = gtid; c <= D.c_total; c += gstride) phaseC_cell(c, B, tp);
  }
  if (!grid_barrier(ctr, B.err, spin_limit, &flag)) goto done;

  // ---- phase D: neighbour scan, one chunk of 32 sorted agents per warp ----
  if (!SPLIT) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = V == 8 ? 8 : insts[0].v;
    char *wbase = smem + (size_t)warp * (sizeof(Inst) + direct_warp_bytes(v, 32, kQueue));
    Inst &sI = *reinterpret_cast<Inst *>(wbase);
    const DirectArea W = direct_area(wbase + sizeof(Inst), v, 32, kQueue);
    int cur = -1;
    for (;;) {
      int c = 0;
      if (lane == 0) c = (int)atomicAdd(&ctr[kCtrTicket], 1u);
      c = __shfl_sync(kFull, c, 0);
      if (c >= D.n_chunks) break;
      const int k = warp_find_inst(cpre, D.n_inst, c);
      if (k != cur) {
        const int *src = reinterpret_cast<const int *>(insts + k);
        int *dst = reinterpret_cast<int *>(&sI);
        for (int w = lane; w < (int)(sizeof(Inst) / 4); w += 32) dst[w] = src[w];
        __syncwarp();
        cur = k;
      }
      const int gp0 = sI.agent_base + (c - __ldg(cpre + k)) * 32;
      const int gp1 = min(gp0 + 32, sI.agent_base + sI.n);
      phaseD_direct<H, V, false>(sI, gp0, gp1, B, W, err);
      // an instance observed without actions goes back to normal stepping
      if (sI.reset && gp0 == sI.agent_base && lane == 0) insts[k].reset = 0;
    }
  }

done:
  if (err) atomicOr(B.err, err);
  // The last block out restores the counters for the next launch.  After an
  // abort the barrier count and the cell counts may be mid-step; the cell
  // counts are cleared here so that no later step scatters with them.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const bool last = atomicAdd(&ctr[kCtrExit], 1u) == gridDim.x - 1;
    flag = last ? (ld_acquire(&ctr[kCtrAbort]) ? 2 : 1) : 0;
  }
  __syncthreads();
  if (flag == 2)
    for (int c = threadIdx.x; c < D.c_total; c += blockDim.x) B.counts[c] = 0;
  if (flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(&ctr[kCtrBarCount], 0u);
      atomicExch(&ctr[kCtrTicket], 0u);
      atomicExch(&ctr[kCtrAbort], 0u);
      atomicExch(&ctr[kCtrExit], 0u);
    }
  }
}

// ---------------------------------------------------------------------------
// Binning as three kernels (mode 4), the single environment's form over the
// flattened agents and cells of all active instances: each kernel walks its
// work list with a grid-stride loop (a fixed grid serves every active set);
// the scan and scatter start under programmatic dependent launch.  No grid
// barrier: the kernel boundaries order the phases.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bbin_apply(const BatchDev *__restrict__ d,
                                                    const Inst *__restrict__ insts,
                                                    const int *__restrict__ apre, unsigned *ctr,
                                                    float2 *bxy) {
  const BatchDev D = *d;
  const Bufs &B = D.B;
  // the chunk ticket of this step's neighbour launch (the previous step's
  // launch has finished: this kernel starts after it in stream order)
  if (blockIdx.x == 0 && threadIdx.x == 0) ctr[kCtrTicket] = 0;
  __shared__ int k0;
  unsigned err = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int f0 = blockIdx.x * blockDim.x; f0 < D.n_total; f0 += stride) {
    const int f = f0 + threadIdx.x;
    const int k = block_inst(apre, D.n_inst, f0, f, &k0);
    if (f < D.n_total) {
      const Inst &I = insts[k];
      const int i = f - I.agent_base;
      const float4 st = phaseA_agent(I, i, B.actions + I.agent_base, nullptr, I.reset, B.counts,
                                     B.cellrank, err);
      bxy[f] = make_float2(st.x, st.y);  // the new position in agent order, for the scatter
    }
  }
  if (err) atomicOr(B.err, err);
}

__global__ void __launch_bounds__(256) k_bbin_scan(const BatchDev *__restrict__ d) {
  __shared__ int sm[kScanTile + 34];
  pdl_wait();
  const BatchDev D = *d;
  for (int t = blockIdx.x; t < D.n_scan_tiles; t += gridDim.x) phaseB_tile(t, D.B, sm);
}

// dynamic shared memory: (scan tiles + 1) ints of tile prefix.  Reads the
// new positions in agent order from bxy (written by k_bbin_apply), so it
// needs no instance lookup.
__global__ void __launch_bounds__(256) k_bbin_scatter(const BatchDev *__restrict__ d,
                                                      const float2 *__restrict__ bxy) {
  extern __shared__ int tp[];
  __shared__ int wsum[33];
  pdl_wait();
  const BatchDev D = *d;
  const Bufs &B = D.B;
  tile_prefix(B, tp, wsum);
  const int stride = gridDim.x * blockDim.x;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < D.n_total; f += stride) {
    const int2 cr = B.cellrank[f];
    if (!dbg_ok(cr.x >= 0 && cr.x < B.c_total && cr.y >= 0)) continue;
    const int pos = tp[cr.x / kScanTile] + B.local[cr.x] + cr.y;
    if ((unsigned)pos >= (unsigned)B.n_total) {  // inconsistent counts: never write out of range
      atomicOr(B.err, FLOCK_ERR_STATE);
      continue;
    }
    B.sxy[pos] = bxy[f];
    B.sidx[pos] = f;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= D.c_total; c += stride)
    phaseC_cell(c, B, tp);
}

// Phase D of the split forms, a launch of its own (so the wide direct scan of
// the standalone kernels has the registers it wants): every warp takes
// chunks of 32 / LPA cell-sorted agents, the first by its index in the grid
// (no atomic round trip before it starts), the rest from a shared ticket
// (zero when the binning ends; balances the load of a mix of instances),
// and keeps its copy of the instance descriptor while its chunks stay in one
// instance.  A step whose persistent binning launch (mode 3) gave up
// at a grid barrier (FLOCK_ERR_TIMEOUT latched) is left unobserved.
// LPA lanes per agent: a chunk is 32 / LPA agents (more lanes keep more warps
// busy when the batch holds few agents).
template <int H, int V, int LPA>
__device__ __forceinline__ void batch_neigh(const BatchDev *__restrict__ d, Inst *insts,
                                            const int *cpre, unsigned *ctr, int after_barriers) {
  constexpr int A = 32 / LPA;
  extern __shared__ __align__(16) char smem[];
  pdl_wait();
  const BatchDev D = *d;
  const Bufs &B = D.B;
  if (after_barriers && (ld_acquire(B.err) & FLOCK_ERR_TIMEOUT)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = V == 8 ? 8 : insts[0].v;
  char *wbase = smem + (size_t)warp * (sizeof(Inst) + direct_warp_bytes(v, A));
  Inst &sI = *reinterpret_cast<Inst *>(wbase);
  const DirectArea W = direct_area(wbase + sizeof(Inst), v, A);
  unsigned err = 0;
  int cur = -1;
  // first chunk: the warp's index in the grid (a block's warps take
  // consecutive chunks, no atomic before the first one); later chunks from
  // the shared ticket, fetched while the current chunk is scanned
  const int wpb = blockDim.x >> 5, nw = gridDim.x * wpb;
  int c = blockIdx.x * wpb + warp;
  while (c < D.n_chunks) {
    int nxt = 0;
    if (lane == 0) nxt = nw + (int)atomicAdd(&ctr[kCtrTicket], 1u);
    const int k = warp_find_inst(cpre, D.n_inst, c);
    if (k != cur) {
      const int *src = reinterpret_cast<const int *>(insts + k);
      int *dst = reinterpret_cast<int *>(&sI);
      for (int w = lane; w < (int)(sizeof(Inst) / 4); w += 32) dst[w] = src[w];
      __syncwarp();
      cur = k;
    }
    const int gp0 = sI.agent_base + (c - cpre[k]) * A;
    const int gp1 = min(gp0 + A, sI.agent_base + sI.n);
    phaseD_direct<H, V, true, LPA, false, true>(sI, gp0, gp1, B, W, err);
    if (sI.reset && gp0 == sI.agent_base && lane == 0) insts[k].reset = 0;
    c = __shfl_sync(kFull, nxt, 0);
  }
  if (err) atomicOr(B.err, err);
}

// The launches.  Registers: one lane per agent keeps the compiler's default
// for blocks of 256 (the large mixes, issue-bound, want the warps: the
// 256-instance mix takes 179.5 us a step, 181.2 at 80 registers); 2 or 4
// lanes get 80 registers and no spills (a batch of one 50,000-agent
// instance 31.6 us a step against 33.6 us at 64 with 24 bytes spilled).
template <int H, int V>
__global__ void __launch_bounds__(256) k_batch_neigh1(const BatchDev *__restrict__ d, Inst *insts,
                                                      const int *cpre, unsigned *ctr,
                                                      int after_barriers) {
  batch_neigh<H, V, 1>(d, insts, cpre, ctr, after_barriers);
}

template <int H, int V, int LPA>
__global__ void __launch_bounds__(256, 3) k_batch_neigh(const BatchDev *__restrict__ d,
                                                        Inst *insts, const int *cpre,
                                                        unsigned *ctr, int after_barriers) {
  batch_neigh<H, V, LPA>(d, insts, cpre, ctr, after_barriers);
}

static size_t neigh_smem(int v, int block, int lanes) {
  return (size_t)(block / 32) * (sizeof(Inst) + direct_warp_bytes(v, 32 / lanes));
}

// Dynamic shared memory of the persistent kernel: the scan tile or the prefix
// of max_tiles scan tiles, and (fused form) the per-warp areas of phase D.
// Sized by the batch's cell capacity, so that the binning-only kernel of the
// two-launch form fits six blocks per SM.
static size_t batch_smem(int v, bool split, int max_tiles) {
  const size_t scan = (size_t)(kScanTile + 34) * 4;
  const size_t prefix = (size_t)(max_tiles + 1) * 4;
  size_t m = scan > prefix ? scan : prefix;
  if (split) return m;
  const size_t warps =
      (size_t)(kBatchBlock / 32) * (sizeof(Inst) + direct_warp_bytes(v, 32, kQueue));
  return m > warps ? m : warps;
}

using KFn = void (*)(const BatchDev *, Inst *, const int *, const int *, unsigned *, unsigned);
using NFn = void (*)(const BatchDev *, Inst *, const int *, unsigned *, int);

// The V = 8 kernels write observation layout 0 only.
static KFn batch_kernel(int halo, int v, int layout, bool split) {
  const bool v8 = v == 8 && layout == 0;
  if (split) {
    if (halo == 1) return v8 ? k_batch_step<1, 8, true> : k_batch_step<1, 0, true>;
    return v8 ? k_batch_step<2, 8, true> : k_batch_step<2, 0, true>;
  }
  if (halo == 1) return v8 ? k_batch_step<1, 8, false> : k_batch_step<1, 0, false>;
  return v8 ? k_batch_step<2, 8, false> : k_batch_step<2, 0, false>;
}

static NFn neigh_kernel(int halo, int v, int layout, int lanes) {
  const bool v8 = v == 8 && layout == 0;
  static const NFn t[2][2][3] = {
      {{k_batch_neigh1<1, 0>, k_batch_neigh<1, 0, 2>, k_batch_neigh<1, 0, 4>},
       {k_batch_neigh1<1, 8>, k_batch_neigh<1, 8, 2>, k_batch_neigh<1, 8, 4>}},
      {{k_batch_neigh1<2, 0>, k_batch_neigh<2, 0, 2>, k_batch_neigh<2, 0, 4>},
       {k_batch_neigh1<2, 8>, k_batch_neigh<2, 8, 2>, k_batch_neigh<2, 8, 4>}}};
  return t[halo - 1][v8 ? 1 : 0][lanes == 1 ? 0 : (lanes == 2 ? 1 : 2)];
}

}  // namespace flock

using namespace flock;

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BLayout {
  size_t dev, insts, apre, cpre, ctr, err, cellrank, bxy, counts, local, cell_start, tile_sum, sxy,
      sidx, total;
};

BLayout batch_layout(int mi, int ma, int mc) {
  BLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) { size_t at = o; o = a256(o + b); return at; };
  const int nT = (mc + kScanTile - 1) / kScanTile;
  L.dev = take(2 * sizeof(BatchDev));  // two slots (see env_batch_step)
  L.insts = take((size_t)mi * sizeof(Inst));
  L.apre = take((size_t)(mi + 1) * 4);
  L.cpre = take((size_t)(mi + 1) * 4);
  L.ctr = take(64);
  L.err = take(64);
  L.cellrank = take((size_t)ma * 8);
  L.counts = take((size_t)mc * 4);
  L.local = take((size_t)mc * 4);
  L.cell_start = take((size_t)(mc + 1) * 4);
  L.tile_sum = take((size_t)(nT + 1) * 4);
  L.sxy = take((size_t)ma * 8);
  L.sidx = take((size_t)ma * 4);
  L.bxy = take((size_t)ma * 8);  // mode 4: new positions in agent order
  L.total = o;
  return L;
}

}  // namespace

struct flock_batch {
  int max_inst, max_agents, max_cells;
  flock_tuning tuning;
  BLayout lay;
  char *ws;
  cudaStream_t stream, cap_stream;
  cudaGraphExec_t graph;
  int grid, v, halo, layout;
  int mode;        // 2: fused persistent; 3: persistent binning + neighbour launch;
                   // 4: binning kernels + neighbour launch
  bool split;      // the neighbour scan is a launch of its own (modes 3, 4)
  bool kbin;       // binning by three kernels (mode 4)
  int nblock;      // threads per block of the neighbour launch
  int lanes;       // lanes per agent of the neighbour launch (chunks of 32 / lanes agents)
  int neigh_grid;  // blocks of the split form's neighbour launch (all resident)
  int bin_grid, scan_grid, scatter_grid;  // mode 4 binning kernels (grid-stride)
  unsigned spin_limit;
  BatchDev dev;  // host copy
  std::vector<Inst> insts;
  std::vector<int> apre, cpre;
  // Two descriptor slots in device memory, each with the output pointers of
  // the steps that use it and a graph reading it: a caller alternating two
  // sets of outputs re-uploads nothing per step.
  struct Slot {
    const void *act, *obs, *rew, *coll;
    cudaGraphExec_t graph;
    bool dirty;  // the device copy is older than the host's
  } slot[2];
  int last;  // slot of the last step
  // Derived descriptors of parameter sets seen before, keyed by the
  // parameter bytes: a serving session's set is derived once, not at every
  // change of the active set.  Cleared when it outgrows 4 x max_inst.
  std::unordered_map<std::string, Inst> derived;
  int timing;
  cudaEvent_t ev[2];
  bool configured;
  // Page-locked staging of the uploads (a copy from pageable memory may wait
  // for the stream, which would stall a caller that keeps steps in flight):
  // two halves for the set's descriptors and prefixes, used in turn, and one
  // BatchDev per slot; an event per buffer marks when its copy has left.
  char *hset = nullptr;
  size_t hset_half = 0;
  int hset_cur = 0;
  cudaEvent_t hset_ev[2] = {nullptr, nullptr};
  bool hset_used[2] = {false, false};
  BatchDev *hdev = nullptr;
  cudaEvent_t hdev_ev[2] = {nullptr, nullptr};
  bool hdev_used[2] = {false, false};
};

// Frees what env_batch_create made besides the workspace.
static void batch_free(flock_batch *b) {
  for (int k = 0; k < 2; ++k) {
    if (b->hset_ev[k]) cudaEventDestroy(b->hset_ev[k]);
    if (b->hdev_ev[k]) cudaEventDestroy(b->hdev_ev[k]);
  }
  if (b->hset) cudaFreeHost(b->hset);
  if (b->hdev) cudaFreeHost(b->hdev);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

extern "C" int flock_instance_cells(const flock_params *p, const flock_tuning *t, int *cells) {
  if (!p || !cells) return FLOCK_EINVAL;
  Inst I;
  int rc = derive(*p, (t && t->stencil) ? t->stencil : 1, I, nullptr);
  if (rc) return rc;
  *cells = I.ncells;
  return FLOCK_OK;
}

extern "C" int flock_batch_workspace_bytes(int mi, int ma, int mc, const flock_tuning *t,
                                           size_t *bytes) {
  (void)t;
  if (!bytes || mi < 1 || ma < 0 || mc < 1 || mc > kMaxScanTiles * kScanTile) return FLOCK_EINVAL;
  *bytes = batch_layout(mi, ma, mc).total;
  return FLOCK_OK;
}

#define BCK(call)                                       \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

extern "C" int env_batch_create(int mi, int ma, int mc, const flock_tuning *t, void *ws,
                                size_t ws_bytes, void *stream, flock_batch **out) {
  NvtxRange nvtx_range("flock:env_batch_create");
  if (!out) return FLOCK_EINVAL;
  *out = nullptr;
  if (mi < 1 || ma < 0 || mc < 1 || mc > kMaxScanTiles * kScanTile) return FLOCK_EINVAL;
  flock_batch *b = new (std::nothrow) flock_batch();
  if (!b) return FLOCK_EINVAL;
  b->max_inst = mi;
  b->max_agents = ma;
  b->max_cells = mc;
  b->tuning = flock_tuning{};
  if (t) b->tuning = *t;
  b->halo = b->tuning.stencil ? b->tuning.stencil : 1;
  if (b->halo != 1 && b->halo != 2) { delete b; return FLOCK_EINVAL; }
  b->tuning.stencil = b->halo;
  // mode 2: one persistent launch runs every phase; mode 3: the persistent
  // launch bins (phases A-C) and a second launch runs the neighbour scan;
  // mode 4 (the default, the fastest measured on mixes of 10 to 256
  // instances): three binning kernels, then the neighbour launch
  b->mode = b->tuning.mode ? b->tuning.mode : 4;
  if (b->mode < 2 || b->mode > 4) {
    delete b;
    return FLOCK_EINVAL;
  }
  b->split = b->mode != 2;
  b->kbin = b->mode == 4;
  // tuning.block: the neighbour launch's block in the split forms
  b->nblock = b->split ? (b->tuning.block ? b->tuning.block : 128) : kBatchBlock;
  if (b->nblock < 64 || b->nblock > 256 || b->nblock % 32) {
    delete b;
    return FLOCK_EINVAL;
  }
  // lanes per agent (the separate neighbour launch): as for one environment,
  // by the most agents the batch holds; the one-launch form takes one
  b->lanes = !b->split ? 1 : (b->tuning.lanes ? b->tuning.lanes
                                               : (ma <= 32768 ? 4 : (ma <= 524288 ? 2 : 1)));
  if (b->lanes != 1 && b->lanes != 2 && b->lanes != 4) {
    delete b;
    return FLOCK_EINVAL;
  }
  b->tuning.mode = b->mode;
  b->tuning.block = b->nblock;
  b->tuning.lanes = b->lanes;
  b->lay = batch_layout(mi, ma, mc);
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < b->lay.total) { delete b; return FLOCK_ENOSPACE; }
  b->ws = (char *)ws;
  b->stream = (cudaStream_t)stream;
  b->spin_limit = 1u << 22;
  b->v = 0;
  b->layout = 0;
  int dev = 0, coop = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!coop && !b->kbin) { delete b; return FLOCK_EINVAL; }
  // grid-stride binning kernels: a few resident blocks per SM
  b->bin_grid = 8 * sms;
  b->scatter_grid = 4 * sms;
  const int max_tiles = (mc + kScanTile - 1) / kScanTile;
  b->scan_grid = max_tiles < 4 * sms ? max_tiles : 4 * sms;
  cudaError_t ce = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (ce != cudaSuccess) { delete b; return cuda_fail(ce, "cudaStreamCreate"); }
  const BLayout &L = b->lay;
  ce = cudaMemsetAsync(b->ws + L.counts, 0, (size_t)mc * 4, b->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(b->ws + L.ctr, 0, 64, b->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(b->ws + L.err, 0, 64, b->stream);
  if (ce != cudaSuccess) {
    batch_free(b);
    return cuda_fail(ce, "env_batch_create memset");
  }
  b->hset_half = ((size_t)mi * sizeof(Inst) + 2 * ((size_t)mi + 1) * 4 + 255) & ~(size_t)255;
  ce = cudaHostAlloc((void **)&b->hset, 2 * b->hset_half, cudaHostAllocDefault);
  if (ce == cudaSuccess) ce = cudaHostAlloc((void **)&b->hdev, 2 * sizeof(BatchDev), cudaHostAllocDefault);
  for (int k = 0; k < 2 && ce == cudaSuccess; ++k) {
    ce = cudaEventCreateWithFlags(&b->hset_ev[k], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->hdev_ev[k], cudaEventDisableTiming);
  }
  if (ce != cudaSuccess) {
    batch_free(b);
    return cuda_fail(ce, "env_batch_create staging");
  }
  *out = b;
  return FLOCK_OK;
}

// Destroys the slots' graphs (re-captured at the next step), after the
// stream has finished with them.
static cudaError_t drop_graphs(flock_batch *b) {
  if (!b->slot[0].graph && !b->slot[1].graph) return cudaSuccess;
  const cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 2; ++k)
    if (b->slot[k].graph) {
      cudaGraphExecDestroy(b->slot[k].graph);
      b->slot[k].graph = nullptr;
    }
  return cudaSuccess;
}

extern "C" int env_batch_set(flock_batch *b, int n_inst, const flock_params *params,
                             const int *n_agents, float *const *state, const int *reset) {
  NvtxRange nvtx_range("flock:env_batch_set");
  if (!b || n_inst < 0 || n_inst > b->max_inst || (n_inst > 0 && (!params || !n_agents || !state)))
    return FLOCK_EINVAL;
  std::vector<Inst> ins((size_t)(n_inst > 0 ? n_inst : 1));
  std::vector<int> apre((size_t)n_inst + 1), cpre((size_t)n_inst + 1);
  long long na = 0, ncell = 0, nchunk = 0;
  int v = 0, layout = 0;
  for (int k = 0; k < n_inst; ++k) {
    Inst &I = ins[k];
    const std::string key(reinterpret_cast<const char *>(&params[k]), sizeof(flock_params));
    auto hit = b->derived.find(key);
    if (hit != b->derived.end()) {
      I = hit->second;
    } else {
      int rc = derive(params[k], b->halo, I, nullptr);
      if (rc) return rc;
      if (b->derived.size() >= (size_t)4 * b->max_inst) b->derived.clear();
      b->derived.emplace(key, I);
    }
    if (n_agents[k] < 0 || (n_agents[k] > 0 && !state[k])) return FLOCK_EINVAL;
    if (k == 0) {
      v = I.v;
      layout = I.obs_layout;
    }
    // one sector count and one observation layout per batch (rows are
    // flattened with a single row length)
    if (I.v != v || I.obs_layout != layout) return FLOCK_EINVAL;
    if (I.kind != 0) return FLOCK_EINVAL;  // the batch steps flock instances
    I.n = n_agents[k];
    I.n_own = n_agents[k];
    I.state = reinterpret_cast<float4 *>(state[k]);
    I.agent_base = (int)na;
    I.cell_base = (int)ncell;
    I.chunk_base = (int)nchunk;
    I.obs_base = na * (long long)I.obs_dim;
    I.reset = reset ? (reset[k] != 0) : 0;
    apre[k] = (int)na;
    cpre[k] = (int)nchunk;
    na += I.n;
    ncell += I.ncells;
    nchunk += (I.n + 32 / b->lanes - 1) / (32 / b->lanes);
    if (na > b->max_agents || ncell > b->max_cells) return FLOCK_EINVAL;
  }
  apre[n_inst] = (int)na;
  cpre[n_inst] = (int)nchunk;
  if (n_inst > 0 && (v != b->v || layout != b->layout)) {
    // the kernel variant (and its shared memory) depends on v and the layout
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!b->kbin) {
      KFn fn = batch_kernel(b->halo, v, layout, b->split);
      const size_t sm = batch_smem(v, b->split, (b->max_cells + kScanTile - 1) / kScanTile);
      BCK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kBatchBlock, sm));
      if (per < 1) return FLOCK_EINVAL;  // too many sectors for one block
      b->grid = per * sms;
    } else {
      b->grid = b->bin_grid;
    }
    if (b->split) {
      NFn nf = neigh_kernel(b->halo, v, layout, b->lanes);
      const size_t nsm = neigh_smem(v, b->nblock, b->lanes);
      int pn = 0;
      BCK(cudaFuncSetAttribute(nf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm));
      BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pn, nf, b->nblock, nsm));
      if (pn < 1) return FLOCK_EINVAL;
      b->neigh_grid = pn * sms;
    }
    b->v = v;
    b->layout = layout;
    BCK(drop_graphs(b));
  }
  const BLayout &L = b->lay;
  BatchDev &D = b->dev;
  D.n_inst = n_inst;
  D.n_total = (int)na;
  D.c_total = (int)ncell;
  D.n_scan_tiles = n_inst > 0 ? (int)((ncell + kScanTile - 1) / kScanTile) : 0;
  D.n_chunks = (int)nchunk;
  Bufs &B = D.B;
  B.cellrank = (int2 *)(b->ws + L.cellrank);
  B.counts = (int *)(b->ws + L.counts);
  B.local = (int *)(b->ws + L.local);
  B.cell_start = (int *)(b->ws + L.cell_start);
  B.tile_sum = (int *)(b->ws + L.tile_sum);
  B.sxy = (float2 *)(b->ws + L.sxy);
  B.sidx = (int *)(b->ws + L.sidx);
  B.err = (unsigned *)(b->ws + L.err);
  B.bar = (unsigned *)(b->ws + L.ctr);
  B.n_total = D.n_total;
  B.c_total = D.c_total;
  B.n_scan_tiles = D.n_scan_tiles;
  b->insts.swap(ins);
  b->apre.swap(apre);
  b->cpre.swap(cpre);
  if (n_inst > 0) {
    // through the staging half not used last, once its previous copy has left
    const int h = b->hset_cur ^= 1;
    if (b->hset_used[h]) BCK(cudaEventSynchronize(b->hset_ev[h]));
    char *hs = b->hset + (size_t)h * b->hset_half;
    const size_t bi = (size_t)n_inst * sizeof(Inst), bp = ((size_t)n_inst + 1) * 4;
    memcpy(hs, b->insts.data(), bi);
    memcpy(hs + bi, b->apre.data(), bp);
    memcpy(hs + bi + bp, b->cpre.data(), bp);
    BCK(cudaMemcpyAsync(b->ws + L.insts, hs, bi, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(b->ws + L.apre, hs + bi, bp, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(b->ws + L.cpre, hs + bi + bp, bp, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaEventRecord(b->hset_ev[h], b->stream));
    b->hset_used[h] = true;
  }
  b->slot[0].dirty = b->slot[1].dirty = true;  // both descriptors re-uploaded when next used
  b->configured = true;
  return FLOCK_OK;
}

static int batch_enqueue_persistent(flock_batch *b, cudaStream_t s, const BatchDev *dv);

static int batch_enqueue(flock_batch *b, cudaStream_t s, int k) {
  const BLayout &L = b->lay;
  if (b->timing) BCK(cudaEventRecordWithFlags(b->ev[0], s, cudaEventRecordExternal));
  const BatchDev *dv = (const BatchDev *)(b->ws + L.dev) + k;
  Inst *ins = (Inst *)(b->ws + L.insts);
  const int *apre = (const int *)(b->ws + L.apre);
  const int *cpre = (const int *)(b->ws + L.cpre);
  unsigned *ctr = (unsigned *)(b->ws + L.ctr);
  if (b->kbin) {
    NvtxRange r("flock:batch_binning");
    const int max_tiles = (b->max_cells + kScanTile - 1) / kScanTile;
    float2 *bxy = (float2 *)(b->ws + L.bxy);
    BCK(launch(false, k_bbin_apply, b->bin_grid, 256, 0, s, dv, (const Inst *)ins, apre, ctr,
               bxy));
    BCK(launch(true, k_bbin_scan, b->scan_grid, 256, 0, s, dv));
    BCK(launch(true, k_bbin_scatter, b->scatter_grid, 256, (size_t)(max_tiles + 1) * 4, s, dv,
               (const float2 *)bxy));
  } else {
    const int rc = batch_enqueue_persistent(b, s, dv);
    if (rc) return rc;
  }
  if (b->split) {
    NvtxRange r("flock:batch_neighbours");
    BCK(launch(b->kbin, neigh_kernel(b->halo, b->v, b->layout, b->lanes), b->neigh_grid,
               b->nblock, neigh_smem(b->v, b->nblock, b->lanes), s, dv, ins, cpre, ctr,
               b->mode == 3 ? 1 : 0));
  }
  if (b->timing) BCK(cudaEventRecordWithFlags(b->ev[1], s, cudaEventRecordExternal));
  return FLOCK_OK;
}

static int batch_enqueue_persistent(flock_batch *b, cudaStream_t s, const BatchDev *dv) {
  const BLayout &L = b->lay;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(kBatchBlock);
  cfg.dynamicSmemBytes = batch_smem(b->v, b->split, (b->max_cells + kScanTile - 1) / kScanTile);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  KFn fn = batch_kernel(b->halo, b->v, b->layout, b->split);
  NvtxRange r("flock:batch_persistent");
  BCK(cudaLaunchKernelEx(&cfg, fn, dv, (Inst *)(b->ws + L.insts),
                         (const int *)(b->ws + L.apre), (const int *)(b->ws + L.cpre),
                         (unsigned *)(b->ws + L.ctr), b->spin_limit));
  return FLOCK_OK;
}

extern "C" int env_batch_step(flock_batch *b, const int32_t *act, float *obs, float *rew,
                              int32_t *coll) {
  NvtxRange nvtx_range("flock:env_batch_step");
  if (!b || !b->configured) return FLOCK_EINVAL;
  if (b->dev.n_total == 0) return FLOCK_OK;
  if (!act || !obs || !rew || !coll || ((uintptr_t)obs & 7)) return FLOCK_EINVAL;
  // the slot holding these pointers, else the one not used last
  int k = -1;
  for (int j = 0; j < 2; ++j) {
    const flock_batch::Slot &q = b->slot[j];
    if (q.act == act && q.obs == obs && q.rew == rew && q.coll == coll) k = j;
  }
  if (k < 0) {
    k = b->last ^ 1;
    flock_batch::Slot &q = b->slot[k];
    q.act = act;
    q.obs = obs;
    q.rew = rew;
    q.coll = coll;
    q.dirty = true;  // the graph reads the slot's descriptor: no re-capture needed
  }
  flock_batch::Slot &q = b->slot[k];
  if (q.dirty) {
    b->dev.B.actions = act;
    b->dev.B.obs = obs;
    b->dev.B.reward = rew;
    b->dev.B.coll = coll;
    if (b->hdev_used[k]) BCK(cudaEventSynchronize(b->hdev_ev[k]));
    b->hdev[k] = b->dev;
    BCK(cudaMemcpyAsync((BatchDev *)(b->ws + b->lay.dev) + k, b->hdev + k, sizeof(BatchDev),
                        cudaMemcpyHostToDevice, b->stream));
    BCK(cudaEventRecord(b->hdev_ev[k], b->stream));
    b->hdev_used[k] = true;
    q.dirty = false;
  }
  if (!q.graph) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = batch_enqueue(b, b->cap_stream, k);
    cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&q.graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      q.graph = nullptr;
      return cuda_fail(ce, "cudaGraphInstantiate");
    }
  }
  b->last = k;
  BCK(cudaGraphLaunch(q.graph, b->stream));
  return FLOCK_OK;
}

#ifdef FLOCK_DEBUG
// Debug build: takes (reads and clears) this translation unit's latched
// FLOCK_ERR_BOUNDS word; waits for the stream.
static unsigned dbg_take(cudaStream_t s) {
  unsigned w = 0;
  const unsigned z = 0;
  if (cudaMemcpyFromSymbolAsync(&w, flock::g_flock_dbg_bits, 4, 0, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyToSymbolAsync(flock::g_flock_dbg_bits, &z, 4, 0, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FLOCK_ERR_BOUNDS;  // could not read it: report the check as failed
  return w;
}
#endif

extern "C" int env_batch_get_error(flock_batch *b, uint32_t *bits) {
  NvtxRange nvtx_range("flock:env_batch_get_error");
  if (!b || !bits) return FLOCK_EINVAL;
  uint32_t w = 0;
  BCK(cudaMemcpyAsync(&w, b->ws + b->lay.err, 4, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaMemsetAsync(b->ws + b->lay.err, 0, 4, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (w & FLOCK_ERR_TIMEOUT) {
    // the kernel restored its counters on the way out; clear them once more
    // from the host in case the step was cut short in an unforeseen place
    BCK(cudaMemsetAsync(b->ws + b->lay.ctr, 0, 64, b->stream));
    BCK(cudaMemsetAsync(b->ws + b->lay.counts, 0, (size_t)b->max_cells * 4, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
  }
#ifdef FLOCK_DEBUG
  w |= dbg_take(b->stream);
#endif
  *bits = w;
  return FLOCK_OK;
}

extern "C" int env_batch_set_spin_limit(flock_batch *b, unsigned limit) {
  if (!b) return FLOCK_EINVAL;
  BCK(drop_graphs(b));
  b->spin_limit = limit;
  return FLOCK_OK;
}

extern "C" int env_batch_get_launch(const flock_batch *b, int *grid, int *block) {
  if (!b || !grid || !block) return FLOCK_EINVAL;
  *grid = b->grid;
  *block = kBatchBlock;
  return FLOCK_OK;
}

extern "C" int env_batch_set_timing(flock_batch *b, int enable) {
  if (!b) return FLOCK_EINVAL;
  if (enable && !b->ev[0])
    for (int k = 0; k < 2; ++k) BCK(cudaEventCreate(&b->ev[k]));
  if ((enable != 0) != (b->timing != 0)) BCK(drop_graphs(b));
  b->timing = enable != 0;
  return FLOCK_OK;
}

extern "C" int env_batch_get_time(flock_batch *b, float *ms) {
  if (!b || !ms || !b->timing) return FLOCK_EINVAL;
  BCK(cudaEventSynchronize(b->ev[1]));
  BCK(cudaEventElapsedTime(ms, b->ev[0], b->ev[1]));
  return FLOCK_OK;
}

extern "C" void env_batch_destroy(flock_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  for (int k = 0; k < 2; ++k)
    if (b->slot[k].graph) cudaGraphExecDestroy(b->slot[k].graph);
  batch_free(b);
}
