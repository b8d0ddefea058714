// Kernels and C ABI of the single-instance flock environment step
// (arXiv 2207.03945, Section 4.1, Eq. 1, Fig. 3, Fig. 4).  See flock.h.
//
// A step is four kernels on the caller's stream, replayed as one CUDA graph:
//   k_apply_bin   phase A   one thread per agent
//   k_scan        phase B   one block per scan tile of 1024 cells
//   k_scatter     phase C   grid-stride over agents and cells
//   k_neighbours  phase D   one block per tile of cells
// or, for at most kFusedScanCells cells, three: the last block of
// k_apply_bin scans all cells (phase B), and k_scatter reads final starts.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "flock_device.cuh"
#include "flock_host.h"

namespace flock {

// The fused scan: one block of kFusedBlock threads, kFusedRounds rounds of
// 4 cells a lane held in registers, so at most kFusedScanCells cells.  It
// pays below about 8k cells (5,000 agents: 21.7 us a step against 23.7 us
// with the separate scan; even at 20,000, slower at 50,000, where the
// separate scan kernel's launch overlaps the binning under programmatic
// dependent launch and one block's scan of 20k cells takes ~4 us).
constexpr int kFusedBlock = 1024;
constexpr int kFusedRounds = 2;
constexpr int kFusedScanCells = kFusedBlock * 4 * kFusedRounds;

// FUSED: blocks of kFusedBlock threads; the last block to finish its agents
// (a ticket in B.bar[0], taken after a fence, so every count atomic of the
// other blocks is complete) scans all cell counts into cell_start and resets
// the ticket.  No block waits for another.
// The policy step (B.wimg set) launches extra blocks past the agents' ones;
// they write the network's operand image while the others bin the agents.
template <bool FUSED>
__global__ void __launch_bounds__(FUSED ? kFusedBlock : 256)
    k_apply_bin(const Inst *__restrict__ gI, Bufs B, int reset) {
  __shared__ Inst sI;
  load_inst(sI, gI);
  __syncthreads();
  unsigned err = 0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < sI.n)
    phaseA_agent(sI, i, B.actions + sI.agent_base, B.cactions ? B.cactions + sI.agent_base : nullptr,
                 reset, B.counts, B.cellrank, err);
  if (err) atomicOr(B.err, err);
  // the policy step: the network's operand image, read three kernels later,
  // by the blocks past the agents' ones
  if (B.wimg) {
    const int first = (sI.n + blockDim.x - 1) / blockDim.x * blockDim.x;
    if (i >= first) policy_image(B.wblob, B.wimg, i - first, gridDim.x * blockDim.x - first);
  }
  if (FUSED) {
    // every count atomic of this block has returned (complete in L2); the
    // barrier and thread 0's fence order them before the ticket
    __shared__ int last;
    __shared__ int wsum[33];
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(B.bar, 1u) == gridDim.x - 1;
      if (last) __threadfence();
    }
    __syncthreads();
    if (last) {
      scan_cells_block<kFusedRounds>(B, wsum);
      if (threadIdx.x == 0) *B.bar = 0u;
    }
  }
}

__global__ void __launch_bounds__(256) k_scan(Bufs B) {
  __shared__ int sm[kScanTile + 34];
  pdl_wait();
  phaseB_tile(blockIdx.x, B, sm);
}

__global__ void __launch_bounds__(256) k_scatter(const Inst *__restrict__ gI, Bufs B) {
  __shared__ int tp[kMaxScanTiles + 1];
  __shared__ int wsum[33];
  pdl_wait();
  tile_prefix(B, tp, wsum);
  const float4 *state = gI->state;
  const int stride = gridDim.x * blockDim.x;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < B.n_total; f += stride)
    phaseC_agent(f, state + f, B, tp);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= B.c_total; c += stride)
    phaseC_cell(c, B, tp);
}

// Phase C after the fused scan: the cell starts are final.
__global__ void __launch_bounds__(256) k_scatter_final(const Inst *__restrict__ gI, Bufs B) {
  pdl_wait();
  const float4 *state = gI->state;
  const int stride = gridDim.x * blockDim.x;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < B.n_total; f += stride)
    phaseC_agent_final(f, state + f, B);
}

template <int H>
__global__ void k_neighbours(const Inst *__restrict__ gI, Bufs B) {
  extern __shared__ __align__(16) char smem[];
  __shared__ Inst sI;
  load_inst(sI, gI);
  pdl_wait();
  __syncthreads();
  unsigned err = 0;
  const int t = blockIdx.x;
  phaseD_tile<H>(sI, t % sI.tiles_x, t / sI.tiles_x, B, smem, err);
  if (err) atomicOr(B.err, err);
}

// LPA lanes per agent: each warp takes 32 / LPA consecutive sorted agents
// (AORDER: consecutive agents in agent order, their observation rows written
// as one block; the host-buffer step's form, whose outputs are in mapped host
// memory).  TAG: the tag environment (two colour channels of sectors).  COMPACT: the
// runs across the square's edges walked by one loop instead of nine inlined
// copies (a warp per agent with a wide view: the paper's flock 126.7 us a
// step against 141.3, tag 152.2 against 181.5, from fewer instruction-fetch
// stalls; with few candidates, 1,000 agents, the inlined runs are faster).
template <int H, int V, int LPA, bool TAG = false, bool COMPACT = false, bool AORDER = false>
__global__ void k_neighbours_direct(const Inst *__restrict__ gI, Bufs B) {
  extern __shared__ __align__(16) char smem[];
  __shared__ Inst sI;
  load_inst(sI, gI);
  pdl_wait();
  __syncthreads();
  unsigned err = 0;
  const int warp = threadIdx.x >> 5;
  constexpr int A = 32 / LPA;
  const int gp0 = (blockIdx.x * (blockDim.x >> 5) + warp) * A;
  if (gp0 < sI.n) {
    const int vs = TAG ? 2 * sI.v : sI.v;
    const DirectArea W = direct_area(smem + (size_t)warp * direct_warp_bytes(vs, A), vs, A);
    phaseD_direct<H, V, true, LPA, TAG, COMPACT, false, AORDER>(sI, gp0, min(gp0 + A, sI.n), B, W,
                                                                 err);
  }
  if (err) atomicOr(B.err, err);
}

// The policy step's neighbour scan with the shared policy network (Section
// 4.3; 18 -> 64 -> 64 -> 9 with tanh) in its epilogue: each warp, once its
// agents' observations are complete in its sector arrays, runs the network
// on them on the tensor cores (policy_warp_rows: mma.sync, BF16 operands,
// FP32 accumulate; the weights from the operand image the binning kernel
// built, L1-resident) and writes their greedy actions (largest logit, lowest
// index on ties) and optionally the logits.  No observation goes through
// memory on the way, and the step keeps its four kernels.  The network's
// accumulators are held by halves of 32 columns, so the kernel needs no
// more registers than the scan (a form with a fifth kernel reading BF16
// observation rows from L2 took 44.3 us a step at 100,000 agents, this one
// 42.2 us).
template <int H, int V, int LPA>
__global__ void k_neighbours_policy(const Inst *__restrict__ gI, Bufs B) {
  extern __shared__ __align__(16) char smem[];
  __shared__ Inst sI;
  load_inst(sI, gI);
  pdl_wait();
  __syncthreads();
  unsigned err = 0;
  const int warp = threadIdx.x >> 5;
  constexpr int A = 32 / LPA;
  const int gp0 = (blockIdx.x * (blockDim.x >> 5) + warp) * A;
  if (gp0 < sI.n) {
    const DirectArea W = direct_area(smem + (size_t)warp * direct_warp_bytes(sI.v, A), sI.v, A);
    phaseD_direct<H, V, true, LPA, false, false, true>(sI, gp0, min(gp0 + A, sI.n), B, W, err);
  }
  if (err) atomicOr(B.err, err);
}

// Copies a step's outputs (observations, rewards, collision counts) from the
// workspace to page-locked, mapped host buffers: one kernel instead of one
// copy per buffer, 16 bytes per store where both ends are 16-byte aligned
// (else 4).  Every size is a multiple of 4 bytes and every pointer 4-byte
// aligned (checked by the host).
struct CopyOut {
  const char *src[3];
  char *dst[3];
  size_t bytes[3];
};

__global__ void __launch_bounds__(256) k_copy_out(CopyOut J) {
  pdl_wait();
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const char *src = J.src[k];
    char *dst = J.dst[k];
    const size_t nb = J.bytes[k];
    size_t done = 0;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
      const size_t n16 = nb / 16;
      const int4 *s4 = reinterpret_cast<const int4 *>(src);
      int4 *d4 = reinterpret_cast<int4 *>(dst);
      for (size_t t = tid; t < n16; t += stride) d4[t] = s4[t];
      done = n16 * 16;
    }
    for (size_t t = done + tid * 4; t < nb; t += stride * 4)
      *reinterpret_cast<int *>(dst + t) = *reinterpret_cast<const int *>(src + t);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static thread_local char g_last_cuda_error[256] = "";

int cuda_fail(cudaError_t e, const char *what) {
  snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s: %s", what, cudaGetErrorString(e));
  return FLOCK_ECUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Derived constants, written out from the model definition: validate the
// parameters, then compute everything a kernel needs in double where a
// transcendental is involved and round once to float.
int derive(const flock_params &p, int stencil, Inst &I, flock_derived *D) {
  memset(&I, 0, sizeof I);
  const double kPi = 3.14159265358979323846;
  const float vals[] = {p.side, p.view_radius, p.fov, p.agent_radius, p.collision_penalty,
                        p.speed_min, p.speed_max, p.speed_step, p.turn_step};
  for (float x : vals)
    if (!std::isfinite(x)) return FLOCK_EINVAL;
  if (p.num_segments < 1 || p.num_segments > FLOCK_MAX_SEGMENTS) return FLOCK_EINVAL;
  if (!(p.view_radius > 0.0f) || !(p.agent_radius >= 0.0f)) return FLOCK_EINVAL;
  if (!(2.0f * p.agent_radius < p.view_radius)) return FLOCK_EINVAL;
  if (!(p.side > 2.0f * p.view_radius)) return FLOCK_EINVAL;
  if (!(p.speed_min >= 0.0f && p.speed_min <= p.speed_max && p.speed_max < p.side))
    return FLOCK_EINVAL;
  if (!(p.collision_penalty >= 0.0f) || !(p.speed_step >= 0.0f)) return FLOCK_EINVAL;
  if (!(p.turn_step >= 0.0f && p.turn_step < (float)kPi)) return FLOCK_EINVAL;
  const float two_pi = (float)(2.0 * kPi);
  if (!(p.fov > 0.0f && p.fov <= two_pi)) return FLOCK_EINVAL;

  I.L = p.side;
  I.HL = 0.5f * p.side;
  I.RV = p.view_radius;
  I.RV2 = p.view_radius * p.view_radius;
  const float two_dr = 2.0f * p.agent_radius;
  I.RC2 = two_dr * two_dr;
  I.INV_SPAN = (float)(1.0 / ((double)p.view_radius - 2.0 * (double)p.agent_radius));
  I.TWO_PI = two_pi;
  I.SMIN = p.speed_min;
  I.SMAX = p.speed_max;
  I.v = p.num_segments;
  I.full = p.fov == two_pi;
  const double fov = I.full ? 2.0 * kPi : (double)p.fov;
  if (I.full) {
    I.CF = -1.0f;  // full circle: sector 0 starts straight behind the agent
    I.SF = 0.0f;
  } else {
    I.CF = (float)cos(0.5 * fov);
    I.SF = (float)sin(0.5 * fov);
  }
  auto pseudo = [](double x, double y) {
    if (y >= 0.0) return x >= 0.0 ? y / (x + y) : 1.0 + (-x) / (-x + y);
    return x < 0.0 ? 2.0 + (-y) / (-x - y) : 3.0 + x / (x - y);
  };
  for (int m = 1; m <= I.v; ++m) {
    const double phi = (double)m * fov / (double)I.v;
    I.T[m] = (float)pseudo(cos(phi), sin(phi));
  }
  I.DT[0] = -p.turn_step; I.DT[1] = 0.0f; I.DT[2] = p.turn_step;
  I.DS[0] = -p.speed_step; I.DS[1] = 0.0f; I.DS[2] = p.speed_step;
  // the strict range test must not admit a distance above d_v
  if (sqrtf(nextafterf(I.RV2, 0.0f)) > p.view_radius) return FLOCK_EINVAL;

  // resolution of the exact reward sum: every ramp term is a float no smaller
  // than the one made by the largest float below d_v, so a multiple of
  // 2^(e - 24) for that float's exponent e; the penalty must be one too
  const float rv = p.view_radius;
  const float t_min = (rv - nextafterf(rv, 0.0f)) * I.INV_SPAN;
  if (!(t_min > 0.0f)) return FLOCK_EINVAL;
  int e = 0;
  frexpf(t_min, &e);
  int K = 24 - e;
  if (p.collision_penalty > 0.0f) {
    int ep = 0;
    frexpf(p.collision_penalty, &ep);
    K = K > 24 - ep ? K : 24 - ep;
  }
  if (K < 0) K = 0;
  if (K > 60) return FLOCK_EINVAL;
  const float t_max = (rv - sqrtf(I.RC2)) * I.INV_SPAN;
  double mt = (double)t_max > (double)p.collision_penalty ? (double)t_max : (double)p.collision_penalty;
  if (mt < 1.0) mt = 1.0;
  const double nmax = floor(ldexp(1.0, 62) / ldexp(mt, K));
  if (nmax < 1.0) return FLOCK_EINVAL;
  I.NMAX = nmax > 9.0e15 ? (long long)9.0e15 : (long long)nmax;
  I.K = K;
  // a term is at most max(t_max, P) * 2^K (P: a tag chaser's term); two
  // 24-bit pieces hold it when that is < 2^48
  const double term_max = (double)t_max > (double)p.collision_penalty ? (double)t_max
                                                                       : (double)p.collision_penalty;
  I.pieces = ldexp(term_max, K) < ldexp(1.0, 48) ? 2 : 3;
  I.scaleK = ldexpf(1.0f, K);
  I.inv_scaleK = ldexpf(1.0f, -K);
  const double pk = ldexp((double)p.collision_penalty, K);
  I.PK = (long long)pk;
  if ((double)I.PK != pk) return FLOCK_EINVAL;

  // cell list: cells at least d_v (3 x 3 stencil) or d_v / 2 (5 x 5) wide,
  // widened by a relative 2^-20 and by L * 2^-21 so that the float binning
  // of x * (nc / L) can never hide an in-range neighbour outside the stencil
  if (stencil != 1 && stencil != 2) return FLOCK_EINVAL;
  const double wmin = ((double)rv * (1.0 + ldexp(1.0, -20)) + (double)p.side * ldexp(1.0, -21)) /
                      (double)stencil;
  // Fewer than 2h+1 cells per side is fine: a stencil then visits some cell
  // twice under different periodic shifts, but with L > 2 d_v at most one
  // image of a neighbour can lie within d_v, so nothing is counted twice.
  // The halo wraps by one period only, which needs nc >= h.
  const double ncd = floor((double)p.side / wmin);
  if (ncd < stencil || ncd * ncd > (double)kMaxScanTiles * kScanTile) return FLOCK_EINVAL;
  I.nc = (int)ncd;
  I.ncells = I.nc * I.nc;
  I.row0 = 0;  // a whole square: every row, every agent observed
  I.nrows = I.nc;
  I.halo = stencil;
  I.invw = (float)((double)I.nc / (double)p.side);
  if (p.obs_layout != 0 && p.obs_layout != 1) return FLOCK_EINVAL;
  if (p.kind != 0 && p.kind != 1) return FLOCK_EINVAL;
  I.obs_layout = p.obs_layout;
  I.kind = p.kind;
  // tag: the two colour channels of distances; flock: the chosen layout
  I.obs_dim = p.kind == 1 ? 2 * I.v : (p.obs_layout == 1 ? I.v + 1 : 2 * I.v + 2);

  if (D) {
    memset(D, 0, sizeof *D);
    D->side = I.L; D->half_side = I.HL; D->view_radius = I.RV; D->rv2 = I.RV2; D->rc2 = I.RC2;
    D->inv_span = I.INV_SPAN; D->two_pi = I.TWO_PI; D->cos_half_fov = I.CF;
    D->sin_half_fov = I.SF; D->speed_min = I.SMIN; D->speed_max = I.SMAX;
    for (int k = 0; k < 3; ++k) { D->turn[k] = I.DT[k]; D->accel[k] = I.DS[k]; }
    for (int m = 0; m <= FLOCK_MAX_SEGMENTS; ++m) D->edge[m] = I.T[m];
    D->v = I.v; D->full_circle = I.full; D->k_exp = I.K; D->penalty_fixed = I.PK;
    D->nmax = I.NMAX; D->cells_per_side = I.nc; D->stencil = stencil; D->inv_cell_width = I.invw;
  }
  return FLOCK_OK;
}

// Fill in the launch shape.  Agents per tile aim at 3/4 of the block.
// Mean candidates an agent tests: the agents in its stencil cells.
static double candidates_per_agent(const Inst &I, int n) {
  const double wc = (double)I.L / I.nc;
  return n > 0 ? (double)n / ((double)I.L * I.L) * (2.0 * I.halo + 1.0) * (2.0 * I.halo + 1.0) *
                     wc * wc
               : 0.0;
}

int choose_tuning(const Inst &I, int n, const flock_tuning *req, flock_tuning &t) {
  flock_tuning r{};
  if (req) r = *req;
  t.stencil = I.halo;
  t.mode = r.mode ? r.mode : 2;
  if (t.mode != 1 && t.mode != 2) return FLOCK_EINVAL;
  // lanes per agent: more lanes keep more warps in flight when there are
  // few agents; with many, one lane per agent has the least overhead.  An
  // agent with hundreds of candidates (a view much wider than the spacing of
  // the agents), or one of at most 4,096 agents, gets a whole warp.
  const double cand = candidates_per_agent(I, n);
  t.lanes = r.lanes ? r.lanes
                    : (cand >= 256.0 || n <= 4096
                           ? 32
                           : (n <= 32768 ? 4 : (n <= 524288 ? 2 : 1)));
  if (t.lanes != 1 && t.lanes != 2 && t.lanes != 4 && t.lanes != 32) return FLOCK_EINVAL;
  if (t.mode == 1) t.lanes = 1;
  t.block = r.block ? r.block : 128;
  if (t.block < 64 || t.block > 512 || t.block % 32) return FLOCK_EINVAL;
  if (I.kind == 1 && t.mode == 1) return FLOCK_EINVAL;  // tag: direct forms only
  const double w = (double)I.L / I.nc;
  const double per_cell = n > 0 ? (double)n / ((double)I.L * I.L) * w * w : 1.0;
  t.tile_h = r.tile_h ? r.tile_h : 2;
  if (t.tile_h < 1 || t.tile_h > kMaxTileH) return FLOCK_EINVAL;
  if (r.tile_w) {
    t.tile_w = r.tile_w;
  } else {
    double tw = 0.75 * t.block / (per_cell * t.tile_h);
    t.tile_w = (int)(tw < 1 ? 1 : (tw > kMaxTileW ? kMaxTileW : tw));
  }
  if (t.tile_w < 1 || t.tile_w > kMaxTileW) return FLOCK_EINVAL;
  if (t.tile_w > I.nc) t.tile_w = I.nc;
  if (t.tile_h > I.nc) t.tile_h = I.nc;
  return FLOCK_OK;
}

// Geometry of the tiles and the shared-memory staging capacity.
void set_tiles(Inst &I, int n, const flock_tuning &t) {
  I.tile_w = t.tile_w;
  I.tile_h = t.tile_h;
  I.tiles_x = (I.nc + t.tile_w - 1) / t.tile_w;
  I.tiles_y = (I.nc + t.tile_h - 1) / t.tile_h;
  const double w = (double)I.L / I.nc;
  const double per_cell = n > 0 ? (double)n / ((double)I.L * I.L) * w * w : 0.0;
  const double staged = (t.tile_w + 2.0 * I.halo) * (t.tile_h + 2.0 * I.halo) * per_cell;
  int cap = (int)(2.0 * staged) + 128;
  cap = cap < 256 ? 256 : (cap > 4096 ? 4096 : cap);
  I.cap = cap;
}

static std::once_flag g_attr_once;
static cudaError_t g_attr_err = cudaSuccess;

cudaError_t set_kernel_attrs() {
  std::call_once(g_attr_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int want = maxsm - (int)sizeof(Inst) - 1024;
    const void *fns[] = {(const void *)k_neighbours<1>, (const void *)k_neighbours<2>,
                         (const void *)k_neighbours_direct<1, 0, 1>,
                         (const void *)k_neighbours_direct<2, 0, 1>,
                         (const void *)k_neighbours_direct<1, 8, 1>,
                         (const void *)k_neighbours_direct<2, 8, 1>,
                         (const void *)k_neighbours_direct<1, 0, 2>,
                         (const void *)k_neighbours_direct<2, 0, 2>,
                         (const void *)k_neighbours_direct<1, 8, 2>,
                         (const void *)k_neighbours_direct<2, 8, 2>,
                         (const void *)k_neighbours_direct<1, 0, 4>,
                         (const void *)k_neighbours_direct<2, 0, 4>,
                         (const void *)k_neighbours_direct<1, 8, 4>,
                         (const void *)k_neighbours_direct<2, 8, 4>,
                         (const void *)k_neighbours_direct<1, 0, 1, true>,
                         (const void *)k_neighbours_direct<2, 0, 1, true>,
                         (const void *)k_neighbours_direct<1, 0, 2, true>,
                         (const void *)k_neighbours_direct<2, 0, 2, true>,
                         (const void *)k_neighbours_direct<1, 0, 4, true>,
                         (const void *)k_neighbours_direct<2, 0, 4, true>,
                         (const void *)k_neighbours_direct<1, 0, 32>,
                         (const void *)k_neighbours_direct<2, 0, 32>,
                         (const void *)k_neighbours_direct<1, 0, 32, true>,
                         (const void *)k_neighbours_direct<2, 0, 32, true>,
                         (const void *)k_neighbours_direct<1, 0, 32, false, true>,
                         (const void *)k_neighbours_direct<2, 0, 32, false, true>,
                         (const void *)k_neighbours_direct<1, 0, 32, true, true>,
                         (const void *)k_neighbours_direct<2, 0, 32, true, true>,
                         (const void *)k_neighbours_policy<1, 8, 1>,
                         (const void *)k_neighbours_policy<2, 8, 1>,
                         (const void *)k_neighbours_policy<1, 8, 2>,
                         (const void *)k_neighbours_policy<2, 8, 2>,
                         (const void *)k_neighbours_policy<1, 8, 4>,
                         (const void *)k_neighbours_policy<2, 8, 4>,
                         (const void *)k_neighbours_policy<1, 0, 32>,
                         (const void *)k_neighbours_policy<2, 0, 32>,
                         (const void *)k_neighbours_direct<1, 8, 1, false, false, true>,
                         (const void *)k_neighbours_direct<1, 8, 2, false, false, true>,
                         (const void *)k_neighbours_direct<1, 8, 4, false, false, true>};
    for (const void *f : fns)
      if (g_attr_err == cudaSuccess) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e != cudaSuccess) g_attr_err = e;
      }
  });
  return g_attr_err;
}

}  // namespace flock

using namespace flock;

struct Layout {
  size_t state, cellrank, counts, local, cell_start, tile_sum, sxy, sidx, types, stype, inst,
      err, h_act, h_obs, h_rew, h_coll, wimg, total;
};

static Layout make_layout(int n, int C, int D) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  const int nT = (C + kScanTile - 1) / kScanTile;
  L.state = take((size_t)n * 16);
  L.cellrank = take((size_t)n * 8);
  L.counts = take((size_t)((C + 3) & ~3) * 4);  // zero padding to a whole 16-byte group
  L.local = take((size_t)C * 4);
  L.cell_start = take((size_t)(C + 4) * 4);
  L.tile_sum = take((size_t)(nT + 1) * 4);
  L.sxy = take((size_t)n * 8);
  L.sidx = take((size_t)n * 4);
  L.types = take((size_t)n);   // tag: agent types
  L.stype = take((size_t)n);   // tag: cell-sorted types
  L.inst = take(sizeof(Inst));
  L.err = take(64);
  L.h_act = take((size_t)n * 4);
  L.h_obs = take((size_t)n * D * 4);
  L.h_rew = take((size_t)n * 4);
  L.h_coll = take((size_t)n * 4);
  L.wimg = take(kImgBytes);  // policy step: the weights' operand image
  L.total = o;
  return L;
}

struct flock_env {
  flock_params params;
  flock_tuning tuning;
  flock_derived derived;
  Inst inst;  // host copy
  int n;
  char *ws;
  Layout lay;
  cudaStream_t stream;
  cudaStream_t cap_stream;
  cudaGraphExec_t graph;
  const void *g_act, *g_obs, *g_rew, *g_coll;
  int g_cont;  // the cached graph takes continuous actions
  Bufs bufs;
  int n_scan_tiles;
  int scatter_grid;
  int copy_grid;  // k_copy_out (host-buffer step)
  bool fused_scan;  // at most kFusedScanCells cells: the binning kernel's last block scans them
  bool wide;        // 256 or more candidates an agent on average (a view much wider than the spacing)
  size_t smemD;
  int timing;
  cudaEvent_t ev[5];
  cudaGraphExec_t pgraph;  // step with the policy
  cudaGraphExec_t rgraph;  // a rollout of T steps
  cudaGraphExec_t hgraph;  // host-buffer step: the step and the copy to mapped buffers
  const void *h_act, *h_dst[3];
  const void *r_act, *r_obs, *r_rew, *r_coll;
  int r_T, r_cont;
  const void *p_w, *p_act, *p_rew, *p_coll, *p_log, *p_obs;
};

extern "C" const char *flock_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" int flock_default_params(float side, flock_params *out) {
  if (!out) return FLOCK_EINVAL;
  const double kPi = 3.14159265358979323846;
  out->side = side;
  out->view_radius = 5.0f;
  out->fov = (float)(250.0 * kPi / 180.0);
  out->agent_radius = 0.5f;
  out->collision_penalty = 1.0f;
  out->speed_min = 0.0f;
  out->speed_max = 1.0f;
  out->speed_step = 0.25f;
  out->turn_step = (float)(kPi / 8.0);
  out->num_segments = 8;
  out->obs_layout = 0;
  out->kind = 0;
  return FLOCK_OK;
}

extern "C" int flock_obs_dim(const flock_params *p) {
  if (!p || p->num_segments < 1 || p->num_segments > FLOCK_MAX_SEGMENTS) return FLOCK_EINVAL;
  if (p->obs_layout != 0 && p->obs_layout != 1) return FLOCK_EINVAL;
  if (p->kind != 0 && p->kind != 1) return FLOCK_EINVAL;
  if (p->kind == 1) return 2 * p->num_segments;
  return p->obs_layout == 1 ? p->num_segments + 1 : 2 * p->num_segments + 2;
}

static int resolve(const flock_params *p, const flock_tuning *t, int n, Inst &I, flock_tuning &tt,
                   flock_derived *D) {
  if (!p || n < 0) return FLOCK_EINVAL;
  int stencil = (t && t->stencil) ? t->stencil : 1;
  int rc = derive(*p, stencil, I, D);
  if (rc) return rc;
  rc = choose_tuning(I, n, t, tt);
  if (rc) return rc;
  I.n = n;
  I.n_own = n;
  set_tiles(I, n, tt);
  return FLOCK_OK;
}

extern "C" int flock_workspace_bytes(const flock_params *p, const flock_tuning *t, int n,
                                     size_t *bytes) {
  if (!bytes) return FLOCK_EINVAL;
  Inst I;
  flock_tuning tt;
  int rc = resolve(p, t, n, I, tt, nullptr);
  if (rc) return rc;
  *bytes = make_layout(n, I.ncells, I.obs_dim).total;
  return FLOCK_OK;
}

extern "C" int flock_derive(const flock_params *p, const flock_tuning *t, flock_derived *out) {
  if (!p || !out) return FLOCK_EINVAL;
  Inst I;
  return derive(*p, (t && t->stencil) ? t->stencil : 1, I, out);
}

// Geometry of a slab (rows [row0, row0 + nrows) of the square's cell grid,
// modulo nc; nrows = 0: the whole square) applied to a resolved descriptor.
static int set_slab(Inst &I, const flock_tuning &t, int row0, int nrows) {
  if (nrows == 0 && row0 == 0) return FLOCK_OK;
  if (t.mode != 2) return FLOCK_EINVAL;  // slabs use the direct neighbour scan
  if (row0 < 0 || row0 >= I.nc || nrows < 2 * I.halo + 1 || nrows > I.nc) return FLOCK_EINVAL;
  I.row0 = row0;
  I.nrows = nrows;
  I.ncells = nrows * I.nc;
  return FLOCK_OK;
}

static int create_env(const flock_params *p, const flock_tuning *t, int n, int row0, int nrows,
                      void *ws, size_t ws_bytes, void *stream, flock_env **out) {
  if (!out) return FLOCK_EINVAL;
  *out = nullptr;
  flock_env *e = new (std::nothrow) flock_env();
  if (!e) return FLOCK_EINVAL;
  int rc = resolve(p, t, n, e->inst, e->tuning, &e->derived);
  if (!rc) rc = set_slab(e->inst, e->tuning, row0, nrows);
  if (rc) { delete e; return rc; }
  e->params = *p;
  e->n = n;
  e->lay = make_layout(n, e->inst.ncells, e->inst.obs_dim);
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < e->lay.total) { delete e; return FLOCK_ENOSPACE; }
  e->ws = (char *)ws;
  e->stream = (cudaStream_t)stream;
  cudaError_t ce = set_kernel_attrs();
  if (ce != cudaSuccess) { delete e; return cuda_fail(ce, "cudaFuncSetAttribute"); }
  ce = cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking);
  if (ce != cudaSuccess) { delete e; return cuda_fail(ce, "cudaStreamCreate"); }
  const Layout &L = e->lay;
  e->inst.state = (float4 *)(e->ws + L.state);
  e->inst.agent_base = 0;
  e->inst.cell_base = 0;
  e->inst.obs_base = 0;
  Bufs &B = e->bufs;
  B.cellrank = (int2 *)(e->ws + L.cellrank);
  B.counts = (int *)(e->ws + L.counts);
  B.local = (int *)(e->ws + L.local);
  B.cell_start = (int *)(e->ws + L.cell_start);
  B.tile_sum = (int *)(e->ws + L.tile_sum);
  B.sxy = (float2 *)(e->ws + L.sxy);
  B.sidx = (int *)(e->ws + L.sidx);
  if (e->inst.kind == 1) {
    B.types = (const uint8_t *)(e->ws + L.types);
    B.stype = (uint8_t *)(e->ws + L.stype);
  }
  B.err = (unsigned *)(e->ws + L.err);
  B.bar = B.err + 4;
  B.n_total = n;
  B.c_total = e->inst.ncells;
  e->n_scan_tiles = (e->inst.ncells + kScanTile - 1) / kScanTile;
  B.n_scan_tiles = e->n_scan_tiles;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int g = (n + 255) / 256;
  e->scatter_grid = g < 1 ? 1 : (g > 4 * sms ? 4 * sms : g);
  // 16-byte units of the outputs, one per thread, at most 8 blocks per SM
  const size_t units = ((size_t)n * e->inst.obs_dim * 4 + (size_t)n * 8) / 16;
  e->copy_grid = (int)std::max<size_t>(1, std::min<size_t>((units + 255) / 256, (size_t)sms * 8));
  e->fused_scan = e->inst.ncells <= kFusedScanCells;
  e->wide = candidates_per_agent(e->inst, n) >= 256.0;
  e->smemD = e->tuning.mode == 1
                 ? phaseD_smem_bytes(e->inst.cap, e->inst.v, e->tuning.block)
                 : (size_t)(e->tuning.block / 32) *
                       direct_warp_bytes(e->inst.kind == 1 ? 2 * e->inst.v : e->inst.v,
                                         32 / e->tuning.lanes);
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e->smemD + sizeof(Inst) + 1024 > (size_t)smem_max) {
    cudaStreamDestroy(e->cap_stream);
    delete e;
    return FLOCK_EINVAL;  // launch shape too large for this many sectors
  }
  // descriptor and cleared scratch, in stream order
  cudaStream_t s = e->stream;
  cudaError_t c1 = cudaMemcpyAsync(e->ws + L.inst, &e->inst, sizeof(Inst), cudaMemcpyHostToDevice, s);
  cudaError_t c2 = cudaMemsetAsync(e->ws + L.counts, 0, (size_t)((e->inst.ncells + 3) & ~3) * 4, s);
  cudaError_t c3 = cudaMemsetAsync(e->ws + L.err, 0, 64, s);
  if (c3 == cudaSuccess && n > 0) c3 = cudaMemsetAsync(e->ws + L.types, 0, (size_t)n, s);  // all runners
  if (c1 != cudaSuccess || c2 != cudaSuccess || c3 != cudaSuccess) {
    cudaStreamDestroy(e->cap_stream);
    delete e;
    return cuda_fail(c1 != cudaSuccess ? c1 : (c2 != cudaSuccess ? c2 : c3), "env_create copies");
  }
  // the host descriptor copy is pageable memory: the copy above has been
  // staged by the time it returns, so e->inst may change afterwards
  *out = e;
  return FLOCK_OK;
}

extern "C" int env_create(const flock_params *p, const flock_tuning *t, int n, void *ws,
                          size_t ws_bytes, void *stream, flock_env **out) {
  NvtxRange nvtx_range("flock:env_create");
  return create_env(p, t, n, 0, 0, ws, ws_bytes, stream, out);
}

// act: discrete actions, or cact (when not null): continuous ones.
// n_run >= 0 (a slab's observation): that many agents this time (at most the
// environment's n); the descriptor in the workspace must say the same.
// Policy step: wblob, the weight blob (the binning kernel writes its operand
// image), and pact and plogits, the actions and logits the neighbour scan's
// epilogue writes; the scan then runs in the direct form.
static int enqueue_step(flock_env *e, cudaStream_t s, const int32_t *act, const float2 *cact,
                        float *obs, float *rew, int32_t *coll, int reset, int n_run = -1,
                        const unsigned short *wblob = nullptr, int32_t *pact = nullptr,
                        float *plogits = nullptr, bool aorder = false) {
  Bufs B = e->bufs;
  B.actions = act;
  B.cactions = cact;
  B.obs = obs;
  B.reward = rew;
  B.coll = coll;
  B.pact = pact;
  B.plogits = plogits;
  B.wblob = wblob;
  B.wimg = wblob ? (uint4 *)(e->ws + e->lay.wimg) : nullptr;
  const Inst *gI = (const Inst *)(e->ws + e->lay.inst);
  const int n = n_run >= 0 ? n_run : e->n;
  B.n_total = n;
  const bool tm = e->timing != 0;
  // with timing events between the kernels, plain stream order
  const bool pdl = !tm;
  if (tm) CK(cudaEventRecordWithFlags(e->ev[0], s, cudaEventRecordExternal));
  // the fused scan needs the binning kernel's last block: with no agents the
  // separate scan zeroes the counts and writes the (empty) cell starts
  const bool fused = e->fused_scan && n > 0;
  {
    NvtxRange r("flock:apply_bin");
    // the policy step's operand image: blocks of its own after the agents'
    const int bs = fused ? kFusedBlock : 256;
    const int img = wblob ? (kImgVecs * 32 + bs - 1) / bs : 0;
    if (fused)
      CK(launch(false, k_apply_bin<true>, (n + bs - 1) / bs + img, bs, 0, s, gI, B, reset));
    else if (n > 0)
      CK(launch(false, k_apply_bin<false>, (n + bs - 1) / bs + img, bs, 0, s, gI, B, reset));
  }
  if (tm) CK(cudaEventRecordWithFlags(e->ev[1], s, cudaEventRecordExternal));
  if (!fused) {
    NvtxRange r("flock:scan");
    // k_scan follows k_apply_bin only when there was one
    CK(launch(pdl && n > 0, k_scan, e->n_scan_tiles, 256, 0, s, B));
  }
  if (tm) CK(cudaEventRecordWithFlags(e->ev[2], s, cudaEventRecordExternal));
  {
    NvtxRange r("flock:scatter");
    if (fused) CK(launch(pdl, k_scatter_final, e->scatter_grid, 256, 0, s, gI, B));
    else CK(launch(pdl, k_scatter, e->scatter_grid, 256, 0, s, gI, B));
  }
  if (tm) CK(cudaEventRecordWithFlags(e->ev[3], s, cudaEventRecordExternal));
  NvtxRange r_neigh("flock:neighbours");
  if (n > 0) {
    const int blk = e->tuning.block;
    const size_t sm = e->smemD;
    if (e->tuning.mode == 1 && !pact && !aorder) {
      const int tiles = e->inst.tiles_x * e->inst.tiles_y;
      if (e->inst.halo == 1) CK(launch(pdl, k_neighbours<1>, tiles, blk, sm, s, gI, B));
      else CK(launch(pdl, k_neighbours<2>, tiles, blk, sm, s, gI, B));
    } else {
      // the agent-order form takes 4 lanes per agent up to 100,000 agents: more
      // warps, so that the first ones' row stores to host memory overlap the
      // later ones' scans (50,000 agents: 46.5 us a host step against 48.7
      // with 2 lanes).  Its warp area is the least of the 1-4 lane forms and of
      // the tile form's, so it also serves a tile-form tuning (mode 1).
      const int lpa =
          aorder && (n <= 100000 || e->tuning.mode == 1) ? 4 : e->tuning.lanes;
      const int per_block = blk / lpa;  // agents per block
      const int blocks = (n + per_block - 1) / per_block;
      using KD = void (*)(const Inst *, Bufs);
      // one agent per warp (32 lanes) has the generic-sector kernel only
      static const KD kd[2][2][4] = {
          {{k_neighbours_direct<1, 0, 1>, k_neighbours_direct<1, 0, 2>, k_neighbours_direct<1, 0, 4>,
            k_neighbours_direct<1, 0, 32>},
           {k_neighbours_direct<1, 8, 1>, k_neighbours_direct<1, 8, 2>, k_neighbours_direct<1, 8, 4>,
            k_neighbours_direct<1, 0, 32>}},
          {{k_neighbours_direct<2, 0, 1>, k_neighbours_direct<2, 0, 2>, k_neighbours_direct<2, 0, 4>,
            k_neighbours_direct<2, 0, 32>},
           {k_neighbours_direct<2, 8, 1>, k_neighbours_direct<2, 8, 2>, k_neighbours_direct<2, 8, 4>,
            k_neighbours_direct<2, 0, 32>}}};
      static const KD kt[2][4] = {
          {k_neighbours_direct<1, 0, 1, true>, k_neighbours_direct<1, 0, 2, true>,
           k_neighbours_direct<1, 0, 4, true>, k_neighbours_direct<1, 0, 32, true>},
          {k_neighbours_direct<2, 0, 1, true>, k_neighbours_direct<2, 0, 2, true>,
           k_neighbours_direct<2, 0, 4, true>, k_neighbours_direct<2, 0, 32, true>}};
      const int li = lpa == 1 ? 0 : (lpa == 2 ? 1 : (lpa == 4 ? 2 : 3));
      // the V = 8 kernels write observation layout 0 only
      const int v8 = e->inst.v == 8 && e->inst.obs_layout == 0 ? 1 : 0;
      const int h = e->inst.halo - 1;
      // a warp per agent with a wide view (hundreds of candidates): the
      // compact walk of the wrapping runs
      static const KD kc[2][2] = {
          {k_neighbours_direct<1, 0, 32, false, true>, k_neighbours_direct<1, 0, 32, true, true>},
          {k_neighbours_direct<2, 0, 32, false, true>, k_neighbours_direct<2, 0, 32, true, true>}};
      // the policy step's scan with the network in its epilogue (8 sectors,
      // layout 0, the flock: the host checks)
      static const KD kp[2][4] = {
          {k_neighbours_policy<1, 8, 1>, k_neighbours_policy<1, 8, 2>,
           k_neighbours_policy<1, 8, 4>, k_neighbours_policy<1, 0, 32>},
          {k_neighbours_policy<2, 8, 1>, k_neighbours_policy<2, 8, 2>,
           k_neighbours_policy<2, 8, 4>, k_neighbours_policy<2, 0, 32>}};
      // agent order (host-buffer step; 3 x 3 cells, 8 sectors, layout 0, 1-4
      // lanes: the caller checks)
      static const KD ka[3] = {k_neighbours_direct<1, 8, 1, false, false, true>,
                               k_neighbours_direct<1, 8, 2, false, false, true>,
                               k_neighbours_direct<1, 8, 4, false, false, true>};
      const KD k = pact ? kp[h][li]
                   : aorder ? ka[li < 3 ? li : 0]
                   : (lpa == 32 && e->wide) ? kc[h][e->inst.kind == 1 ? 1 : 0]
                   : (e->inst.kind == 1 ? kt[h][li] : kd[h][v8][li]);
      CK(launch(pdl, k, blocks, blk, sm, s, gI, B));
    }
  }
  if (tm) CK(cudaEventRecordWithFlags(e->ev[4], s, cudaEventRecordExternal));
  return FLOCK_OK;
}

// The policy step: the step's four kernels, the binning kernel also writing
// the weights' operand image and the neighbour scan running the network on
// each warp's agents in its epilogue.
static int enqueue_policy_step(flock_env *e, cudaStream_t s, const unsigned short *w,
                               int32_t *act, float *rew, int32_t *coll, float *logits,
                               float *obs) {
  return enqueue_step(e, s, act, nullptr, obs, rew, coll, 0, -1, w, act, logits);
}

static bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

static int check_out(const flock_env *e, const float *obs, const float *rew, const int32_t *coll) {
  if (e->n == 0) return FLOCK_OK;
  if (!obs || !rew || !coll || !aligned(obs, 8) || !aligned(rew, 4) || !aligned(coll, 4))
    return FLOCK_EINVAL;
  return FLOCK_OK;
}

extern "C" int env_reset(flock_env *e, const float *state0, float *obs, float *rew, int32_t *coll) {
  NvtxRange nvtx_range("flock:env_reset");
  if (!e || (e->n > 0 && !state0)) return FLOCK_EINVAL;
  int rc = check_out(e, obs, rew, coll);
  if (rc) return rc;
  if (e->n > 0)
    CK(cudaMemcpyAsync(e->ws + e->lay.state, state0, (size_t)e->n * 16, cudaMemcpyDeviceToDevice,
                       e->stream));
  return enqueue_step(e, e->stream, nullptr, nullptr, obs, rew, coll, 1);
}

// Makes `exec` run graph g.  When only kernel arguments differ (new buffer
// pointers), the executable graph is updated in place: launches already
// enqueued keep the old arguments, so nothing waits.  Otherwise (first use,
// or a different topology) it is re-instantiated after the stream drains.
static cudaError_t install_graph(cudaGraphExec_t &exec, cudaGraph_t g, cudaStream_t s) {
  if (exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(exec, g, &info) == cudaSuccess) return cudaSuccess;
    (void)cudaGetLastError();  // the update was refused: rebuild
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) exec = nullptr;
  return e;
}

// One step through the cached graph; act_or_cact is the discrete (cont = 0)
// or continuous (cont = 1) action buffer.
static int step_graph(flock_env *e, const void *act_or_cact, int cont, float *obs, float *rew,
                      int32_t *coll) {
  if (!e || (e->n > 0 && !act_or_cact)) return FLOCK_EINVAL;
  int rc = check_out(e, obs, rew, coll);
  if (rc) return rc;
  if (!e->graph || e->g_act != act_or_cact || e->g_cont != cont || e->g_obs != obs ||
      e->g_rew != rew || e->g_coll != coll) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int32_t *act = cont ? nullptr : (const int32_t *)act_or_cact;
    const float2 *cact = cont ? (const float2 *)act_or_cact : nullptr;
    rc = enqueue_step(e, e->cap_stream, act, cact, obs, rew, coll, 0);
    cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = install_graph(e->graph, g, e->stream);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      e->g_act = nullptr;  // force a rebuild next time
      return cuda_fail(ce, "cudaGraphInstantiate");
    }
    e->g_act = act_or_cact;
    e->g_cont = cont;
    e->g_obs = obs;
    e->g_rew = rew;
    e->g_coll = coll;
  }
  CK(cudaGraphLaunch(e->graph, e->stream));
  return FLOCK_OK;
}

extern "C" int env_step(flock_env *e, const int32_t *act, float *obs, float *rew, int32_t *coll) {
  NvtxRange nvtx_range("flock:env_step");
  return step_graph(e, act, 0, obs, rew, coll);
}

extern "C" int env_step_continuous(flock_env *e, const float *act2, float *obs, float *rew,
                                   int32_t *coll) {
  NvtxRange nvtx_range("flock:env_step_continuous");
  if (act2 && !aligned(act2, 8)) return FLOCK_EINVAL;
  return step_graph(e, act2, 1, obs, rew, coll);
}

extern "C" int env_rollout(flock_env *e, int T, const int32_t *act, const float *act2, float *obs,
                           float *rew, int32_t *coll) {
  NvtxRange nvtx_range("flock:env_rollout");
  if (!e || T < 0) return FLOCK_EINVAL;
  if (T == 0) return FLOCK_OK;
  const int n = e->n;
  if (n > 0 && ((act == nullptr) == (act2 == nullptr))) return FLOCK_EINVAL;
  if (act2 && !aligned(act2, 8)) return FLOCK_EINVAL;
  int rc = check_out(e, obs, rew, coll);
  if (rc) return rc;
  const int cont = act2 != nullptr;
  const void *a = cont ? (const void *)act2 : (const void *)act;
  if (!e->rgraph || e->r_T != T || e->r_cont != cont || e->r_act != a || e->r_obs != obs ||
      e->r_rew != rew || e->r_coll != coll) {
    // T steps in one graph; step t reads actions row t and writes output rows t
    const int timing = e->timing;
    e->timing = 0;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
    const size_t D = (size_t)e->inst.obs_dim;
    for (int t = 0; t < T && rc == FLOCK_OK; ++t) {
      const size_t o = (size_t)t * n;
      rc = enqueue_step(e, e->cap_stream, act ? act + o : nullptr,
                        act2 ? reinterpret_cast<const float2 *>(act2) + o : nullptr,
                        obs ? obs + o * D : nullptr, rew ? rew + o : nullptr,
                        coll ? coll + o : nullptr, 0);
    }
    e->timing = timing;
    cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = install_graph(e->rgraph, g, e->stream);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      e->r_T = 0;  // force a rebuild next time
      return cuda_fail(ce, "cudaGraphInstantiate");
    }
    e->r_T = T;
    e->r_cont = cont;
    e->r_act = a;
    e->r_obs = obs;
    e->r_rew = rew;
    e->r_coll = coll;
  }
  CK(cudaGraphLaunch(e->rgraph, e->stream));
  return FLOCK_OK;
}

extern "C" int env_step_policy(flock_env *e, const uint16_t *weights, int32_t *act, float *rew,
                               int32_t *coll, float *logits, float *obs) {
  NvtxRange nvtx_range("flock:env_step_policy");
  if (!e || e->inst.v != 8 || e->inst.obs_layout != 0 || e->inst.kind != 0) return FLOCK_EINVAL;
  if (e->n > 0 && (!weights || !act || !rew || !coll || !aligned(weights, 4) ||
                   (obs && !aligned(obs, 8))))
    return FLOCK_EINVAL;
  if (!e->pgraph || e->p_w != weights || e->p_act != act || e->p_rew != rew ||
      e->p_coll != coll || e->p_log != logits || e->p_obs != obs) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_policy_step(e, e->cap_stream, (const unsigned short *)weights, act, rew, coll,
                                 logits, obs);
    cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = install_graph(e->pgraph, g, e->stream);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      e->p_w = nullptr;  // force a rebuild next time
      return cuda_fail(ce, "cudaGraphInstantiate");
    }
    e->p_w = weights;
    e->p_act = act;
    e->p_rew = rew;
    e->p_coll = coll;
    e->p_log = logits;
    e->p_obs = obs;
  }
  CK(cudaGraphLaunch(e->pgraph, e->stream));
  return FLOCK_OK;
}

extern "C" int env_step_host(flock_env *e, const int32_t *act_h, float *obs_h, float *rew_h,
                             int32_t *coll_h) {
  NvtxRange nvtx_range("flock:env_step_host");
  if (!e) return FLOCK_EINVAL;
  const size_t n = (size_t)e->n;
  if (n > 0 && (!act_h || !obs_h || !rew_h || !coll_h)) return FLOCK_EINVAL;
  const Layout &L = e->lay;
  const int32_t *act = (const int32_t *)(e->ws + L.h_act);
  float *obs = (float *)(e->ws + L.h_obs);
  float *rew = (float *)(e->ws + L.h_rew);
  int32_t *coll = (int32_t *)(e->ws + L.h_coll);
  // Page-locked, mapped actions (Grace-Blackwell reaches host memory
  // coherently over NVLink-C2C) are read by the binning kernel in place.  The
  // outputs go through the workspace (written in place, their scattered rows
  // crossed the link more slowly than a bulk copy), then to mapped host
  // buffers by one copy kernel captured with the step in one graph, else by
  // one copy each after the step.
  void *da = nullptr;
  if (n > 0 && cudaHostGetDevicePointer(&da, (void *)act_h, 0) == cudaSuccess) {
    act = (const int32_t *)da;
  } else {
    (void)cudaGetLastError();
    if (n > 0) CK(cudaMemcpyAsync((void *)act, act_h, n * 4, cudaMemcpyHostToDevice, e->stream));
  }
  if (n == 0) {
    int rc = env_step(e, act, obs, rew, coll);
    if (rc) return rc;
    CK(cudaStreamSynchronize(e->stream));
    return FLOCK_OK;
  }
  {
    const size_t ob = n * e->inst.obs_dim * 4;
    void *dobs = nullptr, *drew = nullptr, *dcoll = nullptr;
    const bool mapped =
        cudaHostGetDevicePointer(&dobs, obs_h, 0) == cudaSuccess &&
        cudaHostGetDevicePointer(&drew, rew_h, 0) == cudaSuccess &&
        cudaHostGetDevicePointer(&dcoll, coll_h, 0) == cudaSuccess &&
        ((reinterpret_cast<uintptr_t>(dobs) | reinterpret_cast<uintptr_t>(drew) |
          reinterpret_cast<uintptr_t>(dcoll)) & 3) == 0;
    if (mapped) {
      CopyOut J;
      J.src[0] = (const char *)obs;
      J.src[1] = (const char *)rew;
      J.src[2] = (const char *)coll;
      J.dst[0] = (char *)dobs;
      J.dst[1] = (char *)drew;
      J.dst[2] = (char *)dcoll;
      J.bytes[0] = ob;
      J.bytes[1] = n * 4;
      J.bytes[2] = n * 4;
      // One graph, kept while the buffers are the same.  The 8-sector flock
      // with 1-4 lanes per agent runs its neighbour scan in agent order and
      // writes the outputs straight into the mapped buffers, whole blocks of
      // rows at a time, while other warps still compute; otherwise the step
      // writes the workspace and the copy kernel follows it (under
      // programmatic dependent launch).
      const bool ao = e->inst.kind == 0 && e->inst.halo == 1 && e->inst.v == 8 &&
                      e->inst.obs_layout == 0 && e->tuning.lanes != 32;
      if (!e->hgraph || e->h_act != act || e->h_dst[0] != dobs || e->h_dst[1] != drew ||
          e->h_dst[2] != dcoll) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = ao ? enqueue_step(e, e->cap_stream, act, nullptr, (float *)dobs, (float *)drew,
                                   (int32_t *)dcoll, 0, -1, nullptr, nullptr, nullptr, true)
                    : enqueue_step(e, e->cap_stream, act, nullptr, obs, rew, coll, 0);
        cudaError_t le = rc || ao ? cudaSuccess
                                  : launch(true, k_copy_out, e->copy_grid, 256, 0, e->cap_stream, J);
        cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &g);
        if (rc || le != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          return rc ? rc : cuda_fail(le, "cudaLaunchKernelEx");
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        ce = install_graph(e->hgraph, g, e->stream);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
          e->h_act = nullptr;  // force a rebuild next time
          return cuda_fail(ce, "cudaGraphInstantiate");
        }
        e->h_act = act;
        e->h_dst[0] = dobs;
        e->h_dst[1] = drew;
        e->h_dst[2] = dcoll;
      }
      CK(cudaGraphLaunch(e->hgraph, e->stream));
    } else {
      (void)cudaGetLastError();
      int rc = env_step(e, act, obs, rew, coll);
      if (rc) return rc;
      CK(cudaMemcpyAsync(obs_h, obs, ob, cudaMemcpyDeviceToHost, e->stream));
      CK(cudaMemcpyAsync(rew_h, rew, n * 4, cudaMemcpyDeviceToHost, e->stream));
      CK(cudaMemcpyAsync(coll_h, coll, n * 4, cudaMemcpyDeviceToHost, e->stream));
    }
  }
  CK(cudaStreamSynchronize(e->stream));
  return FLOCK_OK;
}

extern "C" int env_get_state(flock_env *e, float *state) {
  if (!e || (e->n > 0 && !state)) return FLOCK_EINVAL;
  if (e->n > 0)
    CK(cudaMemcpyAsync(state, e->ws + e->lay.state, (size_t)e->n * 16, cudaMemcpyDeviceToDevice,
                       e->stream));
  return FLOCK_OK;
}

extern "C" int env_set_types(flock_env *e, const uint8_t *types) {
  if (!e || e->inst.kind != 1 || (e->n > 0 && !types)) return FLOCK_EINVAL;
  if (e->n > 0)
    CK(cudaMemcpyAsync(e->ws + e->lay.types, types, (size_t)e->n, cudaMemcpyDeviceToDevice,
                       e->stream));
  return FLOCK_OK;
}

extern "C" int env_set_state(flock_env *e, const float *state) {
  if (!e || (e->n > 0 && !state)) return FLOCK_EINVAL;
  if (e->n > 0)
    CK(cudaMemcpyAsync(e->ws + e->lay.state, state, (size_t)e->n * 16, cudaMemcpyDeviceToDevice,
                       e->stream));
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

extern "C" int env_get_error(flock_env *e, uint32_t *bits) {
  NvtxRange nvtx_range("flock:env_get_error");
  if (!e || !bits) return FLOCK_EINVAL;
  uint32_t w = 0;
  CK(cudaMemcpyAsync(&w, e->ws + e->lay.err, 4, cudaMemcpyDeviceToHost, e->stream));
  CK(cudaMemsetAsync(e->ws + e->lay.err, 0, 4, e->stream));
  CK(cudaStreamSynchronize(e->stream));
#ifdef FLOCK_DEBUG
  w |= dbg_take(e->stream);
#endif
  *bits = w;
  return FLOCK_OK;
}

extern "C" int env_get_derived(const flock_env *e, flock_derived *out) {
  if (!e || !out) return FLOCK_EINVAL;
  *out = e->derived;
  return FLOCK_OK;
}

extern "C" int env_get_tuning(const flock_env *e, flock_tuning *out) {
  if (!e || !out) return FLOCK_EINVAL;
  *out = e->tuning;
  return FLOCK_OK;
}

extern "C" int env_set_timing(flock_env *e, int enable) {
  if (!e) return FLOCK_EINVAL;
  if (enable && !e->ev[0])
    for (int k = 0; k < 5; ++k) CK(cudaEventCreate(&e->ev[k]));
  if ((enable != 0) != (e->timing != 0) && (e->graph || e->pgraph || e->hgraph)) {
    CK(cudaStreamSynchronize(e->stream));
    // re-captured by the next env_step / env_step_policy / env_step_host
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->pgraph) cudaGraphExecDestroy(e->pgraph);
    if (e->hgraph) cudaGraphExecDestroy(e->hgraph);
    e->graph = nullptr;
    e->pgraph = nullptr;
    e->hgraph = nullptr;
  }
  e->timing = enable != 0;
  return FLOCK_OK;
}

extern "C" int env_get_phase_times(flock_env *e, float *ms) {
  if (!e || !ms || !e->timing) return FLOCK_EINVAL;
  CK(cudaEventSynchronize(e->ev[4]));
  for (int k = 0; k < 4; ++k) CK(cudaEventElapsedTime(&ms[k], e->ev[k], e->ev[k + 1]));
  return FLOCK_OK;
}

extern "C" void env_destroy(flock_env *e) {
  if (!e) return;
  cudaStreamSynchronize(e->stream);
  for (int k = 0; k < 5; ++k)
    if (e->ev[k]) cudaEventDestroy(e->ev[k]);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  if (e->pgraph) cudaGraphExecDestroy(e->pgraph);
  if (e->rgraph) cudaGraphExecDestroy(e->rgraph);
  if (e->hgraph) cudaGraphExecDestroy(e->hgraph);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  delete e;
}


// ---------------------------------------------------------------------------
// Slabs: one square decomposed over several devices.  A slab environment's
// cell list holds a band of rows of the square's grid; each step the caller
// (the decomposition in slab.py) applies the actions of the agents it owns
// (env_slab_apply), moves the agents that crossed into another band to its
// owner and copies the agents near each band edge to the neighbouring band
// as ghosts, then observes its own agents over its own and the ghost agents
// (env_slab_observe).  Positions keep their coordinates on the square, so
// the minimum-image offsets are those of the undivided square.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_apply(const Inst *__restrict__ gI, float4 *state,
                                               const int32_t *__restrict__ actions, int n,
                                               unsigned *errw) {
  const Inst &I = *gI;
  unsigned err = 0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float4 st = state[i];
    if (!state_ok(st, I)) err |= FLOCK_ERR_STATE;
    state[i] = apply_action(st, actions[i], I, err);
  }
  if (err) atomicOr(errw, err);
}

extern "C" int flock_slab_workspace_bytes(const flock_params *p, const flock_tuning *t, int n_max,
                                          int row0, int nrows, size_t *bytes) {
  if (!bytes || nrows <= 0) return FLOCK_EINVAL;
  Inst I;
  flock_tuning tt;
  int rc = resolve(p, t, n_max, I, tt, nullptr);
  if (!rc) rc = set_slab(I, tt, row0, nrows);
  if (rc) return rc;
  *bytes = make_layout(n_max, I.ncells, I.obs_dim).total;
  return FLOCK_OK;
}

extern "C" int env_slab_create(const flock_params *p, const flock_tuning *t, int n_max, int row0,
                               int nrows, void *ws, size_t ws_bytes, void *stream,
                               flock_env **out) {
  NvtxRange nvtx_range("flock:env_slab_create");
  if (nrows <= 0) return FLOCK_EINVAL;
  return create_env(p, t, n_max, row0, nrows, ws, ws_bytes, stream, out);
}

extern "C" int env_slab_apply(flock_env *e, int n, float *state_dev, const int32_t *actions_dev) {
  NvtxRange nvtx_range("flock:env_slab_apply");
  if (!e || n < 0 || n > e->n) return FLOCK_EINVAL;
  if (n == 0) return FLOCK_OK;
  if (!state_dev || !actions_dev || !aligned(state_dev, 16) || !aligned(actions_dev, 4))
    return FLOCK_EINVAL;
  CK(launch(false, k_apply, (n + 255) / 256, 256, 0, e->stream,
            (const Inst *)(e->ws + e->lay.inst), reinterpret_cast<float4 *>(state_dev),
            actions_dev, n, e->bufs.err));
  return FLOCK_OK;
}

extern "C" int env_slab_observe(flock_env *e, int n_own, int n_ghost, const float *state_dev,
                                float *obs, float *rew, int32_t *coll) {
  NvtxRange nvtx_range("flock:env_slab_observe");
  if (!e || n_own < 0 || n_ghost < 0 || n_own + n_ghost > e->n) return FLOCK_EINVAL;
  const int n = n_own + n_ghost;
  if (n > 0 && (!state_dev || !aligned(state_dev, 16))) return FLOCK_EINVAL;
  if (n_own > 0 && (!obs || !rew || !coll || !aligned(obs, 8))) return FLOCK_EINVAL;
  Inst I = e->inst;
  I.n = n;
  I.n_own = n_own;
  // the host copy is staged by the time the call returns (pageable memory)
  CK(cudaMemcpyAsync(e->ws + e->lay.inst, &I, sizeof(Inst), cudaMemcpyHostToDevice, e->stream));
  if (n > 0)
    CK(cudaMemcpyAsync(e->ws + e->lay.state, state_dev, (size_t)n * 16, cudaMemcpyDeviceToDevice,
                       e->stream));
  return enqueue_step(e, e->stream, nullptr, nullptr, obs, rew, coll, 1, n);
}

// ---------------------------------------------------------------------------
// Allocation-free step.
//
// Some callers cannot allocate device memory at all: code that runs inside a
// host callback or a real-time loop where cudaMalloc may block or is
// forbidden, plugins whose host application owns every allocation, and
// processes that must not touch a caching allocator they do not control.
// flock_step_static serves them: the caller passes only the state, the
// actions and the outputs; everything else the step needs (cell counts,
// offsets, sorted copies, the parameter descriptor, the error word) lives in
// the fixed device array below, which every GPU that loads this library
// holds for the lifetime of the process.
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxAgents = FLOCK_STATIC_MAX_AGENTS;
constexpr int kStaticMaxCells = FLOCK_STATIC_MAX_CELLS;
constexpr int kStaticScanTiles = (kStaticMaxCells + kScanTile - 1) / kScanTile;

// Byte offsets inside the array (each 256-byte aligned).
constexpr size_t sa(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kSInst = 0;
constexpr size_t kSErr = sa(kSInst + sizeof(Inst));
constexpr size_t kSCellrank = sa(kSErr + 64);
constexpr size_t kSCounts = sa(kSCellrank + (size_t)kStaticMaxAgents * 8);
constexpr size_t kSLocal = sa(kSCounts + (size_t)kStaticMaxCells * 4);
constexpr size_t kSCellStart = sa(kSLocal + (size_t)kStaticMaxCells * 4);
constexpr size_t kSTileSum = sa(kSCellStart + (size_t)(kStaticMaxCells + 1) * 4);
constexpr size_t kSSxy = sa(kSTileSum + (size_t)(kStaticScanTiles + 1) * 4);
constexpr size_t kSSidx = sa(kSSxy + (size_t)kStaticMaxAgents * 8);
constexpr size_t kSBytes = sa(kSSidx + (size_t)kStaticMaxAgents * 4);
static_assert(kSBytes == FLOCK_STATIC_SCRATCH_BYTES, "flock.h states the scratch size");

}  // namespace

// The scratch of flock_step_static: one per device, shared by every call.
static __device__ __align__(256) char g_flock_static_scratch[kSBytes];

namespace {

std::mutex g_static_mu;
char *g_static_ptr[256];  // device address of the array, per device ordinal

// Device address of the scratch array on the current device (set up on the
// first call for that device).  In host code the array's name is only a
// host-side stand-in, so the address must come from cudaGetSymbolAddress.
int static_scratch(char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return FLOCK_EINVAL;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_flock_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_static_ptr[dev] = (char *)p;
  }
  *out = g_static_ptr[dev];
  return FLOCK_OK;
}

}  // namespace

extern "C" int flock_step_static(const flock_params *p, int n, float *state_dev,
                                 const int32_t *actions_dev, float *obs_dev, float *reward_dev,
                                 int32_t *coll_dev, void *stream, uint32_t *error_bits_out) {
  NvtxRange nvtx_range("flock:flock_step_static");
  if (!p || n < 0) return FLOCK_EINVAL;
  if (n > kStaticMaxAgents) return FLOCK_EINVAL;  // more agents than the fixed scratch holds
  Inst I;
  int rc = derive(*p, 1, I, nullptr);
  if (rc) return rc;
  if (I.ncells > kStaticMaxCells) return FLOCK_EINVAL;  // cell list larger than the scratch
  if (I.kind != 0) return FLOCK_EINVAL;                  // flock only
  if (n > 0 && (!state_dev || !obs_dev || !reward_dev || !coll_dev || ((uintptr_t)obs_dev & 7)))
    return FLOCK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // The call copies its descriptor from pageable host memory and, with
  // error_bits_out, waits for the stream: neither is allowed while the
  // stream is being captured, so such a call is refused before it enqueues
  // anything.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return FLOCK_EINVAL;
  // The scratch address and the grid size below are those of the current
  // device: a stream of another device is refused.
  int cur_dev = 0, stream_dev = 0;
  CK(cudaGetDevice(&cur_dev));
  CK(cudaStreamGetDevice(s, &stream_dev));
  if (stream_dev != cur_dev) return FLOCK_EINVAL;
  char *sp = nullptr;
  rc = static_scratch(&sp);
  if (rc) return rc;
  cudaError_t ce = set_kernel_attrs();
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaFuncSetAttribute");
  flock_tuning t{};
  t.stencil = 1;
  t.mode = 2;
  t.block = 128;
  I.n = n;
  I.n_own = n;
  I.state = reinterpret_cast<float4 *>(state_dev);
  I.agent_base = 0;
  I.cell_base = 0;
  I.obs_base = 0;
  set_tiles(I, n, t);
  Bufs B{};
  B.cellrank = (int2 *)(sp + kSCellrank);
  B.counts = (int *)(sp + kSCounts);
  B.local = (int *)(sp + kSLocal);
  B.cell_start = (int *)(sp + kSCellStart);
  B.tile_sum = (int *)(sp + kSTileSum);
  B.sxy = (float2 *)(sp + kSSxy);
  B.sidx = (int *)(sp + kSSidx);
  B.err = (unsigned *)(sp + kSErr);
  B.bar = B.err + 4;
  B.actions = actions_dev;
  B.obs = obs_dev;
  B.reward = reward_dev;
  B.coll = coll_dev;
  B.n_total = n;
  B.c_total = I.ncells;
  B.n_scan_tiles = (I.ncells + kScanTile - 1) / kScanTile;
  // the array keeps the previous call's contents: start the counts and the
  // error word from zero, and load this call's descriptor
  CK(cudaMemsetAsync(sp + kSCounts, 0, (size_t)I.ncells * 4, s));
  CK(cudaMemsetAsync(sp + kSErr, 0, 64, s));
  CK(cudaMemcpyAsync(sp + kSInst, &I, sizeof(Inst), cudaMemcpyHostToDevice, s));
  const Inst *gI = (const Inst *)(sp + kSInst);
  const int reset = actions_dev ? 0 : 1;
  if (n > 0) {
    k_apply_bin<false><<<(n + 255) / 256, 256, 0, s>>>(gI, B, reset);
    CK(cudaGetLastError());
  }
  k_scan<<<B.n_scan_tiles, 256, 0, s>>>(B);
  CK(cudaGetLastError());
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur_dev));
  int g = (n + 255) / 256;
  g = g < 1 ? 1 : (g > 4 * sms ? 4 * sms : g);
  k_scatter<<<g, 256, 0, s>>>(gI, B);
  CK(cudaGetLastError());
  if (n > 0) {
    const size_t smem = (size_t)(t.block / 32) * direct_warp_bytes(I.v);
    const int blocks = (n + t.block - 1) / t.block;
    // the V = 8 kernel writes observation layout 0 only (float2 entries of
    // 2v + 2 value rows); every other layout takes the generic kernel
    if (I.v == 8 && I.obs_layout == 0) k_neighbours_direct<1, 8, 1><<<blocks, t.block, smem, s>>>(gI, B);
    else k_neighbours_direct<1, 0, 1><<<blocks, t.block, smem, s>>>(gI, B);
    CK(cudaGetLastError());
  }
  if (error_bits_out) {
    uint32_t w = 0;
    CK(cudaMemcpyAsync(&w, sp + kSErr, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
#ifdef FLOCK_DEBUG
    w |= dbg_take(s);
#endif
    *error_bits_out = w;
  }
  return FLOCK_OK;
}
