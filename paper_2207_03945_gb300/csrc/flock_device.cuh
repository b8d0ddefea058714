// Device code of the flock environment step (arXiv 2207.03945, Section 4.1).
//
// One step is four phases over a uniform cell list on the periodic square:
//   A  apply actions (Section 4.1: accelerate, rotate, move), compute each
//      agent's cell, count agents per cell with warp-aggregated atomics;
//   B  exclusive scan of the cell counts, in tiles of SCAN_TILE cells;
//   C  scatter positions into cell order (counting sort), finalise cell starts;
//   D  neighbour scan: per tile of cells, stage the tile plus its halo from
//      the cell-sorted positions into shared memory, then one thread per agent
//      visits the stencil cells and fuses observation (Fig. 3), collision
//      count (Fig. 4) and reward (Eq. 1) into one pass.
//
// Every FP32 operation that decides or produces an output is written with an
// explicit round-to-nearest intrinsic (no contraction, no approximation), so
// the results are exactly those of the plain O(N^2) definition evaluated
// with the same formulas.  The reward sum is exact (64-bit fixed point) and
// therefore independent of the visiting order.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "flock.h"

namespace flock {

constexpr int kMaxV = FLOCK_MAX_SEGMENTS;
constexpr int kScanTile = 1024;        // cells per scan tile (phase B)
constexpr int kMaxScanTiles = 8192;    // => at most 8M cells
constexpr int kMaxTileW = 64, kMaxTileH = 8;
constexpr int kMaxStagedCells = (kMaxTileH + 4) * (kMaxTileW + 4);

// Per-instance descriptor.  A single environment has one; a batch has one
// per active instance.  Lives in device memory (the workspace); 16-byte
// aligned so that per-warp shared copies keep the areas after them aligned.
struct alignas(16) Inst {
  float4 *state;       // resident state (x, y, theta, s), updated in place
  long long obs_base;  // first float of this instance's obs rows
  int n, nc, ncells, v;
  int agent_base, cell_base, tile_base, chunk_base;
  int tiles_x, tiles_y, tile_w, tile_h;
  int halo, full, K, reset;
  int obs_dim, cap;  // cap: staged agents that fit in shared memory
  int pieces;        // 32-bit pieces a reward term needs in shared accumulators (2 or 3)
  int obs_layout;    // 0: (distance, count) per sector, speed, heading; 1: distances, speed
  int kind;          // 0: flock; 1: tag (runners and chasers, Section 4.2)
  // a slab of a larger square (decomposition over devices): its cell list
  // holds the rows [row0, row0 + nrows) of the square's grid (modulo nc),
  // and only its first n_own agents are observed (the rest are ghosts,
  // copies of a neighbouring slab's agents).  A whole square: row0 = 0,
  // nrows = nc, n_own = n.
  int row0, nrows, n_own;
  float L, HL, invw, RV, RV2, RC2, INV_SPAN, SMIN, SMAX, TWO_PI, CF, SF, scaleK, inv_scaleK;
  float DT[3], DS[3];
  long long PK, NMAX;
  float T[kMaxV + 1];
};

static_assert(sizeof(Inst) % 16 == 0, "Inst must keep 16-byte alignment");

// Scratch and output pointers of one step (flattened over all instances).
struct Bufs {
  int2 *cellrank;      // per agent: global cell, rank in cell
  int *counts;         // per cell, zero between steps
  int *local;          // per cell: exclusive prefix within its scan tile
  int *cell_start;     // per cell + 1: first sorted position
  int *tile_sum;       // per scan tile: agents in the tile
  float2 *sxy;         // cell-sorted positions (x, y)
  int *sidx;           // cell-sorted flattened agent index
  unsigned *err;       // latched FLOCK_ERR_* bits
  unsigned *bar;       // grid barrier words (count, generation)
  const int32_t *actions;
  const float2 *cactions;  // continuous actions (acceleration, rotation), or null
  const uint8_t *types;    // tag: agent types (0 runner, 1 chaser), agent order; else null
  uint8_t *stype;          // tag: cell-sorted types; else null
  float *obs;
  float *reward;
  int32_t *coll;
  const unsigned short *wblob;  // policy step: the weight blob, whose operand image the
  uint4 *wimg;                  // binning kernel writes to wimg (both null otherwise)
  int32_t *pact;   // policy step, network in the neighbour scan: greedy actions out
  float *plogits;  // and logits (9 per agent, agent order), or null
  int n_total, c_total, n_scan_tiles, pad;
};

// Debug build (FLOCK_DEBUG, libflock_debug.so): index checks on the step's
// scratch and output accesses.  A failed check latches FLOCK_ERR_BOUNDS in
// this translation unit's word (read and cleared with the error bits) and
// the access is skipped; nothing traps.  In the release build every check
// is the constant true and compiles away.
#ifdef FLOCK_DEBUG
static __device__ unsigned g_flock_dbg_bits;
__device__ __forceinline__ bool dbg_ok(bool cond) {
  if (!cond) atomicOr(&g_flock_dbg_bits, FLOCK_ERR_BOUNDS);
  return cond;
}
#else
__device__ __forceinline__ constexpr bool dbg_ok(bool) { return true; }
#endif

// Shared-memory accesses of the neighbour scan's per-warp areas, issued as
// shared-space instructions on 32-bit shared addresses.  The areas are
// carved from dynamic shared memory and reached through pointers whose
// address space the compiler does not always see; generic-address atomics
// cost several times a shared one.  `red` updates return nothing.
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void sred_add_u32(unsigned a, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sred_min_u32(unsigned a, unsigned v) {
  asm volatile("red.shared.min.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sred_add_u64(unsigned a, unsigned long long v) {
  asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void sst_f4(unsigned a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ float4 sld_f4(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}

// Predicated forms: the predicate is evaluated inside the instruction
// sequence, so a conditional update costs no branch (a branch around a
// side effect in the neighbour scan's pair loop costs the warp far more
// than the update: divergence and reconvergence bookkeeping).
__device__ __forceinline__ void sred_add_u32_if(bool p, unsigned a, unsigned v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.shared.add.u32 [%0], %1;\n\t}"
      ::"r"(a), "r"(v), "r"((unsigned)p)
      : "memory");
}
__device__ __forceinline__ void sred_min_u32_if(bool p, unsigned a, unsigned v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.shared.min.u32 [%0], %1;\n\t}"
      ::"r"(a), "r"(v), "r"((unsigned)p)
      : "memory");
}
__device__ __forceinline__ void sred_add_u64_if(bool p, unsigned a, unsigned long long v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.shared.add.u64 [%0], %1;\n\t}"
      ::"r"(a), "l"(v), "r"((unsigned)p)
      : "memory");
}
__device__ __forceinline__ void sst_f4_if(bool p, unsigned a, float4 v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t@q st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n\t}"
      ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"((unsigned)p)
      : "memory");
}

// A candidate run [a, a + n) of the sorted arrays (n_total entries); in the
// debug build a run outside them is checked, latched and emptied.
__device__ __forceinline__ void dbg_run(int a, int &n, int n_total) {
  if (!dbg_ok(n <= 0 || (a >= 0 && a + n <= n_total))) n = 0;
}

// Programmatic dependent launch: a kernel launched with the programmatic
// serialization attribute is set up while the kernel before it drains; it
// waits here until that kernel has finished and its writes are visible.
// (No early trigger: blocks of the next kernel held resident while this one
// still runs made the step slower.)  Launched without the attribute, the
// wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Exactly-rounded FP32 arithmetic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

// Deterministic sine and cosine (used once per agent, never per pair):
// Cody-Waite reduction by pi/2 with a two-part constant whose high part has 8
// significant bits (so q * hi is exact for the quadrant counts q <= 4 that
// headings in [0, 2pi) produce), then the Taylor polynomials of sin to x^9
// and cos to x^8 in Horner form.  The coefficients are the floats nearest
// to 1/k!.  Error against the exact functions stays below 2e-7.
__device__ __forceinline__ void det_sincos(float th, float &c, float &s) {
  const float kTwoOverPi = 0x1.45f306p-1f;
  const float kHi = 1.5703125f, kLo = 0x1.fb5444p-12f;
  const float s1 = -0x1.555556p-3f, s2 = 0x1.111112p-7f, s3 = -0x1.a01a02p-13f,
              s4 = 0x1.71de3ap-19f;
  const float c1 = -0.5f, c2 = 0x1.555556p-5f, c3 = -0x1.6c16c2p-10f, c4 = 0x1.a01a02p-16f;
  int q = __float2int_rn(fmul(th, kTwoOverPi));
  float qf = (float)q;
  float r = fsub(fsub(th, fmul(qf, kHi)), fmul(qf, kLo));
  float r2 = fmul(r, r);
  float ps = fadd(s3, fmul(r2, s4));
  ps = fadd(s2, fmul(r2, ps));
  ps = fadd(s1, fmul(r2, ps));
  float sr = fadd(r, fmul(fmul(r, r2), ps));
  float pc = fadd(c3, fmul(r2, c4));
  pc = fadd(c2, fmul(r2, pc));
  pc = fadd(c1, fmul(r2, pc));
  float cr = fadd(1.0f, fmul(r2, pc));
  switch (q & 3) {
    case 0: c = cr; s = sr; break;
    case 1: c = -sr; s = cr; break;
    case 2: c = -cr; s = -sr; break;
    default: c = sr; s = -cr; break;
  }
}

// Pseudo-angle of direction (x, y) in [0, 4): one unit per quadrant,
// counter-clockwise from +x, monotone in the true angle.  Per quadrant q it
// is q + n / d with d = |x| + |y| in all four quadrants and n = |y| (q even)
// or |x| (q odd); written with one division and no branch, it gives the
// same bits as the case-by-case form y/(x+y), 1+(-x)/(-x+y), 2+(-y)/(-x-y),
// 3+x/(x-y).
__device__ __forceinline__ float pseudo_angle(float x, float y) {
  const bool yp = y >= 0.0f, xp = x >= 0.0f;
  const int q = yp ? (xp ? 0 : 1) : (xp ? 3 : 2);
  const float ax = fabsf(x), ay = fabsf(y);
  const float num = (q & 1) ? ax : ay;
  return fadd((float)q, fdiv(num, fadd(ax, ay)));
}

__device__ __forceinline__ float wrap_coord(float x, float L) {
  if (x >= L) x = fsub(x, L);
  else if (x < 0.0f) x = fadd(x, L);
  if (x >= L) x = 0.0f;
  return x;
}

__device__ __forceinline__ bool state_ok(const float4 s, const Inst &I) {
  // NaN fails every comparison; infinities fail the range tests
  return s.x >= 0.0f && s.x < I.L && s.y >= 0.0f && s.y < I.L && s.z >= 0.0f &&
         s.z < I.TWO_PI && s.w >= I.SMIN && s.w <= I.SMAX;
}

// Section 4.1: accelerate by ds (speed clamped to [s_min, s_max]), rotate by
// dt (heading kept in [0, 2pi); |dt| < pi), then move one step along the new
// heading on the torus.
__device__ __forceinline__ float4 move_agent(float4 st, float ds, float dt, const Inst &I) {
  float s = fadd(st.w, ds);
  if (s < I.SMIN) s = I.SMIN;
  else if (s > I.SMAX) s = I.SMAX;
  float th = fadd(st.z, dt);
  if (th >= I.TWO_PI) th = fsub(th, I.TWO_PI);
  else if (th < 0.0f) th = fadd(th, I.TWO_PI);
  if (th >= I.TWO_PI) th = 0.0f;
  float c, sn;
  det_sincos(th, c, sn);
  float x = wrap_coord(fadd(st.x, fmul(s, c)), I.L);
  float y = wrap_coord(fadd(st.y, fmul(s, sn)), I.L);
  return make_float4(x, y, th, s);
}

// Discrete action a in [0, 9): turn a / 3 and speed change a % 3 index the
// steps {-Delta, 0, +Delta} and {-a, 0, +a}; other values act as 4 (flagged).
__device__ __forceinline__ float4 apply_action(float4 st, int a, const Inst &I, unsigned &err) {
  if ((unsigned)a >= 9u) {
    a = 4;
    err |= FLOCK_ERR_ACTION;
  }
  const int tu = a / 3, su = a - 3 * tu;
  return move_agent(st, I.DS[su], I.DT[tu], I);
}

// Continuous action (acceleration, rotation), Section 4.1: the ranges
// [-a, a] x [-Delta, Delta] of the discrete steps bound the action (values
// outside are clamped; a non-finite component counts as 0 and is flagged);
// then the same speed clamp, heading wrap and move as above.
__device__ __forceinline__ float4 apply_cont(float4 st, float2 a, const Inst &I, unsigned &err) {
  float acc = a.x, rot = a.y;
  if (!isfinite(acc)) {
    acc = 0.0f;
    err |= FLOCK_ERR_ACTION;
  }
  if (!isfinite(rot)) {
    rot = 0.0f;
    err |= FLOCK_ERR_ACTION;
  }
  const float amax = I.DS[2], tmax = I.DT[2];
  acc = acc < -amax ? -amax : (acc > amax ? amax : acc);
  rot = rot < -tmax ? -tmax : (rot > tmax ? tmax : rot);
  return move_agent(st, acc, rot, I);
}

// Tag action (speed, rotation), Section 4.2: sets the speed, clamped to
// [s_min, s_max], and turns the heading by the rotation clamped to
// [-Delta, Delta]; a non-finite component counts as 0 and is flagged.
__device__ __forceinline__ float4 apply_tag(float4 st, float2 a, const Inst &I, unsigned &err) {
  float spd = a.x, rot = a.y;
  if (!isfinite(spd)) {
    spd = 0.0f;
    err |= FLOCK_ERR_ACTION;
  }
  if (!isfinite(rot)) {
    rot = 0.0f;
    err |= FLOCK_ERR_ACTION;
  }
  const float tmax = I.DT[2];
  rot = rot < -tmax ? -tmax : (rot > tmax ? tmax : rot);
  spd = spd < I.SMIN ? I.SMIN : (spd > I.SMAX ? I.SMAX : spd);
  st.w = spd;
  return move_agent(st, 0.0f, rot, I);
}

// Element e of an observation row: for e < v the sector's (distance, count),
// for e == v (speed, heading); layout 1 keeps the distance (or the speed).
__device__ __forceinline__ void put_obs(const Inst &I, float *row, int e, float2 val) {
  if (I.obs_layout == 0) *reinterpret_cast<float2 *>(row + 2 * e) = val;
  else row[e] = val.x;
}

// Row of the instance's cell list that holds row gr of the square's grid
// (gr - row0 modulo nc; the identity for a whole square).
__device__ __forceinline__ int lrow(const Inst &I, int gr) {
  const int r = gr - I.row0;
  return r < 0 ? r + I.nc : r;
}

__device__ __forceinline__ int cell_of(float x, const Inst &I) {
  int c = __float2int_rz(fmul(x, I.invw));
  c = c < 0 ? 0 : c;
  return c >= I.nc ? I.nc - 1 : c;
}

// Warp-aggregated count of one agent in cell g; returns the agent's rank in
// its cell.  Lanes of a run of consecutive active lanes with the same cell
// share one atomic, taken by the run's first lane (agents stored near their
// cell neighbours form such runs).  A full match of equal cells across the
// warp (__match_any_sync) found almost nothing to merge for agents in random
// order and made the binning pass 40% slower, so only runs are merged.
__device__ __forceinline__ int warp_count(int *counts, int g) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int gp = __shfl_up_sync(m, g, 1);
  const bool head = lane == 0 || !((m >> (lane - 1)) & 1u) || gp != g;
  const unsigned heads = __ballot_sync(m, head);
  if (heads == m) return atomicAdd(&counts[g], 1);  // no runs: one atomic per lane
  // run of this lane: from its head to the lane before the next head (or the
  // end of the active lanes)
  const int first = 31 - __clz(heads & (below | (1u << lane)));
  const unsigned after = heads & ~(below | (1u << lane));
  const unsigned stop = after ? (after & (0u - after)) : 0u;  // lowest later head
  const unsigned span = (stop ? stop - 1u : 0xffffffffu) & ~((1u << first) - 1u) & m;
  int base = 0;
  if (head) base = atomicAdd(&counts[g], __popc(span));
  base = __shfl_sync(m, base, first);
  return base + __popc(span & below);
}

// ---------------------------------------------------------------------------
// Phase A: apply + bin one agent (instance-local index i).
// ---------------------------------------------------------------------------
// actions_inst / cactions_inst: the instance's discrete actions, or (when
// cactions_inst is not null) its continuous ones.
// Returns the agent's new state.
__device__ __forceinline__ float4 phaseA_agent(const Inst &I, int i, const int32_t *actions_inst,
                                               const float2 *cactions_inst, int reset,
                                               int *counts, int2 *cellrank, unsigned &err) {
  float4 st = I.state[i];
  if (!state_ok(st, I)) err |= FLOCK_ERR_STATE;
  if (!reset) {
    if (!cactions_inst) st = apply_action(st, actions_inst[i], I, err);
    else if (I.kind == 1) st = apply_tag(st, cactions_inst[i], I, err);
    else st = apply_cont(st, cactions_inst[i], I, err);
    I.state[i] = st;
  }
  const int g = I.cell_base + lrow(I, cell_of(st.y, I)) * I.nc + cell_of(st.x, I);
  if (!dbg_ok(g >= I.cell_base && g < I.cell_base + I.ncells)) return st;
  cellrank[I.agent_base + i] = make_int2(g, warp_count(counts, g));
  return st;
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan helpers (blockDim.x a multiple of 32, <= 1024).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread; returns the thread's exclusive
// prefix and writes the block total to *total.  wsum: >= 32 ints of smem.
__device__ __forceinline__ int block_excl_scan(int v, int *wsum, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  int inc = warp_incl_scan(v);
  __syncthreads();
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? wsum[lane] : 0;
    int wi = warp_incl_scan(w);
    if (lane < nw) wsum[lane] = wi - w;
    if (lane == nw - 1) wsum[32] = wi;
  }
  __syncthreads();
  int r = wsum[warp] + inc - v;
  *total = wsum[32];
  return r;
}

// In-place exclusive scan of a[0..n) in shared memory; a[n] = total.
__device__ __forceinline__ void block_excl_scan_inplace(int *a, int n, int *wsum) {
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per;
  int s = 0;
  for (int k = 0; k < per; ++k)
    if (lo + k < n) s += a[lo + k];
  int total;
  int run = block_excl_scan(s, wsum, &total);
  for (int k = 0; k < per; ++k)
    if (lo + k < n) {
      int t = a[lo + k];
      a[lo + k] = run;
      run += t;
    }
  if (threadIdx.x == 0) a[n] = total;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Phase B: exclusive scan of one tile of kScanTile cells.  Writes the
// in-tile exclusive prefix to local[], the tile total to tile_sum[t], and
// zeroes the counts for the next step.  sm: kScanTile + 33 ints.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void phaseB_tile(int t, const Bufs &B, int *sm) {
  const int c0 = t * kScanTile;
  const int m = min(kScanTile, B.c_total - c0);
  int *a = sm;
  int *wsum = sm + kScanTile + 1;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    a[k] = B.counts[c0 + k];
    B.counts[c0 + k] = 0;
  }
  __syncthreads();
  block_excl_scan_inplace(a, m, wsum);
  for (int k = threadIdx.x; k < m; k += blockDim.x) B.local[c0 + k] = a[k];
  if (threadIdx.x == 0) B.tile_sum[t] = a[m];
  __syncthreads();
}

// Prefix over the scan tiles, into smem tp[0..n_scan_tiles].
__device__ __forceinline__ void tile_prefix(const Bufs &B, int *tp, int *wsum) {
  for (int k = threadIdx.x; k < B.n_scan_tiles; k += blockDim.x) tp[k] = B.tile_sum[k];
  __syncthreads();
  block_excl_scan_inplace(tp, B.n_scan_tiles, wsum);
}

// Whole-grid exclusive scan of the cell counts by one block (the fused
// scan: the last block of the binning kernel, once every count is final):
// cell_start[c] = sum of counts[0..c), cell_start[C] = the total, counts
// zeroed for the next step.  Warp w takes cells [128 G w, 128 G (w + 1)) as
// G rounds of 32 lanes x 4 cells: coalesced 16-byte loads from L2 (where the
// count atomics landed), all in flight before the first is used.  The
// block scans the warps' totals; each warp then walks its rounds in order,
// a lane's group start being the warp's base, the carry of the earlier
// rounds and the lane's exclusive prefix within the round.  The counts
// array is padded with zeros to a multiple of 4 cells and cell_start holds
// C + 4 entries, so every access is a whole 16-byte group (entries past C
// hold the total).  Needs C <= 128 G (blockDim.x / 32).  wsum: >= 33 ints
// of shared memory.
template <int G>
__device__ __forceinline__ void scan_cells_block(const Bufs &B, int *wsum) {
  const int C = B.c_total, C4 = (C + 3) & ~3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lo = warp * 128 * G + 4 * lane;
  int4 v[G];
#pragma unroll
  for (int j = 0; j < G; ++j) {
    const int c = lo + 128 * j;
    v[j] = c < C4 ? __ldcg(reinterpret_cast<const int4 *>(B.counts + c)) : make_int4(0, 0, 0, 0);
  }
  int gs[G], t = 0;
#pragma unroll
  for (int j = 0; j < G; ++j) {
    gs[j] = v[j].x + v[j].y + v[j].z + v[j].w;
    t += gs[j];
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
  int total = 0;
  int base = block_excl_scan(lane == 0 ? t : 0, wsum, &total);
  base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
  for (int j = 0; j < G; ++j) {
    const int c = lo + 128 * j;
    int incl = gs[j];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int run = base + incl - gs[j];
    base += __shfl_sync(0xffffffffu, incl, 31);
    int4 st;
    st.x = run; run += v[j].x;
    st.y = run; run += v[j].y;
    st.z = run; run += v[j].z;
    st.w = run;
    if (c < C4) {
      *reinterpret_cast<int4 *>(B.cell_start + c) = st;
      *reinterpret_cast<int4 *>(B.counts + c) = make_int4(0, 0, 0, 0);
    }
  }
  if (C4 == C && threadIdx.x == 0) B.cell_start[C] = total;
}

// Writes agent f's sorted entries at position pos.
__device__ __forceinline__ void scatter_agent(int f, float4 st, int pos, const Bufs &B) {
  if ((unsigned)pos >= (unsigned)B.n_total) {  // inconsistent counts: never write out of range
    atomicOr(B.err, FLOCK_ERR_STATE);
    return;
  }
  B.sxy[pos] = make_float2(st.x, st.y);
  B.sidx[pos] = f;
  if (B.stype) B.stype[pos] = B.types[f];
}

// Phase C after the fused scan: position = cell start + rank in the cell.
__device__ __forceinline__ void phaseC_agent_final(int f, const float4 *state_i, const Bufs &B) {
  const int2 cr = B.cellrank[f];
  if (!dbg_ok(cr.x >= 0 && cr.x < B.c_total && cr.y >= 0)) return;
  scatter_agent(f, *state_i, B.cell_start[cr.x] + cr.y, B);
}

// Phase C for one agent (flattened index f, local index i of instance I):
// counting-sort scatter of its state into cell order.
__device__ __forceinline__ void phaseC_agent(int f, const float4 *state_i, const Bufs &B,
                                             const int *tp) {
  const int2 cr = B.cellrank[f];
  if (!dbg_ok(cr.x >= 0 && cr.x < B.c_total && cr.y >= 0)) return;
  scatter_agent(f, *state_i, tp[cr.x / kScanTile] + B.local[cr.x] + cr.y, B);
}

__device__ __forceinline__ void phaseC_cell(int c, const Bufs &B, const int *tp) {
  B.cell_start[c] = c == B.c_total ? B.n_total : tp[c / kScanTile] + B.local[c];
}

// ---------------------------------------------------------------------------
// Phase D: neighbour scan of one tile of cells.
//
// Layout of one tile: the block stages the tile's cells plus an H-cell halo
// (H = 1 for the 3 x 3 stencil, 2 for 5 x 5) from the cell-sorted positions
// into shared memory, row by row, each staged row being at most three
// contiguous runs of the sorted array (left halo across the periodic
// boundary, interior, right halo).  Every staged agent carries the periodic
// shift (0 or +-L per axis) that places its cell next to the tile.
//
// The tile's own agents are split evenly over the warps.  A warp takes up to
// 32 of them (one per lane) and
//   1. scans the candidates: each lane walks its 2H+1 stencil rows (each a
//      contiguous staged range), computes the minimum-image offset and d^2,
//      and appends in-range pairs (dx, dy, d^2, owner lane) to a per-warp
//      queue in shared memory (ballot compaction);
//   2. drains the queue 32 pairs at a time with every lane busy: collision
//      test, reward term, direction in the field-of-view frame, pseudo-angle
//      and sector; each pair updates its owner's accumulators in shared
//      memory with atomics (reward sum, sector minimum and count);
//   3. writes each agent's observation, reward and collision count at the
//      agent's own row.
// A tile whose staged agents exceed the shared buffer (a dense cluster) is
// processed by the direct per-thread path, reading the sorted arrays.
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;
constexpr int kQueue = 128;  // queued pairs per warp (tile form; lean direct form)
constexpr int kQueueWide = 160;  // queued pairs per warp, wide direct form

// x is an integer-valued float in [2^23, 2^62) or 0: its value as an
// integer, with 32-bit integer operations only (a float -> int64 conversion
// would run on the FP64 pipe).
__device__ __forceinline__ unsigned long long float_int_u64(float x) {
  const unsigned u = __float_as_uint(x);
  if (u == 0u) return 0ull;
  const unsigned m = (u & 0x7fffffu) | 0x800000u;
  return (unsigned long long)m << ((int)(u >> 23) - 150);
}

// Sector of pseudo-angle p: number of edges T[1..v-1] at or below p.
__device__ __forceinline__ int sector_of(float p, const float *T, int v) {
  int lo = 0, hi = v - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p >= T[mid]) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct Acc {
  unsigned long long acc;  // sum of ramp terms in units of 2^-K
  int nin, ncoll;
};

// Direct path: one candidate pair with its minimum-image offset (dx, dy).
// md/cn: this thread's per-sector minimum d^2 (as bits) and count, strided.
__device__ __forceinline__ void pair_core(float dx, float dy, const Inst &I, float ux, float uy,
                                          Acc &a, unsigned *md, int *cn, int stride) {
  const float d2 = fadd(fmul(dx, dx), fmul(dy, dy));
  if (!(d2 < I.RV2)) return;  // Eq. 1: d_ij < d_v
  a.nin++;
  if (d2 < I.RC2) {  // Fig. 4: collision below 2 d_r
    a.ncoll++;
  } else {
    const float t = fmul(fsub(I.RV, fsqrt(d2)), I.INV_SPAN);
    a.acc += float_int_u64(fmul(t, I.scaleK));  // exact: t is a multiple of 2^-K
  }
  const float lx = fadd(fmul(dx, ux), fmul(dy, uy));
  const float ly = fsub(fmul(dy, ux), fmul(dx, uy));
  if (lx == 0.0f && ly == 0.0f) return;  // coincident: no direction
  float p = pseudo_angle(lx, ly);
  if (p >= 4.0f) p = 0.0f;
  if (!I.full && p >= I.T[I.v]) return;  // outside the field of view
  const int k = sector_of(p, I.T, I.v);
  unsigned *m = md + k * stride;
  const unsigned db = __float_as_uint(d2);
  if (db < *m) *m = db;
  cn[k * stride] += 1;
}

__device__ __forceinline__ int wrapi(int c, int nc) { return c < 0 ? c + nc : (c >= nc ? c - nc : c); }

// Cooperative copy of a descriptor into shared memory (call, then sync).
__device__ __forceinline__ void load_inst(Inst &dst, const Inst *src) {
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Inst) / 4); k += blockDim.x) d[k] = s[k];
}

// Output of one agent from its accumulators.
__device__ __forceinline__ void write_agent(const Inst &I, const Bufs &B, int i, float s,
                                           float th, unsigned long long acc, int ncoll, int nin,
                                           const unsigned *md, const int *cn, int stride,
                                           unsigned &err) {
  float *o = B.obs + I.obs_base + (long long)i * I.obs_dim;
  for (int k = 0; k < I.v; ++k) {
    const int ck = cn[k * stride];
    const float dk = ck ? fsqrt(__uint_as_float(md[k * stride])) : I.RV;
    put_obs(I, o, k, make_float2(dk, (float)ck));
  }
  put_obs(I, o, I.v, make_float2(s, th));
  const long long total = (long long)acc - (long long)ncoll * I.PK;
  B.reward[I.agent_base + i] = fmul(__ll2float_rn(total), I.inv_scaleK);
  B.coll[I.agent_base + i] = ncoll;
  if ((long long)nin > I.NMAX) err |= FLOCK_ERR_OVERFLOW;
}

// Shared memory of phase D (dynamic), in bytes from the base:
//   float4 stg[cap]                      staged candidates (x, y, shift_x, shift_y)
//   int    cs[kMaxStagedCells + 1]       staged-cell prefix (row-major)
//   int    wsum[33], rs[kMaxTileH], rl[kMaxTileH]   scan scratch, the tile's rows
//   per warp: float4 queue[kQueue]; u64 acc[32]; int ncoll[32], nin[32];
//             u32 md[32 * v]; int cn[32 * v]
// I must be the block's shared-memory copy of the instance descriptor.
__host__ __device__ inline size_t phaseD_warp_bytes(int v) {
  return (size_t)kQueue * 16 + 32 * 8 + 32 * 4 * 2 + (size_t)32 * v * 8;
}
// bytes of the staged-cell prefix plus the scan scratch, rounded to 16
constexpr size_t kCsBytes =
    (((size_t)(kMaxStagedCells + 1) * 4 + (33 + 2 * kMaxTileH) * 4) + 15) & ~(size_t)15;
__host__ __device__ inline size_t phaseD_smem_bytes(int cap, int v, int block) {
  return (size_t)cap * 16 + kCsBytes + (size_t)(block / 32) * phaseD_warp_bytes(v);
}

struct WarpArea {
  float4 *queue;
  unsigned long long *acc;
  int *ncoll, *nin;
  unsigned *md;
  int *cn;
};

// Drain `count` queued pairs (warp-uniform); ux/uy: this lane's own agent.
// Every lane takes one pair per round whatever its owner; the owner's
// accumulators are updated with shared-memory atomics (a round holds pairs of
// many owners, so they rarely collide).  In this path an agent has at most
// `cap` <= 4096 in-range neighbours, so in-range and collision counts share
// one 32-bit word (low and high 16 bits).
__device__ __forceinline__ void drain(const Inst &I, const WarpArea &W, int count, float ux,
                                     float uy) {
  const int lane = threadIdx.x & 31;
  const int v = I.v;
  for (int e0 = 0; e0 < count; e0 += 32) {
    const int e = e0 + lane;
    const bool valid = e < count;
    float4 E = valid ? W.queue[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int o = valid ? __float_as_int(E.w) : lane;
    const float uxo = __shfl_sync(kFull, ux, o), uyo = __shfl_sync(kFull, uy, o);
    if (valid) {
      const float dx = E.x, dy = E.y, d2 = E.z;
      const bool coll = d2 < I.RC2;
      if (!coll) {
        const float t = fmul(fsub(I.RV, fsqrt(d2)), I.INV_SPAN);
        const unsigned long long tv = float_int_u64(fmul(t, I.scaleK));
        if (tv) sred_add_u64(smem_u32(W.acc) + 8u * (unsigned)o, tv);
      }
      sred_add_u32(smem_u32(W.ncoll) + 4u * (unsigned)o, coll ? 0x10001u : 1u);
      const float lx = fadd(fmul(dx, uxo), fmul(dy, uyo));
      const float ly = fsub(fmul(dy, uxo), fmul(dx, uyo));
      if (lx != 0.0f || ly != 0.0f) {
        float p = pseudo_angle(lx, ly);
        if (p >= 4.0f) p = 0.0f;
        if (I.full || p < I.T[v]) {
          const int key = sector_of(p, I.T, v);
          const unsigned off = 4u * (unsigned)(o * v + key);
          sred_min_u32(smem_u32(W.md) + off, __float_as_uint(d2));
          sred_add_u32(smem_u32(W.cn) + off, 1u);
        }
      }
    }
  }
  __syncwarp();
}

// Candidate scan of one lane's stencil rows (smem ranges [ra[r], ra[r]+rn[r])),
// appending in-range pairs to the warp queue; drains when nearly full.
template <int H, bool WRAP>
__device__ __forceinline__ void scan_rows(const Inst &I, const WarpArea &W, const float4 *stg,
                                          const int *ra, const int *rn, int self, float xi,
                                          float yi, float ux, float uy) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int qn = 0;
#pragma unroll
  for (int r = 0; r < 2 * H + 1; ++r) {
    const int n = rn[r];
    const int maxn = __reduce_max_sync(kFull, (unsigned)n);
    for (int j = 0; j < maxn; ++j) {
      const int q = ra[r] + j;
      bool inr = false;
      float dx = 0.f, dy = 0.f, d2 = 0.f;
      if (j < n && q != self) {
        const float4 e = stg[q];
        dx = fsub(e.x, xi);
        dy = fsub(e.y, yi);
        if (WRAP) {
          dx = fadd(dx, e.z);
          dy = fadd(dy, e.w);
        }
        d2 = fadd(fmul(dx, dx), fmul(dy, dy));
        inr = d2 < I.RV2;  // Eq. 1: d_ij < d_v
      }
      const unsigned m = __ballot_sync(kFull, inr);
      if (inr) W.queue[qn + __popc(m & lt)] = make_float4(dx, dy, d2, __int_as_float(lane));
      qn += __popc(m);
      if (qn > kQueue - 32) {
        __syncwarp();
        drain(I, W, qn, ux, uy);
        qn = 0;
      }
    }
  }
  __syncwarp();
  drain(I, W, qn, ux, uy);
}

template <int H>
__device__ void phaseD_tile(const Inst &I, int tx, int ty, const Bufs &B, char *smem,
                            unsigned &err) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  float4 *stg = reinterpret_cast<float4 *>(smem);
  int *cs = reinterpret_cast<int *>(smem + (size_t)I.cap * 16);
  int *wsum = cs + kMaxStagedCells + 1;
  char *wbase = smem + (size_t)I.cap * 16 + kCsBytes;  // 16-byte aligned
  const int nc = I.nc, v = I.v;
  const int c0 = tx * I.tile_w, c1 = min(c0 + I.tile_w, nc);
  const int r0 = ty * I.tile_h, r1 = min(r0 + I.tile_h, nc);
  const int tw = c1 - c0, th = r1 - r0;
  const int nsc = tw + 2 * H, nsr = th + 2 * H, ncell = nsc * nsr;
  const int *cst = B.cell_start;

  // the tile's own rows in the sorted order, and the staged-cell counts
  // (row-major over staged row, staged column)
  int *rs = wsum + 33, *rl = rs + kMaxTileH;
  if (tid < th) {
    const int rg = I.cell_base + (r0 + tid) * nc;
    rs[tid] = cst[rg + c0];
    rl[tid] = cst[rg + c1] - rs[tid];
  }
  for (int e = tid; e < ncell; e += nthr) {
    const int sr = e / nsc, sc = e - sr * nsc;
    const int g = I.cell_base + wrapi(r0 - H + sr, nc) * nc + wrapi(c0 - H + sc, nc);
    cs[e] = cst[g + 1] - cst[g];
  }
  __syncthreads();
  block_excl_scan_inplace(cs, ncell, wsum);
  const int staged = cs[ncell];
  const bool use_smem = staged <= I.cap;
  const bool wraps = c0 - H < 0 || c1 + H > nc || r0 - H < 0 || r1 + H > nc;

  if (use_smem) {
    // one warp per staged row; a row is at most three contiguous runs
    for (int sr = warp; sr < nsr; sr += nwarps) {
      const int vr = r0 - H + sr;
      const float sy = vr < 0 ? -I.L : (vr >= nc ? I.L : 0.0f);
      const int rowg = I.cell_base + wrapi(vr, nc) * nc;
      const int vlo = c0 - H, vhi = c1 + H;
#pragma unroll
      for (int part = 0; part < 3; ++part) {
        int a, b, off;
        float sx;
        if (part == 0) { a = vlo; b = min(0, vhi); off = nc; sx = -I.L; }
        else if (part == 1) { a = max(vlo, 0); b = min(vhi, nc); off = 0; sx = 0.0f; }
        else { a = max(vlo, nc); b = vhi; off = -nc; sx = I.L; }
        if (a >= b) continue;
        const int gs = cst[rowg + a + off], ge = cst[rowg + b + off];
        const int ss = cs[sr * nsc + (a - vlo)];
        for (int q = lane; q < ge - gs; q += 32) {
          const float2 pxy = B.sxy[gs + q];
          stg[ss + q] = make_float4(pxy.x, pxy.y, sx, sy);
        }
      }
    }
  }
  __syncthreads();

  // the tile's own agents: row r (0..th-1) holds sorted positions
  // [rs[r], rs[r] + rl[r]); rs/rl were filled during staging
  int ncent = 0;
  for (int r = 0; r < th; ++r) ncent += rl[r];

  if (use_smem) {
    WarpArea W;
    char *wp = wbase + (size_t)warp * phaseD_warp_bytes(v);
    W.queue = reinterpret_cast<float4 *>(wp);
    W.acc = reinterpret_cast<unsigned long long *>(wp + kQueue * 16);
    W.ncoll = reinterpret_cast<int *>(wp + kQueue * 16 + 32 * 8);
    W.nin = W.ncoll + 32;
    W.md = reinterpret_cast<unsigned *>(W.nin + 32);
    W.cn = reinterpret_cast<int *>(W.md + 32 * v);
    // output rows are written cooperatively: P float2 per row, rpi rows per
    // pass of the warp (lane -> row lane / P, element lane % P)
    const int P = v + 1;
    const int rpi = P <= 32 ? 32 / P : 1;
    const int my_r = P <= 32 ? lane / P : 0, my_e = P <= 32 ? lane % P : lane;
    // contiguous, even share of the tile's agents per warp
    const int per = (ncent + nwarps - 1) / nwarps;
    const int wa0 = warp * per, wa1 = min(wa0 + per, ncent);
    for (int b0 = wa0; b0 < wa1; b0 += 32) {
      const int a = b0 + lane;
      const int nb = min(32, wa1 - b0);
      const bool have = a < wa1;
      int self = -1, i = 0, sr = 0, lc = 0;
      float xi = 0.f, yi = 0.f;
      float2 ts = make_float2(0.f, 0.f);
      if (have) {
        int r = 0, al = a;
        while (al >= rl[r]) {
          al -= rl[r];
          ++r;
        }
        sr = r + H;
        self = cs[sr * nsc + H] + al;  // interior run of the row, in sorted order
        const int gp = rs[r] + al;
        i = B.sidx[gp] - I.agent_base;
        const float4 s4 = I.state[i];  // own heading and speed
        ts = make_float2(s4.z, s4.w);
        const float4 e = stg[self];
        xi = e.x;
        yi = e.y;
        lc = cell_of(xi, I) - c0 + H;
      }
      float c = 1.f, sn = 0.f;
      det_sincos(ts.x, c, sn);
      const float ux = fadd(fmul(c, I.CF), fmul(sn, I.SF));
      const float uy = fsub(fmul(sn, I.CF), fmul(c, I.SF));
      W.acc[lane] = 0ull;
      W.ncoll[lane] = 0;
      for (int k = 0; k < v; ++k) {
        W.md[lane * v + k] = 0x7f800000u;
        W.cn[lane * v + k] = 0;
      }
      int ra[2 * H + 1], rn[2 * H + 1];
#pragma unroll
      for (int r = 0; r < 2 * H + 1; ++r) {
        if (have) {
          const int row = sr - H + r;
          ra[r] = cs[row * nsc + lc - H];
          rn[r] = cs[row * nsc + lc + H + 1] - ra[r];
        } else {
          ra[r] = 0;
          rn[r] = 0;
        }
      }
      __syncwarp();
      if (wraps)
        scan_rows<H, true>(I, W, stg, ra, rn, self, xi, yi, ux, uy);
      else
        scan_rows<H, false>(I, W, stg, ra, rn, self, xi, yi, ux, uy);
      __syncwarp();
      // reward and collisions: one value per agent
      if (have) {
        const unsigned packed = (unsigned)W.ncoll[lane];  // in-range | collisions << 16
        const int ncoll = (int)(packed >> 16);
        const long long total = (long long)W.acc[lane] - (long long)ncoll * I.PK;
        B.reward[I.agent_base + i] = fmul(__ll2float_rn(total), I.inv_scaleK);
        B.coll[I.agent_base + i] = ncoll;
        if ((long long)(packed & 0xffffu) > I.NMAX) err |= FLOCK_ERR_OVERFLOW;
      }
      // observation rows, written whole and contiguous
      float *obs = B.obs + I.obs_base;
      for (int rb = 0; rb < nb; rb += rpi) {
        const int r = min(rb + my_r, 31);
        const int ir = __shfl_sync(kFull, i, r);
        const float sr_ = __shfl_sync(kFull, ts.y, r), tr = __shfl_sync(kFull, ts.x, r);
        if (rb + my_r < nb && my_r < rpi) {
          for (int e = my_e; e < P; e += 32) {
            float2 val;
            if (e < v) {
              const int ck = W.cn[r * v + e];
              val = make_float2(ck ? fsqrt(__uint_as_float(W.md[r * v + e])) : I.RV, (float)ck);
            } else {
              val = make_float2(sr_, tr);
            }
            put_obs(I, obs + (long long)ir * I.obs_dim, e, val);
          }
        }
      }
      __syncwarp();
    }
  } else {
    // dense tile: per-thread scan straight from the sorted arrays, with the
    // per-sector accumulators strided by the block size
    unsigned *md = reinterpret_cast<unsigned *>(wbase);
    int *cn = reinterpret_cast<int *>(md + (size_t)v * nthr);
    for (int a0 = 0; a0 < ncent; a0 += nthr) {
      const int a = a0 + tid;
      if (a >= ncent) continue;
      int r = 0, al = a, rg = 0, rlen = 0;
      for (;; ++r) {
        rg = I.cell_base + (r0 + r) * nc;
        rlen = cst[rg + c1] - cst[rg + c0];
        if (al < rlen) break;
        al -= rlen;
      }
      const int gp = cst[rg + c0] + al;
      const int i = B.sidx[gp] - I.agent_base;
      const float4 me = I.state[i];
      float c, sn;
      det_sincos(me.z, c, sn);
      const float ux = fadd(fmul(c, I.CF), fmul(sn, I.SF));
      const float uy = fsub(fmul(sn, I.CF), fmul(c, I.SF));
      const int cx = cell_of(me.x, I);
      for (int k = 0; k < v; ++k) {
        md[k * nthr + tid] = 0x7f800000u;
        cn[k * nthr + tid] = 0;
      }
      Acc acc{0ull, 0, 0};
      const int cy = r0 + r;
      for (int dr = -H; dr <= H; ++dr) {
        const int vr = cy + dr;
        const float sy = vr < 0 ? -I.L : (vr >= nc ? I.L : 0.0f);
        const int rowg = I.cell_base + wrapi(vr, nc) * nc;
        for (int dc = -H; dc <= H; ++dc) {
          const int vc = cx + dc;
          const float sx = vc < 0 ? -I.L : (vc >= nc ? I.L : 0.0f);
          const int g = rowg + wrapi(vc, nc);
          const int ga = cst[g], gb = cst[g + 1];
          for (int gq = ga; gq < gb; ++gq) {
            if (gq == gp) continue;
            const float2 pxy = B.sxy[gq];
            const float dx = fadd(fsub(pxy.x, me.x), sx);
            const float dy = fadd(fsub(pxy.y, me.y), sy);
            pair_core(dx, dy, I, ux, uy, acc, md + tid, cn + tid, nthr);
          }
        }
      }
      write_agent(I, B, i, me.w, me.z, acc.acc, acc.ncoll, acc.nin, md + tid, cn + tid, nthr,
                  err);
    }
  }
  __syncthreads();  // smem is reused by the next tile
}


// ---------------------------------------------------------------------------
// Phase D, direct form: one warp handles up to 32 consecutive cell-sorted
// agents of one instance (sorted positions [gp0, gp1)), with no block-level
// staging.  Neighbouring lanes are in the same or adjacent cells, so their
// stencil rows overlap and the candidate reads hit L1; nothing waits on
// other warps.  Per stencil row a lane's candidates are at most three
// contiguous runs of the sorted array (cells across the left boundary, the
// cells inside, cells across the right boundary), each with its own
// periodic shift.  Pair processing (queue, drain) and the output are the
// same as in the staged form.  smem: this warp's WarpArea.
// ---------------------------------------------------------------------------
struct DirectArea {
  float4 *queue;
  unsigned long long *acc;  // [32]: each owner lane's reward sum (units of 2^-K)
  unsigned *accp;           // [3][32]: pieces of the current drain (bits 0-23, 24-47, 48-)
  int *nin, *ncoll;
  unsigned *md;  // per-sector minimum distance (bits of a non-negative float)
  int *cn;
};

// Bytes of one warp's area for v sectors and A agents per warp (32 / lanes
// per agent): the per-sector minima and counts take A rows of v.
// q: the queue capacity (kQueueWide for the standalone kernels, kQueue for
// the batched kernel).  Rounded up to 16 bytes: the warps' areas follow one
// another and each starts with the float4 queue (one agent per warp with an
// odd v leaves A v 8 = 8 mod 16).
__host__ __device__ inline size_t direct_warp_bytes(int v, int A = 32, int q = kQueueWide) {
  const size_t b = (size_t)q * 16 + 32 * 8 + 3 * 32 * 4 + 32 + 32 * 4 * 2 + (size_t)A * v * 8;
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ DirectArea direct_area(char *base, int v, int A = 32,
                                                  int q = kQueueWide) {
  DirectArea W;
  W.queue = reinterpret_cast<float4 *>(base);
  W.acc = reinterpret_cast<unsigned long long *>(base + q * 16);
  W.accp = reinterpret_cast<unsigned *>(base + q * 16 + 32 * 8);
  W.nin = reinterpret_cast<int *>(base + q * 16 + 32 * 8 + 3 * 32 * 4 + 32);
  W.ncoll = W.nin + 32;
  W.md = reinterpret_cast<unsigned *>(W.ncoll + 32);
  W.cn = reinterpret_cast<int *>(W.md + A * v);
  return W;
}

// Sector search with the edges in registers: for V = 8 a three-level
// binary search over T[1..7] with selects; otherwise the generic search.
template <int V>
struct Edges {
  float t[8];
  __device__ __forceinline__ void load(const Inst &I) {
    if (V == 8) {
#pragma unroll
      for (int m = 0; m < 8; ++m) t[m] = I.T[m + 1];
    }
  }
  // returns the sector, or -1 when outside the field of view
  __device__ __forceinline__ int sector(const Inst &I, float p) const {
    if (V == 8) {
      const bool out = !I.full && p >= t[7];
      const bool b2 = p >= t[3];
      const float t1 = b2 ? t[5] : t[1];
      const bool b1 = p >= t1;
      const float t0 = b2 ? (b1 ? t[6] : t[4]) : (b1 ? t[2] : t[0]);
      const bool b0 = p >= t0;
      const int k = (b2 ? 4 : 0) + (b1 ? 2 : 0) + (b0 ? 1 : 0);
      return out ? -1 : k;
    } else {
      if (!I.full && p >= I.T[I.v]) return -1;
      return sector_of(p, I.T, I.v);
    }
  }
};

// Adds one reward term (units of 2^-K) to owner o's sum.  PIECES: as 24-bit
// pieces with 32-bit atomics (a drain holds at most kQueueWide terms, so each
// piece sum stays below 2^24 * kQueueWide and exact); else one 64-bit atomic.
template <bool PIECES>
__device__ __forceinline__ void add_term(const Inst &I, const DirectArea &W, int o,
                                         unsigned long long tv) {
  if (!tv) return;
  if (PIECES) {
    const unsigned a = smem_u32(W.accp) + 4u * (unsigned)o;
    sred_add_u32(a, (unsigned)tv & 0xffffffu);
    sred_add_u32(a + 128u, (unsigned)(tv >> 24) & 0xffffffu);
    if (I.pieces > 2) sred_add_u32(a + 256u, (unsigned)(tv >> 48));
  } else {
    sred_add_u64(smem_u32(W.acc) + 8u * (unsigned)o, tv);
  }
}

// x[r] for a run-time r < N, by selects (a dynamic index would put x in
// local memory).
template <int N>
__device__ __forceinline__ int pick(const int (&x)[N], int r) {
  int v = x[0];
#pragma unroll
  for (int k = 1; k < N; ++k) v = r == k ? x[k] : v;
  return v;
}

// Drain for the direct form.  In-range and collision counts are kept by the
// owner lanes during the candidate scan; here each queued pair adds its ramp
// term (non-colliding pairs) and its sector minimum and count.
// PIECES: add each term as 24-bit pieces with 32-bit shared atomics and fold
// them into the 64-bit sums once per drain (64-bit shared atomics are slow);
// without it, one 64-bit atomic per term (fewer registers, which the batched
// kernel needs to keep four blocks per SM).  Both sums are exact integers.
//
// TAG (Section 4.2): the queue entry's owner word also carries the
// neighbour's type (bit 8); ti is each lane's own agent type.  A runner's
// ramp terms come from runners only (its touches cost -P through the
// collision count, whatever the type); a chaser adds +P per touched runner.
// The sector accumulators hold two channels of v, the neighbour's type
// choosing the channel.
//
// ONE (one agent per warp, 32 lanes per agent): every queued pair belongs to
// that agent, so each lane adds its terms to its own register sum `racc`
// (added up over the warp at the end) instead of shared-memory atomics that
// would all hit one word, and the agent's frame needs no shuffle.
template <int V, bool PIECES, bool TAG = false, bool ONE = false>
__device__ __forceinline__ int drain_direct(const Inst &I, const DirectArea &W, int count,
                                           float ux, float uy, const Edges<V> &E8, int ti,
                                           unsigned long long &racc, bool all = true) {
  const int lane = threadIdx.x & 31;
  const int v = V == 8 ? 8 : I.v;
  const int vs = TAG ? 2 * v : v;  // accumulator row length
  const unsigned q_s = smem_u32(W.queue), md_s = smem_u32(W.md), cn_s = smem_u32(W.cn);
  const unsigned ap_s = smem_u32(W.accp), a64_s = smem_u32(W.acc);
  // mid-scan, only whole rounds of 32 pairs are taken; the rest stays queued
  const int take = all ? count : (count & ~31);
  // Branch-free pair body: every lane computes every quantity (an idle lane
  // on a harmless stand-in pair) and the shared-memory updates carry their
  // condition as a predicate.
  for (int e0 = 0; e0 < take; e0 += 32) {
    const int e = e0 + lane;
    const bool valid = e < take;
    const float4 E = sld_f4(q_s + 16u * (unsigned)(valid ? e : 0));
    const int w = valid ? __float_as_int(E.w) : 0;
    const int o = ONE ? 0 : (TAG ? (w & 0xff) : w);
    const int tj = TAG ? (w >> 8) : 0;
    const float uxo = ONE ? ux : __shfl_sync(kFull, ux, o);
    const float uyo = ONE ? uy : __shfl_sync(kFull, uy, o);
    const int tio = TAG ? (ONE ? ti : __shfl_sync(kFull, ti, o)) : 0;
    const float dx = valid ? E.x : 1.0f, dy = valid ? E.y : 0.0f;
    const float d2 = valid ? E.z : 1.0f;
    const bool coll = d2 < I.RC2;
    // the distance: the ramp term's, and the sector minimum's (sqrt is
    // monotone, so the minimum of the rounded roots is the rounded root of
    // the minimum d^2)
    const float dist = fsqrt(d2);
    // reward term of this pair for its owner (units of 2^-K): the ramp of
    // Fig. 4 for a non-colliding pair; for tag a runner's ramp counts runners
    // only, and a chaser earns P per runner it touches
    bool ramp, touch = false;
    if constexpr (!TAG) {
      ramp = valid && !coll;
    } else {
      ramp = valid && tio == 0 && tj == 0 && !coll;
      touch = valid && tio == 1 && tj == 0 && coll;
    }
    const float t = fmul(fsub(I.RV, dist), I.INV_SPAN);
    unsigned long long tv = float_int_u64(fmul(ramp ? t : 0.0f, I.scaleK));
    if (TAG) tv = touch ? (unsigned long long)I.PK : tv;
    if (ONE) {
      racc += tv;
    } else if (PIECES) {
      const unsigned pa = ap_s + 4u * (unsigned)o;
      const bool nz = tv != 0ull;
      sred_add_u32_if(nz, pa, (unsigned)tv & 0xffffffu);
      sred_add_u32_if(nz, pa + 128u, (unsigned)(tv >> 24) & 0xffffffu);
      sred_add_u32_if(nz && I.pieces > 2, pa + 256u, (unsigned)(tv >> 48));
    } else {
      sred_add_u64_if(tv != 0ull, a64_s + 8u * (unsigned)o, tv);
    }
    // direction in the owner's field-of-view frame, pseudo-angle, sector
    const float lx = fadd(fmul(dx, uxo), fmul(dy, uyo));
    const float ly = fsub(fmul(dy, uxo), fmul(dx, uyo));
    const bool dir = lx != 0.0f || ly != 0.0f;  // coincident agents have none
    float p = pseudo_angle(dir ? lx : 1.0f, ly);
    if (p >= 4.0f) p = 0.0f;
    int key = E8.sector(I, p);
    const bool seen = valid && dir && key >= 0 && dbg_ok(key < v && o < 32);
    if (TAG) key += tj * v;  // colour channel of the neighbour's type
    const unsigned off = 4u * (unsigned)(o * vs + (seen ? key : 0));
    sred_min_u32_if(seen, md_s + off, __float_as_uint(dist));
    sred_add_u32_if(seen, cn_s + off, 1u);
  }
  __syncwarp();
  // the pairs not taken move to the front of the queue
  const int rest = count - take;
  if (rest > 0) {
    const bool mv = lane < rest;
    const float4 E = sld_f4(q_s + 16u * (unsigned)(take + (mv ? lane : 0)));
    __syncwarp();
    sst_f4_if(mv, q_s + 16u * (unsigned)lane, E);
    __syncwarp();
  }
  if (!PIECES || ONE) return rest;
  // each lane folds its own pieces into its 64-bit sum
  W.acc[lane] += (unsigned long long)W.accp[lane] +
                 ((unsigned long long)W.accp[32 + lane] << 24) +
                 ((unsigned long long)W.accp[64 + lane] << 48);
  W.accp[lane] = 0u;
  W.accp[32 + lane] = 0u;
  W.accp[64 + lane] = 0u;
  __syncwarp();
  return rest;
}

// One run of candidates [a, a + n) with shifts (sx, sy); appends in-range
// pairs to the queue (warp-uniform loop), draining when nearly full.
// With LPA lanes per agent, lane l serves agent slot l % (32 / LPA) and
// takes every LPA-th candidate of the run, starting at l / (32 / LPA).
template <bool SHIFT, int V, bool PIECES, int LPA, bool TAG = false>
__device__ __forceinline__ void direct_run(const Inst &I, const DirectArea &W, const float2 *sxy,
                                           int a, int n, int self, float sx, float sy, float xi,
                                           float yi, float ux, float uy, int &qn, int &nin,
                                           int &ncoll, const Edges<V> &E8,
                                           const uint8_t *stype, int ti,
                                           unsigned long long &racc) {
  constexpr int A = 32 / LPA;
  constexpr bool ONE = A == 1;
  const int lane = threadIdx.x & 31;
  const int slot = lane & (A - 1), sub = lane / A;
  const unsigned lt = (1u << lane) - 1u;
  const int maxn = __reduce_max_sync(kFull, (unsigned)n);
  if constexpr (!PIECES) {
    // lean form (the batched kernel, 64 registers): one candidate per lane
    // and pass, the agent itself skipped
    for (int j0 = 0; j0 < maxn; j0 += LPA) {
      const int j = j0 + sub;
      const int q = a + j;
      bool inr = false;
      float dx = 0.f, dy = 0.f, d2 = 0.f;
      if (j < n && q != self) {
        const float2 p = __ldg(sxy + q);
        dx = fsub(p.x, xi);
        dy = fsub(p.y, yi);
        if (SHIFT) {
          dx = fadd(dx, sx);
          dy = fadd(dy, sy);
        }
        d2 = fadd(fmul(dx, dx), fmul(dy, dy));
        inr = d2 < I.RV2;  // Eq. 1: d_ij < d_v
        if (inr) {
          nin++;
          ncoll += d2 < I.RC2 ? 1 : 0;  // Fig. 4: collision below 2 d_r
        }
      }
      const unsigned m = __ballot_sync(kFull, inr);
      const int w = TAG ? (slot | ((int)(inr && stype[q] != 0) << 8)) : slot;
      sst_f4_if(inr, smem_u32(W.queue) + 16u * (unsigned)(qn + __popc(m & lt)),
                make_float4(dx, dy, d2, __int_as_float(w)));
      qn += __popc(m);
      if (qn > kQueue - 32) {
        __syncwarp();
        qn = drain_direct<V, PIECES, TAG, ONE>(I, W, qn, ux, uy, E8, ti, racc, false);
      }
    }
    return;
  }
  // wide form: two candidates per lane and pass (their loads in flight
  // together), one drain test per pass
  for (int j0 = 0; j0 < maxn; j0 += 2 * LPA) {
    const int ja = j0 + sub, jb = ja + LPA;
    bool ina = false, inb = false;
    float dxa = 0.f, dya = 0.f, d2a = 0.f, dxb = 0.f, dyb = 0.f, d2b = 0.f;
    float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
    if (ja < n) pa = __ldg(sxy + a + ja);
    if (jb < n) pb = __ldg(sxy + a + jb);
    if (ja < n) {
      dxa = fsub(pa.x, xi);
      dya = fsub(pa.y, yi);
      if (SHIFT) {
        dxa = fadd(dxa, sx);
        dya = fadd(dya, sy);
      }
      d2a = fadd(fmul(dxa, dxa), fmul(dya, dya));
      ina = d2a < I.RV2 && a + ja != self;  // Eq. 1: d_ij < d_v, j != i
    }
    if (jb < n) {
      dxb = fsub(pb.x, xi);
      dyb = fsub(pb.y, yi);
      if (SHIFT) {
        dxb = fadd(dxb, sx);
        dyb = fadd(dyb, sy);
      }
      d2b = fadd(fmul(dxb, dxb), fmul(dyb, dyb));
      inb = d2b < I.RV2 && a + jb != self;
    }
    nin += (ina ? 1 : 0) + (inb ? 1 : 0);
    ncoll += (ina && d2a < I.RC2 ? 1 : 0) + (inb && d2b < I.RC2 ? 1 : 0);  // Fig. 4
    const unsigned ma = __ballot_sync(kFull, ina), mb = __ballot_sync(kFull, inb);
    const unsigned q_s = smem_u32(W.queue);
    {
      const int w = TAG ? (slot | ((int)(ina && stype[a + ja] != 0) << 8)) : slot;
      sst_f4_if(ina, q_s + 16u * (unsigned)(qn + __popc(ma & lt)),
                make_float4(dxa, dya, d2a, __int_as_float(w)));
    }
    qn += __popc(ma);
    {
      const int w = TAG ? (slot | ((int)(inb && stype[a + jb] != 0) << 8)) : slot;
      sst_f4_if(inb, q_s + 16u * (unsigned)(qn + __popc(mb & lt)),
                make_float4(dxb, dyb, d2b, __int_as_float(w)));
    }
    qn += __popc(mb);
    if (qn > kQueueWide - 64) {
      __syncwarp();
      qn = drain_direct<V, PIECES, TAG, ONE>(I, W, qn, ux, uy, E8, ti, racc, false);
    }
  }
}

// ---------------------------------------------------------------------------
// Policy network: the shared MLP of the learners (Section 4.3; two hidden
// layers of 64 with tanh, here 18 -> 64 -> 64 -> 9 on the 18-value
// observation), run in the neighbour scan's epilogue on each warp's own
// agents (policy_warp_rows).  BF16 operands on the tensor cores (mma.sync
// m16n8k16 and m16n8k8), FP32 accumulate; the greedy action (largest logit,
// lowest index on ties) is written back.  The weights reach the lanes as an
// operand image built from the blob at the start of the step (see
// policy_image); each layer's accumulators, rounded to BF16 pairs and passed
// through the hardware BF16 tanh, are the next layer's A fragments without
// leaving the registers.
// ---------------------------------------------------------------------------
// offsets in the 5,961-value BF16 blob: W1[64][18] b1[64] W2[64][64] b2[64] W3[9][64] b3[9]
constexpr int kOffB1 = 64 * 18, kOffW2 = kOffB1 + 64, kOffB2 = kOffW2 + 64 * 64,
              kOffW3 = kOffB2 + 64, kOffB3 = kOffW3 + 9 * 64, kBlobLen = kOffB3 + 9;
static_assert(kOffB1 % 2 == 0 && kOffW2 % 2 == 0 && kOffB2 % 2 == 0 && kOffW3 % 2 == 0 &&
                  kOffB3 % 2 == 0,
              "every matrix and bias of the blob starts on a BF16 pair");

// Operand image: for lane (g, t) = (lane / 4, lane % 4) the 116 words it
// feeds the forward pass, in the order of use, as 29 uint4 stored
// lane-interleaved (vector j of lane l at j * 32 + l: a warp-wide load is 512
// contiguous bytes).  Every pair of B words an m16n8k16 takes sits in one
// aligned half of a vector.  The biases enter as products with a constant 1
// in an m16n8k8 step (no accumulator initialisation).  n = 8 nt + g is the
// output row a word serves.  Word ranges per lane:
//   [0, 16)    layer 1, columns 0-15, word 2 nt + r: W1[n][2t + 8r, 2t + 8r + 1]
//   [16, 24)   layer 1, columns 16-23, word 16 + nt: (t = 0) W1[n][16, 17],
//              (t = 1) (b1[n], 0): the observation's column 18 is the constant 1
//   [24, 88)   layer 2, q = s - 24: k-step q / 16, n-tile (q / 2) % 8, the
//              pair at column offset 8 (q % 2)
//   [88, 96)   b2, word 88 + nt: (t = 0) (b2[n], 0)
//   [96, 112)  layer 3, q = s - 96: k-step q / 4, n-tile (q / 2) % 2, pair
//              q % 2; rows 9-15 of W3 are zero
//   [112, 116) b3, word 112 + nt (nt < 2): (t = 0, n < 9) (b3[n], 0); 0, 0
constexpr int kImgWords = 116, kImgVecs = kImgWords / 4;
constexpr int kImgL1K8 = 16, kImgL2 = 24, kImgB2 = 88, kImgL3 = 96, kImgB3 = 112;
constexpr size_t kImgBytes = (size_t)kImgVecs * 32 * 16;

__device__ __forceinline__ unsigned blob_pair(const unsigned short *__restrict__ blob, int e) {
  return *reinterpret_cast<const unsigned *>(blob + e);  // e even, blob 4-byte aligned
}

__device__ __forceinline__ unsigned image_word(const unsigned short *__restrict__ blob, int s, int g,
                                               int t) {
  if (s < kImgL1K8) {
    const int nt = s >> 1, r = s & 1;
    return blob_pair(blob, (8 * nt + g) * 18 + 2 * t + 8 * r);
  }
  if (s < kImgL2) {
    const int n = 8 * (s - kImgL1K8) + g;
    if (t == 0) return blob_pair(blob, n * 18 + 16);
    return t == 1 ? (unsigned)blob[kOffB1 + n] : 0u;
  }
  if (s < kImgB2) {
    const int q = s - kImgL2, kk = q >> 4, nt = (q >> 1) & 7, r = q & 1;
    return blob_pair(blob, kOffW2 + (8 * nt + g) * 64 + 16 * kk + 2 * t + 8 * r);
  }
  if (s < kImgL3) return t == 0 ? (unsigned)blob[kOffB2 + 8 * (s - kImgB2) + g] : 0u;
  if (s < kImgB3) {
    const int q = s - kImgL3, kk = q >> 2, nt = (q >> 1) & 1, r = q & 1, n = 8 * nt + g;
    return n < 9 ? blob_pair(blob, kOffW3 + n * 64 + 16 * kk + 2 * t + 8 * r) : 0u;
  }
  const int n = 8 * (s - kImgB3) + g;
  return s < kImgB3 + 2 && t == 0 && n < 9 ? (unsigned)blob[kOffB3 + n] : 0u;
}

// Writes image vectors idx, idx + stride, ... (call with the grid's thread
// index and size; kImgVecs * 32 vectors in all).
__device__ __forceinline__ void policy_image(const unsigned short *__restrict__ blob, uint4 *img,
                                             int idx, int stride) {
  for (; idx < kImgVecs * 32; idx += stride) {
    const int j = idx >> 5, l = idx & 31, g = l >> 2, t = l & 3;
    img[idx] = make_uint4(image_word(blob, 4 * j, g, t), image_word(blob, 4 * j + 1, g, t),
                          image_word(blob, 4 * j + 2, g, t), image_word(blob, 4 * j + 3, g, t));
  }
}

__device__ __forceinline__ unsigned u4c(const uint4 &v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// The two FP32 values of a BF16 pair.
__device__ __forceinline__ float2 bf16x2_float2(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// d += a b (m16n8k16, BF16 operands, FP32 accumulate)
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                               unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d = a b (m16n8k8, BF16 operands, FP32 result): the first product of an
// accumulator chain.  a0, a1: rows g and g + 8, columns 2t, 2t + 1; b: rows
// 2t, 2t + 1 of column g.
__device__ __forceinline__ void mma_bf16_1688_first(float (&d)[4], unsigned a0, unsigned a1,
                                                    unsigned b) {
  const float z = 0.f;
  asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%7,%7,%7,%7};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(b), "f"(z));
}

// round-to-nearest-even pair of floats to packed bf16 (lo in the low half)
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned *>(&v);
}

// tanh of a pair of pre-activations: rounded to a bf16 pair, then one
// hardware approximation for both halves (half the special-function issue
// of two FP32 tanh); the result is the next layer's packed BF16 operand.
__device__ __forceinline__ unsigned tanh_pair_bf16(float lo, float hi) {
  unsigned y;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(pack_bf16(lo, hi)));
  return y;
}

constexpr unsigned kOneLo = 0x3f80u;  // BF16 pair (1, 0)

// tanh of four accumulator tiles (n-tiles 4q .. 4q + 3 of a layer, this
// lane's values) as the next layer's A fragments of k-steps 2q (lo) and
// 2q + 1 (hi).
__device__ __forceinline__ void tanh_fragments(const float (&acc)[4][4], unsigned (&lo)[4],
                                               unsigned (&hi)[4]) {
  lo[0] = tanh_pair_bf16(acc[0][0], acc[0][1]);
  lo[1] = tanh_pair_bf16(acc[0][2], acc[0][3]);
  lo[2] = tanh_pair_bf16(acc[1][0], acc[1][1]);
  lo[3] = tanh_pair_bf16(acc[1][2], acc[1][3]);
  hi[0] = tanh_pair_bf16(acc[2][0], acc[2][1]);
  hi[1] = tanh_pair_bf16(acc[2][2], acc[2][3]);
  hi[2] = tanh_pair_bf16(acc[3][0], acc[3][1]);
  hi[3] = tanh_pair_bf16(acc[3][2], acc[3][3]);
}

// Forward pass of one m-tile (16 agents).  im: this lane's first image
// vector (vector j at im[32 j]).  a0: this lane's A fragment of observation
// columns 0-15 (rows g and g + 8); a8lo, a8hi: its m16n8k8 fragment of
// columns 16-23 for rows g and g + 8, where column 16, 17 is the row's
// (speed, heading) pair (t = 0), column 18 the constant 1 (t = 1: the word
// kOneLo) and the rest zero.  Returns, for this lane, the greedy action and
// the 4 logit columns it holds for rows g and g + 8.
__device__ __forceinline__ void policy_mtile(const uint4 *__restrict__ im, const unsigned (&a0)[4],
                                             unsigned a8lo, unsigned a8hi, int &act_lo,
                                             int &act_hi, float (&lg)[2][4]) {
  const int lane = threadIdx.x & 31, t = lane & 3;
  const unsigned one = t == 0 ? kOneLo : 0u;  // column 0 of a bias step: the constant 1
  // layer 1: [16 x 19] x [W1 | b1]^T, tanh -> [16 x 64], kept as layer 2's A
  // fragments (h1[k]: columns 16k .. 16k + 15); by halves of 32 columns, so
  // that the accumulators take 16 registers
  unsigned h1[4][4];
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const uint4 w0 = __ldg(im + 32 * (2 * hf)), w1 = __ldg(im + 32 * (2 * hf + 1));
    const uint4 w8 = __ldg(im + 32 * (kImgL1K8 / 4 + hf));
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // n-tile 4 hf + j
      const uint4 &w = j < 2 ? w0 : w1;
      mma_bf16_1688_first(acc[j], a8lo, a8hi, u4c(w8, j));
      mma_bf16_16816(acc[j], a0, u4c(w, 2 * (j & 1)), u4c(w, 2 * (j & 1) + 1));
    }
    tanh_fragments(acc, h1[2 * hf], h1[2 * hf + 1]);
  }
  // layer 2: [16 x 64] x W2^T + b2, tanh, by halves of 32 columns; each half
  // goes straight into layer 3: [16 x 64] x W3^T + b3 -> [16 x 16], the 9
  // logits (columns 9-15 zero)
  float o[2][4];
  {
    const uint4 bb = __ldg(im + 32 * (kImgB3 / 4));
    mma_bf16_1688_first(o[0], one, one, bb.x);
    mma_bf16_1688_first(o[1], one, one, bb.y);
  }
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    float acc[4][4];
    const uint4 bv = __ldg(im + 32 * (kImgB2 / 4 + hf));
#pragma unroll
    for (int j = 0; j < 4; ++j) mma_bf16_1688_first(acc[j], one, one, u4c(bv, j));
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint4 w0 = __ldg(im + 32 * (kImgL2 / 4 + 4 * kk + 2 * hf));
      const uint4 w1 = __ldg(im + 32 * (kImgL2 / 4 + 4 * kk + 2 * hf + 1));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 &w = j < 2 ? w0 : w1;
        mma_bf16_16816(acc[j], h1[kk], u4c(w, 2 * (j & 1)), u4c(w, 2 * (j & 1) + 1));
      }
    }
    unsigned h2[2][4];
    tanh_fragments(acc, h2[0], h2[1]);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint4 w = __ldg(im + 32 * (kImgL3 / 4 + 2 * hf + q));
      mma_bf16_16816(o[0], h2[q], w.x, w.y);
      mma_bf16_16816(o[1], h2[q], w.z, w.w);
    }
  }
  // greedy action per row (largest logit, lowest column on ties; NaN never
  // chosen): this thread holds columns 2t, 2t + 1 (logits), 8 + 2t (a logit
  // for t = 0 only) and 9 + 2t (never one).  The row's maximum over the
  // quad first, then the lowest column that holds it.
  const float ninf = -__int_as_float(0x7f800000);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float x0 = o[0][2 * h], x1 = o[0][2 * h + 1], x8 = t == 0 ? o[1][2 * h] : ninf;
    lg[h][0] = x0;
    lg[h][1] = x1;
    lg[h][2] = o[1][2 * h];
    lg[h][3] = o[1][2 * h + 1];
    float m = fmaxf(fmaxf(x0, x1), x8);
    m = fmaxf(m, __shfl_xor_sync(kFull, m, 1));
    m = fmaxf(m, __shfl_xor_sync(kFull, m, 2));
    int bi = x0 == m ? 2 * t : (x1 == m ? 2 * t + 1 : (t == 0 && x8 == m ? 8 : 16));
    bi = min(bi, __shfl_xor_sync(kFull, bi, 1));
    bi = min(bi, __shfl_xor_sync(kFull, bi, 2));
    if (h == 0) act_lo = bi;
    else act_hi = bi;
  }
}

// The network on a warp's own A agents, in the neighbour scan's epilogue:
// their observation rows go from the warp's sector arrays straight into
// BF16 A fragments (16 rows an m-tile; rows past the warp's nb agents are
// zero but for the bias column), and the greedy actions and logits go to
// the agents' rows.  A row is the observation in BF16: (distance, count)
// per sector, the range for an empty sector, then (speed, heading).  Every
// lane of the warp takes part (mma.sync); i and ts are this lane's agent
// and own state as the scan loaded them (lane r < A holds row r).
template <int A>
__device__ __forceinline__ void policy_warp_rows(const Inst &I, const DirectArea &W,
                                                 const Bufs &B, int i, float2 ts, int nb) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int v = I.v;  // 8 (the host runs the network on 8-sector flocks only)
  const uint4 *im = B.wimg + lane;
#pragma unroll 1
  for (int mt = 0; mt < (A + 15) / 16; ++mt) {
    unsigned f[2][3];
    int ir[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int r = 16 * mt + g + 8 * m;  // < 32: a lane's index
      ir[m] = __shfl_sync(kFull, i, r);
      const float sp = __shfl_sync(kFull, ts.y, r), hd = __shfl_sync(kFull, ts.x, r);
      const bool ok = r < nb;
      unsigned w0 = 0u, w1 = 0u;
      if (ok) {
        const int c0 = W.cn[r * v + t], c1 = W.cn[r * v + 4 + t];
        w0 = pack_bf16(c0 ? __uint_as_float(W.md[r * v + t]) : I.RV, (float)c0);
        w1 = pack_bf16(c1 ? __uint_as_float(W.md[r * v + 4 + t]) : I.RV, (float)c1);
      }
      f[m][0] = w0;
      f[m][1] = w1;
      f[m][2] = t == 0 ? (ok ? pack_bf16(sp, hd) : 0u) : (t == 1 ? kOneLo : 0u);
    }
    const unsigned a0[4] = {f[0][0], f[1][0], f[0][1], f[1][1]};
    int alo = 0, ahi = 0;
    float lg[2][4];
    policy_mtile(im, a0, f[0][2], f[1][2], alo, ahi, lg);
    const int rlo = 16 * mt + g, rhi = rlo + 8;
    if (t == 0) {
      if (rlo < nb) B.pact[I.agent_base + ir[0]] = alo;
      if (rhi < nb) B.pact[I.agent_base + ir[1]] = ahi;
    }
    if (B.plogits) {
      const int c4[4] = {2 * t, 2 * t + 1, 8 + 2 * t, 9 + 2 * t};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (c4[j] < 9) {
          if (rlo < nb) B.plogits[(long long)(I.agent_base + ir[0]) * 9 + c4[j]] = lg[0][j];
          if (rhi < nb) B.plogits[(long long)(I.agent_base + ir[1]) * 9 + c4[j]] = lg[1][j];
        }
      }
    }
  }
}

// A warp takes the 32 / LPA consecutive sorted agents [gp0, gp1); LPA lanes
// share each agent's candidates (LPA = 1, 2, 4 or 32).  LPA = 32 gives a whole warp to one agent: the form for agents with
// hundreds of candidates (a wide view), whose few agents would otherwise
// leave most of the GPU idle.
// TAG: the tag environment (needs V == 0 and no policy): two colour
// channels of sectors, type-dependent rewards (see drain_direct), and the
// observation row is the 2v channel distances.
// COMPACT: the runs of wrapping chunks are walked by a loop that is not
// unrolled, so that form of the candidate scan appears once in the code (the
// batched kernels, whose mix of small instances wraps often, run faster with
// the smaller instruction footprint; a single large instance rarely wraps and
// runs faster fully unrolled).
// POLICY: the policy step's network runs in the epilogue on the warp's own
// agents (policy_warp_rows) and writes their actions and logits.
// AORDER: [gp0, gp1) are agent indices (flattened), not sorted positions:
// the warp's agents are consecutive in agent order, so that its observation
// rows form one contiguous block, which the warp assembles in its queue area
// and writes with 16-byte stores (the form for outputs in mapped host
// memory, where scattered rows cross the link slowly).  An agent's own
// position is read from its state row, and its sorted position (the
// candidate that is itself) from its cell and rank.  Flock, 8 sectors,
// layout 0, at most 32 rows of 72 bytes (the queue holds 2,560).
template <int H, int V, bool PIECES = true, int LPA = 1, bool TAG = false, bool COMPACT = false,
          bool POLICY = false, bool AORDER = false>
__device__ __forceinline__ void phaseD_direct(const Inst &I, int gp0, int gp1, const Bufs &B,
                              const DirectArea &W, unsigned &err) {
  static_assert(LPA == 1 || LPA == 2 || LPA == 4 || LPA == 32, "lanes per agent");
  static_assert(!TAG || V == 0, "tag uses the generic sector count");
  static_assert(!POLICY || !TAG, "the network reads flock observations");
  static_assert(!AORDER || (V == 8 && !TAG && !POLICY && LPA != 32 && (32 / LPA) * 72 <= kQueueWide * 16),
                "agent-order rows: 8-sector flock rows staged in the queue area");
  constexpr int A = 32 / LPA;
  const int lane = threadIdx.x & 31;
  const int slot = lane & (A - 1);
  const int nc = I.nc, v = V == 8 ? 8 : I.v;
  const int vs = TAG ? 2 * v : v;  // accumulator row length
  Edges<V> E8;
  E8.load(I);
  const int gp = gp0 + slot;
  bool have = gp < gp1;
  const int nb = gp1 - gp0;
  float xi = 0.f, yi = 0.f;
  float2 ts = make_float2(0.f, 0.f);
  int i = 0, cx = 0, cy = 0, sp = -1;
  if (AORDER) {
    if (have && dbg_ok(gp >= 0 && gp < B.n_total)) {
      i = gp - I.agent_base;
      if (!dbg_ok(i >= 0 && i < I.n)) i = 0;
      const float4 s4 = I.state[i];  // the new position, heading and speed
      xi = s4.x;
      yi = s4.y;
      ts = make_float2(s4.z, s4.w);
      cx = cell_of(xi, I);
      cy = cell_of(yi, I);
      const int2 cr = B.cellrank[gp];
      if (dbg_ok(cr.x >= 0 && cr.x < B.c_total)) sp = B.cell_start[cr.x] + cr.y;
    }
  } else if (have && dbg_ok(gp >= 0 && gp < B.n_total)) {
    sp = gp;
    const float2 p = B.sxy[gp];
    xi = p.x;
    yi = p.y;
    i = B.sidx[gp] - I.agent_base;
    if (!dbg_ok(i >= 0 && i < I.n)) i = 0;
    const float4 s4 = I.state[i];  // own heading and speed (only the owner needs them)
    ts = make_float2(s4.z, s4.w);
    cx = cell_of(xi, I);
    cy = cell_of(yi, I);
  }
  // a slab's ghosts (agents past its first n_own) are candidates only
  if (i >= I.n_own) have = false;
  const int ti = TAG && have ? (int)(B.stype[gp] != 0) : 0;  // own type (tag)
  // the cell starts of the stencil rows are read before anything waits on
  // the agent's own state row, so that the two reads are in flight together
  // stencil columns [cx - H, cx + H] split into runs that do not wrap
  const int vlo = cx - H, vhi = cx + H + 1;
  const int ma = max(vlo, 0), mb = min(vhi, nc);  // interior run
  const bool lw = vlo < 0, rw = vhi > nc;         // left / right boundary runs
  const bool wrap_any = __any_sync(kFull, have && (lw || rw || cy - H < 0 || cy + H >= nc));
  const int *cst = B.cell_start;
  int ra[2 * H + 1], rn[2 * H + 1];
#pragma unroll
  for (int r = 0; r < 2 * H + 1; ++r) {
    const int rowg = I.cell_base + lrow(I, wrapi(cy - H + r, nc)) * nc;
    ra[r] = have ? cst[rowg + ma] : 0;
    rn[r] = have ? cst[rowg + mb] - ra[r] : 0;
    dbg_run(ra[r], rn[r], B.n_total);
  }
  float c = 1.f, sn = 0.f;
  det_sincos(ts.x, c, sn);
  const float ux = fadd(fmul(c, I.CF), fmul(sn, I.SF));
  const float uy = fsub(fmul(sn, I.CF), fmul(c, I.SF));
  W.acc[lane] = 0ull;
  if (PIECES) {
    W.accp[lane] = 0u;
    W.accp[32 + lane] = 0u;
    W.accp[64 + lane] = 0u;
  }
  // per-sector minima and counts of the warp's A agents (A rows of v)
  if (V == 8) {
    if (lane < A) {
      uint4 *m4 = reinterpret_cast<uint4 *>(W.md + lane * 8);
      int4 *c4 = reinterpret_cast<int4 *>(W.cn + lane * 8);
      const unsigned inf = 0x7f800000u;
      m4[0] = make_uint4(inf, inf, inf, inf);
      m4[1] = make_uint4(inf, inf, inf, inf);
      c4[0] = make_int4(0, 0, 0, 0);
      c4[1] = make_int4(0, 0, 0, 0);
    }
  } else {
    for (int t = lane; t < A * vs; t += 32) {
      W.md[t] = 0x7f800000u;
      W.cn[t] = 0;
    }
  }
  int nin = 0, ncoll = 0;
  unsigned long long racc = 0;  // one agent per warp: this lane's share of its reward sum
  __syncwarp();
  int qn = 0;
  // the agent's own sorted position: its candidate scan skips it
  const int self = have ? sp : -1;
  if (!wrap_any) {
#pragma unroll
    for (int r = 0; r < 2 * H + 1; ++r)
      direct_run<false, V, PIECES, LPA, TAG>(I, W, B.sxy, ra[r], rn[r], self, 0.f, 0.f, xi, yi,
                                             ux, uy, qn, nin, ncoll, E8, B.stype, ti, racc);
  } else if (COMPACT) {
    // per stencil row three runs: the interior, the cells across the left
    // boundary (virtual columns [vlo, 0) -> [vlo + nc, nc)) and those across
    // the right one (virtual columns [nc, vhi) -> [0, vhi - nc))
#pragma unroll 1
    for (int t = 0; t < 3 * (2 * H + 1); ++t) {
      const int r = t / 3, kind = t - 3 * r;
      const int vr = cy - H + r;
      const float sy = vr < 0 ? -I.L : (vr >= nc ? I.L : 0.0f);
      const int rowg = I.cell_base + lrow(I, wrapi(vr, nc)) * nc;
      int a = 0, n = 0;
      float sx = 0.f;
      if (kind == 0) {
        a = pick<2 * H + 1>(ra, r);
        n = pick<2 * H + 1>(rn, r);
      } else if (kind == 1) {
        sx = -I.L;
        if (have && lw) {
          a = cst[rowg + vlo + nc];
          n = cst[rowg + nc] - a;
        }
      } else {
        sx = I.L;
        if (have && rw) {
          a = cst[rowg];
          n = cst[rowg + vhi - nc] - a;
        }
      }
      dbg_run(a, n, B.n_total);
      direct_run<true, V, PIECES, LPA, TAG>(I, W, B.sxy, a, n, self, sx, sy, xi, yi, ux, uy, qn,
                                            nin, ncoll, E8, B.stype, ti, racc);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 2 * H + 1; ++r) {
      const int vr = cy - H + r;
      const float sy = vr < 0 ? -I.L : (vr >= nc ? I.L : 0.0f);
      const int rowg = I.cell_base + lrow(I, wrapi(vr, nc)) * nc;
      direct_run<true, V, PIECES, LPA, TAG>(I, W, B.sxy, ra[r], rn[r], self, 0.f, sy, xi, yi,
                                            ux, uy, qn, nin, ncoll, E8, B.stype, ti, racc);
      // cells across the left boundary: virtual columns [vlo, 0) -> [vlo + nc, nc)
      int a = 0, n = 0;
      if (have && lw) {
        a = cst[rowg + vlo + nc];
        n = cst[rowg + nc] - a;
      }
      dbg_run(a, n, B.n_total);
      direct_run<true, V, PIECES, LPA, TAG>(I, W, B.sxy, a, n, self, -I.L, sy, xi, yi, ux, uy,
                                            qn, nin, ncoll, E8, B.stype, ti, racc);
      // cells across the right boundary: virtual columns [nc, vhi) -> [0, vhi - nc)
      a = 0;
      n = 0;
      if (have && rw) {
        a = cst[rowg];
        n = cst[rowg + vhi - nc] - a;
      }
      dbg_run(a, n, B.n_total);
      direct_run<true, V, PIECES, LPA, TAG>(I, W, B.sxy, a, n, self, I.L, sy, xi, yi, ux, uy,
                                            qn, nin, ncoll, E8, B.stype, ti, racc);
    }
  }
  __syncwarp();
  drain_direct<V, PIECES, TAG, A == 1>(I, W, qn, ux, uy, E8, ti, racc, true);
  if (A == 1) {
    // one agent per warp: the lanes' register sums make its reward sum
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) racc += __shfl_xor_sync(kFull, racc, m);
    if (lane == 0) W.acc[0] = racc;
    __syncwarp();
  }
  // the lanes of an agent add up their counts
#pragma unroll
  for (int m = A; m < 32; m <<= 1) {
    nin += __shfl_xor_sync(kFull, nin, m);
    ncoll += __shfl_xor_sync(kFull, ncoll, m);
  }
  // reward and collisions
  if (have && lane < A) {
    // a chaser's touches earn through its terms; everyone else's cost P each
    const long long pen = TAG && ti ? 0ll : (long long)ncoll * I.PK;
    const long long total = (long long)W.acc[lane] - pen;
    B.reward[I.agent_base + i] = fmul(__ll2float_rn(total), I.inv_scaleK);
    B.coll[I.agent_base + i] = ncoll;
    if ((long long)nin > I.NMAX) err |= FLOCK_ERR_OVERFLOW;
  }
  // observation rows (when asked for).  The last entry of a flock row,
  // (speed, heading) (layout 1: the speed), comes from the agent's own lane;
  // the v sector entries of several rows at a time from all lanes, each
  // row's contiguous.  Tag rows are the 2v distances.
  float *obs = B.obs ? B.obs + I.obs_base : nullptr;
  if (AORDER && obs) {
    // the warp's nb rows are contiguous from agent i0: assembled in the queue
    // area (free after the final drain), then stored 16 bytes at a time
    __syncwarp();  // the drain's last reads of the queue and writes of the sectors
    const int i0 = gp0 - I.agent_base;
    float *stage = reinterpret_cast<float *>(W.queue);
    for (int t = lane; t < nb * 16; t += 32) {
      const int r = t >> 4, e = (t & 15) >> 1;
      const int ck = W.cn[r * 8 + e];
      stage[r * 18 + (t & 15)] =
          (t & 1) ? (float)ck : (ck ? __uint_as_float(W.md[r * 8 + e]) : I.RV);
    }
    if (have && lane < A) {
      stage[slot * 18 + 16] = ts.y;
      stage[slot * 18 + 17] = ts.x;
    }
    __syncwarp();
    float *dst = obs + (long long)i0 * 18;
    const int words = nb * 18;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      const float4 *s4 = reinterpret_cast<const float4 *>(stage);
      float4 *d4 = reinterpret_cast<float4 *>(dst);
      for (int t = lane; t < words / 4; t += 32) d4[t] = s4[t];
      done = words & ~3;
    }
    for (int t = done + lane; t < words; t += 32) dst[t] = stage[t];
  } else if (obs) {
    const int P = TAG ? 2 * v : v;  // entries per row from the sector arrays
    const int rpi = P <= 32 ? 32 / P : 1;
    const int my_r = P <= 32 ? lane / P : 0, my_e = P <= 32 ? lane % P : lane;
    // the V = 8 kernels serve layout 0 only (the host picks V = 0 for layout 1)
    const bool lay0 = V == 8 || I.obs_layout == 0;
    if (!TAG && have && lane < A) {
      const float2 val = make_float2(ts.y, ts.x);
      float *row = obs + (long long)i * I.obs_dim;
      if (lay0) *reinterpret_cast<float2 *>(row + 2 * v) = val;
      else row[v] = val.x;
    }
    for (int rb = 0; rb < nb; rb += rpi) {
      const int r = min(rb + my_r, 31);
      const int ir = __shfl_sync(kFull, i, r);
      const bool hr = __shfl_sync(kFull, have, r);  // a ghost's row gets no output
      if (rb + my_r < nb && my_r < rpi && hr) {
        for (int e = my_e; e < P; e += 32) {
          const int ck = W.cn[r * vs + e];
          const float d = ck ? __uint_as_float(W.md[r * vs + e]) : I.RV;
          float *row = obs + (long long)ir * I.obs_dim;
          if (TAG || !lay0) row[e] = d;  // tag: the channel distances; layout 1: the distance only
          else *reinterpret_cast<float2 *>(row + 2 * e) = make_float2(d, (float)ck);
        }
      }
    }
  }
  if (POLICY) {
    __syncwarp();
    policy_warp_rows<A>(I, W, B, i, ts, nb);
  }
  __syncwarp();
}

}  // namespace flock
