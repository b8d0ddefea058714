/*
 * flock.h -- C ABI of the GB300 flock environment step.
 *
 * The library advances the flock multi-agent environment of arXiv 2207.03945
 * ("High Performance Simulation for Scalable Multi-Agent Reinforcement
 * Learning", Section 4.1) on one GPU.  One step applies every agent's action
 * (accelerate within [s_min, s_max], rotate, move on the periodic square),
 * then, with the new positions, gives every agent its sector-vision
 * observation (Section 4 and Fig. 3), its collision count (Fig. 4) and its
 * reward r_i = sum_j f(d_ij) over d_ij < d_v (Eq. 1).
 *
 * Memory: the caller owns every device buffer, including the workspace the
 * library carves its scratch from (query its size first).  The library never
 * allocates device memory; it owns only small host structs and, for graph
 * replay, a CUDA stream and graph of its own.  All pointers named *_dev are
 * device pointers; *_host are host pointers (pinned memory gives true
 * asynchronous copies).  Buffers must not overlap.
 *
 * Streams: every call enqueues work on the stream given at create time (a
 * cudaStream_t passed as void*; NULL is the legacy default stream) and
 * returns without waiting, except where stated.  One handle per stream; a
 * handle is not safe for concurrent use from several host threads.
 *
 * Errors: calls return FLOCK_OK (0) or a negative FLOCK_E* code.  Conditions
 * found on the device (bad action values, bad state values, a timed-out
 * grid barrier, reward accumulator overflow) are latched as FLOCK_ERR_* bits
 * and read, then cleared, by env_get_error / env_batch_get_error.  Device
 * code never traps.
 *
 * Layouts (row-major, no padding):
 *   state       n x 4 float : (x, y, theta, s), x, y in [0, side), theta in
 *                             [0, (float)2pi), s in [speed_min, speed_max]
 *   actions     n int32     : a in [0, 9): turn = a / 3 picks {-turn_step, 0,
 *                             +turn_step}, speed change = a % 3 picks
 *                             {-speed_step, 0, +speed_step}; a = 4 is "keep"
 *   continuous actions  n x 2 float : (acceleration, rotation), the paper's
 *                             two-dimensional action space (Section 4.1),
 *                             clamped to [-speed_step, speed_step] x
 *                             [-turn_step, turn_step] (env_step_continuous)
 *   obs, layout 0  n x (2v+2) float : for sector k = 0..v-1, (distance to the
 *                             nearest agent in sector k, or view_radius when
 *                             empty; number of agents in sector k), then
 *                             (s, theta).  Sectors split the field of view
 *                             (centred on the heading) into v equal angles,
 *                             numbered counter-clockwise from its right edge.
 *   obs, layout 1  n x (v+1) float : the distances of the v sectors, then s
 *                             (the paper's observation: 129 values for v = 128)
 *   obs, tag       n x 2v float : the v sector distances of the nearest runner,
 *                             then of the nearest chaser (128 values for v = 64)
 *   reward      n float, coll n int32 (collisions: pairs closer than
 *                             2 * agent_radius)
 * Row i of every output belongs to agent i of the state (never reordered).
 */
#ifndef FLOCK_H
#define FLOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FLOCK_OK 0
#define FLOCK_EINVAL (-1)   /* bad argument, parameter or size */
#define FLOCK_ENOSPACE (-2) /* workspace too small or not 256-byte aligned */
#define FLOCK_ECUDA (-3)    /* a CUDA runtime call failed (see flock_last_cuda_error) */

/* ---- device-side condition bits (env_get_error) ---- */
#define FLOCK_ERR_ACTION 1u   /* an action outside [0, 9) was read (it acted as 4), or a
                                 continuous action component was not finite (it acted as 0) */
#define FLOCK_ERR_STATE 2u    /* an input state value was non-finite or out of range */
#define FLOCK_ERR_TIMEOUT 4u  /* a grid barrier of the batched kernel gave up waiting */
#define FLOCK_ERR_OVERFLOW 8u /* an agent had more in-range neighbours than the exact
                                 reward sum holds (see flock_derived.nmax) */
#define FLOCK_ERR_BOUNDS 16u  /* debug build (FLOCK_DEBUG, libflock_debug.so) only: an
                                 index check failed; the access was skipped */

#define FLOCK_MAX_SEGMENTS 128

/* Model parameters (Section 4.1; readings of the paper in parentheses). */
typedef struct flock_params {
  float side;              /* L: the periodic square [0, L)^2 */
  float view_radius;       /* d_v: neighbours at distance < d_v are seen (Eq. 1) */
  float fov;               /* field of view, radians, in (0, (float)2pi];
                              (float)2pi means the full circle */
  float agent_radius;      /* d_r: a pair collides when closer than 2 d_r (Fig. 4) */
  float collision_penalty; /* P: reward contribution of a colliding pair is -P */
  float speed_min, speed_max; /* speed clamp (the printed min/max are swapped) */
  float speed_step;        /* speed change of an accelerate/decelerate action */
  float turn_step;         /* heading change of a rotate action, radians */
  int num_segments;        /* v: sectors of the field of view, 1..128 */
  int obs_layout;          /* 0: (distance, count) per sector, speed, heading (2v + 2
                              values); 1: distance per sector, speed (v + 1 values) */
  int kind;                /* 0: flock; 1: tag (Section 4.2), see env_set_types */
} flock_params;

/* Launch shape of the neighbour scan.  Every field may be 0 (library
 * choice).  Results are identical for every valid setting. */
typedef struct flock_tuning {
  int stencil; /* 1: cells of width >= d_v, 3 x 3 stencil; 2: width >= d_v/2, 5 x 5 */
  int tile_w;  /* mode 1: cells per tile along x, 1..64 */
  int tile_h;  /* mode 1: cells per tile along y, 1..8 */
  int block;   /* threads per block, multiple of 32 in 64..512 (0: 128;
                  batch, modes 3 and 4: the neighbour launch's block,
                  64..256) */
  int mode;    /* neighbour scan: 1 = tiles of cells staged in shared memory,
                  2 = each warp takes 32 / lanes consecutive cell-sorted agents
                  and reads their stencil cells through the L1 cache.
                  Batch: 2 = every phase in one persistent launch; 3 = binning
                  in the persistent launch, the neighbour scan (direct form)
                  in a second launch; 4 (0: the default) = binning by three
                  kernels (apply and count, scan, scatter) over all
                  instances, then the neighbour launch.  Results are
                  identical. */
  int lanes;   /* mode 2: lanes per agent, 1, 2, 4 or 32 (0: 32 when an agent
                  has 256 or more candidates in its stencil cells on average
                  or there are at most 4,096 agents, else 4 up to 32,768
                  agents, 2 up to 524,288, else 1); the
                  lanes of an agent share its candidates.  Mode 1 uses 1.
                  Batch, modes 3 and 4: 1, 2 or 4 for the neighbour launch (0:
                  by the batch's maximum agent count, as above); mode 2: 1. */
} flock_tuning;

/* Constants the library derives from flock_params (host, double precision
 * where a transcendental is involved, rounded once to float). */
typedef struct flock_derived {
  float side, half_side, view_radius, rv2, rc2, inv_span, two_pi, cos_half_fov,
      sin_half_fov, speed_min, speed_max;
  float turn[3], accel[3];
  float edge[FLOCK_MAX_SEGMENTS + 1]; /* edge[m], m = 1..v: pseudo-angle of sector edge m */
  int v, full_circle, k_exp;          /* reward sum resolution 2^-k_exp */
  int64_t penalty_fixed;              /* P * 2^k_exp */
  int64_t nmax;                       /* in-range neighbours the exact sum holds */
  int cells_per_side, stencil;        /* cell list geometry */
  float inv_cell_width;
} flock_derived;

typedef struct flock_env flock_env;
typedef struct flock_batch flock_batch;

/* Fills *out with this library's defaults for a square of side `side`:
 * d_v = 5, d_r = 0.5, P = 1, s in [0, 1], speed_step 0.25, turn_step pi/8,
 * v = 8, fov = 250 degrees.  Returns FLOCK_EINVAL for a NULL out. */
int flock_default_params(float side, flock_params *out);

/* Values per observation row for valid params: 2v + 2 (obs_layout 0),
 * v + 1 (obs_layout 1), 2v (tag); else FLOCK_EINVAL. */
int flock_obs_dim(const flock_params *params);

/* Device workspace (bytes) that env_create needs for n_agents agents. */
int flock_workspace_bytes(const flock_params *params, const flock_tuning *tuning_or_null,
                          int n_agents, size_t *bytes_out);

/* The derived constants and cell geometry env_create would use (no GPU
 * needed).  tuning_or_null selects the stencil. */
int flock_derive(const flock_params *params, const flock_tuning *tuning_or_null,
                 flock_derived *out);

/* Creates an environment of n_agents (>= 0) agents.  workspace_dev: caller
 * buffer of at least flock_workspace_bytes, 256-byte aligned, owned by the
 * caller until env_destroy; the agent state lives in it.  stream: the
 * cudaStream_t all calls enqueue on.  No kernel runs; the workspace is
 * cleared with cudaMemsetAsync. */
int env_create(const flock_params *params, const flock_tuning *tuning_or_null, int n_agents,
               void *workspace_dev, size_t workspace_bytes, void *stream, flock_env **out);

/* Loads state0_dev (n x 4) as the current state and writes the initial
 * observation, rewards and collisions of that state (no action applied). */
int env_reset(flock_env *env, const float *state0_dev, float *obs_dev, float *reward_dev,
              int32_t *coll_dev);

/* One step (the hot path): applies actions_dev, then observes.  Enqueues a
 * CUDA graph of the binning and neighbour-scan kernels (captured on the
 * first call; when a buffer pointer changes, the graph is updated in place
 * and launches already enqueued keep their pointers). */
int env_step(flock_env *env, const int32_t *actions_dev, float *obs_dev, float *reward_dev,
             int32_t *coll_dev);

/* env_step with the paper's continuous actions (Section 4.1): actions2_dev
 * holds n x 2 floats (acceleration, rotation; for tag (speed, rotation)),
 * 8-byte aligned.  Each is
 * clamped to [-speed_step, speed_step] and [-turn_step, turn_step]; a
 * component that is not finite acts as 0 and latches FLOCK_ERR_ACTION.  The
 * speed clamp, heading wrap, move and observation are those of env_step.
 * Shares env_step's cached graph (updated in place when the kind of action
 * or a pointer changes). */
int env_step_continuous(flock_env *env, const float *actions2_dev, float *obs_dev,
                        float *reward_dev, int32_t *coll_dev);

/* A rollout: T consecutive steps (env_step or env_step_continuous) as one
 * launch of a CUDA graph of 4T kernels -- the t = 128 environment updates of
 * a training step (Section 5).  Exactly one of actions_dev (T x n int32) and
 * actions2_dev (T x n x 2 float, 8-byte aligned) is given; step t reads row
 * t and writes rows t of obs_dev (T x n x obs_dim), reward_dev (T x n) and
 * coll_dev (T x n), so the buffers hold the whole trajectory of every agent.
 * The graph is kept for the next call with the same T and pointers (and
 * updated in place when only the pointers change).  T = 0 does nothing. */
int env_rollout(flock_env *env, int T, const int32_t *actions_dev, const float *actions2_dev,
                float *obs_dev, float *reward_dev, int32_t *coll_dev);

/* Advantages and value targets over a rollout (the trajectory processing of
 * PPO, Section 4.3), by generalised advantage estimation in FP32:
 *   delta_t = (r_t + gamma v_{t+1}) - v_t,  A_t = delta_t + (gamma lambda) A_{t+1},
 *   A_T = 0,  R_t = A_t + v_t,
 * evaluated in that order from t = T-1 down, one rounding per operation
 * (gamma lambda rounded once).  reward_dev: T x n, value_dev: (T+1) x n (row
 * T bootstraps the last step; the flock never terminates), adv_dev and
 * ret_dev: T x n, all step-major, device memory, not overlapping.  gamma and
 * lambda in [0, 1].  Enqueues one kernel on `stream` (a cudaStream_t). */
int flock_gae(int T, int n, const float *reward_dev, const float *value_dev, float gamma,
              float lambda, float *adv_dev, float *ret_dev, void *stream);

/* Initial states drawn on the device from a seed (an episode's start where
 * the state lives, e.g. a serving session admitted by seed; the paper leaves
 * initial conditions open, uniform is this library's reading): row i of the
 * n x 4 state_dev is (x, y, theta, s) with
 *   x = min(u(4i) * side, side-),  y = min(u(4i+1) * side, side-),
 *   theta = min(u(4i+2) * (float)2pi, (float)2pi-),  s = speed,
 * where v- is the float below v, each product rounded once, and u(k) is
 * output k (from 0) of SplitMix64 seeded with `seed` (Steele, Lea and Flood,
 * OOPSLA 2014: z = seed + (k+1) * 0x9E3779B97F4A7C15, then the finaliser
 * z ^= z >> 30, z *= 0xBF58476D1CE4E5B9, z ^= z >> 27, z *= 0x94D049BB133111EB,
 * z ^= z >> 31) reduced to its top 24 bits times 2^-24.  state_dev: device
 * memory, 16-byte aligned; side > 0 and speed finite, else FLOCK_EINVAL.
 * Enqueues one kernel on `stream` (a cudaStream_t); n == 0 does nothing. */
int flock_seed_states(float *state_dev, int n, float side, float speed, uint64_t seed,
                      void *stream);

/* One step whose next actions come from the policy: applies
 * actions_inout_dev, observes, and feeds each agent's observation through the
 * shared policy network (the learners' shared MLP of Section 4.3, here
 * 18 -> 64 -> 64 -> 9 with tanh, as the 18-value observation needs; needs
 * num_segments == 8 and obs_layout 0), then overwrites actions_inout_dev with
 * the greedy actions (largest logit, lowest index on ties) for the next step.
 * The network runs in the neighbour scan's epilogue: each warp feeds its own
 * agents' observations to it straight from its registers and shared memory
 * (as BF16), so the step keeps its four kernels.  The binning launch copies
 * the weights into a lane-interleaved operand image in the workspace (14,848
 * bytes, rebuilt every call, so weights may change between calls).
 * weights_bf16_dev: 5,961 bfloat16 values, W1[64][18] b1[64] W2[64][64]
 * b2[64] W3[9][64] b3[9], each W row-major [out][in].  Operands are BF16 on
 * the tensor cores, accumulation FP32, tanh the hardware approximation.
 * logits_dev (n x 9 floats) and obs_dev (n x 18) may be NULL (with NULL obs
 * no FP32 observation is written). */
int env_step_policy(flock_env *env, const uint16_t *weights_bf16_dev, int32_t *actions_inout_dev,
                    float *reward_dev, int32_t *coll_dev, float *logits_dev, float *obs_dev);

/* env_step from and to host memory, waiting for the stream: returns after
 * the outputs are in the host buffers.  Page-locked, mapped actions
 * (cudaHostAlloc / pinned tensors; the GPU reaches them coherently over
 * NVLink-C2C on Grace-Blackwell) are read by the step's first kernel in
 * place, others are copied in.  Page-locked, mapped output buffers of a
 * flock with 8 sectors, observation layout 0, the 3 x 3 stencil and 1-4
 * lanes per agent are written by the neighbour scan itself, run in agent
 * order so that each warp stores its block of rows whole; other page-locked
 * outputs are written to the workspace and copied out by one copy kernel;
 * pageable ones by one copy per buffer.  The step (and its copy) is one CUDA
 * graph, kept while the buffers are the same. */
int env_step_host(flock_env *env, const int32_t *actions_host, float *obs_host,
                  float *reward_host, int32_t *coll_host);

/* Tag (params.kind == 1, Section 4.2): agents of type 0 are runners, of
 * type 1 (any non-zero byte) chasers.  types_dev: n bytes, copied into the
 * workspace (all runners after env_create).  A runner's reward is the flock
 * reward (Eq. 1) over runners, with -collision_penalty for every agent it
 * touches (closer than 2 agent_radius, either type); a chaser's reward is
 * +collision_penalty per runner it touches.  The view has two colour
 * channels (runners, chasers) of num_segments sectors.  With
 * env_step_continuous the action is (speed, rotation): the speed is set,
 * clamped to [speed_min, speed_max].  Tag uses the direct neighbour scan
 * (tuning mode 2) of a single environment; the batch, the policy step and
 * flock_step_static take flock instances only.  FLOCK_EINVAL for a flock
 * environment. */
int env_set_types(flock_env *env, const uint8_t *types_dev);

/* Copies the current state (n x 4) out of / into the workspace. */
int env_get_state(flock_env *env, float *state_dev);
int env_set_state(flock_env *env, const float *state_dev);

/* Waits for the stream, returns the latched FLOCK_ERR_* bits in *bits_out and
 * clears them. */
int env_get_error(flock_env *env, uint32_t *bits_out);

/* The library's derived constants and the tuning in use. */
int env_get_derived(const flock_env *env, flock_derived *out);
int env_get_tuning(const flock_env *env, flock_tuning *out);

/* Kernel timing.  With enable != 0 the step graph is re-captured with a CUDA
 * event around each of its four kernels (apply+bin, scan, scatter,
 * neighbour scan); env_get_phase_times waits for the stream and returns the
 * last step's kernel durations in milliseconds.  Off by default. */
int env_set_timing(flock_env *env, int enable);
int env_get_phase_times(flock_env *env, float ms_out[4]);

/* Frees the host handle and the library's graph and stream; frees nothing
 * the caller owns.  Waits for the stream first. */
void env_destroy(flock_env *env);

/* ---------------------------------------------------------------------------
 * Batched step: many independent flock instances advanced by ONE persistent
 * cooperative kernel per step (apply+bin, scan, scatter and neighbour scan as
 * phases separated by grid barriers).  Instances may differ in agent count and
 * in every parameter except num_segments and obs_layout; all share the
 * batch's tuning.  Actions are discrete (int32).
 *
 * Instance k of the active set owns rows [off_k, off_k + n_k) of every
 * flattened per-agent buffer (actions, reward, coll, and obs rows of the
 * layout's length), off_k = n_0 + ... + n_{k-1}.  Its state lives in caller memory
 * (state_dev[k], n_k x 4 floats) and is updated in place, so sessions stay
 * resident across steps and may join or leave between steps.
 * ------------------------------------------------------------------------- */

/* Cells one instance uses (cells_per_side^2) under the given tuning. */
int flock_instance_cells(const flock_params *params, const flock_tuning *tuning_or_null,
                         int *cells_out);

/* Workspace for a batch of at most max_instances instances holding at most
 * max_agents agents and max_cells cells in total. */
int flock_batch_workspace_bytes(int max_instances, int max_agents, int max_cells,
                                const flock_tuning *tuning_or_null, size_t *bytes_out);

/* Creates a batch (no instance active).  Same ownership and stream rules as
 * env_create.  Needs a device that supports cooperative launches. */
int env_batch_create(int max_instances, int max_agents, int max_cells,
                     const flock_tuning *tuning_or_null, void *workspace_dev,
                     size_t workspace_bytes, void *stream, flock_batch **out);

/* Sets the active instances (replacing the previous set), in order.
 * params/n_agents/state_dev/reset are arrays of n_inst entries; reset[k] != 0
 * (or reset == NULL for none) makes the next step observe instance k without
 * applying its actions (its initial observation).  The descriptors are
 * copied to the device in stream order; no kernel is re-captured.
 * Returns FLOCK_EINVAL if a parameter set is invalid, if num_segments or
 * obs_layout differs between instances, if an instance is a tag instance,
 * or if a total exceeds the batch's maxima. */
int env_batch_set(flock_batch *batch, int n_inst, const flock_params *params,
                  const int *n_agents, float *const *state_dev, const int *reset);

/* One step of every active instance (the batched hot path). */
int env_batch_step(flock_batch *batch, const int32_t *actions_dev, float *obs_dev,
                   float *reward_dev, int32_t *coll_dev);

/* Waits for the stream, returns and clears the latched FLOCK_ERR_* bits; after
 * a FLOCK_ERR_TIMEOUT it also resets the grid-barrier counters. */
int env_batch_get_error(flock_batch *batch, uint32_t *bits_out);

/* Bound on the polls of one grid-barrier wait (default 1<<22, about a
 * second); a wait that runs out sets FLOCK_ERR_TIMEOUT and the kernel
 * returns.  0 makes every wait give up at once (for tests of that path). */
int env_batch_set_spin_limit(flock_batch *batch, unsigned limit);

/* Grid size (blocks) and block size of the persistent kernel, and the
 * duration of the last step in ms when timing is on (events around the
 * kernel, recorded inside the replayed graph). */
int env_batch_get_launch(const flock_batch *batch, int *grid_out, int *block_out);
int env_batch_set_timing(flock_batch *batch, int enable);
int env_batch_get_time(flock_batch *batch, float *ms_out);

void env_batch_destroy(flock_batch *batch);

/* ---------------------------------------------------------------------------
 * Slabs: one square decomposed over several devices (a square too large for
 * one GPU's memory).  Band b of R owns the rows [r_b, r_{b+1}) of the
 * square's cell grid (flock_derive: cells_per_side rows of width side /
 * cells_per_side).  A slab environment holds the cell list of its band plus
 * H rows on each side (H = the stencil's halo, 1 for the 3 x 3 stencil):
 * rows [row0, row0 + nrows) modulo cells_per_side, row0 = r_b - H, nrows =
 * r_{b+1} - r_b + 2H.  Each step (Section 4.1: all agents act, then all
 * observe the new positions):
 *   1. env_slab_apply: the band's own agents take their actions;
 *   2. the caller moves agents that left the band to the band that now owns
 *      them, and copies every own agent in the H rows next to a band edge to
 *      the band across that edge (a ghost; coordinates on the square, never
 *      shifted, so offsets across the square's edge are formed as on the
 *      undivided square);
 *   3. env_slab_observe: own agents observe own and ghost agents.
 * The outputs equal those of the undivided square, bit for bit (same
 * pairs, same FP32 operations, exact reward sums).  Agents must not move
 * more than one band per step (speed_max below the band height).  The
 * decomposition itself (which agents move, which are ghosts, the exchange)
 * is in the Python package (slab.py); these calls compute on one device.
 * ------------------------------------------------------------------------- */

/* Workspace of a slab environment of at most n_max agents (own + ghosts)
 * and rows [row0, row0 + nrows) (0 <= row0 < cells_per_side, 2H + 1 <=
 * nrows <= cells_per_side).  The tuning must use the direct neighbour scan
 * (mode 0 or 2). */
int flock_slab_workspace_bytes(const flock_params *params, const flock_tuning *tuning_or_null,
                               int n_max, int row0, int nrows, size_t *bytes_out);

/* Creates a slab environment (the ownership and stream rules of env_create).
 * Use env_slab_apply / env_slab_observe (and env_get_error, env_destroy) with
 * it, not env_reset / env_step. */
int env_slab_create(const flock_params *params, const flock_tuning *tuning_or_null, int n_max,
                    int row0, int nrows, void *workspace_dev, size_t workspace_bytes,
                    void *stream, flock_env **out);

/* Applies actions_dev (n int32, the discrete actions of env_step) to the n
 * agents of state_dev (n x 4 floats, 16-byte aligned) in place.  Invalid
 * actions and states latch FLOCK_ERR_ACTION / FLOCK_ERR_STATE. */
int env_slab_apply(flock_env *env, int n, float *state_dev, const int32_t *actions_dev);

/* Observes the first n_own agents of state_dev ((n_own + n_ghost) x 4
 * floats: the band's own agents, then its ghosts, all already moved) over
 * all of them: obs_dev (n_own x obs_dim), reward_dev and coll_dev (n_own)
 * as for env_step.  n_own + n_ghost <= n_max.  Every agent must lie in the
 * slab's rows. */
int env_slab_observe(flock_env *env, int n_own, int n_ghost, const float *state_dev,
                     float *obs_dev, float *reward_dev, int32_t *coll_dev);

/* ---------------------------------------------------------------------------
 * Allocation-free step.  (The paper has no counterpart: this entry point exists
 * for callers of this library that cannot allocate device memory -- code in a
 * host callback or real-time loop where cudaMalloc may block or is not
 * allowed, or a plugin whose host application owns all device memory.)
 *
 * One step of a flock environment of n_agents agents, with every scratch
 * buffer taken from a fixed array of FLOCK_STATIC_SCRATCH_BYTES bytes that
 * the library declares in device memory.  Each GPU that loads the library
 * holds that array until the process exits.  The caller passes only:
 *   state_dev    n x 4 floats, read and updated in place;
 *   actions_dev  n int32, or NULL to observe the state without moving it;
 *   obs_dev, reward_dev, coll_dev  the outputs, as for env_step.
 * The call enqueues on `stream` and returns; with error_bits_out non-NULL it
 * waits for the stream and stores the FLOCK_ERR_* bits of this call.  Any
 * observation layout is accepted; obs_dev holds flock_obs_dim(params) values
 * per row, 8-byte aligned.  `stream` must belong to the current device, and
 * must not be in stream capture: each call copies its parameter descriptor
 * from pageable host memory (and may wait for the stream), so a call made
 * while `stream` is being captured, or with a stream of another device,
 * returns FLOCK_EINVAL and enqueues nothing.
 *
 * Limits: at most FLOCK_STATIC_MAX_AGENTS agents and a cell list of at most
 * FLOCK_STATIC_MAX_CELLS cells (cells_per_side^2 of flock_derive with the
 * default 3 x 3 stencil); larger sizes return FLOCK_EINVAL.  The call does
 * no cudaMalloc or cudaFree and calls no allocating library routine.
 *
 * Every call on a device uses the same array, which keeps the previous
 * call's contents; the call clears what must start at zero itself.  Calls
 * whose work overlaps on the GPU (different streams, or threads without
 * ordering) race on the array: order them on one stream.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) for that
 * device; make that first call before any stream capture is in progress.
 * ------------------------------------------------------------------------- */
#define FLOCK_STATIC_MAX_AGENTS 65536
#define FLOCK_STATIC_MAX_CELLS 32768
#define FLOCK_STATIC_SCRATCH_BYTES 1705472
int flock_step_static(const flock_params *params, int n_agents, float *state_dev,
                      const int32_t *actions_dev, float *obs_dev, float *reward_dev,
                      int32_t *coll_dev, void *stream, uint32_t *error_bits_out);

/* Last CUDA error string seen by the library in this process (or ""). */
const char *flock_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLOCK_H */
