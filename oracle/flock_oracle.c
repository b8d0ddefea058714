/*
 * Flock environment oracle -- TEST INFRASTRUCTURE, NOT THE PRODUCT PATH.
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * may load this library.  It shares no code, header, table or constant
 * generator with the CUDA library under paper_2207_03945_gb300/.
 *
 * What it computes: one update of the flock environment of "High Performance
 * Simulation for Scalable Multi-Agent Reinforcement Learning" (arXiv
 * 2207.03945), Section 4.1, as the plain brute-force definition over every
 * ordered pair (i, j), i != j, with no cell list:
 *
 *   1. every agent applies its action: accelerate (speed clamped to
 *      [s_min, s_max]) and rotate, then moves along its heading on the
 *      periodic square (Section 4.1: actions are applied first);
 *   2. with the new positions, every agent observes every other agent
 *      (Section 4.1, "for all pairs of agents in spatial proximity"):
 *        - range: d_ij < d_v (Eq. 1, strict);
 *        - reward r_i = sum_j f(d_ij) over in-range j (Eq. 1), with f from
 *          Fig. 4: -P when the agents collide (d < 2 d_r), otherwise the
 *          linear ramp (d_v - d) / (d_v - 2 d_r);
 *        - vision (Section 4, Fig. 3): the field of view, centred on the
 *          heading, is cut into v equal angular sectors numbered
 *          counter-clockwise from its right edge; each sector records the
 *          distance to the nearest in-range agent whose centre falls in it
 *          (d_v when empty) and how many such agents there are.
 *
 * Arithmetic: IEEE binary32, round to nearest, one operation at a time (build
 * with -ffp-contract=off, no fast-math), denormals kept.  Every FP32 formula
 * below is written out so that a second implementation that follows the same
 * formulas reaches identical bits.  The angular sector of a neighbour is taken
 * from a division-based pseudo-angle ("diamond angle") that is monotone in the
 * true angle; the sector edges are the pseudo-angles of the exact edge angles,
 * computed in double and rounded once.
 *
 * The reward sum (Eq. 1) is evaluated exactly: each FP32 term f(d_ij) is an
 * integer multiple of 2^-K (K derived below from the parameters), the terms
 * are added as 64-bit integers, and the exact total is rounded once to FP32.
 * The result therefore does not depend on the order of the j loop.
 *
 * Readings where the paper is silent or garbled (Section 4.1 prints the speed
 * update with min and max swapped; Fig. 4 shows f only as a plot; the paper
 * gives no boundary behaviour) are stated next to the code that takes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXV 128

/* Status codes and latched condition bits (same meaning as the product's). */
#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_FLAG_ACTION 1u   /* an action outside [0, 9) was replaced by 4, or a
                               continuous action component was not finite */
#define OR_FLAG_STATE 2u    /* a state component was non-finite or out of range */
#define OR_FLAG_OVERFLOW 8u /* more in-range neighbours than the 64-bit sum holds */

typedef struct {
  float side;              /* L, the periodic square is [0, L)^2 */
  float view_radius;       /* d_v */
  float fov;               /* field of view in radians, (0, 2pi]; (float)2pi = full circle */
  float agent_radius;      /* d_r; agents collide when d < 2 d_r (Fig. 4) */
  float collision_penalty; /* P */
  float speed_min, speed_max;
  float speed_step; /* a: speed change of one acceleration action */
  float turn_step;  /* Delta: heading change of one rotation action, radians */
  int num_segments; /* v */
} oracle_params;

typedef struct {
  float L, HL, RV, RV2, RC2, INV_SPAN, TWO_PI, CF, SF, SMIN, SMAX;
  float DT[3], DS[3];
  float T[OR_MAXV + 1]; /* T[m], m = 1..v: pseudo-angle of sector edge m */
  int v, full, K;
  int64_t PK;   /* P * 2^K, exact */
  int64_t NMAX; /* largest in-range count whose worst-case sum fits in 62 bits */
} oracle_derived;

/* ------------------------------------------------------------------ */
/* Deterministic sine/cosine: Cody-Waite reduction by pi/2 followed by */
/* Taylor polynomials, FP32 throughout.                                */
/* ------------------------------------------------------------------ */
static const float TWO_OVER_PI = 0x1.45f306p-1f; /* (float)(2/pi) */
static const float PIO2_HI = 1.5703125f;         /* 8 significant bits: q*hi exact for q <= 4 */
static const float PIO2_LO = 0x1.fb5444p-12f;    /* (float)(pi/2 - 1.5703125) */
/* Taylor coefficients, each the float nearest to the exact rational. */
static const float S1 = -0x1.555556p-3f; /* -1/3!  */
static const float S2 = 0x1.111112p-7f;  /*  1/5!  */
static const float S3 = -0x1.a01a02p-13f;/* -1/7!  */
static const float S4 = 0x1.71de3ap-19f; /*  1/9!  */
static const float C1 = -0.5f;           /* -1/2!  */
static const float C2 = 0x1.555556p-5f;  /*  1/4!  */
static const float C3 = -0x1.6c16c2p-10f;/* -1/6!  */
static const float C4 = 0x1.a01a02p-16f; /*  1/8!  */

void oracle_sincos(float th, float *c_out, float *s_out) {
  int q = (int)rintf(th * TWO_OVER_PI);
  float qf = (float)q;
  float r = (th - qf * PIO2_HI) - qf * PIO2_LO;
  float r2 = r * r;
  float ps = S3 + r2 * S4;
  ps = S2 + r2 * ps;
  ps = S1 + r2 * ps;
  float sr = r + (r * r2) * ps;
  float pc = C3 + r2 * C4;
  pc = C2 + r2 * pc;
  pc = C1 + r2 * pc;
  float cr = 1.0f + r2 * pc;
  switch (q & 3) {
    case 0: *c_out = cr; *s_out = sr; break;
    case 1: *c_out = -sr; *s_out = cr; break;
    case 2: *c_out = -cr; *s_out = -sr; break;
    default: *c_out = sr; *s_out = -cr; break;
  }
}

/* Pseudo-angle of the direction (x, y) in [0, 4): 0 along +x, increasing
 * counter-clockwise, one unit per quadrant; monotone in the true angle. */
float oracle_diamond(float x, float y) {
  if (y >= 0.0f) {
    if (x >= 0.0f) return y / (x + y);
    return 1.0f + (-x) / (-x + y);
  }
  if (x < 0.0f) return 2.0f + (-y) / (-x - y);
  return 3.0f + x / (x - y);
}

static double diamond_d(double x, double y) {
  if (y >= 0.0) {
    if (x >= 0.0) return y / (x + y);
    return 1.0 + (-x) / (-x + y);
  }
  if (x < 0.0) return 2.0 + (-y) / (-x - y);
  return 3.0 + x / (x - y);
}

/* Derived constants, computed from the parameters in double where a
 * transcendental is involved and rounded once to float.  Returns OR_EINVAL
 * for parameters the model cannot take. */
int oracle_derive(const oracle_params *p, oracle_derived *d) {
  memset(d, 0, sizeof *d);
  const double PI = 3.14159265358979323846;
  if (!(isfinite(p->side) && isfinite(p->view_radius) && isfinite(p->fov) &&
        isfinite(p->agent_radius) && isfinite(p->collision_penalty) &&
        isfinite(p->speed_min) && isfinite(p->speed_max) &&
        isfinite(p->speed_step) && isfinite(p->turn_step)))
    return OR_EINVAL;
  if (p->num_segments < 1 || p->num_segments > OR_MAXV) return OR_EINVAL;
  if (!(p->view_radius > 0.0f) || !(p->agent_radius >= 0.0f)) return OR_EINVAL;
  if (!(2.0f * p->agent_radius < p->view_radius)) return OR_EINVAL;
  if (!(p->side > 2.0f * p->view_radius)) return OR_EINVAL;
  if (!(p->speed_min >= 0.0f && p->speed_min <= p->speed_max && p->speed_max < p->side))
    return OR_EINVAL;
  if (!(p->collision_penalty >= 0.0f)) return OR_EINVAL;
  if (!(p->turn_step >= 0.0f && p->turn_step < (float)PI)) return OR_EINVAL;
  if (!(p->speed_step >= 0.0f)) return OR_EINVAL;

  d->L = p->side;
  d->HL = 0.5f * p->side;
  d->RV = p->view_radius;
  d->RV2 = p->view_radius * p->view_radius;
  float two_dr = 2.0f * p->agent_radius;
  d->RC2 = two_dr * two_dr;
  d->INV_SPAN = (float)(1.0 / ((double)p->view_radius - 2.0 * (double)p->agent_radius));
  d->TWO_PI = (float)(2.0 * PI);
  d->SMIN = p->speed_min;
  d->SMAX = p->speed_max;
  if (!(p->fov > 0.0f && p->fov <= d->TWO_PI)) return OR_EINVAL;
  d->full = p->fov == d->TWO_PI;
  d->v = p->num_segments;
  double fov = d->full ? 2.0 * PI : (double)p->fov;
  if (d->full) {
    /* full circle: the sectors start straight behind the agent */
    d->CF = -1.0f;
    d->SF = 0.0f;
  } else {
    d->CF = (float)cos(0.5 * fov);
    d->SF = (float)sin(0.5 * fov);
  }
  for (int m = 1; m <= d->v; ++m) {
    double phi = (double)m * fov / (double)d->v;
    d->T[m] = (float)diamond_d(cos(phi), sin(phi));
  }
  d->DT[0] = -p->turn_step; d->DT[1] = 0.0f; d->DT[2] = p->turn_step;
  d->DS[0] = -p->speed_step; d->DS[1] = 0.0f; d->DS[2] = p->speed_step;

  /* The in-range test d2 < RV2 must never admit sqrtf(d2) > d_v. */
  float rv = p->view_radius;
  if (sqrtf(nextafterf(d->RV2, 0.0f)) > rv) return OR_EINVAL;

  /* Fixed-point exponent K for the exact reward sum.  The smallest positive
   * ramp term comes from the largest float below d_v; every ramp term is at
   * least that and so a multiple of 2^(e_min - 23).  -P must be one too. */
  float diff_min = rv - nextafterf(rv, 0.0f);
  float t_min = diff_min * d->INV_SPAN;
  if (!(t_min > 0.0f)) return OR_EINVAL;
  int e;
  frexpf(t_min, &e); /* t_min in [2^(e-1), 2^e) */
  int K = 24 - e;
  if (p->collision_penalty > 0.0f) {
    int ep;
    frexpf(p->collision_penalty, &ep);
    if (24 - ep > K) K = 24 - ep;
  }
  if (K < 0) K = 0;
  if (K > 60) return OR_EINVAL;
  float s_lo = sqrtf(d->RC2); /* smallest distance of a non-colliding pair */
  float t_max = (rv - s_lo) * d->INV_SPAN;
  double max_term = (double)t_max > (double)p->collision_penalty ? (double)t_max
                                                                  : (double)p->collision_penalty;
  if (max_term < 1.0) max_term = 1.0;
  double scaled = ldexp(max_term, K);
  double nmax = floor(ldexp(1.0, 62) / scaled);
  if (nmax < 1.0) return OR_EINVAL;
  d->NMAX = nmax > 9.0e15 ? (int64_t)9.0e15 : (int64_t)nmax;
  d->K = K;
  d->PK = (int64_t)ldexp((double)p->collision_penalty, K);
  if ((double)d->PK != ldexp((double)p->collision_penalty, K)) return OR_EINVAL;
  return OR_OK;
}

int oracle_derive_export(const oracle_params *p, oracle_derived *d) { return oracle_derive(p, d); }
int oracle_derived_size(void) { return (int)sizeof(oracle_derived); }

/* ------------------------------------------------------------------ */
/* Step part 1: apply the actions (Section 4.1).                       */
/* ------------------------------------------------------------------ */
static float wrap_coord(float x, float L) {
  if (x >= L) x = x - L;
  else if (x < 0.0f) x = x + L;
  if (x >= L) x = 0.0f; /* x + L rounded up to L */
  return x;
}

static int state_ok(const oracle_derived *d, const float *st) {
  for (int c = 0; c < 4; ++c)
    if (!isfinite(st[c])) return 0;
  return st[0] >= 0.0f && st[0] < d->L && st[1] >= 0.0f && st[1] < d->L && st[2] >= 0.0f &&
         st[2] < d->TWO_PI && st[3] >= d->SMIN && st[3] <= d->SMAX;
}

/* Speed change ds and heading change dt of one agent, then the move: the
 * speed update is read as a clamp to [s_min, s_max] (the printed formula has
 * min and max swapped), the heading wraps into [0, 2pi) (|dt| < pi, so one
 * wrap is enough), and the agent moves one step along the new heading. */
static void move_one(const oracle_derived *d, float *st, float ds, float dt) {
  float s = st[3] + ds;
  if (s < d->SMIN) s = d->SMIN;
  else if (s > d->SMAX) s = d->SMAX;
  float th = st[2] + dt;
  if (th >= d->TWO_PI) th = th - d->TWO_PI;
  else if (th < 0.0f) th = th + d->TWO_PI;
  if (th >= d->TWO_PI) th = 0.0f;
  float c, sn;
  oracle_sincos(th, &c, &sn);
  float x = st[0] + s * c;
  float y = st[1] + s * sn;
  st[0] = wrap_coord(x, d->L);
  st[1] = wrap_coord(y, d->L);
  st[2] = th;
  st[3] = s;
}

/* Discrete action a in [0, 9): turn = a / 3 picks {-Delta, 0, +Delta}, speed
 * = a % 3 picks {-a, 0, +a}. */
static void apply_one(const oracle_derived *d, float *st, int32_t a, uint32_t *flags) {
  if (a < 0 || a >= 9) {
    a = 4;
    *flags |= OR_FLAG_ACTION;
  }
  int tu = a / 3, su = a % 3;
  move_one(d, st, d->DS[su], d->DT[tu]);
}

/* Continuous action (acceleration, rotation), the two-dimensional action
 * space of the paper's flock (Section 4.1): the acceleration lies in
 * [-a_max, a_max] and the rotation in [-theta_max, theta_max]; here
 * a_max = speed_step and theta_max = turn_step, and values outside are
 * clamped to the range (reading: the ranges bound the action).  A component
 * that is not finite counts as 0 and raises OR_FLAG_ACTION. */
static void apply_cont(const oracle_derived *d, float *st, const float *a, uint32_t *flags) {
  float acc = a[0], rot = a[1];
  if (!isfinite(acc)) {
    acc = 0.0f;
    *flags |= OR_FLAG_ACTION;
  }
  if (!isfinite(rot)) {
    rot = 0.0f;
    *flags |= OR_FLAG_ACTION;
  }
  const float amax = d->DS[2], tmax = d->DT[2];
  if (acc < -amax) acc = -amax;
  else if (acc > amax) acc = amax;
  if (rot < -tmax) rot = -tmax;
  else if (rot > tmax) rot = tmax;
  move_one(d, st, acc, rot);
}

/* ------------------------------------------------------------------ */
/* Step part 2: observation, collisions and reward of agent i over all */
/* other agents (Eq. 1, Fig. 3, Fig. 4), brute force.                  */
/* ------------------------------------------------------------------ */
static void observe_one(const oracle_derived *d, int n, const float *state, int i,
                        float *obs_row, float *reward_i, int32_t *coll_i, uint32_t *flags) {
  const int v = d->v;
  float mind2[OR_MAXV];
  int32_t cnt[OR_MAXV];
  for (int k = 0; k < v; ++k) {
    mind2[k] = INFINITY;
    cnt[k] = 0;
  }
  const float xi = state[4 * i + 0], yi = state[4 * i + 1];
  const float thi = state[4 * i + 2], si = state[4 * i + 3];
  float c, sn;
  oracle_sincos(thi, &c, &sn);
  /* start edge of the field of view: the heading turned clockwise by fov/2 */
  const float ux = c * d->CF + sn * d->SF;
  const float uy = sn * d->CF - c * d->SF;
  const float scaleK = ldexpf(1.0f, d->K);
  int64_t acc = 0;
  int64_t nin = 0;
  int32_t ncoll = 0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    /* minimum-image difference on the periodic square */
    float dx = state[4 * j + 0] - xi;
    if (dx > d->HL) dx = dx - d->L;
    else if (dx < -d->HL) dx = dx + d->L;
    float dy = state[4 * j + 1] - yi;
    if (dy > d->HL) dy = dy - d->L;
    else if (dy < -d->HL) dy = dy + d->L;
    float d2 = dx * dx + dy * dy;
    if (!(d2 < d->RV2)) continue; /* Eq. 1: d_ij < d_v, strict */
    nin++;
    if (d2 < d->RC2) { /* Fig. 4: collision at a distance below 2 d_r */
      ncoll++;
      acc -= d->PK;
    } else {
      float dist = sqrtf(d2);
      float t = (d->RV - dist) * d->INV_SPAN;
      acc += (int64_t)(t * scaleK); /* exact: t is a multiple of 2^-K */
    }
    /* neighbour direction in the frame whose x axis is the FOV start edge */
    float lx = dx * ux + dy * uy;
    float ly = dy * ux - dx * uy;
    if (lx == 0.0f && ly == 0.0f) continue; /* coincident: no direction */
    float pa = oracle_diamond(lx, ly);
    if (pa >= 4.0f) pa = 0.0f;
    if (!d->full && pa >= d->T[v]) continue; /* outside the field of view */
    int k = 0;
    for (int m = 1; m < v; ++m)
      if (pa >= d->T[m]) k++;
    if (d2 < mind2[k]) mind2[k] = d2;
    cnt[k]++;
  }
  for (int k = 0; k < v; ++k) {
    obs_row[2 * k] = cnt[k] ? sqrtf(mind2[k]) : d->RV;
    obs_row[2 * k + 1] = (float)cnt[k];
  }
  obs_row[2 * v] = si;
  obs_row[2 * v + 1] = thi;
  *reward_i = (float)acc * ldexpf(1.0f, -d->K);
  *coll_i = ncoll;
  if (nin > d->NMAX) *flags |= OR_FLAG_OVERFLOW;
}

/* One environment update.  state: n x 4 floats (x, y, theta, s), updated in
 * place.  actions: n int32 in [0, 9), or NULL for a reset (observe only).
 * obs: n x (2v+2) floats; reward: n floats; coll: n int32.  flags receives
 * the OR of the condition bits.  threads <= 0 uses the OpenMP default. */
int oracle_step(const oracle_params *p, int n, float *state, const int32_t *actions, float *obs,
                float *reward, int32_t *coll, uint32_t *flags_out, int threads) {
  oracle_derived d;
  int rc = oracle_derive(p, &d);
  if (rc != OR_OK) return rc;
  if (n < 0) return OR_EINVAL;
  const size_t D = (size_t)(2 * d.v + 2);
  uint32_t flags = 0;
  for (int i = 0; i < n; ++i) {
    if (!state_ok(&d, state + 4 * i)) flags |= OR_FLAG_STATE;
    if (actions) apply_one(&d, state + 4 * i, actions[i], &flags);
  }
#ifdef _OPENMP
  int nt = threads > 0 ? threads : omp_get_max_threads();
  uint32_t oflags = 0;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(| : oflags)
  for (int i = 0; i < n; ++i) {
    uint32_t f = 0;
    observe_one(&d, n, state, i, obs + (size_t)i * D, reward + i, coll + i, &f);
    oflags |= f;
  }
  flags |= oflags;
#else
  (void)threads;
  for (int i = 0; i < n; ++i)
    observe_one(&d, n, state, i, obs + (size_t)i * D, reward + i, coll + i, &flags);
#endif
  if (flags_out) *flags_out = flags;
  return OR_OK;
}

/* Observation of a subset of agents (rows idx[0..m)) only, for sampled
 * checks at sizes where the full O(N^2) step is too slow.  state must already
 * hold the post-action positions. */
int oracle_observe_rows(const oracle_params *p, int n, const float *state, int m,
                        const int32_t *idx, float *obs_rows, float *reward_rows,
                        int32_t *coll_rows, int threads) {
  oracle_derived d;
  int rc = oracle_derive(p, &d);
  if (rc != OR_OK) return rc;
  const int D = 2 * d.v + 2;
#ifdef _OPENMP
  int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
#else
  (void)threads;
#endif
  for (int r = 0; r < m; ++r) {
    int i = idx[r];
    if (i < 0 || i >= n) continue;
    uint32_t f = 0;
    observe_one(&d, n, state, i, obs_rows + (size_t)r * D, reward_rows + r, coll_rows + r, &f);
  }
  return OR_OK;
}

/* Apply actions only (no observation); for sampled checks at large N. */
int oracle_apply(const oracle_params *p, int n, float *state, const int32_t *actions,
                 uint32_t *flags_out) {
  oracle_derived d;
  int rc = oracle_derive(p, &d);
  if (rc != OR_OK) return rc;
  uint32_t flags = 0;
  for (int i = 0; i < n; ++i) apply_one(&d, state + 4 * i, actions[i], &flags);
  if (flags_out) *flags_out = flags;
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* The paper's own flock variant: continuous actions and the view-only */
/* observation (Section 4.1: the view of v sectors and the speed).     */
/* ------------------------------------------------------------------ */

/* Observation layouts: 0 = per sector (distance, count), then speed and
 * heading (2v + 2 values); 1 = per sector the distance, then the speed
 * (v + 1 values), the 129-value observation of Section 4.1 for v = 128. */
int oracle_obs_dim(const oracle_params *p, int layout) {
  return layout == 1 ? p->num_segments + 1 : 2 * p->num_segments + 2;
}

/* One update with continuous actions.  actions: n x 2 floats (acceleration,
 * rotation) or NULL for a reset; obs: n x oracle_obs_dim(p, layout). */
int oracle_step_cont(const oracle_params *p, int n, float *state, const float *actions,
                     int layout, float *obs, float *reward, int32_t *coll, uint32_t *flags_out,
                     int threads) {
  oracle_derived d;
  int rc = oracle_derive(p, &d);
  if (rc != OR_OK) return rc;
  if (n < 0 || (layout != 0 && layout != 1)) return OR_EINVAL;
  const int v = d.v;
  const size_t D = (size_t)oracle_obs_dim(p, layout);
  uint32_t flags = 0;
  for (int i = 0; i < n; ++i) {
    if (!state_ok(&d, state + 4 * i)) flags |= OR_FLAG_STATE;
    if (actions) apply_cont(&d, state + 4 * i, actions + 2 * i, &flags);
  }
#ifdef _OPENMP
  int nt = threads > 0 ? threads : omp_get_max_threads();
  uint32_t oflags = 0;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(| : oflags)
#else
  (void)threads;
  uint32_t oflags = 0;
#endif
  for (int i = 0; i < n; ++i) {
    uint32_t f = 0;
    float row[2 * OR_MAXV + 2];
    observe_one(&d, n, state, i, row, reward + i, coll + i, &f);
    float *o = obs + (size_t)i * D;
    if (layout == 0) {
      memcpy(o, row, (2 * (size_t)v + 2) * sizeof(float));
    } else {
      for (int k = 0; k < v; ++k) o[k] = row[2 * k]; /* distances */
      o[v] = row[2 * v];                             /* speed */
    }
    oflags |= f;
  }
  flags |= oflags;
  if (flags_out) *flags_out = flags;
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Advantages over a rollout (the trajectory processing of Section 4.3: */
/* PPO on the n x t trajectories of one training step).                 */
/* ------------------------------------------------------------------ */
/* Generalised advantage estimation over T steps of n agents, FP32, one
 * operation at a time, in this order (the definition written out):
 *   gl = gamma * lambda
 *   for t = T-1 down to 0:
 *     delta_t = (r_t + gamma * v_{t+1}) - v_t
 *     A_t     = delta_t + gl * A_{t+1}        (A_T = 0)
 *     R_t     = A_t + v_t                     (the value target)
 * reward: T x n, value: (T+1) x n (v_T bootstraps the last step: the flock
 * never terminates), adv and ret: T x n, all row-major by step. */
int oracle_gae(int T, int n, const float *reward, const float *value, float gamma, float lambda,
               float *adv, float *ret) {
  if (T < 0 || n < 0) return OR_EINVAL;
  if (!(gamma >= 0.0f && gamma <= 1.0f && lambda >= 0.0f && lambda <= 1.0f)) return OR_EINVAL;
  const float gl = gamma * lambda;
  for (int i = 0; i < n; ++i) {
    float a = 0.0f;
    for (int t = T - 1; t >= 0; --t) {
      const size_t k = (size_t)t * n + i;
      const float delta = (reward[k] + gamma * value[k + n]) - value[k];
      a = delta + gl * a;
      adv[k] = a;
      ret[k] = a + value[k];
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Tag (Section 4.2): runners and chasers.                             */
/* ------------------------------------------------------------------ */
/* Agents of type 0 are runners, of type 1 chasers.  Readings (the section
 * describes the rewards in words only):
 *   - a runner gets the flock reward from runners (Eq. 1 with f of Fig. 4:
 *     the linear ramp for 2 d_r <= d < d_v) and -P for every agent it
 *     touches (d < 2 d_r), runner or chaser ("penalised for touching a
 *     chaser"; touching a runner is the flock's collision);
 *   - a chaser gets +P for every runner it touches and nothing else;
 *   - the view has two colour channels of v sectors: channel 0 holds the
 *     nearest runner per sector, channel 1 the nearest chaser (d_v when
 *     empty); the observation is the 2v distances, runners first;
 *   - the action (speed, rotation) sets the speed, clamped to
 *     [s_min, s_max], and turns the heading by the rotation clamped to
 *     [-Delta, Delta]; a non-finite component acts as 0 and is flagged;
 *   - coll counts every touching pair, whatever the types. */
static void apply_tag(const oracle_derived *d, float *st, const float *a, uint32_t *flags) {
  float spd = a[0], rot = a[1];
  if (!isfinite(spd)) {
    spd = 0.0f;
    *flags |= OR_FLAG_ACTION;
  }
  if (!isfinite(rot)) {
    rot = 0.0f;
    *flags |= OR_FLAG_ACTION;
  }
  const float tmax = d->DT[2];
  if (rot < -tmax) rot = -tmax;
  else if (rot > tmax) rot = tmax;
  /* setting the speed is a change of (spd - s); the clamp follows in move_one */
  if (spd < d->SMIN) spd = d->SMIN;
  else if (spd > d->SMAX) spd = d->SMAX;
  st[3] = spd;
  move_one(d, st, 0.0f, rot);
}

static void observe_tag(const oracle_derived *d, int n, const float *state, const uint8_t *type,
                        int i, float *obs_row, float *reward_i, int32_t *coll_i, uint32_t *flags) {
  const int v = d->v;
  float mind2[2 * OR_MAXV];
  for (int k = 0; k < 2 * v; ++k) mind2[k] = INFINITY;
  const float xi = state[4 * i + 0], yi = state[4 * i + 1];
  const float thi = state[4 * i + 2];
  const int ti = type[i] != 0;
  float c, sn;
  oracle_sincos(thi, &c, &sn);
  const float ux = c * d->CF + sn * d->SF;
  const float uy = sn * d->CF - c * d->SF;
  const float scaleK = ldexpf(1.0f, d->K);
  int64_t acc = 0;
  int64_t nin = 0;
  int32_t ncoll = 0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    const int tj = type[j] != 0;
    float dx = state[4 * j + 0] - xi;
    if (dx > d->HL) dx = dx - d->L;
    else if (dx < -d->HL) dx = dx + d->L;
    float dy = state[4 * j + 1] - yi;
    if (dy > d->HL) dy = dy - d->L;
    else if (dy < -d->HL) dy = dy + d->L;
    float d2 = dx * dx + dy * dy;
    if (!(d2 < d->RV2)) continue;
    nin++;
    const int touch = d2 < d->RC2;
    if (touch) ncoll++;
    if (ti == 0) {
      if (touch) acc -= d->PK;               /* any touch costs a runner P */
      else if (tj == 0) {                    /* proximity to runners */
        float t = (d->RV - sqrtf(d2)) * d->INV_SPAN;
        acc += (int64_t)(t * scaleK);
      }
    } else if (touch && tj == 0) {
      acc += d->PK;                          /* a chaser touching a runner */
    }
    float lx = dx * ux + dy * uy;
    float ly = dy * ux - dx * uy;
    if (lx == 0.0f && ly == 0.0f) continue;
    float pa = oracle_diamond(lx, ly);
    if (pa >= 4.0f) pa = 0.0f;
    if (!d->full && pa >= d->T[v]) continue;
    int k = 0;
    for (int m = 1; m < v; ++m)
      if (pa >= d->T[m]) k++;
    k += tj * v; /* colour channel of the neighbour's type */
    if (d2 < mind2[k]) mind2[k] = d2;
  }
  for (int k = 0; k < 2 * v; ++k) obs_row[k] = isinf(mind2[k]) ? d->RV : sqrtf(mind2[k]);
  *reward_i = (float)acc * ldexpf(1.0f, -d->K);
  *coll_i = ncoll;
  if (nin > d->NMAX) *flags |= OR_FLAG_OVERFLOW;
}

/* One tag update.  type: n bytes (0 runner, 1 chaser); actions: n x 2 floats
 * (speed, rotation) or NULL for a reset; obs: n x 2v floats. */
int oracle_step_tag(const oracle_params *p, int n, float *state, const uint8_t *type,
                    const float *actions, float *obs, float *reward, int32_t *coll,
                    uint32_t *flags_out, int threads) {
  oracle_derived d;
  int rc = oracle_derive(p, &d);
  if (rc != OR_OK) return rc;
  if (n < 0) return OR_EINVAL;
  /* a chaser's reward is +P per touched runner: P * 2^K must fit as well */
  const size_t D = 2 * (size_t)d.v;
  uint32_t flags = 0;
  for (int i = 0; i < n; ++i) {
    if (!state_ok(&d, state + 4 * i)) flags |= OR_FLAG_STATE;
    if (actions) apply_tag(&d, state + 4 * i, actions + 2 * i, &flags);
  }
  uint32_t oflags = 0;
#ifdef _OPENMP
  int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(| : oflags)
#else
  (void)threads;
#endif
  for (int i = 0; i < n; ++i) {
    uint32_t f = 0;
    observe_tag(&d, n, state, type, i, obs + (size_t)i * D, reward + i, coll + i, &f);
    oflags |= f;
  }
  flags |= oflags;
  if (flags_out) *flags_out = flags;
  return OR_OK;
}
