// Advantages over a rollout: the trajectory processing that follows the
// environment steps of one training step (arXiv 2207.03945, Section 4.3:
// PPO on the n x t trajectories gathered across all agents).
//
// Generalised advantage estimation, FP32 with explicit round-to-nearest
// operations in this order (the flock never terminates, so v_T bootstraps):
//   gl = gamma * lambda                      (rounded once, on the host)
//   for t = T-1 down to 0:
//     delta_t = (r_t + gamma * v_{t+1}) - v_t
//     A_t     = delta_t + gl * A_{t+1}        (A_T = 0)
//     R_t     = A_t + v_t
// A block takes 32 agents (one warp's columns) and walks the rollout from
// the last step back in chunks of kChunk steps: all its threads stage the
// chunk's rewards and values in shared memory (each step row of 32 agents is
// 128 contiguous bytes), one warp runs the recurrence over the chunk (lane =
// agent) in place, and all threads write the advantages and targets back.
// Many blocks per SM keep the loads in flight while others compute.
// HBM-bound: 16 bytes per (step, agent).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "flock.h"
#include "flock_host.h"

namespace flock {

constexpr int kChunk = 64;     // steps staged per pass
constexpr int kGaeBlock = 256;  // threads per block; 32 agents per block

__global__ void __launch_bounds__(kGaeBlock) k_gae(int T, int n, const float *__restrict__ r,
                                                   const float *__restrict__ v, float gamma,
                                                   float gl, float *__restrict__ adv,
                                                   float *__restrict__ ret) {
  __shared__ float sr[kChunk][32], sv[kChunk][32];
  const int i0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, row0 = threadIdx.x >> 5;
  const int i = i0 + lane;
  const bool have = i < n;
  float a = 0.0f;
  float vnext = 0.0f;
  if (threadIdx.x < 32 && have) vnext = v[(size_t)T * n + i];
  for (int t1 = T; t1 > 0; t1 -= kChunk) {
    const int c = t1 < kChunk ? t1 : kChunk;  // steps t1-1 down to t1-c, row u = t1-1-u
    for (int u = row0; u < c; u += kGaeBlock / 32) {
      if (have) {
        const size_t k = (size_t)(t1 - 1 - u) * n + i;
        sr[u][lane] = r[k];
        sv[u][lane] = v[k];
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      for (int u = 0; u < c; ++u) {
        const float vt = sv[u][lane];
        const float delta = __fsub_rn(__fadd_rn(sr[u][lane], __fmul_rn(gamma, vnext)), vt);
        a = __fadd_rn(delta, __fmul_rn(gl, a));
        sr[u][lane] = a;                  // advantage
        sv[u][lane] = __fadd_rn(a, vt);   // value target
        vnext = vt;
      }
    }
    __syncthreads();
    for (int u = row0; u < c; u += kGaeBlock / 32) {
      if (have) {
        const size_t k = (size_t)(t1 - 1 - u) * n + i;
        adv[k] = sr[u][lane];
        ret[k] = sv[u][lane];
      }
    }
    __syncthreads();
  }
}

// Initial states from a seed (a serving session's episode start, drawn where
// the state lives).  Random numbers: SplitMix64 (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014): output k of
// seed S mixes S + (k + 1) * 0x9E3779B97F4A7C15 through the variant-13
// finaliser, so each output is computed on its own; agent i takes outputs
// 4i, 4i + 1 and 4i + 2 (the fourth is unused), and a uniform in [0, 1) is
// the output's top 24 bits times 2^-24 (exact in FP32).  A thread per agent.
__device__ __forceinline__ unsigned long long splitmix64_out(unsigned long long seed,
                                                             unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float unit24(unsigned long long x) {
  return __uint2float_rn((unsigned)(x >> 40)) * 0x1p-24f;  // 24 bits: exact
}

__global__ void __launch_bounds__(256) k_seed_states(float4 *state, int n, float side,
                                                     float side_below, float two_pi,
                                                     float two_pi_below, float speed,
                                                     unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long k = 4ull * (unsigned long long)i;
  const float x = fminf(__fmul_rn(unit24(splitmix64_out(seed, k)), side), side_below);
  const float y = fminf(__fmul_rn(unit24(splitmix64_out(seed, k + 1)), side), side_below);
  const float th = fminf(__fmul_rn(unit24(splitmix64_out(seed, k + 2)), two_pi), two_pi_below);
  state[i] = make_float4(x, y, th, speed);
}

}  // namespace flock

using namespace flock;

extern "C" int flock_gae(int T, int n, const float *reward, const float *value, float gamma,
                         float lambda, float *adv, float *ret, void *stream) {
  flock::NvtxRange nvtx_range("flock:gae");
  if (T < 0 || n < 0) return FLOCK_EINVAL;
  if (!(gamma >= 0.0f && gamma <= 1.0f && lambda >= 0.0f && lambda <= 1.0f)) return FLOCK_EINVAL;
  if (T == 0 || n == 0) return FLOCK_OK;
  if (!reward || !value || !adv || !ret) return FLOCK_EINVAL;
  const float gl = gamma * lambda;
  const int blocks = (n + 31) / 32;
  k_gae<<<blocks, kGaeBlock, 0, (cudaStream_t)stream>>>(T, n, reward, value, gamma, gl, adv,
                                                        ret);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FLOCK_OK : cuda_fail(e, "k_gae launch");
}

extern "C" int flock_seed_states(float *state, int n, float side, float speed, uint64_t seed,
                                 void *stream) {
  NvtxRange nvtx_range("flock:seed_states");
  if (n < 0 || !(side > 0.0f) || !std::isfinite(side) || !std::isfinite(speed)) return FLOCK_EINVAL;
  if (n == 0) return FLOCK_OK;
  if (!state || (reinterpret_cast<uintptr_t>(state) & 15)) return FLOCK_EINVAL;
  const float two_pi = (float)(2.0 * 3.14159265358979323846);
  k_seed_states<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<float4 *>(state), n, side, std::nextafter(side, 0.0f), two_pi,
      std::nextafter(two_pi, 0.0f), speed, (unsigned long long)seed);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FLOCK_OK : cuda_fail(e, "k_seed_states launch");
}
