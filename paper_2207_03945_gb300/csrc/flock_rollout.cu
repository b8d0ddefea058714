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
