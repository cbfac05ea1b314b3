// Critic value targets of the short-horizon actor-critic learner (FP32, sm_103a).
//
// TD-lambda targets (Sec. 3.2, Eq. td-lambda): for the states s_t of a window
// (t = 0..h-1) the exponentially weighted average of the k-step returns
//   G_t^k = sum_{l<k} gamma^l r_{t+l} + gamma^k V(s_{t+k}),
//   target_t = (1 - lambda) sum_{k=1}^{H-1} lambda^{k-1} G_t^k + lambda^{H-1} G_t^H,
// H = h - t.  Summing the geometric weights backwards in time gives the same
// value in one pass per environment:
//   target_{h-1} = r_{h-1} + gamma V(s_h),
//   target_t     = r_t + gamma ((1 - lambda) V(s_{t+1}) + lambda target_{t+1}).
// An environment whose episode ended at step t (done_t: its state after step t
// is terminal and was replaced by a reset state) takes no return beyond step t:
// target_t = r_t, and the states before it look no further (the states after
// it start a new episode with their own returns).
//
// Memory-bound and tiny: one thread per environment walks its column of the
// [h][N] arrays backwards; consecutive threads read consecutive environments
// (coalesced).
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/shacsim.h"

namespace shac {

__global__ void k_td_lambda(int h, int64_t n, const float* __restrict__ reward, const float* __restrict__ value,
                            const unsigned char* __restrict__ done, float gamma, float lambda,
                            float* __restrict__ target) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  float v_next = value[(int64_t)h * n + e];   // V(s_{t+1})
  float g_next = v_next;                        // target_{t+1} (at t = h-1 the bootstrap V(s_h))
  for (int t = h - 1; t >= 0; --t) {
    const int64_t i = (int64_t)t * n + e;
    const bool end = done != nullptr && done[i] != 0;
    const float g = reward[i] + (end ? 0.f : gamma * ((1.f - lambda) * v_next + lambda * g_next));
    target[i] = g;
    v_next = value[i];
    g_next = g;
  }
}

}  // namespace shac

extern "C" shac_status shac_td_lambda(void* stream, int32_t h, int64_t n_envs, const float* reward, const float* value,
                                      const uint8_t* done, float gamma, float lambda, float* target) {
  if (h < 1 || n_envs < 0 || !reward || !value || !target || !(gamma >= 0.f && gamma <= 1.f) ||
      !(lambda >= 0.f && lambda <= 1.f))
    return SHAC_ERR_INVALID_ARG;
  if (n_envs == 0) return SHAC_OK;
  const int block = 256;
  const int64_t grid = (n_envs + block - 1) / block;
  shac::k_td_lambda<<<(unsigned)grid, block, 0, (cudaStream_t)stream>>>(h, n_envs, reward, value, done, gamma, lambda,
                                                                         target);
  return cudaGetLastError() == cudaSuccess ? SHAC_OK : SHAC_ERR_CUDA;
}
