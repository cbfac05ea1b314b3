// Kernels of the two execution forms.
//
// PLAIN   one environment per thread; each stage of a substep is its own
//         kernel and all per-environment intermediates live in global
//         scratch laid out [component][N] (coalesced across threads).
// BATCHED a persistent kernel; each warp takes work items from an atomic
//         counter (items are pre-sorted by cost, largest first) and runs
//         32 / T environments in teams of T lanes, every stage of every
//         substep of every step fused, with the per-environment scratch in
//         shared memory.  One launch covers a whole window (or one step).
#include "shac_kernels.cuh"

namespace shac {

// ------------------------------------------------------------------ PLAIN --

__global__ void k_plain_stage(PlainGroup g, int stage) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const DevModel& M = g.M;
  GMem w{g.ws + e, g.N};
  switch (stage) {
    case PS_KIN:
      sw_forward(M, w, 0, 1);
      break;
    case PS_BIAS:
      sw_gather(M, w, 0, 1); st_rhs(M, w, 0, 1);
      break;
    case PS_CRBA:
      st_mass_rows(M, w, 0, 1);
      break;
    case PS_SOLVE:
      st_chol(M, w, 0, 1); st_solve(M, w, 0, 1, M.o_B, M.o_QDD);
      break;
    case PS_INTEGRATE:
      st_integrate(M, w, 0, 1);
      break;
    case PS_ADJ_INTEGRATE:
      st_integrate_adj(M, w, 0, 1);
      break;
    case PS_ADJ_DYN:
      st_dynamics_adj(M, w, 0, 1, 0);
      break;
    default:
      break;
  }
}

__global__ void k_plain_load(PlainGroup g, const float* __restrict__ q, const float* __restrict__ qd,
                             const float* __restrict__ act) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const DevModel& M = g.M;
  GMem w{g.ws + e, g.N};
  if (q) for (int j = 0; j < M.nq; ++j) w[M.o_Q + j] = q[(size_t)j * g.N + e];
  if (qd) for (int j = 0; j < M.nv; ++j) w[M.o_QD + j] = qd[(size_t)j * g.N + e];
  if (act) {   // every step starts by loading its action: clear the integration compensation
    for (int j = 0; j < M.na; ++j) w[M.o_ACT + j] = act[(size_t)j * g.N + e];
    clear_comp(M, w, 0, 1);
  }
}

__global__ void k_plain_store(PlainGroup g, float* __restrict__ q, float* __restrict__ qd, float* __restrict__ rew,
                              unsigned int* flags) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const DevModel& M = g.M;
  GMem w{g.ws + e, g.N};
  for (int j = 0; j < M.nq; ++j) q[(size_t)j * g.N + e] = w[M.o_Q + j];
  for (int j = 0; j < M.nv; ++j) qd[(size_t)j * g.N + e] = w[M.o_QD + j];
  rew[e] = reward_value(M, w);
  if (!state_finite(M, w)) atomicOr(flags, FLAG_NONFINITE);
}

__global__ void k_plain_tape(PlainGroup g, int k, int save) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const DevModel& M = g.M;
  GMem w{g.ws + e, g.N};
  const int S = M.nq + M.nv;
  float* t = g.tape + (size_t)k * S * g.N + e;
  if (save) {
    for (int j = 0; j < M.nq; ++j) t[(size_t)j * g.N] = w[M.o_Q + j];
    for (int j = 0; j < M.nv; ++j) t[(size_t)(M.nq + j) * g.N] = w[M.o_QD + j];
  } else {
    for (int j = 0; j < M.nq; ++j) w[M.o_Q + j] = t[(size_t)j * g.N];
    for (int j = 0; j < M.nv; ++j) w[M.o_QD + j] = t[(size_t)(M.nq + j) * g.N];
  }
}

// Start of a step's reverse pass: o_Q/o_QD hold the post-step state; load the
// incoming cotangents (if load_bar), clear the action cotangent, add the reward adjoint.
__global__ void k_plain_adj_begin(PlainGroup g, const float* __restrict__ qb, const float* __restrict__ qdb,
                                  const float* __restrict__ rb, int mode) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const DevModel& M = g.M;
  GMem w{g.ws + e, g.N};
  if (mode == 1) {
    for (int j = 0; j < M.nq; ++j) w[M.o_QB + j] = qb[(size_t)j * g.N + e];
    for (int j = 0; j < M.nv; ++j) w[M.o_QDB + j] = qdb[(size_t)j * g.N + e];
  } else if (qb) {
    for (int j = 0; j < M.nq; ++j) w[M.o_QB + j] += qb[(size_t)j * g.N + e];
    for (int j = 0; j < M.nv; ++j) w[M.o_QDB + j] += qdb[(size_t)j * g.N + e];
  }
  for (int j = 0; j < M.na; ++j) w[M.o_ACTB + j] = 0.f;
  reward_adjoint(M, w, rb[e]);
}

__global__ void k_plain_adj_store_act(PlainGroup g, float* __restrict__ ab) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const DevModel& M = g.M;
  GMem w{g.ws + e, g.N};
  for (int j = 0; j < M.na; ++j) ab[(size_t)j * g.N + e] = w[M.o_ACTB + j];
}

__global__ void k_plain_adj_store_state(PlainGroup g, float* __restrict__ qb, float* __restrict__ qdb,
                                        const float* __restrict__ qba, const float* __restrict__ qdba) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const DevModel& M = g.M;
  GMem w{g.ws + e, g.N};
  for (int j = 0; j < M.nq; ++j) qb[(size_t)j * g.N + e] = w[M.o_QB + j] + (qba ? qba[(size_t)j * g.N + e] : 0.f);
  for (int j = 0; j < M.nv; ++j) qdb[(size_t)j * g.N + e] = w[M.o_QDB + j] + (qdba ? qdba[(size_t)j * g.N + e] : 0.f);
}

static inline dim3 plain_grid(int N) { return dim3((N + 63) / 64); }

void launch_plain_stage(const PlainGroup& g, int stage, cudaStream_t s) {
  k_plain_stage<<<plain_grid(g.N), 64, 0, s>>>(g, stage);
}
void launch_plain_load(const PlainGroup& g, const float* q, const float* qd, const float* act, int64_t q_off,
                       int64_t qd_off, int64_t act_off, cudaStream_t s) {
  k_plain_load<<<plain_grid(g.N), 64, 0, s>>>(g, q ? q + q_off : nullptr, qd ? qd + qd_off : nullptr,
                                               act ? act + act_off : nullptr);
}
void launch_plain_store(const PlainGroup& g, float* q, float* qd, float* reward, int64_t q_off, int64_t qd_off,
                        int64_t env_off, unsigned int* flags, cudaStream_t s) {
  k_plain_store<<<plain_grid(g.N), 64, 0, s>>>(g, q + q_off, qd + qd_off, reward + env_off, flags);
}
void launch_plain_tape(const PlainGroup& g, int k, bool save, cudaStream_t s) {
  k_plain_tape<<<plain_grid(g.N), 64, 0, s>>>(g, k, save ? 1 : 0);
}
void launch_plain_adj_begin(const PlainGroup& g, const float* qb, const float* qdb, const float* rb, int64_t q_off,
                            int64_t qd_off, int64_t env_off, int mode, cudaStream_t s) {
  k_plain_adj_begin<<<plain_grid(g.N), 64, 0, s>>>(g, qb ? qb + q_off : nullptr, qdb ? qdb + qd_off : nullptr,
                                                    rb + env_off, mode);
}
void launch_plain_adj_store_act(const PlainGroup& g, float* act_bar, int64_t act_off, cudaStream_t s) {
  k_plain_adj_store_act<<<plain_grid(g.N), 64, 0, s>>>(g, act_bar + act_off);
}
void launch_plain_adj_store_state(const PlainGroup& g, float* qb, float* qdb, const float* qb_add,
                                  const float* qdb_add, int64_t q_off, int64_t qd_off, cudaStream_t s) {
  k_plain_adj_store_state<<<plain_grid(g.N), 64, 0, s>>>(g, qb + q_off, qdb + qd_off, qb_add ? qb_add + q_off : nullptr,
                                                          qdb_add ? qdb_add + qd_off : nullptr);
}

// ---------------------------------------------------------------- BATCHED --
}  // namespace shac

#include "shac_batched.cuh"

namespace shac {

#define k_batched_forward k_batched<false>
#define k_batched_adjoint k_batched<true>

void launch_batched_forward(const BatchedArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
  k_batched_forward<<<grid, block, smem, s>>>(a);
}
void launch_batched_adjoint(const BatchedArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
  k_batched_adjoint<<<grid, block, smem, s>>>(a);
}
cudaError_t batched_set_smem_limit(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_batched_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_batched_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
cudaError_t batched_occupancy(int* blocks_per_sm, int block, size_t smem, bool adjoint) {
  if (adjoint) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batched_adjoint, block, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batched_forward, block, smem);
}

}  // namespace shac
