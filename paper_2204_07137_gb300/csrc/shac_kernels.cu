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

// Register caps of the batched kernels (forward, adjoint): the live state of
// the chain carries and of the 32-row dense path fits without spills; the
// host launches at most 8 warps per CTA (8 x 32 x 208 registers fit an SM's
// 64 Ki).
#define BATCHED_REGS_FORWARD 184
#define BATCHED_REGS_ADJOINT 208

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

struct Team {
  int lane, nl, team, env, active;
};

// Copy a [dim][N] block slice for one environment into scratch (team lanes).
__device__ __forceinline__ void team_load(const SMem& w, int o, const float* src, int dim, int N, int e, int lane,
                                          int nl) {
  for (int j = lane; j < dim; j += nl) w[o + j] = __ldg(src + (size_t)j * N + e);
}
__device__ __forceinline__ void team_store(const SMem& w, int o, float* dst, int dim, int N, int e, int lane, int nl,
                                           bool active) {
  if (!active) return;
  for (int j = lane; j < dim; j += nl) dst[(size_t)j * N + e] = w[o + j];
}

__device__ __forceinline__ bool next_item(const BatchedArgs& a, int& item) {
  int v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(a.counter, 1);
  item = __shfl_sync(0xffffffffu, v, 0);
  return item < a.n_items;
}

__device__ __forceinline__ void setup_team(const BatchedArgs& a, const WorkItem& it, Team& t) {
  const int nl = a.lanes[it.group];
  const int lane32 = threadIdx.x & 31;
  t.nl = nl;
  t.lane = lane32 % nl;
  t.team = lane32 / nl;
  t.active = t.team < it.count;
  t.env = it.env0 + (t.active ? t.team : 0);
}

// Copy a substep record (n floats, a multiple of 4) between an environment's
// scratch and its slot in the workspace, 16 bytes per access (both sides are
// 16-byte aligned: the scratch stride and the record length are multiples of 4
// floats, the dynamic shared memory and the workspace slots 16-byte aligned).
__device__ __forceinline__ void record_save(float* dst, const SMem& w, int n, int lane, int nl) {
  float4* d4 = reinterpret_cast<float4*>(dst);
  const float4* s4 = reinterpret_cast<const float4*>(&w[0]);
  for (int j = lane; j < n / 4; j += nl) d4[j] = s4[j];
}

// One work item of the forward window (all steps, all substeps).
__device__ __forceinline__ void forward_item(const BatchedArgs& a, const DevModel& M, const WorkItem& it,
                                             const SMem& w, const Team& t) {
  const int nm = a.dense_nm[it.group];
  const GroupIO& io = a.io.g[it.group];
  team_load(w, M.o_Q, a.q_in + io.q_off, M.nq, io.N, t.env, t.lane, t.nl);
  team_load(w, M.o_QD, a.qd_in + io.qd_off, M.nv, io.N, t.env, t.lane, t.nl);
  if (a.q_copy0) {
    team_store(w, M.o_Q, a.q_copy0 + io.q_off, M.nq, io.N, t.env, t.lane, t.nl, t.active);
    team_store(w, M.o_QD, a.qd_copy0 + io.qd_off, M.nv, io.N, t.env, t.lane, t.nl, t.active);
  }
  int ep = 0;   // episodic window: steps since the last reset (team lane 0)
  if (a.done && t.lane == 0) ep = a.ep_step[io.env_off + t.env];
  const int REC = M.rec_floats;
  float* wtape = a.tape_window ? a.tape + a.tape_off[it.group] +
                                     (size_t)(it.env0 + t.team) * a.tape_hmax * a.tape_step[it.group]
                               : nullptr;
  for (int step = 0; step < a.h; ++step) {
    team_load(w, M.o_ACT, a.act + (size_t)step * a.io.act_size + io.act_off, M.na, io.N, t.env, t.lane, t.nl);
    clear_comp(M, w, t.lane, t.nl);
    team_sync(t.nl);
    float* wt = wtape ? wtape + (size_t)step * a.tape_step[it.group] : nullptr;
    for (int k = 0; k < M.K; ++k) {
      substep_dynamics(M, w, t.lane, t.nl, nm);
      if (wt) {   // keep the substep record for the adjoint
        record_save(wt + (size_t)k * REC, w, REC, t.lane, t.nl);
        team_sync(t.nl);
      }
      st_integrate(M, w, t.lane, t.nl);
    }
    if (wt) {     // post-step state (before any reset): the reward adjoint's input
      float* post = wt + (size_t)M.K * REC;
      for (int j = t.lane; j < M.nq; j += t.nl) post[j] = w[M.o_Q + j];
      for (int j = t.lane; j < M.nv; j += t.nl) post[M.nq + j] = w[M.o_QD + j];
    }
    if (t.lane == 0 && t.active) {
      a.reward[(size_t)step * a.io.n_envs + io.env_off + t.env] = reward_value(M, w);
      if (!state_finite(M, w)) atomicOr(a.flags, FLAG_NONFINITE);
    }
    if (a.done) {   // early termination (root below the task height, or the episode length) and reset
      team_sync(t.nl);
      int d = 0;
      if (t.lane == 0) {
        ++ep;
        d = ((M.height_q >= 0 && w[M.o_Q + M.height_q] < a.term_h[it.group]) || (a.max_ep[it.group] > 0 && ep >= a.max_ep[it.group])) ? 1 : 0;
        if (d) ep = 0;
        if (t.active) a.done[(size_t)step * a.io.n_envs + io.env_off + t.env] = (unsigned char)d;
      }
      d = __shfl_sync(0xffffffffu, d, 0, t.nl);
      if (d) {
        team_load(w, M.o_Q, a.q_reset + io.q_off, M.nq, io.N, t.env, t.lane, t.nl);
        team_load(w, M.o_QD, a.qd_reset + io.qd_off, M.nv, io.N, t.env, t.lane, t.nl);
      }
      team_sync(t.nl);
    }
    team_store(w, M.o_Q, a.q_out + (size_t)step * a.io.q_size + io.q_off, M.nq, io.N, t.env, t.lane, t.nl, t.active);
    team_store(w, M.o_QD, a.qd_out + (size_t)step * a.io.qd_size + io.qd_off, M.nv, io.N, t.env, t.lane, t.nl,
               t.active);
    team_sync(t.nl);
  }
  if (a.done && t.lane == 0 && t.active) a.ep_step[io.env_off + t.env] = ep;
}

// Reload a substep record (global -> shared) with asynchronous copies, all in
// flight together, then wait for this lane's copies (the caller's team barrier
// makes them visible to the team).
__device__ __forceinline__ void record_load(const SMem& w, const float* src, int n, int lane, int nl) {
  for (int j = lane; j < n / 4; j += nl) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(&w[4 * j]);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + 4 * j) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// One work item of the window adjoint (reverse over steps).  Each step's
// substeps are recomputed once from its checkpoint; every substep's record
// (start state and forward intermediates, scratch [0, rec_floats)) is kept in
// the workspace and reloaded by the reverse pass.  With the window tape the
// forward window already kept every record (and the post-step state), and the
// recompute is skipped.
__device__ __forceinline__ void adjoint_item(const BatchedArgs& a, const DevModel& M, const WorkItem& it,
                                             const SMem& w, const Team& t) {
  const int nm = a.dense_nm[it.group];
  const GroupIO& io = a.io.g[it.group];
  const int REC = M.rec_floats;
  float* tape = a.tape + a.tape_off[it.group] + (size_t)(it.env0 + t.team) * ((size_t)M.K * REC);
  team_load(w, M.o_QB, a.qT_bar + io.q_off, M.nq, io.N, t.env, t.lane, t.nl);
  team_load(w, M.o_QDB, a.qdT_bar + io.qd_off, M.nv, io.N, t.env, t.lane, t.nl);
  for (int step = a.h - 1; step >= 0; --step) {
    team_load(w, M.o_Q, a.q_traj + (size_t)step * a.io.q_size + io.q_off, M.nq, io.N, t.env, t.lane, t.nl);
    team_load(w, M.o_QD, a.qd_traj + (size_t)step * a.io.qd_size + io.qd_off, M.nv, io.N, t.env, t.lane, t.nl);
    team_load(w, M.o_ACT, a.act + (size_t)step * a.io.act_size + io.act_off, M.na, io.N, t.env, t.lane, t.nl);
    zero_range(w, M.o_ACTB, M.na, t.lane, t.nl);
    if (a.done_in && a.done_in[(size_t)step * a.io.n_envs + io.env_off + t.env]) {
      // the state after this step was a reset state: no gradient crosses the reset
      zero_range(w, M.o_QB, M.nq, t.lane, t.nl);
      zero_range(w, M.o_QDB, M.nv, t.lane, t.nl);
    }
    clear_comp(M, w, t.lane, t.nl);
    team_sync(t.nl);
    const float* recs = tape;   // this step's substep records
    if (a.tape_window) {        // kept by the forward window: the post-step state is read back
      recs = a.tape + a.tape_off[it.group] +
             ((size_t)(it.env0 + t.team) * a.tape_hmax + step) * a.tape_step[it.group];
      const float* post = recs + (size_t)M.K * REC;
      for (int j = t.lane; j < M.nq; j += t.nl) w[M.o_Q + j] = post[j];
      for (int j = t.lane; j < M.nv; j += t.nl) w[M.o_QD + j] = post[M.nq + j];
      team_sync(t.nl);
    } else {                    // recomputed once from the checkpoint
      for (int k = 0; k < M.K; ++k) {
        substep_dynamics(M, w, t.lane, t.nl, nm);
        record_save(tape + (size_t)k * REC, w, REC, t.lane, t.nl);
        team_sync(t.nl);
        st_integrate(M, w, t.lane, t.nl);
      }
    }
    if (t.lane == 0) reward_adjoint(M, w, a.reward_bar[(size_t)step * a.io.n_envs + io.env_off + t.env]);
    team_sync(t.nl);
    for (int k = M.K - 1; k >= 0; --k) {
      record_load(w, recs + (size_t)k * REC, REC, t.lane, t.nl);
      team_sync(t.nl);
      st_integrate_adj(M, w, t.lane, t.nl);
      st_dynamics_adj(M, w, t.lane, t.nl, nm);
    }
    team_store(w, M.o_ACTB, a.act_bar + (size_t)step * a.io.act_size + io.act_off, M.na, io.N, t.env, t.lane, t.nl,
               t.active);
    if (a.qtb) {   // cotangent read directly from checkpoint `step`
      const float* qa = a.qtb + (size_t)step * a.io.q_size + io.q_off;
      const float* qda = a.qdtb + (size_t)step * a.io.qd_size + io.qd_off;
      for (int j = t.lane; j < M.nq; j += t.nl) w[M.o_QB + j] += __ldg(qa + (size_t)j * io.N + t.env);
      for (int j = t.lane; j < M.nv; j += t.nl) w[M.o_QDB + j] += __ldg(qda + (size_t)j * io.N + t.env);
    }
    team_sync(t.nl);
  }
  team_store(w, M.o_QB, a.q0_bar + io.q_off, M.nq, io.N, t.env, t.lane, t.nl, t.active);
  team_store(w, M.o_QDB, a.qd0_bar + io.qd_off, M.nv, io.N, t.env, t.lane, t.nl, t.active);
}

// Persistent kernels: warps pull work items (the dense path's register
// capacity of each group is dispatched inside the substep).  Everything a
// kernel runs is inlined into it (forward_item, adjoint_item, the substep
// and its adjoint are forced inline): inside one body the compiler sees that
// the scratch (dynamic shared memory) and the model table (s_models) are
// different arrays, so model fields are not reloaded after every scratch
// store, and no call boundary splits the register allocation (measured on
// the ant-like 2048-environment window: forward 5.99 -> 5.36 ms).
template <bool ADJ>
__global__ void __maxnreg__(ADJ ? BATCHED_REGS_ADJOINT : BATCHED_REGS_FORWARD) k_batched(BatchedArgs a) {
  extern __shared__ __align__(16) float smem[];
  __shared__ DevModel s_models[MAX_GROUPS];
  for (int g = threadIdx.x; g < a.n_groups; g += blockDim.x) s_models[g] = a.models[g];
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  float* wsm = smem + (size_t)warp * a.smem_warp_floats;
  int item_idx;
  while (next_item(a, item_idx)) {
    const WorkItem it = a.items[item_idx];
    const DevModel& M = s_models[it.group];
    Team t;
    setup_team(a, it, t);
    SMem w{wsm + (size_t)t.team * a.env_stride[it.group]};
    if (ADJ) adjoint_item(a, M, it, w, t);
    else forward_item(a, M, it, w, t);
    __syncwarp();
  }
}
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
