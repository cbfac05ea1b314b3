// The batched form's persistent kernels (one work item = 32 / T environments
// of one group on one warp, every stage of every substep of every step fused).
//
// This header is compiled twice: into the library by nvcc (the generic
// kernels, any model and launch shape read from the arguments), and at run
// time for one model and launch shape (shac_batch_specialize): the model's
// counts and scratch offsets, the team size, the dense row capacity and the
// scratch stride are then literals in the source, so the compiler folds the
// address arithmetic and the loop bounds they control.
#pragma once
#include "shac_kernels.cuh"

// Launch-shape values of a specialised build (the generic build reads them
// from the launch arguments).
#ifdef SHAC_SPEC_LANES
#define SHAC_TEAM_LANES(x) (SHAC_SPEC_LANES)
#define SHAC_DENSE_ROWS(x) (SHAC_SPEC_ROWS)
#define SHAC_ENV_STRIDE(x) (SHAC_SPEC_STRIDE)
#else
#define SHAC_TEAM_LANES(x) (x)
#define SHAC_DENSE_ROWS(x) (x)
#define SHAC_ENV_STRIDE(x) (x)
#endif

namespace shac {

// Register caps of the batched kernels (forward, adjoint): the live state of
// the chain carries and of the 32-row dense path fits without spills; the
// host launches at most 8 warps per CTA (8 x 32 x 216 registers fit an SM's
// 64 Ki, and two 4-warp CTAs stay resident per SM).
#define BATCHED_REGS_FORWARD 184
#define BATCHED_REGS_ADJOINT 216


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
  const int nl = SHAC_TEAM_LANES(a.lanes[it.group]);
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
  const int nm = SHAC_DENSE_ROWS(a.dense_nm[it.group]);
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
  const int nm = SHAC_DENSE_ROWS(a.dense_nm[it.group]);
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
#ifdef SHAC_SPEC_KEY
  // a specialised kernel runs only the batch and launch shape it was built for
  if (a.spec_key != SHAC_SPEC_KEY) {
    if (threadIdx.x == 0) atomicOr(a.flags, FLAG_SPEC_MISMATCH);
    return;
  }
#endif
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
    SMem w{wsm + (size_t)t.team * SHAC_ENV_STRIDE(a.env_stride[it.group])};
    if (ADJ) adjoint_item(a, M, it, w, t);
    else forward_item(a, M, it, w, t);
    __syncwarp();
  }
}

}  // namespace shac
