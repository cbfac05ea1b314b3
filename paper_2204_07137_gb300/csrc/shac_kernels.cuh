// Kernel launch arguments shared by the host code and the kernels.
#pragma once
#include "shac_device.cuh"

namespace shac {

constexpr int MAX_GROUPS = 8;

// Per-group addressing of the caller's structure-of-arrays buffers.
struct GroupIO {
  int N;                 // environments in the group
  int64_t q_off, qd_off, act_off, env_off;   // offsets of the group's block
};

struct IOArgs {
  int n_groups;
  GroupIO g[MAX_GROUPS];
  int64_t q_size, qd_size, act_size, n_envs;   // per-time-step strides
};

// Batched form: one work item = up to (32 / lanes) consecutive environments
// of one group, executed by one warp.
struct WorkItem {
  int group, env0, count;
};

struct BatchedArgs {
  const DevModel* models;   // [n_groups] device array
  int n_groups;
  IOArgs io;
  int lanes[MAX_GROUPS];    // lanes per environment (team size) per group
  int dense_nm[MAX_GROUPS]; // register row capacity of the dense path (0: shared-memory form)
  int smem_warp_floats;     // shared floats per warp
  int env_stride[MAX_GROUPS];   // padded env_floats per group (shared memory)
  const WorkItem* items;
  int n_items;
  int* counter;             // work counter (zeroed before each launch)
  float* tape;              // substep tape base (workspace)
  int64_t tape_off[MAX_GROUPS];   // per-group float offset; slot per env (N_g + 31 slots)
  // window tape: the forward keeps every step's substep records and post-step
  // state, the adjoint reads them instead of recomputing (0: recompute)
  int tape_window;
  int tape_hmax;                  // steps per environment slot
  int64_t tape_step[MAX_GROUPS];  // floats per step: K records + post-step q, qd
  unsigned int* flags;
  int h;
  // window / step buffers
  const float* q_in;        // start state (step input or q0)
  const float* qd_in;
  const float* act;         // [h][act_size]
  float* q_out;             // states after each step: [h][q_size] (t = 1..h)
  float* qd_out;
  float* reward;            // [h][n_envs]
  float* q_copy0;           // optional copy of the start state (trajectory entry 0)
  float* qd_copy0;
  // adjoint
  const float* q_traj;      // [h][q_size] states at the start of each step
  const float* qd_traj;
  const float* reward_bar;  // [h][n_envs]
  const float* qT_bar;       // cotangent of the final state
  const float* qdT_bar;
  const float* qtb;          // optional [h][q_size] cotangents of the checkpoints t = 0..h-1
  const float* qdtb;
  float* q0_bar;
  float* qd0_bar;
  float* act_bar;           // [h][act_size]
  // episodic window (early termination with reset); null / unused otherwise
  const float* q_reset;     // reset states, layout of q_in
  const float* qd_reset;
  float term_h[MAX_GROUPS]; // root-height threshold per group (-inf / NaN: none)
  int max_ep[MAX_GROUPS];   // episode length limit per group (<= 0: none)
  int* ep_step;             // [n_envs] steps since the last reset (in/out)
  unsigned char* done;      // forward: [h][n_envs] episode ended by step t
  const unsigned char* done_in;   // adjoint: the forward's done mask
  // key of the model-specialised kernels these arguments are for (0: the
  // generic kernels); a specialised kernel given another key does nothing but
  // raise FLAG_SPEC_MISMATCH
  unsigned int spec_key;
};

#ifndef __CUDACC_RTC__
void launch_batched_forward(const BatchedArgs& a, int grid, int block, size_t smem, cudaStream_t s);
void launch_batched_adjoint(const BatchedArgs& a, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t batched_occupancy(int* blocks_per_sm, int block, size_t smem, bool adjoint);
cudaError_t batched_set_smem_limit(size_t smem);

// Plain form: one environment per thread, one kernel per stage.
struct PlainGroup {
  DevModel M;
  int N;
  float* ws;        // scratch [env_floats][N]
  float* tape;      // [K * (nq + nv)][N]
};

enum PlainStage {
  PS_KIN = 0,       // root-first sweep: kinematics, inertias, subspaces, velocities, contact/muscle
                    // forces, Newton-Euler accelerations and local forces
  PS_BIAS,          // leaves-first sweep: total forces, composite inertias; right-hand side
  PS_CRBA,          // composite-rigid-body mass matrix rows
  PS_SOLVE,         // Cholesky factorisation and solve
  PS_INTEGRATE,     // semi-implicit Euler
  PS_ADJ_INTEGRATE, // integrator adjoint
  PS_ADJ_DYN        // dynamics adjoint (solve with the cached factor + inverse-dynamics VJP)
};
void launch_plain_stage(const PlainGroup& g, int stage, cudaStream_t s);
// state movement between the caller's buffers / tape and the scratch
void launch_plain_load(const PlainGroup& g, const float* q, const float* qd, const float* act, int64_t q_off,
                       int64_t qd_off, int64_t act_off, cudaStream_t s);
void launch_plain_store(const PlainGroup& g, float* q, float* qd, float* reward, int64_t q_off, int64_t qd_off,
                        int64_t env_off, unsigned int* flags, cudaStream_t s);
void launch_plain_tape(const PlainGroup& g, int k, bool save, cudaStream_t s);
// mode 1: set (QB, QDB) = (qb, qdb); mode 0: add (qb, qdb) if non-null
void launch_plain_adj_begin(const PlainGroup& g, const float* qb, const float* qdb, const float* rb, int64_t q_off,
                            int64_t qd_off, int64_t env_off, int mode, cudaStream_t s);
void launch_plain_adj_store_act(const PlainGroup& g, float* act_bar, int64_t act_off, cudaStream_t s);
// writes (QB + qb_add, QDB + qdb_add) (adds skipped when null)
void launch_plain_adj_store_state(const PlainGroup& g, float* qb, float* qdb, const float* qb_add,
                                  const float* qdb_add, int64_t q_off, int64_t qd_off, cudaStream_t s);
#endif

}  // namespace shac
