/*
 * shacsim.h -- C ABI of the GB300 parallel differentiable articulated-body
 * simulator: the batched step s_{t+1} = F(s_t, a_t) of many independent
 * environments and its reverse-mode adjoint (Short-Horizon Actor-Critic,
 * arXiv 2204.07137, Sec. 3.1 "GPU-Based Differentiable Dynamics Simulation",
 * Eq. backward and Eq. fwd_dynamics; appendix A.1 for the window recursion).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All floating point data is FP32.  Device arrays are structure-of-arrays
 *    per articulation group: a quantity with D components for a group of N_g
 *    environments occupies D*N_g floats laid out [D][N_g] (component-major,
 *    environment fastest).  Groups are concatenated in the order given to
 *    shac_batch_create.  Per-step trajectories stack these blocks over time:
 *    [t][sum_g D_g*N_g].
 *  - State s = (q, qd).  q holds joint coordinates (free root: position xyz
 *    then unit quaternion xyzw; revolute/prismatic: one coordinate), qd joint
 *    velocities (free root: body-frame angular velocity then body-frame
 *    velocity of the root origin).  Actions a: per-DOF torque commands
 *    (scaled by the model gear) followed by muscle activations.
 *  - Ownership: the caller owns every device buffer it passes, including the
 *    workspace (size from shac_batch_workspace_bytes).  The library owns only
 *    its handles and the device copies of the model constants, allocated once
 *    in shac_batch_create and freed in shac_batch_destroy.
 *  - step / window calls are asynchronous on the given CUDA stream (a
 *    cudaStream_t passed as void*; NULL = legacy default stream), perform no
 *    allocation, no host synchronisation and no host read-back, so they can
 *    be captured in CUDA graphs.  Arguments are validated on the host; an
 *    invalid argument returns an error status and launches nothing.
 *  - Device-side problems (a non-finite state produced by a step) set a
 *    sticky flag word read with shac_get_status.
 *  - *_bar outputs are overwritten (not accumulated).
 */
#ifndef SHACSIM_H
#define SHACSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SHAC_OK = 0,
  SHAC_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum */
  SHAC_ERR_MODEL = 2,         /* not a tree / parent after child / free joint not at a root / bad index */
  SHAC_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  SHAC_ERR_NONFINITE = 4,     /* sticky: a step produced a non-finite state */
  SHAC_ERR_CAPACITY = 5,      /* model exceeds a compiled limit (e.g. more than 32 DOF) */
  SHAC_ERR_UNSUPPORTED = 6    /* requested form/option not available */
} shac_status;

/* Joint types (Sec. 3.1: articulated rigid bodies in generalised coordinates) */
enum { SHAC_JOINT_FREE = 0, SHAC_JOINT_REVOLUTE = 1, SHAC_JOINT_PRISMATIC = 2, SHAC_JOINT_FIXED = 3 };

/* Execution forms */
enum {
  SHAC_FORM_PLAIN = 0,   /* one environment per thread, one kernel per stage per substep */
  SHAC_FORM_BATCHED = 1  /* lane teams per environment, every stage and substep fused in one
                            persistent launch per window (or per step) */
};

typedef struct shac_model shac_model;
typedef struct shac_batch shac_batch;

/*
 * Host-side description of one articulation (paper Sec. 3.1: a joint tree
 * with masses, inertias, contact shapes, joint limits and actuation).  The
 * library copies everything; the caller keeps ownership of its arrays.
 *
 *  n_links          links, numbered so that parent[i] < i (-1 = world).
 *  joint_type[L]    SHAC_JOINT_*; a FREE joint must be a root (parent -1) and
 *                   ignores joint_pos/joint_quat.
 *  joint_axis[L][3] unit axis in the joint frame (revolute/prismatic).
 *  joint_pos[L][3], joint_quat[L][4] (xyzw): joint frame in the parent link
 *                   frame.  The link frame coincides with the joint frame at
 *                   zero joint coordinate.
 *  mass[L], com[L][3], inertia[L][6] (xx yy zz xy xz yz about the COM, link frame).
 *  n_contacts, contact_link[C], contact_pos[C][3] (sphere centre, link frame),
 *                   contact_radius[C]: spheres against the ground plane z = 0.
 *  q_lower/q_upper[nv]: per-DOF joint limits (use +-1e30 for none; only
 *                   revolute/prismatic DOFs are limited), k_limit: stiffness.
 *  armature[nv], joint_damping[nv].
 *  n_tact, act_dof[n_tact], act_gear[n_tact]: torque actuator k drives DOF
 *                   act_dof[k] with torque act_gear[k] * a[k] (one actuator per DOF).
 *  n_muscles, muscle_ptr[n_muscles+1], via_link[V], via_pos[V][3] (link frame),
 *                   muscle_fmax[n_muscles]: muscle m pulls consecutive via
 *                   points together with force clamp(a, 0, 1) * fmax; its
 *                   activation is a[n_tact + m].
 *  dt: control step; substeps: K semi-implicit Euler substeps per step,
 *                   action held; gravity[3].
 *  ke, kd, kt, mu:  contact normal stiffness, damping, friction stiffness, friction coefficient.
 *  rw_q[nq], rw_qd[nv], reward_coef[10]: reward on the post-step state,
 *     r = -sum rw_q q^2 - sum rw_qd qd^2 - c0 |a|^2 + c1 vx + Rh(clip(z - c4, c5, c6))
 *         + (free root only) c2 up_z + c3 head_x,
 *     Rh(D) = c7 D^2 + c8 D (D < 0), c9 D (D >= 0).  With a free root, vx is
 *     the world x velocity of the root origin and z = q[2] its height; without
 *     one, vx = qd[vx_dof] and z = q[height_q] (a term whose index is -1 is
 *     dropped: planar models driven through slide joints along x and z).
 *  height_q, vx_dof: see the reward; height_q is also the root height of the
 *     episodic window's termination rule for models without a free root.
 *     Ignored for a free root.
 */
typedef struct {
  int32_t n_links;
  const int32_t* parent;
  const int32_t* joint_type;
  const float* joint_axis;
  const float* joint_pos;
  const float* joint_quat;
  const float* mass;
  const float* com;
  const float* inertia;
  int32_t n_contacts;
  const int32_t* contact_link;
  const float* contact_pos;
  const float* contact_radius;
  const float* q_lower;
  const float* q_upper;
  float k_limit;
  const float* armature;
  const float* joint_damping;
  int32_t n_tact;
  const int32_t* act_dof;
  const float* act_gear;
  int32_t n_muscles;
  const int32_t* muscle_ptr;
  const int32_t* via_link;
  const float* via_pos;
  const float* muscle_fmax;
  float dt;
  int32_t substeps;
  float gravity[3];
  float ke, kd, kt, mu;
  const float* rw_q;
  const float* rw_qd;
  float reward_coef[10];
  int32_t height_q;
  int32_t vx_dof;
} shac_model_desc;

/* Validate and copy a model description.  Returns SHAC_ERR_MODEL for a
 * malformed tree or index, SHAC_ERR_CAPACITY beyond the compiled limits
 * (64 links, 32 DOF, 64 contacts). */
shac_status shac_model_create(const shac_model_desc* desc, shac_model** out);
void shac_model_destroy(shac_model* model);
/* nq, nv, na of a model (any pointer may be NULL). */
void shac_model_dims(const shac_model* model, int32_t* nq, int32_t* nv, int32_t* na);

/* A batch of n_groups articulation groups (models[g] with n_envs[g] >= 0
 * environments each) executed in one form (Sec. 3.1: the simulator runs the
 * environments in parallel on the GPU, the dense routines and the contact and
 * joint forces of every environment at once).  Environments of a batch are
 * independent.  Uploads the model constants and the work-item table to the
 * current CUDA device, which the batch stays bound to (the one allocation
 * point).  window_h_max bounds the h accepted by the window calls.  Errors:
 * SHAC_ERR_INVALID_ARG (null pointers, n_groups outside 1..8, a negative
 * count, an unknown form, window_h_max < 1); SHAC_ERR_CUDA. */
shac_status shac_batch_create(const shac_model* const* models, const int32_t* n_envs, int32_t n_groups,
                              int32_t form, int32_t window_h_max, shac_batch** out);
void shac_batch_destroy(shac_batch* batch);
/* Totals over groups: sum nq_g N_g, sum nv_g N_g, sum na_g N_g, sum N_g. */
void shac_batch_dims(const shac_batch* batch, int64_t* q_size, int64_t* qd_size, int64_t* act_size,
                     int64_t* n_envs);
/* Bytes of caller-allocated device workspace the batch needs (the caller
 * passes a 256-byte aligned pointer to every step and window call).  It holds
 * the scratch of one control step for every environment: the per-substep
 * records that Sec. 3.1 keeps for the backward pass (link poses, inertias,
 * contact items, the Cholesky factor) and, with the window tape, those of
 * every step of a window.  0 for a null batch. */
size_t shac_batch_workspace_bytes(const shac_batch* batch);

/* One control step s_{t+1} = F(s_t, a_t) (Sec. 3.1): K substeps with the
 * action held, each solving Eq. fwd_dynamics for the joint accelerations (CRBA
 * mass matrix, Cholesky factorisation) and taking a semi-implicit Euler step;
 * then the reward on the post-step state.  q/qd/act: [q_size]/[qd_size]/
 * [act_size] device arrays; q_next/qd_next likewise; reward: [n_envs].
 * Inputs and outputs must not alias.  Errors: SHAC_ERR_INVALID_ARG (null
 * pointer, unaligned workspace), SHAC_ERR_CUDA (launch failure). */
shac_status shac_step(shac_batch* batch, void* stream, void* workspace,
                      const float* q, const float* qd, const float* act,
                      float* q_next, float* qd_next, float* reward);

/* Eq. backward for one step: given the step input (q, qd, act) and the
 * cotangents of its outputs (q_next_bar, qd_next_bar, reward_bar), write
 * q_bar = dL/dq, qd_bar = dL/dqd, act_bar = dL/dact.  Substeps are recomputed
 * from the input state. */
shac_status shac_step_adjoint(shac_batch* batch, void* stream, void* workspace,
                              const float* q, const float* qd, const float* act,
                              const float* q_next_bar, const float* qd_next_bar, const float* reward_bar,
                              float* q_bar, float* qd_bar, float* act_bar);

/* h steps: act [h][act_size]; q_traj/qd_traj [h+1][..] (entry 0 = q0/qd0 copy),
 * reward [h][n_envs].  The trajectory is the per-control-step checkpoint tape. */
shac_status shac_window_forward(shac_batch* batch, void* stream, void* workspace, int32_t h,
                                const float* q0, const float* qd0, const float* act,
                                float* q_traj, float* qd_traj, float* reward);

/* Appendix A.1 recursion (without the policy term): reverse over the h
 * steps of a window given its checkpoint tape (q_traj, qd_traj [h+1][..] from
 * shac_window_forward), the per-step reward cotangents reward_bar [h][n_envs]
 * and the cotangents of every checkpoint q_traj_bar/qd_traj_bar [h+1][..]
 * (entry h = final state; pass zeros where the loss does not read a
 * checkpoint directly).  Writes q0_bar/qd0_bar (total cotangent of the start
 * state, including entry 0) and act_bar [h][act_size].  Substeps of each step
 * are recomputed from its checkpoint. */
shac_status shac_window_adjoint(shac_batch* batch, void* stream, void* workspace, int32_t h,
                                const float* q_traj, const float* qd_traj, const float* act,
                                const float* reward_bar, const float* q_traj_bar, const float* qd_traj_bar,
                                float* q0_bar, float* qd0_bar, float* act_bar);

/* Episodic window: early termination with an in-kernel reset and the gradient
 * cut at the reset (Sec. 3.2: the environment is reset when the task terminates
 * early and no gradient crosses the reset; appendix A.3: a task terminates when
 * the root falls below a task height, or at the task horizon).  BATCHED form
 * only (SHAC_ERR_UNSUPPORTED for PLAIN).
 *
 * shac_window_forward_episodic does what shac_window_forward does and, after
 * every step t, for every environment:
 *   e <- e + 1   (e = steps since the environment's last reset)
 *   done_t = (root height < term_height[g]: q[2] for a free root, else
 *             q[height_q] when height_q >= 0)  or  (max_episode_steps[g] > 0 and e >= max_episode_steps[g])
 *   if done_t: state <- the environment's reset state, e <- 0.
 * reward[t] is the reward of step t before any reset; q_traj/qd_traj[t + 1]
 * hold the state after the reset (the state step t + 1 starts from).
 *   q_reset, qd_reset  reset states, same layout as q0/qd0 (device, read only).
 *   term_height        HOST array [n_groups], copied; -INFINITY or NaN: no
 *                      height rule for that group.
 *   max_episode_steps  HOST array [n_groups], copied: task horizon per group
 *                      in control steps; <= 0: none.
 *   episode_step       device int32 [n_envs] (groups concatenated): e, read at
 *                      the start of the window and written at its end.
 *   done               device uint8 [h][n_envs]: 1 where step t ended an
 *                      episode, else 0.
 * The discount restart at a reset (Sec. 3.2) belongs to the caller's loss: it
 * weights reward_bar with the done mask.
 *
 * shac_window_adjoint_episodic does what shac_window_adjoint does with the
 * done mask of the forward window: where done_t, the cotangent of the state
 * after step t (a reset state, a constant of the window), including
 * q_traj_bar[t + 1], is dropped before step t is reversed; step t's reward
 * cotangent still enters. */
shac_status shac_window_forward_episodic(shac_batch* batch, void* stream, void* workspace, int32_t h,
                                         const float* q0, const float* qd0, const float* act,
                                         const float* q_reset, const float* qd_reset,
                                         const float* term_height, const int32_t* max_episode_steps,
                                         int32_t* episode_step, float* q_traj, float* qd_traj, float* reward,
                                         uint8_t* done);
shac_status shac_window_adjoint_episodic(shac_batch* batch, void* stream, void* workspace, int32_t h,
                                         const float* q_traj, const float* qd_traj, const float* act,
                                         const uint8_t* done, const float* reward_bar,
                                         const float* q_traj_bar, const float* qd_traj_bar,
                                         float* q0_bar, float* qd0_bar, float* act_bar);

/* Step adjoint for callers that cannot allocate device memory when they call
 * the simulator (e.g. inside a CUDA graph capture that forbids allocation, or
 * runtimes that only pass pre-registered buffers).  The paper has no
 * counterpart: this is a deployment variant of shac_step_adjoint.
 *
 * Same arguments and results as shac_step_adjoint minus the workspace: the
 * scratch (work counter and substep records) lives in a 64 MiB device array
 * compiled into the library, resident on every GPU that loads it until the
 * process exits.  Nothing is allocated by the call.  A batch whose step-level
 * scratch exceeds 64 MiB is rejected with SHAC_ERR_CAPACITY: that is what
 * shac_batch_workspace_bytes reports with the window tape off (for the
 * ant-like model: up to about 1500 environments); the window tape's share is
 * never used by step calls, so turning the tape on does not change the limit.
 * The current device must be the one the batch was created on
 * (SHAC_ERR_INVALID_ARG otherwise, nothing launched).  The first call on a
 * device looks up the array's device address with that device current and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not use the library across a device reset.  Every
 * call on a device shares the one array, and it keeps the last call's
 * contents (the work counter is cleared by each call): calls that may overlap
 * on the GPU (different streams, or concurrent host threads) race on it and
 * must be serialised by the caller. */
shac_status shac_step_adjoint_static(shac_batch* batch, void* stream,
                                     const float* q, const float* qd, const float* act,
                                     const float* q_next_bar, const float* qd_next_bar, const float* reward_bar,
                                     float* q_bar, float* qd_bar, float* act_bar);

/* Batched-form launch shape: lanes per environment for group g (1,2,4,8,16,32;
 * 0 = automatic) and warps per CTA.  Does not change results beyond FP32
 * reassociation inside a team. */
shac_status shac_batch_set_launch(shac_batch* batch, int32_t group, int32_t lanes_per_env, int32_t warps_per_cta);
shac_status shac_batch_get_launch(const shac_batch* batch, int32_t group, int32_t* lanes_per_env,
                                  int32_t* warps_per_cta);

/* Measured choice of the batched launch shape (the environment-to-warp
 * packing per group and the CTA size; the paper has no counterpart: its
 * kernels are one thread per environment).  Coordinate descent: each group's
 * lanes per environment in turn (1, 2, 4, 8, 16, 32; the others fixed), then
 * the warps per CTA (1, 2, 4, 8); every candidate is timed as a window forward
 * + window adjoint of min(h_max, 8) steps with CUDA events on `stream` (one
 * warm-up, median of three).  The timed windows start from q0 [q_size] and
 * qd0 [qd_size] and apply act [min(h_max, 8)][act_size] (device pointers, the
 * layouts of the window calls; read once at the start), so the search sees the
 * caller's workload (its contacts and joint ranges); a null pointer takes the
 * rest configuration instead (joint coordinates 0, free joints at the origin
 * with the identity orientation, zero velocities, zero actions).  A candidate replaces the best shape so far only when it is more
 * than 3 % faster (timing noise between equal shapes stays below that); the
 * best shape is applied to the batch (as shac_batch_set_launch would) and
 * kept.  A batch using model-specialised kernels (shac_batch_specialize) keeps
 * its team size and searches the warps per CTA only, timed with those
 * kernels (they stay in use).  `workspace`: a caller buffer of
 * shac_autotune_workspace_bytes (256-byte aligned), overwritten: the batch's
 * workspace followed by the inputs and outputs of the timed windows; the call
 * allocates no device memory.  budget_ms: wall-clock limit of the search
 * (> 0; the best shape found so far is kept when it runs out).  Synchronises
 * the stream, so it must not be called during a stream capture.  A PLAIN
 * batch, or one with no environment, returns SHAC_OK unchanged.  Errors:
 * SHAC_ERR_INVALID_ARG for a null batch, an unaligned workspace or
 * budget_ms <= 0; SHAC_ERR_CUDA if a CUDA call fails (the launch shape is then
 * left as it was). */
shac_status shac_autotune(shac_batch* batch, void* stream, void* workspace, int32_t budget_ms, const float* q0,
                          const float* qd0, const float* act);
/* Bytes of the workspace shac_autotune needs (shac_batch_workspace_bytes plus
 * the timed windows' buffers). */
size_t shac_autotune_workspace_bytes(const shac_batch* batch);

/* Model-specialised batched kernels.  The paper generates its forward and
 * backward simulation kernels by source-code transformation (Sec. 3.1); here
 * run-time compilation serves another end: the library's own batched kernels
 * are compiled again with one model's counts, scratch offsets and link parents
 * and the current team size written into their source as constants, so that
 * the compiler folds the address arithmetic and the loop bounds they control
 * and unrolls the tree sums over the links.  enable = 1 builds the forward
 * and adjoint kernels for the batch's model and current launch shape with
 * NVRTC on the current device (which must be the batch's; a few seconds, once
 * per distinct model layout, tree and team size in a process) and makes every
 * batched step and window call of the batch use them while group 0 keeps that
 * team size (after shac_batch_set_launch or shac_autotune change it, the calls
 * use the generic kernels again until the next shac_batch_specialize);
 * enable = 0 returns to the generic kernels.  Results equal the generic
 * kernels' up to FP32 rounding (constant operands can change how the compiler
 * contracts multiply-adds).  BATCHED batches with one group only
 * (SHAC_ERR_UNSUPPORTED otherwise).  Synchronous; not for a stream capture.
 * Errors: SHAC_ERR_INVALID_ARG (null batch, enable not 0/1, another device
 * current); SHAC_ERR_CUDA if the run-time compiler or the module load fails. */
shac_status shac_batch_specialize(shac_batch* batch, int32_t enable);

/* Window tape (BATCHED form; SHAC_ERR_UNSUPPORTED for PLAIN): keep = 1 makes
 * shac_window_forward (and its episodic variant) store every substep record of
 * every step (link poses, inertias, subspaces, velocities, external wrenches,
 * contact items, Cholesky factor, accelerations) and each step's post-step state
 * in the workspace, and shac_window_adjoint (episodic too) read them back instead
 * of recomputing each step's substeps: the reverse pass skips one forward
 * recompute, at K * record + nq + nv floats per env-step of workspace (ant-like
 * model, h_max = 32, 2048 environments: 2.9 GB; shac_batch_workspace_bytes
 * reports the new size, reallocate after the call).  Contract: the adjoint
 * window must follow the forward window on the same workspace with the same h,
 * q_traj/qd_traj, act (and done mask), with no other window call in between; it
 * then returns what the recomputing adjoint returns, bit for bit.  Step-level
 * calls (shac_step, shac_step_adjoint, shac_step_adjoint_static) never use the
 * tape.  keep = 0 (the default) recomputes.  (Sec. 3.1 keeps each substep's
 * Cholesky factor for the backward pass; the tape keeps every intermediate.) */
shac_status shac_batch_set_window_tape(shac_batch* batch, int32_t keep);

/* Critic value targets of the learner (Sec. 3.2, Eq. td-lambda): for every
 * environment and t = 0..h-1 the TD-lambda average of the k-step returns
 * G_t^k = sum_{l<k} gamma^l r_{t+l} + gamma^k V(s_{t+k}) over the window,
 *   target_t = (1 - lambda) sum_{k=1}^{h-t-1} lambda^{k-1} G_t^k + lambda^{h-t-1} G_t^{h-t}.
 * Where done_t is set (the episode ended at step t, as written by
 * shac_window_forward_episodic) the returns of the states up to t stop at step
 * t with no bootstrap.  Layout [t][n_envs] (environment fastest), device
 * pointers: reward [h][N], value [h+1][N] (V of the window's states, entry h the
 * final state), done [h][N] uint8 or NULL (no episode ends), target [h][N]
 * (written).  Asynchronous on the stream; no allocation.  INVALID_ARG for
 * null pointers, h < 1, n_envs < 0, gamma or lambda outside [0, 1]. */
shac_status shac_td_lambda(void* stream, int32_t h, int64_t n_envs, const float* reward, const float* value,
                           const uint8_t* done, float gamma, float lambda, float* target);

/* Synchronises the stream and returns the sticky device flags
 * (bit 0: non-finite state); clear != 0 resets them.  Not capturable. */
shac_status shac_get_status(shac_batch* batch, void* stream, uint32_t* sticky_flags, int32_t clear);

const char* shac_status_string(shac_status status);

#ifdef __cplusplus
}
#endif
#endif /* SHACSIM_H */
