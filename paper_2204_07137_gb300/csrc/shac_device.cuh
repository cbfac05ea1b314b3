// Per-environment simulator stages and their adjoints (FP32, sm_103a).
//
// The simulator step F (paper Sec. 3.1) is evaluated with spatial (6-D)
// vectors expressed in world-aligned coordinates about one reference point
// (Plücker coordinates, angular part first): the world origin for a model
// without a free root, the free root's origin otherwise (the dynamics are
// translation invariant; the contact depth adds the root height back).  With
// that choice the motion subspaces, spatial inertias and forces of all links
// live in one frame, so the composite-rigid-body mass matrix needs no frame
// transforms and the Newton-Euler recursion is a plain sum along the tree.
//
//   forward dynamics (Eq. fwd_dynamics):  (M + diag(armature)) qdd = tau_j - C(q, qd)
//   C = ID(q, qd, 0) with gravity as a base acceleration and the external
//       contact / muscle wrenches subtracted (the J^T f and c terms);
//   M  by CRBA: M_ab = S_b . (Ic_i S_a), i = link of DOF a, b in i or ancestors;
//   Cholesky M = L L^T (cached per substep for the backward pass, Sec. 3.1);
//   semi-implicit Euler integration.
//
// Adjoint of one substep (Eq. backward): reverse the integrator to obtain the
// cotangent of qdd, then use G(q, qd, qdd, a) = ID(q, qd, qdd) + arm*qdd -
// tau_j = 0 at the solution: with lambda = M^{-1} qdd_bar (one solve with the
// cached factor), (q_bar, qd_bar, a_bar) += -lambda^T dG/d(q, qd, a),
// a single reverse sweep of the Newton-Euler recursion (inverse-dynamics
// derivative) plus the contact, muscle, limit and actuation terms.
//
// Every stage is written for a "team" of nl lanes working on one
// environment: loops stride by nl and team_sync() separates dependent
// phases.  With nl = 1 (one environment per thread, PLAIN form) the loops are
// the serial algorithm, team_sync() is a no-op and the tree recursions are
// chain walks with register carries; the BATCHED form runs teams of 1..32
// lanes inside a warp on shared-memory scratch, where a team of two or more
// lanes computes the tree recursions as per-lane tree sums (one component per
// lane, links in a fixed order) and the world poses by rows.  Each phase
// writes any given scratch slot from exactly one lane and every sum runs in a
// fixed order, so a team's results do not depend on its size beyond the
// dense stage (the register path needs nl >= nv, narrower teams use the
// shared-memory stages) and the muscle wrenches (summed in as many partial
// sums per link as the team has lanes per link); they differ from one
// thread's chain walks by the reassociation of those sums.
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#else
// compiled at run time (a model-specialised build of the batched kernels):
// no host headers
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef int int32_t;
typedef unsigned int uint32_t;
#endif

namespace shac {

// Compile-time integer sequences (the dense path expands its column loops
// through them).
template <int... I> struct iseq {};
template <int N, int... I> struct make_iseq_t : make_iseq_t<N - 1, N - 1, I...> {};
template <int... I> struct make_iseq_t<0, I...> { using type = iseq<I...>; };
template <int N> using make_iseq = typename make_iseq_t<N>::type;

enum { J_FREE = 0, J_REV = 1, J_PRIS = 2, J_FIXED = 3 };
enum { FLAG_NONFINITE = 1u, FLAG_SPEC_MISMATCH = 2u };

constexpr int MAX_LINKS = 64;
constexpr int MAX_DOF = 32;
constexpr int MAX_CONTACTS = 64;

// Device-resident description of one articulation group.  All pointers point
// into one device blob owned by the batch.
struct DevModel {
  int L, nq, nv, na, ntact, nc, nm, nseg, nitems, K, nlev;
  float h;                               // substep length dt / K
  float grav[3], ke, kd, kt, mu, klim;
  float rc[10];
  int root_free;                         // link 0 is a free joint
  int height_q, vx_dof;                  // root height / forward velocity coordinates (q[2] / world vx with a free root)
  // links
  const int *parent, *jtype, *qs, *ds, *nd;
  const int *lvl_ptr, *lvl_link;         // chain heads grouped by chain depth
  const int *chain_tail;                 // last link of the chain starting at a head
  const int *ch_ptr, *ch_idx;            // children lists
  const int *lc_ptr, *lc_idx;            // contact items attached to each link
  const int *lm_ptr, *lm_idx;            // muscle via-point items attached to each link
  const float *axis, *jpos, *jrot, *mass, *com, *icom;
  // dofs
  const int *dof_link, *dof_k, *dof_act;
  const unsigned *anc_mask;              // per DOF a: bit b set when DOF b <= a moves an ancestor-or-self link of a
  const float *qlo, *qhi, *arm, *damp, *gear;
  // force items: contacts [0, nc) then muscle segment ends [nc, nc + 2 nseg)
  const int *item_link;
  const float *item_pos, *crad;
  const int *seg_mus, *mus_seg_ptr;
  const float *fmax;
  // reward weights
  const float *rwq, *rwqd;
  // per-environment scratch layout (float offsets)
  int o_Q, o_QD, o_ACT, o_QB, o_QDB, o_ACTB;
  int o_LR, o_LW;                        // per-link records: LREC floats each (in the substep record), LWORK (work)
  int o_S, o_IT, o_M, o_LD, o_B, o_T, o_QDD;
  int o_QC, o_QDC;                       // compensation (low parts) of q, qd within a step
  int o_LAM, o_ITB, o_SEGA, o_MW, o_RDB;
  int rec_floats;       // floats of the substep record: scratch [0, rec_floats) (o_Q first)
  int env_floats;
};

// Per-link scratch: two records per link with fields at fixed offsets, so a
// pass over link i computes one base address per record.  The record part is
// inside the substep record the reverse pass reloads; the work part holds the
// recursions' intermediates and the reverse pass's cotangents.  Both strides
// are odd, so the lanes of a one-lane-per-link pass hit distinct banks.
constexpr int LREC = 35;    // R 9, P 3, spatial inertia 10, V 6, external wrench 6, pad
constexpr int LR_R = 0, LR_P = 9, LR_SI = 12, LR_V = 22, LR_FX = 28;
// The work record's fields are ordered so that every tree sum of a team runs
// over one block of consecutive floats: [A, F_bar] (root first, reverse),
// [Ic, F] (leaves first, forward), [F, A_bar], V_bar and [R_bar, P_bar]
// (leaves first, reverse).
constexpr int LWORK = 65;   // A 6, F_bar 6, Ic 10, F 6, A_bar 6, V_bar 6, R_bar 9, P_bar 3, pose cotangent to parent 12, pad
constexpr int LW_A = 0, LW_FB = 6, LW_IC = 12, LW_F = 22, LW_AB = 28, LW_VB = 34, LW_RB = 40, LW_PB = 49, LW_TP = 52;
static_assert(LW_FB == LW_A + 6 && LW_F == LW_IC + 10 && LW_AB == LW_F + 6 && LW_PB == LW_RB + 9,
              "tree-sum blocks must be contiguous");

// ------------------------------------------------------------ accessors --
// Global-memory scratch: component c of an environment at base[c * stride].
struct GMem {
  float* b;
  int s;
  __device__ __forceinline__ float& operator[](int i) const { return b[(size_t)i * s]; }
};
// Shared-memory scratch: contiguous per environment.
struct SMem {
  float* b;
  __device__ __forceinline__ float& operator[](int i) const { return b[i]; }
};

__device__ __forceinline__ int lrec(const DevModel& M, int i) { return M.o_LR + LREC * i; }
__device__ __forceinline__ int lwork(const DevModel& M, int i) { return M.o_LW + LWORK * i; }

// Parent of link i (-1: a root).  A model-specialised build has the parent
// table as a literal list (SHAC_SPEC_PARENTS), so in a loop over the links that
// the compiler unrolls, every parent and every scratch address derived from it
// is a constant; for a link index only known at run time use the table read.
__device__ __forceinline__ int link_parent(const DevModel& M, int i) {
#ifdef SHAC_SPEC_PARENTS
  constexpr int kParent[] = {SHAC_SPEC_PARENTS};
  (void)M;
  return kParent[i];
#else
  return __ldg(M.parent + i);
#endif
}

// Subtree sums of NC consecutive floats of every link's work record starting
// at field f, one component per lane: x_p += x_i for each link i > 0 with a
// parent, in descending order.  Links are numbered parent first, so link i's
// subtree is complete when i is reached; every lane runs the same link
// sequence (no barrier per tree level, no chain lookups) and the lanes of one
// link access consecutive words.  A model may have several roots (parent -1).
// REC: the field is in the link record instead of the work record.
template <bool REC>
__device__ __forceinline__ int lbase(const DevModel& M, int i) { return REC ? lrec(M, i) : lwork(M, i); }

template <int NC, bool REC = false, class Mem>
__device__ __forceinline__ void subtree_sums(const DevModel& M, const Mem& w, int f, int lane, int nl) {
  for (int c = lane; c < NC; c += nl) {
#pragma unroll
    for (int i = M.L - 1; i > 0; --i) {
      const int p = link_parent(M, i);
      if (p >= 0) w[lbase<REC>(M, p) + f + c] += w[lbase<REC>(M, i) + f + c];
    }
  }
}

// Ancestor sums, the root-first counterpart: x_i += x_p for each link i > 0
// with a parent, in ascending order (the parent's value is final when i is
// reached).
template <int NC, bool REC = false, class Mem>
__device__ __forceinline__ void ancestor_sums(const DevModel& M, const Mem& w, int f, int lane, int nl) {
  for (int c = lane; c < NC; c += nl) {
#pragma unroll
    for (int i = 1; i < M.L; ++i) {
      const int p = link_parent(M, i);
      if (p >= 0) w[lbase<REC>(M, i) + f + c] += w[lbase<REC>(M, p) + f + c];
    }
  }
}

__device__ __forceinline__ void team_sync(int nl) {
  if (nl > 1) __syncwarp();
}

// ----------------------------------------------------------- small math --
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float a, float b, float c) { return {a, b, c}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class Mem> __device__ __forceinline__ V3 ld3(const Mem& w, int o) { return {w[o], w[o + 1], w[o + 2]}; }
template <class Mem> __device__ __forceinline__ void st3(const Mem& w, int o, V3 v) { w[o] = v.x; w[o + 1] = v.y; w[o + 2] = v.z; }
template <class Mem> __device__ __forceinline__ void add3(const Mem& w, int o, V3 v) { w[o] += v.x; w[o + 1] += v.y; w[o + 2] += v.z; }
__device__ __forceinline__ V3 cld3(const float* p) { return {__ldg(p), __ldg(p + 1), __ldg(p + 2)}; }

struct M33 { float m[9]; };   // row major
template <class Mem> __device__ __forceinline__ M33 ldm(const Mem& w, int o) {
  M33 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.m[i] = w[o + i];
  return r;
}
template <class Mem> __device__ __forceinline__ void stm(const Mem& w, int o, const M33& r) {
#pragma unroll
  for (int i = 0; i < 9; ++i) w[o + i] = r.m[i];
}
__device__ __forceinline__ M33 cldm(const float* p) {
  M33 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.m[i] = __ldg(p + i);
  return r;
}
__device__ __forceinline__ V3 mul(const M33& R, V3 x) {
  return {R.m[0] * x.x + R.m[1] * x.y + R.m[2] * x.z, R.m[3] * x.x + R.m[4] * x.y + R.m[5] * x.z,
          R.m[6] * x.x + R.m[7] * x.y + R.m[8] * x.z};
}
__device__ __forceinline__ V3 mulT(const M33& R, V3 x) {
  return {R.m[0] * x.x + R.m[3] * x.y + R.m[6] * x.z, R.m[1] * x.x + R.m[4] * x.y + R.m[7] * x.z,
          R.m[2] * x.x + R.m[5] * x.y + R.m[8] * x.z};
}
__device__ __forceinline__ M33 mul(const M33& A, const M33& B) {
  M33 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C.m[3 * i + j] = A.m[3 * i] * B.m[j] + A.m[3 * i + 1] * B.m[3 + j] + A.m[3 * i + 2] * B.m[6 + j];
  return C;
}
__device__ __forceinline__ M33 mulBT(const M33& A, const M33& B) {   // A B^T
  M33 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C.m[3 * i + j] = A.m[3 * i] * B.m[3 * j] + A.m[3 * i + 1] * B.m[3 * j + 1] + A.m[3 * i + 2] * B.m[3 * j + 2];
  return C;
}
__device__ __forceinline__ V3 col(const M33& R, int k) { return {R.m[k], R.m[3 + k], R.m[6 + k]}; }

// unit-quaternion (x, y, z, w) rotation matrix
__device__ __forceinline__ M33 quat_to_R(float x, float y, float z, float w) {
  M33 R;
  R.m[0] = 1.f - 2.f * (y * y + z * z); R.m[1] = 2.f * (x * y - z * w); R.m[2] = 2.f * (x * z + y * w);
  R.m[3] = 2.f * (x * y + z * w); R.m[4] = 1.f - 2.f * (x * x + z * z); R.m[5] = 2.f * (y * z - x * w);
  R.m[6] = 2.f * (x * z - y * w); R.m[7] = 2.f * (y * z + x * w); R.m[8] = 1.f - 2.f * (x * x + y * y);
  return R;
}
// adjoint of quat_to_R: accumulate dR : Rbar into (xb, yb, zb, wb)
__device__ __forceinline__ void quat_to_R_adj(float x, float y, float z, float w, const M33& B,
                                              float& xb, float& yb, float& zb, float& wb) {
  const float* b = B.m;
  xb += 2.f * (b[1] * y + b[2] * z + b[3] * y - b[5] * w + b[6] * z + b[7] * w) - 4.f * x * (b[4] + b[8]);
  yb += 2.f * (b[1] * x + b[2] * w + b[3] * x + b[5] * z - b[6] * w + b[7] * z) - 4.f * y * (b[0] + b[8]);
  zb += 2.f * (-b[1] * w + b[2] * x + b[3] * w + b[5] * y + b[6] * x + b[7] * y) - 4.f * z * (b[0] + b[4]);
  wb += 2.f * (-b[1] * z + b[2] * y + b[3] * z - b[5] * x - b[6] * y + b[7] * x);
}
// rotation by angle t about unit axis a
__device__ __forceinline__ M33 axis_angle(V3 a, float t) {
  float s, c;
  sincosf(t, &s, &c);
  float k = 1.f - c;
  M33 R;
  R.m[0] = c + k * a.x * a.x; R.m[1] = k * a.x * a.y - s * a.z; R.m[2] = k * a.x * a.z + s * a.y;
  R.m[3] = k * a.y * a.x + s * a.z; R.m[4] = c + k * a.y * a.y; R.m[5] = k * a.y * a.z - s * a.x;
  R.m[6] = k * a.z * a.x - s * a.y; R.m[7] = k * a.z * a.y + s * a.x; R.m[8] = c + k * a.z * a.z;
  return R;
}

// spatial inertia at the world origin, 10 floats: m, h = m c (3), Io (xx yy zz xy xz yz)
// product I * (w, v) = (Io w + h x v, m v - h x w)
template <class Mem>
__device__ __forceinline__ void si_mul(const Mem& w, int o, V3 xw, V3 xv, V3& yn, V3& yf) {
  float m = w[o];
  V3 h = ld3(w, o + 1);
  float ixx = w[o + 4], iyy = w[o + 5], izz = w[o + 6], ixy = w[o + 7], ixz = w[o + 8], iyz = w[o + 9];
  V3 Iw = {ixx * xw.x + ixy * xw.y + ixz * xw.z, ixy * xw.x + iyy * xw.y + iyz * xw.z,
           ixz * xw.x + iyz * xw.y + izz * xw.z};
  yn = Iw + cross(h, xv);
  yf = m * xv - cross(h, xw);
}

// ================================================================= FORWARD ==
//
// Each link's work is one function called by one lane; the recursions over
// the tree are tree sums and poses by rows (a team) or chain walks (one
// thread).  A forward substep is the root-first part, the local pass, the
// leaves-first sums and the dense solve; the plain form calls the same
// functions from one thread per environment.

__device__ __forceinline__ M33 com_inertia(const DevModel& M, int i) {
  const float* ic = M.icom + 6 * i;
  M33 Ic;
  Ic.m[0] = __ldg(ic); Ic.m[4] = __ldg(ic + 1); Ic.m[8] = __ldg(ic + 2);
  Ic.m[1] = Ic.m[3] = __ldg(ic + 3); Ic.m[2] = Ic.m[6] = __ldg(ic + 4); Ic.m[5] = Ic.m[7] = __ldg(ic + 5);
  return Ic;
}

// joint spatial velocity u_i = sum_{d in i} S_d qd_d
template <class Mem>
__device__ __forceinline__ void joint_vel(const DevModel& M, const Mem& w, int i, V3& uw, V3& uv) {
  uw = v3(0.f, 0.f, 0.f); uv = v3(0.f, 0.f, 0.f);
  const int d0 = __ldg(M.ds + i), n = __ldg(M.nd + i);
  for (int d = d0; d < d0 + n; ++d) {
    const float qd = w[M.o_QD + d];
    uw = uw + qd * ld3(w, M.o_S + 6 * d);
    uv = uv + qd * ld3(w, M.o_S + 6 * d + 3);
  }
}

// Muscles (Sec. 3.1): force clamp(a, 0, 1) fmax along each via segment,
// pulling its two ends together.
template <class Mem>
__device__ __forceinline__ void seg_forward(const DevModel& M, const Mem& w, int sg) {
  const int e0 = M.nc + 2 * sg, e1 = e0 + 1;
  const int l0 = __ldg(M.item_link + e0), l1 = __ldg(M.item_link + e1);
  const V3 x0 = ld3(w, lrec(M, l0) + LR_P) + mul(ldm(w, lrec(M, l0) + LR_R), cld3(M.item_pos + 3 * e0));
  const V3 x1 = ld3(w, lrec(M, l1) + LR_P) + mul(ldm(w, lrec(M, l1) + LR_R), cld3(M.item_pos + 3 * e1));
  const int mu_ = __ldg(M.seg_mus + sg);
  const float a = fminf(fmaxf(w[M.o_ACT + M.ntact + mu_], 0.f), 1.f);
  const float F = a * __ldg(M.fmax + mu_);
  const V3 dv = x1 - x0;
  const V3 u = (1.f / sqrtf(dot(dv, dv))) * dv;
  st3(w, M.o_IT + 7 * e0, x0);
  st3(w, M.o_IT + 7 * e0 + 3, F * u);
  st3(w, M.o_IT + 7 * e1, x1);
  st3(w, M.o_IT + 7 * e1 + 3, -F * u);
}

// Wrench of part r (of parts) of the muscle via points attached to link i:
// the link's items r, r + parts, r + 2 parts, ...
template <class Mem>
__device__ __forceinline__ void lk_muscle_wrench(const DevModel& M, const Mem& w, int i, int r, int parts, V3& wn,
                                                 V3& wf) {
  wn = v3(0.f, 0.f, 0.f); wf = v3(0.f, 0.f, 0.f);
  for (int k = __ldg(M.lm_ptr + i) + r; k < __ldg(M.lm_ptr + i + 1); k += parts) {
    const int e = __ldg(M.lm_idx + k);
    const V3 x = ld3(w, M.o_IT + 7 * e), f = ld3(w, M.o_IT + 7 * e + 3);
    wn = wn + cross(x, f);
    wf = wf + f;
  }
}

// Lanes per link in the per-link muscle sums (at most 32 (link, part) slots).
__device__ __forceinline__ int muscle_parts(const DevModel& M, int nl) { return nl >= 2 * M.L ? nl / M.L : 1; }

// The chain walks of the PLAIN form (and of a one-lane team) visit chains:
// maximal runs of links in which every link but the last has exactly one
// child, walked parent-first (root-first sweeps) or child-first (leaves-first
// sweeps) with the carried values in registers.  Teams use the tree sums and
// the poses by rows instead.
__device__ __forceinline__ int chain_next(const DevModel& M, int i) { return __ldg(M.ch_idx + __ldg(M.ch_ptr + i)); }

// Sweep 1 is split into passes.  Everything local to a link runs with one
// lane per link for all links at once: the joint's own transform before the
// root-first part (lk_joint_local), the inertia, contacts and local force
// after it (lk_local).  In between, what flows down the tree - the world pose,
// velocity and acceleration of the parent: a team computes the poses by rows
// (poses_by_rows) and the velocities and accelerations as ancestor sums of
// per-link terms; a single thread (PLAIN form) walks the chains keeping the
// parent's values in registers (KinCarry, lk_kin).
//
// lk_joint_local: pose of link i in its parent's frame (joint frame times
// joint motion: Rot(axis, q) for revolute, q axis for prismatic; the free
// root's pose from its quaternion), written to the pose fields of link i's record.
// TO_WORK: write the local pose to the pose-cotangent slot of link i's work
// record (its [R, P] layout; free in the forward pass) instead of its record,
// for poses_by_rows.
template <bool TO_WORK = false, class Mem>
__device__ __forceinline__ void lk_joint_local(const DevModel& M, const Mem& w, int i) {
  const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i);
  M33 R;
  V3 P;
  if (jt == J_FREE) {
    R = quat_to_R(w[M.o_Q + s + 3], w[M.o_Q + s + 4], w[M.o_Q + s + 5], w[M.o_Q + s + 6]);
    P = v3(0.f, 0.f, 0.f);
  } else {
    R = cldm(M.jrot + 9 * i);
    P = cld3(M.jpos + 3 * i);
    const V3 ax = cld3(M.axis + 3 * i);
    if (jt == J_REV) R = mul(R, axis_angle(ax, w[M.o_Q + s]));
    else if (jt == J_PRIS) P = P + w[M.o_Q + s] * mul(R, ax);
  }
  const int o = TO_WORK ? lwork(M, i) + LW_TP : lrec(M, i);
  static_assert(LR_P == LR_R + 9, "a pose is R (9) then P (3)");
  stm(w, o + LR_R, R);
  st3(w, o + LR_P, P);
}

// World poses by rows (team form): the lane owning row r (lanes r, r + T, ...
// for the three rows; a team of two lanes gives the first lane rows 0 and 2)
// computes row r of R_i = R_p R_local and P_i[r] = P_p[r] + (row r of R_p) .
// P_local for every link in ascending order (parents first; a root keeps its
// local pose).  Row r of a link's pose depends only on row r of its parent's,
// which the same lane wrote, so the lanes never wait for one another; the local
// poses come from the work records (lk_joint_local<true>).
template <class Mem>
__device__ __forceinline__ void poses_by_rows(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int r = lane; r < 3; r += nl) {
#pragma unroll
    for (int i = 0; i < M.L; ++i) {
      const int ol = lwork(M, i) + LW_TP, o = lrec(M, i);
      const int p = link_parent(M, i);
      V3 row = ld3(w, ol + LR_R + 3 * r);
      float pr = w[ol + LR_P + r];
      if (p >= 0) {
        const int op = lrec(M, p);
        const V3 rp = ld3(w, op + LR_R + 3 * r);
        row = rp.x * ld3(w, ol + LR_R) + rp.y * ld3(w, ol + LR_R + 3) + rp.z * ld3(w, ol + LR_R + 6);
        pr = w[op + LR_P + r] + dot(rp, ld3(w, ol + LR_P));
      }
      st3(w, o + LR_R + 3 * r, row);
      w[o + LR_P + r] = pr;
    }
  }
}

// World pose, velocity and acceleration carried from a link to its child.
struct KinCarry {
  M33 R;
  V3 P, Vw, Vv, aw, av;
};

// Parent state of a chain head (the tree root: identity frame at rest, with
// gravity as the base acceleration -g).
template <class Mem>
__device__ __forceinline__ void kin_parent(const DevModel& M, const Mem& w, int p, KinCarry& c) {
  if (p >= 0) {
    c.R = ldm(w, lrec(M, p) + LR_R);
    c.P = ld3(w, lrec(M, p) + LR_P);
    c.Vw = ld3(w, lrec(M, p) + LR_V); c.Vv = ld3(w, lrec(M, p) + LR_V + 3);
    c.aw = ld3(w, lwork(M, p) + LW_A); c.av = ld3(w, lwork(M, p) + LW_A + 3);
  } else {
    c.Vw = c.Vv = c.aw = v3(0.f, 0.f, 0.f);
    c.av = v3(-M.grav[0], -M.grav[1], -M.grav[2]);
  }
}

// lk_kin: world pose R_i = R_p R_local, P_i = P_p + R_p P_local (the root and
// a free joint: the local pose), the motion-subspace columns (revolute
// (a, P x a), prismatic (0, a), free (R e_k, P x R e_k) for the body rates and
// (0, R e_k) for v_body), the velocity V_i = V_p + u_i and the Newton-Euler
// acceleration A_i = A_p + V_i x u_i with qdd = 0.  c holds the parent's state
// on entry and link i's on return.
template <class Mem>
__device__ __forceinline__ void lk_kin(const DevModel& M, const Mem& w, int i, KinCarry& c) {
  const int jt = __ldg(M.jtype + i), p = __ldg(M.parent + i);
  const int d0 = __ldg(M.ds + i), nd = __ldg(M.nd + i);
  const V3 ax = cld3(M.axis + 3 * i);
  const M33 Rl = ldm(w, lrec(M, i) + LR_R);
  const V3 Pl = ld3(w, lrec(M, i) + LR_P);
  float qdv[6];
  if (jt == J_FREE) {
#pragma unroll
    for (int k = 0; k < 6; ++k) qdv[k] = w[M.o_QD + d0 + k];
  } else {
    qdv[0] = nd == 1 ? w[M.o_QD + d0] : 0.f;
  }
  M33 R;
  V3 P;
  if (jt == J_FREE || p < 0) {
    R = Rl;
    P = Pl;
  } else {
    R = mul(c.R, Rl);
    P = c.P + mul(c.R, Pl);
  }
  stm(w, lrec(M, i) + LR_R, R);
  st3(w, lrec(M, i) + LR_P, P);
  V3 uw = v3(0.f, 0.f, 0.f), uv = v3(0.f, 0.f, 0.f);
  auto subspace = [&](int k, V3 sw, V3 sv) {
    st3(w, M.o_S + 6 * (d0 + k), sw);
    st3(w, M.o_S + 6 * (d0 + k) + 3, sv);
    const float qd = qdv[k];
    uw = uw + qd * sw;
    uv = uv + qd * sv;
  };
  // DOF counts are fixed by the joint type (free 6, revolute / prismatic 1,
  // fixed 0), so every column index below is a compile-time constant
  if (jt == J_FREE) {
#pragma unroll
    for (int k = 0; k < 3; ++k) subspace(k, col(R, k), cross(P, col(R, k)));
#pragma unroll
    for (int k = 0; k < 3; ++k) subspace(3 + k, v3(0.f, 0.f, 0.f), col(R, k));
  } else if (nd == 1) {
    const V3 a = mul(R, ax);
    if (jt == J_REV) subspace(0, a, cross(P, a));
    else subspace(0, v3(0.f, 0.f, 0.f), a);
  }
  const V3 Vw = c.Vw + uw, Vv = c.Vv + uv;
  const V3 aw = c.aw + cross(Vw, uw);
  const V3 av = c.av + cross(Vw, uv) + cross(Vv, uw);
  st3(w, lrec(M, i) + LR_V, Vw); st3(w, lrec(M, i) + LR_V + 3, Vv);
  st3(w, lwork(M, i) + LW_A, aw); st3(w, lwork(M, i) + LW_A + 3, av);
  c.R = R; c.P = P; c.Vw = Vw; c.Vv = Vv; c.aw = aw; c.av = av;
}

// Team form of sweep 1: the world poses by rows (poses_by_rows), the rest of
// lk_kin a pass per link and two ancestor sums, since V_i = V_p + u_i and
// A_i = A_p + V_i x u_i (the roots' A_p: -g) are sums of terms of each link
// along its path from the root.
// Link i's motion-subspace columns (as in lk_kin) and its joint velocity u_i,
// the own term of V_i, stored in the V field and, for lk_bias_acc_own, in the
// F_bar field (unused by the forward pass).
template <class Mem>
__device__ __forceinline__ void lk_subspace_vel(const DevModel& M, const Mem& w, int i) {
  const int jt = __ldg(M.jtype + i), d0 = __ldg(M.ds + i), nd = __ldg(M.nd + i);
  const M33 R = ldm(w, lrec(M, i) + LR_R);
  const V3 P = ld3(w, lrec(M, i) + LR_P);
  V3 uw = v3(0.f, 0.f, 0.f), uv = v3(0.f, 0.f, 0.f);
  auto subspace = [&](int k, V3 sw, V3 sv) {
    st3(w, M.o_S + 6 * (d0 + k), sw);
    st3(w, M.o_S + 6 * (d0 + k) + 3, sv);
    const float qd = w[M.o_QD + d0 + k];
    uw = uw + qd * sw;
    uv = uv + qd * sv;
  };
  if (jt == J_FREE) {
#pragma unroll
    for (int k = 0; k < 3; ++k) subspace(k, col(R, k), cross(P, col(R, k)));
#pragma unroll
    for (int k = 0; k < 3; ++k) subspace(3 + k, v3(0.f, 0.f, 0.f), col(R, k));
  } else if (nd == 1) {
    const V3 a = mul(R, cld3(M.axis + 3 * i));
    if (jt == J_REV) subspace(0, a, cross(P, a));
    else subspace(0, v3(0.f, 0.f, 0.f), a);
  }
  st3(w, lrec(M, i) + LR_V, uw); st3(w, lrec(M, i) + LR_V + 3, uv);
  st3(w, lwork(M, i) + LW_FB, uw); st3(w, lwork(M, i) + LW_FB + 3, uv);
}
// The own term of A_i after the velocity sums: V_i x u_i, and -g at a root.
template <class Mem>
__device__ __forceinline__ void lk_bias_acc_own(const DevModel& M, const Mem& w, int i) {
  const V3 Vw = ld3(w, lrec(M, i) + LR_V), Vv = ld3(w, lrec(M, i) + LR_V + 3);
  const V3 uw = ld3(w, lwork(M, i) + LW_FB), uv = ld3(w, lwork(M, i) + LW_FB + 3);
  const V3 aw = cross(Vw, uw);
  V3 av = cross(Vw, uv) + cross(Vv, uw);
  if (__ldg(M.parent + i) < 0) av = av + v3(-M.grav[0], -M.grav[1], -M.grav[2]);
  st3(w, lwork(M, i) + LW_A, aw); st3(w, lwork(M, i) + LW_A + 3, av);
}

// lk_local: the spatial inertia about the reference point (m, h = m c, Io),
// the contact forces of link i and its local force
// F_i = I_i A_i + V_i x* (I_i V_i) - Fext_i, from the pose, velocity and
// acceleration lk_kin stored.
template <class Mem>
__device__ __forceinline__ void lk_local(const DevModel& M, const Mem& w, int i) {
  const M33 R = ldm(w, lrec(M, i) + LR_R);
  const V3 P = ld3(w, lrec(M, i) + LR_P);
  const V3 Vw = ld3(w, lrec(M, i) + LR_V), Vv = ld3(w, lrec(M, i) + LR_V + 3);
  const V3 aw = ld3(w, lwork(M, i) + LW_A), av = ld3(w, lwork(M, i) + LW_A + 3);
  const float m = __ldg(M.mass + i);
  const V3 c = P + mul(R, cld3(M.com + 3 * i));
  const M33 Iw = mulBT(mul(R, com_inertia(M, i)), R);
  const float cc = dot(c, c);
  const V3 h = m * c;
  const float ixx = Iw.m[0] + m * (cc - c.x * c.x), iyy = Iw.m[4] + m * (cc - c.y * c.y);
  const float izz = Iw.m[8] + m * (cc - c.z * c.z), ixy = Iw.m[1] - m * c.x * c.y;
  const float ixz = Iw.m[2] - m * c.x * c.z, iyz = Iw.m[5] - m * c.y * c.z;
  {   // the link's own spatial inertia, in the record and as the start of its composite inertia
    const int o = lrec(M, i) + LR_SI, oc = lwork(M, i) + LW_IC;
    w[o] = m; st3(w, o + 1, h);
    w[o + 4] = ixx; w[o + 5] = iyy; w[o + 6] = izz; w[o + 7] = ixy; w[o + 8] = ixz; w[o + 9] = iyz;
    w[oc] = m; st3(w, oc + 1, h);
    w[oc + 4] = ixx; w[oc + 5] = iyy; w[oc + 6] = izz; w[oc + 7] = ixy; w[oc + 8] = ixz; w[oc + 9] = iyz;
  }
  auto imul = [&](V3 xw, V3 xv, V3& yn, V3& yf) {
    yn = v3(ixx * xw.x + ixy * xw.y + ixz * xw.z, ixy * xw.x + iyy * xw.y + iyz * xw.z,
            ixz * xw.x + iyz * xw.y + izz * xw.z) + cross(h, xv);
    yf = m * xv - cross(h, xw);
  };
  // Sec. 3.1 contact model on the ground plane z = 0 (n = +z) for the contact
  // spheres of link i, applied at the lowest point x of each sphere:
  //   f_n = (-ke + kd ddot) min(d, 0),  d = height of x, ddot = v_x . n
  //   f_t = -v_t/|v_t| min(kt |v_t|, mu |f_n|)  (viscous branch when kt|v_t| <= mu|f_n|)
  V3 wn = v3(0.f, 0.f, 0.f), wf = v3(0.f, 0.f, 0.f);
  const int k0 = __ldg(M.lc_ptr + i), k1 = __ldg(M.lc_ptr + i + 1);
  if (k0 != k1) {
    const float zroot = M.root_free ? w[M.o_Q + 2] : 0.f;
    for (int k = k0; k < k1; ++k) {
      const int ci = __ldg(M.lc_idx + k);
      V3 x = P + mul(R, cld3(M.item_pos + 3 * ci));
      x.z -= __ldg(M.crad + ci);
      const float d = x.z + zroot;
      V3 f = v3(0.f, 0.f, 0.f);
      if (d < 0.f) {
        const V3 vp = Vv + cross(Vw, x);
        const float fn = (-M.ke + M.kd * vp.z) * d;
        const float vt = sqrtf(vp.x * vp.x + vp.y * vp.y);
        const float afn = fabsf(fn);
        if (M.kt * vt <= M.mu * afn) { f.x = -M.kt * vp.x; f.y = -M.kt * vp.y; }
        else { const float sc = M.mu * afn / vt; f.x = -sc * vp.x; f.y = -sc * vp.y; }
        f.z = fn;
      }
      st3(w, M.o_IT + 7 * ci, x);
      st3(w, M.o_IT + 7 * ci + 3, f);
      w[M.o_IT + 7 * ci + 6] = d;
      wn = wn + cross(x, f);
      wf = wf + f;
    }
  }
  st3(w, lrec(M, i) + LR_FX, wn);
  st3(w, lrec(M, i) + LR_FX + 3, wf);
  V3 fn, ff, bn, bf;
  imul(aw, av, fn, ff);
  imul(Vw, Vv, bn, bf);
  fn = fn + cross(Vw, bn) + cross(Vv, bf) - wn;
  ff = ff + cross(Vw, bf) - wf;
  st3(w, lwork(M, i) + LW_F, fn);
  st3(w, lwork(M, i) + LW_F + 3, ff);
}

// Sweep 1: one lane per link the joint transforms; root first the world
// poses, subspaces, velocities and Newton-Euler accelerations (qdd = 0) of
// every link (a team: poses by rows, per-link terms and ancestor sums; one
// thread: chain walks); one lane per link the inertias, contact forces and
// local forces; then the muscle wrenches (their segments span two links).
template <class Mem>
__device__ void sw_forward(const DevModel& M, const Mem& w, int lane, int nl) {
  if (nl > 1) {   // a team: poses by rows, the rest per link and by ancestor sums
    for (int i = lane; i < M.L; i += nl) lk_joint_local<true>(M, w, i);
    team_sync(nl);
    poses_by_rows(M, w, lane, nl);
    team_sync(nl);
    for (int i = lane; i < M.L; i += nl) lk_subspace_vel(M, w, i);
    team_sync(nl);
    ancestor_sums<6, true>(M, w, LR_V, lane, nl);
    team_sync(nl);
    for (int i = lane; i < M.L; i += nl) lk_bias_acc_own(M, w, i);
    team_sync(nl);
    ancestor_sums<6>(M, w, LW_A, lane, nl);
    team_sync(nl);
  } else {        // one thread: chain walks carrying pose, velocity and acceleration
    for (int i = 0; i < M.L; ++i) lk_joint_local(M, w, i);
    for (int l = 0; l < M.nlev; ++l) {
      for (int ii = __ldg(M.lvl_ptr + l); ii < __ldg(M.lvl_ptr + l + 1); ++ii) {
        const int hd = __ldg(M.lvl_link + ii), tl = __ldg(M.chain_tail + hd);
        KinCarry c;
        kin_parent(M, w, __ldg(M.parent + hd), c);
        for (int i = hd;; i = chain_next(M, i)) {
          lk_kin(M, w, i, c);
          if (i == tl) break;
        }
      }
    }
  }
  for (int i = lane; i < M.L; i += nl) lk_local(M, w, i);
  team_sync(nl);
  if (M.nseg > 0) {
    for (int sg = lane; sg < M.nseg; sg += nl) seg_forward(M, w, sg);
    team_sync(nl);
    // each link's muscle wrench in `parts` partial sums on as many lanes,
    // then added in part order
    const int parts = muscle_parts(M, nl);
    for (int sl = lane; sl < M.L * parts; sl += nl) {
      V3 wn, wf;
      lk_muscle_wrench(M, w, sl / parts, sl % parts, parts, wn, wf);
      st3(w, M.o_MW + 6 * sl, wn);
      st3(w, M.o_MW + 6 * sl + 3, wf);
    }
    team_sync(nl);
    for (int i = lane; i < M.L; i += nl) {
      V3 wn = v3(0.f, 0.f, 0.f), wf = v3(0.f, 0.f, 0.f);
      for (int r = 0; r < parts; ++r) {
        wn = wn + ld3(w, M.o_MW + 6 * (i * parts + r));
        wf = wf + ld3(w, M.o_MW + 6 * (i * parts + r) + 3);
      }
      add3(w, lrec(M, i) + LR_FX, wn);
      add3(w, lrec(M, i) + LR_FX + 3, wf);
      add3(w, lwork(M, i) + LW_F, -wn);
      add3(w, lwork(M, i) + LW_F + 3, -wf);
    }
    team_sync(nl);
  }
}

// Total force and composite inertia of the link a chain walk just finished,
// carried in registers to its parent (the next link up the chain).
struct GatherCarry {
  V3 fn, ff;
  float ic[10];
};

// F_i += sum_children F_c (total forces) and Ic_i += sum_children Ic_c
// (composite inertias, CRBA part 1; lk_local starts Ic_i at the link's own
// inertia).  Inside a chain the only child is the link walked before (carried
// in g); the chain's tail reads its children from scratch.
template <class Mem>
__device__ __forceinline__ void lk_gather(const DevModel& M, const Mem& w, int i, bool tail, GatherCarry& g) {
  V3 fn = ld3(w, lwork(M, i) + LW_F), ff = ld3(w, lwork(M, i) + LW_F + 3);
  float ic[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) ic[k] = w[lwork(M, i) + LW_IC + k];
  if (tail) {
    const int c0 = __ldg(M.ch_ptr + i), c1 = __ldg(M.ch_ptr + i + 1);
    for (int kk = c0; kk < c1; ++kk) {
      const int c = __ldg(M.ch_idx + kk);
      fn = fn + ld3(w, lwork(M, c) + LW_F);
      ff = ff + ld3(w, lwork(M, c) + LW_F + 3);
#pragma unroll
      for (int k = 0; k < 10; ++k) ic[k] += w[lwork(M, c) + LW_IC + k];
    }
  } else {
    fn = fn + g.fn;
    ff = ff + g.ff;
#pragma unroll
    for (int k = 0; k < 10; ++k) ic[k] += g.ic[k];
  }
  st3(w, lwork(M, i) + LW_F, fn);
  st3(w, lwork(M, i) + LW_F + 3, ff);
#pragma unroll
  for (int k = 0; k < 10; ++k) w[lwork(M, i) + LW_IC + k] = ic[k];
  g.fn = fn;
  g.ff = ff;
#pragma unroll
  for (int k = 0; k < 10; ++k) g.ic[k] = ic[k];
}

// Sweep 2, leaves first: total forces and composite inertias (Ic and F are the
// 16 consecutive floats from LW_IC).  A team sums them one component per lane;
// a single thread (PLAIN form) walks the chains with register carries.
template <class Mem>
__device__ void sw_gather(const DevModel& M, const Mem& w, int lane, int nl) {
  if (nl > 1) {
    subtree_sums<16>(M, w, LW_IC, lane, nl);
    team_sync(nl);
    return;
  }
  for (int l = M.nlev - 1; l >= 0; --l) {
    for (int ii = __ldg(M.lvl_ptr + l); ii < __ldg(M.lvl_ptr + l + 1); ++ii) {
      const int hd = __ldg(M.lvl_link + ii), tl = __ldg(M.chain_tail + hd);
      GatherCarry g;
      for (int i = tl;; i = __ldg(M.parent + i)) {
        lk_gather(M, w, i, i == tl, g);
        if (i == hd) break;
      }
    }
  }
}

// joint-space actuation, limit penalty (Sec. 3.1) and damping
template <class Mem>
__device__ __forceinline__ float joint_force(const DevModel& M, const Mem& w, int d) {
  float t = 0.f;
  const int a = __ldg(M.dof_act + d);
  if (a >= 0) t = __ldg(M.gear + d) * w[M.o_ACT + a];
  const int i = __ldg(M.dof_link + d), jt = __ldg(M.jtype + i);
  if (jt == J_REV || jt == J_PRIS) {
    const float q = w[M.o_Q + __ldg(M.qs + i)];
    const float lo = __ldg(M.qlo + d), hi = __ldg(M.qhi + d);
    if (q < lo) t += M.klim * (lo - q);
    else if (q > hi) t += M.klim * (hi - q);
  }
  return t - __ldg(M.damp + d) * w[M.o_QD + d];
}

// right-hand side of DOF d: b_d = tau_j - S_d . F_total (bias with qdd = 0)
template <class Mem>
__device__ __forceinline__ float dof_rhs(const DevModel& M, const Mem& w, int d) {
  const int i = __ldg(M.dof_link + d);
  const float c = dot(ld3(w, M.o_S + 6 * d), ld3(w, lwork(M, i) + LW_F)) +
                  dot(ld3(w, M.o_S + 6 * d + 3), ld3(w, lwork(M, i) + LW_F + 3));
  return joint_force(M, w, d) - c;
}

template <class Mem>
__device__ void st_rhs(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int d = lane; d < M.nv; d += nl) w[M.o_B + d] = dof_rhs(M, w, d);
  team_sync(nl);
}

// CRBA part 2, shared-memory form: lower triangle of M row by row (row a
// owns M[a][b], b <= a; zero unless b moves an ancestor-or-self link of a),
// armature on the diagonal.
template <class Mem>
__device__ void st_mass_rows(const DevModel& M, const Mem& w, int lane, int nl) {
  const int n = M.nv;
  for (int a = lane; a < n; a += nl) {
    const int i = __ldg(M.dof_link + a);
    for (int b = 0; b < a; ++b) w[M.o_M + a * n + b] = 0.f;
    V3 fn, ff;
    si_mul(w, lwork(M, i) + LW_IC, ld3(w, M.o_S + 6 * a), ld3(w, M.o_S + 6 * a + 3), fn, ff);
    for (int j = i; j >= 0; j = __ldg(M.parent + j)) {
      const int b0 = __ldg(M.ds + j), nb = __ldg(M.nd + j);
      for (int b = b0; b < b0 + nb && b <= a; ++b)
        w[M.o_M + a * n + b] = dot(ld3(w, M.o_S + 6 * b), fn) + dot(ld3(w, M.o_S + 6 * b + 3), ff);
    }
    w[M.o_M + a * n + a] += __ldg(M.arm + a);
  }
  team_sync(nl);
}

// Cholesky factorisation in place (strict lower part in o_M, diagonal in
// o_LD), right-looking; the trailing update of each row is done by one lane.
template <class Mem>
__device__ void st_chol(const DevModel& M, const Mem& w, int lane, int nl) {
  const int n = M.nv;
  for (int k = 0; k < n; ++k) {
    const float dkk = sqrtf(w[M.o_M + k * n + k]);
    const float inv = 1.f / dkk;
    if (lane == 0) w[M.o_LD + k] = dkk;
    for (int i = k + 1 + lane; i < n; i += nl) w[M.o_M + i * n + k] *= inv;
    team_sync(nl);
    for (int i = k + 1 + lane; i < n; i += nl) {
      const float lik = w[M.o_M + i * n + k];
      for (int j = k + 1; j <= i; ++j) w[M.o_M + i * n + j] -= lik * w[M.o_M + j * n + k];
    }
    team_sync(nl);
  }
}

// x = (L L^T)^{-1} b using the cached factor; b (o_in) is consumed, o_T is scratch.
template <class Mem>
__device__ void st_solve(const DevModel& M, const Mem& w, int lane, int nl, int o_in, int o_out) {
  const int n = M.nv;
  for (int k = 0; k < n; ++k) {
    const float yk = w[o_in + k] / w[M.o_LD + k];
    if (lane == 0) w[M.o_T + k] = yk;
    for (int i = k + 1 + lane; i < n; i += nl) w[o_in + i] -= w[M.o_M + i * n + k] * yk;
    team_sync(nl);
  }
  for (int k = n - 1; k >= 0; --k) {
    const float xk = w[M.o_T + k] / w[M.o_LD + k];
    if (lane == 0) w[o_out + k] = xk;
    for (int i = lane; i < k; i += nl) w[M.o_T + i] -= w[M.o_M + k * n + i] * xk;
    team_sync(nl);
  }
}

// Exact sum of two floats: s + e == a + b (Knuth's two-sum).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bp = s - a;
  const float ap = s - bp;
  e = (a - ap) + (b - bp);
  return s;
}

// Semi-implicit Euler for link i's joint: qd += h qdd, then q += h qd (new
// velocity); free root: p += h R v_b, quat <- normalise(quat + h/2 quat (x)
// (w_b, 0)).  The state stays FP32 between substeps; the rounding of each
// accumulation is carried in o_QC/o_QDC (zeroed at every step start) and fed
// back into the next substep's update, so a step of K substeps rounds its
// state once.
// The velocity update of DOF d (first, for every DOF) ...
template <class Mem>
__device__ __forceinline__ void dof_integrate(const DevModel& M, const Mem& w, int d) {
  float e;
  const float y = M.h * w[M.o_QDD + d] + w[M.o_QDC + d];
  w[M.o_QD + d] = two_sum(w[M.o_QD + d], y, e);
  w[M.o_QDC + d] = e;
}
// ... then the position update of link i's joint from the new velocities.
template <class Mem>
__device__ __forceinline__ void lk_integrate(const DevModel& M, const Mem& w, int i) {
  const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i), d0 = __ldg(M.ds + i);
  if (jt == J_FREE) {
    const M33 R = ldm(w, lrec(M, i) + LR_R);
    const V3 dp = M.h * mul(R, ld3(w, M.o_QD + d0 + 3)) + M.h * mul(R, ld3(w, M.o_QDC + d0 + 3));
    float e;
    w[M.o_Q + s] = two_sum(w[M.o_Q + s], dp.x + w[M.o_QC + s], e); w[M.o_QC + s] = e;
    w[M.o_Q + s + 1] = two_sum(w[M.o_Q + s + 1], dp.y + w[M.o_QC + s + 1], e); w[M.o_QC + s + 1] = e;
    w[M.o_Q + s + 2] = two_sum(w[M.o_Q + s + 2], dp.z + w[M.o_QC + s + 2], e); w[M.o_QC + s + 2] = e;
    const float x = w[M.o_Q + s + 3], y = w[M.o_Q + s + 4], z = w[M.o_Q + s + 5], qw = w[M.o_Q + s + 6];
    const V3 om = ld3(w, M.o_QD + d0);
    const V3 u = v3(x, y, z);
    const V3 pv = qw * om + cross(u, om);
    const float pw = -dot(u, om);
    const float hh = 0.5f * M.h;
    const float nx = x + hh * pv.x, ny = y + hh * pv.y, nz = z + hh * pv.z, nw = qw + hh * pw;
    const float inv = rsqrtf(nx * nx + ny * ny + nz * nz + nw * nw);
    w[M.o_Q + s + 3] = nx * inv; w[M.o_Q + s + 4] = ny * inv; w[M.o_Q + s + 5] = nz * inv; w[M.o_Q + s + 6] = nw * inv;
  } else if (jt == J_REV || jt == J_PRIS) {
    float e;
    const float y = M.h * w[M.o_QD + d0] + (M.h * w[M.o_QDC + d0] + w[M.o_QC + s]);
    w[M.o_Q + s] = two_sum(w[M.o_Q + s], y, e);
    w[M.o_QC + s] = e;
  }
}

template <class Mem>
__device__ void st_integrate(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int d = lane; d < M.nv; d += nl) dof_integrate(M, w, d);
  team_sync(nl);
  for (int i = lane; i < M.L; i += nl) lk_integrate(M, w, i);
  team_sync(nl);
}

// Clear the integration compensation at a step start (team-parallel).
template <class Mem>
__device__ __forceinline__ void clear_comp(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int j = lane; j < M.nq; j += nl) w[M.o_QC + j] = 0.f;
  for (int j = lane; j < M.nv; j += nl) w[M.o_QDC + j] = 0.f;
}

// ---- register-resident dense path (teams with at least nv lanes) ----------
// Lane a of the team owns row a of M and DOF a of the right-hand side.  The
// matrix is padded to NM x NM (nv <= NM <= team size) with identity rows.
// Every column loop is expanded at compile time through index sequences, so
// each row element is a named register (a runtime-bounded or partially
// unrolled loop would leave the row array in local memory) and no shuffle
// sits under a lane-dependent branch.  The row is assembled in registers
// (CRBA part 2, ancestor DOFs from a bit mask) and factorised by a
// right-looking Cholesky whose column k is broadcast with team shuffles; the
// strict lower part of L goes to o_M and the reciprocal diagonal 1/L_kk to
// o_LD for the solves and the backward pass.

// row[J] -= L_ik L_jk for the lanes i >= J of the trailing block.
template <int J, int NM>
__device__ __forceinline__ void chol_update(float (&row)[NM], float lik, int lane, int nl) {
  const float ljk = __shfl_sync(0xffffffffu, lik, J, nl);   // every lane takes part
  if (lane >= J) row[J] = fmaf(-lik, ljk, row[J]);
}
template <int K, int NM, int... J>
__device__ __forceinline__ void chol_trailing(float (&row)[NM], float lik, int lane, int nl,
                                              iseq<J...>) {
  (chol_update<K + 1 + J, NM>(row, lik, lane, nl), ...);
}
// Column K: L_KK = sqrt(pivot) (lane K), L_iK = M_iK / L_KK (lanes i > K).
// Every lane also keeps its own diagonal entry in `diag`, updated with its own
// L_iK (the same multiply-adds the trailing update applies to row[i] on lane
// i), so the next column's pivot is broadcast from a register that does not
// wait for this column's shuffles.
template <int K, int NM>
__device__ __forceinline__ void chol_column(float (&row)[NM], float& diag, float& inv_diag, int lane, int nl) {
  const float inv = rsqrtf(__shfl_sync(0xffffffffu, diag, K, nl));
  const float lik = row[K] * inv;
  if (lane >= K) row[K] = lik;
  if (lane == K) inv_diag = inv;
  if (lane > K) diag = fmaf(-lik, lik, diag);
  chol_trailing<K, NM>(row, lik, lane, nl, make_iseq<NM - K - 1>{});
}
template <int NM, int... K>
__device__ __forceinline__ void chol_columns(float (&row)[NM], float& diag, float& inv_diag, int lane, int nl,
                                             iseq<K...>) {
  (chol_column<K, NM>(row, diag, inv_diag, lane, nl), ...);
}

// Forward substitution y = L^{-1} b, step K: lane a holds b_a, row a of L in
// its registers.
template <int K, int NM>
__device__ __forceinline__ void fsub_step(const float (&row)[NM], float inv_diag, float& b, int lane, int nl) {
  const float yk = __shfl_sync(0xffffffffu, b * inv_diag, K, nl);
  if (lane > K) b = fmaf(-row[K], yk, b);
  else if (lane == K) b = yk;
}
template <int NM, int... K>
__device__ __forceinline__ void fsub(const float (&row)[NM], float inv_diag, float& b, int lane, int nl,
                                     iseq<K...>) {
  (fsub_step<K, NM>(row, inv_diag, b, lane, nl), ...);
}
// Backward substitution x = L^{-T} y, step K (descending): lane a < K needs
// L_Ka, read from the stored factor; the address is always valid so the load
// does not wait on the substitution chain.
template <int K, class Mem>
__device__ __forceinline__ void bsub_step(const DevModel& M, const Mem& w, float inv_diag, float& b, int lane,
                                          int nl) {
  const int n = M.nv;
  const bool use = lane < K && K < n;
  const float lka = w[M.o_M + (use ? K * n + lane : 0)];
  const float xk = __shfl_sync(0xffffffffu, b * inv_diag, K, nl);
  if (use) b = fmaf(-lka, xk, b);
  else if (lane == K) b = xk;
}
template <int NM, class Mem, int... K>
__device__ __forceinline__ void bsub(const DevModel& M, const Mem& w, float inv_diag, float& b, int lane, int nl,
                                     iseq<K...>) {
  (bsub_step<NM - 1 - K>(M, w, inv_diag, b, lane, nl), ...);
}

// Row a of M (CRBA part 2) into registers; padding rows are identity rows.
template <int B, int NM, class Mem>
__device__ __forceinline__ void row_entry(const DevModel& M, const Mem& w, float (&row)[NM], float& diag,
                                          unsigned mask, V3 fn, V3 ff, float arm, int lane) {
  // every lane reads column B's subspace (a broadcast; padding columns read
  // other scratch) and keeps the product only where DOF B moves an ancestor
  const float p = dot(ld3(w, M.o_S + 6 * B), fn) + dot(ld3(w, M.o_S + 6 * B + 3), ff);
  float v = ((mask >> B) & 1u) ? p : 0.f;
  if (B == lane) {
    v += arm;
    diag = v;
  }
  row[B] = v;
}
template <int NM, class Mem, int... B>
__device__ __forceinline__ void row_assemble(const DevModel& M, const Mem& w, float (&row)[NM], float& diag, int lane,
                                             iseq<B...>) {
  V3 fn = v3(0.f, 0.f, 0.f), ff = v3(0.f, 0.f, 0.f);
  unsigned mask = 0u;
  const bool own = lane < M.nv;
  if (own) {
    const int i = __ldg(M.dof_link + lane);
    si_mul(w, lwork(M, i) + LW_IC, ld3(w, M.o_S + 6 * lane), ld3(w, M.o_S + 6 * lane + 3), fn, ff);
    mask = __ldg(M.anc_mask + lane);
  }
  const float arm = own ? __ldg(M.arm + lane) : 1.f;
  (row_entry<B, NM>(M, w, row, diag, mask, fn, ff, arm, lane), ...);
}
template <int B, int NM, class Mem>
__device__ __forceinline__ void row_store_entry(const DevModel& M, const Mem& w, const float (&row)[NM], int lane) {
  if (B < lane && lane < M.nv) w[M.o_M + lane * M.nv + B] = row[B];
}
template <int NM, class Mem, int... B>
__device__ __forceinline__ void row_store(const DevModel& M, const Mem& w, const float (&row)[NM], int lane,
                                          iseq<B...>) {
  (row_store_entry<B, NM>(M, w, row, lane), ...);
}
template <int B, int NM, class Mem>
__device__ __forceinline__ void row_load_entry(const DevModel& M, const Mem& w, float (&row)[NM], int lane) {
  const bool use = B < lane && lane < M.nv;
  const float v = w[M.o_M + (use ? lane * M.nv + B : 0)];
  row[B] = use ? v : 0.f;
}
template <int NM, class Mem, int... B>
__device__ __forceinline__ void row_load(const DevModel& M, const Mem& w, float (&row)[NM], int lane,
                                         iseq<B...>) {
  (row_load_entry<B, NM>(M, w, row, lane), ...);
}

// Forward substep's dense part: assemble, factor, store the factor, solve
// (M + diag(arm)) qdd = b into o_QDD.  b is lane a's right-hand side.
template <int NM, class Mem>
__device__ __forceinline__ void dense_substep(const DevModel& M, const Mem& w, int lane, int nl, float b) {
  using Seq = make_iseq<NM>;
  const bool own = lane < M.nv;
  float row[NM];
  float diag = 1.f;
  row_assemble<NM>(M, w, row, diag, lane, Seq{});
  float inv_diag = 1.f;
  chol_columns<NM>(row, diag, inv_diag, lane, nl, Seq{});
  row_store<NM>(M, w, row, lane, Seq{});
  if (own) w[M.o_LD + lane] = inv_diag;
  team_sync(nl);
  if (!own) b = 0.f;
  fsub<NM>(row, inv_diag, b, lane, nl, Seq{});
  bsub<NM>(M, w, inv_diag, b, lane, nl, Seq{});
  if (own) w[M.o_QDD + lane] = b;
  team_sync(nl);
}

// x = (L L^T)^{-1} b with the stored factor (o_M strict lower, o_LD = 1/L_kk):
// o_in -> o_out.
template <int NM, class Mem>
__device__ __forceinline__ void dense_stored_solve(const DevModel& M, const Mem& w, int lane, int nl, int o_in,
                                                   int o_out) {
  using Seq = make_iseq<NM>;
  const bool own = lane < M.nv;
  float row[NM];
  row_load<NM>(M, w, row, lane, Seq{});
  const float inv_diag = own ? w[M.o_LD + lane] : 1.f;
  float b = own ? w[o_in + lane] : 0.f;
  fsub<NM>(row, inv_diag, b, lane, nl, Seq{});
  bsub<NM>(M, w, inv_diag, b, lane, nl, Seq{});
  if (own) w[o_out + lane] = b;
  team_sync(nl);
}

// Row capacities of the register path (see dense_class on the host).
#define SHAC_DENSE_CASES(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(20) X(24) X(28) X(32)

template <class Mem>
__device__ __forceinline__ void dense_substep_nm(const DevModel& M, const Mem& w, int lane, int nl, int nm, float b) {
  switch (nm) {
#define SHAC_CASE(N) case N: dense_substep<N>(M, w, lane, nl, b); break;
    SHAC_DENSE_CASES(SHAC_CASE)
#undef SHAC_CASE
    default: break;
  }
}
template <class Mem>
__device__ __forceinline__ void dense_stored_solve_nm(const DevModel& M, const Mem& w, int lane, int nl, int nm,
                                                      int o_in, int o_out) {
  switch (nm) {
#define SHAC_CASE(N) case N: dense_stored_solve<N>(M, w, lane, nl, o_in, o_out); break;
    SHAC_DENSE_CASES(SHAC_CASE)
#undef SHAC_CASE
    default: break;
  }
}

// One forward substep up to the accelerations (integration is separate).
// nm = 0: shared-memory dense stages (any team size, incl. one thread per
// environment); nm > 0: register-resident dense path of that row capacity.
template <class Mem>
__device__ __forceinline__ void substep_dynamics(const DevModel& M, const Mem& w, int lane, int nl, int nm) {
  sw_forward(M, w, lane, nl);
  sw_gather(M, w, lane, nl);
  if (nm > 0) {
    dense_substep_nm(M, w, lane, nl, nm, lane < M.nv ? dof_rhs(M, w, lane) : 0.f);
  } else {
    st_rhs(M, w, lane, nl);
    st_mass_rows(M, w, lane, nl);
    st_chol(M, w, lane, nl);
    st_solve(M, w, lane, nl, M.o_B, M.o_QDD);
  }
}

// Reward on the post-step state (appendix A.3 reward shapes; see shacsim.h).
template <class Mem>
__device__ float reward_value(const DevModel& M, const Mem& w) {
  float r = 0.f;
  for (int j = 0; j < M.nq; ++j) { float q = w[M.o_Q + j]; r -= __ldg(M.rwq + j) * q * q; }
  for (int j = 0; j < M.nv; ++j) { float v = w[M.o_QD + j]; r -= __ldg(M.rwqd + j) * v * v; }
  float a2 = 0.f;
  for (int j = 0; j < M.na; ++j) { float a = w[M.o_ACT + j]; a2 += a * a; }
  r -= M.rc[0] * a2;
  if (M.root_free) {
    M33 R = quat_to_R(w[M.o_Q + 3], w[M.o_Q + 4], w[M.o_Q + 5], w[M.o_Q + 6]);
    V3 vw = mul(R, ld3(w, M.o_QD + 3));
    r += M.rc[1] * vw.x + M.rc[2] * R.m[8] + M.rc[3] * R.m[0];
  } else if (M.vx_dof >= 0) {
    r += M.rc[1] * w[M.o_QD + M.vx_dof];
  }
  if (M.height_q >= 0) {
    float D = fminf(fmaxf(w[M.o_Q + M.height_q] - M.rc[4], M.rc[5]), M.rc[6]);
    r += D < 0.f ? (M.rc[7] * D * D + M.rc[8] * D) : M.rc[9] * D;
  }
  return r;
}

// adjoint of reward_value: accumulate into o_QB, o_QDB, o_ACTB (single lane)
template <class Mem>
__device__ void reward_adjoint(const DevModel& M, const Mem& w, float rb) {
  for (int j = 0; j < M.nq; ++j) w[M.o_QB + j] -= 2.f * __ldg(M.rwq + j) * w[M.o_Q + j] * rb;
  for (int j = 0; j < M.nv; ++j) w[M.o_QDB + j] -= 2.f * __ldg(M.rwqd + j) * w[M.o_QD + j] * rb;
  for (int j = 0; j < M.na; ++j) w[M.o_ACTB + j] -= 2.f * M.rc[0] * w[M.o_ACT + j] * rb;
  if (M.root_free) {
    float x = w[M.o_Q + 3], y = w[M.o_Q + 4], z = w[M.o_Q + 5], qw = w[M.o_Q + 6];
    M33 R = quat_to_R(x, y, z, qw);
    V3 vb = ld3(w, M.o_QD + 3);
    // vx = R row 0 . v_b
    const float cv = M.rc[1] * rb;
    w[M.o_QDB + 3] += cv * R.m[0]; w[M.o_QDB + 4] += cv * R.m[1]; w[M.o_QDB + 5] += cv * R.m[2];
    M33 B;
#pragma unroll
    for (int k = 0; k < 9; ++k) B.m[k] = 0.f;
    B.m[0] = cv * vb.x + M.rc[3] * rb; B.m[1] = cv * vb.y; B.m[2] = cv * vb.z;
    B.m[8] = M.rc[2] * rb;
    float xb = 0.f, yb = 0.f, zb = 0.f, wb = 0.f;
    quat_to_R_adj(x, y, z, qw, B, xb, yb, zb, wb);
    w[M.o_QB + 3] += xb; w[M.o_QB + 4] += yb; w[M.o_QB + 5] += zb; w[M.o_QB + 6] += wb;
  } else if (M.vx_dof >= 0) {
    w[M.o_QDB + M.vx_dof] += M.rc[1] * rb;
  }
  if (M.height_q >= 0) {
    const float raw = w[M.o_Q + M.height_q] - M.rc[4];
    if (raw > M.rc[5] && raw < M.rc[6]) {
      const float dD = raw < 0.f ? (2.f * M.rc[7] * raw + M.rc[8]) : M.rc[9];
      w[M.o_QB + M.height_q] += dD * rb;
    }
  }
}

// Zero a range of scratch (team-parallel).
template <class Mem>
__device__ __forceinline__ void zero_range(const Mem& w, int o, int n, int lane, int nl) {
  for (int k = lane; k < n; k += nl) w[o + k] = 0.f;
}

// ================================================================= ADJOINT ==

// Reverse of lk_integrate for link i.  Inputs: o_Q/o_QD hold the substep
// START state, o_QDD its accelerations, the link records its rotations; o_QB/o_QDB hold the
// cotangents of the substep END state.  Outputs (link i's entries): o_QB/o_QDB
// partial cotangents of the start state (integrator paths only) and
// o_T = qdd_bar.
template <class Mem>
__device__ __forceinline__ void lk_integrate_adj(const DevModel& M, const Mem& w, int i) {
  const float h = M.h;
  const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i), d = __ldg(M.ds + i), nd = __ldg(M.nd + i);
  if (jt == J_REV || jt == J_PRIS) {
    w[M.o_QDB + d] += h * w[M.o_QB + s];          // q' = q + h qd'
  } else if (jt == J_FREE) {
    const M33 R = ldm(w, lrec(M, i) + LR_R);
    const V3 vb1 = ld3(w, M.o_QD + d + 3) + h * ld3(w, M.o_QDD + d + 3);   // new body velocity
    const V3 om1 = ld3(w, M.o_QD + d) + h * ld3(w, M.o_QDD + d);
    const V3 pb = ld3(w, M.o_QB + s);
    // p' = p + h R v_b'
    add3(w, M.o_QDB + d + 3, h * mulT(R, pb));
    M33 B;
    B.m[0] = h * pb.x * vb1.x; B.m[1] = h * pb.x * vb1.y; B.m[2] = h * pb.x * vb1.z;
    B.m[3] = h * pb.y * vb1.x; B.m[4] = h * pb.y * vb1.y; B.m[5] = h * pb.y * vb1.z;
    B.m[6] = h * pb.z * vb1.x; B.m[7] = h * pb.z * vb1.y; B.m[8] = h * pb.z * vb1.z;
    const float x = w[M.o_Q + s + 3], y = w[M.o_Q + s + 4], z = w[M.o_Q + s + 5], qw = w[M.o_Q + s + 6];
    float xb = 0.f, yb = 0.f, zb = 0.f, wb = 0.f;
    quat_to_R_adj(x, y, z, qw, B, xb, yb, zb, wb);
    // quat' = n / |n|, n = quat + h/2 quat (x) (w', 0)
    const V3 u = v3(x, y, z);
    const float hh = 0.5f * h;
    const V3 nu = u + hh * (qw * om1 + cross(u, om1));
    const float nw = qw - hh * dot(u, om1);
    const float inv = 1.f / sqrtf(dot(nu, nu) + nw * nw);
    const V3 qu1 = inv * nu;
    const float qw1 = inv * nw;
    const V3 qub = ld3(w, M.o_QB + s + 3);
    const float qwb = w[M.o_QB + s + 6];
    const float pr = dot(qu1, qub) + qw1 * qwb;
    const V3 nub = inv * (qub - pr * qu1);
    const float nwb = inv * (qwb - pr * qw1);
    const V3 ub = nub + hh * cross(om1, nub) - (hh * nwb) * om1;
    const float wbq = nwb + hh * dot(om1, nub);
    const V3 omb = hh * (qw * nub + cross(nub, u)) - (hh * nwb) * u;
    add3(w, M.o_QDB + d, omb);
    w[M.o_QB + s + 3] = ub.x + xb; w[M.o_QB + s + 4] = ub.y + yb; w[M.o_QB + s + 5] = ub.z + zb;
    w[M.o_QB + s + 6] = wbq + wb;
  }
  for (int k = d; k < d + nd; ++k) w[M.o_T + k] = h * w[M.o_QDB + k];   // qd' = qd + h qdd
}

template <class Mem>
__device__ void st_integrate_adj(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int i = lane; i < M.L; i += nl) lk_integrate_adj(M, w, i);
  team_sync(nl);
}

__device__ __forceinline__ void add_outer(M33& A, V3 a, V3 b) {   // A += a b^T
  A.m[0] += a.x * b.x; A.m[1] += a.x * b.y; A.m[2] += a.x * b.z;
  A.m[3] += a.y * b.x; A.m[4] += a.y * b.y; A.m[5] += a.y * b.z;
  A.m[6] += a.z * b.x; A.m[7] += a.z * b.y; A.m[8] += a.z * b.z;
}

// Adjoint sweep 1 is split like the forward sweep, with w = -lambda as the
// cotangent of tau = S^T F_total (G = ID(q, qd, qdd) + arm qdd - tau_j).
//
// lk_adj_acc, root first: the accelerations A_i = A_p + sum_{d in i} S_d qdd_d
// + V_i x u_i with the solved qdd, and the force cotangent
// F_bar_i = F_bar_p + sum_{d in i} w_d S_d.  c carries (A, F_bar) of the
// parent in registers on entry and link i's on return.
struct AccCarry {
  V3 aw, av, nb, fb;
};
template <class Mem>
__device__ __forceinline__ void acc_parent(const DevModel& M, const Mem& w, int p, AccCarry& c) {
  if (p >= 0) {
    c.aw = ld3(w, lwork(M, p) + LW_A); c.av = ld3(w, lwork(M, p) + LW_A + 3);
    c.nb = ld3(w, lwork(M, p) + LW_FB); c.fb = ld3(w, lwork(M, p) + LW_FB + 3);
  } else {
    c.aw = c.nb = c.fb = v3(0.f, 0.f, 0.f);
    c.av = v3(-M.grav[0], -M.grav[1], -M.grav[2]);
  }
}
template <class Mem>
__device__ __forceinline__ void lk_adj_acc(const DevModel& M, const Mem& w, int i, AccCarry& c) {
  const int d0 = __ldg(M.ds + i), nd = __ldg(M.nd + i);
  const V3 Vw = ld3(w, lrec(M, i) + LR_V), Vv = ld3(w, lrec(M, i) + LR_V + 3);
  V3 aw = c.aw, av = c.av, nb = c.nb, fb = c.fb;
  V3 uw = v3(0.f, 0.f, 0.f), uv = v3(0.f, 0.f, 0.f);
  for (int d = d0; d < d0 + nd; ++d) {
    const V3 sw = ld3(w, M.o_S + 6 * d), sv = ld3(w, M.o_S + 6 * d + 3);
    const float qd = w[M.o_QD + d], qdd = w[M.o_QDD + d], lam = w[M.o_LAM + d];
    uw = uw + qd * sw; uv = uv + qd * sv;
    aw = aw + qdd * sw; av = av + qdd * sv;
    nb = nb - lam * sw; fb = fb - lam * sv;
  }
  aw = aw + cross(Vw, uw);
  av = av + cross(Vw, uv) + cross(Vv, uw);
  st3(w, lwork(M, i) + LW_A, aw); st3(w, lwork(M, i) + LW_A + 3, av);
  st3(w, lwork(M, i) + LW_FB, nb); st3(w, lwork(M, i) + LW_FB + 3, fb);
  c.aw = aw; c.av = av; c.nb = nb; c.fb = fb;
}

// Team form of adjoint sweep 1: link i's own terms of (A, F_bar) (its DOFs'
// S qdd and -lambda S, V_i x u_i and, for a root, the base acceleration -g),
// which ancestor_sums over [A, F_bar] then turn into the recursion's values.
template <class Mem>
__device__ __forceinline__ void lk_adj_acc_own(const DevModel& M, const Mem& w, int i) {
  AccCarry c;
  acc_parent(M, w, -1, c);
  if (__ldg(M.parent + i) >= 0) c.av = v3(0.f, 0.f, 0.f);
  lk_adj_acc(M, w, i, c);
}

// Cotangent of the spatial inertia from y = I x (y_bar given): h_bar and the
// (full 3 x 3) cotangent G of Io, accumulated in registers (no mass
// cotangent: masses are constants).
__device__ __forceinline__ void si_adj(V3& hb, M33& G, V3 xw, V3 xv, V3 yn_b, V3 yf_b) {
  hb = hb + cross(xv, yn_b) + cross(yf_b, xw);
  add_outer(G, yn_b, xw);
}

// The joint forces of DOF d (actuation, limit penalty, damping): their
// cotangents from tau_bar = lambda_d.  One lane per DOF, in the same pass as
// lk_adj_local (the two write disjoint scratch).
template <class Mem>
__device__ __forceinline__ void dof_adj_force(const DevModel& M, const Mem& w, int d) {
  const float lam = w[M.o_LAM + d];
  const int a = __ldg(M.dof_act + d);
  if (a >= 0) w[M.o_ACTB + a] += lam * __ldg(M.gear + d);
  const int i = __ldg(M.dof_link + d), jt = __ldg(M.jtype + i);
  if (jt == J_REV || jt == J_PRIS) {
    const int s = __ldg(M.qs + i);
    const float q = w[M.o_Q + s];
    if (q < __ldg(M.qlo + d) || q > __ldg(M.qhi + d)) w[M.o_QB + s] -= lam * M.klim;
  }
  w[M.o_QDB + d] -= lam * __ldg(M.damp + d);
}

// lk_adj_local, one lane per link, everything of adjoint sweep 1 that is local
// to link i but its DOFs' joint forces (dof_adj_force): the local force
// F_i = I A + V x* (I V) - Fext recomputed with the solved accelerations; the
// reverse of F_i (A_bar = I F_bar, V_bar and the inertia cotangent, carried
// through h = m c, Io = R Ic R^T + m(|c|^2 1 - c c^T), c = P + R com to the
// pose); and the reverse of link i's contacts (their external wrench enters
// F_i with a minus).  Stores link i's V_bar, R_bar and P_bar accumulators.
template <bool KEEP_RLOCAL, class Mem>
__device__ __forceinline__ void lk_adj_local(const DevModel& M, const Mem& w, int i) {
  const int jt = __ldg(M.jtype + i);
  const int osi = lrec(M, i) + LR_SI;
  const float m = w[osi];
  const V3 h = ld3(w, osi + 1);
  const float ixx = w[osi + 4], iyy = w[osi + 5], izz = w[osi + 6], ixy = w[osi + 7], ixz = w[osi + 8],
              iyz = w[osi + 9];
  auto imul = [&](V3 xw, V3 xv, V3& yn, V3& yf) {
    yn = v3(ixx * xw.x + ixy * xw.y + ixz * xw.z, ixy * xw.x + iyy * xw.y + iyz * xw.z,
            ixz * xw.x + iyz * xw.y + izz * xw.z) + cross(h, xv);
    yf = m * xv - cross(h, xw);
  };
  const V3 Vw = ld3(w, lrec(M, i) + LR_V), Vv = ld3(w, lrec(M, i) + LR_V + 3);
  const V3 aw = ld3(w, lwork(M, i) + LW_A), av = ld3(w, lwork(M, i) + LW_A + 3);
  const V3 nb = ld3(w, lwork(M, i) + LW_FB), fb = ld3(w, lwork(M, i) + LW_FB + 3);
  {
    V3 fn, ff, bn, bf;
    imul(aw, av, fn, ff);
    imul(Vw, Vv, bn, bf);
    fn = fn + cross(Vw, bn) + cross(Vv, bf) - ld3(w, lrec(M, i) + LR_FX);
    ff = ff + cross(Vw, bf) - ld3(w, lrec(M, i) + LR_FX + 3);
    st3(w, lwork(M, i) + LW_F, fn); st3(w, lwork(M, i) + LW_F + 3, ff);
  }
  // A_bar = I F_bar (I symmetric)
  V3 abn, abf;
  imul(nb, fb, abn, abf);
  st3(w, lwork(M, i) + LW_AB, abn);
  st3(w, lwork(M, i) + LW_AB + 3, abf);
  V3 hb = v3(0.f, 0.f, 0.f);
  M33 G;
#pragma unroll
  for (int k = 0; k < 9; ++k) G.m[k] = 0.f;
  si_adj(hb, G, aw, av, nb, fb);
  // momentum B = I V and V x* B
  V3 Bn, Bf;
  imul(Vw, Vv, Bn, Bf);
  V3 vwb = cross(Bn, nb) + cross(Bf, fb);
  V3 vvb = cross(Bf, nb);
  const V3 Bnb = cross(nb, Vw);
  const V3 Bfb = cross(nb, Vv) + cross(fb, Vw);
  V3 t1, t2;
  imul(Bnb, Bfb, t1, t2);
  vwb = vwb + t1;
  vvb = vvb + t2;
  si_adj(hb, G, Vw, Vv, Bnb, Bfb);
  // spatial inertia about the reference point -> pose cotangents
  const M33 R = ldm(w, lrec(M, i) + LR_R);
  const V3 P = ld3(w, lrec(M, i) + LR_P);
  V3 Pb = v3(0.f, 0.f, 0.f);
  M33 Rb;
#pragma unroll
  for (int k = 0; k < 9; ++k) Rb.m[k] = 0.f;
  if (m != 0.f || __ldg(M.icom + 6 * i) != 0.f || __ldg(M.icom + 6 * i + 1) != 0.f || __ldg(M.icom + 6 * i + 2) != 0.f) {
    const V3 com = cld3(M.com + 3 * i);
    const V3 c = P + mul(R, com);
    const float trG = G.m[0] + G.m[4] + G.m[8];
    M33 Gs;   // G + G^T
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Gs.m[3 * a + b] = G.m[3 * a + b] + G.m[3 * b + a];
    const V3 cb = m * hb + m * (2.f * trG * c - mul(Gs, c));
    Rb = mul(mul(Gs, R), com_inertia(M, i));
    Pb = cb;
    add_outer(Rb, cb, com);
  }
  // contacts of link i: Fext cotangent = -F_bar
  const int k0 = __ldg(M.lc_ptr + i), k1 = __ldg(M.lc_ptr + i + 1);
  for (int k = k0; k < k1; ++k) {
    const int c = __ldg(M.lc_idx + k);
    const float dep = w[M.o_IT + 7 * c + 6];
    float db = 0.f;
    if (dep < 0.f) {
      const V3 x = ld3(w, M.o_IT + 7 * c), f = ld3(w, M.o_IT + 7 * c + 3);
      const V3 neb = -nb, feb = -fb;
      const V3 fbar = cross(neb, x) + feb;
      V3 xb = cross(f, neb);
      const V3 vp = Vv + cross(Vw, x);
      const float fn = f.z;
      const float vt = sqrtf(vp.x * vp.x + vp.y * vp.y);
      const float afn = fabsf(fn);
      float fnb = fbar.z;
      V3 vpb = v3(0.f, 0.f, 0.f);
      if (M.kt * vt <= M.mu * afn) {
        vpb.x = -M.kt * fbar.x;
        vpb.y = -M.kt * fbar.y;
      } else {
        const float sc = M.mu * afn / vt;
        const float sb = -(fbar.x * vp.x + fbar.y * vp.y);
        vpb.x = -sc * fbar.x;
        vpb.y = -sc * fbar.y;
        fnb += sb * M.mu * (fn >= 0.f ? 1.f : -1.f) / vt;
        const float vtb = -sb * sc / vt;
        vpb.x += vtb * vp.x / vt;
        vpb.y += vtb * vp.y / vt;
      }
      // fn = (-ke + kd ddot) d, d = x.z + root height
      db = fnb * (-M.ke + M.kd * vp.z);
      xb.z += db;
      vpb.z += fnb * M.kd * dep;
      vwb = vwb + cross(x, vpb);
      vvb = vvb + vpb;
      xb = xb + cross(vpb, Vw);
      Pb = Pb + xb;
      add_outer(Rb, xb, cld3(M.item_pos + 3 * c));
    }
    w[M.o_ITB + 10 * c + 9] = db;
  }
  st3(w, lwork(M, i) + LW_VB, vwb);
  st3(w, lwork(M, i) + LW_VB + 3, vvb);
  st3(w, lwork(M, i) + LW_PB, Pb);
  stm(w, lwork(M, i) + LW_RB, Rb);
  // joint-local rotation R_local = jrot Rot(axis, q) of a revolute joint with
  // a parent, kept in link i's pose-cotangent slot until the leaves-first
  // chain sweep replaces it (the team form's world-frame sums need none)
  if (KEEP_RLOCAL && jt == J_REV && __ldg(M.parent + i) >= 0)
    stm(w, lwork(M, i) + LW_TP, mul(cldm(M.jrot + 9 * i), axis_angle(cld3(M.axis + 3 * i), w[M.o_Q + __ldg(M.qs + i)])));
}

// Reverse of one muscle segment: cotangents of both via points and of the
// activation (stored per segment).
template <class Mem>
__device__ __forceinline__ void seg_adjoint(const DevModel& M, const Mem& w, int sg) {
  const int e0 = M.nc + 2 * sg, e1 = e0 + 1;
  const int l0 = __ldg(M.item_link + e0), l1 = __ldg(M.item_link + e1);
  const V3 x0 = ld3(w, M.o_IT + 7 * e0), f0 = ld3(w, M.o_IT + 7 * e0 + 3);
  const V3 x1 = ld3(w, M.o_IT + 7 * e1), f1 = ld3(w, M.o_IT + 7 * e1 + 3);
  const V3 n0b = -ld3(w, lwork(M, l0) + LW_FB), f0eb = -ld3(w, lwork(M, l0) + LW_FB + 3);
  const V3 n1b = -ld3(w, lwork(M, l1) + LW_FB), f1eb = -ld3(w, lwork(M, l1) + LW_FB + 3);
  const V3 f0b = cross(n0b, x0) + f0eb, f1b = cross(n1b, x1) + f1eb;
  V3 x0b = cross(f0, n0b), x1b = cross(f1, n1b);
  const int mu_ = __ldg(M.seg_mus + sg);
  const float araw = w[M.o_ACT + M.ntact + mu_];
  const float a = fminf(fmaxf(araw, 0.f), 1.f);
  const float fm = __ldg(M.fmax + mu_);
  const float F = a * fm;
  const V3 dv = x1 - x0;
  const float len = sqrtf(dot(dv, dv));
  const V3 u = (1.f / len) * dv;
  const V3 g = f0b - f1b;
  const V3 ub = F * g;
  const float Fb = dot(u, g);
  const V3 dvb = (1.f / len) * (ub - dot(u, ub) * u);
  x1b = x1b + dvb;
  x0b = x0b - dvb;
  w[M.o_SEGA + sg] = (araw > 0.f && araw < 1.f) ? Fb * fm : 0.f;
  st3(w, M.o_ITB + 10 * e0, x0b);
  st3(w, M.o_ITB + 10 * e1, x1b);
}

// Children's contributions carried up a chain in registers: subtree sums of
// the total force and of A_bar, the child's V_bar and its cotangent of this
// link's pose (what the pose-cotangent slot holds for a chain head).
struct BwdCarry {
  V3 Fn, Ff, an, af, vw, vv, tP;
  M33 tR;
};

// Adjoint sweep 2 (leaves first), chain form (one thread), at link i: gather the children (total
// forces, A_bar, V_bar, kinematic cotangents; inside a chain the only child
// is the link walked before, carried in g), reverse the Newton-Euler
// accelerations and velocities and the motion subspaces, and pass the pose
// cotangent through the joint transform to the parent (R_p_bar, P_p_bar in
// the pose-cotangent slot).  The inertia's share of the pose cotangents was added by
// lk_adj_local; the joint's own q_bar is taken after the sweep (lk_adj_qbar)
// from the final R_bar, P_bar left in its work record.
template <class Mem>
__device__ __forceinline__ void lk_adj_bwd(const DevModel& M, const Mem& w, int i, bool tail, BwdCarry& g) {
  V3 Fn = ld3(w, lwork(M, i) + LW_F), Ff = ld3(w, lwork(M, i) + LW_F + 3);
  V3 an = ld3(w, lwork(M, i) + LW_AB), af = ld3(w, lwork(M, i) + LW_AB + 3);
  V3 vw = ld3(w, lwork(M, i) + LW_VB), vv = ld3(w, lwork(M, i) + LW_VB + 3);
  M33 Rb = ldm(w, lwork(M, i) + LW_RB);
  V3 Pb = ld3(w, lwork(M, i) + LW_PB);
  V3 cvw = v3(0.f, 0.f, 0.f), cvv = v3(0.f, 0.f, 0.f);
  if (tail) {
    const int c0 = __ldg(M.ch_ptr + i), c1 = __ldg(M.ch_ptr + i + 1);
    for (int k = c0; k < c1; ++k) {
      const int c = __ldg(M.ch_idx + k);
      Fn = Fn + ld3(w, lwork(M, c) + LW_F);
      Ff = Ff + ld3(w, lwork(M, c) + LW_F + 3);
      an = an + ld3(w, lwork(M, c) + LW_AB);
      af = af + ld3(w, lwork(M, c) + LW_AB + 3);
      cvw = cvw + ld3(w, lwork(M, c) + LW_VB);
      cvv = cvv + ld3(w, lwork(M, c) + LW_VB + 3);
#pragma unroll
      for (int t = 0; t < 9; ++t) Rb.m[t] += w[lwork(M, c) + LW_TP + t];
      Pb = Pb + ld3(w, lwork(M, c) + LW_TP + 9);
    }
  } else {
    Fn = Fn + g.Fn; Ff = Ff + g.Ff;
    an = an + g.an; af = af + g.af;
    cvw = g.vw; cvv = g.vv;
#pragma unroll
    for (int t = 0; t < 9; ++t) Rb.m[t] += g.tR.m[t];
    Pb = Pb + g.tP;
  }
  // the rest of link i's scratch reads come before its first store
  V3 uw, uv;
  joint_vel(M, w, i, uw, uv);
  const V3 Vw = ld3(w, lrec(M, i) + LR_V), Vv = ld3(w, lrec(M, i) + LR_V + 3);
  const M33 R = ldm(w, lrec(M, i) + LR_R);
  const V3 P = ld3(w, lrec(M, i) + LR_P);
  const int jt = __ldg(M.jtype + i), d0 = __ldg(M.ds + i), nd = __ldg(M.nd + i);
  const int p = __ldg(M.parent + i);
  M33 Rloc;   // joint-local rotation kept in the pose-cotangent slot by lk_adj_local (revolute with a parent)
  if (jt == J_REV && p >= 0) Rloc = ldm(w, lwork(M, i) + LW_TP);
  float lam1 = 0.f, qdd1 = 0.f, qd1 = 0.f, qdb1 = 0.f;   // a one-DOF joint's terms
  V3 s1w = v3(0.f, 0.f, 0.f), s1v = v3(0.f, 0.f, 0.f);
  if (jt != J_FREE && nd == 1) {
    lam1 = w[M.o_LAM + d0]; qdd1 = w[M.o_QDD + d0]; qd1 = w[M.o_QD + d0]; qdb1 = w[M.o_QDB + d0];
    s1w = ld3(w, M.o_S + 6 * d0); s1v = ld3(w, M.o_S + 6 * d0 + 3);
  }
  st3(w, lwork(M, i) + LW_F, Fn);
  st3(w, lwork(M, i) + LW_F + 3, Ff);
  st3(w, lwork(M, i) + LW_AB, an);
  st3(w, lwork(M, i) + LW_AB + 3, af);
  // A_i = A_p + sum S qdd + V_i x u_i
  vw = vw + cross(uw, an) + cross(uv, af) + cvw;
  vv = vv + cross(uw, af) + cvv;
  st3(w, lwork(M, i) + LW_VB, vw);
  st3(w, lwork(M, i) + LW_VB + 3, vv);
  const V3 ubw = cross(an, Vw) + cross(af, Vv);
  const V3 ubv = cross(af, Vw);
  // motion subspaces of the DOFs of i: tau = S^T F_total, A and V terms
  const V3 ax = cld3(M.axis + 3 * i);
  if (jt == J_FREE) {
    // a free joint is the root: its six DOF terms feed only its own q_bar, so
    // they run after the sweep, one DOF per lane (root_dof_terms)
  } else if (nd == 1) {
    const float wd = -lam1;
    w[M.o_QDB + d0] = qdb1 + (dot(s1w, ubw + vw) + dot(s1v, ubv + vv));
    const V3 sbw = wd * Fn + qdd1 * an + qd1 * (ubw + vw);
    const V3 sbv = wd * Ff + qdd1 * af + qd1 * (ubv + vv);
    V3 ab;
    if (jt == J_REV) {   // (a, P x a), a = R ax
      const V3 a = mul(R, ax);
      ab = sbw + cross(sbv, P);
      Pb = Pb + cross(a, sbv);
    } else {             // (0, a)
      ab = sbv;
    }
    add_outer(Rb, ab, ax);
  }
  stm(w, lwork(M, i) + LW_RB, Rb);
  st3(w, lwork(M, i) + LW_PB, Pb);
  g.Fn = Fn; g.Ff = Ff; g.an = an; g.af = af; g.vw = vw; g.vv = vv;
  if (p >= 0 && jt != J_FREE) {
    // Rj = Rp jrot (joint frame in world), R = Rj Rot(ax, q), Pj = Pp + Rp jpos
    M33 tp;
    if (jt == J_REV) {
      tp = mulBT(Rb, Rloc);   // R_p_bar = R_bar R_local^T
    } else {
      M33 Rjb = Rb;
      if (jt == J_PRIS) add_outer(Rjb, w[M.o_Q + __ldg(M.qs + i)] * Pb, ax);   // P = Pj + q Rj ax
      tp = mulBT(Rjb, cldm(M.jrot + 9 * i));
    }
    add_outer(tp, Pb, cld3(M.jpos + 3 * i));
    stm(w, lwork(M, i) + LW_TP, tp);
    st3(w, lwork(M, i) + LW_TP + 9, Pb);
    g.tR = tp;
    g.tP = Pb;
  }
}

// Team form of adjoint sweep 2 (leaves first): every recursion of lk_adj_bwd
// as subtree sums of the links' own terms.  F_total and A_bar are sums of the
// links' own values; V_bar_i = V_bar_own_i + (terms of u_i and A_bar_i) + the
// children's V_bar is a sum of lk_adj_vbar_own's terms.  The pose cotangents
// pass through the joint transforms (R_i = R_p R_local, P_i = P_p + R_p P_local):
// with the world-frame moment Q_k = R_bar_k R_k^T + P_bar_k P_k^T of each link's
// own cotangents, the total of link p is
//   R_bar_p = (sum_{k in sub(p)} Q_k - (sum_{k in sub(p)} P_bar_k) P_p^T) R_p,
//   P_bar_p = sum_{k in sub(p)} P_bar_k,
// because R_local^T R_p^T = R_c^T and R_p P_local = P_c - P_p telescope along
// every path of the subtree; so no transform runs along the tree.
template <class Mem>
__device__ __forceinline__ void lk_adj_vbar_own(const DevModel& M, const Mem& w, int i) {
  V3 uw, uv;
  joint_vel(M, w, i, uw, uv);
  const V3 an = ld3(w, lwork(M, i) + LW_AB), af = ld3(w, lwork(M, i) + LW_AB + 3);
  add3(w, lwork(M, i) + LW_VB, cross(uw, an) + cross(uv, af));
  add3(w, lwork(M, i) + LW_VB + 3, cross(uw, af));
}

// After the F, A_bar and V_bar sums: link i's one-DOF joint terms (qd_bar and
// the subspace cotangent's share of the pose cotangents; a free root's six DOFs
// run in root_dof_terms), then its moment Q_i over R_bar (P_bar stays).
template <class Mem>
__device__ __forceinline__ void lk_adj_pose(const DevModel& M, const Mem& w, int i) {
  const int ow = lwork(M, i), orc = lrec(M, i);
  M33 Rb = ldm(w, ow + LW_RB);
  V3 Pb = ld3(w, ow + LW_PB);
  const M33 R = ldm(w, orc + LR_R);
  const V3 P = ld3(w, orc + LR_P);
  const int jt = __ldg(M.jtype + i), nd = __ldg(M.nd + i);
  if (jt != J_FREE && nd == 1) {
    const int d0 = __ldg(M.ds + i);
    const V3 Fn = ld3(w, ow + LW_F), Ff = ld3(w, ow + LW_F + 3);
    const V3 an = ld3(w, ow + LW_AB), af = ld3(w, ow + LW_AB + 3);
    const V3 Vw = ld3(w, orc + LR_V), Vv = ld3(w, orc + LR_V + 3);
    const V3 s1w = ld3(w, M.o_S + 6 * d0), s1v = ld3(w, M.o_S + 6 * d0 + 3);
    const float wd = -w[M.o_LAM + d0], qdd1 = w[M.o_QDD + d0], qd1 = w[M.o_QD + d0];
    const V3 uw = cross(an, Vw) + cross(af, Vv) + ld3(w, ow + LW_VB);
    const V3 uv = cross(af, Vw) + ld3(w, ow + LW_VB + 3);
    w[M.o_QDB + d0] += dot(s1w, uw) + dot(s1v, uv);
    const V3 sbw = wd * Fn + qdd1 * an + qd1 * uw;
    const V3 sbv = wd * Ff + qdd1 * af + qd1 * uv;
    const V3 ax = cld3(M.axis + 3 * i);
    V3 ab;
    if (jt == J_REV) {   // (a, P x a), a = R ax
      ab = sbw + cross(sbv, P);
      Pb = Pb + cross(mul(R, ax), sbv);
    } else {             // (0, a)
      ab = sbv;
    }
    add_outer(Rb, ab, ax);
  }
  M33 Q = mulBT(Rb, R);
  add_outer(Q, Pb, P);
  stm(w, ow + LW_RB, Q);
  st3(w, ow + LW_PB, Pb);
}

// The free root's DOF d (0..5) after the leaves-first sweep: tau = S^T F_total
// gives qd_bar_d and the subspace cotangents (sbw, sbv), whose share of the
// root's rotation cotangent (column d mod 3: (R e_k, P x R e_k) for the body
// rates, (0, R e_k) for v_body) is kept in o_RDB for lk_adj_qbar.  The root's
// position cotangent is not needed (the root origin is the reference point).
template <class Mem>
__device__ __forceinline__ void root_dof_terms(const DevModel& M, const Mem& w, int d) {
  const V3 Fn = ld3(w, lwork(M, 0) + LW_F), Ff = ld3(w, lwork(M, 0) + LW_F + 3);
  const V3 an = ld3(w, lwork(M, 0) + LW_AB), af = ld3(w, lwork(M, 0) + LW_AB + 3);
  const V3 Vw = ld3(w, lrec(M, 0) + LR_V), Vv = ld3(w, lrec(M, 0) + LR_V + 3);
  // cotangent of the root's velocity terms: V_bar plus the V x u part of A
  const V3 uw = cross(an, Vw) + cross(af, Vv) + ld3(w, lwork(M, 0) + LW_VB);
  const V3 uv = cross(af, Vw) + ld3(w, lwork(M, 0) + LW_VB + 3);
  const float wd = -w[M.o_LAM + d], qdd = w[M.o_QDD + d], qd = w[M.o_QD + d];
  const V3 sw = ld3(w, M.o_S + 6 * d), sv = ld3(w, M.o_S + 6 * d + 3);
  w[M.o_QDB + d] += dot(sw, uw) + dot(sv, uv);
  const V3 sbw = wd * Fn + qdd * an + qd * uw;
  const V3 sbv = wd * Ff + qdd * af + qd * uv;
  st3(w, M.o_RDB + 3 * d, d < 3 ? sbw + cross(sbv, ld3(w, lrec(M, 0) + LR_P)) : sbv);
}

// q_bar of link i's joint from its final pose cotangents: revolute
// dR/dq = [a]x R with a = R ax; prismatic dP/dq = a; free root: the
// quaternion's share through R(quat), and the root height receives every
// contact depth's cotangent (depth = x.z + root height).
// WORLD: the R_bar slot holds the subtree sum of Q and the P_bar slot that of
// P_bar (team form); R_bar = (Q - P_bar P^T) R is formed first.
template <bool WORLD, class Mem>
__device__ __forceinline__ void lk_adj_qbar(const DevModel& M, const Mem& w, int i) {
  const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i);
  M33 Rb = ldm(w, lwork(M, i) + LW_RB);
  if (WORLD) {
    if (jt == J_FIXED) return;
    add_outer(Rb, -ld3(w, lwork(M, i) + LW_PB), ld3(w, lrec(M, i) + LR_P));
    Rb = mul(Rb, ldm(w, lrec(M, i) + LR_R));
  }
  if (jt == J_FREE) {   // the root origin is the reference point: no position cotangent here
#pragma unroll
    for (int k = 0; k < 3; ++k) {   // the six DOF terms' shares, column k from DOFs k and 3 + k
      const V3 a = ld3(w, M.o_RDB + 3 * k), b = ld3(w, M.o_RDB + 3 * (3 + k));
      Rb.m[k] += a.x; Rb.m[3 + k] += a.y; Rb.m[6 + k] += a.z;
      Rb.m[k] += b.x; Rb.m[3 + k] += b.y; Rb.m[6 + k] += b.z;
    }
    float xb = 0.f, yb = 0.f, zb = 0.f, wb = 0.f;
    quat_to_R_adj(w[M.o_Q + s + 3], w[M.o_Q + s + 4], w[M.o_Q + s + 5], w[M.o_Q + s + 6], Rb, xb, yb, zb, wb);
    w[M.o_QB + s + 3] += xb; w[M.o_QB + s + 4] += yb; w[M.o_QB + s + 5] += zb; w[M.o_QB + s + 6] += wb;
    if (M.root_free && i == 0) {
      float sd = 0.f;
      for (int c = 0; c < M.nc; ++c) sd += w[M.o_ITB + 10 * c + 9];
      w[M.o_QB + 2] += sd;
    }
  } else if (jt == J_REV) {
    const M33 R = ldm(w, lrec(M, i) + LR_R);
    const V3 a = mul(R, cld3(M.axis + 3 * i));
    float qb = 0.f;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const V3 dcol = cross(a, col(R, cc));
      qb += Rb.m[cc] * dcol.x + Rb.m[3 + cc] * dcol.y + Rb.m[6 + cc] * dcol.z;
    }
    w[M.o_QB + s] += qb;
  } else if (jt == J_PRIS) {
    const M33 R = ldm(w, lrec(M, i) + LR_R);
    w[M.o_QB + s] += dot(ld3(w, lwork(M, i) + LW_PB), mul(R, cld3(M.axis + 3 * i)));
  }
}

// Adjoint of the dynamics solve: given o_T = qdd_bar and the recomputed
// substep (o_QDD holds the solved accelerations, o_M/o_LD the factor), add
// -lambda^T dG/d(q, qd, a) to o_QB, o_QDB, o_ACTB with lambda = M^{-1} qdd_bar.
template <class Mem>
__device__ __forceinline__ void st_dynamics_adj(const DevModel& M, const Mem& w, int lane, int nl, int nm) {
  if (nm > 0) {
    dense_stored_solve_nm(M, w, lane, nl, nm, M.o_T, M.o_LAM);
  } else {
    for (int d = lane; d < M.nv; d += nl) w[M.o_B + d] = w[M.o_T + d];
    team_sync(nl);
    st_solve(M, w, lane, nl, M.o_B, M.o_LAM);
  }
  // root first: accelerations with the solved qdd and force cotangents (a
  // team: each link's own terms, then ancestor sums; one thread: chain walks
  // with register carries)
  if (nl > 1) {
    for (int i = lane; i < M.L; i += nl) lk_adj_acc_own(M, w, i);
    team_sync(nl);
    ancestor_sums<12>(M, w, LW_A, lane, nl);
    team_sync(nl);
  } else {
    for (int l = 0; l < M.nlev; ++l) {
      for (int ii = __ldg(M.lvl_ptr + l); ii < __ldg(M.lvl_ptr + l + 1); ++ii) {
        const int hd = __ldg(M.lvl_link + ii), tl = __ldg(M.chain_tail + hd);
        AccCarry c;
        acc_parent(M, w, __ldg(M.parent + hd), c);
        for (int i = hd;; i = chain_next(M, i)) {
          lk_adj_acc(M, w, i, c);
          if (i == tl) break;
        }
      }
    }
  }
  // one pass: links from the first lane up, DOFs' joint forces from the last
  // lane down (a free root's six DOFs do not load the root's lane)
  if (nl > 1) {
    for (int i = lane; i < M.L; i += nl) lk_adj_local<false>(M, w, i);
  } else {
    for (int i = 0; i < M.L; ++i) lk_adj_local<true>(M, w, i);
  }
  for (int d = nl - 1 - lane; d < M.nv; d += nl) dof_adj_force(M, w, d);
  team_sync(nl);
  if (M.nseg > 0) {
    for (int sg = lane; sg < M.nseg; sg += nl) seg_adjoint(M, w, sg);
    team_sync(nl);
    for (int mu_ = lane; mu_ < M.nm; mu_ += nl) {
      float sa = 0.f;
      for (int sg = __ldg(M.mus_seg_ptr + mu_); sg < __ldg(M.mus_seg_ptr + mu_ + 1); ++sg) sa += w[M.o_SEGA + sg];
      w[M.o_ACTB + M.ntact + mu_] += sa;
    }
    // each link's via-point pose cotangents in `parts` partial sums, then
    // added in part order
    const int parts = muscle_parts(M, nl);
    for (int sl = lane; sl < M.L * parts; sl += nl) {
      const int i = sl / parts, r = sl % parts;
      V3 Pb = v3(0.f, 0.f, 0.f);
      M33 Rb;
#pragma unroll
      for (int k = 0; k < 9; ++k) Rb.m[k] = 0.f;
      for (int k = __ldg(M.lm_ptr + i) + r; k < __ldg(M.lm_ptr + i + 1); k += parts) {
        const int e = __ldg(M.lm_idx + k);
        const V3 xb = ld3(w, M.o_ITB + 10 * e);
        Pb = Pb + xb;
        add_outer(Rb, xb, cld3(M.item_pos + 3 * e));
      }
      st3(w, M.o_MW + 12 * sl, Pb);
      stm(w, M.o_MW + 12 * sl + 3, Rb);
    }
    team_sync(nl);
    for (int i = lane; i < M.L; i += nl) {
      V3 Pb = v3(0.f, 0.f, 0.f);
      M33 Rb;
#pragma unroll
      for (int k = 0; k < 9; ++k) Rb.m[k] = 0.f;
      for (int r = 0; r < parts; ++r) {
        const int o = M.o_MW + 12 * (i * parts + r);
        Pb = Pb + ld3(w, o);
#pragma unroll
        for (int k = 0; k < 9; ++k) Rb.m[k] += w[o + 3 + k];
      }
      add3(w, lwork(M, i) + LW_PB, Pb);
#pragma unroll
      for (int k = 0; k < 9; ++k) w[lwork(M, i) + LW_RB + k] += Rb.m[k];
    }
    team_sync(nl);
  }
  if (nl > 1) {
    // leaves first as subtree sums of world-frame terms (lk_adj_vbar_own,
    // lk_adj_pose): F_total and A_bar, V_bar, then the pose moments
    subtree_sums<12>(M, w, LW_F, lane, nl);
    team_sync(nl);
    for (int i = lane; i < M.L; i += nl) lk_adj_vbar_own(M, w, i);
    team_sync(nl);
    subtree_sums<6>(M, w, LW_VB, lane, nl);
    team_sync(nl);
    for (int i = lane; i < M.L; i += nl) lk_adj_pose(M, w, i);
    if (M.root_free)   // the root's DOFs on the lanes counted down from the last
      for (int d = nl - 1 - lane; d < 6; d += nl) root_dof_terms(M, w, d);
    team_sync(nl);
    subtree_sums<12>(M, w, LW_RB, lane, nl);
    team_sync(nl);
    for (int i = lane; i < M.L; i += nl) lk_adj_qbar<true>(M, w, i);
    team_sync(nl);
    return;
  }
  for (int l = M.nlev - 1; l >= 0; --l) {
    for (int ii = __ldg(M.lvl_ptr + l); ii < __ldg(M.lvl_ptr + l + 1); ++ii) {
      const int hd = __ldg(M.lvl_link + ii), tl = __ldg(M.chain_tail + hd);
      BwdCarry g;
      for (int i = tl;; i = __ldg(M.parent + i)) {
        lk_adj_bwd(M, w, i, i == tl, g);
        if (i == hd) break;
      }
    }
  }
  if (M.root_free)
    for (int d = 0; d < 6; ++d) root_dof_terms(M, w, d);
  for (int i = 0; i < M.L; ++i) lk_adj_qbar<false>(M, w, i);
}

// One reverse substep: o_Q/o_QD hold the substep start state, o_QB/o_QDB the
// cotangents of its end state; on return they hold the start-state cotangents,
// and o_ACTB has accumulated the action cotangent.
template <class Mem>
__device__ void substep_adjoint(const DevModel& M, const Mem& w, int lane, int nl, int nm) {
  substep_dynamics(M, w, lane, nl, nm);     // recompute; the factor is kept for lambda
  st_integrate_adj(M, w, lane, nl);
  st_dynamics_adj(M, w, lane, nl, nm);
}

// non-finite check of the state (one lane)
template <class Mem>
__device__ __forceinline__ bool state_finite(const DevModel& M, const Mem& w) {
  bool ok = true;
  for (int j = 0; j < M.nq; ++j) ok &= isfinite(w[M.o_Q + j]);
  for (int j = 0; j < M.nv; ++j) ok &= isfinite(w[M.o_QD + j]);
  return ok;
}

}  // namespace shac
