// Per-environment simulator stages and their adjoints (FP32, sm_103a).
//
// The simulator step F (paper Sec. 3.1) is evaluated with spatial (6-D)
// vectors expressed in world coordinates at the world origin (Plücker
// coordinates, angular part first): with that choice the motion subspaces,
// spatial inertias and forces of all links live in one frame, so the
// composite-rigid-body mass matrix needs no frame transforms and the
// Newton-Euler recursion is a plain sum along the tree.
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
// phases.  With nl = 1 (one environment per thread, PLAIN form) the loops
// are the serial algorithm and team_sync() is a no-op; the BATCHED form runs
// teams of 1..32 lanes inside a warp on shared-memory scratch.  Each phase
// writes any given scratch slot from exactly one lane, so results do not
// depend on the team size beyond floating-point reassociation of the sums
// that a team performs in a different order (there is none: every
// reduction below is a fixed-order gather).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace shac {

enum { J_FREE = 0, J_REV = 1, J_PRIS = 2, J_FIXED = 3 };
enum { FLAG_NONFINITE = 1u };

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
  // links
  const int *parent, *jtype, *qs, *ds, *nd;
  const int *lvl_ptr, *lvl_link;         // links grouped by depth
  const int *ch_ptr, *ch_idx;            // children lists
  const int *li_ptr, *li_idx;            // force items attached to each link
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
  int o_R, o_P, o_SI, o_S, o_V, o_A, o_F, o_FX, o_IT, o_IC, o_M, o_LD, o_B, o_T, o_QDD;
  int o_QC, o_QDC;                       // compensation (low parts) of q, qd within a step
  int o_LAM, o_SB, o_VB, o_AB, o_FB, o_SIB, o_RB, o_PB, o_ITB, o_TP, o_SEGA;
  int env_floats;
};

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

// Forward kinematics, level by level: link rotation R_i and origin P_i (world).
template <class Mem>
__device__ void st_fk(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int l = 0; l < M.nlev; ++l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii);
      const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i), p = __ldg(M.parent + i);
      M33 R;
      V3 P;
      if (jt == J_FREE) {
        // Spatial quantities use the free root's origin as reference point
        // (translation invariance); only contact depths need its height back.
        R = quat_to_R(w[M.o_Q + s + 3], w[M.o_Q + s + 4], w[M.o_Q + s + 5], w[M.o_Q + s + 6]);
        P = v3(0.f, 0.f, 0.f);
      } else {
        M33 Rj = cldm(M.jrot + 9 * i);
        V3 Pj = cld3(M.jpos + 3 * i);
        if (p >= 0) {
          M33 Rp = ldm(w, M.o_R + 9 * p);
          Pj = ld3(w, M.o_P + 3 * p) + mul(Rp, Pj);
          Rj = mul(Rp, Rj);
        }
        if (jt == J_REV) {
          R = mul(Rj, axis_angle(cld3(M.axis + 3 * i), w[M.o_Q + s]));
          P = Pj;
        } else if (jt == J_PRIS) {
          R = Rj;
          P = Pj + w[M.o_Q + s] * mul(Rj, cld3(M.axis + 3 * i));
        } else {
          R = Rj;
          P = Pj;
        }
      }
      stm(w, M.o_R + 9 * i, R);
      st3(w, M.o_P + 3 * i, P);
    }
    team_sync(nl);
  }
}

// Spatial inertias at the origin and motion-subspace columns of every DOF.
template <class Mem>
__device__ void st_linkq(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int i = lane; i < M.L; i += nl) {
    M33 R = ldm(w, M.o_R + 9 * i);
    V3 P = ld3(w, M.o_P + 3 * i);
    const float m = __ldg(M.mass + i);
    V3 c = P + mul(R, cld3(M.com + 3 * i));
    const float* ic = M.icom + 6 * i;
    M33 Ic;
    Ic.m[0] = __ldg(ic); Ic.m[4] = __ldg(ic + 1); Ic.m[8] = __ldg(ic + 2);
    Ic.m[1] = Ic.m[3] = __ldg(ic + 3); Ic.m[2] = Ic.m[6] = __ldg(ic + 4); Ic.m[5] = Ic.m[7] = __ldg(ic + 5);
    M33 Iw = mulBT(mul(R, Ic), R);
    float cc = dot(c, c);
    const int o = M.o_SI + 10 * i;
    w[o] = m;
    st3(w, o + 1, m * c);
    w[o + 4] = Iw.m[0] + m * (cc - c.x * c.x);
    w[o + 5] = Iw.m[4] + m * (cc - c.y * c.y);
    w[o + 6] = Iw.m[8] + m * (cc - c.z * c.z);
    w[o + 7] = Iw.m[1] - m * c.x * c.y;
    w[o + 8] = Iw.m[2] - m * c.x * c.z;
    w[o + 9] = Iw.m[5] - m * c.y * c.z;
  }
  for (int d = lane; d < M.nv; d += nl) {
    const int i = __ldg(M.dof_link + d), k = __ldg(M.dof_k + d), jt = __ldg(M.jtype + i);
    M33 R = ldm(w, M.o_R + 9 * i);
    V3 P = ld3(w, M.o_P + 3 * i);
    V3 sw, sv;
    if (jt == J_FREE) {
      if (k < 3) { sw = col(R, k); sv = cross(P, sw); }
      else { sw = v3(0.f, 0.f, 0.f); sv = col(R, k - 3); }
    } else {
      V3 a = mul(R, cld3(M.axis + 3 * i));
      if (jt == J_REV) { sw = a; sv = cross(P, a); }
      else { sw = v3(0.f, 0.f, 0.f); sv = a; }
    }
    st3(w, M.o_S + 6 * d, sw);
    st3(w, M.o_S + 6 * d + 3, sv);
  }
  team_sync(nl);
}

// joint spatial velocity u_i = sum_{d in i} S_d qd_d
template <class Mem>
__device__ __forceinline__ void joint_vel(const DevModel& M, const Mem& w, int i, V3& uw, V3& uv) {
  uw = v3(0.f, 0.f, 0.f); uv = v3(0.f, 0.f, 0.f);
  const int d0 = __ldg(M.ds + i), n = __ldg(M.nd + i);
  for (int d = d0; d < d0 + n; ++d) {
    float qd = w[M.o_QD + d];
    uw = uw + qd * ld3(w, M.o_S + 6 * d);
    uv = uv + qd * ld3(w, M.o_S + 6 * d + 3);
  }
}

// Link spatial velocities V_i = V_parent + u_i.
template <class Mem>
__device__ void st_vel(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int l = 0; l < M.nlev; ++l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii), p = __ldg(M.parent + i);
      V3 uw, uv;
      joint_vel(M, w, i, uw, uv);
      if (p >= 0) { uw = uw + ld3(w, M.o_V + 6 * p); uv = uv + ld3(w, M.o_V + 6 * p + 3); }
      st3(w, M.o_V + 6 * i, uw);
      st3(w, M.o_V + 6 * i + 3, uv);
    }
    team_sync(nl);
  }
}

// Sec. 3.1 contact model on the ground plane z = 0 (n = +z), applied at the
// lowest point x of each contact sphere:
//   f_n = (-ke + kd ddot) min(d, 0),  d = x_z, ddot = v_x . n
//   f_t = -v_t/|v_t| min(kt |v_t|, mu |f_n|)  (viscous branch when kt|v_t| <= mu|f_n|)
// Muscles: force clamp(a,0,1) fmax along each via segment, pulling its ends together.
// Each item stores its world point x and force f; then per-link external wrenches.
template <class Mem>
__device__ void st_items(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int c = lane; c < M.nc; c += nl) {
    const int i = __ldg(M.item_link + c);
    M33 R = ldm(w, M.o_R + 9 * i);
    const V3 lp = cld3(M.item_pos + 3 * c);
    V3 x = ld3(w, M.o_P + 3 * i) + mul(R, lp);
    x.z -= __ldg(M.crad + c);
    const float d = x.z + (M.root_free ? w[M.o_Q + 2] : 0.f);   // height above the plane
    V3 f = v3(0.f, 0.f, 0.f);
    if (d < 0.f) {
      V3 vp = ld3(w, M.o_V + 6 * i + 3) + cross(ld3(w, M.o_V + 6 * i), x);
      float fn = (-M.ke + M.kd * vp.z) * d;
      float vt2 = vp.x * vp.x + vp.y * vp.y;
      float vt = sqrtf(vt2);
      float afn = fabsf(fn);
      if (M.kt * vt <= M.mu * afn) { f.x = -M.kt * vp.x; f.y = -M.kt * vp.y; }
      else { float s = M.mu * afn / vt; f.x = -s * vp.x; f.y = -s * vp.y; }
      f.z = fn;
    }
    st3(w, M.o_IT + 7 * c, x);
    st3(w, M.o_IT + 7 * c + 3, f);
    w[M.o_IT + 7 * c + 6] = d;
  }
  for (int sg = lane; sg < M.nseg; sg += nl) {
    const int e0 = M.nc + 2 * sg, e1 = e0 + 1;
    const int l0 = __ldg(M.item_link + e0), l1 = __ldg(M.item_link + e1);
    V3 x0 = ld3(w, M.o_P + 3 * l0) + mul(ldm(w, M.o_R + 9 * l0), cld3(M.item_pos + 3 * e0));
    V3 x1 = ld3(w, M.o_P + 3 * l1) + mul(ldm(w, M.o_R + 9 * l1), cld3(M.item_pos + 3 * e1));
    const int mu_ = __ldg(M.seg_mus + sg);
    float a = fminf(fmaxf(w[M.o_ACT + M.ntact + mu_], 0.f), 1.f);
    float F = a * __ldg(M.fmax + mu_);
    V3 dv = x1 - x0;
    float inv = 1.f / sqrtf(dot(dv, dv));
    V3 u = inv * dv;
    st3(w, M.o_IT + 7 * e0, x0);
    st3(w, M.o_IT + 7 * e0 + 3, F * u);
    st3(w, M.o_IT + 7 * e1, x1);
    st3(w, M.o_IT + 7 * e1 + 3, -F * u);
  }
  team_sync(nl);
  for (int i = lane; i < M.L; i += nl) {
    V3 n = v3(0.f, 0.f, 0.f), f = v3(0.f, 0.f, 0.f);
    for (int k = __ldg(M.li_ptr + i); k < __ldg(M.li_ptr + i + 1); ++k) {
      const int e = __ldg(M.li_idx + k);
      V3 x = ld3(w, M.o_IT + 7 * e), fe = ld3(w, M.o_IT + 7 * e + 3);
      n = n + cross(x, fe);
      f = f + fe;
    }
    st3(w, M.o_FX + 6 * i, n);
    st3(w, M.o_FX + 6 * i + 3, f);
  }
  team_sync(nl);
}

// Newton-Euler inverse dynamics in world spatial coordinates.
//   A_i = A_parent + sum_d S_d qdd_d + V_i x u_i          (A_root parent = -gravity)
//   F_i = I_i A_i + V_i x* (I_i V_i) - Fext_i,  F_parent += F_i (gather)
// use_qdd = 0 gives the bias C (qdd = 0).  Leaves total F_i in o_F.
template <class Mem>
__device__ void st_id(const DevModel& M, const Mem& w, int lane, int nl, bool use_qdd) {
  for (int l = 0; l < M.nlev; ++l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii), p = __ldg(M.parent + i);
      V3 aw, av;
      if (p >= 0) { aw = ld3(w, M.o_A + 6 * p); av = ld3(w, M.o_A + 6 * p + 3); }
      else { aw = v3(0.f, 0.f, 0.f); av = v3(-M.grav[0], -M.grav[1], -M.grav[2]); }
      V3 uw, uv;
      joint_vel(M, w, i, uw, uv);
      V3 Vw = ld3(w, M.o_V + 6 * i), Vv = ld3(w, M.o_V + 6 * i + 3);
      aw = aw + cross(Vw, uw);
      av = av + cross(Vw, uv) + cross(Vv, uw);
      if (use_qdd) {
        const int d0 = __ldg(M.ds + i), n = __ldg(M.nd + i);
        for (int d = d0; d < d0 + n; ++d) {
          float a = w[M.o_QDD + d];
          aw = aw + a * ld3(w, M.o_S + 6 * d);
          av = av + a * ld3(w, M.o_S + 6 * d + 3);
        }
      }
      st3(w, M.o_A + 6 * i, aw);
      st3(w, M.o_A + 6 * i + 3, av);
    }
    team_sync(nl);
  }
  for (int i = lane; i < M.L; i += nl) {
    V3 aw = ld3(w, M.o_A + 6 * i), av = ld3(w, M.o_A + 6 * i + 3);
    V3 Vw = ld3(w, M.o_V + 6 * i), Vv = ld3(w, M.o_V + 6 * i + 3);
    V3 fn, ff, bn, bf;
    si_mul(w, M.o_SI + 10 * i, aw, av, fn, ff);
    si_mul(w, M.o_SI + 10 * i, Vw, Vv, bn, bf);
    fn = fn + cross(Vw, bn) + cross(Vv, bf) - ld3(w, M.o_FX + 6 * i);
    ff = ff + cross(Vw, bf) - ld3(w, M.o_FX + 6 * i + 3);
    st3(w, M.o_F + 6 * i, fn);
    st3(w, M.o_F + 6 * i + 3, ff);
  }
  team_sync(nl);
  for (int l = M.nlev - 1; l >= 0; --l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii);
      const int c0 = __ldg(M.ch_ptr + i), c1 = __ldg(M.ch_ptr + i + 1);
      if (c0 == c1) continue;
      V3 fn = ld3(w, M.o_F + 6 * i), ff = ld3(w, M.o_F + 6 * i + 3);
      for (int k = c0; k < c1; ++k) {
        const int c = __ldg(M.ch_idx + k);
        fn = fn + ld3(w, M.o_F + 6 * c);
        ff = ff + ld3(w, M.o_F + 6 * c + 3);
      }
      st3(w, M.o_F + 6 * i, fn);
      st3(w, M.o_F + 6 * i + 3, ff);
    }
    team_sync(nl);
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
    float q = w[M.o_Q + __ldg(M.qs + i)];
    float lo = __ldg(M.qlo + d), hi = __ldg(M.qhi + d);
    if (q < lo) t += M.klim * (lo - q);
    else if (q > hi) t += M.klim * (hi - q);
  }
  return t - __ldg(M.damp + d) * w[M.o_QD + d];
}

// right-hand side b = tau_j - S^T F (bias from st_id with qdd = 0)
template <class Mem>
__device__ void st_rhs(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int d = lane; d < M.nv; d += nl) {
    const int i = __ldg(M.dof_link + d);
    float c = dot(ld3(w, M.o_S + 6 * d), ld3(w, M.o_F + 6 * i)) + dot(ld3(w, M.o_S + 6 * d + 3), ld3(w, M.o_F + 6 * i + 3));
    w[M.o_B + d] = joint_force(M, w, d) - c;
  }
  team_sync(nl);
}

// CRBA part 1: composite spatial inertias Ic_i = I_i + sum_children Ic_c
// (gather, leaves first).
template <class Mem>
__device__ void st_composite(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int l = M.nlev - 1; l >= 0; --l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii);
      float acc[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) acc[k] = w[M.o_SI + 10 * i + k];
      for (int kk = __ldg(M.ch_ptr + i); kk < __ldg(M.ch_ptr + i + 1); ++kk) {
        const int c = __ldg(M.ch_idx + kk);
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] += w[M.o_IC + 10 * c + k];
      }
#pragma unroll
      for (int k = 0; k < 10; ++k) w[M.o_IC + 10 * i + k] = acc[k];
    }
    team_sync(nl);
  }
}

// Lower triangle of M row by row (row a owns M[a][b], b <= a), armature on
// the diagonal (shared-memory form).
template <class Mem>
__device__ void st_mass_rows(const DevModel& M, const Mem& w, int lane, int nl) {
  const int n = M.nv;
  for (int a = lane; a < n; a += nl) {
    const int i = __ldg(M.dof_link + a);
    for (int b = 0; b < a; ++b) w[M.o_M + a * n + b] = 0.f;   // zero unless b is an ancestor DOF
    V3 fn, ff;
    si_mul(w, M.o_IC + 10 * i, ld3(w, M.o_S + 6 * a), ld3(w, M.o_S + 6 * a + 3), fn, ff);
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

// Semi-implicit Euler: qd += h qdd, then q += h qd (new velocity); free root:
// p += h R v_b, quat <- normalise(quat + h/2 quat (x) (w_b, 0)).
// The state stays FP32 between substeps; the rounding of each accumulation
// is carried in o_QC/o_QDC (zeroed at every step start) and fed back into the
// next substep's update, so a step of K substeps rounds its state once.
template <class Mem>
__device__ void st_integrate(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int d = lane; d < M.nv; d += nl) {
    float e;
    const float y = M.h * w[M.o_QDD + d] + w[M.o_QDC + d];
    w[M.o_QD + d] = two_sum(w[M.o_QD + d], y, e);
    w[M.o_QDC + d] = e;
  }
  team_sync(nl);
  for (int i = lane; i < M.L; i += nl) {
    const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i), d = __ldg(M.ds + i);
    if (jt == J_FREE) {
      M33 R = ldm(w, M.o_R + 9 * i);
      V3 dp = M.h * mul(R, ld3(w, M.o_QD + d + 3)) + M.h * mul(R, ld3(w, M.o_QDC + d + 3));
      float e;
      w[M.o_Q + s] = two_sum(w[M.o_Q + s], dp.x + w[M.o_QC + s], e); w[M.o_QC + s] = e;
      w[M.o_Q + s + 1] = two_sum(w[M.o_Q + s + 1], dp.y + w[M.o_QC + s + 1], e); w[M.o_QC + s + 1] = e;
      w[M.o_Q + s + 2] = two_sum(w[M.o_Q + s + 2], dp.z + w[M.o_QC + s + 2], e); w[M.o_QC + s + 2] = e;
      float x = w[M.o_Q + s + 3], y = w[M.o_Q + s + 4], z = w[M.o_Q + s + 5], qw = w[M.o_Q + s + 6];
      V3 om = ld3(w, M.o_QD + d);
      V3 u = v3(x, y, z);
      V3 pv = qw * om + cross(u, om);
      float pw = -dot(u, om);
      const float hh = 0.5f * M.h;
      float nx = x + hh * pv.x, ny = y + hh * pv.y, nz = z + hh * pv.z, nw = qw + hh * pw;
      float inv = rsqrtf(nx * nx + ny * ny + nz * nz + nw * nw);
      w[M.o_Q + s + 3] = nx * inv; w[M.o_Q + s + 4] = ny * inv; w[M.o_Q + s + 5] = nz * inv; w[M.o_Q + s + 6] = nw * inv;
    } else if (jt == J_REV || jt == J_PRIS) {
      float e;
      const float y = M.h * w[M.o_QD + d] + (M.h * w[M.o_QDC + d] + w[M.o_QC + s]);
      w[M.o_Q + s] = two_sum(w[M.o_Q + s], y, e);
      w[M.o_QC + s] = e;
    }
  }
  team_sync(nl);
}

// Clear the integration compensation at a step start (team-parallel).
template <class Mem>
__device__ __forceinline__ void clear_comp(const DevModel& M, const Mem& w, int lane, int nl) {
  for (int j = lane; j < M.nq; j += nl) w[M.o_QC + j] = 0.f;
  for (int j = lane; j < M.nv; j += nl) w[M.o_QDC + j] = 0.f;
}

// ---- register-resident dense path (teams with at least nv lanes) ----------
// Lane a of the team owns row a of M.  The row is assembled in registers
// (CRBA part 2), factorised by a right-looking Cholesky whose column k is
// broadcast with team shuffles, and the factor is stored to o_M/o_LD for the
// triangular solves and for the backward pass.  NM >= nv is the register
// capacity of a row (compile-time), nl >= nv the team size.
template <int NM, class Mem>
__device__ void dense_factor(const DevModel& M, const Mem& w, int lane, int nl) {
  const int n = M.nv;
  const bool own = lane < n;
  float row[NM];
  {
    V3 fn = v3(0.f, 0.f, 0.f), ff = v3(0.f, 0.f, 0.f);
    unsigned mask = 0u;
    if (own) {
      const int i = __ldg(M.dof_link + lane);
      si_mul(w, M.o_IC + 10 * i, ld3(w, M.o_S + 6 * lane), ld3(w, M.o_S + 6 * lane + 3), fn, ff);
      mask = __ldg(M.anc_mask + lane);
    }
    const float arm = own ? __ldg(M.arm + lane) : 1.f;
#pragma unroll
    for (int b = 0; b < NM; ++b) {
      float v = 0.f;
      if ((mask >> b) & 1u) v = dot(ld3(w, M.o_S + 6 * b), fn) + dot(ld3(w, M.o_S + 6 * b + 3), ff);
      if (b == lane) v += arm;
      row[b] = v;
    }
  }
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    if (k < n) {
      const float rk = row[k];
      const float dkk = sqrtf(__shfl_sync(0xffffffffu, rk, k, nl));
      const float lik = rk * (1.f / dkk);
      if (lane > k) row[k] = lik;
      else if (lane == k) row[k] = dkk;
#pragma unroll
      for (int j = k + 1; j < NM; ++j) {
        if (j < n) {
          const float ljk = __shfl_sync(0xffffffffu, lik, j, nl);
          if (lane >= j) row[j] -= lik * ljk;
        }
      }
    }
  }
  if (own) {
#pragma unroll
    for (int b = 0; b < NM; ++b) {
      if (b < lane) w[M.o_M + lane * n + b] = row[b];
      else if (b == lane) w[M.o_LD + lane] = row[b];
    }
  }
  team_sync(nl);
}

// x = (L L^T)^{-1} b with the stored factor; lane a holds b_a, the columns of
// the substitution are broadcast with team shuffles (no barriers).
template <class Mem>
__device__ void dense_solve(const DevModel& M, const Mem& w, int lane, int nl, int o_in, int o_out) {
  const int n = M.nv;
  const bool own = lane < n;
  float b = own ? w[o_in + lane] : 0.f;
  const float invd = own ? 1.f / w[M.o_LD + lane] : 0.f;
  for (int k = 0; k < n; ++k) {
    const float yk = __shfl_sync(0xffffffffu, b * invd, k, nl);
    if (lane > k && own) b -= w[M.o_M + lane * n + k] * yk;
    else if (lane == k) b = yk;
  }
  for (int k = n - 1; k >= 0; --k) {
    const float xk = __shfl_sync(0xffffffffu, b * invd, k, nl);
    if (lane < k) b -= w[M.o_M + k * n + lane] * xk;
    else if (lane == k) b = xk;
  }
  if (own) w[o_out + lane] = b;
  team_sync(nl);
}

// One forward substep up to the accelerations (integration is separate).
// NM = 0: shared-memory dense stages (any team size, incl. one thread per
// environment); NM > 0: register-resident dense path.
template <int NM, class Mem>
__device__ void substep_dynamics(const DevModel& M, const Mem& w, int lane, int nl) {
  st_fk(M, w, lane, nl);
  st_linkq(M, w, lane, nl);
  st_vel(M, w, lane, nl);
  st_items(M, w, lane, nl);
  st_id(M, w, lane, nl, false);
  st_rhs(M, w, lane, nl);
  st_composite(M, w, lane, nl);
  if constexpr (NM > 0) {
    dense_factor<NM>(M, w, lane, nl);
    dense_solve(M, w, lane, nl, M.o_B, M.o_QDD);
  } else {
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
    float D = fminf(fmaxf(w[M.o_Q + 2] - M.rc[4], M.rc[5]), M.rc[6]);
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
    float raw = w[M.o_Q + 2] - M.rc[4];
    if (raw > M.rc[5] && raw < M.rc[6]) {
      float D = raw;
      float dD = D < 0.f ? (2.f * M.rc[7] * D + M.rc[8]) : M.rc[9];
      w[M.o_QB + 2] += dD * rb;
    }
  }
}

// ================================================================= ADJOINT ==

// Reverse of st_integrate.  Inputs: o_Q/o_QD hold the substep START state,
// o_QDD its accelerations, o_R its rotations; o_QB/o_QDB hold the cotangents
// of the substep END state.  Outputs: o_QB/o_QDB partial cotangents of the
// start state (integrator paths only) and o_T = qdd_bar.
template <class Mem>
__device__ void st_integrate_adj(const DevModel& M, const Mem& w, int lane, int nl) {
  const float h = M.h;
  for (int i = lane; i < M.L; i += nl) {
    const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i), d = __ldg(M.ds + i);
    if (jt == J_REV || jt == J_PRIS) {
      w[M.o_QDB + d] += h * w[M.o_QB + s];          // q' = q + h qd'
    } else if (jt == J_FREE) {
      M33 R = ldm(w, M.o_R + 9 * i);
      V3 vb1 = ld3(w, M.o_QD + d + 3) + h * ld3(w, M.o_QDD + d + 3);   // new body velocity
      V3 om1 = ld3(w, M.o_QD + d) + h * ld3(w, M.o_QDD + d);
      V3 pb = ld3(w, M.o_QB + s);
      // p' = p + h R v_b'
      add3(w, M.o_QDB + d + 3, h * mulT(R, pb));
      M33 B;
      B.m[0] = h * pb.x * vb1.x; B.m[1] = h * pb.x * vb1.y; B.m[2] = h * pb.x * vb1.z;
      B.m[3] = h * pb.y * vb1.x; B.m[4] = h * pb.y * vb1.y; B.m[5] = h * pb.y * vb1.z;
      B.m[6] = h * pb.z * vb1.x; B.m[7] = h * pb.z * vb1.y; B.m[8] = h * pb.z * vb1.z;
      float x = w[M.o_Q + s + 3], y = w[M.o_Q + s + 4], z = w[M.o_Q + s + 5], qw = w[M.o_Q + s + 6];
      float xb = 0.f, yb = 0.f, zb = 0.f, wb = 0.f;
      quat_to_R_adj(x, y, z, qw, B, xb, yb, zb, wb);
      // quat' = n / |n|, n = quat + h/2 quat (x) (w', 0)
      V3 u = v3(x, y, z);
      const float hh = 0.5f * h;
      V3 nu = u + hh * (qw * om1 + cross(u, om1));
      float nw = qw - hh * dot(u, om1);
      float nn = sqrtf(dot(nu, nu) + nw * nw);
      float inv = 1.f / nn;
      V3 qu1 = inv * nu;
      float qw1 = inv * nw;
      V3 qub = ld3(w, M.o_QB + s + 3);
      float qwb = w[M.o_QB + s + 6];
      float pr = dot(qu1, qub) + qw1 * qwb;
      V3 nub = inv * (qub - pr * qu1);
      float nwb = inv * (qwb - pr * qw1);
      V3 ub = nub + hh * cross(om1, nub) - (hh * nwb) * om1;
      float wbq = nwb + hh * dot(om1, nub);
      V3 omb = hh * (qw * nub + cross(nub, u)) - (hh * nwb) * u;
      add3(w, M.o_QDB + d, omb);
      w[M.o_QB + s + 3] = ub.x + xb; w[M.o_QB + s + 4] = ub.y + yb; w[M.o_QB + s + 5] = ub.z + zb;
      w[M.o_QB + s + 6] = wbq + wb;
    }
  }
  team_sync(nl);
  for (int d = lane; d < M.nv; d += nl) w[M.o_T + d] = h * w[M.o_QDB + d];   // qd' = qd + h qdd
  team_sync(nl);
}

// y_bar, x -> accumulate cotangents of the 10-float spatial inertia for y = I x
// into (hbar[3], G[9]) at o (mass cotangent not needed: masses are constants).
template <class Mem>
__device__ __forceinline__ void si_mul_adj(const Mem& w, int o, V3 xw, V3 xv, V3 yn_b, V3 yf_b) {
  add3(w, o, cross(xv, yn_b) + cross(yf_b, xw));
  w[o + 3] += yn_b.x * xw.x; w[o + 4] += yn_b.x * xw.y; w[o + 5] += yn_b.x * xw.z;
  w[o + 6] += yn_b.y * xw.x; w[o + 7] += yn_b.y * xw.y; w[o + 8] += yn_b.y * xw.z;
  w[o + 9] += yn_b.z * xw.x; w[o + 10] += yn_b.z * xw.y; w[o + 11] += yn_b.z * xw.z;
}

// Zero a range of scratch (team-parallel).
template <class Mem>
__device__ __forceinline__ void zero_range(const Mem& w, int o, int n, int lane, int nl) {
  for (int k = lane; k < n; k += nl) w[o + k] = 0.f;
}

// Adjoint of the dynamics solve: given o_T = qdd_bar and the recomputed
// substep (o_QDD holds the solved accelerations), add -lambda^T dG/d(q,qd,a)
// to o_QB, o_QDB, o_ACTB.
template <int NM, class Mem>
__device__ void st_dynamics_adj(const DevModel& M, const Mem& w, int lane, int nl) {
  // lambda = M^{-1} qdd_bar (cached factor)
  if constexpr (NM > 0) {
    dense_solve(M, w, lane, nl, M.o_T, M.o_LAM);
  } else {
    for (int d = lane; d < M.nv; d += nl) w[M.o_B + d] = w[M.o_T + d];
    team_sync(nl);
    st_solve(M, w, lane, nl, M.o_B, M.o_LAM);
  }
  // accelerations and forces with the actual qdd (the C pass used qdd = 0)
  st_id(M, w, lane, nl, true);
  // clear accumulators
  zero_range(w, M.o_VB, 6 * M.L, lane, nl);
  zero_range(w, M.o_SIB, 12 * M.L, lane, nl);
  zero_range(w, M.o_RB, 9 * M.L, lane, nl);
  zero_range(w, M.o_PB, 3 * M.L, lane, nl);
  team_sync(nl);
  // joint forces: tau_j_bar = lambda
  for (int d = lane; d < M.nv; d += nl) {
    const float lam = w[M.o_LAM + d];
    const int a = __ldg(M.dof_act + d);
    if (a >= 0) w[M.o_ACTB + a] += lam * __ldg(M.gear + d);
    const int i = __ldg(M.dof_link + d), jt = __ldg(M.jtype + i);
    if (jt == J_REV || jt == J_PRIS) {
      const int s = __ldg(M.qs + i);
      float q = w[M.o_Q + s];
      if (q < __ldg(M.qlo + d) || q > __ldg(M.qhi + d)) w[M.o_QB + s] -= lam * M.klim;
    }
    w[M.o_QDB + d] -= lam * __ldg(M.damp + d);
    // tau_d = S_d . F_total: S_bar = w_d F, with w = -lambda
    const float wd = -lam;
    st3(w, M.o_SB + 6 * d, wd * ld3(w, M.o_F + 6 * i));
    st3(w, M.o_SB + 6 * d + 3, wd * ld3(w, M.o_F + 6 * i + 3));
  }
  team_sync(nl);
  // F_bar_total_i = sum_{d in i} w_d S_d + F_bar_total_parent (root first)
  for (int l = 0; l < M.nlev; ++l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii), p = __ldg(M.parent + i);
      V3 bn = v3(0.f, 0.f, 0.f), bf = v3(0.f, 0.f, 0.f);
      if (p >= 0) { bn = ld3(w, M.o_FB + 6 * p); bf = ld3(w, M.o_FB + 6 * p + 3); }
      const int d0 = __ldg(M.ds + i), n = __ldg(M.nd + i);
      for (int d = d0; d < d0 + n; ++d) {
        const float wd = -w[M.o_LAM + d];
        bn = bn + wd * ld3(w, M.o_S + 6 * d);
        bf = bf + wd * ld3(w, M.o_S + 6 * d + 3);
      }
      st3(w, M.o_FB + 6 * i, bn);
      st3(w, M.o_FB + 6 * i + 3, bf);
    }
    team_sync(nl);
  }
  // local force F_i = I A + V x* (I V) - Fext
  for (int i = lane; i < M.L; i += nl) {
    V3 nb = ld3(w, M.o_FB + 6 * i), fb = ld3(w, M.o_FB + 6 * i + 3);
    V3 aw = ld3(w, M.o_A + 6 * i), av = ld3(w, M.o_A + 6 * i + 3);
    V3 Vw = ld3(w, M.o_V + 6 * i), Vv = ld3(w, M.o_V + 6 * i + 3);
    const int osi = M.o_SI + 10 * i, osb = M.o_SIB + 12 * i;
    // A_bar = I F_bar (I symmetric)
    V3 abn, abf;
    si_mul(w, osi, nb, fb, abn, abf);
    st3(w, M.o_AB + 6 * i, abn);
    st3(w, M.o_AB + 6 * i + 3, abf);
    si_mul_adj(w, osb, aw, av, nb, fb);
    // momentum B = I V and V x* B
    V3 Bn, Bf;
    si_mul(w, osi, Vw, Vv, Bn, Bf);
    V3 vwb = cross(Bn, nb) + cross(Bf, fb);
    V3 vvb = cross(Bf, nb);
    V3 Bnb = cross(nb, Vw);
    V3 Bfb = cross(nb, Vv) + cross(fb, Vw);
    V3 t1, t2;
    si_mul(w, osi, Bnb, Bfb, t1, t2);
    vwb = vwb + t1;
    vvb = vvb + t2;
    si_mul_adj(w, osb, Vw, Vv, Bnb, Bfb);
    add3(w, M.o_VB + 6 * i, vwb);
    add3(w, M.o_VB + 6 * i + 3, vvb);
  }
  team_sync(nl);
  // accelerations, leaves first: A_i = A_p + sum S qdd + V_i x u_i
  for (int l = M.nlev - 1; l >= 0; --l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii);
      V3 an = ld3(w, M.o_AB + 6 * i), af = ld3(w, M.o_AB + 6 * i + 3);
      for (int k = __ldg(M.ch_ptr + i); k < __ldg(M.ch_ptr + i + 1); ++k) {
        const int c = __ldg(M.ch_idx + k);
        an = an + ld3(w, M.o_AB + 6 * c);
        af = af + ld3(w, M.o_AB + 6 * c + 3);
      }
      st3(w, M.o_AB + 6 * i, an);
      st3(w, M.o_AB + 6 * i + 3, af);
      V3 uw, uv;
      joint_vel(M, w, i, uw, uv);
      V3 Vw = ld3(w, M.o_V + 6 * i), Vv = ld3(w, M.o_V + 6 * i + 3);
      add3(w, M.o_VB + 6 * i, cross(uw, an) + cross(uv, af));
      add3(w, M.o_VB + 6 * i + 3, cross(uw, af));
      V3 ubw = cross(an, Vw) + cross(af, Vv);
      V3 ubv = cross(af, Vw);
      const int d0 = __ldg(M.ds + i), n = __ldg(M.nd + i);
      for (int d = d0; d < d0 + n; ++d) {
        const float qdd = w[M.o_QDD + d], qd = w[M.o_QD + d];
        add3(w, M.o_SB + 6 * d, qdd * an + qd * ubw);
        add3(w, M.o_SB + 6 * d + 3, qdd * af + qd * ubv);
        w[M.o_QDB + d] += dot(ld3(w, M.o_S + 6 * d), ubw) + dot(ld3(w, M.o_S + 6 * d + 3), ubv);
      }
    }
    team_sync(nl);
  }
  // force items (external wrench Fext_i enters F_i with a minus sign)
  for (int c = lane; c < M.nc; c += nl) {
    const int i = __ldg(M.item_link + c);
    V3 x = ld3(w, M.o_IT + 7 * c), f = ld3(w, M.o_IT + 7 * c + 3);
    const float dep = w[M.o_IT + 7 * c + 6];
    V3 xb = v3(0.f, 0.f, 0.f), wb = v3(0.f, 0.f, 0.f), vob = v3(0.f, 0.f, 0.f);
    float db = 0.f;
    if (dep < 0.f) {
      V3 neb = -ld3(w, M.o_FB + 6 * i), feb = -ld3(w, M.o_FB + 6 * i + 3);
      V3 fbar = cross(neb, x) + feb;
      xb = cross(f, neb);
      V3 Vw = ld3(w, M.o_V + 6 * i);
      V3 vp = ld3(w, M.o_V + 6 * i + 3) + cross(Vw, x);
      float fn = f.z;
      float vt = sqrtf(vp.x * vp.x + vp.y * vp.y);
      float afn = fabsf(fn);
      float fnb = fbar.z;
      V3 vpb = v3(0.f, 0.f, 0.f);
      if (M.kt * vt <= M.mu * afn) {
        vpb.x = -M.kt * fbar.x;
        vpb.y = -M.kt * fbar.y;
      } else {
        float s = M.mu * afn / vt;
        float sb = -(fbar.x * vp.x + fbar.y * vp.y);
        vpb.x = -s * fbar.x;
        vpb.y = -s * fbar.y;
        fnb += sb * M.mu * (fn >= 0.f ? 1.f : -1.f) / vt;
        float vtb = -sb * s / vt;
        vpb.x += vtb * vp.x / vt;
        vpb.y += vtb * vp.y / vt;
      }
      // fn = (-ke + kd ddot) d, d = x.z + root height
      db = fnb * (-M.ke + M.kd * vp.z);
      xb.z += db;
      vpb.z += fnb * M.kd * dep;
      vob = vpb;
      wb = cross(x, vpb);
      xb = xb + cross(vpb, Vw);
    }
    st3(w, M.o_ITB + 10 * c, xb);
    st3(w, M.o_ITB + 10 * c + 3, wb);
    st3(w, M.o_ITB + 10 * c + 6, vob);
    w[M.o_ITB + 10 * c + 9] = db;
  }
  for (int sg = lane; sg < M.nseg; sg += nl) {
    const int e0 = M.nc + 2 * sg, e1 = e0 + 1;
    const int l0 = __ldg(M.item_link + e0), l1 = __ldg(M.item_link + e1);
    V3 x0 = ld3(w, M.o_IT + 7 * e0), f0 = ld3(w, M.o_IT + 7 * e0 + 3);
    V3 x1 = ld3(w, M.o_IT + 7 * e1), f1 = ld3(w, M.o_IT + 7 * e1 + 3);
    V3 n0b = -ld3(w, M.o_FB + 6 * l0), f0eb = -ld3(w, M.o_FB + 6 * l0 + 3);
    V3 n1b = -ld3(w, M.o_FB + 6 * l1), f1eb = -ld3(w, M.o_FB + 6 * l1 + 3);
    V3 f0b = cross(n0b, x0) + f0eb, f1b = cross(n1b, x1) + f1eb;
    V3 x0b = cross(f0, n0b), x1b = cross(f1, n1b);
    const int mu_ = __ldg(M.seg_mus + sg);
    float araw = w[M.o_ACT + M.ntact + mu_];
    float a = fminf(fmaxf(araw, 0.f), 1.f);
    float fm = __ldg(M.fmax + mu_);
    float F = a * fm;
    V3 dv = x1 - x0;
    float len = sqrtf(dot(dv, dv));
    V3 u = (1.f / len) * dv;
    V3 g = f0b - f1b;
    V3 ub = F * g;
    float Fb = dot(u, g);
    V3 db = (1.f / len) * (ub - dot(u, ub) * u);
    x1b = x1b + db;
    x0b = x0b - db;
    w[M.o_SEGA + sg] = (araw > 0.f && araw < 1.f) ? Fb * fm : 0.f;
    st3(w, M.o_ITB + 10 * e0, x0b);
    st3(w, M.o_ITB + 10 * e1, x1b);
  }
  team_sync(nl);
  if (lane == 0 && M.root_free) {   // depth = x.z + root height: the root height gets every d_bar
    float s = 0.f;
    for (int c = 0; c < M.nc; ++c) s += w[M.o_ITB + 10 * c + 9];
    w[M.o_QB + 2] += s;
  }
  for (int mu_ = lane; mu_ < M.nm; mu_ += nl) {
    float s = 0.f;
    for (int sg = __ldg(M.mus_seg_ptr + mu_); sg < __ldg(M.mus_seg_ptr + mu_ + 1); ++sg) s += w[M.o_SEGA + sg];
    w[M.o_ACTB + M.ntact + mu_] += s;
  }
  for (int i = lane; i < M.L; i += nl) {
    V3 pb = v3(0.f, 0.f, 0.f), wb = v3(0.f, 0.f, 0.f), vb = v3(0.f, 0.f, 0.f);
    M33 Rb;
#pragma unroll
    for (int k = 0; k < 9; ++k) Rb.m[k] = 0.f;
    for (int k = __ldg(M.li_ptr + i); k < __ldg(M.li_ptr + i + 1); ++k) {
      const int e = __ldg(M.li_idx + k);
      V3 xb = ld3(w, M.o_ITB + 10 * e);
      V3 lp = cld3(M.item_pos + 3 * e);
      pb = pb + xb;
      Rb.m[0] += xb.x * lp.x; Rb.m[1] += xb.x * lp.y; Rb.m[2] += xb.x * lp.z;
      Rb.m[3] += xb.y * lp.x; Rb.m[4] += xb.y * lp.y; Rb.m[5] += xb.y * lp.z;
      Rb.m[6] += xb.z * lp.x; Rb.m[7] += xb.z * lp.y; Rb.m[8] += xb.z * lp.z;
      if (e < M.nc) {
        wb = wb + ld3(w, M.o_ITB + 10 * e + 3);
        vb = vb + ld3(w, M.o_ITB + 10 * e + 6);
      }
    }
    add3(w, M.o_PB + 3 * i, pb);
#pragma unroll
    for (int k = 0; k < 9; ++k) w[M.o_RB + 9 * i + k] += Rb.m[k];
    add3(w, M.o_VB + 6 * i, wb);
    add3(w, M.o_VB + 6 * i + 3, vb);
  }
  team_sync(nl);
  // velocities, leaves first: V_i = V_p + u_i
  for (int l = M.nlev - 1; l >= 0; --l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii);
      V3 vw = ld3(w, M.o_VB + 6 * i), vv = ld3(w, M.o_VB + 6 * i + 3);
      for (int k = __ldg(M.ch_ptr + i); k < __ldg(M.ch_ptr + i + 1); ++k) {
        const int c = __ldg(M.ch_idx + k);
        vw = vw + ld3(w, M.o_VB + 6 * c);
        vv = vv + ld3(w, M.o_VB + 6 * c + 3);
      }
      st3(w, M.o_VB + 6 * i, vw);
      st3(w, M.o_VB + 6 * i + 3, vv);
      const int d0 = __ldg(M.ds + i), n = __ldg(M.nd + i);
      for (int d = d0; d < d0 + n; ++d) {
        const float qd = w[M.o_QD + d];
        add3(w, M.o_SB + 6 * d, qd * vw);
        add3(w, M.o_SB + 6 * d + 3, qd * vv);
        w[M.o_QDB + d] += dot(ld3(w, M.o_S + 6 * d), vw) + dot(ld3(w, M.o_S + 6 * d + 3), vv);
      }
    }
    team_sync(nl);
  }
  // link quantities: motion subspaces and spatial inertias -> R_bar, P_bar
  for (int i = lane; i < M.L; i += nl) {
    M33 R = ldm(w, M.o_R + 9 * i);
    V3 P = ld3(w, M.o_P + 3 * i);
    M33 Rb = ldm(w, M.o_RB + 9 * i);
    V3 Pb = ld3(w, M.o_PB + 3 * i);
    const int jt = __ldg(M.jtype + i), d0 = __ldg(M.ds + i), n = __ldg(M.nd + i);
    for (int d = d0; d < d0 + n; ++d) {
      V3 sbw = ld3(w, M.o_SB + 6 * d), sbv = ld3(w, M.o_SB + 6 * d + 3);
      const int k = d - d0;
      if (jt == J_FREE) {
        if (k < 3) {
          V3 r = col(R, k);
          V3 rb = sbw + cross(sbv, P);
          Pb = Pb + cross(r, sbv);
          Rb.m[k] += rb.x; Rb.m[3 + k] += rb.y; Rb.m[6 + k] += rb.z;
        } else {
          Rb.m[k - 3] += sbv.x; Rb.m[3 + k - 3] += sbv.y; Rb.m[6 + k - 3] += sbv.z;
        }
      } else {
        V3 ax = cld3(M.axis + 3 * i);
        V3 ab;
        if (jt == J_REV) {
          V3 a = mul(R, ax);
          ab = sbw + cross(sbv, P);
          Pb = Pb + cross(a, sbv);
        } else {
          ab = sbv;
        }
        Rb.m[0] += ab.x * ax.x; Rb.m[1] += ab.x * ax.y; Rb.m[2] += ab.x * ax.z;
        Rb.m[3] += ab.y * ax.x; Rb.m[4] += ab.y * ax.y; Rb.m[5] += ab.y * ax.z;
        Rb.m[6] += ab.z * ax.x; Rb.m[7] += ab.z * ax.y; Rb.m[8] += ab.z * ax.z;
      }
    }
    // spatial inertia: h = m c, Io = R Ic R^T + m(|c|^2 1 - c c^T), c = P + R com
    const float m = __ldg(M.mass + i);
    if (m != 0.f || __ldg(M.icom + 6 * i) != 0.f || __ldg(M.icom + 6 * i + 1) != 0.f || __ldg(M.icom + 6 * i + 2) != 0.f) {
      const int osb = M.o_SIB + 12 * i;
      V3 hb = ld3(w, osb);
      M33 G;
#pragma unroll
      for (int k = 0; k < 9; ++k) G.m[k] = w[osb + 3 + k];
      V3 com = cld3(M.com + 3 * i);
      V3 c = P + mul(R, com);
      const float trG = G.m[0] + G.m[4] + G.m[8];
      M33 Gs;   // G + G^T
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Gs.m[3 * a + b] = G.m[3 * a + b] + G.m[3 * b + a];
      V3 cb = m * hb + m * (2.f * trG * c - mul(Gs, c));
      const float* ic = M.icom + 6 * i;
      M33 Ic;
      Ic.m[0] = __ldg(ic); Ic.m[4] = __ldg(ic + 1); Ic.m[8] = __ldg(ic + 2);
      Ic.m[1] = Ic.m[3] = __ldg(ic + 3); Ic.m[2] = Ic.m[6] = __ldg(ic + 4); Ic.m[5] = Ic.m[7] = __ldg(ic + 5);
      M33 GRI = mul(mul(Gs, R), Ic);
#pragma unroll
      for (int k = 0; k < 9; ++k) Rb.m[k] += GRI.m[k];
      Pb = Pb + cb;
      Rb.m[0] += cb.x * com.x; Rb.m[1] += cb.x * com.y; Rb.m[2] += cb.x * com.z;
      Rb.m[3] += cb.y * com.x; Rb.m[4] += cb.y * com.y; Rb.m[5] += cb.y * com.z;
      Rb.m[6] += cb.z * com.x; Rb.m[7] += cb.z * com.y; Rb.m[8] += cb.z * com.z;
    }
    stm(w, M.o_RB + 9 * i, Rb);
    st3(w, M.o_PB + 3 * i, Pb);
  }
  team_sync(nl);
  // forward kinematics, leaves first; each link gathers its children's
  // contributions (o_TP: R_bar 9 + P_bar 3 destined to the parent)
  for (int l = M.nlev - 1; l >= 0; --l) {
    for (int ii = __ldg(M.lvl_ptr + l) + lane; ii < __ldg(M.lvl_ptr + l + 1); ii += nl) {
      const int i = __ldg(M.lvl_link + ii);
      M33 Rb = ldm(w, M.o_RB + 9 * i);
      V3 Pb = ld3(w, M.o_PB + 3 * i);
      for (int k = __ldg(M.ch_ptr + i); k < __ldg(M.ch_ptr + i + 1); ++k) {
        const int c = __ldg(M.ch_idx + k);
#pragma unroll
        for (int t = 0; t < 9; ++t) Rb.m[t] += w[M.o_TP + 12 * c + t];
        Pb = Pb + ld3(w, M.o_TP + 12 * c + 9);
      }
      const int jt = __ldg(M.jtype + i), s = __ldg(M.qs + i), p = __ldg(M.parent + i);
      if (jt == J_FREE) {   // the root origin is the reference point: no position cotangent here
        float xb = 0.f, yb = 0.f, zb = 0.f, wb = 0.f;
        quat_to_R_adj(w[M.o_Q + s + 3], w[M.o_Q + s + 4], w[M.o_Q + s + 5], w[M.o_Q + s + 6], Rb, xb, yb, zb, wb);
        w[M.o_QB + s + 3] += xb; w[M.o_QB + s + 4] += yb; w[M.o_QB + s + 5] += zb; w[M.o_QB + s + 6] += wb;
        continue;
      }
      M33 R = ldm(w, M.o_R + 9 * i);
      V3 ax = cld3(M.axis + 3 * i);
      M33 Rjb;   // cotangent of Rj (joint frame in world)
      if (jt == J_REV) {
        // R = Rj Rot(ax, q); dR/dq = [a]x R with a = R ax
        V3 a = mul(R, ax);
        float qb = 0.f;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          V3 rc = col(R, cc);
          V3 d = cross(a, rc);
          qb += Rb.m[cc] * d.x + Rb.m[3 + cc] * d.y + Rb.m[6 + cc] * d.z;
        }
        w[M.o_QB + s] += qb;
        M33 Rot = axis_angle(ax, w[M.o_Q + s]);
        Rjb = mulBT(Rb, Rot);
      } else if (jt == J_PRIS) {
        // P = Pj + q Rj ax
        V3 a = mul(R, ax);
        w[M.o_QB + s] += dot(Pb, a);
        const float q = w[M.o_Q + s];
        Rjb = Rb;
        Rjb.m[0] += q * Pb.x * ax.x; Rjb.m[1] += q * Pb.x * ax.y; Rjb.m[2] += q * Pb.x * ax.z;
        Rjb.m[3] += q * Pb.y * ax.x; Rjb.m[4] += q * Pb.y * ax.y; Rjb.m[5] += q * Pb.y * ax.z;
        Rjb.m[6] += q * Pb.z * ax.x; Rjb.m[7] += q * Pb.z * ax.y; Rjb.m[8] += q * Pb.z * ax.z;
      } else {
        Rjb = Rb;
      }
      if (p >= 0) {
        // Rj = Rp jrot, Pj = Pp + Rp jpos
        M33 tp = mulBT(Rjb, cldm(M.jrot + 9 * i));
        V3 jp = cld3(M.jpos + 3 * i);
        tp.m[0] += Pb.x * jp.x; tp.m[1] += Pb.x * jp.y; tp.m[2] += Pb.x * jp.z;
        tp.m[3] += Pb.y * jp.x; tp.m[4] += Pb.y * jp.y; tp.m[5] += Pb.y * jp.z;
        tp.m[6] += Pb.z * jp.x; tp.m[7] += Pb.z * jp.y; tp.m[8] += Pb.z * jp.z;
#pragma unroll
        for (int t = 0; t < 9; ++t) w[M.o_TP + 12 * i + t] = tp.m[t];
        st3(w, M.o_TP + 12 * i + 9, Pb);
      }
    }
    team_sync(nl);
  }
}

// One reverse substep: o_Q/o_QD hold the substep start state, o_QB/o_QDB the
// cotangents of its end state; on return they hold the start-state cotangents,
// and o_ACTB has accumulated the action cotangent.
template <int NM, class Mem>
__device__ void substep_adjoint(const DevModel& M, const Mem& w, int lane, int nl) {
  substep_dynamics<NM>(M, w, lane, nl);     // recompute; the factor is kept for lambda
  st_integrate_adj(M, w, lane, nl);
  st_dynamics_adj<NM>(M, w, lane, nl);
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
