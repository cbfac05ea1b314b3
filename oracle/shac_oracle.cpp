// FP64 CPU oracle for the simulator step s_{t+1} = F(s_t, a_t) and its adjoint
// (paper Sec. 3.1, Eq. "backward" and Eq. "fwd_dynamics"; appendix A.1).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
// CUDA path is checked against.  It shares no code, header, table or helper
// with the CUDA library; only tests, the smoke check and the bench's CPU
// baseline leg load it.
//
// What it computes, written as the textbook definitions rather than as a fast
// algorithm:
//   * forward kinematics by composing link transforms parent -> child;
//   * the joint-space mass matrix M = sum_i (m_i Jv_i^T Jv_i + Jw_i^T I_i Jw_i)
//     from per-link COM Jacobians (the Lagrangian definition of M, used in
//     Sec. 3.1 through CRBA);
//   * the bias / inverse dynamics by the classical vector Newton-Euler
//     recursion (Luh-Walker-Paul), including gravity and the external contact
//     and muscle forces (the J^T f and c terms of Eq. fwd_dynamics);
//   * contact: the normal penalty with damping and the friction "linear step
//     function" of Sec. 3.1 (the contact-force equation), joint limits by the
//     penalty equation of Sec. 3.1;
//   * Cholesky factorisation and solve for the joint accelerations (Sec. 3.1);
//   * semi-implicit Euler integration (Sec. 3.1);
//   * the adjoint of Eq. backward as the literal product of the cotangent row
//     with the step Jacobian dF/ds, dF/da, where the Jacobian is obtained
//     exactly by forward-mode dual numbers (no hand-written reverse code);
//   * the window adjoint as the concatenation of step adjoints (appendix A.1).
//
// All functions are templated on the scalar T (double or a dual number).
// Branches (contact, friction regime, joint limits, clipping) are decided on
// the value part.
//
// FP32 error floor (a diagnostic, never a reference value): the same functions
// instantiated on Monte Carlo Arithmetic scalars (Parker, "Monte Carlo
// Arithmetic", 1997), whose every operation result is multiplied by a random
// factor 1 + u r, r uniform in [-1, 1), u = 2^-24 (the unit roundoff of
// FP32).  Over a few seeded runs, the spread of an output measures how far
// rounding every intermediate result to FP32 moves it: the floor below which
// an FP32 implementation of the map cannot be expected to agree with the
// exact FP64 result.  With u = 0 the perturbed runs equal the FP64 oracle bit
// for bit.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <array>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ---------------------------------------------------------------- scalars --
constexpr int ND = 16;   // tangent directions carried per dual pass

// Monte Carlo Arithmetic state of the calling thread: a splitmix64 generator
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// 2014) and the relative perturbation size u (0: exact FP64).
struct McaState { uint64_t s = 0; double u = 0.0; };
static thread_local McaState g_mca;

inline uint64_t splitmix64_next(uint64_t& x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
inline void mca_seed(uint64_t seed, uint64_t stream, double u) {
  g_mca.s = seed * 0xD1B54A32D192ED03ull + stream;
  splitmix64_next(g_mca.s);
  g_mca.u = u;
}
// x (1 + u r), r uniform in [-1, 1) from the top 53 bits of the generator
inline double mca_round(double x) {
  if (g_mca.u == 0.0) return x;
  const double r = (double)(splitmix64_next(g_mca.s) >> 11) * 0x1.0p-53 * 2.0 - 1.0;
  return x * (1.0 + g_mca.u * r);
}

// Rounding policies of the dual numbers: exact (the oracle), the value part
// perturbed after every operation (tangents exact), or values and tangents
// perturbed (every operation of the derivative computation as well).
struct Exact { static double fix(double x) { return x; } static double fixd(double x) { return x; } };
struct McaValue { static double fix(double x) { return mca_round(x); } static double fixd(double x) { return x; } };
struct McaFull { static double fix(double x) { return mca_round(x); } static double fixd(double x) { return mca_round(x); } };

template <class P>
struct DualT {
  double v;
  double d[ND];
  DualT() : v(0.0) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }
  DualT(double x) : v(x) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }
};
template <class P> inline DualT<P> operator+(const DualT<P>& a, const DualT<P>& b) { DualT<P> r; r.v = P::fix(a.v + b.v); for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(a.d[i] + b.d[i]); return r; }
template <class P> inline DualT<P> operator-(const DualT<P>& a, const DualT<P>& b) { DualT<P> r; r.v = P::fix(a.v - b.v); for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(a.d[i] - b.d[i]); return r; }
template <class P> inline DualT<P> operator-(const DualT<P>& a) { DualT<P> r; r.v = -a.v; for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r; }
template <class P> inline DualT<P> operator*(const DualT<P>& a, const DualT<P>& b) { DualT<P> r; r.v = P::fix(a.v * b.v); for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(P::fixd(a.d[i] * b.v) + P::fixd(a.v * b.d[i])); return r; }
template <class P> inline DualT<P> operator/(const DualT<P>& a, const DualT<P>& b) {
  DualT<P> r; r.v = P::fix(a.v / b.v); double ib = P::fixd(1.0 / P::fixd(b.v * b.v));
  for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(P::fixd(P::fixd(a.d[i] * b.v) - P::fixd(a.v * b.d[i])) * ib); return r;
}
template <class P> inline DualT<P> operator+(const DualT<P>& a, double b) { DualT<P> r = a; r.v = P::fix(r.v + b); return r; }
template <class P> inline DualT<P> operator+(double a, const DualT<P>& b) { DualT<P> r = b; r.v = P::fix(r.v + a); return r; }
template <class P> inline DualT<P> operator-(const DualT<P>& a, double b) { DualT<P> r = a; r.v = P::fix(r.v - b); return r; }
template <class P> inline DualT<P> operator-(double a, const DualT<P>& b) { DualT<P> r = -b; r.v = P::fix(r.v + a); return r; }
template <class P> inline DualT<P> operator*(const DualT<P>& a, double b) { DualT<P> r; r.v = P::fix(a.v * b); for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(a.d[i] * b); return r; }
template <class P> inline DualT<P> operator*(double a, const DualT<P>& b) { return b * a; }
template <class P> inline DualT<P> operator/(const DualT<P>& a, double b) { return a * (1.0 / b); }
template <class P> inline DualT<P>& operator+=(DualT<P>& a, const DualT<P>& b) { a = a + b; return a; }
template <class P> inline DualT<P>& operator-=(DualT<P>& a, const DualT<P>& b) { a = a - b; return a; }
template <class P> inline DualT<P>& operator*=(DualT<P>& a, const DualT<P>& b) { a = a * b; return a; }
template <class P> inline DualT<P> sqrt(const DualT<P>& a) { DualT<P> r; r.v = P::fix(std::sqrt(a.v)); double k = P::fixd(0.5 / r.v); for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(a.d[i] * k); return r; }
template <class P> inline DualT<P> sin(const DualT<P>& a) { DualT<P> r; r.v = P::fix(std::sin(a.v)); double k = P::fixd(std::cos(a.v)); for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(a.d[i] * k); return r; }
template <class P> inline DualT<P> cos(const DualT<P>& a) { DualT<P> r; r.v = P::fix(std::cos(a.v)); double k = P::fixd(-std::sin(a.v)); for (int i = 0; i < ND; ++i) r.d[i] = P::fixd(a.d[i] * k); return r; }
template <class P> inline double val(const DualT<P>& a) { return a.v; }
using Dual = DualT<Exact>;

// Monte Carlo Arithmetic scalar: a double whose every operation result is
// perturbed (mca_round).
struct Mca {
  double v;
  Mca() : v(0.0) {}
  Mca(double x) : v(x) {}
};
inline Mca operator+(const Mca& a, const Mca& b) { return Mca(mca_round(a.v + b.v)); }
inline Mca operator-(const Mca& a, const Mca& b) { return Mca(mca_round(a.v - b.v)); }
inline Mca operator-(const Mca& a) { return Mca(-a.v); }
inline Mca operator*(const Mca& a, const Mca& b) { return Mca(mca_round(a.v * b.v)); }
inline Mca operator/(const Mca& a, const Mca& b) { return Mca(mca_round(a.v / b.v)); }
inline Mca operator+(const Mca& a, double b) { return Mca(mca_round(a.v + b)); }
inline Mca operator+(double a, const Mca& b) { return Mca(mca_round(a + b.v)); }
inline Mca operator-(const Mca& a, double b) { return Mca(mca_round(a.v - b)); }
inline Mca operator-(double a, const Mca& b) { return Mca(mca_round(a - b.v)); }
inline Mca operator*(const Mca& a, double b) { return Mca(mca_round(a.v * b)); }
inline Mca operator*(double a, const Mca& b) { return Mca(mca_round(a * b.v)); }
inline Mca operator/(const Mca& a, double b) { return Mca(mca_round(a.v / b)); }
inline Mca& operator+=(Mca& a, const Mca& b) { a = a + b; return a; }
inline Mca& operator-=(Mca& a, const Mca& b) { a = a - b; return a; }
inline Mca& operator*=(Mca& a, const Mca& b) { a = a * b; return a; }
inline Mca sqrt(const Mca& a) { return Mca(mca_round(std::sqrt(a.v))); }
inline Mca sin(const Mca& a) { return Mca(mca_round(std::sin(a.v))); }
inline Mca cos(const Mca& a) { return Mca(mca_round(std::cos(a.v))); }
inline double val(const Mca& a) { return a.v; }

inline double val(double a) { return a; }
using std::sqrt; using std::sin; using std::cos;

// ------------------------------------------------------------------ model --
enum { J_FREE = 0, J_REVOLUTE = 1, J_PRISMATIC = 2, J_FIXED = 3 };

struct Model {
  int L = 0, nq = 0, nv = 0, na = 0, ntact = 0, nc = 0, nm = 0;
  std::vector<int> parent, jtype, qs, ds;
  std::vector<double> axis, jpos, jrot, mass, com, inert;   // jrot 9/link, inert 9/link (about COM)
  std::vector<int> clink; std::vector<double> cpos, crad;
  std::vector<double> qlo, qhi, arm, damp; double klim = 0;
  std::vector<int> act_dof; std::vector<double> act_gear;
  std::vector<int> mptr, vlink; std::vector<double> vpos, fmax;
  double dt = 0; int K = 1; double g[3] = {0, 0, 0}; double ke = 0, kd = 0, kt = 0, mu = 0;
  std::vector<double> rwq, rwqd; double rc[10] = {0};
  int height_q = -1, vx_dof = -1;   // reward coordinates of a model without a free root
};

template <class T> using V3 = std::array<T, 3>;
template <class T> using M3 = std::array<T, 9>;   // row major

template <class T> V3<T> add(const V3<T>& a, const V3<T>& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
template <class T> V3<T> sub(const V3<T>& a, const V3<T>& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
template <class T, class S> V3<T> scale(const V3<T>& a, const S& s) { return {a[0] * s, a[1] * s, a[2] * s}; }
template <class T> T dot(const V3<T>& a, const V3<T>& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T> V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
template <class T> V3<T> mv(const M3<T>& R, const V3<T>& x) {
  return {R[0] * x[0] + R[1] * x[1] + R[2] * x[2], R[3] * x[0] + R[4] * x[1] + R[5] * x[2],
          R[6] * x[0] + R[7] * x[1] + R[8] * x[2]};
}
template <class T> V3<T> mtv(const M3<T>& R, const V3<T>& x) {   // R^T x
  return {R[0] * x[0] + R[3] * x[1] + R[6] * x[2], R[1] * x[0] + R[4] * x[1] + R[7] * x[2],
          R[2] * x[0] + R[5] * x[1] + R[8] * x[2]};
}
template <class T> M3<T> mm(const M3<T>& A, const M3<T>& B) {
  M3<T> C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
  return C;
}
template <class T> M3<T> to_T(const double* r) { M3<T> o; for (int i = 0; i < 9; ++i) o[i] = T(r[i]); return o; }
template <class T> V3<T> to_T3(const double* r) { return {T(r[0]), T(r[1]), T(r[2])}; }

// Unit-quaternion rotation matrix, quaternion stored x, y, z, w.
template <class T> M3<T> quat_rot(const T& x, const T& y, const T& z, const T& w) {
  return {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - z * w), 2.0 * (x * z + y * w),
          2.0 * (x * y + z * w), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - x * w),
          2.0 * (x * z - y * w), 2.0 * (y * z + x * w), 1.0 - 2.0 * (x * x + y * y)};
}
// Rotation by angle t about unit axis a (Rodrigues' formula).
template <class T> M3<T> axis_rot(const double* a, const T& t) {
  T c = cos(t), s = sin(t); T omc = 1.0 - c;
  return {c + omc * (a[0] * a[0]), omc * (a[0] * a[1]) - s * a[2], omc * (a[0] * a[2]) + s * a[1],
          omc * (a[1] * a[0]) + s * a[2], c + omc * (a[1] * a[1]), omc * (a[1] * a[2]) - s * a[0],
          omc * (a[2] * a[0]) - s * a[1], omc * (a[2] * a[1]) + s * a[0], c + omc * (a[2] * a[2])};
}

// Per-link world quantities.
template <class T> struct Kin {
  std::vector<M3<T>> R;           // link orientation
  std::vector<V3<T>> o, c, ax;    // link origin (= joint position), COM, joint axis (world)
  std::vector<V3<T>> w, vo;       // angular velocity, velocity of the link origin
};

template <class T>
void kinematics(const Model& m, const T* q, const T* qd, Kin<T>& k, bool with_vel) {
  k.R.resize(m.L); k.o.resize(m.L); k.c.resize(m.L); k.ax.resize(m.L);
  k.w.resize(m.L); k.vo.resize(m.L);
  for (int i = 0; i < m.L; ++i) {
    int p = m.parent[i];
    const int s = m.qs[i], d = m.ds[i];
    if (m.jtype[i] == J_FREE) {
      k.R[i] = quat_rot(q[s + 3], q[s + 4], q[s + 5], q[s + 6]);
      k.o[i] = {q[s], q[s + 1], q[s + 2]};
      k.ax[i] = {T(0.0), T(0.0), T(0.0)};
    } else {
      M3<T> Rp; V3<T> op;
      if (p < 0) { Rp = {T(1.0), T(0.0), T(0.0), T(0.0), T(1.0), T(0.0), T(0.0), T(0.0), T(1.0)}; op = {T(0.0), T(0.0), T(0.0)}; }
      else { Rp = k.R[p]; op = k.o[p]; }
      M3<T> Rj = mm(Rp, to_T<T>(&m.jrot[9 * i]));
      V3<T> oj = add(op, mv(Rp, to_T3<T>(&m.jpos[3 * i])));
      V3<T> a = mv(Rj, to_T3<T>(&m.axis[3 * i]));
      k.ax[i] = a;
      if (m.jtype[i] == J_REVOLUTE) { k.R[i] = mm(Rj, axis_rot(&m.axis[3 * i], q[s])); k.o[i] = oj; }
      else if (m.jtype[i] == J_PRISMATIC) { k.R[i] = Rj; k.o[i] = add(oj, scale(a, q[s])); }
      else { k.R[i] = Rj; k.o[i] = oj; }
    }
    k.c[i] = add(k.o[i], mv(k.R[i], to_T3<T>(&m.com[3 * i])));
    if (!with_vel) continue;
    V3<T> wp{T(0.0), T(0.0), T(0.0)}, vp{T(0.0), T(0.0), T(0.0)}, op{T(0.0), T(0.0), T(0.0)};
    if (p >= 0) { wp = k.w[p]; vp = k.vo[p]; op = k.o[p]; }
    switch (m.jtype[i]) {
      case J_FREE:
        k.w[i] = mv(k.R[i], V3<T>{qd[d], qd[d + 1], qd[d + 2]});
        k.vo[i] = mv(k.R[i], V3<T>{qd[d + 3], qd[d + 4], qd[d + 5]});
        break;
      case J_REVOLUTE:
        k.w[i] = add(wp, scale(k.ax[i], qd[d]));
        k.vo[i] = add(vp, cross(wp, sub(k.o[i], op)));
        break;
      case J_PRISMATIC:
        k.w[i] = wp;
        k.vo[i] = add(add(vp, cross(wp, sub(k.o[i], op))), scale(k.ax[i], qd[d]));
        break;
      default:
        k.w[i] = wp;
        k.vo[i] = add(vp, cross(wp, sub(k.o[i], op)));
    }
  }
}

// velocity of the material point x of link i
template <class T> V3<T> point_vel(const Kin<T>& k, int i, const V3<T>& x) {
  return add(k.vo[i], cross(k.w[i], sub(x, k.o[i])));
}

// External point forces (contact + muscles): list of (link, point, force).
template <class T> struct PointForce { int link; V3<T> x; V3<T> f; };

template <class T>
void contact_forces(const Model& m, const Kin<T>& k, std::vector<PointForce<T>>& out) {
  // Sec. 3.1 contact model against the ground plane z = 0, normal n = +z:
  //   f_c = (-k_n + k_d ddot) min(d, 0) n,
  //   f_t = -v_t/|v_t| min(k_t |v_t|, mu |f_c|).
  for (int c = 0; c < m.nc; ++c) {
    int i = m.clink[c];
    V3<T> centre = add(k.o[i], mv(k.R[i], to_T3<T>(&m.cpos[3 * c])));
    V3<T> x = {centre[0], centre[1], centre[2] - m.crad[c]};   // lowest point of the sphere
    T d = x[2];                                                 // signed gap
    if (!(val(d) < 0.0)) continue;                              // min(d, 0) = 0: no force
    V3<T> vp = point_vel(k, i, x);
    T ddot = vp[2];
    T fn = (-m.ke + m.kd * ddot) * d;                           // n-component of f_c
    T vtx = vp[0], vty = vp[1];
    T vt2 = vtx * vtx + vty * vty;
    T afn = val(fn) >= 0.0 ? fn : -fn;                          // |f_c|
    T fx, fy;
    // viscous branch when k_t |v_t| <= mu |f_c| (ties go to it; both agree there)
    if (m.kt * std::sqrt(val(vt2)) <= m.mu * val(afn)) {
      fx = -m.kt * vtx; fy = -m.kt * vty;
    } else {
      T vt = sqrt(vt2);
      T s = m.mu * afn / vt;
      fx = -s * vtx; fy = -s * vty;
    }
    out.push_back({i, x, V3<T>{fx, fy, fn}});
  }
}

template <class T>
void muscle_forces(const Model& m, const Kin<T>& k, const T* act, std::vector<PointForce<T>>& out) {
  // Sec. 3.1 muscles: a list of attachment sites; a purely contractive force of
  // magnitude activation * Fmax pulls each pair of consecutive sites together.
  for (int mu_ = 0; mu_ < m.nm; ++mu_) {
    T a = act[m.ntact + mu_];
    if (val(a) < 0.0) a = T(0.0);
    if (val(a) > 1.0) a = T(1.0);
    T F = a * m.fmax[mu_];
    for (int v = m.mptr[mu_]; v + 1 < m.mptr[mu_ + 1]; ++v) {
      int l0 = m.vlink[v], l1 = m.vlink[v + 1];
      V3<T> x0 = add(k.o[l0], mv(k.R[l0], to_T3<T>(&m.vpos[3 * v])));
      V3<T> x1 = add(k.o[l1], mv(k.R[l1], to_T3<T>(&m.vpos[3 * (v + 1)])));
      V3<T> dvec = sub(x1, x0);
      T len = sqrt(dot(dvec, dvec));
      V3<T> u = scale(dvec, T(1.0) / len);
      out.push_back({l0, x0, scale(u, F)});
      out.push_back({l1, x1, scale(u, -F)});
    }
  }
}

template <class T>
T muscle_length(const Model& m, const Kin<T>& k, int mu_) {
  T len = T(0.0);
  for (int v = m.mptr[mu_]; v + 1 < m.mptr[mu_ + 1]; ++v) {
    int l0 = m.vlink[v], l1 = m.vlink[v + 1];
    V3<T> x0 = add(k.o[l0], mv(k.R[l0], to_T3<T>(&m.vpos[3 * v])));
    V3<T> x1 = add(k.o[l1], mv(k.R[l1], to_T3<T>(&m.vpos[3 * (v + 1)])));
    V3<T> dvec = sub(x1, x0);
    len = len + sqrt(dot(dvec, dvec));
  }
  return len;
}

template <class T> M3<T> world_inertia(const Model& m, const Kin<T>& k, int i) {
  // R I_com R^T
  M3<T> I = to_T<T>(&m.inert[9 * i]);
  M3<T> RI = mm(k.R[i], I);
  M3<T> out;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      out[3 * a + b] = RI[3 * a] * k.R[i][3 * b] + RI[3 * a + 1] * k.R[i][3 * b + 1] + RI[3 * a + 2] * k.R[i][3 * b + 2];
  return out;
}

// Inverse dynamics by the vector Newton-Euler recursion: returns the joint
// forces that produce accelerations qdd under gravity and the given external
// point forces (tau = M qdd + c - J^T f in the notation of Eq. fwd_dynamics).
template <class T>
void inverse_dynamics(const Model& m, const Kin<T>& k, const T* qd, const T* qdd,
                      const std::vector<PointForce<T>>& ext, T* tau) {
  const int L = m.L;
  std::vector<V3<T>> al(L), ao(L), f(L), n(L), F(L), N(L);
  V3<T> z{T(0.0), T(0.0), T(0.0)};
  // outward pass: angular acceleration and acceleration of each link origin
  for (int i = 0; i < L; ++i) {
    int p = m.parent[i];
    const int d = m.ds[i];
    V3<T> wp = z, alp = z, aop = z, op = z;
    if (p >= 0) { wp = k.w[p]; alp = al[p]; aop = ao[p]; op = k.o[p]; }
    switch (m.jtype[i]) {
      case J_FREE: {
        V3<T> wb{qd[d], qd[d + 1], qd[d + 2]};
        V3<T> dwb{qdd[d], qdd[d + 1], qdd[d + 2]};
        V3<T> dvb{qdd[d + 3], qdd[d + 4], qdd[d + 5]};
        (void)wb;
        al[i] = mv(k.R[i], dwb);                                  // d/dt (R w_b) = R dw_b
        ao[i] = add(mv(k.R[i], dvb), cross(k.w[i], k.vo[i]));     // d/dt (R v_b)
        break;
      }
      case J_REVOLUTE: {
        V3<T> r = sub(k.o[i], op);
        al[i] = add(add(alp, scale(k.ax[i], qdd[d])), cross(wp, scale(k.ax[i], qd[d])));
        ao[i] = add(add(aop, cross(alp, r)), cross(wp, cross(wp, r)));
        break;
      }
      case J_PRISMATIC: {
        V3<T> r = sub(k.o[i], op);
        al[i] = alp;
        ao[i] = add(add(add(aop, cross(alp, r)), cross(wp, cross(wp, r))),
                    add(scale(cross(wp, scale(k.ax[i], qd[d])), 2.0), scale(k.ax[i], qdd[d])));
        break;
      }
      default: {
        V3<T> r = sub(k.o[i], op);
        al[i] = alp;
        ao[i] = add(add(aop, cross(alp, r)), cross(wp, cross(wp, r)));
      }
    }
    // Newton-Euler about the COM
    V3<T> rc = sub(k.c[i], k.o[i]);
    V3<T> ac = add(add(ao[i], cross(al[i], rc)), cross(k.w[i], cross(k.w[i], rc)));
    V3<T> g = to_T3<T>(m.g);
    f[i] = scale(sub(ac, g), T(m.mass[i]));
    M3<T> Iw = world_inertia(m, k, i);
    n[i] = add(mv(Iw, al[i]), cross(k.w[i], mv(Iw, k.w[i])));
  }
  for (const auto& e : ext) {
    f[e.link] = sub(f[e.link], e.f);
    n[e.link] = sub(n[e.link], cross(sub(e.x, k.c[e.link]), e.f));
  }
  // inward pass: joint force F_i and moment N_i about the joint origin o_i
  for (int i = 0; i < L; ++i) { F[i] = f[i]; N[i] = add(n[i], cross(sub(k.c[i], k.o[i]), f[i])); }
  for (int i = L - 1; i >= 0; --i) {
    int p = m.parent[i];
    if (p >= 0) {
      F[p] = add(F[p], F[i]);
      N[p] = add(N[p], add(N[i], cross(sub(k.o[i], k.o[p]), F[i])));
    }
  }
  for (int i = 0; i < L; ++i) {
    const int d = m.ds[i];
    switch (m.jtype[i]) {
      case J_FREE: {
        V3<T> tw = mtv(k.R[i], N[i]), tv = mtv(k.R[i], F[i]);
        for (int a = 0; a < 3; ++a) { tau[d + a] = tw[a]; tau[d + 3 + a] = tv[a]; }
        break;
      }
      case J_REVOLUTE: tau[d] = dot(k.ax[i], N[i]); break;
      case J_PRISMATIC: tau[d] = dot(k.ax[i], F[i]); break;
      default: break;
    }
  }
}

// Per-link COM Jacobians (world frame): Jv (3 x nv) and Jw (3 x nv), row major.
template <class T>
void com_jacobian(const Model& m, const Kin<T>& k, int i, std::vector<T>& Jv, std::vector<T>& Jw) {
  Jv.assign(3 * m.nv, T(0.0)); Jw.assign(3 * m.nv, T(0.0));
  for (int j = i; j >= 0; j = m.parent[j]) {
    const int d = m.ds[j];
    if (m.jtype[j] == J_FREE) {
      V3<T> r = sub(k.c[i], k.o[j]);
      for (int a = 0; a < 3; ++a) {
        V3<T> col{k.R[j][a], k.R[j][3 + a], k.R[j][6 + a]};   // world image of body axis a
        for (int row = 0; row < 3; ++row) Jw[row * m.nv + d + a] = col[row];
        V3<T> lin = cross(col, r);
        for (int row = 0; row < 3; ++row) Jv[row * m.nv + d + a] = lin[row];
        for (int row = 0; row < 3; ++row) Jv[row * m.nv + d + 3 + a] = col[row];
      }
    } else if (m.jtype[j] == J_REVOLUTE) {
      V3<T> lin = cross(k.ax[j], sub(k.c[i], k.o[j]));
      for (int row = 0; row < 3; ++row) { Jw[row * m.nv + d] = k.ax[j][row]; Jv[row * m.nv + d] = lin[row]; }
    } else if (m.jtype[j] == J_PRISMATIC) {
      for (int row = 0; row < 3; ++row) Jv[row * m.nv + d] = k.ax[j][row];
    }
  }
}

template <class T>
void mass_matrix(const Model& m, const Kin<T>& k, T* M) {
  const int n = m.nv;
  for (int a = 0; a < n * n; ++a) M[a] = T(0.0);
  std::vector<T> Jv, Jw;
  for (int i = 0; i < m.L; ++i) {
    if (m.mass[i] == 0.0 && m.inert[9 * i] == 0.0 && m.inert[9 * i + 4] == 0.0 && m.inert[9 * i + 8] == 0.0) continue;
    com_jacobian(m, k, i, Jv, Jw);
    M3<T> Iw = world_inertia(m, k, i);
    for (int a = 0; a < n; ++a) {
      V3<T> wa{Jw[a], Jw[n + a], Jw[2 * n + a]};
      V3<T> Iwa = mv(Iw, wa);
      for (int b = 0; b < n; ++b) {
        T s = m.mass[i] * (Jv[a] * Jv[b] + Jv[n + a] * Jv[n + b] + Jv[2 * n + a] * Jv[2 * n + b]);
        s = s + Iwa[0] * Jw[b] + Iwa[1] * Jw[n + b] + Iwa[2] * Jw[2 * n + b];
        M[a * n + b] = M[a * n + b] + s;
      }
    }
  }
}

// Joint-space forces from actuation, joint limits and joint damping.
template <class T>
void joint_forces(const Model& m, const T* q, const T* qd, const T* act, T* tau) {
  for (int a = 0; a < m.nv; ++a) tau[a] = T(0.0);
  for (int a = 0; a < m.ntact; ++a) tau[m.act_dof[a]] = tau[m.act_dof[a]] + m.act_gear[a] * act[a];
  for (int i = 0; i < m.L; ++i) {
    if (m.jtype[i] != J_REVOLUTE && m.jtype[i] != J_PRISMATIC) continue;
    const int d = m.ds[i], s = m.qs[i];
    // Sec. 3.1 joint-limit penalty; zero inside [lower, upper]
    if (val(q[s]) < m.qlo[d]) tau[d] = tau[d] + m.klim * (m.qlo[d] - q[s]);
    else if (val(q[s]) > m.qhi[d]) tau[d] = tau[d] + m.klim * (m.qhi[d] - q[s]);
  }
  for (int a = 0; a < m.nv; ++a) tau[a] = tau[a] - m.damp[a] * qd[a];
}

// Cholesky M = L L^T (lower, row major) and the solve L L^T x = b.
template <class T> void cholesky(int n, const T* A, T* Lc) {
  for (int i = 0; i < n * n; ++i) Lc[i] = T(0.0);
  for (int j = 0; j < n; ++j) {
    T s = A[j * n + j];
    for (int k2 = 0; k2 < j; ++k2) s = s - Lc[j * n + k2] * Lc[j * n + k2];
    Lc[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      T t = A[i * n + j];
      for (int k2 = 0; k2 < j; ++k2) t = t - Lc[i * n + k2] * Lc[j * n + k2];
      Lc[i * n + j] = t / Lc[j * n + j];
    }
  }
}
template <class T> void chol_solve(int n, const T* Lc, const T* b, T* x) {
  std::vector<T> y(n);
  for (int i = 0; i < n; ++i) {
    T s = b[i];
    for (int k2 = 0; k2 < i; ++k2) s = s - Lc[i * n + k2] * y[k2];
    y[i] = s / Lc[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = y[i];
    for (int k2 = i + 1; k2 < n; ++k2) s = s - Lc[k2 * n + i] * x[k2];
    x[i] = s / Lc[i * n + i];
  }
}

// Joint accelerations from Eq. fwd_dynamics:
//   (M + diag(armature)) qdd = tau_joint + J^T f - c   with c incl. gravity.
template <class T>
void forward_accel(const Model& m, const T* q, const T* qd, const T* act, T* qdd) {
  const int n = m.nv;
  Kin<T> k;
  kinematics(m, q, qd, k, true);
  std::vector<PointForce<T>> ext;
  contact_forces(m, k, ext);
  muscle_forces(m, k, act, ext);
  std::vector<T> zero(n, T(0.0)), bias(n), tj(n), rhs(n), M(n * n), Lc(n * n);
  inverse_dynamics(m, k, qd, zero.data(), ext, bias.data());
  joint_forces(m, q, qd, act, tj.data());
  for (int a = 0; a < n; ++a) rhs[a] = tj[a] - bias[a];
  mass_matrix(m, k, M.data());
  for (int a = 0; a < n; ++a) M[a * n + a] = M[a * n + a] + m.arm[a];
  cholesky(n, M.data(), Lc.data());
  chol_solve(n, Lc.data(), rhs.data(), qdd);
}

// Semi-implicit Euler: velocities first, then positions with the new velocity.
// Free joint: p += dt R(quat) v_b ; quat <- normalise(quat + dt/2 quat (x) (w_b, 0)).
template <class T>
void integrate(const Model& m, T* q, T* qd, const T* qdd, double h) {
  for (int a = 0; a < m.nv; ++a) qd[a] = qd[a] + h * qdd[a];
  for (int i = 0; i < m.L; ++i) {
    const int s = m.qs[i], d = m.ds[i];
    if (m.jtype[i] == J_FREE) {
      T x = q[s + 3], y = q[s + 4], z = q[s + 5], w = q[s + 6];
      M3<T> R = quat_rot(x, y, z, w);
      V3<T> vw = mv(R, V3<T>{qd[d + 3], qd[d + 4], qd[d + 5]});
      for (int a = 0; a < 3; ++a) q[s + a] = q[s + a] + h * vw[a];
      T wx = qd[d], wy = qd[d + 1], wz = qd[d + 2];
      // quaternion product (x,y,z,w) (x) (wx,wy,wz,0)
      T px = w * wx + (y * wz - z * wy);
      T py = w * wy + (z * wx - x * wz);
      T pz = w * wz + (x * wy - y * wx);
      T pw = -(x * wx + y * wy + z * wz);
      T nx = x + 0.5 * h * px, ny = y + 0.5 * h * py, nz = z + 0.5 * h * pz, nw = w + 0.5 * h * pw;
      T inv = T(1.0) / sqrt(nx * nx + ny * ny + nz * nz + nw * nw);
      q[s + 3] = nx * inv; q[s + 4] = ny * inv; q[s + 5] = nz * inv; q[s + 6] = nw * inv;
    } else if (m.jtype[i] == J_REVOLUTE || m.jtype[i] == J_PRISMATIC) {
      q[s] = q[s] + h * qd[d];
    }
  }
}

// Per-step reward on the post-step state (appendix A.3 reward shapes).
template <class T>
T reward(const Model& m, const T* q, const T* qd, const T* act) {
  T r = T(0.0);
  for (int j = 0; j < m.nq; ++j) r = r - m.rwq[j] * q[j] * q[j];
  for (int j = 0; j < m.nv; ++j) r = r - m.rwqd[j] * qd[j] * qd[j];
  T a2 = T(0.0);
  for (int j = 0; j < m.na; ++j) a2 = a2 + act[j] * act[j];
  r = r - m.rc[0] * a2;
  // forward velocity, uprightness and heading, height: with a free root its
  // world x velocity, R[2][2], R[0][0] and q[2]; without one (planar models on
  // slide joints) qd[vx_dof] and q[height_q] when given
  int hq = -1;
  if (m.L > 0 && m.jtype[0] == J_FREE) {
    M3<T> R = quat_rot(q[3], q[4], q[5], q[6]);
    V3<T> vw = mv(R, V3<T>{qd[3], qd[4], qd[5]});
    r = r + m.rc[1] * vw[0] + m.rc[2] * R[8] + m.rc[3] * R[0];
    hq = 2;
  } else {
    if (m.vx_dof >= 0) r = r + m.rc[1] * qd[m.vx_dof];
    hq = m.height_q;
  }
  if (hq >= 0) {
    T D = q[hq] - m.rc[4];
    if (val(D) < m.rc[5]) D = T(m.rc[5]);
    if (val(D) > m.rc[6]) D = T(m.rc[6]);
    if (val(D) < 0.0) r = r + m.rc[7] * D * D + m.rc[8] * D;
    else r = r + m.rc[9] * D;
  }
  return r;
}

// One control step: K substeps with the action held, then the reward.
template <class T>
void step(const Model& m, const T* q, const T* qd, const T* act, T* qn, T* qdn, T* r) {
  for (int j = 0; j < m.nq; ++j) qn[j] = q[j];
  for (int j = 0; j < m.nv; ++j) qdn[j] = qd[j];
  std::vector<T> qdd(m.nv);
  const double h = m.dt / m.K;
  for (int s = 0; s < m.K; ++s) {
    forward_accel(m, qn, qdn, act, qdd.data());
    integrate(m, qn, qdn, qdd.data(), h);
  }
  *r = reward(m, qn, qdn, act);
}

// Exact step Jacobian: rows (q_next[nq], qd_next[nv], reward[1]),
// columns (q[nq], qd[nv], act[na]); row-major, by dual-number passes (D = Dual;
// DualT<McaValue> gives the derivatives along an FP32-perturbed evaluation).
template <class D = Dual>
void step_jacobian(const Model& m, const double* q, const double* qd, const double* act, double* J) {
  const int nin = m.nq + m.nv + m.na, nout = m.nq + m.nv + 1;
  std::vector<D> x(nin), qn(m.nq), qdn(m.nv);
  D r;
  for (int base = 0; base < nin; base += ND) {
    for (int i = 0; i < nin; ++i) {
      double v = i < m.nq ? q[i] : (i < m.nq + m.nv ? qd[i - m.nq] : act[i - m.nq - m.nv]);
      x[i] = D(v);
      if (i >= base && i < base + ND) x[i].d[i - base] = 1.0;
    }
    step(m, x.data(), x.data() + m.nq, x.data() + m.nq + m.nv, qn.data(), qdn.data(), &r);
    for (int o = 0; o < nout; ++o) {
      const D& y = o < m.nq ? qn[o] : (o < m.nq + m.nv ? qdn[o - m.nq] : r);
      for (int i = base; i < std::min(nin, base + ND); ++i) J[o * nin + i] = y.d[i - base];
    }
  }
}

// Eq. backward: (dL/ds_t, dL/da_t) = (dL/ds_{t+1}, dL/dr_t) [dF/ds_t, dF/da_t].
template <class D = Dual>
void step_vjp(const Model& m, const double* q, const double* qd, const double* act,
              const double* qn_bar, const double* qdn_bar, double r_bar,
              double* q_bar, double* qd_bar, double* act_bar) {
  const int nin = m.nq + m.nv + m.na, nout = m.nq + m.nv + 1;
  std::vector<double> J((size_t)nout * nin), ybar(nout);
  step_jacobian<D>(m, q, qd, act, J.data());
  for (int o = 0; o < m.nq; ++o) ybar[o] = qn_bar[o];
  for (int o = 0; o < m.nv; ++o) ybar[m.nq + o] = qdn_bar[o];
  ybar[nout - 1] = r_bar;
  for (int i = 0; i < nin; ++i) {
    double s = 0.0;
    for (int o = 0; o < nout; ++o) s += ybar[o] * J[(size_t)o * nin + i];
    if (i < m.nq) q_bar[i] = s;
    else if (i < m.nq + m.nv) qd_bar[i - m.nq] = s;
    else act_bar[i - m.nq - m.nv] = s;
  }
}

}  // namespace orc

// ------------------------------------------------------------------ C ABI --
extern "C" {

typedef struct {
  int32_t n_links; const int32_t* parent; const int32_t* joint_type;
  const double* joint_axis; const double* joint_pos; const double* joint_quat;
  const double* mass; const double* com; const double* inertia;
  int32_t n_contacts; const int32_t* contact_link; const double* contact_pos; const double* contact_radius;
  const double* q_lower; const double* q_upper; const double* armature; const double* damping; double k_limit;
  int32_t n_tact; const int32_t* act_dof; const double* act_gear;
  int32_t n_muscles; const int32_t* muscle_ptr; const int32_t* via_link; const double* via_pos; const double* muscle_fmax;
  double dt; int32_t substeps; double gravity[3]; double ke, kd, kt, mu;
  const double* rw_q; const double* rw_qd; double reward_coef[10];
  int32_t height_q; int32_t vx_dof;
} orc_desc;

static orc::Model make_model(const orc_desc* d) {
  orc::Model m;
  m.L = d->n_links;
  m.parent.assign(d->parent, d->parent + m.L);
  m.jtype.assign(d->joint_type, d->joint_type + m.L);
  m.qs.resize(m.L); m.ds.resize(m.L);
  int nq = 0, nv = 0;
  for (int i = 0; i < m.L; ++i) {
    m.qs[i] = nq; m.ds[i] = nv;
    int t = m.jtype[i];
    nq += t == orc::J_FREE ? 7 : (t == orc::J_FIXED ? 0 : 1);
    nv += t == orc::J_FREE ? 6 : (t == orc::J_FIXED ? 0 : 1);
  }
  m.nq = nq; m.nv = nv;
  m.axis.assign(d->joint_axis, d->joint_axis + 3 * m.L);
  m.jpos.assign(d->joint_pos, d->joint_pos + 3 * m.L);
  m.jrot.resize(9 * m.L);
  for (int i = 0; i < m.L; ++i) {
    const double* qq = d->joint_quat + 4 * i;
    orc::M3<double> R = orc::quat_rot(qq[0], qq[1], qq[2], qq[3]);
    for (int a = 0; a < 9; ++a) m.jrot[9 * i + a] = R[a];
  }
  m.mass.assign(d->mass, d->mass + m.L);
  m.com.assign(d->com, d->com + 3 * m.L);
  m.inert.resize(9 * m.L);
  for (int i = 0; i < m.L; ++i) {
    const double* s = d->inertia + 6 * i;   // xx yy zz xy xz yz
    double full[9] = {s[0], s[3], s[4], s[3], s[1], s[5], s[4], s[5], s[2]};
    for (int a = 0; a < 9; ++a) m.inert[9 * i + a] = full[a];
  }
  m.nc = d->n_contacts;
  m.clink.assign(d->contact_link, d->contact_link + m.nc);
  m.cpos.assign(d->contact_pos, d->contact_pos + 3 * m.nc);
  m.crad.assign(d->contact_radius, d->contact_radius + m.nc);
  m.qlo.assign(d->q_lower, d->q_lower + nv); m.qhi.assign(d->q_upper, d->q_upper + nv);
  m.arm.assign(d->armature, d->armature + nv); m.damp.assign(d->damping, d->damping + nv);
  m.klim = d->k_limit;
  m.ntact = d->n_tact;
  m.act_dof.assign(d->act_dof, d->act_dof + m.ntact);
  m.act_gear.assign(d->act_gear, d->act_gear + m.ntact);
  m.nm = d->n_muscles;
  m.mptr.assign(d->muscle_ptr, d->muscle_ptr + m.nm + 1);
  int nvia = m.mptr[m.nm];
  m.vlink.assign(d->via_link, d->via_link + nvia);
  m.vpos.assign(d->via_pos, d->via_pos + 3 * nvia);
  m.fmax.assign(d->muscle_fmax, d->muscle_fmax + m.nm);
  m.na = m.ntact + m.nm;
  m.dt = d->dt; m.K = d->substeps;
  for (int a = 0; a < 3; ++a) m.g[a] = d->gravity[a];
  m.ke = d->ke; m.kd = d->kd; m.kt = d->kt; m.mu = d->mu;
  m.rwq.assign(d->rw_q, d->rw_q + nq);
  m.rwqd.assign(d->rw_qd, d->rw_qd + nv);
  for (int a = 0; a < 10; ++a) m.rc[a] = d->reward_coef[a];
  m.height_q = d->height_q;
  m.vx_dof = d->vx_dof;
  return m;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Environment-batched entry points; every per-env array is [N][dim] (row per env).
void orc_step(const orc_desc* d, int32_t N, const double* q, const double* qd, const double* act,
              double* qn, double* qdn, double* r) {
  orc::Model m = make_model(d);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < N; ++e)
    orc::step<double>(m, q + (size_t)e * m.nq, qd + (size_t)e * m.nv, act + (size_t)e * m.na,
                      qn + (size_t)e * m.nq, qdn + (size_t)e * m.nv, r + e);
}

void orc_step_jacobian(const orc_desc* d, int32_t N, const double* q, const double* qd, const double* act, double* J) {
  orc::Model m = make_model(d);
  const size_t sz = (size_t)(m.nq + m.nv + 1) * (m.nq + m.nv + m.na);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < N; ++e)
    orc::step_jacobian(m, q + (size_t)e * m.nq, qd + (size_t)e * m.nv, act + (size_t)e * m.na, J + e * sz);
}

void orc_step_vjp(const orc_desc* d, int32_t N, const double* q, const double* qd, const double* act,
                  const double* qn_bar, const double* qdn_bar, const double* r_bar,
                  double* q_bar, double* qd_bar, double* act_bar) {
  orc::Model m = make_model(d);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < N; ++e)
    orc::step_vjp(m, q + (size_t)e * m.nq, qd + (size_t)e * m.nv, act + (size_t)e * m.na,
                  qn_bar + (size_t)e * m.nq, qdn_bar + (size_t)e * m.nv, r_bar[e],
                  q_bar + (size_t)e * m.nq, qd_bar + (size_t)e * m.nv, act_bar + (size_t)e * m.na);
}

// Window of h steps.  Trajectories are [t][N][dim].
void orc_window_forward(const orc_desc* d, int32_t N, int32_t h, const double* q0, const double* qd0,
                        const double* act, double* q_traj, double* qd_traj, double* rew) {
  orc::Model m = make_model(d);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < N; ++e) {
    for (int j = 0; j < m.nq; ++j) q_traj[(size_t)e * m.nq + j] = q0[(size_t)e * m.nq + j];
    for (int j = 0; j < m.nv; ++j) qd_traj[(size_t)e * m.nv + j] = qd0[(size_t)e * m.nv + j];
    for (int t = 0; t < h; ++t) {
      const double* qt = q_traj + ((size_t)t * N + e) * m.nq;
      const double* qdt = qd_traj + ((size_t)t * N + e) * m.nv;
      orc::step<double>(m, qt, qdt, act + ((size_t)t * N + e) * m.na,
                        q_traj + ((size_t)(t + 1) * N + e) * m.nq, qd_traj + ((size_t)(t + 1) * N + e) * m.nv,
                        rew + (size_t)t * N + e);
    }
  }
}

// Appendix A.1 recursion without the policy term: the state cotangent is
// carried backwards through each step's exact VJP, the reward cotangents
// r_bar[t] entering at step t (reward on the post-step state).
void orc_window_adjoint(const orc_desc* d, int32_t N, int32_t h, const double* q_traj, const double* qd_traj,
                        const double* act, const double* r_bar, const double* qT_bar, const double* qdT_bar,
                        double* q0_bar, double* qd0_bar, double* act_bar) {
  orc::Model m = make_model(d);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < N; ++e) {
    std::vector<double> qb(qT_bar + (size_t)e * m.nq, qT_bar + (size_t)(e + 1) * m.nq);
    std::vector<double> qdb(qdT_bar + (size_t)e * m.nv, qdT_bar + (size_t)(e + 1) * m.nv);
    std::vector<double> qb2(m.nq), qdb2(m.nv);
    for (int t = h - 1; t >= 0; --t) {
      orc::step_vjp(m, q_traj + ((size_t)t * N + e) * m.nq, qd_traj + ((size_t)t * N + e) * m.nv,
                    act + ((size_t)t * N + e) * m.na, qb.data(), qdb.data(), r_bar[(size_t)t * N + e],
                    qb2.data(), qdb2.data(), act_bar + ((size_t)t * N + e) * m.na);
      qb.swap(qb2); qdb.swap(qdb2);
    }
    for (int j = 0; j < m.nq; ++j) q0_bar[(size_t)e * m.nq + j] = qb[j];
    for (int j = 0; j < m.nv; ++j) qd0_bar[(size_t)e * m.nv + j] = qdb[j];
  }
}

// ---- FP32 error floor: Monte Carlo Arithmetic runs -------------------------
// Each environment e draws its perturbations from its own stream (seed, e), so
// results do not depend on the thread that runs it.  u = 0 gives the exact
// FP64 results.

void orc_mca_step(const orc_desc* d, int32_t N, const double* q, const double* qd, const double* act,
                  double* qn, double* qdn, double* r, uint64_t seed, double u) {
  orc::Model m = make_model(d);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < N; ++e) {
    orc::mca_seed(seed, (uint64_t)e, u);
    std::vector<orc::Mca> x(m.nq + m.nv + m.na), yq(m.nq), yqd(m.nv);
    for (int j = 0; j < m.nq; ++j) x[j] = orc::Mca(q[(size_t)e * m.nq + j]);
    for (int j = 0; j < m.nv; ++j) x[m.nq + j] = orc::Mca(qd[(size_t)e * m.nv + j]);
    for (int j = 0; j < m.na; ++j) x[m.nq + m.nv + j] = orc::Mca(act[(size_t)e * m.na + j]);
    orc::Mca rr;
    orc::step<orc::Mca>(m, x.data(), x.data() + m.nq, x.data() + m.nq + m.nv, yq.data(), yqd.data(), &rr);
    for (int j = 0; j < m.nq; ++j) qn[(size_t)e * m.nq + j] = yq[j].v;
    for (int j = 0; j < m.nv; ++j) qdn[(size_t)e * m.nv + j] = yqd[j].v;
    r[e] = rr.v;
    orc::mca_seed(0, 0, 0.0);
  }
}

// The window adjoint (as orc_window_adjoint) with every step's Jacobian taken
// along an FP32-perturbed evaluation of the step; tangents != 0 perturbs the
// derivative arithmetic too.
void orc_mca_window_adjoint(const orc_desc* d, int32_t N, int32_t h, const double* q_traj, const double* qd_traj,
                            const double* act, const double* r_bar, const double* qT_bar, const double* qdT_bar,
                            double* q0_bar, double* qd0_bar, double* act_bar, uint64_t seed, double u,
                            int32_t tangents) {
  orc::Model m = make_model(d);
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < N; ++e) {
    orc::mca_seed(seed, (uint64_t)e, u);
    std::vector<double> qb(qT_bar + (size_t)e * m.nq, qT_bar + (size_t)(e + 1) * m.nq);
    std::vector<double> qdb(qdT_bar + (size_t)e * m.nv, qdT_bar + (size_t)(e + 1) * m.nv);
    std::vector<double> qb2(m.nq), qdb2(m.nv);
    for (int t = h - 1; t >= 0; --t) {
      const double* qt = q_traj + ((size_t)t * N + e) * m.nq;
      const double* qdt = qd_traj + ((size_t)t * N + e) * m.nv;
      const double* at = act + ((size_t)t * N + e) * m.na;
      double* abt = act_bar + ((size_t)t * N + e) * m.na;
      if (tangents)
        orc::step_vjp<orc::DualT<orc::McaFull>>(m, qt, qdt, at, qb.data(), qdb.data(), r_bar[(size_t)t * N + e],
                                                 qb2.data(), qdb2.data(), abt);
      else
        orc::step_vjp<orc::DualT<orc::McaValue>>(m, qt, qdt, at, qb.data(), qdb.data(), r_bar[(size_t)t * N + e],
                                                  qb2.data(), qdb2.data(), abt);
      qb.swap(qb2); qdb.swap(qdb2);
    }
    for (int j = 0; j < m.nq; ++j) q0_bar[(size_t)e * m.nq + j] = qb[j];
    for (int j = 0; j < m.nv; ++j) qd0_bar[(size_t)e * m.nv + j] = qdb[j];
    orc::mca_seed(0, 0, 0.0);
  }
}

// Cholesky factorisation and solve of one n x n system in Monte Carlo
// Arithmetic (the pins check the floor's scaling with the condition number).
void orc_mca_chol_solve(int32_t n, const double* A, const double* b, double* x, uint64_t seed, double u) {
  orc::mca_seed(seed, 0, u);
  std::vector<orc::Mca> Am(A, A + (size_t)n * n), Lc((size_t)n * n), bm(b, b + n), xm(n);
  orc::cholesky<orc::Mca>(n, Am.data(), Lc.data());
  orc::chol_solve<orc::Mca>(n, Lc.data(), bm.data(), xm.data());
  for (int i = 0; i < n; ++i) x[i] = xm[i].v;
  orc::mca_seed(0, 0, 0.0);
}

// ---- single-state helpers used by the pins --------------------------------
void orc_forward_accel(const orc_desc* d, const double* q, const double* qd, const double* act, double* qdd) {
  orc::Model m = make_model(d);
  orc::forward_accel<double>(m, q, qd, act, qdd);
}

void orc_mass_matrix(const orc_desc* d, const double* q, double* M) {
  orc::Model m = make_model(d);
  orc::Kin<double> k;
  std::vector<double> qd(m.nv, 0.0);
  orc::kinematics(m, q, qd.data(), k, false);
  orc::mass_matrix(m, k, M);
}

// with_ext: include contact and muscle forces (act used for muscles only)
void orc_inverse_dynamics(const orc_desc* d, const double* q, const double* qd, const double* qdd,
                          const double* act, int32_t with_ext, double* tau) {
  orc::Model m = make_model(d);
  orc::Kin<double> k;
  orc::kinematics(m, q, qd, k, true);
  std::vector<orc::PointForce<double>> ext;
  if (with_ext) { orc::contact_forces(m, k, ext); orc::muscle_forces(m, k, act, ext); }
  orc::inverse_dynamics(m, k, qd, qdd, ext, tau);
}

void orc_joint_forces(const orc_desc* d, const double* q, const double* qd, const double* act, double* tau) {
  orc::Model m = make_model(d);
  orc::joint_forces<double>(m, q, qd, act, tau);
}

// out: [0] kinetic energy, [1] potential energy (-sum m g.c),
//      [2..4] linear momentum, [5..7] angular momentum about the world origin,
//      [8..10] centre of mass
void orc_energy_momentum(const orc_desc* d, const double* q, const double* qd, double* out) {
  orc::Model m = make_model(d);
  orc::Kin<double> k;
  orc::kinematics(m, q, qd, k, true);
  double T = 0, V = 0, P[3] = {0, 0, 0}, H[3] = {0, 0, 0}, C[3] = {0, 0, 0}, mt = 0;
  for (int i = 0; i < m.L; ++i) {
    orc::V3<double> vc = orc::point_vel(k, i, k.c[i]);
    orc::M3<double> Iw = orc::world_inertia(m, k, i);
    orc::V3<double> Iw_w = orc::mv(Iw, k.w[i]);
    T += 0.5 * m.mass[i] * orc::dot(vc, vc) + 0.5 * orc::dot(k.w[i], Iw_w);
    V -= m.mass[i] * (m.g[0] * k.c[i][0] + m.g[1] * k.c[i][1] + m.g[2] * k.c[i][2]);
    orc::V3<double> lin = orc::scale(vc, m.mass[i]);
    orc::V3<double> ang = orc::add(orc::cross(k.c[i], lin), Iw_w);
    for (int a = 0; a < 3; ++a) { P[a] += lin[a]; H[a] += ang[a]; C[a] += m.mass[i] * k.c[i][a]; }
    mt += m.mass[i];
  }
  out[0] = T; out[1] = V;
  for (int a = 0; a < 3; ++a) { out[2 + a] = P[a]; out[5 + a] = H[a]; out[8 + a] = C[a] / mt; }
}

// Link poses: R [L][9] row major, origin [L][3], COM [L][3].
void orc_link_poses(const orc_desc* d, const double* q, double* R, double* o, double* c) {
  orc::Model m = make_model(d);
  orc::Kin<double> k;
  std::vector<double> qd(m.nv, 0.0);
  orc::kinematics(m, q, qd.data(), k, false);
  for (int i = 0; i < m.L; ++i) {
    for (int a = 0; a < 9; ++a) R[9 * i + a] = k.R[i][a];
    for (int a = 0; a < 3; ++a) { o[3 * i + a] = k.o[i][a]; c[3 * i + a] = k.c[i][a]; }
  }
}

void orc_muscle_lengths(const orc_desc* d, const double* q, double* len) {
  orc::Model m = make_model(d);
  orc::Kin<double> k;
  std::vector<double> qd(m.nv, 0.0);
  orc::kinematics(m, q, qd.data(), k, false);
  for (int i = 0; i < m.nm; ++i) len[i] = orc::muscle_length(m, k, i);
}

void orc_cholesky(int32_t n, const double* A, double* Lc) { orc::cholesky<double>(n, A, Lc); }

}  // extern "C"
