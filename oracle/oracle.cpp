/*
 * ComFree step oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of one step of the complementarity-free contact method
 * of "ComFree-Sim" (arxiv 2603.12185).  It exists to check the CUDA path and to serve as the
 * timed CPU baseline; only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg
 * may load it.  It shares no code with the CUDA library.
 *
 * Every function is templated on the scalar type so that a forward-mode dual number gives
 * exact directional derivatives of a rollout (the reference gradient for the adjoint).
 *
 * The step follows the paper's order (Sec. III-A, Algorithm 1):
 *   1. forward kinematics of the bodies                       (Sec. III-A, multi-joint systems)
 *   2. joint-space inertia M (its definition sum_b J_b^T M_b J_b) and bias c (Newton-Euler),
 *      M~ = M + dt diag(damping) (implicit joint damping)
 *   3. smooth prediction  v_s = v + M~^-1 (tau - c - b.v) dt                  (Eq. smooth_vel)
 *   4. all-pairs narrowphase -> contacts (phi, point, normal)
 *   5. per contact: frame, relative Jacobian blocks J_n, J_t, J_tor, J_rol      (Sec. III-A)
 *      and the constraint-space impedance M(phi)                    (Eqs. k_d_setting, r_scaling)
 *      (or, trace_mode 2, the exact diagonal impedance of each facet, Sec. III-B; or,
 *      trace_mode 3, M(phi) scaled by a learned function of the contact's configuration,
 *      the learning-based K(q), D(q) that Sec. III-B allows)
 *   6. per facet: J~ = J_n - mu_s d_j^T J_s, s = J~ v_s,
 *      lambda dt = ( -k M(phi) (s dt + phi) - d M(phi) s )_+        (Eqs. tilde_defs, cf_wrench)
 *   7. p = sum J~^T lambda dt                                         (Algorithm 1, Kernel III)
 *   8. v+ = v_s + M~^-1 p                                              (Eq. vel_correction)
 *   9. semi-implicit Euler with the exact quaternion exponential.
 *
 * Where the paper is silent or garbled, the reading taken is restated at the function that
 * applies it.
 *
 * Parity pins (tests/test_oracle_pins.py) tie every stage to closed forms, hand-derived
 * worked examples, invariants, brute force or finite differences; tests/test_oracle_mutants.py
 * plants mistakes in copies of this file and checks that a pin catches each.  The paper's
 * penetration-depth table pins the order of its six impedance settings and, for a resting
 * sphere, their magnitudes within a third; parity unpinned: the paper's MJWarp-relative claims.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------
 * scalar types
 * ---------------------------------------------------------------------------------------- */
struct Dual {  // value + one directional derivative
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
static inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
static inline Dual& operator/=(Dual& a, Dual b) { a = a / b; return a; }
static inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
static inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
static inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
static inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
static inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, s > 0 ? a.d / (2 * s) : 0.0); }
static inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
static inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
static inline Dual fabs(Dual a) { return a.v < 0 ? -a : a; }
static inline Dual pow(Dual a, double p) {
  double r = std::pow(a.v, p);
  return Dual(r, a.v != 0 ? p * std::pow(a.v, p - 1) * a.d : 0.0);
}
static inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
static inline Dual tanh(Dual a) { double t = std::tanh(a.v); return Dual(t, (1.0 - t * t) * a.d); }
static inline double val(double a) { return a; }
static inline double val(Dual a) { return a.v; }
using std::sqrt; using std::sin; using std::cos; using std::fabs; using std::pow;

/* ------------------------------------------------------------------------------------------
 * C interface structs (doubles; layouts documented in oracle/oracle.py)
 * ---------------------------------------------------------------------------------------- */
extern "C" {
typedef struct {
  int nbody, ngeom;
  const int* body_parent;      /* [nbody] -1 = world                                   */
  const int* body_jnt;         /* [nbody] 0 free, 1 hinge                              */
  const double* body_pos;      /* [nbody*3] hinge frame origin in parent frame         */
  const double* body_quat;     /* [nbody*4] hinge frame orientation in parent frame    */
  const double* body_axis;     /* [nbody*3] hinge axis in body frame                   */
  const double* body_ipos;     /* [nbody*3] centre of mass in body frame               */
  const double* body_mass;     /* [nbody]                                              */
  const double* body_inertia;  /* [nbody*3] principal inertia, principal axes = body axes */
  const double* body_damping;  /* [nbody] hinge damping                                */
  const int* geom_type;        /* [ngeom] 0 plane 1 sphere 2 capsule 3 box             */
  const int* geom_body;        /* [ngeom] -1 static                                    */
  const double* geom_pos;      /* [ngeom*3] in body frame (world for static)           */
  const double* geom_quat;     /* [ngeom*4]                                            */
  const double* geom_size;     /* [ngeom*3]                                            */
  const double* geom_mu;       /* [ngeom*3] tangential, torsional, rolling             */
  const double* body_range;    /* [nbody*2] hinge limits (lower, upper); lower < upper limits */
  const double* body_frictionloss; /* [nbody] hinge dry friction (N m)                  */
} ow_world;

typedef struct {
  double gravity[3];
  double k_user, d_user;
  double solimp[5]; /* r_min, r_max, width, midpoint, power */
  double margin;
  int n_t, n_tor, n_rol;
  int trace_mode; /* 0: tr(J_i M~^-1 J_i^T) of the translational point Jacobian, 1: 1/m_i,
                     2: the exact diagonal impedance of Sec. III-B, one value per facet,
                     3: the mode-0 M(phi) times exp(g(x)), g the impedance network below */
  const double* impnet; /* trace_mode 3: the network's IMP_PARAMS parameters */
} ow_params;

/* one detected contact, for tests */
typedef struct {
  int geom_a, geom_b, body_a, body_b, sub;
  double phi, pos[3], normal[3], t1[3], t2[3];
  double trace_a, trace_b, r, mphi;
  double lam_sum;        /* sum of facet impulses (lambda dt)              */
  double wrench[6];      /* resultant impulse on A in the contact frame:
                            normal, t1, t2, torsional, rolling t1, rolling t2 */
  int nfacet;
  int nactive;
  double feat[4];        /* the impedance network's input x (see impnet_features)     */
  double m_exact;        /* mean over the facets of the exact diagonal impedance
                            M_j = 1 / ((k dt + d) J~_j M~^-1 J~_j^T) (Sec. III-B)       */
} ow_contact;
}

namespace orc {

enum { PLANE = 0, SPHERE = 1, CAPSULE = 2, BOX = 3, CYLINDER = 4, ELLIPSOID = 5 };
enum { FREE = 0, HINGE = 1 };

template <class S> struct V3 {
  S x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(S a, S b, S c) : x(a), y(b), z(c) {}
};
template <class S> V3<S> operator+(const V3<S>& a, const V3<S>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class S> V3<S> operator-(const V3<S>& a, const V3<S>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S> V3<S> operator-(const V3<S>& a) { return {-a.x, -a.y, -a.z}; }
template <class S> V3<S> operator*(S s, const V3<S>& a) { return {s * a.x, s * a.y, s * a.z}; }
template <class S> S dot(const V3<S>& a, const V3<S>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class S> S norm(const V3<S>& a) { return sqrt(dot(a, a)); }
template <class S> S comp(const V3<S>& a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

/* 3x3 matrix, row major */
template <class S> struct M3 {
  S m[9];
  M3() { for (int i = 0; i < 9; ++i) m[i] = S(0.0); }
  static M3 eye() { M3 r; r.m[0] = r.m[4] = r.m[8] = S(1.0); return r; }
  V3<S> col(int j) const { return {m[j], m[3 + j], m[6 + j]}; }
};
template <class S> V3<S> mul(const M3<S>& a, const V3<S>& v) {
  return {a.m[0] * v.x + a.m[1] * v.y + a.m[2] * v.z, a.m[3] * v.x + a.m[4] * v.y + a.m[5] * v.z,
          a.m[6] * v.x + a.m[7] * v.y + a.m[8] * v.z};
}
template <class S> V3<S> mulT(const M3<S>& a, const V3<S>& v) {
  return {a.m[0] * v.x + a.m[3] * v.y + a.m[6] * v.z, a.m[1] * v.x + a.m[4] * v.y + a.m[7] * v.z,
          a.m[2] * v.x + a.m[5] * v.y + a.m[8] * v.z};
}
template <class S> M3<S> mul(const M3<S>& a, const M3<S>& b) {
  M3<S> r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      S s(0.0);
      for (int k = 0; k < 3; ++k) s += a.m[3 * i + k] * b.m[3 * k + j];
      r.m[3 * i + j] = s;
    }
  return r;
}

/* quaternion (w, x, y, z) -> rotation matrix (normalised first) */
template <class S> M3<S> quat_to_mat(const S* qin) {
  S n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  S w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
  M3<S> r;
  r.m[0] = S(1.0) - S(2.0) * (y * y + z * z); r.m[1] = S(2.0) * (x * y - w * z); r.m[2] = S(2.0) * (x * z + w * y);
  r.m[3] = S(2.0) * (x * y + w * z); r.m[4] = S(1.0) - S(2.0) * (x * x + z * z); r.m[5] = S(2.0) * (y * z - w * x);
  r.m[6] = S(2.0) * (x * z - w * y); r.m[7] = S(2.0) * (y * z + w * x); r.m[8] = S(1.0) - S(2.0) * (x * x + y * y);
  return r;
}
template <class S> void quat_mul(const S* a, const S* b, S* out) {
  S r0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  S r1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  S r2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  S r3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  out[0] = r0; out[1] = r1; out[2] = r2; out[3] = r3;
}
/* rotation by angle about a unit axis (Rodrigues) */
template <class S> M3<S> axis_angle(const V3<S>& a, S th) {
  S c = cos(th), s = sin(th), t = S(1.0) - c;
  M3<S> r;
  r.m[0] = t * a.x * a.x + c;       r.m[1] = t * a.x * a.y - s * a.z; r.m[2] = t * a.x * a.z + s * a.y;
  r.m[3] = t * a.x * a.y + s * a.z; r.m[4] = t * a.y * a.y + c;       r.m[5] = t * a.y * a.z - s * a.x;
  r.m[6] = t * a.x * a.z - s * a.y; r.m[7] = t * a.y * a.z + s * a.x; r.m[8] = t * a.z * a.z + c;
  return r;
}

template <class S> static S smax(S a, S b) { return a > b ? a : b; }
template <class S> static S smin(S a, S b) { return a < b ? a : b; }
template <class S> static S clampv(S a, S lo, S hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* ------------------------------------------------------------------------------------------
 * model structure derived from the description
 * ---------------------------------------------------------------------------------------- */
struct Structure {
  int nbody, ngeom, nq, nv;
  std::vector<int> qadr, vadr, tree;   /* per body */
  std::vector<std::vector<int>> tree_bodies, tree_dofs;
  std::vector<int> dof_tree, dof_local;
};

static bool build_structure(const ow_world* w, Structure& st) {
  st.nbody = w->nbody; st.ngeom = w->ngeom;
  st.qadr.resize(w->nbody); st.vadr.resize(w->nbody); st.tree.resize(w->nbody);
  int nq = 0, nv = 0;
  for (int b = 0; b < w->nbody; ++b) {
    int p = w->body_parent[b];
    if (p >= b) return false;                          /* topological order required   */
    if (w->body_jnt[b] == FREE && p != -1) return false; /* free joints only at the root */
    if (p >= 0 && w->body_jnt[p] == FREE) return false;  /* no children of free bodies  */
    st.qadr[b] = nq; st.vadr[b] = nv;
    nq += w->body_jnt[b] == FREE ? 7 : 1;
    nv += w->body_jnt[b] == FREE ? 6 : 1;
    if (p < 0) {
      st.tree[b] = (int)st.tree_bodies.size();
      st.tree_bodies.push_back({});
      st.tree_dofs.push_back({});
    } else {
      st.tree[b] = st.tree[p];
    }
    st.tree_bodies[st.tree[b]].push_back(b);
    int nd = w->body_jnt[b] == FREE ? 6 : 1;
    for (int k = 0; k < nd; ++k) st.tree_dofs[st.tree[b]].push_back(st.vadr[b] + k);
  }
  st.nq = nq; st.nv = nv;
  st.dof_tree.assign(nv, 0); st.dof_local.assign(nv, 0);
  for (size_t t = 0; t < st.tree_dofs.size(); ++t)
    for (size_t i = 0; i < st.tree_dofs[t].size(); ++i) {
      st.dof_tree[st.tree_dofs[t][i]] = (int)t;
      st.dof_local[st.tree_dofs[t][i]] = (int)i;
    }
  return true;
}

template <class S> static V3<S> vload(const double* p) { return {S(p[0]), S(p[1]), S(p[2])}; }

/* ------------------------------------------------------------------------------------------
 * 1. forward kinematics
 * ---------------------------------------------------------------------------------------- */
template <class S> struct Pose {
  V3<S> x;     /* body frame origin (joint anchor for hinges) */
  M3<S> R;     /* body frame orientation                      */
  V3<S> com;   /* centre of mass                              */
  V3<S> axis;  /* world hinge axis                            */
};

template <class S>
static void forward_kinematics(const ow_world* w, const Structure& st, const S* q, std::vector<Pose<S>>& P) {
  P.resize(w->nbody);
  for (int b = 0; b < w->nbody; ++b) {
    Pose<S>& o = P[b];
    if (w->body_jnt[b] == FREE) {
      const S* qb = q + st.qadr[b];
      o.x = {qb[0], qb[1], qb[2]};
      o.R = quat_to_mat(qb + 3);
      o.axis = V3<S>();
    } else {
      int p = w->body_parent[b];
      V3<S> xp; M3<S> Rp = M3<S>::eye();
      if (p >= 0) { xp = P[p].x; Rp = P[p].R; }
      S bq[4] = {S(w->body_quat[4 * b]), S(w->body_quat[4 * b + 1]), S(w->body_quat[4 * b + 2]), S(w->body_quat[4 * b + 3])};
      M3<S> Rfix = mul(Rp, quat_to_mat(bq));
      V3<S> ax = vload<S>(w->body_axis + 3 * b);
      ax = S(1.0) / norm(ax) * ax;
      o.R = mul(Rfix, axis_angle(ax, q[st.qadr[b]]));
      o.x = xp + mul(Rp, vload<S>(w->body_pos + 3 * b));
      o.axis = mul(Rfix, ax);
    }
    o.com = o.x + mul(o.R, vload<S>(w->body_ipos + 3 * b));
  }
}

/* Point Jacobian of body b at world point p, as dense rows over all nv DoFs:
 * v_point = Jl v, omega_world = Ja v.  Free joint: v = (world linear velocity of the body
 * origin, body-frame angular velocity).  Hinge: column = (axis x (p - anchor), axis). */
template <class S>
static void point_jacobian(const ow_world* w, const Structure& st, const std::vector<Pose<S>>& P, int b,
                           const V3<S>& p, std::vector<S>* Jl, std::vector<S>* Ja) {
  for (int r = 0; r < 3; ++r) {
    Jl[r].assign(st.nv, S(0.0));
    Ja[r].assign(st.nv, S(0.0));
  }
  for (int a = b; a >= 0; a = w->body_parent[a]) {
    if (w->body_jnt[a] == FREE) {
      int d = st.vadr[a];
      V3<S> rp = p - P[a].x;
      for (int i = 0; i < 3; ++i) {
        Jl[i][d + i] = S(1.0);
        V3<S> c = P[a].R.col(i);
        V3<S> lin = cross(c, rp);
        for (int r = 0; r < 3; ++r) {
          Ja[r][d + 3 + i] = comp(c, r);
          Jl[r][d + 3 + i] = comp(lin, r);
        }
      }
    } else {
      int d = st.vadr[a];
      V3<S> lin = cross(P[a].axis, p - P[a].x);
      for (int r = 0; r < 3; ++r) {
        Jl[r][d] = comp(lin, r);
        Ja[r][d] = comp(P[a].axis, r);
      }
    }
  }
}

/* ------------------------------------------------------------------------------------------
 * 2. joint-space inertia and bias forces
 * ---------------------------------------------------------------------------------------- */
/* M = sum_b Jl(b, com_b)^T m_b Jl(b, com_b) + Ja(b)^T I_b,world Ja(b)   (kinetic energy
 * 1/2 v^T M v).  Bodies of different trees share no DoFs, so M is block diagonal by tree;
 * block t is returned as a dense n_t x n_t matrix over the tree's DoF list. */
template <class S>
static void mass_matrix(const ow_world* w, const Structure& st, const std::vector<Pose<S>>& P,
                        std::vector<std::vector<S>>& Mt) {
  size_t ntree = st.tree_bodies.size();
  Mt.assign(ntree, {});
  std::vector<S> Jl[3], Ja[3];
  for (size_t t = 0; t < ntree; ++t) {
    const std::vector<int>& D = st.tree_dofs[t];
    int n = (int)D.size();
    Mt[t].assign((size_t)n * n, S(0.0));
    for (int b : st.tree_bodies[t]) {
      point_jacobian(w, st, P, b, P[b].com, Jl, Ja);
      S m(w->body_mass[b]);
      /* world inertia R diag(I) R^T */
      M3<S> Iw;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          S s(0.0);
          for (int k = 0; k < 3; ++k) s += P[b].R.m[3 * i + k] * S(w->body_inertia[3 * b + k]) * P[b].R.m[3 * j + k];
          Iw.m[3 * i + j] = s;
        }
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          int di = D[i], dj = D[j];
          S s(0.0);
          for (int r = 0; r < 3; ++r) s += m * Jl[r][di] * Jl[r][dj];
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) s += Ja[r][di] * Iw.m[3 * r + c] * Ja[c][dj];
          Mt[t][(size_t)i * n + j] += s;
        }
    }
  }
}

/* Bias forces c(q, v) (Coriolis, centrifugal, gravity), recursive Newton-Euler with zero joint
 * acceleration and the world accelerating at -g.  Free body (Euler's equations in the body
 * frame with the origin at the centre of mass): c = (-m g, w x I w). */
template <class S>
static void bias_forces(const ow_world* w, const Structure& st, const std::vector<Pose<S>>& P, const S* v,
                        const double* grav, std::vector<S>& c) {
  c.assign(st.nv, S(0.0));
  V3<S> g = vload<S>(grav);
  int nb = w->nbody;
  std::vector<V3<S>> om(nb), omd(nb), acom(nb), F(nb), N(nb);
  for (int b = 0; b < nb; ++b) {
    S m(w->body_mass[b]);
    V3<S> I = vload<S>(w->body_inertia + 3 * b);
    if (w->body_jnt[b] == FREE) {
      int d = st.vadr[b];
      V3<S> wb = {v[d + 3], v[d + 4], v[d + 5]};
      V3<S> Iw = {I.x * wb.x, I.y * wb.y, I.z * wb.z};
      V3<S> gyro = cross(wb, Iw);
      for (int i = 0; i < 3; ++i) c[d + i] = -m * comp(g, i);
      c[d + 3] = gyro.x; c[d + 4] = gyro.y; c[d + 5] = gyro.z;
      continue;
    }
    int p = w->body_parent[b];
    V3<S> omp, omdp, ap, comp_p;
    if (p >= 0) { omp = om[p]; omdp = omd[p]; ap = acom[p]; comp_p = P[p].com; }
    else { ap = -g; }
    S qd = v[st.vadr[b]];
    om[b] = omp + qd * P[b].axis;
    omd[b] = omdp + cross(omp, qd * P[b].axis);
    V3<S> ro = P[b].x - comp_p;
    V3<S> aanchor = p >= 0 ? ap + cross(omdp, ro) + cross(omp, cross(omp, ro)) : ap;
    V3<S> rc = P[b].com - P[b].x;
    acom[b] = aanchor + cross(omd[b], rc) + cross(om[b], cross(om[b], rc));
    /* world inertia times vector: R diag(I) R^T u */
    auto Iw = [&](const V3<S>& u) {
      V3<S> ul = mulT(P[b].R, u);
      V3<S> t = {I.x * ul.x, I.y * ul.y, I.z * ul.z};
      return mul(P[b].R, t);
    };
    F[b] = m * acom[b];
    N[b] = Iw(omd[b]) + cross(om[b], Iw(om[b]));
  }
  /* backward pass: total force and moment about the world origin of each subtree */
  std::vector<V3<S>> ft(nb), nt(nb);
  for (int b = nb - 1; b >= 0; --b) {
    if (w->body_jnt[b] == FREE) continue;
    ft[b] = ft[b] + F[b];
    nt[b] = nt[b] + N[b] + cross(P[b].com, F[b]);
    c[st.vadr[b]] = dot(P[b].axis, nt[b] - cross(P[b].x, ft[b]));
    int p = w->body_parent[b];
    if (p >= 0) { ft[p] = ft[p] + ft[b]; nt[p] = nt[p] + nt[b]; }
  }
}

/* Cholesky factor of a dense SPD block (lower triangle, row major); false if not SPD. */
template <class S> static bool cholesky(std::vector<S>& A, int n) {
  for (int j = 0; j < n; ++j) {
    S s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(val(s) > 0.0)) return false;
    S d = sqrt(s);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      S t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = t / d;
    }
    for (int i = 0; i < j; ++i) A[(size_t)i * n + j] = S(0.0);
  }
  return true;
}
template <class S> static void chol_solve(const std::vector<S>& L, int n, S* x) {
  for (int i = 0; i < n; ++i) {
    S s = x[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * x[k];
    x[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    S s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];
    x[i] = s / L[(size_t)i * n + i];
  }
}

/* Solve M~ x = b in place for a dense nv vector using the per-tree factors. */
template <class S>
static void solve_all(const Structure& st, const std::vector<std::vector<S>>& L, std::vector<S>& x) {
  std::vector<S> tmp;
  for (size_t t = 0; t < st.tree_dofs.size(); ++t) {
    const std::vector<int>& D = st.tree_dofs[t];
    int n = (int)D.size();
    tmp.resize(n);
    for (int i = 0; i < n; ++i) tmp[i] = x[D[i]];
    chol_solve(L[t], n, tmp.data());
    for (int i = 0; i < n; ++i) x[D[i]] = tmp[i];
  }
}

/* ------------------------------------------------------------------------------------------
 * 4. narrowphase
 * Contact normal n points from geom B to geom A; phi is the signed distance (negative =
 * penetration); the contact point is the midpoint of the two surface points.
 * ---------------------------------------------------------------------------------------- */
template <class S> struct GeomPose { V3<S> c; M3<S> R; };
template <class S> struct RawContact { S phi; V3<S> p, n; int sub = 0; };

template <class S>
static void sphere_sphere(const V3<S>& ca, S ra, const V3<S>& cb, S rb, std::vector<RawContact<S>>& out) {
  V3<S> d = ca - cb;
  S dist = norm(d);
  V3<S> n = dist > S(0.0) ? (S(1.0) / dist) * d : V3<S>(S(0.0), S(0.0), S(1.0));
  RawContact<S> k;
  k.phi = dist - ra - rb;
  V3<S> sa = ca - ra * n, sb = cb + rb * n;
  k.p = S(0.5) * (sa + sb);
  k.n = n;
  out.push_back(k);
}

/* sphere (centre c, radius r) against a plane through o with unit normal nz */
template <class S>
static void sphere_plane(const V3<S>& c, S r, const V3<S>& o, const V3<S>& nz, std::vector<RawContact<S>>& out) {
  S dist = dot(nz, c - o);
  RawContact<S> k;
  k.phi = dist - r;
  V3<S> sa = c - r * nz, sb = c - dist * nz;
  k.p = S(0.5) * (sa + sb);
  k.n = nz;
  out.push_back(k);
}

/* closest points of segments [p1,q1], [p2,q2]; near-parallel segments (1 - cos^2 < 1e-3)
 * take the midpoint of the overlap of segment 2's projection onto segment 1. */
template <class S>
static void segment_segment(const V3<S>& p1, const V3<S>& q1, const V3<S>& p2, const V3<S>& q2, S& s, S& t) {
  V3<S> d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
  S a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r), c = dot(d1, r), b = dot(d1, d2);
  S denom = a * e - b * b;
  S zero(0.0), one(1.0);
  if (val(denom) > 1e-3 * val(a * e)) {
    s = clampv((b * f - c * e) / denom, zero, one);
  } else {
    S sp = dot(p2 - p1, d1) / a, sq = dot(q2 - p1, d1) / a;
    S lo = smax(zero, smin(sp, sq)), hi = smin(one, smax(sp, sq));
    if (lo <= hi) s = S(0.5) * (lo + hi);
    else s = smax(sp, sq) < zero ? zero : one;
    t = clampv((b * s + f) / e, zero, one);
    return;
  }
  t = (b * s + f) / e;
  if (t < zero) { t = zero; s = clampv(-c / a, zero, one); }
  else if (t > one) { t = one; s = clampv((b - c) / a, zero, one); }
}

/* sphere (centre c, radius r) against a box (centre bc, rotation R, half extents hs).
 * `sphere_is_a` selects the normal orientation (n from B to A). */
template <class S>
static void sphere_box(const V3<S>& c, S r, const V3<S>& bc, const M3<S>& R, const V3<S>& hs, bool sphere_is_a,
                       std::vector<RawContact<S>>& out) {
  V3<S> l = mulT(R, c - bc);
  S lc[3] = {l.x, l.y, l.z}, h[3] = {hs.x, hs.y, hs.z};
  bool inside = true;
  S cl[3];
  for (int i = 0; i < 3; ++i) {
    cl[i] = clampv(lc[i], -h[i], h[i]);
    if (lc[i] < -h[i] || lc[i] > h[i]) inside = false;
  }
  V3<S> nb;      /* normal pointing from the box toward the sphere */
  S dist;        /* signed distance of the centre to the box surface */
  V3<S> sbox;    /* closest surface point of the box */
  if (!inside) {
    V3<S> q = bc + mul(R, V3<S>(cl[0], cl[1], cl[2]));
    V3<S> d = c - q;
    dist = norm(d);
    nb = (S(1.0) / dist) * d;
    sbox = q;
  } else {
    int k = 0;
    S best = h[0] - fabs(lc[0]);
    for (int i = 1; i < 3; ++i) {
      S gap = h[i] - fabs(lc[i]);
      if (gap < best) { best = gap; k = i; }
    }
    S sg = lc[k] >= S(0.0) ? S(1.0) : S(-1.0);
    nb = sg * R.col(k);
    dist = -best;
    S sl[3] = {lc[0], lc[1], lc[2]};
    sl[k] = sg * h[k];
    sbox = bc + mul(R, V3<S>(sl[0], sl[1], sl[2]));
  }
  RawContact<S> k;
  k.phi = dist - r;
  V3<S> ssph = c - r * nb;
  k.p = S(0.5) * (ssph + sbox);
  k.n = sphere_is_a ? nb : -nb;
  out.push_back(k);
}

/* Box-box contacts (the paper delegates collision detection to MJWarp and names no method;
 * this is the reading taken here): the separating-axis test over the six face axes (A's three,
 * then B's) picks the axis of least overlap, whose box is the reference and whose face toward
 * the other (incident) box is the reference face.  The incident box's face most anti-parallel
 * to it is clipped by the reference face's four side planes (Sutherland-Hodgman: incident
 * vertices in cyclic order from (+,+) of its two in-face axes, planes in the order +k1, -k1,
 * +k2, -k2 with k1, k2 the reference face's in-plane axes after the normal axis); each clipped
 * vertex (at most 8, subs in polygon order) gives a contact with gap = its signed distance to
 * the reference plane, point = its midpoint with its projection, normal = the reference face
 * normal oriented from B to A.  Edge-edge contacts of crossed edges are not generated. */
template <class S>
static void box_box(const V3<S>& ca, const M3<S>& Ra, const V3<S>& ha, const V3<S>& cb, const M3<S>& Rb,
                    const V3<S>& hb, std::vector<RawContact<S>>& out) {
  const V3<S> d = cb - ca;
  const S hav[3] = {ha.x, ha.y, ha.z}, hbv[3] = {hb.x, hb.y, hb.z};
  int best = 0;
  S best_sep(0.0);
  for (int k = 0; k < 6; ++k) {
    const V3<S> u = k < 3 ? Ra.col(k) : Rb.col(k - 3);
    S ra(0.0), rb(0.0);
    for (int i = 0; i < 3; ++i) {
      ra += hav[i] * fabs(dot(Ra.col(i), u));
      rb += hbv[i] * fabs(dot(Rb.col(i), u));
    }
    const S sep = fabs(dot(d, u)) - ra - rb;
    if (k == 0 || sep > best_sep) { best_sep = sep; best = k; }
  }
  const bool refA = best < 3;
  const int jr = best % 3;
  const V3<S> cR = refA ? ca : cb, cI = refA ? cb : ca;
  const M3<S>& RR = refA ? Ra : Rb;
  const M3<S>& RI = refA ? Rb : Ra;
  const S* hR = refA ? hav : hbv;
  const S* hI = refA ? hbv : hav;
  const V3<S> nR = (dot(cI - cR, RR.col(jr)) >= S(0.0) ? S(1.0) : S(-1.0)) * RR.col(jr);
  int ji = 0;
  S most(0.0);
  for (int i = 0; i < 3; ++i) {
    const S c = fabs(dot(RI.col(i), nR));
    if (i == 0 || c > most) { most = c; ji = i; }
  }
  const S si = dot(RI.col(ji), nR) > S(0.0) ? S(-1.0) : S(1.0);  /* incident face faces the reference */
  const int i1 = (ji + 1) % 3, i2 = (ji + 2) % 3;
  const V3<S> fc = cI + (si * hI[ji]) * RI.col(ji);
  const V3<S> e1 = hI[i1] * RI.col(i1), e2 = hI[i2] * RI.col(i2);
  std::vector<V3<S>> poly = {fc + e1 + e2, fc - e1 + e2, fc - e1 - e2, fc + e1 - e2};
  const int k1 = (jr + 1) % 3, k2 = (jr + 2) % 3;
  const int axes[4] = {k1, k1, k2, k2};
  const S sg[4] = {S(1.0), S(-1.0), S(1.0), S(-1.0)};
  for (int pl = 0; pl < 4 && !poly.empty(); ++pl) {
    const V3<S> u = sg[pl] * RR.col(axes[pl]);
    const S h = hR[axes[pl]];
    std::vector<V3<S>> next;
    for (size_t v = 0; v < poly.size(); ++v) {
      const V3<S>& P = poly[v];
      const V3<S>& Q = poly[(v + 1) % poly.size()];
      const S dP = dot(P - cR, u) - h, dQ = dot(Q - cR, u) - h;
      if (dP <= S(0.0)) next.push_back(P);
      if ((dP <= S(0.0)) != (dQ <= S(0.0))) next.push_back(P + (dP / (dP - dQ)) * (Q - P));
    }
    poly.swap(next);
  }
  for (size_t v = 0; v < poly.size(); ++v) {
    RawContact<S> k;
    const S dist = dot(poly[v] - cR, nR) - hR[jr];
    k.phi = dist;
    k.p = poly[v] - (S(0.5) * dist) * nR;
    k.n = refA ? -nR : nR;
    out.push_back(k);
  }
}

/* Ellipsoid (centre c, rotation R, semi-axes e along the body axes) against a plane (point o,
 * unit normal n); the paper names no method, and the reading taken is the support point against n,
 * p = c - R D^2 R^T n / |D R^T n| with D = diag(e), is the lowest point; gap = its height. */
template <class S>
static void ellipsoid_plane(const V3<S>& c, const M3<S>& R, const V3<S>& e, const V3<S>& o, const V3<S>& n,
                            std::vector<RawContact<S>>& out) {
  const V3<S> nl = mulT(R, n);
  const V3<S> dn(e.x * nl.x, e.y * nl.y, e.z * nl.z);
  const S len = norm(dn);
  const V3<S> pl(e.x * dn.x / len, e.y * dn.y / len, e.z * dn.z / len);
  const V3<S> p = c - mul(R, pl);
  RawContact<S> k;
  const S dist = dot(n, p - o);
  k.phi = dist;
  k.p = p - (S(0.5) * dist) * n;
  k.n = n;
  out.push_back(k);
}

/* Cylinder (centre c, rotation R, radius r, half length h along the body z axis) against a
 * plane; the paper names no method, and in the reading taken each end cap contributes three rim points 120 degrees apart, starting from
 * the rim's lowest direction w = -(n - (n.u) u)/|.| (the body x axis when the cap is parallel
 * to the plane): a tilted cylinder touches with its lowest rim point, a lying one along a line,
 * a standing one on a tripod.  Subs 3 cap + k (cap 0 at -h). */
template <class S>
static void cylinder_plane(const V3<S>& c, const M3<S>& R, S r, S h, const V3<S>& o, const V3<S>& n,
                           std::vector<RawContact<S>>& out) {
  const V3<S> u = R.col(2);
  V3<S> w = -(n - dot(n, u) * u);
  const S wl = norm(w);
  w = wl > S(1e-6) ? (S(1.0) / wl) * w : R.col(0);
  const V3<S> w2 = cross(u, w);
  for (int cap = 0; cap < 2; ++cap) {
    const V3<S> ce = c + (cap ? h : -h) * u;
    for (int k = 0; k < 3; ++k) {
      const double th = 2.0 * M_PI * k / 3.0;
      const V3<S> p = ce + (r * S(std::cos(th))) * w + (r * S(std::sin(th))) * w2;
      RawContact<S> kc;
      const S dist = dot(n, p - o);
      kc.phi = dist;
      kc.p = p - (S(0.5) * dist) * n;
      kc.n = n;
      out.push_back(kc);
    }
  }
}

/* Sphere (centre s, radius rs) against a solid cylinder (centre c, axis u, radius r, half
 * length h); the paper names no method, and the reading taken is: with t = u.(s - c) and the radial offset d = (s - c) - t u, a centre
 * outside the cylinder is pushed from the closest point c + clamp(t) u + min(|d|, r) d/|d|; a
 * centre inside leaves through the nearer of the side (depth r - |d|) and the cap (depth
 * h - |t|).  The normal points from the cylinder toward the sphere. */
template <class S>
static void sphere_cylinder(const V3<S>& sc, S rs, const V3<S>& c, const M3<S>& R, S r, S h, bool sphere_is_a,
                            std::vector<RawContact<S>>& out) {
  const V3<S> u = R.col(2);
  const V3<S> rel = sc - c;
  const S t = dot(u, rel);
  const V3<S> d = rel - t * u;
  const S rho = norm(d);
  const V3<S> dr = rho > S(1e-12) ? (S(1.0) / rho) * d : R.col(0);
  V3<S> nb, q;
  S dist;
  if (fabs(t) <= h && rho <= r) {
    const S side = r - rho, cap = h - fabs(t);
    if (side <= cap) {
      nb = dr;
      dist = -side;
      q = c + t * u + r * dr;
    } else {
      const S sg = t >= S(0.0) ? S(1.0) : S(-1.0);
      nb = sg * u;
      dist = -cap;
      q = c + (sg * h) * u + d;
    }
  } else {
    const S tc = clampv(t, -h, h);
    const S rc = rho < r ? rho : r;
    q = c + tc * u + rc * dr;
    const V3<S> g = sc - q;
    dist = norm(g);
    nb = (S(1.0) / dist) * g;
  }
  RawContact<S> k;
  k.phi = dist - rs;
  k.p = S(0.5) * ((sc - rs * nb) + q);
  k.n = sphere_is_a ? nb : -nb;
  out.push_back(k);
}

/* Box signed distance along the capsule axis: f(t) = sdf_box(x0 + t w), t in [-h, h], in box
 * coordinates.  f is convex; t* = argmin f.  If the axis stays outside the box, f^2 is the
 * C1 piecewise quadratic sum_k max(|x_k(t)| - s_k, 0)^2, and t* is the root of its
 * nondecreasing, piecewise linear derivative: found exactly by walking the <= 6 slab
 * breakpoints (a flat stretch takes its midpoint).  If the axis enters the box, f is the
 * maximum of the six linear functions +-x_k(t) - s_k and t* is the best of the endpoints and
 * the pairwise crossings of those lines. */
template <class S>
static S capsule_box_param(const V3<S>& x0v, const V3<S>& wv, S h, const V3<S>& sv) {
  S x0[3] = {x0v.x, x0v.y, x0v.z}, w[3] = {wv.x, wv.y, wv.z}, s[3] = {sv.x, sv.y, sv.z};
  auto sdf = [&](S t) {
    S out2(0.0), inmax(-1e300);
    bool outside = false;
    for (int k = 0; k < 3; ++k) {
      S e = fabs(x0[k] + t * w[k]) - s[k];
      if (e > S(0.0)) { outside = true; out2 += e * e; }
      inmax = smax(inmax, e);
    }
    return outside ? sqrt(out2) : inmax;
  };
  /* does the segment touch the box?  (clip against the three slabs) */
  S lo = -h, hi = h;
  bool hits = true;
  for (int k = 0; k < 3 && hits; ++k) {
    if (val(w[k]) == 0.0) {
      if (fabs(x0[k]) > s[k]) hits = false;
    } else {
      S ta = (-s[k] - x0[k]) / w[k], tb = (s[k] - x0[k]) / w[k];
      if (ta > tb) std::swap(ta, tb);
      lo = smax(lo, ta); hi = smin(hi, tb);
      if (lo > hi) hits = false;
    }
  }
  if (!hits) {
    /* derivative of G = sum_k max(|x_k| - s_k, 0)^2, up to the factor 2 */
    auto dG = [&](S t) {
      S g(0.0);
      for (int k = 0; k < 3; ++k) {
        S xk = x0[k] + t * w[k];
        S e = fabs(xk) - s[k];
        if (e > S(0.0)) g += e * (xk >= S(0.0) ? w[k] : -w[k]);
      }
      return g;
    };
    if (dG(-h) >= S(0.0)) return -h;
    if (dG(h) <= S(0.0)) return h;
    std::vector<S> bp = {-h, h};
    for (int k = 0; k < 3; ++k)
      if (val(w[k]) != 0.0)
        for (int sg = -1; sg <= 1; sg += 2) {
          S tb = (S(double(sg)) * s[k] - x0[k]) / w[k];
          if (tb > -h && tb < h) bp.push_back(tb);
        }
    std::sort(bp.begin(), bp.end(), [](const S& a, const S& b) { return val(a) < val(b); });
    for (size_t i = 0; i + 1 < bp.size(); ++i) {
      S ta = bp[i], tb = bp[i + 1];
      S ga = dG(ta), gb = dG(tb);
      if (ga <= S(0.0) && gb >= S(0.0)) {
        if (val(ga) == 0.0 && val(gb) == 0.0) return S(0.5) * (ta + tb);
        if (val(ga) == 0.0) return ta;
        if (val(gb) == 0.0) return tb;
        /* linear on the piece: solve with the active set at its midpoint */
        S tm = S(0.5) * (ta + tb), num(0.0), den(0.0);
        for (int k = 0; k < 3; ++k) {
          S xk = x0[k] + tm * w[k];
          if (fabs(xk) - s[k] > S(0.0)) {
            S sg = xk >= S(0.0) ? S(1.0) : S(-1.0);
            num += w[k] * (sg * s[k] - x0[k]);
            den += w[k] * w[k];
          }
        }
        return num / den;
      }
    }
    return S(0.0); /* unreachable for a convex G */
  }
  /* the axis enters the box: f = max of six lines a t + b */
  S la[6], lb[6];
  for (int k = 0; k < 3; ++k) {
    la[2 * k] = w[k];  lb[2 * k] = x0[k] - s[k];
    la[2 * k + 1] = -w[k]; lb[2 * k + 1] = -x0[k] - s[k];
  }
  std::vector<S> cand = {-h, h};
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      S da = la[i] - la[j];
      if (val(fabs(da)) > 1e-12) {
        S tc = (lb[j] - lb[i]) / da;
        if (tc > -h && tc < h) cand.push_back(tc);
      }
    }
  S best = cand[0], fbest = sdf(cand[0]);
  for (size_t i = 1; i < cand.size(); ++i) {
    S fi = sdf(cand[i]);
    if (fi < fbest || (val(fi) == val(fbest) && cand[i] < best)) { fbest = fi; best = cand[i]; }
  }
  return best;
}

/* ------------------------------------------------------------------------------------------
 * 5. contact frame (reading: the paper does not fix it)
 * plane contacts: t1 = the plane's local x axis; otherwise t1 = normalize(e_z x n) when
 * |n_z| < 0.5, else normalize(e_x x n); t2 = n x t1.
 * ---------------------------------------------------------------------------------------- */
template <class S> static void contact_frame(const V3<S>& n, const V3<S>* plane_x, V3<S>& t1, V3<S>& t2) {
  if (plane_x) {
    t1 = *plane_x;
  } else {
    V3<S> a = fabs(n.z) < S(0.5) ? V3<S>(S(0.0), S(0.0), S(1.0)) : V3<S>(S(1.0), S(0.0), S(0.0));
    V3<S> c = cross(a, n);
    t1 = (S(1.0) / norm(c)) * c;
  }
  t2 = cross(n, t1);
}

/* r(|phi|) of Eq. r_scaling with x clamped to [0, 1] (reading: beyond the width the impedance
 * saturates at r_max) */
template <class S> static S solimp_r(S aphi, const double* si) {
  S x = clampv(aphi / S(si[2]), S(0.0), S(1.0));
  S m(si[3]);
  S g = x < m ? m * pow(x / m, si[4]) : S(1.0) - (S(1.0) - m) * pow((S(1.0) - x) / (S(1.0) - m), si[4]);
  return S(si[0]) + (S(si[1]) - S(si[0])) * g;
}

/* ------------------------------------------------------------------------------------------
 * learned impedance (Sec. III-B: K(q) and D(q) may be learned instead of set by the
 * heuristic).  The paper fixes neither the model nor its inputs; the readings here:
 * K = k M_theta / dt, D = d M_theta / dt as in Eq. k_d_setting, with
 *   M_theta = M(phi) exp(clamp(g(x), -IMP_CLAMP, IMP_CLAMP)),
 *   g(x) = b2 + sum_h w2_h tanh(b1_h + sum_i W1_hi x_i)   (IMP_HIDDEN tanh units),
 * theta = [W1 (IMP_HIDDEN x IMP_IN, row-major), b1, w2, b2], and the contact's configuration
 * features
 *   x0 = clamp(phi / solimp width, -1, 1)            (where r(|phi|) of Eq. r_scaling moves)
 *   x1 = clamp(1 - 3 (1/m_A + 1/m_B) / (tr_A + tr_B), -1, 1)
 *        (the share of the point-Jacobian trace that comes from rotation; 1/m of a static
 *        side is 0, tr is the mode-0 trace)
 *   x2 = clamp(w_n / (tr_A + tr_B), 0, 4), w_n = sum over the dynamic sides of
 *        1/m_b + (l_b x n)^T I_b^-1 (l_b x n) with l_b the lever from body b's centre of mass
 *        and I_b its world inertia: the normal row's J M^-1 J^T with every body taken as a
 *        free body (exact for free bodies, a cheap stand-in for links of a tree)
 *   x3 = 1 if side B is static, else 0.
 * g = 0 gives back the heuristic exactly.
 * ---------------------------------------------------------------------------------------- */
enum { IMP_IN = 4, IMP_HIDDEN = 8, IMP_PARAMS = IMP_HIDDEN * IMP_IN + 2 * IMP_HIDDEN + 1 };
static const double IMP_CLAMP = 8.0;

template <class S> static S impnet_g(const double* th, const S* x) {
  const double* W1 = th;
  const double* b1 = th + IMP_HIDDEN * IMP_IN;
  const double* w2 = b1 + IMP_HIDDEN;
  const double b2 = w2[IMP_HIDDEN];
  S g(b2);
  for (int h = 0; h < IMP_HIDDEN; ++h) {
    S a(b1[h]);
    for (int i = 0; i < IMP_IN; ++i) a += S(W1[h * IMP_IN + i]) * x[i];
    g += S(w2[h]) * tanh(a);
  }
  return g;
}

template <class S>
static void impnet_features(S phi, double width, S trace_sum, double im_sum, S w_n, bool b_static, S* x) {
  x[0] = clampv(phi / S(width), S(-1.0), S(1.0));
  x[1] = clampv(S(1.0) - S(3.0 * im_sum) / trace_sum, S(-1.0), S(1.0));
  x[2] = clampv(w_n / trace_sum, S(0.0), S(4.0));
  x[3] = S(b_static ? 1.0 : 0.0);
}

/* 1/m + (l x n)^T I^-1 (l x n) of body b taken as a free body, l = p - its centre of mass */
template <class S>
static S free_normal_inverse_mass(const ow_world* w, const std::vector<Pose<S>>& P, int b, const V3<S>& p,
                                  const V3<S>& n) {
  V3<S> u = mulT(P[b].R, cross(p - P[b].com, n));
  const double* I = w->body_inertia + 3 * b;
  return S(1.0 / w->body_mass[b]) + u.x * u.x / S(I[0]) + u.y * u.y / S(I[1]) + u.z * u.z / S(I[2]);
}

/* ------------------------------------------------------------------------------------------
 * the step
 * ---------------------------------------------------------------------------------------- */
template <class S> struct StepRecord {
  std::vector<S> vs, p, c;
  std::vector<ow_contact> contacts;
  bool detail = false;  /* also the mean exact facet impedance of every contact */
};

template <class S>
static int step_world(const ow_world* w, const ow_params* prm, const Structure& st, double dt, S* q, S* v,
                      const S* tau, StepRecord<S>* rec) {
  S DT(dt);
  /* 1. kinematics */
  std::vector<Pose<S>> P;
  forward_kinematics(w, st, q, P);
  /* 2. inertia, bias, implicit damping, factorisation */
  std::vector<std::vector<S>> L;
  mass_matrix(w, st, P, L);
  std::vector<S> c;
  bias_forces(w, st, P, v, prm->gravity, c);
  std::vector<S> damp(st.nv, S(0.0));
  for (int b = 0; b < w->nbody; ++b)
    if (w->body_jnt[b] == HINGE) damp[st.vadr[b]] = S(w->body_damping[b]);
  for (size_t t = 0; t < L.size(); ++t) {
    int n = (int)st.tree_dofs[t].size();
    for (int i = 0; i < n; ++i) L[t][(size_t)i * n + i] += DT * damp[st.tree_dofs[t][i]];
    if (!cholesky(L[t], n)) return -1;
  }
  /* 3. smooth prediction, Eq. smooth_vel (with implicit damping) */
  std::vector<S> vs(st.nv);
  for (int i = 0; i < st.nv; ++i) vs[i] = (tau ? tau[i] : S(0.0)) - c[i] - damp[i] * v[i];
  solve_all(st, L, vs);
  for (int i = 0; i < st.nv; ++i) vs[i] = v[i] + vs[i] * DT;

  /* 4.-7. contacts, facets, impulses, generalised impulse */
  std::vector<GeomPose<S>> G(w->ngeom);
  for (int g = 0; g < w->ngeom; ++g) {
    S gq[4] = {S(w->geom_quat[4 * g]), S(w->geom_quat[4 * g + 1]), S(w->geom_quat[4 * g + 2]), S(w->geom_quat[4 * g + 3])};
    int b = w->geom_body[g];
    if (b < 0) {
      G[g].c = vload<S>(w->geom_pos + 3 * g);
      G[g].R = quat_to_mat(gq);
    } else {
      G[g].c = P[b].x + mul(P[b].R, vload<S>(w->geom_pos + 3 * g));
      G[g].R = mul(P[b].R, quat_to_mat(gq));
    }
  }
  std::vector<S> pgen(st.nv, S(0.0));
  std::vector<S> JlA[3], JaA[3], JlB[3], JaB[3];
  std::vector<S> tmp(st.nv);
  const double margin = prm->margin;
  for (int gi = 0; gi < w->ngeom; ++gi)
    for (int gj = gi + 1; gj < w->ngeom; ++gj) {
      int bi = w->geom_body[gi], bj = w->geom_body[gj];
      int ti = w->geom_type[gi], tj = w->geom_type[gj];
      if (bi < 0 && bj < 0) continue;
      if (bi == bj) continue;
      if (bi >= 0 && bj >= 0 && (w->body_parent[bi] == bj || w->body_parent[bj] == bi)) continue;
      /* orient the pair: A = non-plane geom, else the lower index */
      int ga = gi, gb = gj;
      if (ti == PLANE) std::swap(ga, gb);
      int ta = w->geom_type[ga], tb = w->geom_type[gb];
      if (ta == PLANE) continue;
      std::vector<RawContact<S>> raw;
      const double* sa = w->geom_size + 3 * ga;
      const double* sb = w->geom_size + 3 * gb;
      V3<S> axa = G[ga].R.col(2), axb = G[gb].R.col(2);
      bool plane_pair = (tb == PLANE);
      if (plane_pair) {
        V3<S> nz = G[gb].R.col(2), o = G[gb].c;
        if (ta == SPHERE) sphere_plane(G[ga].c, S(sa[0]), o, nz, raw);
        else if (ta == CAPSULE) {
          sphere_plane(G[ga].c - S(sa[1]) * axa, S(sa[0]), o, nz, raw);
          sphere_plane(G[ga].c + S(sa[1]) * axa, S(sa[0]), o, nz, raw);
        } else if (ta == ELLIPSOID) {
          ellipsoid_plane(G[ga].c, G[ga].R, vload<S>(sa), o, nz, raw);
        } else if (ta == CYLINDER) {
          cylinder_plane(G[ga].c, G[ga].R, S(sa[0]), S(sa[1]), o, nz, raw);
        } else if (ta == BOX) {
          for (int cx = -1; cx <= 1; cx += 2)
            for (int cy = -1; cy <= 1; cy += 2)
              for (int cz = -1; cz <= 1; cz += 2) {
                V3<S> corner = G[ga].c + mul(G[ga].R, V3<S>(S(cx * sa[0]), S(cy * sa[1]), S(cz * sa[2])));
                sphere_plane(corner, S(0.0), o, nz, raw);
              }
        }
      } else if (ta == SPHERE && tb == SPHERE) {
        sphere_sphere(G[ga].c, S(sa[0]), G[gb].c, S(sb[0]), raw);
      } else if ((ta == SPHERE && tb == CAPSULE) || (ta == CAPSULE && tb == SPHERE)) {
        bool capA = ta == CAPSULE;
        const GeomPose<S>& cg = capA ? G[ga] : G[gb];
        const GeomPose<S>& sg = capA ? G[gb] : G[ga];
        const double* cs = capA ? sa : sb;
        const double* ss = capA ? sb : sa;
        V3<S> u = cg.R.col(2);
        S t = clampv(dot(sg.c - cg.c, u), S(-cs[1]), S(cs[1]));
        V3<S> qn = cg.c + t * u;
        if (capA) sphere_sphere(qn, S(cs[0]), sg.c, S(ss[0]), raw);
        else sphere_sphere(sg.c, S(ss[0]), qn, S(cs[0]), raw);
      } else if (ta == CAPSULE && tb == CAPSULE) {
        V3<S> p1 = G[ga].c - S(sa[1]) * axa, q1 = G[ga].c + S(sa[1]) * axa;
        V3<S> p2 = G[gb].c - S(sb[1]) * axb, q2 = G[gb].c + S(sb[1]) * axb;
        S s(0.0), t(0.0);
        segment_segment(p1, q1, p2, q2, s, t);
        sphere_sphere(p1 + s * (q1 - p1), S(sa[0]), p2 + t * (q2 - p2), S(sb[0]), raw);
      } else if ((ta == SPHERE && tb == BOX) || (ta == BOX && tb == SPHERE)) {
        bool sphA = ta == SPHERE;
        const GeomPose<S>& sg = sphA ? G[ga] : G[gb];
        const GeomPose<S>& bg = sphA ? G[gb] : G[ga];
        const double* ss = sphA ? sa : sb;
        const double* bs = sphA ? sb : sa;
        sphere_box(sg.c, S(ss[0]), bg.c, bg.R, vload<S>(bs), sphA, raw);
      } else if ((ta == CAPSULE && tb == BOX) || (ta == BOX && tb == CAPSULE)) {
        bool capA = ta == CAPSULE;
        const GeomPose<S>& cg = capA ? G[ga] : G[gb];
        const GeomPose<S>& bg = capA ? G[gb] : G[ga];
        const double* cs = capA ? sa : sb;
        const double* bs = capA ? sb : sa;
        V3<S> x0 = mulT(bg.R, cg.c - bg.c), wl = mulT(bg.R, cg.R.col(2));
        S t = capsule_box_param(x0, wl, S(cs[1]), vload<S>(bs));
        sphere_box(cg.c + t * cg.R.col(2), S(cs[0]), bg.c, bg.R, vload<S>(bs), capA, raw);
      } else if ((ta == SPHERE && tb == CYLINDER) || (ta == CYLINDER && tb == SPHERE)) {
        const bool sphA = ta == SPHERE;
        const GeomPose<S>& sg = sphA ? G[ga] : G[gb];
        const GeomPose<S>& cg = sphA ? G[gb] : G[ga];
        const double* ss = sphA ? sa : sb;
        const double* cs = sphA ? sb : sa;
        sphere_cylinder(sg.c, S(ss[0]), cg.c, cg.R, S(cs[0]), S(cs[1]), sphA, raw);
      } else if (ta == BOX && tb == BOX) {
        box_box(G[ga].c, G[ga].R, vload<S>(sa), G[gb].c, G[gb].R, vload<S>(sb), raw);
      } else {
        continue;
      }
      for (size_t ri = 0; ri < raw.size(); ++ri) raw[ri].sub = (int)ri;
      for (RawContact<S>& k : raw) {
        if (!(val(k.phi) < margin)) continue;
        int ba = w->geom_body[ga], bb = w->geom_body[gb];
        /* frame */
        V3<S> t1, t2;
        V3<S> px = G[gb].R.col(0);
        contact_frame(k.n, plane_pair ? &px : nullptr, t1, t2);
        /* relative Jacobian J = J_A(p) - J_B(p): linear and angular rows */
        std::vector<S> Jl[3], Ja[3];
        for (int r = 0; r < 3; ++r) { Jl[r].assign(st.nv, S(0.0)); Ja[r].assign(st.nv, S(0.0)); }
        S trace[2] = {S(0.0), S(0.0)};
        for (int side = 0; side < 2; ++side) {
          int bdy = side == 0 ? ba : bb;
          if (bdy < 0) continue;
          std::vector<S>* jl = side == 0 ? JlA : JlB;
          std::vector<S>* ja = side == 0 ? JaA : JaB;
          point_jacobian(w, st, P, bdy, k.p, jl, ja);
          S sgn(side == 0 ? 1.0 : -1.0);
          for (int r = 0; r < 3; ++r)
            for (int i = 0; i < st.nv; ++i) { Jl[r][i] += sgn * jl[r][i]; Ja[r][i] += sgn * ja[r][i]; }
          /* trace of J_i M~^-1 J_i^T over the translational point Jacobian of body i (also the
             input of the learned impedance's features, and of the heuristic that the exact
             impedance is compared with) */
          if (prm->trace_mode != 1) {
            for (int r = 0; r < 3; ++r) {
              tmp = jl[r];
              solve_all(st, L, tmp);
              for (int i = 0; i < st.nv; ++i) trace[side] += jl[r][i] * tmp[i];
            }
          } else {
            trace[side] = S(1.0) / S(w->body_mass[bdy]);
          }
        }
        /* contact-space rows */
        auto row = [&](std::vector<S>* J, const V3<S>& d, std::vector<S>& out) {
          out.assign(st.nv, S(0.0));
          for (int i = 0; i < st.nv; ++i) out[i] = d.x * J[0][i] + d.y * J[1][i] + d.z * J[2][i];
        };
        std::vector<S> Jn, Jt1, Jt2, Jtor, Jr1, Jr2;
        row(Jl, k.n, Jn); row(Jl, t1, Jt1); row(Jl, t2, Jt2);
        row(Ja, k.n, Jtor); row(Ja, t1, Jr1); row(Ja, t2, Jr2);
        /* impedance: Eq. k_d_setting with M(phi) = r/(1-r) / (tr_i + tr_j), Eq. r_scaling */
        S r = solimp_r(fabs(k.phi), prm->solimp);
        S mphi = r / (S(1.0) - r) / (trace[0] + trace[1]);
        /* the learned impedance's inputs, and (trace_mode 3) its scaling of M(phi) */
        S feat[4];
        {
          double im_sum = (ba >= 0 ? 1.0 / w->body_mass[ba] : 0.0) + (bb >= 0 ? 1.0 / w->body_mass[bb] : 0.0);
          S w_n(0.0);
          if (ba >= 0) w_n += free_normal_inverse_mass(w, P, ba, k.p, k.n);
          if (bb >= 0) w_n += free_normal_inverse_mass(w, P, bb, k.p, k.n);
          impnet_features(k.phi, prm->solimp[2], trace[0] + trace[1], im_sum, w_n, bb < 0, feat);
        }
        if (prm->trace_mode == 3) mphi *= exp(clampv(impnet_g(prm->impnet, feat), S(-IMP_CLAMP), S(IMP_CLAMP)));
        S kM = S(prm->k_user) * mphi, dM = S(prm->d_user) * mphi;
        /* friction coefficients of the pair: the larger of the two geoms' */
        S mu[3];
        for (int i = 0; i < 3; ++i) mu[i] = S(std::max(w->geom_mu[3 * ga + i], w->geom_mu[3 * gb + i]));
        ow_contact rc;
        std::memset(&rc, 0, sizeof(rc));
        S wrench[6] = {S(0.0), S(0.0), S(0.0), S(0.0), S(0.0), S(0.0)};
        S m_exact_sum(0.0);
        int nf = 0, nact = 0;
        /* facets, Eqs. dual_polyhedral, tilde_defs, cf_wrench */
        auto facet = [&](int sub, S ca, S sa_) {
          /* sub 0: tangential (direction ca t1 + sa_ t2), 1: torsional (sign ca), 2: rolling */
          std::vector<S> Jf(st.nv);
          for (int i = 0; i < st.nv; ++i) {
            S dj;
            if (sub == 0) dj = ca * Jt1[i] + sa_ * Jt2[i];
            else if (sub == 1) dj = ca * Jtor[i];
            else dj = ca * Jr1[i] + sa_ * Jr2[i];
            Jf[i] = Jn[i] - mu[sub] * dj;
          }
          S sv(0.0);
          for (int i = 0; i < st.nv; ++i) sv += Jf[i] * vs[i];
          S lam;
          S Mj(0.0);
          if (prm->trace_mode == 2 || (rec && rec->detail)) {
            /* Sec. III-B, the diagonal form K dt + D = 1/(dt w_j), w_j = J~_j M~^-1 J~_j^T; the
               user's (k, d) keep splitting it between the gap and the velocity term:
               M_j = 1 / ((k dt + d) w_j) in place of M(phi) */
            tmp = Jf;
            solve_all(st, L, tmp);
            S wj(0.0);
            for (int i = 0; i < st.nv; ++i) wj += Jf[i] * tmp[i];
            Mj = S(1.0) / ((S(prm->k_user) * DT + S(prm->d_user)) * wj);
            m_exact_sum += Mj;
          }
          if (prm->trace_mode == 2) {
            lam = -S(prm->k_user) * Mj * (sv * DT + k.phi) - S(prm->d_user) * Mj * sv;
          } else {
            lam = -kM * (sv * DT + k.phi) - dM * sv;
          }
          if (lam < S(0.0)) lam = S(0.0);
          else ++nact;
          ++nf;
          for (int i = 0; i < st.nv; ++i) pgen[i] += Jf[i] * lam;
          wrench[0] += lam;
          if (sub == 0) { wrench[1] -= mu[0] * ca * lam; wrench[2] -= mu[0] * sa_ * lam; }
          else if (sub == 1) wrench[3] -= mu[1] * ca * lam;
          else { wrench[4] -= mu[2] * ca * lam; wrench[5] -= mu[2] * sa_ * lam; }
        };
        for (int j = 0; j < prm->n_t; ++j) {
          double th = 2.0 * M_PI * j / prm->n_t;
          facet(0, S(std::cos(th)), S(std::sin(th)));
        }
        for (int j = 0; j < prm->n_tor; ++j) facet(1, S(j % 2 == 0 ? 1.0 : -1.0), S(0.0));
        for (int j = 0; j < prm->n_rol; ++j) {
          double th = 2.0 * M_PI * j / prm->n_rol;
          facet(2, S(std::cos(th)), S(std::sin(th)));
        }
        if (rec) {
          rc.geom_a = ga; rc.geom_b = gb; rc.body_a = ba; rc.body_b = bb; rc.sub = k.sub;
          rc.phi = val(k.phi);
          rc.pos[0] = val(k.p.x); rc.pos[1] = val(k.p.y); rc.pos[2] = val(k.p.z);
          rc.normal[0] = val(k.n.x); rc.normal[1] = val(k.n.y); rc.normal[2] = val(k.n.z);
          rc.t1[0] = val(t1.x); rc.t1[1] = val(t1.y); rc.t1[2] = val(t1.z);
          rc.t2[0] = val(t2.x); rc.t2[1] = val(t2.y); rc.t2[2] = val(t2.z);
          rc.trace_a = val(trace[0]); rc.trace_b = val(trace[1]);
          rc.r = val(r); rc.mphi = prm->trace_mode == 2 ? 0.0 : val(mphi); rc.lam_sum = val(wrench[0]);
          for (int i = 0; i < 6; ++i) rc.wrench[i] = val(wrench[i]);
          rc.nfacet = nf; rc.nactive = nact;
          for (int i = 0; i < 4; ++i) rc.feat[i] = val(feat[i]);
          rc.m_exact = nf ? val(m_exact_sum) / nf : 0.0;
          rec->contacts.push_back(rc);
        }
      }
    }
  /* joint limits and dry joint friction (Sec. III-A names them in the system model; the paper
     gives no formula, so these are readings):
     - a limit is a one-row frictionless constraint J = +e_k (lower, gap q - lo) or -e_k (upper,
       gap hi - q) under the same impulse law as a contact facet, its "trace" (M~^-1)_kk;
     - dry friction applies the impulse that alone would stop the predicted joint velocity,
       clamped to +-frictionloss dt.
     Both act on the smooth prediction and add to p like the contacts. */
  for (int b = 0; b < w->nbody; ++b) {
    if (w->body_jnt[b] != HINGE) continue;
    const double lo = w->body_range ? w->body_range[2 * b] : 0.0;
    const double hi = w->body_range ? w->body_range[2 * b + 1] : 0.0;
    const double fl = w->body_frictionloss ? w->body_frictionloss[b] : 0.0;
    if (!(lo < hi) && !(fl > 0.0)) continue;
    const int kd = st.vadr[b];
    tmp.assign(st.nv, S(0.0));
    tmp[kd] = S(1.0);
    solve_all(st, L, tmp);
    const S wkk = tmp[kd];
    if (lo < hi) {
      for (int side = 0; side < 2; ++side) {
        const S gap = side == 0 ? q[st.qadr[b]] - S(lo) : S(hi) - q[st.qadr[b]];
        if (!(val(gap) < margin)) continue;
        const S sgn(side == 0 ? 1.0 : -1.0);
        const S sv = sgn * vs[kd];
        S Mk;
        if (prm->trace_mode == 2) {
          Mk = S(1.0) / ((S(prm->k_user) * DT + S(prm->d_user)) * wkk);
        } else {
          const S r = solimp_r(fabs(gap), prm->solimp);
          Mk = r / (S(1.0) - r) / wkk;
        }
        S lam = -S(prm->k_user) * Mk * (sv * DT + gap) - S(prm->d_user) * Mk * sv;
        if (lam > S(0.0)) pgen[kd] += sgn * lam;
      }
    }
    if (fl > 0.0) {
      S lam = -vs[kd] / wkk;
      const S cap = S(fl) * DT;
      if (lam > cap) lam = cap;
      if (lam < -cap) lam = -cap;
      pgen[kd] += lam;
    }
  }

  /* 8. velocity correction, Eq. vel_correction */
  std::vector<S> dv = pgen;
  solve_all(st, L, dv);
  for (int i = 0; i < st.nv; ++i) v[i] = vs[i] + dv[i];
  if (rec) { rec->vs = vs; rec->p = pgen; rec->c = c; }

  /* 9. semi-implicit Euler */
  for (int b = 0; b < w->nbody; ++b) {
    if (w->body_jnt[b] == HINGE) {
      q[st.qadr[b]] += v[st.vadr[b]] * DT;
      continue;
    }
    S* qb = q + st.qadr[b];
    const S* vb = v + st.vadr[b];
    for (int i = 0; i < 3; ++i) qb[i] += vb[i] * DT;
    /* body-frame angular velocity: quat <- quat (x) exp(omega dt / 2) */
    V3<S> om = {vb[3], vb[4], vb[5]};
    S wn = norm(om);
    S half = S(0.5) * wn * DT;
    S dq[4];
    if (val(wn) > 0.0) {
      S sc = sin(half) / wn;
      dq[0] = cos(half); dq[1] = sc * om.x; dq[2] = sc * om.y; dq[3] = sc * om.z;
    } else {
      dq[0] = S(1.0); dq[1] = dq[2] = dq[3] = S(0.0);
    }
    S nq[4];
    quat_mul(qb + 3, dq, nq);
    S nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    for (int i = 0; i < 4; ++i) qb[3 + i] = nq[i] / nn;
  }
  return 0;
}

}  // namespace orc

using namespace orc;

/* ------------------------------------------------------------------------------------------
 * C entry points
 * ---------------------------------------------------------------------------------------- */
extern "C" {

int ow_sizes(const ow_world* w, int* nq, int* nv) {
  Structure st;
  if (!build_structure(w, st)) return -1;
  *nq = st.nq; *nv = st.nv;
  return 0;
}

/* Advance one world nsteps.  q[nq], v[nv] in/out; tau [nsteps][nv] or NULL; returns 0 or -1. */
int ow_step(const ow_world* w, const ow_params* prm, double dt, int nsteps, double* q, double* v,
            const double* tau, int* ncontact_total) {
  Structure st;
  if (!build_structure(w, st)) return -1;
  long nc = 0;
  for (int s = 0; s < nsteps; ++s) {
    StepRecord<double> rec;
    int rc = step_world<double>(w, prm, st, dt, q, v, tau ? tau + (size_t)s * st.nv : nullptr,
                                ncontact_total ? &rec : nullptr);
    if (rc) return rc;
    nc += (long)rec.contacts.size();
  }
  if (ncontact_total) *ncontact_total = (int)nc;
  return 0;
}

/* Many worlds in parallel (OpenMP over worlds), each advanced nsteps.  q/v are concatenated
 * per world at qadr/vadr.  Returns the number of failing worlds. */
int ow_step_batch(int nworld, const ow_world* const* worlds, const ow_params* prm, double dt, int nsteps,
                  double* q, const long* qadr, double* v, const long* vadr, long* contacts, int nthreads) {
  int fails = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : fails)
#endif
  for (int i = 0; i < nworld; ++i) {
    int nc = 0;
    int rc = ow_step(worlds[i], prm, dt, nsteps, q + qadr[i], v + vadr[i], nullptr, contacts ? &nc : nullptr);
    if (contacts) contacts[i] = nc;
    if (rc) ++fails;
  }
  return fails;
}

int ow_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* One step with a record of its intermediates: vs[nv], p[nv], c[nv], and up to cap contacts. */
int ow_step_record(const ow_world* w, const ow_params* prm, double dt, double* q, double* v, const double* tau,
                   double* vs, double* p, double* c, ow_contact* contacts, int cap, int* ncontact) {
  Structure st;
  if (!build_structure(w, st)) return -1;
  StepRecord<double> rec;
  rec.detail = true;
  int rc = step_world<double>(w, prm, st, dt, q, v, tau, &rec);
  if (rc) return rc;
  for (int i = 0; i < st.nv; ++i) {
    if (vs) vs[i] = rec.vs[i];
    if (p) p[i] = rec.p[i];
    if (c) c[i] = rec.c[i];
  }
  *ncontact = (int)rec.contacts.size();
  for (int i = 0; i < (int)rec.contacts.size() && i < cap; ++i) contacts[i] = rec.contacts[i];
  return 0;
}

/* Dense joint-space inertia (nv x nv, zeros off the tree blocks), bias c, body poses
 * (x[3], R[9], com[3] per body) at state (q, v). */
int ow_dynamics(const ow_world* w, const double* gravity, const double* q, const double* v, double* M, double* c,
                double* poses) {
  Structure st;
  if (!build_structure(w, st)) return -1;
  std::vector<Pose<double>> P;
  forward_kinematics(w, st, q, P);
  std::vector<std::vector<double>> Mt;
  mass_matrix(w, st, P, Mt);
  if (M) {
    std::memset(M, 0, sizeof(double) * st.nv * st.nv);
    for (size_t t = 0; t < Mt.size(); ++t) {
      const std::vector<int>& D = st.tree_dofs[t];
      int n = (int)D.size();
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) M[(size_t)D[i] * st.nv + D[j]] = Mt[t][(size_t)i * n + j];
    }
  }
  if (c) {
    std::vector<double> cc;
    bias_forces(w, st, P, v, gravity, cc);
    for (int i = 0; i < st.nv; ++i) c[i] = cc[i];
  }
  if (poses)
    for (int b = 0; b < w->nbody; ++b) {
      double* o = poses + 15 * b;
      o[0] = P[b].x.x; o[1] = P[b].x.y; o[2] = P[b].x.z;
      for (int i = 0; i < 9; ++i) o[3 + i] = P[b].R.m[i];
      o[12] = P[b].com.x; o[13] = P[b].com.y; o[14] = P[b].com.z;
    }
  return 0;
}

/* Cholesky factor of a dense SPD matrix (tests the oracle's factorisation routine). */
int ow_cholesky(double* A, int n) {
  std::vector<double> a(A, A + (size_t)n * n);
  if (!cholesky(a, n)) return -1;
  std::memcpy(A, a.data(), sizeof(double) * n * n);
  return 0;
}

/* Capsule-box closest-axis parameter (tests the narrowphase minimiser). */
double ow_capsule_box_param(const double* x0, const double* w, double h, const double* half) {
  return capsule_box_param(V3<double>(x0[0], x0[1], x0[2]), V3<double>(w[0], w[1], w[2]), h,
                           V3<double>(half[0], half[1], half[2]));
}

double ow_solimp_r(double aphi, const double* solimp) { return solimp_r(aphi, solimp); }

int ow_impnet_params(void) { return IMP_PARAMS; }

/* The learned impedance network at n inputs x[n][IMP_IN]: out[n] = g(x) (unclamped). */
void ow_impnet_eval(const double* theta, const double* x, int n, double* out) {
  for (int i = 0; i < n; ++i) out[i] = impnet_g(theta, x + (size_t)i * IMP_IN);
}

/* Mean squared error of the network on (x[n][IMP_IN], y[n]), L = (1/n) sum_i (g(x_i) - y_i)^2,
 * and its gradient by the chain rule through g: grad[IMP_PARAMS]. */
double ow_impnet_loss_grad(const double* theta, const double* x, const double* y, int n, double* grad) {
  const double* W1 = theta;
  const double* b1 = theta + IMP_HIDDEN * IMP_IN;
  const double* w2 = b1 + IMP_HIDDEN;
  for (int p = 0; p < IMP_PARAMS; ++p) grad[p] = 0.0;
  double loss = 0.0;
  for (int i = 0; i < n; ++i) {
    const double* xi = x + (size_t)i * IMP_IN;
    double hid[IMP_HIDDEN];
    double g = w2[IMP_HIDDEN];
    for (int h = 0; h < IMP_HIDDEN; ++h) {
      double a = b1[h];
      for (int k = 0; k < IMP_IN; ++k) a += W1[h * IMP_IN + k] * xi[k];
      hid[h] = std::tanh(a);
      g += w2[h] * hid[h];
    }
    const double e = g - y[i];
    loss += e * e;
    const double dg = 2.0 * e / n;                      /* dL/dg_i */
    grad[IMP_PARAMS - 1] += dg;                         /* b2 */
    for (int h = 0; h < IMP_HIDDEN; ++h) {
      grad[IMP_HIDDEN * IMP_IN + IMP_HIDDEN + h] += dg * hid[h];        /* w2_h */
      const double da = dg * w2[h] * (1.0 - hid[h] * hid[h]);         /* through tanh */
      grad[IMP_HIDDEN * IMP_IN + h] += da;                             /* b1_h */
      for (int k = 0; k < IMP_IN; ++k) grad[h * IMP_IN + k] += da * xi[k];  /* W1_hk */
    }
  }
  return loss / n;
}

/* The MPC costs of one state (Sec. V, Eq. mpc and its running and terminal cost terms).
 * The object is the free body `cost_body`; goal[7] = its target position and quaternion (wxyz);
 * qref[nq] = the home pose, of which only hinge coordinates count; wts[8] = w_quat, w_pos,
 * w_contact, w_joint, w_fallen (the paper's Omega), fall_radius, term_pos (phi_1), term_quat
 * (phi_2).  Running cost:
 *   w_quat (1 - (q*^T q)^2) + w_pos (|p_x - p*_x| + |p_y - p*_y| + |p_z - p*_z|)
 *   + w_contact sum_tips |p - tip|^2 + w_joint sum_hinges (q_k - qref_k)^2 + w_fallen [fallen],
 * where a fingertip is the far end (centre + half length along the geom's z axis) of every
 * capsule carried by a hinge body that has no child body, and "fallen" means the object's
 * horizontal distance from the target exceeds fall_radius (the synthetic palm is the floor, so
 * the paper's height test cannot tell a dropped object).  Terminal cost:
 *   term_pos |p - p*|^2 + term_quat (1 - (q*^T q)^2). */
int ow_mpc_cost(const ow_world* w, int cost_body, const double* q, const double* goal, const double* qref,
                const double* wts, double* running, double* terminal) {
  Structure st;
  if (!build_structure(w, st)) return -1;
  if (cost_body < 0 || cost_body >= w->nbody || w->body_jnt[cost_body] != FREE) return -1;
  std::vector<Pose<double>> P;
  forward_kinematics(w, st, q, P);
  const double* qo = q + st.qadr[cost_body];
  const double align = goal[3] * qo[3] + goal[4] * qo[4] + goal[5] * qo[5] + goal[6] * qo[6];
  const double c_quat = 1.0 - align * align;
  double c = wts[0] * c_quat;
  c += wts[1] * (std::fabs(qo[0] - goal[0]) + std::fabs(qo[1] - goal[1]) + std::fabs(qo[2] - goal[2]));
  double tips = 0.0;
  for (int g = 0; g < w->ngeom; ++g) {
    const int b = w->geom_body[g];
    if (b < 0 || w->geom_type[g] != CAPSULE || w->body_jnt[b] != HINGE) continue;
    bool leaf = true;
    for (int k = 0; k < w->nbody; ++k)
      if (w->body_parent[k] == b) leaf = false;
    if (!leaf) continue;
    const double gq[4] = {w->geom_quat[4 * g], w->geom_quat[4 * g + 1], w->geom_quat[4 * g + 2], w->geom_quat[4 * g + 3]};
    const M3<double> Rg = mul(P[b].R, quat_to_mat(gq));
    const V3<double> centre = P[b].x + mul(P[b].R, vload<double>(w->geom_pos + 3 * g));
    const V3<double> tip = centre + w->geom_size[3 * g + 1] * Rg.col(2);
    const V3<double> d = V3<double>(qo[0], qo[1], qo[2]) - tip;
    tips += dot(d, d);
  }
  c += wts[2] * tips;
  double cj = 0.0;
  for (int b = 0; b < w->nbody; ++b)
    if (w->body_jnt[b] == HINGE) {
      const double e = q[st.qadr[b]] - qref[st.qadr[b]];
      cj += e * e;
    }
  c += wts[3] * cj;
  if (std::hypot(qo[0] - goal[0], qo[1] - goal[1]) > wts[5]) c += wts[4];
  *running = c;
  const double dx = qo[0] - goal[0], dy = qo[1] - goal[1], dz = qo[2] - goal[2];
  *terminal = wts[6] * (dx * dx + dy * dy + dz * dz) + wts[7] * c_quat;
  return 0;
}

/* Rollout loss of body `body` after T steps, L = |x_T - x*|^2 + (1 - (quat*^T quat_T)^2), and
 * its directional derivative along (dq0, dv0, dtau) by forward-mode dual numbers.
 * tau and dtau are [T][nv]. */
int ow_rollout_loss_dir(const ow_world* w, const ow_params* prm, double dt, int T, const double* q0,
                        const double* v0, const double* tau, const double* dq0, const double* dv0,
                        const double* dtau, int body, const double* target_pos, const double* target_quat,
                        double* loss, double* dloss) {
  Structure st;
  if (!build_structure(w, st)) return -1;
  if (w->body_jnt[body] != FREE) return -1;
  std::vector<Dual> q(st.nq), v(st.nv), u(st.nv);
  for (int i = 0; i < st.nq; ++i) q[i] = Dual(q0[i], dq0 ? dq0[i] : 0.0);
  for (int i = 0; i < st.nv; ++i) v[i] = Dual(v0[i], dv0 ? dv0[i] : 0.0);
  for (int s = 0; s < T; ++s) {
    for (int i = 0; i < st.nv; ++i)
      u[i] = Dual(tau ? tau[(size_t)s * st.nv + i] : 0.0, dtau ? dtau[(size_t)s * st.nv + i] : 0.0);
    if (step_world<Dual>(w, prm, st, dt, q.data(), v.data(), u.data(), nullptr)) return -1;
  }
  const Dual* qb = q.data() + st.qadr[body];
  Dual L(0.0);
  for (int i = 0; i < 3; ++i) { Dual e = qb[i] - Dual(target_pos[i]); L += e * e; }
  Dual dq(0.0);
  for (int i = 0; i < 4; ++i) dq += Dual(target_quat[i]) * qb[3 + i];
  L += Dual(1.0) - dq * dq;
  *loss = L.v;
  *dloss = L.d;
  return 0;
}

}  /* extern "C" */
