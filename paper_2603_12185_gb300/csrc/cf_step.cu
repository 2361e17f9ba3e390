// The fused ComFree step: one group of warps per world, the world's state staged in shared
// memory for the whole step (or nsteps steps), persistent CTAs pulling work units.
//
// Per world and step (ComFree-Sim, Sec. III and Algorithm 1):
//   A. smooth prediction v_s = v + M~^-1 (tau - c - b v) dt            (Eq. smooth_vel; Kernel I)
//   B. pair loop: bounding-sphere broadphase compacted into per-warp queues, narrowphase,
//      contact frame, M(phi), per-facet closed-form impulses and the scatter of J~^T lambda
//      (articulated worlds) or of M^-1 J~^T lambda (free bodies) into fixed-point shared
//      accumulators                                    (Eqs. tilde_defs, cf_wrench; Kernels II-III)
//   C. v+ = v_s + M~^-1 p, semi-implicit Euler                      (Eq. vel_correction; Kernel IV)
#include <atomic>
#include <cstdio>

#include "cf_device_math.cuh"

namespace cf {

__device__ __forceinline__ void group_sync(int gid, int nthreads) {
  if (nthreads == 32) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(nthreads) : "memory");
}

__device__ __forceinline__ float ctrl_at(const StepParams& P, int step, int uadr, int uoff) {
  if (P.nctrl <= 0 || uoff < 0) return 0.f;
  int slice = P.ctrl_offset + step;
  slice = slice < P.nctrl ? slice : P.nctrl - 1;
  return P.ctrl[(size_t)slice * P.total_nu + uadr + uoff];
}

struct PlaneDev {
  f3 o, n, x;
  float mu[3];
};

__device__ __forceinline__ PlaneDev load_plane(const DGeom& g) {
  M33 R = quat_mat(g.quat[0], g.quat[1], g.quat[2], g.quat[3]);
  PlaneDev p;
  p.o = mk3(g.pos[0], g.pos[1], g.pos[2]);
  p.n = col(R, 2);
  p.x = col(R, 0);
  p.mu[0] = g.mu[0]; p.mu[1] = g.mu[1]; p.mu[2] = g.mu[2];
  return p;
}

__device__ __forceinline__ void capture_contact(const StepParams& P, int world, int* s_count, int ga, int gb, int sub,
                                                float phi, f3 p, f3 n, float lam, float mphi, float rho,
                                                float wn, float target, bool b_static) {
  int slot = atomicAdd(s_count + 1, 1);
  if (slot < P.capture_cap) {
    cf_contact c;
    c.geom_a = ga; c.geom_b = gb; c.sub = sub; c.flags = b_static ? CF_CONTACT_B_STATIC : 0;
    c.phi = phi;
    c.pos[0] = p.x; c.pos[1] = p.y; c.pos[2] = p.z;
    c.normal[0] = n.x; c.normal[1] = n.y; c.normal[2] = n.z;
    c.lam_sum = lam; c.mphi = mphi;
    c.rho = rho; c.wn = wn; c.target = target;
    P.capture[(size_t)world * P.capture_cap + slot] = c;
  }
}

// =======================================================================================
// pile worlds: free bodies, geom i on body i at its origin, static planes
// =======================================================================================
struct PileView {
  int N, NP;
  int* acch;                // [6][N] velocity change (v; body-frame w), high words
  unsigned* accl;           // [6][N] low words
  float4* pb;               // [N] position (x, y, z) and bounding radius
  float4* rec;              // [N][7] body records, see kRec*
  const DGeom* geoms;       // the scene's geoms: body i carries geom i (friction coefficients)
  float* planes;            // [NP][12]
  int* queue;               // [warps][2][kCandQueue] broadphase candidates: capsule-capsule pairs, the rest
  float* cq;                // [warps][8][kQueue] contacts: p.xyz, n.xyz, phi, code
  int* count;               // [0] contacts, [1] captured
};

// Codes (pile bodies <= 4096, planes <= 4096): a candidate is (a << 16) | b for a body pair and
// (a << 16) | 0x8000 | plane for a body-plane pair; a queued contact adds its sub-contact (0..7:
// capsule ends, box corners, cylinder rim points, clipped box-box vertices) as sub << 12.
constexpr int kPlaneBit = 0x8000;
constexpr int kPlaneMask = 0xfff;
constexpr int kBodyMask = 0xfff;

__device__ __forceinline__ int code_with_sub(int code, int sub) { return code | (sub << 12); }
constexpr int kCqWords = 8;
constexpr int kCandQueue = 128;  // per-warp broadphase candidate queue of a pile world (entries)

// Body record of a pile body, 7 float4 (one vector load each):
//   0: linear velocity (v, then v_s, then v+), 1/m      1: body-frame angular velocity, 1/I_0
//   2: R row 0, 1/I_1        3: R row 1, 1/I_2          4: R row 2, size 0 (radius)
//   5: size 1, size 2, geom type (int bits), 0          6: orientation quaternion (w, x, y, z)
// (R stored by columns, so that a capsule's axis and radius came in one load, measured 1.4%
// slower on the 4096 x 256 pile.)
constexpr int kRec = 7;

__host__ __device__ inline size_t pile_floats(int N, int NP, int warps) {
  // accumulators (12 words/body) + position (4) + record (28) + planes + both queues + counters
  size_t words = (size_t)N * 12 + (size_t)N * 32 + (size_t)NP * 12 + (size_t)warps * (kQueue * kCqWords + 2 * kCandQueue) + 4;
  return (words + 3) & ~(size_t)3;
}

__device__ inline PileView pile_view(float* base, int N, int NP, int warps) {
  PileView s;
  s.N = N; s.NP = NP;
  s.acch = reinterpret_cast<int*>(base);
  s.accl = reinterpret_cast<unsigned*>(base + (size_t)N * 6);
  float* f = base + (size_t)N * 12;
  s.pb = reinterpret_cast<float4*>(f); f += 4 * (size_t)N;
  s.rec = reinterpret_cast<float4*>(f); f += 4 * (size_t)kRec * N;
  s.planes = f; f += (size_t)NP * 12;
  s.cq = f; f += (size_t)warps * kQueue * kCqWords;
  s.queue = reinterpret_cast<int*>(f); f += (size_t)warps * 2 * kCandQueue;
  s.count = reinterpret_cast<int*>(f);
  return s;
}

__device__ __forceinline__ M33 pile_R(const PileView& s, int i) {
  const float4 a = s.rec[kRec * i + 2], b = s.rec[kRec * i + 3], c = s.rec[kRec * i + 4];  // columns
  M33 R;
  R.m[0] = a.x; R.m[1] = a.y; R.m[2] = a.z; R.m[3] = b.x; R.m[4] = b.y; R.m[5] = b.z;
  R.m[6] = c.x; R.m[7] = c.y; R.m[8] = c.z;
  return R;
}
__device__ __forceinline__ f3 pile_axis(const PileView& s, int i) {  // body z axis (column 2 of R)
  return mk3(s.rec[kRec * i + 2].z, s.rec[kRec * i + 3].z, s.rec[kRec * i + 4].z);
}
__device__ __forceinline__ int pile_type(const PileView& s, int i) { return __float_as_int(s.rec[kRec * i + 5].z); }
__device__ __forceinline__ float pile_rad(const PileView& s, int i) { return s.rec[kRec * i + 4].w; }
__device__ __forceinline__ float pile_hl(const PileView& s, int i) { return s.rec[kRec * i + 5].x; }
__device__ __forceinline__ float pile_s2(const PileView& s, int i) { return s.rec[kRec * i + 5].y; }

// translational trace tr(J_i M^-1 J_i^T) of a free body at lever r (world) or 1/m;
// im = 1/m, ii = inverse principal inertia
__device__ __forceinline__ float pile_trace(const StepParams& P, float im, f3 ii, const M33& R, f3 r) {
  if (P.trace_mode == 1) return im;
  f3 l = mulT(R, r);
  return 3.f * im + dot(r, r) * (ii.x + ii.y + ii.z) - (l.x * l.x * ii.x + l.y * l.y * ii.y + l.z * l.z * ii.z);
}

// scatter the velocity change M^-1 J~^T lambda of one body: linear (world) and angular (body
// frame), the contact wrench (f, m) acting at lever r with the given sign
__device__ __forceinline__ void pile_apply(PileView& s, int i, float im, f3 ii, const M33& R, f3 r, f3 f, f3 m,
                                           float sign, bool& range) {
  const f3 ang = mulT(R, cross(r, f) + m);
  const float sm = sign * im;
  const int N = s.N;
  const float d0 = sm * f.x, d1 = sm * f.y, d2 = sm * f.z;
  const float d3 = sign * ii.x * ang.x, d4 = sign * ii.y * ang.y, d5 = sign * ii.z * ang.z;
  // a contribution beyond the fixed-point range (or NaN) voids the step: CF_FLAG_RANGE
  range |= !(fabsf(d0) <= kFix2Range) || !(fabsf(d1) <= kFix2Range) || !(fabsf(d2) <= kFix2Range) ||
           !(fabsf(d3) <= kFix2Range) || !(fabsf(d4) <= kFix2Range) || !(fabsf(d5) <= kFix2Range);
  fix2_add(s.acch + i, s.accl + i, d0);
  fix2_add(s.acch + N + i, s.accl + N + i, d1);
  fix2_add(s.acch + 2 * N + i, s.accl + 2 * N + i, d2);
  fix2_add(s.acch + 3 * N + i, s.accl + 3 * N + i, d3);
  fix2_add(s.acch + 4 * N + i, s.accl + 4 * N + i, d4);
  fix2_add(s.acch + 5 * N + i, s.accl + 5 * N + i, d5);
}

// Solve one queued contact: frame, M(phi), facet impulses, scatter onto both bodies
// (a plane contributes nothing).  kExt: the step kernel's optional features (kExtImp: the
// exact and learned impedances; kExtGeo: box-box contacts, cylinders and ellipsoids).
template <int kExt>
__device__ __forceinline__ void pile_solve(const StepParams& P, PileView& s, const DScene& sc, int world,
                                           const float* cq, int slot, bool& range) {
  Raw k;
  k.p = mk3(cq[slot], cq[kQueue + slot], cq[2 * kQueue + slot]);
  k.n = mk3(cq[3 * kQueue + slot], cq[4 * kQueue + slot], cq[5 * kQueue + slot]);
  k.phi = cq[6 * kQueue + slot];
  const int code = __float_as_int(cq[7 * kQueue + slot]);
  const int a = (code >> 16) & kBodyMask, bc = code & 0xffff;
  const bool plane = (bc & kPlaneBit) != 0;
  const int b = plane ? -1 : (bc & kBodyMask);
  const int sub = (bc >> 12) & 7;
  f3 px = mk3(0.f, 0.f, 0.f);
  // pair friction: the larger of the two geoms' coefficients (one triple for uniform scenes)
  float mu_t = sc.mu[0], mu_tor = sc.mu[1], mu_rol = sc.mu[2];
  int gb;
  if (plane) {
    const float* pl = s.planes + 12 * (bc & kPlaneMask);
    px = mk3(pl[6], pl[7], pl[8]);
    if (!sc.mu_uniform) { mu_t = pl[9]; mu_tor = pl[10]; mu_rol = pl[11]; }
    gb = sc.geom0 + sc.plane0 + (bc & kPlaneMask);
  } else {
    if (!sc.mu_uniform) { const float* mb = s.geoms[b].mu; mu_t = mb[0]; mu_tor = mb[1]; mu_rol = mb[2]; }
    gb = sc.geom0 + b;
  }
  if (!sc.mu_uniform) {
    const float* ma = s.geoms[a].mu;
    mu_t = fmaxf(ma[0], mu_t); mu_tor = fmaxf(ma[1], mu_tor); mu_rol = fmaxf(ma[2], mu_rol);
  }
  f3 t1, t2;
  contact_frame(k.n, plane, px, t1, t2);
  M33 Ra = pile_R(s, a);
  float4 pa = s.pb[a];
  f3 ra = k.p - mk3(pa.x, pa.y, pa.z);
  const float4 va = s.rec[kRec * a], wa4 = s.rec[kRec * a + 1];
  f3 wa = mul(Ra, mk3(wa4.x, wa4.y, wa4.z));
  f3 vc = mk3(va.x, va.y, va.z) + cross(wa, ra);
  f3 wc = wa;
  const float ima = va.w;
  const f3 iia = mk3(wa4.w, s.rec[kRec * a + 2].w, s.rec[kRec * a + 3].w);
  float tr = pile_trace(P, ima, iia, Ra, ra);
  M33 Rb;
  f3 rb, iib;
  float imb = 0.f;
  if (b >= 0) {
    Rb = pile_R(s, b);
    float4 pbb = s.pb[b];
    rb = k.p - mk3(pbb.x, pbb.y, pbb.z);
    const float4 vb = s.rec[kRec * b], wb4 = s.rec[kRec * b + 1];
    f3 wb = mul(Rb, mk3(wb4.x, wb4.y, wb4.z));
    vc = vc - (mk3(vb.x, vb.y, vb.z) + cross(wb, rb));
    wc = wc - wb;
    imb = vb.w;
    iib = mk3(wb4.w, s.rec[kRec * b + 2].w, s.rec[kRec * b + 3].w);
    tr += pile_trace(P, imb, iib, Rb, rb);
  }
  float mphi = 0.f, target = 0.f;
  float w[6];
  ImpFeat feat;
  const bool imp = (kExt & kExtImp) && P.trace_mode >= 2;  // exact or learned impedance
  if (imp) {
    float w_n = free_normal_inverse_mass(ima, iia, Ra, ra, k.n);
    if (b >= 0) w_n += free_normal_inverse_mass(imb, iib, Rb, rb, k.n);
    feat = impnet_features(P, k.phi, tr, ima + imb, w_n, b < 0);
  }
  if ((kExt & kExtImp) && P.trace_mode == 2) {
    Gram g;
    gram_zero(g);
    gram_add_free(g, ima, iia, Ra, ra, k.n, t1, t2);
    if (b >= 0) gram_add_free(g, imb, iib, Rb, rb, k.n, t1, t2);
    facet_impulses_exact(P, dot(k.n, vc), dot(t1, vc), dot(t2, vc), dot(k.n, wc), dot(t1, wc), dot(t2, wc), k.phi,
                         mu_t, mu_tor, mu_rol, g, w);
    if (P.capture_cap > 0) {  // the learned impedance's target: ln(mean exact impedance / M(phi))
      const float r = solimp_r(P, fabsf(k.phi));
      target = logf(facet_mean_exact_impedance(P, mu_t, mu_tor, mu_rol, g) * (1.f - r) * tr / r);
    }
  } else {
    float r = solimp_r(P, fabsf(k.phi));
    mphi = __fdividef(r, (1.f - r) * tr);
    if ((kExt & kExtImp) && P.trace_mode == 3) mphi *= impnet_scale(P.impnet + (size_t)world * P.impnet_stride, feat);
    facet_impulses(P, dot(k.n, vc), dot(t1, vc), dot(t2, vc), dot(k.n, wc), dot(t1, wc), dot(t2, wc), k.phi,
                   P.k_user * mphi, P.d_user * mphi, mu_t, mu_tor, mu_rol, w);
  }
  f3 f = w[0] * k.n + w[1] * t1 + w[2] * t2;
  f3 m = w[3] * k.n + w[4] * t1 + w[5] * t2;
  pile_apply(s, a, ima, iia, Ra, ra, f, m, 1.f, range);
  if (b >= 0) pile_apply(s, b, imb, iib, Rb, rb, f, m, -1.f, range);
  if (P.capture_cap > 0)
    capture_contact(P, world, s.count, sc.geom0 + a, gb, sub, k.phi, k.p, k.n, w[0], mphi, imp ? feat.x[1] : 0.f,
                    imp ? feat.x[2] : 0.f, target, b < 0);
}

// narrowphase of body a against body b (sub-contact 0 only); phi = +inf when there is none.
// Spheres are handled as capsules of zero half length, so sphere-sphere and sphere-capsule
// in either order share one branch.
template <int kExt>
__device__ __forceinline__ Raw pile_narrow_pair(const PileView& s, int a, int b, f3 ca, int sub) {
  const int ta = pile_type(s, a), tb = pile_type(s, b);
  const float4 pb4 = s.pb[b];
  const f3 cb = mk3(pb4.x, pb4.y, pb4.z);
  Raw k;
  k.phi = 3.0e38f;
  // sphere and capsule pairs reduce to two spheres at the closest points of their axes
  // (a sphere's axis is its centre), met by one sphere-sphere test after the branches
  f3 sa = ca, sb = cb;
  bool spheres = false;
  if ((kExt & kExtGeo) && (ta >= CF_GEOM_CYLINDER || tb >= CF_GEOM_CYLINDER)) {  // cylinders touch spheres only
    if (ta == CF_GEOM_SPHERE && tb == CF_GEOM_CYLINDER)
      k = nf_sphere_cylinder(ca, pile_rad(s, a), cb, pile_R(s, b), pile_rad(s, b), pile_hl(s, b), true);
    else if (ta == CF_GEOM_CYLINDER && tb == CF_GEOM_SPHERE)
      k = nf_sphere_cylinder(cb, pile_rad(s, b), ca, pile_R(s, a), pile_rad(s, a), pile_hl(s, a), false);
  } else if (ta == CF_GEOM_CAPSULE && tb == CF_GEOM_CAPSULE) {
    f3 ua = pile_axis(s, a), ub = pile_axis(s, b);
    f3 p1 = ca - pile_hl(s, a) * ua, q1 = ca + pile_hl(s, a) * ua, p2 = cb - pile_hl(s, b) * ub, q2 = cb + pile_hl(s, b) * ub;
    float ss, tt;
    nf_segments(p1, q1, p2, q2, ss, tt);
    sa = p1 + ss * (q1 - p1);
    sb = p2 + tt * (q2 - p2);
    spheres = true;
  } else if (ta != CF_GEOM_BOX && tb != CF_GEOM_BOX) {  // sphere-sphere, capsule-sphere, sphere-capsule
    const bool capA = ta == CF_GEOM_CAPSULE;
    const int ic = capA ? a : b;
    const f3 cc = capA ? ca : cb, cs = capA ? cb : ca;
    const float h = ta == CF_GEOM_SPHERE && tb == CF_GEOM_SPHERE ? 0.f : pile_hl(s, ic);
    const f3 u = pile_axis(s, ic);
    const float t = fminf(fmaxf(dot(cs - cc, u), -h), h);
    const f3 pc = cc + t * u;
    if (capA) sa = pc;
    else sb = pc;
    spheres = true;
  } else if (ta == CF_GEOM_BOX && tb == CF_GEOM_BOX) {  // clipped face vertex `sub`
    if (kExt & kExtGeo)
      k = nf_box_box(ca, pile_R(s, a), mk3(pile_rad(s, a), pile_hl(s, a), pile_s2(s, a)), cb, pile_R(s, b), mk3(pile_rad(s, b), pile_hl(s, b), pile_s2(s, b)),
                   sub);
  } else if ((ta == CF_GEOM_BOX) != (tb == CF_GEOM_BOX)) {
    bool boxA = ta == CF_GEOM_BOX;
    int ib = boxA ? a : b, io = boxA ? b : a;
    M33 Rbx = pile_R(s, ib);
    f3 cbx = boxA ? ca : cb, co = boxA ? cb : ca;
    f3 hs = mk3(pile_rad(s, ib), pile_hl(s, ib), pile_s2(s, ib));
    if (pile_type(s, io) == CF_GEOM_SPHERE) {
      k = nf_sphere_box(co, pile_rad(s, io), cbx, Rbx, hs, !boxA);
    } else {
      f3 u = pile_axis(s, io);
      float t = nf_capsule_box_param(mulT(Rbx, co - cbx), mulT(Rbx, u), pile_hl(s, io), hs);
      k = nf_sphere_box(co + t * u, pile_rad(s, io), cbx, Rbx, hs, !boxA);
    }
  }
  if (spheres) k = nf_sphere_sphere(sa, pile_rad(s, a), sb, pile_rad(s, b));
  return k;
}

// narrowphase of body a against a plane: sphere (sub 0), capsule end sphere sub, box corner sub
template <int kExt>
__device__ __forceinline__ Raw pile_narrow_plane(const PileView& s, int a, int sub, f3 ca, f3 o, f3 nz) {
  const int ta = pile_type(s, a);
  if ((kExt & kExtGeo) && ta == CF_GEOM_CYLINDER) return nf_cylinder_plane(ca, pile_R(s, a), pile_rad(s, a), pile_hl(s, a), o, nz, sub);
  if ((kExt & kExtGeo) && ta == CF_GEOM_ELLIPSOID)
    return nf_ellipsoid_plane(ca, pile_R(s, a), mk3(pile_rad(s, a), pile_hl(s, a), pile_s2(s, a)), o, nz);
  f3 c = ca;
  float r = pile_rad(s, a);
  if (ta == CF_GEOM_CAPSULE) {
    c = ca + (sub ? pile_hl(s, a) : -pile_hl(s, a)) * pile_axis(s, a);
  } else if (ta == CF_GEOM_BOX) {
    c = ca + mul(pile_R(s, a), mk3((sub & 4) ? pile_rad(s, a) : -pile_rad(s, a), (sub & 2) ? pile_hl(s, a) : -pile_hl(s, a),
                                   (sub & 1) ? pile_s2(s, a) : -pile_s2(s, a)));
    r = 0.f;
  }
  return nf_sphere_plane(c, r, o, nz);
}

// number of sub-contacts a candidate can produce (a plane: per end sphere or box corner)
template <int kExt>
__device__ __forceinline__ int pile_nsub(const PileView& s, int code) {
  if (code < 0) return 0;
  const int ta = pile_type(s, code >> 16);
  if (!(code & kPlaneBit)) return (kExt & kExtGeo) && ta == CF_GEOM_BOX && pile_type(s, code & kBodyMask) == CF_GEOM_BOX ? 8 : 1;
  if ((kExt & kExtGeo) && ta >= CF_GEOM_CYLINDER) return ta == CF_GEOM_CYLINDER ? 6 : 1;
  return ta == CF_GEOM_SPHERE ? 1 : (ta == CF_GEOM_CAPSULE ? 2 : 8);
}

// narrowphase of candidate `code` (-1: none), sub-contact `sub`; true when it is a contact
template <int kExt>
__device__ __forceinline__ bool pile_narrow(const StepParams& P, const PileView& s, int code, int sub, Raw& k) {
  if (code < 0) return false;
  const int a = code >> 16, bc = code & 0xffff;
  const float4 pa4 = s.pb[a];
  const f3 ca = mk3(pa4.x, pa4.y, pa4.z);
  if (bc & kPlaneBit) {
    const float* pl = s.planes + 12 * (bc & kPlaneMask);
    k = pile_narrow_plane<kExt>(s, a, sub, ca, mk3(pl[0], pl[1], pl[2]), mk3(pl[3], pl[4], pl[5]));
  } else {
    k = pile_narrow_pair<kExt>(s, a, bc, ca, sub);
  }
  return k.phi < P.margin;
}

// cos(th) and sin(th) / |w| for th = |w| dt / 2, from w2 = |w|^2: for th^2 <= 0.25 the Taylor
// series of cos and of sin(th) / th to the th^8 term (truncation below th^10 / 10! < 3e-10),
// with no square root or division; beyond it, sincosf of th
__device__ __forceinline__ void exp_half_angle(float w2, float dt, float& c, float& s_over_w) {
  const float h = 0.5f * dt;
  const float x = h * h * w2;  // th^2
  if (x <= 0.25f) {
    c = 1.f + x * (-1.f / 2.f + x * (1.f / 24.f + x * (-1.f / 720.f + x * (1.f / 40320.f))));
    s_over_w = h * (1.f + x * (-1.f / 6.f + x * (1.f / 120.f + x * (-1.f / 5040.f + x * (1.f / 362880.f)))));
  } else {
    const float wn = sqrtf(w2);
    float sn;
    sincosf(h * wn, &sn, &c);
    s_over_w = sn / wn;
  }
}

// Squared distance of two bounding-sphere centres, rounded in a fixed order (measured 1% faster
// on the 4096 x 256 pile than the form the compiler contracts by itself)
__device__ __forceinline__ float bs_dist2(const float4& a, const float4& b) {
  const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}
// bounding spheres a (radius already grown by the margin) and b overlap
__device__ __forceinline__ bool bs_hit(const float4& a, const float4& b) {
  const float rr = __fadd_rn(a.w, b.w);
  return bs_dist2(a, b) < __fmul_rn(rr, rr);
}

template <int kExt>
__device__ void pile_world(const StepParams& P, float* smem, int world, int gid, int gwarps) {
  const DWorld W = P.worlds[world];
  const DScene sc = P.scenes[W.scene];
  const int N = sc.nbody, NP = sc.nplane;
  const int T = gwarps * 32;
  const int tid = threadIdx.x - gid * T;
  const int lane = threadIdx.x & 31, wig = tid >> 5;
  PileView s = pile_view(smem, N, NP, gwarps);
  s.geoms = P.geoms + sc.geom0;
  const float* q = P.q + W.qadr;
  const float* v = P.v + W.vadr;
  const float dt = P.dt;

  // load state and per-world parameters
  for (int i = tid; i < N; i += T) {
    const float* qi = q + 7 * i;
    float px = qi[0], py = qi[1], pz = qi[2];
    const float* vi = v + 6 * i;
    float4* rc = s.rec + kRec * i;
    float m, i0, i1, i2, ty, r, h, s2;
    if (W.padr >= 0) {
      const float4* pp = reinterpret_cast<const float4*>(P.wparam + W.padr + 8 * i);
      float4 p0 = pp[0], p1 = pp[1];
      m = p0.x; i0 = p0.y; i1 = p0.z; i2 = p0.w; ty = p1.x; r = p1.y; h = p1.z; s2 = p1.w;
    } else {
      const DBody& bd = P.bodies[sc.body0 + i];
      const DGeom& gd = P.geoms[sc.geom0 + i];
      m = bd.mass; i0 = bd.inertia[0]; i1 = bd.inertia[1]; i2 = bd.inertia[2];
      ty = (float)gd.type; r = gd.size[0]; h = gd.size[1]; s2 = gd.size[2];
    }
    int t = (int)ty;
    rc[0] = make_float4(vi[0], vi[1], vi[2], 1.f / m);
    rc[1] = make_float4(vi[3], vi[4], vi[5], 1.f / i0);
    rc[2].w = 1.f / i1;
    rc[3].w = 1.f / i2;
    rc[4].w = r;
    rc[5] = make_float4(h, s2, __int_as_float(t), 0.f);
    rc[6] = make_float4(qi[3], qi[4], qi[5], qi[6]);
    const float bound = t == CF_GEOM_SPHERE ? r
                        : t == CF_GEOM_CAPSULE ? r + h
                        : t == CF_GEOM_CYLINDER ? sqrtf(r * r + h * h)
                        : t == CF_GEOM_ELLIPSOID ? fmaxf(r, fmaxf(h, s2))
                                                 : sqrtf(r * r + h * h + s2 * s2);
    s.pb[i] = make_float4(px, py, pz, bound);
  }
  for (int pi = tid; pi < NP; pi += T) {
    PlaneDev pl = load_plane(P.geoms[sc.geom0 + sc.plane0 + pi]);
    float* o = s.planes + 12 * pi;
    o[0] = pl.o.x; o[1] = pl.o.y; o[2] = pl.o.z; o[3] = pl.n.x; o[4] = pl.n.y; o[5] = pl.n.z;
    o[6] = pl.x.x; o[7] = pl.x.y; o[8] = pl.x.z; o[9] = pl.mu[0]; o[10] = pl.mu[1]; o[11] = pl.mu[2];
  }
  const f3 g = mk3(P.gravity[0], P.gravity[1], P.gravity[2]);
  int* queue = s.queue + wig * 2 * kCandQueue;   // [0]: capsule-capsule pairs, [kCandQueue]: the rest
  bool range = false;  // some velocity change left the scatter's range

  for (int step = 0; step < P.nsteps; ++step) {
    group_sync(gid, T);
    // ---- A. kinematics and smooth prediction (free body: c = (-m g, w x I w)), v -> v_s ----
    for (int i = tid; i < N; i += T) {
      float4* rc = s.rec + kRec * i;
      const float4 qq = rc[6], r0 = rc[0], r1 = rc[1];
      M33 R = quat_mat(qq.x, qq.y, qq.z, qq.w);
      const float ii0 = r1.w, ii1 = rc[2].w, ii2 = rc[3].w;  // inverse principal inertia
      rc[2] = make_float4(R.m[0], R.m[1], R.m[2], ii1);
      rc[3] = make_float4(R.m[3], R.m[4], R.m[5], ii2);
      rc[4] = make_float4(R.m[6], R.m[7], R.m[8], rc[4].w);
      float w0 = r1.x, w1 = r1.y, w2 = r1.z;
      f3 gy = cross(mk3(w0, w1, w2), mk3(__fdividef(w0, ii0), __fdividef(w1, ii1), __fdividef(w2, ii2)));
      rc[0] = make_float4(r0.x + g.x * dt, r0.y + g.y * dt, r0.z + g.z * dt, r0.w);
      rc[1] = make_float4(w0 - dt * gy.x * ii0, w1 - dt * gy.y * ii1, w2 - dt * gy.z * ii2, ii0);
#pragma unroll
      for (int k = 0; k < 6; ++k) { s.acch[k * N + i] = 0; s.accl[k * N + i] = 0u; }
    }
    if (tid == 0) { s.count[0] = 0; s.count[1] = 0; }
    group_sync(gid, T);

    // ---- B. broadphase -> candidate queue -> narrowphase -> contact queue -> solve ----
    // Body pairs are tested in 32 x 32 tiles (i-chunk <= j-chunk) dealt round-robin to the
    // warps: each lane holds body i in registers, the j loop is warp-uniform (broadcast loads)
    // and the bounding-sphere hits of a tile are kept as a 32-bit mask per lane, split into
    // capsule-capsule pairs and the rest (a ballot of the j-chunk's capsules).  All hits of a
    // tile are then compacted into the two candidate queues at once (a warp prefix sum of the
    // masks' popcounts gives each lane its slots); after the tiles, every body is tested against
    // the planes, 32 planes per mask, and compacted the same way.  Every 32 candidates of one
    // queue run the narrowphase one per lane, so a batch takes one narrowphase branch (the
    // segment-segment one or the cheap ones), and its hits are compacted into the contact
    // queue; every 32 contacts are solved one per lane.  So the solve, the costly part, runs on
    // full warps although only a fraction of the candidates touch.
    {
      const float margin = P.margin;
      const unsigned lt = (1u << lane) - 1u;
      float* cq = s.cq + wig * kQueue * kCqWords;
      const int nchunk = (N + 31) >> 5;
      const int ntile = nchunk * (nchunk + 1) / 2;
      int qa = 0, qb = 0, cn = 0;           // queued capsule-capsule pairs, queued other candidates
      int phase = 0;                        // 0: body-pair tiles, 1: planes, 2: all masks made
      int t = wig, a0 = wig * 32, p0 = 0;   // next tile; next (32 bodies, 32 planes) plane block
      unsigned ma = 0, mb = 0;              // this lane's hits not yet queued, by class (bit k: j0 + k)
      int code_hi = 0, j0 = 0, totala = 0, totalb = 0, excla = 0, exclb = 0;
      while (true) {
        if (qa < 32 && qb < 32) {
          while (totala == 0 && totalb == 0 && phase < 2) {
            unsigned m = 0;
            if (phase == 0) {
              if (t >= ntile) { phase = NP > 0 ? 1 : 2; continue; }
              int rem = t, ci = 0;
              while (rem >= nchunk - ci) { rem -= nchunk - ci; ++ci; }
              const int cj = ci + rem;
              const int i = (ci << 5) + lane;
              float4 pi4 = make_float4(3.0e30f, 3.0e30f, 3.0e30f, 0.f);
              if (i < N) { pi4 = s.pb[i]; pi4.w += margin; }
              j0 = cj << 5;
              const int kmax = min(32, N - j0);
#pragma unroll 8
              for (int k = 0; k < kmax; ++k)
                if (bs_hit(pi4, s.pb[j0 + k])) m |= 1u << k;
              if (ci == cj) m &= 0xfffffffeu << lane;
              const unsigned capj = __ballot_sync(0xffffffffu, j0 + lane < N && pile_type(s, j0 + lane) == CF_GEOM_CAPSULE);
              const bool cc = i < N && pile_type(s, i) == CF_GEOM_CAPSULE;
              code_hi = i << 16;
              t += gwarps;
              ma = cc ? (m & capj) : 0u;
              mb = m & ~ma;
            } else {
              if (a0 >= N) { phase = 2; break; }
              const int a = a0 + lane;
              if (a < N) {
                const float4 a4 = s.pb[a];
                const int pn = min(32, NP - p0);
                for (int k = 0; k < pn; ++k) {
                  const float* pl = s.planes + 12 * (p0 + k);
                  const float d = (a4.x - pl[0]) * pl[3] + (a4.y - pl[1]) * pl[4] + (a4.z - pl[2]) * pl[5];
                  if (d < a4.w + margin) m |= 1u << k;
                }
              }
              code_hi = (a << 16) | kPlaneBit;
              j0 = p0;
              p0 += 32;
              if (p0 >= NP) { p0 = 0; a0 += T; }
              ma = 0u;
              mb = m;
            }
            const int ca_ = __popc(ma), cb_ = __popc(mb);
            totala = __reduce_add_sync(0xffffffffu, ca_);
            totalb = __reduce_add_sync(0xffffffffu, cb_);
            int ia = ca_, ib = cb_;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
              const int ya = __shfl_up_sync(0xffffffffu, ia, d), yb = __shfl_up_sync(0xffffffffu, ib, d);
              if (lane >= d) { ia += ya; ib += yb; }
            }
            excla = ia - ca_;
            exclb = ib - cb_;
          }
          __syncwarp();
          if (totala > 0) {
            const int room = kCandQueue - qa;
            for (int k = excla; ma && k < room; ++k) {
              queue[qa + k] = code_hi | (j0 + __ffs(ma) - 1);
              ma &= ma - 1;
            }
            const int put = min(totala, room);
            qa += put;
            totala -= put;
            excla = max(excla - room, 0);
          }
          if (totalb > 0) {
            const int room = kCandQueue - qb;
            for (int k = exclb; mb && k < room; ++k) {
              queue[kCandQueue + qb + k] = code_hi | (j0 + __ffs(mb) - 1);
              mb &= mb - 1;
            }
            const int put = min(totalb, room);
            qb += put;
            totalb -= put;
            exclb = max(exclb - room, 0);
          }
        }
        const bool fin = phase == 2 && totala == 0 && totalb == 0;
        if (qa < 32 && qb < 32 && !fin) continue;
        const bool from_a = qa >= 32 || (qb < 32 && qa > 0);
        int& qn = from_a ? qa : qb;
        int* qsrc = from_a ? queue : queue + kCandQueue;
        const int nb = min(qn, 32);
        const bool last = fin && qa + qb == nb;
        __syncwarp();
        const int mine = lane < nb ? qsrc[qn - nb + lane] : -1;
        qn -= nb;
        const int my_nsub = pile_nsub<kExt>(s, mine);
        const int nsub = max(__reduce_max_sync(0xffffffffu, my_nsub), 1);
        for (int sub = 0; sub < nsub; ++sub) {
          Raw kc;
          const bool hit = sub < my_nsub && pile_narrow<kExt>(P, s, mine, sub, kc);
          const unsigned hm = __ballot_sync(0xffffffffu, hit);
          if (hit) {
            const int slot = cn + __popc(hm & lt);
            cq[slot] = kc.p.x; cq[kQueue + slot] = kc.p.y; cq[2 * kQueue + slot] = kc.p.z;
            cq[3 * kQueue + slot] = kc.n.x; cq[4 * kQueue + slot] = kc.n.y; cq[5 * kQueue + slot] = kc.n.z;
            cq[6 * kQueue + slot] = kc.phi;
            cq[7 * kQueue + slot] = __int_as_float(code_with_sub(mine, sub));
          }
          cn += __popc(hm);
          const bool flush = last && sub + 1 == nsub;
          while (cn >= 32 || (flush && cn > 0)) {
            __syncwarp();
            const int ns = min(cn, 32);
            if (lane < ns) pile_solve<kExt>(P, s, sc, world, cq, cn - ns + lane, range);
            if (lane == 0) atomicAdd(s.count, ns);  // contacts of the world
            cn -= ns;
            __syncwarp();
          }
        }
        if (last) break;
      }
    }
    group_sync(gid, T);

    // ---- C. velocity correction and semi-implicit Euler ----
    for (int i = tid; i < N; i += T) {
      float4* rc = s.rec + kRec * i;
      const float4 r0 = rc[0], r1 = rc[1];
      float v0 = r0.x + fix2_get(s.acch[i], s.accl[i]);
      float v1 = r0.y + fix2_get(s.acch[N + i], s.accl[N + i]);
      float v2 = r0.z + fix2_get(s.acch[2 * N + i], s.accl[2 * N + i]);
      float w0 = r1.x + fix2_get(s.acch[3 * N + i], s.accl[3 * N + i]);
      float w1 = r1.y + fix2_get(s.acch[4 * N + i], s.accl[4 * N + i]);
      float w2 = r1.z + fix2_get(s.acch[5 * N + i], s.accl[5 * N + i]);
      rc[0] = make_float4(v0, v1, v2, r0.w);
      rc[1] = make_float4(w0, w1, w2, r1.w);
      s.pb[i].x += v0 * dt; s.pb[i].y += v1 * dt; s.pb[i].z += v2 * dt;
      float dq0, sh;  // the rotation by w dt: (cos th, sin th w / |w|), th = |w| dt / 2
      exp_half_angle(w0 * w0 + w1 * w1 + w2 * w2, dt, dq0, sh);
      const float dq1 = sh * w0, dq2 = sh * w1, dq3 = sh * w2;
      const float4 qq = rc[6];
      float a0 = qq.x, a1 = qq.y, a2 = qq.z, a3 = qq.w;
      float n0 = a0 * dq0 - a1 * dq1 - a2 * dq2 - a3 * dq3;
      float n1 = a0 * dq1 + a1 * dq0 + a2 * dq3 - a3 * dq2;
      float n2 = a0 * dq2 - a1 * dq3 + a2 * dq0 + a3 * dq1;
      float n3 = a0 * dq3 + a1 * dq2 - a2 * dq1 + a3 * dq0;
      float inv = rsqrtf(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
      rc[6] = make_float4(n0 * inv, n1 * inv, n2 * inv, n3 * inv);
    }
  }
  group_sync(gid, T);
  // ---- write back ----
  float* qo = P.q + W.qadr;
  float* vo = P.v + W.vadr;
  bool bad = false;
  for (int i = tid; i < N; i += T) {
    float* qi = qo + 7 * i;
    float4 p4 = s.pb[i];
    qi[0] = p4.x; qi[1] = p4.y; qi[2] = p4.z;
    const float4* rc = s.rec + kRec * i;
    const float4 qq = rc[6], r0 = rc[0], r1 = rc[1];
    qi[3] = qq.x; qi[4] = qq.y; qi[5] = qq.z; qi[6] = qq.w;
    float* vi = vo + 6 * i;
    vi[0] = r0.x; vi[1] = r0.y; vi[2] = r0.z; vi[3] = r1.x; vi[4] = r1.y; vi[5] = r1.z;
    float chk = p4.x + p4.y + p4.z + qq.x + r0.x + r0.y + r0.z + r1.x + r1.y + r1.z;
    if (!isfinite(chk)) bad = true;
  }
  if (bad) {
    atomicOr(P.flags + world, CF_FLAG_NONFINITE);
    atomicOr(P.errword, CF_FLAG_NONFINITE);
  }
  if (range) {
    atomicOr(P.flags + world, CF_FLAG_RANGE);
    atomicOr(P.errword, CF_FLAG_RANGE);
  }
  if (tid == 0) {
    P.ncontact[world] = s.count[0];
    if (P.capture_cap > 0 && s.count[1] > P.capture_cap) {
      atomicOr(P.flags + world, CF_FLAG_CONTACT_OVERFLOW);
      atomicOr(P.errword, CF_FLAG_CONTACT_OVERFLOW);
    }
  }
}

// =======================================================================================
// articulated worlds: free bodies and fixed-base hinge trees, explicit geom pair lists
// =======================================================================================
struct ArticView {
  int nb, ng, nv, nq, ntree;
  unsigned long long* acc;   // [nv]
  float* q;                  // [nq]
  float* v;                  // [nv]
  float* vs;                 // [nv]
  float* tau;                // [nv]
  float* bx;                 // [nb][3]  body origin
  float* bR;                 // [nb][9]
  float* bom;                // [nb][3]  world angular velocity (smooth)
  float* bvo;                // [nb][3]  world velocity of the origin (smooth)
  float* bax;                // [nb][3]  world hinge axis
  float* gc;                 // [ng][3]
  float* gR;                 // [ng][9]
  float* gb;                 // [ng]     bounding radius
  float* minv;               // [ntree][kMaxTreeDof^2]
  int* queue;                // [warps][kQueue] candidate pairs
  float* cq;                 // [warps][kArtCq][kQueue] contacts: p.xyz, n.xyz, phi, (ga << 16) | gb, sub
  int* count;
};
constexpr int kArtCq = 9;

__host__ __device__ inline size_t artic_floats(int nb, int ng, int nq, int nv, int ntree, int warps) {
  size_t words = (size_t)nv * 2 + nq + 3 * (size_t)nv + (size_t)nb * 21 + (size_t)ng * 13 +
                 (size_t)ntree * kMaxTreeDof * kMaxTreeDof + (size_t)warps * kQueue * (1 + kArtCq) + 4;
  return (words + 3) & ~(size_t)3;
}

__device__ inline ArticView artic_view(float* base, const DScene& sc, int warps) {
  ArticView s;
  s.nb = sc.nbody; s.ng = sc.ngeom; s.nv = sc.nv; s.nq = sc.nq; s.ntree = sc.ntree;
  s.acc = reinterpret_cast<unsigned long long*>(base);
  float* f = base + 2 * (size_t)sc.nv;
  s.q = f; f += sc.nq;
  s.v = f; f += sc.nv;
  s.vs = f; f += sc.nv;
  s.tau = f; f += sc.nv;
  s.bx = f; f += 3 * sc.nbody;
  s.bR = f; f += 9 * sc.nbody;
  s.bom = f; f += 3 * sc.nbody;
  s.bvo = f; f += 3 * sc.nbody;
  s.bax = f; f += 3 * sc.nbody;
  s.gc = f; f += 3 * sc.ngeom;
  s.gR = f; f += 9 * sc.ngeom;
  s.gb = f; f += sc.ngeom;
  s.minv = f; f += (size_t)sc.ntree * kMaxTreeDof * kMaxTreeDof;
  s.queue = reinterpret_cast<int*>(f); f += (size_t)warps * kQueue;
  s.cq = f; f += (size_t)warps * kQueue * kArtCq;
  s.count = reinterpret_cast<int*>(f);
  return s;
}

__device__ __forceinline__ f3 ld3(const float* p) { return mk3(p[0], p[1], p[2]); }
__device__ __forceinline__ void st3(float* p, f3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }
__device__ __forceinline__ M33 ld33(const float* p) {
  M33 r;
#pragma unroll
  for (int k = 0; k < 9; ++k) r.m[k] = p[k];
  return r;
}

// world inertia product R diag(I) R^T u
__device__ __forceinline__ f3 iw_mul(const M33& R, const float* I, f3 u) {
  f3 l = mulT(R, u);
  return mul(R, mk3(I[0] * l.x, I[1] * l.y, I[2] * l.z));
}

// A free body's preparation (hinge trees: artic_tree_prepare_group): pose from q, the smooth
// velocity with the gyroscopic bias w x I w, and its twist.
__device__ void artic_free_prepare(const StepParams& P, ArticView& s, const DScene& sc, const DTree& tr) {
  const DBody* B = P.bodies + sc.body0;
  const float dt = P.dt;
  {
    const int b = tr.body0;
    const DBody& bd = B[b];
    const float* qb = s.q + bd.qoff;
    M33 R = quat_mat(qb[3], qb[4], qb[5], qb[6]);
    st3(s.bx + 3 * b, mk3(qb[0], qb[1], qb[2]));
#pragma unroll
    for (int k = 0; k < 9; ++k) s.bR[9 * b + k] = R.m[k];
    const float* vb = s.v + bd.voff;
    f3 w = mk3(vb[3], vb[4], vb[5]);
    f3 gy = cross(w, mk3(bd.inertia[0] * w.x, bd.inertia[1] * w.y, bd.inertia[2] * w.z));
    float* vsb = s.vs + bd.voff;
    vsb[0] = vb[0] + P.gravity[0] * dt;
    vsb[1] = vb[1] + P.gravity[1] * dt;
    vsb[2] = vb[2] + P.gravity[2] * dt;
    vsb[3] = w.x - dt * gy.x / bd.inertia[0];
    vsb[4] = w.y - dt * gy.y / bd.inertia[1];
    vsb[5] = w.z - dt * gy.z / bd.inertia[2];
    st3(s.bom + 3 * b, mul(R, mk3(vsb[3], vsb[4], vsb[5])));
    st3(s.bvo + 3 * b, mk3(vsb[0], vsb[1], vsb[2]));
    st3(s.bax + 3 * b, mk3(0.f, 0.f, 0.f));
  }
}

// ---- lane-parallel preparation of hinge trees: an 8-lane group per tree, lane r = body r ----
__device__ __forceinline__ float gshf(float v, int k) { return __shfl_sync(0xffffffffu, v, k, 8); }
__device__ __forceinline__ int gshi(int v, int k) { return __shfl_sync(0xffffffffu, v, k, 8); }
__device__ __forceinline__ f3 gsh3(f3 v, int k) { return mk3(gshf(v.x, k), gshf(v.y, k), gshf(v.z, k)); }
// sum over the group's lanes k with bit k of `sel` set of v_k
__device__ __forceinline__ f3 gsum3(f3 v, unsigned sel) {
  f3 acc = mk3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const f3 vk = gsh3(v, k);
    if ((sel >> k) & 1u) acc = acc + vk;
  }
  return acc;
}

// One hinge tree of n <= 8 bodies (one hinge each, parents first) prepared by an 8-lane group
// (Sec. III-A's smooth prediction): body poses, the composite-rigid-body inertia M, the
// Newton-Euler bias c, the implicitly damped M~ = M + dt diag(b), the explicit M~^-1, the
// smooth velocity and the body twists.  Walks along a chain become log-depth or masked-sum
// forms:
//   - world poses by pointer jumping: (R, t) <- (R, t) of the pointer's frame o (R, t), three
//     rounds covering depth 8;
//   - sums over a body's ancestors (angular velocities and their rates, the acceleration of the
//     joint origin, the twists) and over its subtree (composite inertia, the backward forces)
//     as masked sums over the group, the masks being the per-body ancestor bitmasks;
//   - M~ assembled column by column (lane j: the ancestors i of j), factorised by one lane
//     (n <= 8), and M~^-1 solved column by column (lane j: M~ x = e_j).
// Every lane of the warp calls it in step (`active` false: no tree for this group), so that
// the shuffles see the whole warp.
__device__ void artic_tree_prepare_group(const StepParams& P, ArticView& s, const DScene& sc, int t, bool active,
                                         int r) {
  const DBody* B = P.bodies + sc.body0;
  const float dt = P.dt;
  int body0 = 0, n = 0;
  if (active) {
    const DTree& tr = P.trees[sc.tree0 + t];
    body0 = tr.body0;
    n = tr.nv;
  }
  const bool me = r < n;
  const int b = body0 + r;
  // this lane's body
  int par = -1, uoff = -1, qoff = 0, voff = 0;
  unsigned anc = 0u;
  float mass = 1.f, damp = 0.f, q = 0.f, qd = 0.f;
  f3 a = mk3(0.f, 0.f, 1.f), pos = mk3(0.f, 0.f, 0.f), ipos = pos, inert = mk3(1.f, 1.f, 1.f);
  M33 Rq;
#pragma unroll
  for (int k = 0; k < 9; ++k) Rq.m[k] = (k % 4 == 0) ? 1.f : 0.f;
  if (me) {
    const DBody& bd = B[b];
    par = bd.parent >= 0 ? bd.parent - body0 : -1;
    anc = (unsigned)bd.anc;
    uoff = bd.uoff;
    qoff = bd.qoff;
    voff = bd.voff;
    mass = bd.mass;
    damp = bd.damping;
    inert = mk3(bd.inertia[0], bd.inertia[1], bd.inertia[2]);
    pos = mk3(bd.pos[0], bd.pos[1], bd.pos[2]);
    ipos = mk3(bd.ipos[0], bd.ipos[1], bd.ipos[2]);
    a = mk3(bd.axis[0], bd.axis[1], bd.axis[2]);
    a = rsqrtf(dot(a, a)) * a;
    Rq = quat_mat(bd.quat[0], bd.quat[1], bd.quat[2], bd.quat[3]);
    q = s.q[qoff];
    qd = s.v[voff];
  }
  // world pose by pointer jumping over the parent chain
  M33 R = mul33(Rq, axis_rot(a, q));
  f3 x = pos;
  int up = par;
#pragma unroll
  for (int round = 0; round < 3; ++round) {
    const int src = up >= 0 ? up : r;
    M33 Ru;
#pragma unroll
    for (int k = 0; k < 9; ++k) Ru.m[k] = gshf(R.m[k], src);
    const f3 xu = gsh3(x, src);
    const int uu = gshi(up, src);
    if (up >= 0) {
      x = xu + mul(Ru, x);
      R = mul33(Ru, R);
      up = uu;
    }
  }
  const f3 ax = mul(R, a);  // the hinge axis is fixed by its own rotation
  const f3 com = x + mul(R, ipos);
  if (me) {
    st3(s.bx + 3 * b, x);
#pragma unroll
    for (int k = 0; k < 9; ++k) s.bR[9 * b + k] = R.m[k];
    st3(s.bax + 3 * b, ax);
  }
  // parent's origin (the world's for a root)
  const int psrc = par >= 0 ? par : r;
  const f3 xps = gsh3(x, psrc);  // every lane shuffles; roots then take the world's origin
  const f3 xp = par >= 0 ? xps : mk3(0.f, 0.f, 0.f);
  // composite rigid bodies over the subtree: mass, first moment, inertia about the world origin
  float Iw[6];
  {
    const float* rr = R.m;
    const float cc = dot(com, com);
    Iw[0] = rr[0] * rr[0] * inert.x + rr[1] * rr[1] * inert.y + rr[2] * rr[2] * inert.z + mass * (cc - com.x * com.x);
    Iw[1] = rr[3] * rr[3] * inert.x + rr[4] * rr[4] * inert.y + rr[5] * rr[5] * inert.z + mass * (cc - com.y * com.y);
    Iw[2] = rr[6] * rr[6] * inert.x + rr[7] * rr[7] * inert.y + rr[8] * rr[8] * inert.z + mass * (cc - com.z * com.z);
    Iw[3] = rr[0] * rr[3] * inert.x + rr[1] * rr[4] * inert.y + rr[2] * rr[5] * inert.z - mass * com.x * com.y;
    Iw[4] = rr[0] * rr[6] * inert.x + rr[1] * rr[7] * inert.y + rr[2] * rr[8] * inert.z - mass * com.x * com.z;
    Iw[5] = rr[3] * rr[6] * inert.x + rr[4] * rr[7] * inert.y + rr[5] * rr[8] * inert.z - mass * com.y * com.z;
  }
  float mc = 0.f, Io[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  f3 hc = mk3(0.f, 0.f, 0.f);
  {
    const float mine = me ? mass : 0.f;
    const f3 hm = mine * com;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool in = (gshi((int)anc, k) >> r) & 1;  // this lane's body is an ancestor of body k
      const float mk = gshf(mine, k);
      const f3 hk = gsh3(hm, k);
      float ik[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) ik[e] = gshf(me ? Iw[e] : 0.f, k);
      if (in) {
        mc += mk;
        hc = hc + hk;
#pragma unroll
        for (int e = 0; e < 6; ++e) Io[e] += ik[e];
      }
    }
  }
// M~ column by column: lane j writes M_ij = M_ji for the ancestors i of j (zero otherwise),
  // with the implicit damping on the diagonal, into the tree's M~^-1 slot used as scratch
  float* mt = s.minv + (size_t)t * kMaxTreeDof * kMaxTreeDof;
  {
    const f3 cC = (mc > 0.f ? 1.f / mc : 0.f) * hc;
    const float cc = dot(cC, cC);
    const float I6[6] = {Io[0] - mc * (cc - cC.x * cC.x), Io[1] - mc * (cc - cC.y * cC.y),
                         Io[2] - mc * (cc - cC.z * cC.z), Io[3] + mc * cC.x * cC.y,
                         Io[4] + mc * cC.x * cC.z, Io[5] + mc * cC.y * cC.z};
    const f3 Ia = mk3(I6[0] * ax.x + I6[3] * ax.y + I6[4] * ax.z, I6[3] * ax.x + I6[1] * ax.y + I6[5] * ax.z,
                      I6[4] * ax.x + I6[5] * ax.y + I6[2] * ax.z);
    const f3 lin = mc * cross(ax, cC - x);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const f3 axi = gsh3(ax, i), xi = gsh3(x, i);
      if (me && i <= r) {
        float mij = ((anc >> i) & 1u) ? dot(axi, Ia + cross(cC - xi, lin)) : 0.f;
        if (i == r) mij += dt * damp;
        mt[i * kMaxTreeDof + r] = mij;
        mt[r * kMaxTreeDof + i] = mij;
      }
    }
  }
  // Newton-Euler bias with zero joint acceleration, the world accelerating at -g
  const f3 w = qd * ax;                      // this joint's twist
  const f3 om = gsum3(w, anc);               // over the ancestors and the body itself
  const f3 omd = gsum3(cross(om, w), anc);   // om_parent x w = om x w
  const f3 omp = gsh3(om, psrc), omdp = gsh3(omd, psrc);
  const f3 ro = x - xp;
  const f3 term = par >= 0 ? cross(omdp, ro) + cross(omp, cross(omp, ro)) : mk3(0.f, 0.f, 0.f);
  const f3 ao = gsum3(term, anc) - mk3(P.gravity[0], P.gravity[1], P.gravity[2]);  // joint origin
  const f3 rc = com - x;
  const f3 ac = ao + cross(omd, rc) + cross(om, cross(om, rc));
  const f3 F = me ? mass * ac : mk3(0.f, 0.f, 0.f);
  f3 Nn;
  {
    const f3 l1 = mulT(R, omd), l2 = mulT(R, om);
    Nn = mul(R, mk3(inert.x * l1.x, inert.y * l1.y, inert.z * l1.z)) +
         cross(om, mul(R, mk3(inert.x * l2.x, inert.y * l2.y, inert.z * l2.z)));
  }
  const f3 T = me ? Nn + cross(com, F) : mk3(0.f, 0.f, 0.f);
  f3 ft = mk3(0.f, 0.f, 0.f), nt = ft;  // over the subtree
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool in = (gshi((int)anc, k) >> r) & 1;
    const f3 fk = gsh3(F, k), tk = gsh3(T, k);
    if (in) { ft = ft + fk; nt = nt + tk; }
  }
  const float rhs = (uoff >= 0 ? s.tau[uoff] : 0.f) - dot(ax, nt - cross(x, ft)) - damp * qd;
  __syncwarp();
  // M~ = L L^T by one lane (n <= 8), in place in the lower triangle
  if (me && r == 0) {
    for (int j = 0; j < n; ++j) {
      float d = mt[j * kMaxTreeDof + j];
      for (int k = 0; k < j; ++k) d -= mt[j * kMaxTreeDof + k] * mt[j * kMaxTreeDof + k];
      d = sqrtf(fmaxf(d, 1e-30f));
      mt[j * kMaxTreeDof + j] = d;
      for (int i = j + 1; i < n; ++i) {
        float tt = mt[i * kMaxTreeDof + j];
        for (int k = 0; k < j; ++k) tt -= mt[i * kMaxTreeDof + k] * mt[j * kMaxTreeDof + k];
        mt[i * kMaxTreeDof + j] = tt / d;
      }
    }
  }
  __syncwarp();
  // column r of M~^-1: L y = e_r, then L^T x = y
  float col[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float yi = 0.f;
    if (me && i < n) {
      yi = i == r ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < i; ++k) yi -= mt[i * kMaxTreeDof + k] * col[k];
      yi /= mt[i * kMaxTreeDof + i];
    }
    col[i] = yi;
  }
#pragma unroll
  for (int i = 7; i >= 0; --i) {
    if (me && i < n) {
      float xi = col[i];
#pragma unroll
      for (int k = i + 1; k < 8; ++k)
        if (k < n) xi -= mt[k * kMaxTreeDof + i] * col[k];
      col[i] = xi / mt[i * kMaxTreeDof + i];
    }
  }
  __syncwarp();
  if (me)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < n) mt[i * kMaxTreeDof + r] = col[i];
  __syncwarp();
  // smooth velocity v_s = v + dt M~^-1 rhs (row r), then the body twists over the ancestors
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float rk = gshf(rhs, k);
    if (me && k < n) acc += mt[r * kMaxTreeDof + k] * rk;
  }
  const float vs = qd + dt * acc;
  if (me) s.vs[voff] = vs;
  const f3 bom = gsum3(vs * ax, anc);
  const f3 bomp = gsh3(bom, psrc);
  const f3 bvo = gsum3(par >= 0 ? cross(bomp, ro) : mk3(0.f, 0.f, 0.f), anc);
  if (me) {
    st3(s.bom + 3 * b, bom);
    st3(s.bvo + 3 * b, bvo);
  }
}

// trace of the translational point Jacobian of body b at world point p through M~^-1
__device__ float artic_trace(const StepParams& P, const ArticView& s, const DScene& sc, int b, f3 p) {
  const DBody* B = P.bodies + sc.body0;
  const DBody& bd = B[b];
  if (P.trace_mode == 1) return 1.f / bd.mass;
  const DTree& tr = P.trees[sc.tree0 + bd.tree];
  if (tr.free) {
    M33 R = ld33(s.bR + 9 * b);
    f3 r = p - ld3(s.bx + 3 * b);
    f3 l = mulT(R, r);
    float i0 = 1.f / bd.inertia[0], i1 = 1.f / bd.inertia[1], i2 = 1.f / bd.inertia[2];
    return 3.f / bd.mass + dot(r, r) * (i0 + i1 + i2) - (l.x * l.x * i0 + l.y * l.y * i1 + l.z * l.z * i2);
  }
  // hinge chain: sum over the chain's joints i, j of (M~^-1)_ij (a_i x (p - o_i)) . (a_j x (p - o_j)),
  // the chain read from the body's ancestor mask (no local arrays, no parent-pointer chasing);
  // M~^-1 is symmetric, so the pairs j > i count twice and j < i are skipped
  const float* mi = s.minv + (size_t)bd.tree * kMaxTreeDof * kMaxTreeDof;
  float t = 0.f;
  for (unsigned mi_ = (unsigned)bd.anc; mi_; mi_ &= mi_ - 1) {
    const int i = __ffs(mi_) - 1, bi = tr.body0 + i;
    const f3 ci = cross(ld3(s.bax + 3 * bi), p - ld3(s.bx + 3 * bi));
    f3 acc = (0.5f * mi[i * kMaxTreeDof + i]) * ci;
    for (unsigned mj = mi_ & (mi_ - 1); mj; mj &= mj - 1) {
      const int j = __ffs(mj) - 1, bj = tr.body0 + j;
      acc = acc + mi[i * kMaxTreeDof + j] * cross(ld3(s.bax + 3 * bj), p - ld3(s.bx + 3 * bj));
    }
    t += 2.f * dot(ci, acc);
  }
  return t;
}

__device__ void artic_apply(const StepParams& P, ArticView& s, const DScene& sc, int b, f3 p, f3 f, f3 m) {
  const DBody* B = P.bodies + sc.body0;
  const DBody& bd = B[b];
  const DTree& tr = P.trees[sc.tree0 + bd.tree];
  if (tr.free) {
    M33 R = ld33(s.bR + 9 * b);
    f3 ang = mulT(R, cross(p - ld3(s.bx + 3 * b), f) + m);
    unsigned long long* a = s.acc + bd.voff;
    atomicAdd(a + 0, to_fix(f.x)); atomicAdd(a + 1, to_fix(f.y)); atomicAdd(a + 2, to_fix(f.z));
    atomicAdd(a + 3, to_fix(ang.x)); atomicAdd(a + 4, to_fix(ang.y)); atomicAdd(a + 5, to_fix(ang.z));
    return;
  }
  for (unsigned mk = (unsigned)bd.anc; mk; mk &= mk - 1) {  // the chain's joints
    const int i = __ffs(mk) - 1, a = tr.body0 + i;
    const float gen = dot(ld3(s.bax + 3 * a), cross(p - ld3(s.bx + 3 * a), f) + m);
    atomicAdd(s.acc + tr.voff + i, to_fix(gen));
  }
}

// Gram matrix of a contact's six basis rows through M~^-1 (exact diagonal impedance): free
// bodies in closed form; hinge chains through their joint-space rows and the tree's explicit
// M~^-1, with the rows of two bodies of one tree combined first (J = J_A - J_B).
__device__ __noinline__ void artic_gram(const StepParams& P, const ArticView& s, const DScene& sc, int ba, int bb,
                                        f3 p, f3 n, f3 t1, f3 t2, Gram& g) {
  const DBody* B = P.bodies + sc.body0;
  float G[2][6][kMaxTreeDof];
  int gtree[2] = {-1, -1}, gnv[2] = {0, 0};
  int ng = 0;
  gram_zero(g);
  for (int side = 0; side < 2; ++side) {
    const int b = side ? bb : ba;
    if (b < 0) continue;
    const float sg = side ? -1.f : 1.f;
    const DBody& bd = B[b];
    const DTree& tr = P.trees[sc.tree0 + bd.tree];
    if (tr.free) {
      gram_add_free(g, 1.f / bd.mass, mk3(1.f / bd.inertia[0], 1.f / bd.inertia[1], 1.f / bd.inertia[2]),
                    ld33(s.bR + 9 * b), p - ld3(s.bx + 3 * b), n, t1, t2);
      continue;
    }
    int slot = (ng > 0 && gtree[0] == bd.tree) ? 0 : ng;
    if (slot == ng) {
      gtree[slot] = bd.tree; gnv[slot] = tr.nv;
      for (int x = 0; x < 6; ++x)
        for (int i = 0; i < kMaxTreeDof; ++i) G[slot][x][i] = 0.f;
      ++ng;
    }
    for (int a = b; a >= 0; a = B[a].parent) {
      const int k = B[a].voff - tr.voff;
      const f3 ax = ld3(s.bax + 3 * a);
      const f3 lin = cross(ax, p - ld3(s.bx + 3 * a));  // point velocity per unit joint rate
      G[slot][0][k] += sg * dot(n, lin); G[slot][1][k] += sg * dot(t1, lin); G[slot][2][k] += sg * dot(t2, lin);
      G[slot][3][k] += sg * dot(n, ax); G[slot][4][k] += sg * dot(t1, ax); G[slot][5][k] += sg * dot(t2, ax);
    }
  }
  for (int slot = 0; slot < ng; ++slot) {
    const float* mi = s.minv + (size_t)gtree[slot] * kMaxTreeDof * kMaxTreeDof;
    const int nv = gnv[slot];
    float H[6][kMaxTreeDof];  // M~^-1 G_y
    for (int y = 0; y < 6; ++y)
      for (int i = 0; i < nv; ++i) {
        float acc = 0.f;
        for (int j = 0; j < nv; ++j) acc += mi[i * kMaxTreeDof + j] * G[slot][y][j];
        H[y][i] = acc;
      }
    auto q = [&](int x, int y) {
      float acc = 0.f;
      for (int i = 0; i < nv; ++i) acc += G[slot][x][i] * H[y][i];
      return acc;
    };
    g.nn += q(0, 0); g.n1 += q(0, 1); g.n2 += q(0, 2); g.t11 += q(1, 1); g.t12 += q(1, 2); g.t22 += q(2, 2);
    g.n3 += q(0, 3); g.r33 += q(3, 3);
    g.n4 += q(0, 4); g.n5 += q(0, 5); g.r44 += q(4, 4); g.r45 += q(4, 5); g.r55 += q(5, 5);
  }
}

template <int kExt>
__device__ __noinline__ void artic_contact(const StepParams& P, ArticView& s, const DScene& sc, int world,
                                           const float* cq, int slot) {
  Raw k;
  k.p = mk3(cq[slot], cq[kQueue + slot], cq[2 * kQueue + slot]);
  k.n = mk3(cq[3 * kQueue + slot], cq[4 * kQueue + slot], cq[5 * kQueue + slot]);
  k.phi = cq[6 * kQueue + slot];
  const int code = __float_as_int(cq[7 * kQueue + slot]), sub = __float_as_int(cq[8 * kQueue + slot]);
  const int ga = code >> 16, gb = code & 0xffff;
  const DGeom& GA = P.geoms[sc.geom0 + ga];
  const DGeom& GB = P.geoms[sc.geom0 + gb];
  const bool plane = GB.type == CF_GEOM_PLANE;
  const f3 px = plane ? mk3(s.gR[9 * gb], s.gR[9 * gb + 3], s.gR[9 * gb + 6]) : mk3(0.f, 0.f, 0.f);
  const int ba = GA.body, bb = GB.body;
  f3 t1, t2;
  contact_frame(k.n, plane, px, t1, t2);
  f3 oma = ld3(s.bom + 3 * ba);
  f3 vc = ld3(s.bvo + 3 * ba) + cross(oma, k.p - ld3(s.bx + 3 * ba));
  f3 wc = oma;
  float tr = artic_trace(P, s, sc, ba, k.p);
  if (bb >= 0) {
    f3 omb = ld3(s.bom + 3 * bb);
    vc = vc - (ld3(s.bvo + 3 * bb) + cross(omb, k.p - ld3(s.bx + 3 * bb)));
    wc = wc - omb;
    tr += artic_trace(P, s, sc, bb, k.p);
  }
  float mphi = 0.f, target = 0.f;
  float w[6];
  const float mu_t = fmaxf(GA.mu[0], GB.mu[0]), mu_tor = fmaxf(GA.mu[1], GB.mu[1]), mu_rol = fmaxf(GA.mu[2], GB.mu[2]);
  ImpFeat feat;
  const bool imp = (kExt & kExtImp) && P.trace_mode >= 2;  // exact or learned impedance
  if (imp) {
    const DBody* B = P.bodies + sc.body0;
    auto side = [&](int b) {  // the link taken as a free body about its centre of mass
      const DBody& bd = B[b];
      const M33 R = ld33(s.bR + 9 * b);
      const f3 com = ld3(s.bx + 3 * b) + mul(R, mk3(bd.ipos[0], bd.ipos[1], bd.ipos[2]));
      return free_normal_inverse_mass(1.f / bd.mass, mk3(1.f / bd.inertia[0], 1.f / bd.inertia[1], 1.f / bd.inertia[2]),
                                      R, k.p - com, k.n);
    };
    const float im_sum = 1.f / B[ba].mass + (bb >= 0 ? 1.f / B[bb].mass : 0.f);
    const float w_n = side(ba) + (bb >= 0 ? side(bb) : 0.f);
    feat = impnet_features(P, k.phi, tr, im_sum, w_n, bb < 0);
  }
  if ((kExt & kExtImp) && P.trace_mode == 2) {
    Gram g;
    artic_gram(P, s, sc, ba, bb, k.p, k.n, t1, t2, g);
    facet_impulses_exact(P, dot(k.n, vc), dot(t1, vc), dot(t2, vc), dot(k.n, wc), dot(t1, wc), dot(t2, wc), k.phi,
                         mu_t, mu_tor, mu_rol, g, w);
    if (P.capture_cap > 0) {  // the learned impedance's target: ln(mean exact impedance / M(phi))
      const float r = solimp_r(P, fabsf(k.phi));
      target = logf(facet_mean_exact_impedance(P, mu_t, mu_tor, mu_rol, g) * (1.f - r) * tr / r);
    }
  } else {
    float r = solimp_r(P, fabsf(k.phi));
    mphi = __fdividef(r, (1.f - r) * tr);
    if ((kExt & kExtImp) && P.trace_mode == 3) mphi *= impnet_scale(P.impnet + (size_t)world * P.impnet_stride, feat);
    facet_impulses(P, dot(k.n, vc), dot(t1, vc), dot(t2, vc), dot(k.n, wc), dot(t1, wc), dot(t2, wc), k.phi,
                   P.k_user * mphi, P.d_user * mphi, mu_t, mu_tor, mu_rol, w);
  }
  f3 f = w[0] * k.n + w[1] * t1 + w[2] * t2;
  f3 m = w[3] * k.n + w[4] * t1 + w[5] * t2;
  artic_apply(P, s, sc, ba, k.p, f, m);
  if (bb >= 0) artic_apply(P, s, sc, bb, k.p, -f, -m);
  atomicAdd(s.count, 1);
  if (P.capture_cap > 0)
    capture_contact(P, world, s.count, sc.geom0 + ga, sc.geom0 + gb, sub, k.phi, k.p, k.n, w[0], mphi,
                    imp ? feat.x[1] : 0.f, imp ? feat.x[2] : 0.f, target, bb < 0);
}

// Joint limits and dry joint friction of one hinge tree (Sec. III-A's system model), closed
// form from the smooth prediction like the contacts: a limit is a one-row frictionless
// constraint J = +-e_k with gap q - lower or upper - q under the facet impulse law, its trace
// (M~^-1)_kk; dry friction applies the impulse that alone stops the predicted joint velocity,
// clamped to +-frictionloss dt.
__device__ void artic_joint_constraints(const StepParams& P, ArticView& s, const DScene& sc, const DTree& tr, int t) {
  if (tr.free) return;
  const DBody* B = P.bodies + sc.body0;
  const float* mi = s.minv + (size_t)t * kMaxTreeDof * kMaxTreeDof;
  for (int j = 0; j < tr.nbody; ++j) {
    const DBody& bd = B[tr.body0 + j];
    if (!bd.limited && !(bd.frictionloss > 0.f)) continue;
    const int k = bd.voff - tr.voff;
    const float wkk = mi[k * kMaxTreeDof + k];
    const float vsk = s.vs[bd.voff];
    float pk = 0.f;
    if (bd.limited) {
      const float q = s.q[bd.qoff];
      for (int side = 0; side < 2; ++side) {
        const float gap = side ? bd.range[1] - q : q - bd.range[0];
        if (!(gap < P.margin)) continue;
        const float sg = side ? -1.f : 1.f;
        const float sv = sg * vsk;
        float Mk;
        if (P.trace_mode == 2) {
          Mk = 1.f / (fmaf(P.k_user, P.dt, P.d_user) * wkk);
        } else {
          const float r = solimp_r(P, fabsf(gap));
          Mk = r / ((1.f - r) * wkk);
        }
        const float lam = -P.k_user * Mk * fmaf(sv, P.dt, gap) - P.d_user * Mk * sv;
        if (lam > 0.f) pk += sg * lam;
      }
    }
    if (bd.frictionloss > 0.f) {
      const float cap = bd.frictionloss * P.dt;
      pk += fminf(fmaxf(-vsk / wkk, -cap), cap);
    }
    atomicAdd(s.acc + bd.voff, to_fix(pk));
  }
}

// number of sub-contacts a candidate pair can produce: a plane against a capsule's end spheres,
// a box's corners or a cylinder's rim points; box-box clipped vertices; otherwise one
template <int kExt>
__device__ __forceinline__ int artic_nsub(const DGeom* G, int code) {
  if (code < 0) return 0;
  int ta = G[code >> 16].type, tb = G[code & 0xffff].type;
  if (ta == CF_GEOM_PLANE) { const int t = ta; ta = tb; tb = t; }
  if (tb == CF_GEOM_PLANE) {
    if (ta == CF_GEOM_CAPSULE) return 2;
    if (ta == CF_GEOM_BOX) return 8;
    if ((kExt & kExtGeo) && ta == CF_GEOM_CYLINDER) return 6;
    return 1;
  }
  return (kExt & kExtGeo) && ta == CF_GEOM_BOX && tb == CF_GEOM_BOX ? 8 : 1;
}

// narrowphase of sub-contact `sub` of one scene pair, oriented so that a plane is always B;
// (ga, gb) receive the oriented pair.  True when it is a contact.
template <int kExt>
__device__ bool artic_narrow(const StepParams& P, const ArticView& s, const DScene& sc, int code, int sub, Raw& k,
                             int& ga, int& gb) {
  ga = code >> 16;
  gb = code & 0xffff;
  const DGeom* G = P.geoms + sc.geom0;
  int ta = G[ga].type, tb = G[gb].type;
  if (ta == CF_GEOM_PLANE) { int t = ga; ga = gb; gb = t; t = ta; ta = tb; tb = t; }
  f3 ca = ld3(s.gc + 3 * ga), cb = ld3(s.gc + 3 * gb);
  M33 Ra = ld33(s.gR + 9 * ga), Rb = ld33(s.gR + 9 * gb);
  const float* sa = G[ga].size;
  const float* sb = G[gb].size;
  k.phi = 3.0e38f;
  if (tb == CF_GEOM_PLANE) {
    f3 nz = col(Rb, 2);
    if (ta == CF_GEOM_SPHERE) {
      k = nf_sphere_plane(ca, sa[0], cb, nz);
    } else if (ta == CF_GEOM_CAPSULE) {
      k = nf_sphere_plane(ca + (sub ? sa[1] : -sa[1]) * col(Ra, 2), sa[0], cb, nz);
    } else if ((kExt & kExtGeo) && ta == CF_GEOM_CYLINDER) {
      k = nf_cylinder_plane(ca, Ra, sa[0], sa[1], cb, nz, sub);
    } else if ((kExt & kExtGeo) && ta == CF_GEOM_ELLIPSOID) {
      k = nf_ellipsoid_plane(ca, Ra, mk3(sa[0], sa[1], sa[2]), cb, nz);
    } else if (ta == CF_GEOM_BOX) {
      f3 corner = ca + mul(Ra, mk3((sub & 4) ? sa[0] : -sa[0], (sub & 2) ? sa[1] : -sa[1], (sub & 1) ? sa[2] : -sa[2]));
      k = nf_sphere_plane(corner, 0.f, cb, nz);
    }
    return k.phi < P.margin;
  }
  if ((kExt & kExtGeo) && (ta >= CF_GEOM_CYLINDER || tb >= CF_GEOM_CYLINDER)) {  // cylinders touch spheres only
    if (ta == CF_GEOM_SPHERE && tb == CF_GEOM_CYLINDER) k = nf_sphere_cylinder(ca, sa[0], cb, Rb, sb[0], sb[1], true);
    else if (ta == CF_GEOM_CYLINDER && tb == CF_GEOM_SPHERE) k = nf_sphere_cylinder(cb, sb[0], ca, Ra, sa[0], sa[1], false);
  } else if (ta == CF_GEOM_SPHERE && tb == CF_GEOM_SPHERE) {
    k = nf_sphere_sphere(ca, sa[0], cb, sb[0]);
  } else if (ta == CF_GEOM_CAPSULE && tb == CF_GEOM_CAPSULE) {
    f3 ua = col(Ra, 2), ub = col(Rb, 2);
    f3 p1 = ca - sa[1] * ua, q1 = ca + sa[1] * ua, p2 = cb - sb[1] * ub, q2 = cb + sb[1] * ub;
    float ss, tt;
    nf_segments(p1, q1, p2, q2, ss, tt);
    k = nf_sphere_sphere(p1 + ss * (q1 - p1), sa[0], p2 + tt * (q2 - p2), sb[0]);
  } else if (ta == CF_GEOM_CAPSULE && tb == CF_GEOM_SPHERE) {
    f3 u = col(Ra, 2);
    float t = fminf(fmaxf(dot(cb - ca, u), -sa[1]), sa[1]);
    k = nf_sphere_sphere(ca + t * u, sa[0], cb, sb[0]);
  } else if (ta == CF_GEOM_SPHERE && tb == CF_GEOM_CAPSULE) {
    f3 u = col(Rb, 2);
    float t = fminf(fmaxf(dot(ca - cb, u), -sb[1]), sb[1]);
    k = nf_sphere_sphere(ca, sa[0], cb + t * u, sb[0]);
  } else if (ta == CF_GEOM_BOX || tb == CF_GEOM_BOX) {
    if (ta == CF_GEOM_BOX && tb == CF_GEOM_BOX) {  // clipped face vertex `sub`
      if (kExt & kExtGeo) k = nf_box_box(ca, Ra, mk3(sa[0], sa[1], sa[2]), cb, Rb, mk3(sb[0], sb[1], sb[2]), sub);
      return k.phi < P.margin;
    }
    bool boxA = ta == CF_GEOM_BOX;
    const M33& Rbx = boxA ? Ra : Rb;
    f3 cbx = boxA ? ca : cb, co = boxA ? cb : ca;
    const float* bs = boxA ? sa : sb;
    const float* os = boxA ? sb : sa;
    int to = boxA ? tb : ta;
    f3 hs = mk3(bs[0], bs[1], bs[2]);
    if (to == CF_GEOM_SPHERE) {
      k = nf_sphere_box(co, os[0], cbx, Rbx, hs, !boxA);
    } else {
      f3 u = col(boxA ? Rb : Ra, 2);
      float t = nf_capsule_box_param(mulT(Rbx, co - cbx), mulT(Rbx, u), os[1], hs);
      k = nf_sphere_box(co + t * u, os[0], cbx, Rbx, hs, !boxA);
    }
  }
  return k.phi < P.margin;
}

// MPC running cost of the state at the start of a step (Sec. V, Eq. mpc cost terms): object
// orientation error 1 - (q*^T q)^2, absolute position errors, squared distances from the object
// to the fingertips (the +z ends of the capsules of leaf bodies), squared deviation of the
// hinges from the home pose, and a penalty once the object leaves the fall radius.
__device__ float artic_running_cost(const StepParams& P, const ArticView& s, const DScene& sc, const DWorld& W,
                                    int world, int lane) {
  // one warp: lanes take the fingertip geoms and the hinges, then a butterfly sum
  const DBody* B = P.bodies + sc.body0;
  const DGeom* G = P.geoms + sc.geom0;
  const float* gl = P.goal + 7 * world;
  const float* qo = s.q + B[P.cost_body].qoff;
  const f3 po = mk3(qo[0], qo[1], qo[2]);
  float part = 0.f;
  for (int g = lane; g < sc.ngeom; g += 32) {
    if (!G[g].tip) continue;
    const f3 tip = ld3(s.gc + 3 * g) + G[g].size[1] * mk3(s.gR[9 * g + 2], s.gR[9 * g + 5], s.gR[9 * g + 8]);
    const f3 d = po - tip;
    part += P.cw[2] * dot(d, d);
  }
  for (int b = lane; b < sc.nbody; b += 32)
    if (B[b].jnt == CF_JOINT_HINGE) {
      const float e = s.q[B[b].qoff] - P.qref[W.qadr + B[b].qoff];
      part += P.cw[3] * e * e;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const float dq = gl[3] * qo[3] + gl[4] * qo[4] + gl[5] * qo[5] + gl[6] * qo[6];
  float c = P.cw[0] * (1.f - dq * dq);
  c += P.cw[1] * (fabsf(qo[0] - gl[0]) + fabsf(qo[1] - gl[1]) + fabsf(qo[2] - gl[2]));
  c += part;
  const float rx = qo[0] - gl[0], ry = qo[1] - gl[1];
  if (rx * rx + ry * ry > P.cw[5] * P.cw[5]) c += P.cw[4];
  return c;
}

template <int kExt>
__device__ void artic_world(const StepParams& P, float* smem, int world, int gid, int gwarps) {
  const DWorld W = P.worlds[world];
  const DScene sc = P.scenes[W.scene];
  const int T = gwarps * 32;
  const int tid = threadIdx.x - gid * T;
  const int lane = threadIdx.x & 31, wig = tid >> 5;
  ArticView s = artic_view(smem, sc, gwarps);
  const DBody* B = P.bodies + sc.body0;
  const DGeom* G = P.geoms + sc.geom0;
  for (int i = tid; i < sc.nq; i += T) s.q[i] = P.q[W.qadr + i];
  for (int i = tid; i < sc.nv; i += T) s.v[i] = P.v[W.vadr + i];
  int* queue = s.queue + wig * kQueue;
  const float dt = P.dt;
  float cost_acc = 0.f;
  // the first step's actuator torques in shared memory (each later step's are staged at the end
  // of the step before), so that the trees' serial chains read no global memory for them
  for (int k = tid; k < sc.nu; k += T) s.tau[k] = ctrl_at(P, 0, W.uadr, k);

  for (int step = 0; step < P.nsteps; ++step) {
    group_sync(gid, T);
    // hinge trees by 8-lane groups (every thread of the world steps through the same loop, so
    // that each warp's shuffles see all its lanes), then free bodies by their group's lane 0
    for (int t0 = 0; t0 < sc.ntree; t0 += T / 8) {
      const int t = t0 + tid / 8;
      const bool hinge = t < sc.ntree && !P.trees[sc.tree0 + t].free;
      artic_tree_prepare_group(P, s, sc, t, hinge, tid & 7);
      if (t < sc.ntree && !hinge && (tid & 7) == 0) artic_free_prepare(P, s, sc, P.trees[sc.tree0 + t]);
    }
    for (int i = tid; i < sc.nv; i += T) s.acc[i] = 0ull;
    if (tid == 0) { s.count[0] = 0; s.count[1] = 0; }
    group_sync(gid, T);
    for (int g = tid; g < sc.ngeom; g += T) {
      const DGeom& gd = G[g];
      M33 Rl = quat_mat(gd.quat[0], gd.quat[1], gd.quat[2], gd.quat[3]);
      f3 c;
      M33 R;
      if (gd.body >= 0) {
        M33 Rb = ld33(s.bR + 9 * gd.body);
        c = ld3(s.bx + 3 * gd.body) + mul(Rb, mk3(gd.pos[0], gd.pos[1], gd.pos[2]));
        R = mul33(Rb, Rl);
      } else {
        c = mk3(gd.pos[0], gd.pos[1], gd.pos[2]);
        R = Rl;
      }
      st3(s.gc + 3 * g, c);
#pragma unroll
      for (int k = 0; k < 9; ++k) s.gR[9 * g + k] = R.m[k];
      s.gb[g] = gd.type == CF_GEOM_SPHERE ? gd.size[0]
                : gd.type == CF_GEOM_CAPSULE ? gd.size[0] + gd.size[1]
                : gd.type == CF_GEOM_CYLINDER ? sqrtf(gd.size[0] * gd.size[0] + gd.size[1] * gd.size[1])
                : gd.type == CF_GEOM_ELLIPSOID ? fmaxf(gd.size[0], fmaxf(gd.size[1], gd.size[2]))
                : sqrtf(gd.size[0] * gd.size[0] + gd.size[1] * gd.size[1] + gd.size[2] * gd.size[2]);
    }
    group_sync(gid, T);
    if (P.cost && wig == 0) {
      const float c = artic_running_cost(P, s, sc, W, world, lane);
      if (lane == 0) cost_acc += c;
    }
    // ---- B. pair loop: bounding-sphere tests compacted into the candidate queue; every 32
    // candidates run the narrowphase one per lane and sub-contact by sub-contact, whose hits
    // are compacted into the contact queue; every 32 contacts are solved one per lane ----
    {
      const unsigned lt = (1u << lane) - 1u;
      float* cq = s.cq + wig * kQueue * kArtCq;
      int qn = 0, cn = 0;
      int base = wig * 32;
      while (true) {
        if (qn < 32 && base < sc.npair) {
          const int k = base + lane;
          int code = -1;
          if (k < sc.npair) {
            uint32_t pr = P.pairs[sc.pair0 + k];
            int ga = pr >> 16, gb = pr & 0xffff;
            bool pa = G[ga].type == CF_GEOM_PLANE, pb = G[gb].type == CF_GEOM_PLANE;
            if (pa || pb) {
              int gp = pa ? ga : gb, go = pa ? gb : ga;
              f3 nz = mk3(s.gR[9 * gp + 2], s.gR[9 * gp + 5], s.gR[9 * gp + 8]);
              float d = dot(nz, ld3(s.gc + 3 * go) - ld3(s.gc + 3 * gp));
              if (d < s.gb[go] + P.margin) code = (int)pr;
            } else {
              f3 d = ld3(s.gc + 3 * ga) - ld3(s.gc + 3 * gb);
              float rr = s.gb[ga] + s.gb[gb] + P.margin;
              if (dot(d, d) < rr * rr) code = (int)pr;
            }
          }
          __syncwarp();
          const unsigned m = __ballot_sync(0xffffffffu, code >= 0);
          if (code >= 0) queue[qn + __popc(m & lt)] = code;
          qn += __popc(m);
          base += T;
        }
        const bool done = base >= sc.npair;
        if (qn < 32 && !done) continue;
        const int nb = min(qn, 32);
        const bool last = done && qn <= 32;
        __syncwarp();
        const int mine = lane < nb ? queue[qn - nb + lane] : -1;
        qn -= nb;
        const int my_nsub = artic_nsub<kExt>(G, mine);
        const int nsub = max(__reduce_max_sync(0xffffffffu, my_nsub), 1);
        for (int sub = 0; sub < nsub; ++sub) {
          Raw kc;
          int ga = 0, gb = 0;
          const bool hit = sub < my_nsub && artic_narrow<kExt>(P, s, sc, mine, sub, kc, ga, gb);
          const unsigned hm = __ballot_sync(0xffffffffu, hit);
          if (hit) {
            const int slot = cn + __popc(hm & lt);
            cq[slot] = kc.p.x; cq[kQueue + slot] = kc.p.y; cq[2 * kQueue + slot] = kc.p.z;
            cq[3 * kQueue + slot] = kc.n.x; cq[4 * kQueue + slot] = kc.n.y; cq[5 * kQueue + slot] = kc.n.z;
            cq[6 * kQueue + slot] = kc.phi;
            cq[7 * kQueue + slot] = __int_as_float((ga << 16) | gb);
            cq[8 * kQueue + slot] = __int_as_float(sub);
          }
          cn += __popc(hm);
          const bool flush = last && sub + 1 == nsub;
          while (cn >= 32 || (flush && cn > 0)) {
            __syncwarp();
            const int ns = min(cn, 32);
            if (lane < ns) artic_contact<kExt>(P, s, sc, world, cq, cn - ns + lane);
            cn -= ns;
            __syncwarp();
          }
        }
        if (last) break;
      }
    }
    if (sc.joints)
      for (int t = tid; t < sc.ntree; t += T) artic_joint_constraints(P, s, sc, P.trees[sc.tree0 + t], t);
    group_sync(gid, T);
    // ---- C. correction and integration, per tree ----
    for (int t = tid; t < sc.ntree; t += T) {
      const DTree& tr = P.trees[sc.tree0 + t];
      if (tr.free) {
        const DBody& bd = B[tr.body0];
        float* vb = s.v + bd.voff;
        const float* vsb = s.vs + bd.voff;
        float im = 1.f / bd.mass;
        for (int k = 0; k < 3; ++k) vb[k] = vsb[k] + from_fix(s.acc[bd.voff + k]) * im;
        for (int k = 0; k < 3; ++k) vb[3 + k] = vsb[3 + k] + from_fix(s.acc[bd.voff + 3 + k]) / bd.inertia[k];
        float* qb = s.q + bd.qoff;
        for (int k = 0; k < 3; ++k) qb[k] += vb[k] * dt;
        float w0 = vb[3], w1 = vb[4], w2 = vb[5];
        float wn = sqrtf(w0 * w0 + w1 * w1 + w2 * w2);
        float dq0 = 1.f, dq1 = 0.f, dq2 = 0.f, dq3 = 0.f;
        if (wn > 0.f) {
          float sn, cs;
          sincosf(0.5f * wn * dt, &sn, &cs);
          float sc_ = sn / wn;
          dq0 = cs; dq1 = sc_ * w0; dq2 = sc_ * w1; dq3 = sc_ * w2;
        }
        float a0 = qb[3], a1 = qb[4], a2 = qb[5], a3 = qb[6];
        float n0 = a0 * dq0 - a1 * dq1 - a2 * dq2 - a3 * dq3;
        float n1 = a0 * dq1 + a1 * dq0 + a2 * dq3 - a3 * dq2;
        float n2 = a0 * dq2 - a1 * dq3 + a2 * dq0 + a3 * dq1;
        float n3 = a0 * dq3 + a1 * dq2 - a2 * dq1 + a3 * dq0;
        float inv = rsqrtf(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
        qb[3] = n0 * inv; qb[4] = n1 * inv; qb[5] = n2 * inv; qb[6] = n3 * inv;
      } else {
        const float* mi = s.minv + (size_t)t * kMaxTreeDof * kMaxTreeDof;
        float pv[kMaxTreeDof];
        for (int j = 0; j < tr.nv; ++j) pv[j] = from_fix(s.acc[tr.voff + j]);
        for (int i = 0; i < tr.nv; ++i) {
          float acc = 0.f;
          for (int j = 0; j < tr.nv; ++j) acc += mi[i * kMaxTreeDof + j] * pv[j];
          s.v[tr.voff + i] = s.vs[tr.voff + i] + acc;
        }
        for (int j = 0; j < tr.nbody; ++j) {
          const DBody& bd = B[tr.body0 + j];
          s.q[bd.qoff] += s.v[bd.voff] * dt;
        }
      }
    }
    if (step + 1 < P.nsteps)
      for (int k = tid; k < sc.nu; k += T) s.tau[k] = ctrl_at(P, step + 1, W.uadr, k);
  }
  group_sync(gid, T);
  bool bad = false;
  for (int i = tid; i < sc.nq; i += T) {
    P.q[W.qadr + i] = s.q[i];
    if (!isfinite(s.q[i])) bad = true;
  }
  for (int i = tid; i < sc.nv; i += T) {
    P.v[W.vadr + i] = s.v[i];
    if (!isfinite(s.v[i])) bad = true;
  }
  if (bad) {
    atomicOr(P.flags + world, CF_FLAG_NONFINITE);
    atomicOr(P.errword, CF_FLAG_NONFINITE);
  }
  if (tid == 0) {
    P.ncontact[world] = s.count[0];
    if (P.capture_cap > 0 && s.count[1] > P.capture_cap) {
      atomicOr(P.flags + world, CF_FLAG_CONTACT_OVERFLOW);
      atomicOr(P.errword, CF_FLAG_CONTACT_OVERFLOW);
    }
    if (P.cost) {
      // terminal cost of the final state: phi1 |p - p*|^2 + phi2 (1 - (q*^T q)^2)
      const float* gl = P.goal + 7 * world;
      const float* qo = s.q + P.bodies[sc.body0 + P.cost_body].qoff;
      float dx = qo[0] - gl[0], dy = qo[1] - gl[1], dz = qo[2] - gl[2];
      float dq = gl[3] * qo[3] + gl[4] * qo[4] + gl[5] * qo[5] + gl[6] * qo[6];
      P.cost[world] += cost_acc + P.cw[6] * (dx * dx + dy * dy + dz * dz) + P.cw[7] * (1.f - dq * dq);
    }
  }
}

// =======================================================================================
// persistent kernel: CTAs pull work units (sorted by decreasing cost); a unit holds
// kWarps / warps worlds, one per group of `warps` warps
// =======================================================================================
// kArtic: articulated worlds compiled in; kExt: the optional features compiled in, a mask of
// kExtImp (the exact and learned impedances, trace_mode 2 and 3) and kExtGeo (box-box
// contacts, cylinders, ellipsoids), so that the other instantiations keep their register budget.
template <bool kArtic, int kMinBlocks, int kExt>
__global__ void __launch_bounds__(kBlock, kMinBlocks) step_kernel(StepParams P) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_unit;
  __shared__ int s_world[kWarps];
  const int warp = threadIdx.x >> 5;
  // group_warps > 0: every world takes that many warps, and each warp group pulls its next
  // world as soon as it is done (worlds of one CTA do not wait for each other); otherwise the
  // CTA pulls a unit of worlds and its warp groups take one world each
  const bool grouped = P.group_warps > 0;
  for (;;) {
    int world = -1, gid = 0, warps = 0;
    if (grouped) {
      warps = P.group_warps;
      gid = warp / warps;
      const int tid = threadIdx.x - gid * 32 * warps;
      if (tid == 0) s_world[gid] = atomicAdd(P.queue, 1);
      group_sync(gid, 32 * warps);
      const int k = s_world[gid];
      group_sync(gid, 32 * warps);
      if (k >= P.nunits) break;
      world = P.order[k];
    } else {
      if (threadIdx.x == 0) s_unit = atomicAdd(P.queue, 1);
      __syncthreads();
      const int u = s_unit;
      if (u >= P.nunits) break;
      const DUnit U = P.units[u];
      warps = U.warps;
      gid = warp / warps;
      if (gid < U.count) world = P.order[U.first + gid];
    }
    if (world >= 0) {
      const DScene& sc = P.scenes[P.worlds[world].scene];
      size_t per = sc.pile ? pile_floats(sc.nbody, sc.nplane, warps)
                           : artic_floats(sc.nbody, sc.ngeom, sc.nq, sc.nv, sc.ntree, warps);
      float* base = smem + per * gid;
      if (!kArtic || sc.pile) pile_world<kExt>(P, base, world, gid, warps);
      else artic_world<kExt>(P, base, world, gid, warps);
    }
    if (!grouped) __syncthreads();
  }
  __syncthreads();
  // the last CTA to finish resets the work counters for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    int done = atomicAdd(P.queue + 1, 1);
    if (done == (int)gridDim.x - 1) {
      P.queue[0] = 0;
      P.queue[1] = 0;
      __threadfence();
    }
  }
}

size_t world_smem_bytes(const DScene& s, int warps) {
  size_t f = s.pile ? pile_floats(s.nbody, s.nplane, warps) : artic_floats(s.nbody, s.ngeom, s.nq, s.nv, s.ntree, warps);
  return f * sizeof(float);
}

// kernel variants: pile-only with 2, 3 or 4 resident CTAs per SM (register budget), the mixed
// (articulated) instantiation, the extended one (articulated, every optional feature) and the
// pile-only one with the exact and learned impedances
using StepFn = void (*)(StepParams);
static const StepFn kVariants[kStepVariants] = {step_kernel<false, 2, 0>,
                                                step_kernel<false, 3, 0>,
                                                step_kernel<false, 4, 0>,
                                                step_kernel<true, 2, 0>,
                                                step_kernel<true, 2, kExtImp | kExtGeo>,
                                                step_kernel<false, 2, kExtImp>};
// the opted-in dynamic shared memory of each variant, per device (the attribute is set on the
// current device; 0 = not yet set there)
constexpr int kAttrDevices = 64;
static std::atomic<size_t> g_max_dyn[kAttrDevices][kStepVariants];

static int variant_index(bool artic, int variant) {
  if (variant == kExtVariant) return 4;
  if (variant == kImpVariant) return artic ? 4 : 5;
  return artic ? 3 : (variant < 0 ? 0 : (variant > 2 ? 2 : variant));
}

static cudaError_t ensure_attr(int vi, size_t* out) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kAttrDevices) return cudaErrorInvalidDevice;
  const size_t cached = g_max_dyn[dev][vi].load();
  if (cached) {
    *out = cached;
    return cudaSuccess;
  }
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kVariants[vi]);
  if (e != cudaSuccess) return e;
  size_t dyn = (size_t)optin - fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(kVariants[vi], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  // prefer the largest shared-memory carveout so several CTAs fit per SM
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kVariants[vi], cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  g_max_dyn[dev][vi].store(dyn);
  *out = dyn;
  return cudaSuccess;
}

size_t step_max_dynamic_smem() {
  size_t m = 0;
  for (int i = 0; i < kStepVariants; ++i) {
    size_t d = 0;
    if (ensure_attr(i, &d) != cudaSuccess) return 0;
    m = (m == 0 || d < m) ? d : m;
  }
  return m;
}

cudaError_t launch_step(const StepParams& p, bool artic, int variant, int grid, size_t smem, cudaStream_t stream) {
  int vi = variant_index(artic, variant);
  size_t dyn = 0;
  cudaError_t e = ensure_attr(vi, &dyn);
  if (e != cudaSuccess) return e;
  if (smem > dyn) return cudaErrorInvalidValue;
  kVariants[vi]<<<grid, kBlock, smem, stream>>>(p);
  return cudaGetLastError();
}

int step_max_blocks_per_sm(bool artic, int variant, size_t smem) {
  int vi = variant_index(artic, variant);
  size_t dyn = 0;
  if (ensure_attr(vi, &dyn) != cudaSuccess) return 1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kVariants[vi], kBlock, smem) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace cf
