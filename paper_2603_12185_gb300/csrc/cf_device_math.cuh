// Device math shared by the step and adjoint kernels: vectors, rotations, narrowphase,
// contact frame, the solimp gap scaling and the closed-form facet impulses.
#pragma once
#include <cuda_runtime.h>

#include "cf_internal.cuh"

namespace cf {

struct f3 {
  float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator-(f3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float norm3(f3 a) { return sqrtf(dot(a, a)); }

// 3x3 rotation, row major
struct M33 {
  float m[9];
};
__device__ __forceinline__ f3 mul(const M33& R, f3 v) {
  return {R.m[0] * v.x + R.m[1] * v.y + R.m[2] * v.z, R.m[3] * v.x + R.m[4] * v.y + R.m[5] * v.z,
          R.m[6] * v.x + R.m[7] * v.y + R.m[8] * v.z};
}
__device__ __forceinline__ f3 mulT(const M33& R, f3 v) {
  return {R.m[0] * v.x + R.m[3] * v.y + R.m[6] * v.z, R.m[1] * v.x + R.m[4] * v.y + R.m[7] * v.z,
          R.m[2] * v.x + R.m[5] * v.y + R.m[8] * v.z};
}
__device__ __forceinline__ f3 col(const M33& R, int j) { return {R.m[j], R.m[3 + j], R.m[6 + j]}; }
__device__ __forceinline__ M33 mul33(const M33& a, const M33& b) {
  M33 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      r.m[3 * i + j] = a.m[3 * i] * b.m[j] + a.m[3 * i + 1] * b.m[3 + j] + a.m[3 * i + 2] * b.m[6 + j];
  return r;
}
// rotation matrix of the (re-normalised) quaternion (w, x, y, z)
__device__ __forceinline__ M33 quat_mat(float w, float x, float y, float z) {
  float s = rsqrtf(w * w + x * x + y * y + z * z);
  w *= s; x *= s; y *= s; z *= s;
  M33 r;
  r.m[0] = 1.f - 2.f * (y * y + z * z); r.m[1] = 2.f * (x * y - w * z); r.m[2] = 2.f * (x * z + w * y);
  r.m[3] = 2.f * (x * y + w * z); r.m[4] = 1.f - 2.f * (x * x + z * z); r.m[5] = 2.f * (y * z - w * x);
  r.m[6] = 2.f * (x * z - w * y); r.m[7] = 2.f * (y * z + w * x); r.m[8] = 1.f - 2.f * (x * x + y * y);
  return r;
}
// rotation by angle th about the unit axis a (Rodrigues)
__device__ __forceinline__ M33 axis_rot(f3 a, float th) {
  float s, c;
  sincosf(th, &s, &c);
  float t = 1.f - c;
  M33 r;
  r.m[0] = t * a.x * a.x + c; r.m[1] = t * a.x * a.y - s * a.z; r.m[2] = t * a.x * a.z + s * a.y;
  r.m[3] = t * a.x * a.y + s * a.z; r.m[4] = t * a.y * a.y + c; r.m[5] = t * a.y * a.z - s * a.x;
  r.m[6] = t * a.x * a.z - s * a.y; r.m[7] = t * a.y * a.z + s * a.x; r.m[8] = t * a.z * a.z + c;
  return r;
}

// ---------------------------------------------------------------------------------------
// narrowphase: phi (signed gap), midpoint contact point p, normal n from geom B to geom A
// ---------------------------------------------------------------------------------------
struct Raw {
  float phi;
  f3 p, n;
};

__device__ __forceinline__ Raw nf_sphere_sphere(f3 ca, float ra, f3 cb, float rb) {
  f3 d = ca - cb;
  const float d2 = dot(d, d);
  const float inv = rsqrtf(d2);
  const float dist = d2 > 0.f ? d2 * inv : 0.f;
  f3 n = d2 > 0.f ? inv * d : mk3(0.f, 0.f, 1.f);
  Raw k;
  k.phi = dist - ra - rb;
  k.p = 0.5f * ((ca - ra * n) + (cb + rb * n));
  k.n = n;
  return k;
}

__device__ __forceinline__ Raw nf_sphere_plane(f3 c, float r, f3 o, f3 nz) {
  float dist = dot(nz, c - o);
  Raw k;
  k.phi = dist - r;
  k.p = 0.5f * ((c - r * nz) + (c - dist * nz));
  k.n = nz;
  return k;
}

// closest points of segments [p1,q1], [p2,q2] (parameters s, t in [0,1]); near-parallel
// segments (1 - cos^2 <= 1e-3) take the midpoint of the overlap of 2's projection onto 1.
__device__ __forceinline__ void nf_segments(f3 p1, f3 q1, f3 p2, f3 q2, float& s, float& t) {
  f3 d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
  float a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r), c = dot(d1, r), b = dot(d1, d2);
  float denom = a * e - b * b;
  if (denom > 1e-3f * (a * e)) {
    s = fminf(fmaxf(__fdividef(b * f - c * e, denom), 0.f), 1.f);
    t = __fdividef(b * s + f, e);
    if (t < 0.f) {
      t = 0.f;
      s = fminf(fmaxf(__fdividef(-c, a), 0.f), 1.f);
    } else if (t > 1.f) {
      t = 1.f;
      s = fminf(fmaxf(__fdividef(b - c, a), 0.f), 1.f);
    }
  } else {
    float sp = dot(p2 - p1, d1) / a, sq = dot(q2 - p1, d1) / a;
    float lo = fmaxf(0.f, fminf(sp, sq)), hi = fminf(1.f, fmaxf(sp, sq));
    if (lo <= hi) s = 0.5f * (lo + hi);
    else s = fmaxf(sp, sq) < 0.f ? 0.f : 1.f;
    t = fminf(fmaxf((b * s + f) / e, 0.f), 1.f);
  }
}

// sphere (centre c, radius r) against a box (centre bc, rotation R, half extents hs)
__device__ __forceinline__ Raw nf_sphere_box(f3 c, float r, f3 bc, const M33& R, f3 hs, bool sphere_is_a) {
  f3 l = mulT(R, c - bc);
  float lc[3] = {l.x, l.y, l.z}, h[3] = {hs.x, hs.y, hs.z}, cl[3];
  bool inside = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cl[i] = fminf(fmaxf(lc[i], -h[i]), h[i]);
    if (lc[i] < -h[i] || lc[i] > h[i]) inside = false;
  }
  f3 nb, sbox;
  float dist;
  if (!inside) {
    f3 qb = bc + mul(R, mk3(cl[0], cl[1], cl[2]));
    f3 d = c - qb;
    dist = norm3(d);
    nb = (1.f / dist) * d;
    sbox = qb;
  } else {
    int k = 0;
    float best = h[0] - fabsf(lc[0]);
#pragma unroll
    for (int i = 1; i < 3; ++i) {
      float g = h[i] - fabsf(lc[i]);
      if (g < best) { best = g; k = i; }
    }
    float sg = lc[k] >= 0.f ? 1.f : -1.f;
    nb = sg * col(R, k);
    dist = -best;
    float sl[3] = {lc[0], lc[1], lc[2]};
    sl[k] = sg * h[k];
    sbox = bc + mul(R, mk3(sl[0], sl[1], sl[2]));
  }
  Raw o;
  o.phi = dist - r;
  o.p = 0.5f * ((c - r * nb) + sbox);
  o.n = sphere_is_a ? nb : -nb;
  return o;
}

// argmin over t in [-h, h] of the box SDF at x0 + t w (box coordinates).  Outside the box:
// root of the nondecreasing piecewise-linear derivative of sum_k max(|x_k| - s_k, 0)^2,
// walking the slab breakpoints (a flat stretch takes its midpoint).  Through the box: best of
// the endpoints and the pairwise crossings of the six lines +-x_k(t) - s_k.
__device__ __forceinline__ float box_sdf_along(const float* x0, const float* w, const float* s, float t) {
  float out2 = 0.f, inmax = -3.0e38f;
  bool outside = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float e = fabsf(fmaf(t, w[k], x0[k])) - s[k];
    if (e > 0.f) { outside = true; out2 = fmaf(e, e, out2); }
    inmax = fmaxf(inmax, e);
  }
  return outside ? sqrtf(out2) : inmax;
}
__device__ __forceinline__ float box_dG(const float* x0, const float* w, const float* s, float t) {
  float g = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float xk = fmaf(t, w[k], x0[k]);
    float e = fabsf(xk) - s[k];
    if (e > 0.f) g = fmaf(e, xk >= 0.f ? w[k] : -w[k], g);
  }
  return g;
}
__device__ inline float nf_capsule_box_param(f3 x0v, f3 wv, float h, f3 sv) {
  float x0[3] = {x0v.x, x0v.y, x0v.z}, w[3] = {wv.x, wv.y, wv.z}, s[3] = {sv.x, sv.y, sv.z};
  float lo = -h, hi = h;
  bool hits = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (!hits) break;
    if (w[k] == 0.f) {
      if (fabsf(x0[k]) > s[k]) hits = false;
    } else {
      float ta = (-s[k] - x0[k]) / w[k], tb = (s[k] - x0[k]) / w[k];
      if (ta > tb) { float tt = ta; ta = tb; tb = tt; }
      lo = fmaxf(lo, ta);
      hi = fminf(hi, tb);
      if (lo > hi) hits = false;
    }
  }
  if (!hits) {
    if (box_dG(x0, w, s, -h) >= 0.f) return -h;
    if (box_dG(x0, w, s, h) <= 0.f) return h;
    float bp[8];
    int nb = 0;
    bp[nb++] = -h;
    bp[nb++] = h;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (w[k] != 0.f)
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
          float tb = ((float)sg * s[k] - x0[k]) / w[k];
          if (tb > -h && tb < h) bp[nb++] = tb;
        }
    for (int i = 1; i < nb; ++i) {  // insertion sort (<= 8 values)
      float v = bp[i];
      int j = i - 1;
      while (j >= 0 && bp[j] > v) { bp[j + 1] = bp[j]; --j; }
      bp[j + 1] = v;
    }
    for (int i = 0; i + 1 < nb; ++i) {
      float ta = bp[i], tb = bp[i + 1];
      float ga = box_dG(x0, w, s, ta), gb = box_dG(x0, w, s, tb);
      if (ga <= 0.f && gb >= 0.f) {
        if (ga == 0.f && gb == 0.f) return 0.5f * (ta + tb);
        if (ga == 0.f) return ta;
        if (gb == 0.f) return tb;
        float tm = 0.5f * (ta + tb), num = 0.f, den = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float xk = fmaf(tm, w[k], x0[k]);
          if (fabsf(xk) - s[k] > 0.f) {
            float sg = xk >= 0.f ? 1.f : -1.f;
            num = fmaf(w[k], sg * s[k] - x0[k], num);
            den = fmaf(w[k], w[k], den);
          }
        }
        return num / den;
      }
    }
    return 0.f;
  }
  float la[6], lb[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    la[2 * k] = w[k];
    lb[2 * k] = x0[k] - s[k];
    la[2 * k + 1] = -w[k];
    lb[2 * k + 1] = -x0[k] - s[k];
  }
  float best = -h, fbest = box_sdf_along(x0, w, s, -h);
  {
    float fh = box_sdf_along(x0, w, s, h);
    if (fh < fbest) { fbest = fh; best = h; }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      float da = la[i] - la[j];
      if (fabsf(da) > 1e-12f) {
        float tc = (lb[j] - lb[i]) / da;
        if (tc > -h && tc < h) {
          float fc = box_sdf_along(x0, w, s, tc);
          if (fc < fbest || (fc == fbest && tc < best)) { fbest = fc; best = tc; }
        }
      }
    }
  return best;
}

// contact frame: plane contacts use the plane's local x axis as t1; otherwise
// t1 = normalize(e_z x n) when |n_z| < 0.5, else normalize(e_x x n); t2 = n x t1.
__device__ __forceinline__ void contact_frame(f3 n, bool plane, f3 px, f3& t1, f3& t2) {
  if (plane) {
    t1 = px;
  } else {
    f3 c = fabsf(n.z) < 0.5f ? mk3(-n.y, n.x, 0.f) : mk3(0.f, -n.z, n.y);
    t1 = rsqrtf(dot(c, c)) * c;
  }
  t2 = cross(n, t1);
}

// r(|phi|) of Eq. r_scaling, x clamped to [0, 1]; the default power p = 2 is a square
__device__ __forceinline__ float solimp_pow(float y, float p) { return p == 2.f ? y * y : powf(y, p); }
__device__ __forceinline__ float solimp_r(const StepParams& P, float aphi) {
  float x = fminf(fmaxf(__fdividef(aphi, P.solimp[2]), 0.f), 1.f);
  float m = P.solimp[3];
  float g = x < m ? m * solimp_pow(__fdividef(x, m), P.solimp[4])
                  : 1.f - (1.f - m) * solimp_pow(__fdividef(1.f - x, 1.f - m), P.solimp[4]);
  return P.solimp[0] + (P.solimp[1] - P.solimp[0]) * g;
}

// Eight facets at angles j * 45 degrees: lambda_j = max(0, a + c_j b1 + s_j b2); returns
// sum lambda_j, sum c_j lambda_j and sum s_j lambda_j.
__device__ __forceinline__ void octa_facets(float a, float b1, float b2, float h, float& sn, float& s1, float& s2) {
  const float u = h * b1, v = h * b2;
  const float l0 = fmaxf(a + b1, 0.f), l2 = fmaxf(a + b2, 0.f), l4 = fmaxf(a - b1, 0.f), l6 = fmaxf(a - b2, 0.f);
  const float l1 = fmaxf(a + u + v, 0.f), l3 = fmaxf(a - u + v, 0.f), l5 = fmaxf(a - u - v, 0.f),
              l7 = fmaxf(a + u - v, 0.f);
  sn = ((l0 + l4) + (l2 + l6)) + ((l1 + l5) + (l3 + l7));
  s1 = (l0 - l4) + h * ((l1 - l5) + (l7 - l3));
  s2 = (l2 - l6) + h * ((l1 - l5) + (l3 - l7));
}

// Box-box contact `sub` (0..7) of two boxes (centres, rotations, half extents): the
// separating-axis test over the six face axes (A's first; the least overlap wins) picks the
// reference face; the incident box's face most anti-parallel to it is clipped by the reference
// face's side planes (vertices from (+,+) of its in-face axes in cyclic order; planes +k1, -k1,
// +k2, -k2); clipped vertex `sub` gives gap = its distance to the reference plane, point = the
// midpoint with its projection, normal = the reference normal from B to A.  phi = +inf when the
// polygon has fewer vertices.  Crossed edges give no contact.
static __device__ __noinline__ Raw nf_box_box(f3 ca, M33 Ra, f3 ha, f3 cb, M33 Rb, f3 hb, int sub) {
  Raw o;
  o.phi = 3.0e38f;
  o.p = ca;
  o.n = mk3(0.f, 0.f, 1.f);
  const f3 d = cb - ca;
  const float hav[3] = {ha.x, ha.y, ha.z}, hbv[3] = {hb.x, hb.y, hb.z};
  int best = 0;
  float best_sep = 0.f;
  for (int k = 0; k < 6; ++k) {
    const f3 u = k < 3 ? col(Ra, k) : col(Rb, k - 3);
    float ra = 0.f, rb = 0.f;
    for (int i = 0; i < 3; ++i) {
      ra += hav[i] * fabsf(dot(col(Ra, i), u));
      rb += hbv[i] * fabsf(dot(col(Rb, i), u));
    }
    const float sep = fabsf(dot(d, u)) - ra - rb;
    if (k == 0 || sep > best_sep) { best_sep = sep; best = k; }
  }
  const bool refA = best < 3;
  const int jr = best % 3;
  const f3 cR = refA ? ca : cb, cI = refA ? cb : ca;
  const M33 RR = refA ? Ra : Rb, RI = refA ? Rb : Ra;
  const float* hR = refA ? hav : hbv;
  const float* hI = refA ? hbv : hav;
  const f3 nR = (dot(cI - cR, col(RR, jr)) >= 0.f ? 1.f : -1.f) * col(RR, jr);
  int ji = 0;
  float most = 0.f;
  for (int i = 0; i < 3; ++i) {
    const float c = fabsf(dot(col(RI, i), nR));
    if (i == 0 || c > most) { most = c; ji = i; }
  }
  const float si = dot(col(RI, ji), nR) > 0.f ? -1.f : 1.f;
  const int i1 = (ji + 1) % 3, i2 = (ji + 2) % 3;
  const f3 fc = cI + (si * hI[ji]) * col(RI, ji);
  const f3 e1 = hI[i1] * col(RI, i1), e2 = hI[i2] * col(RI, i2);
  f3 poly[8], tmp[8];
  poly[0] = fc + e1 + e2; poly[1] = fc - e1 + e2; poly[2] = fc - e1 - e2; poly[3] = fc + e1 - e2;
  int n = 4;
  const int k1 = (jr + 1) % 3, k2 = (jr + 2) % 3;
  for (int pl = 0; pl < 4 && n > 0; ++pl) {
    const int ax = pl < 2 ? k1 : k2;
    const f3 u = ((pl & 1) ? -1.f : 1.f) * col(RR, ax);
    const float h = hR[ax];
    int m = 0;
    for (int v = 0; v < n; ++v) {
      const f3 P = poly[v], Q = poly[v + 1 < n ? v + 1 : 0];
      const float dP = dot(P - cR, u) - h, dQ = dot(Q - cR, u) - h;
      if (dP <= 0.f && m < 8) tmp[m++] = P;
      if ((dP <= 0.f) != (dQ <= 0.f) && m < 8) tmp[m++] = P + (dP / (dP - dQ)) * (Q - P);
    }
    for (int v = 0; v < m; ++v) poly[v] = tmp[v];
    n = m;
  }
  if (sub < n) {
    const f3 v = poly[sub];
    const float dist = dot(v - cR, nR) - hR[jr];
    o.phi = dist;
    o.p = v - (0.5f * dist) * nR;
    o.n = refA ? -1.f * nR : nR;
  }
  return o;
}

// Ellipsoid (centre c, rotation R, semi-axes e) against a plane (point o, normal n): the
// support point against n, c - R D^2 R^T n / |D R^T n| (D = diag(e)), is the lowest point.
__device__ __forceinline__ Raw nf_ellipsoid_plane(f3 c, const M33& R, f3 e, f3 o, f3 n) {
  const f3 nl = mulT(R, n);
  const f3 dn = mk3(e.x * nl.x, e.y * nl.y, e.z * nl.z);
  const float il = rsqrtf(dot(dn, dn));
  const f3 p = c - mul(R, mk3(e.x * dn.x * il, e.y * dn.y * il, e.z * dn.z * il));
  Raw k;
  k.phi = dot(n, p - o);
  k.p = p - (0.5f * k.phi) * n;
  k.n = n;
  return k;
}

// Cylinder (centre c, rotation R, radius r, half length h along body z) against a plane: rim
// point `sub` = 3 cap + k of the cap at -h (cap 0) or +h (cap 1), at 120 k degrees from the
// rim's lowest direction -(n - (n.u) u)/|.| (the body x axis when the cap is parallel).
__device__ __forceinline__ Raw nf_cylinder_plane(f3 c, const M33& R, float r, float h, f3 o, f3 n, int sub) {
  const f3 u = col(R, 2);
  // -(n - (n.u) u) written as u x (u x n): the direct form cancels in 1 - (n.u)^2 when the
  // cylinder stands nearly upright, which FP32 resolves too coarsely
  f3 w = cross(u, cross(u, n));
  const float wl2 = dot(w, w);
  w = wl2 > 1e-12f ? rsqrtf(wl2) * w : col(R, 0);
  const f3 w2 = cross(u, w);
  const int k = sub % 3;
  const float cs = k == 0 ? 1.f : -0.5f, sn = k == 0 ? 0.f : (k == 1 ? 0.8660254f : -0.8660254f);
  const f3 p = c + (sub >= 3 ? h : -h) * u + (r * cs) * w + (r * sn) * w2;
  Raw o2;
  o2.phi = dot(n, p - o);
  o2.p = p - (0.5f * o2.phi) * n;
  o2.n = n;
  return o2;
}

// Sphere (centre sc, radius rs) against a solid cylinder (centre c, rotation R, radius r, half
// length h): a centre outside meets the closest point; one inside leaves through the nearer of
// the side and the cap.  The normal points from B to A (sphere_is_a: the sphere is A).
__device__ __forceinline__ Raw nf_sphere_cylinder(f3 sc, float rs, f3 c, const M33& R, float r, float h,
                                                  bool sphere_is_a) {
  const f3 u = col(R, 2);
  const f3 rel = sc - c;
  const float t = dot(u, rel);
  const f3 d = rel - t * u;
  const float rho = sqrtf(dot(d, d));
  const f3 dr = rho > 1e-12f ? (1.f / rho) * d : col(R, 0);
  f3 nb, q;
  float dist;
  if (fabsf(t) <= h && rho <= r) {
    const float side = r - rho, cap = h - fabsf(t);
    if (side <= cap) {
      nb = dr;
      dist = -side;
      q = c + t * u + r * dr;
    } else {
      const float sg = t >= 0.f ? 1.f : -1.f;
      nb = sg * u;
      dist = -cap;
      q = c + (sg * h) * u + d;
    }
  } else {
    const float tc = fminf(fmaxf(t, -h), h), rc = fminf(rho, r);
    q = c + tc * u + rc * dr;
    const f3 g = sc - q;
    dist = sqrtf(dot(g, g));
    nb = (1.f / dist) * g;
  }
  Raw k;
  k.phi = dist - rs;
  k.p = 0.5f * ((sc - rs * nb) + q);
  k.n = sphere_is_a ? nb : -1.f * nb;
  return k;
}

// Gram matrix, through M~^-1, of a contact's six basis rows: point velocity along n, t1, t2
// (0..2) and relative angular velocity about n, t1, t2 (3..5) -- the entries the facet rows
// J~_j = J_n - mu d_j^T J_s need for their diagonals w_j = J~_j M~^-1 J~_j^T.
struct Gram {
  float nn, n1, n2, t11, t12, t22;  // translational block
  float n3, r33;                    // torsional
  float n4, n5, r44, r45, r55;      // rolling
};

__device__ __forceinline__ void gram_zero(Gram& g) {
  g.nn = g.n1 = g.n2 = g.t11 = g.t12 = g.t22 = g.n3 = g.r33 = g.n4 = g.n5 = g.r44 = g.r45 = g.r55 = 0.f;
}

// add a free body: inverse mass im, inverse principal inertia ii, rotation R, lever r
__device__ __forceinline__ void gram_add_free(Gram& g, float im, f3 ii, const M33& R, f3 r, f3 n, f3 t1, f3 t2) {
  const f3 a0 = mulT(R, cross(r, n)), a1 = mulT(R, cross(r, t1)), a2 = mulT(R, cross(r, t2));
  const f3 e0 = mulT(R, n), e1 = mulT(R, t1), e2 = mulT(R, t2);
  auto q = [&](f3 x, f3 y) { return x.x * y.x * ii.x + x.y * y.y * ii.y + x.z * y.z * ii.z; };
  g.nn += im + q(a0, a0); g.n1 += q(a0, a1); g.n2 += q(a0, a2);
  g.t11 += im + q(a1, a1); g.t12 += q(a1, a2); g.t22 += im + q(a2, a2);
  g.n3 += q(a0, e0); g.r33 += q(e0, e0);
  g.n4 += q(a0, e1); g.n5 += q(a0, e2); g.r44 += q(e1, e1); g.r45 += q(e1, e2); g.r55 += q(e2, e2);
}

// the diagonal of a facet row n_row - mu (c x + s y) for the Gram entries of its rows:
// nn, (n.x, n.y), (x.x, x.y, y.y)
__device__ __forceinline__ float gram_facet(float nn, float nx, float ny, float xx, float xy, float yy, float mu,
                                            float c, float s) {
  return nn - 2.f * mu * (c * nx + s * ny) + mu * mu * (c * c * xx + 2.f * c * s * xy + s * s * yy);
}

// Facet impulses with the exact diagonal impedance of Sec. III-B: K_j dt + D_j = 1/(dt w_j),
// split between the gap and the velocity term as k : d, i.e. M(phi) replaced per facet by
// M_j = 1 / ((k dt + d) w_j).  Same inputs and output as facet_impulses.
__device__ __forceinline__ void facet_impulses_exact(const StepParams& P, float vn, float vt1, float vt2, float wn,
                                                     float wr1, float wr2, float phi, float mu_t, float mu_tor,
                                                     float mu_rol, const Gram& g, float w[6]) {
  const float kd = fmaf(P.k_user, P.dt, P.d_user);
  const float a = -P.k_user * phi - kd * vn;
  float N = 0.f, F1 = 0.f, F2 = 0.f, T = 0.f, R1 = 0.f, R2 = 0.f;
  for (int j = 0; j < P.n_t; ++j) {
    const float c = P.tcos[j], s = P.tsin[j];
    const float gj = a + kd * mu_t * (c * vt1 + s * vt2);
    if (gj > 0.f) {
      const float lam = gj / (kd * gram_facet(g.nn, g.n1, g.n2, g.t11, g.t12, g.t22, mu_t, c, s));
      N += lam; F1 = fmaf(c, lam, F1); F2 = fmaf(s, lam, F2);
    }
  }
  for (int j = 0; j < P.n_tor; ++j) {
    const float sg = (j & 1) ? -1.f : 1.f;
    const float gj = a + kd * mu_tor * sg * wn;
    if (gj > 0.f) {
      const float lam = gj / (kd * (g.nn - 2.f * mu_tor * sg * g.n3 + mu_tor * mu_tor * g.r33));
      N += lam; T = fmaf(sg, lam, T);
    }
  }
  for (int j = 0; j < P.n_rol; ++j) {
    const float c = P.rcos[j], s = P.rsin[j];
    const float gj = a + kd * mu_rol * (c * wr1 + s * wr2);
    if (gj > 0.f) {
      const float lam = gj / (kd * gram_facet(g.nn, g.n4, g.n5, g.r44, g.r45, g.r55, mu_rol, c, s));
      N += lam; R1 = fmaf(c, lam, R1); R2 = fmaf(s, lam, R2);
    }
  }
  w[0] = N; w[1] = -mu_t * F1; w[2] = -mu_t * F2; w[3] = -mu_tor * T; w[4] = -mu_rol * R1; w[5] = -mu_rol * R2;
}

// Mean over the facets of the exact diagonal impedance M_j = 1 / ((k dt + d) w_j) of Sec. III-B
// (the learned impedance's regression target), from the contact's Gram blocks.
__device__ __forceinline__ float facet_mean_exact_impedance(const StepParams& P, float mu_t, float mu_tor,
                                                            float mu_rol, const Gram& g) {
  const float kd = fmaf(P.k_user, P.dt, P.d_user);
  float sum = 0.f;
  for (int j = 0; j < P.n_t; ++j)
    sum += 1.f / (kd * gram_facet(g.nn, g.n1, g.n2, g.t11, g.t12, g.t22, mu_t, P.tcos[j], P.tsin[j]));
  for (int j = 0; j < P.n_tor; ++j) {
    const float sg = (j & 1) ? -1.f : 1.f;
    sum += 1.f / (kd * (g.nn - 2.f * mu_tor * sg * g.n3 + mu_tor * mu_tor * g.r33));
  }
  for (int j = 0; j < P.n_rol; ++j)
    sum += 1.f / (kd * gram_facet(g.nn, g.n4, g.n5, g.r44, g.r45, g.r55, mu_rol, P.rcos[j], P.rsin[j]));
  const int nf = P.n_t + P.n_tor + P.n_rol;
  return nf ? sum / (float)nf : 0.f;
}

// Learned impedance (Sec. III-B allows K(q), D(q) to be learned): the contact's configuration
// features x = (clamp(phi / solimp width, -1, 1), clamp(1 - 3 (1/m_A + 1/m_B) / (tr_A + tr_B),
// -1, 1), clamp(w_n / (tr_A + tr_B), 0, 4), side B static), tr the mode-0 trace and w_n the
// normal row n^T J M^-1 J^T n with every body taken as a free body.
struct ImpFeat {
  float x[kImpIn];
};
__device__ __forceinline__ ImpFeat impnet_features(const StepParams& P, float phi, float tr, float im_sum, float w_n,
                                                   bool b_static) {
  ImpFeat f;
  f.x[0] = fminf(fmaxf(phi / P.solimp[2], -1.f), 1.f);
  f.x[1] = fminf(fmaxf(1.f - 3.f * im_sum / tr, -1.f), 1.f);
  f.x[2] = fminf(fmaxf(w_n / tr, 0.f), 4.f);
  f.x[3] = b_static ? 1.f : 0.f;
  return f;
}

// 1/m + (l x n)^T I^-1 (l x n) of a free body with orientation R, inverse principal inertia ii
// and lever l from its centre of mass
__device__ __forceinline__ float free_normal_inverse_mass(float im, f3 ii, const M33& R, f3 l, f3 n) {
  const f3 u = mulT(R, cross(l, n));
  return im + u.x * u.x * ii.x + u.y * u.y * ii.y + u.z * u.z * ii.z;
}

// The factor exp(clamp(g(x), -8, 8)) that scales M(phi), g(x) = b2 + sum_h w2_h
// tanh(b1_h + sum_i W1_hi x_i), parameters [W1 (8 x 4, row-major), b1, w2, b2].
__device__ __forceinline__ float impnet_scale(const float* __restrict__ th, const ImpFeat& f) {
  float g = __ldg(th + kImpParams - 1);
#pragma unroll
  for (int h = 0; h < kImpHidden; ++h) {
    float a = __ldg(th + kImpHidden * kImpIn + h);
#pragma unroll
    for (int i = 0; i < kImpIn; ++i) a = fmaf(__ldg(th + h * kImpIn + i), f.x[i], a);
    g = fmaf(__ldg(th + kImpHidden * kImpIn + kImpHidden + h), tanhf(a), g);
  }
  return expf(fminf(fmaxf(g, -kImpClamp), kImpClamp));
}

// Closed-form facet impulses of one contact (Eqs. tilde_defs, cf_wrench with
// K = k M(phi)/dt, D = d M(phi)/dt, impulse lambda dt = (-kM (s dt + phi) - dM s)_+).
// In: the contact-space velocities of the smooth prediction (normal, tangential pair,
// torsion, rolling pair).  Out: the resultant impulse on A in the contact frame
// w = (normal, t1, t2, torsion, rolling t1, rolling t2).
// With a = A - B v_n and the facet velocity s_j = v_n - mu (c_j v_1 + s_j v_2), each facet is
// lambda_j = max(0, a + c_j (B mu v_1) + s_j (B mu v_2)).
__device__ __forceinline__ void facet_impulses(const StepParams& P, float vn, float vt1, float vt2, float wn,
                                               float wr1, float wr2, float phi, float kM, float dM, float mu_t,
                                               float mu_tor, float mu_rol, float w[6]) {
  const float B = fmaf(kM, P.dt, dM);
  const float a = -kM * phi - B * vn;
  float N = 0.f, F1 = 0.f, F2 = 0.f, T = 0.f, R1 = 0.f, R2 = 0.f;
  if (P.n_t == 8 && P.n_tor == 2 && P.n_rol == 8) {
    // the 6D cone with 8 + 2 + 8 facets: directions at multiples of 45 degrees, so the facet
    // sums reduce to signed combinations (h = cos 45 = sin 45)
    const float h = 0.70710678f;
    float sn, s1, s2;
    octa_facets(a, B * mu_t * vt1, B * mu_t * vt2, h, sn, s1, s2);
    N = sn; F1 = -mu_t * s1; F2 = -mu_t * s2;
    const float bt = B * mu_tor * wn;
    const float lp = fmaxf(a + bt, 0.f), lm = fmaxf(a - bt, 0.f);
    N += lp + lm;
    T = -mu_tor * (lp - lm);
    octa_facets(a, B * mu_rol * wr1, B * mu_rol * wr2, h, sn, s1, s2);
    N += sn; R1 = -mu_rol * s1; R2 = -mu_rol * s2;
    w[0] = N; w[1] = F1; w[2] = F2; w[3] = T; w[4] = R1; w[5] = R2;
    return;
  }
  if (P.n_t == 4 && P.n_tor == 0 && P.n_rol == 0) {  // the 4-facet pyramid: directions +-t1, +-t2
    const float b1 = B * mu_t * vt1, b2 = B * mu_t * vt2;
    const float l0 = fmaxf(a + b1, 0.f), l1 = fmaxf(a + b2, 0.f), l2 = fmaxf(a - b1, 0.f), l3 = fmaxf(a - b2, 0.f);
    w[0] = (l0 + l2) + (l1 + l3); w[1] = -mu_t * (l0 - l2); w[2] = -mu_t * (l1 - l3);
    w[3] = 0.f; w[4] = 0.f; w[5] = 0.f;
    return;
  }
  {
    const float b1 = B * mu_t * vt1, b2 = B * mu_t * vt2;
    for (int j = 0; j < P.n_t; ++j) {
      const float c = P.tcos[j], s = P.tsin[j];
      const float lam = fmaxf(fmaf(c, b1, fmaf(s, b2, a)), 0.f);
      N += lam;
      F1 = fmaf(c, lam, F1);
      F2 = fmaf(s, lam, F2);
    }
    F1 *= -mu_t;
    F2 *= -mu_t;
  }
  if (P.n_tor == 2) {
    const float bt = B * mu_tor * wn;
    const float lp = fmaxf(a + bt, 0.f), lm = fmaxf(a - bt, 0.f);
    N += lp + lm;
    T = -mu_tor * (lp - lm);
  }
  {
    const float b1 = B * mu_rol * wr1, b2 = B * mu_rol * wr2;
    for (int j = 0; j < P.n_rol; ++j) {
      const float c = P.rcos[j], s = P.rsin[j];
      const float lam = fmaxf(fmaf(c, b1, fmaf(s, b2, a)), 0.f);
      N += lam;
      R1 = fmaf(c, lam, R1);
      R2 = fmaf(s, lam, R2);
    }
    R1 *= -mu_rol;
    R2 *= -mu_rol;
  }
  w[0] = N; w[1] = F1; w[2] = F2; w[3] = T; w[4] = R1; w[5] = R2;
}

__device__ __forceinline__ unsigned long long to_fix(float x) {
  x = fminf(fmaxf(x, -kFixClamp), kFixClamp);
  return (unsigned long long)__float2ll_rn(x * kFixScale);
}
__device__ __forceinline__ float from_fix(unsigned long long a) {
  return __ll2float_rn((long long)a) * kFixInv;
}

// Two-word fixed point for the pile scatter: x 2^16 = h + f with h = floor(x 2^16) and the
// fraction f in [0, 1) (both exact in FP32); h goes to a signed 32-bit word and round(f 2^20)
// to an unsigned one, by native 32-bit shared atomics.  Integer sums do not depend on the
// order, so the result is deterministic; the quantum is 2^-36 and the sum is exact while
// |sum| < 2^15 and a word receives fewer than 4096 contributions.
__device__ __forceinline__ void fix2_add(int* hi, unsigned* lo, float x) {
  // the caller has checked |x| <= kFix2Range (else it raises CF_FLAG_RANGE and the result is
  // void); the float-to-integer conversions saturate, so no value faults here
  x *= kFix2Hi;
  const float h = floorf(x);
  atomicAdd(hi, __float2int_rz(h));
  atomicAdd(lo, __float2uint_rn((x - h) * kFix2Lo));
}
__device__ __forceinline__ float fix2_get(int hi, unsigned lo) {
  return fmaf((float)hi, kFix2HiInv, (float)lo * kFix2LoInv);
}

}  // namespace cf
