// Adjoint of the ComFree step for articulated scenes (hinge trees and free bodies).
//
// Reverse sweep with checkpoint recomputation:
//   forward:  the step kernel advances the batch T steps, saving the state every `ckpt` steps;
//   backward: per segment (last first) the step kernel recomputes the segment's states, then
//             for each step t (last first) one launch applies the transpose of the step's
//             Jacobian to the adjoint:  a_t = J_t^T a_{t+1},  dL/dtau_t = J_tau,t^T a_{t+1}.
// The vector-Jacobian product is exact: a CTA per world runs the step below in forward-mode
// tangent arithmetic, one lane per input coordinate (q, v, tau of the world), all lanes on the
// same primal path (no divergence), and each lane reduces its Jacobian column against the
// incoming adjoint.  Kinks -- facet activation (.)_+, clamps, branch choices in the narrowphase
// -- take the derivative of the branch the primal state selects, like the oracle's duals.
#include <cstdio>

#include "cf_grad.cuh"

namespace cf {

// ---------------------------------------------------------------------------------------
// scalar types: float and a float tangent pair
// ---------------------------------------------------------------------------------------
struct DF {
  float v, d;
  __device__ DF() : v(0.f), d(0.f) {}
  __device__ DF(float a) : v(a), d(0.f) {}
  __device__ DF(float a, float b) : v(a), d(b) {}
};
__device__ __forceinline__ DF operator+(DF a, DF b) { return DF(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return DF(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.v, -a.d); }
__device__ __forceinline__ DF operator*(DF a, DF b) { return DF(a.v * b.v, fmaf(a.d, b.v, a.v * b.d)); }
__device__ __forceinline__ DF operator/(DF a, DF b) {
  float inv = 1.f / b.v, r = a.v * inv;
  return DF(r, (a.d - r * b.d) * inv);
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { a = a + b; return a; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { a = a - b; return a; }
__device__ __forceinline__ bool operator<(DF a, DF b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(DF a, DF b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(DF a, DF b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(DF a, DF b) { return a.v >= b.v; }
__device__ __forceinline__ float val(DF a) { return a.v; }
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ DF ssqrt(DF a) {
  float s = sqrtf(a.v);
  return DF(s, s > 0.f ? 0.5f * a.d / s : 0.f);
}
__device__ __forceinline__ float ssqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ void ssincos(DF a, DF& sn, DF& cs) {
  float s, c;
  sincosf(a.v, &s, &c);
  sn = DF(s, c * a.d);
  cs = DF(c, -s * a.d);
}
__device__ __forceinline__ void ssincos(float a, float& sn, float& cs) { sincosf(a, &sn, &cs); }
__device__ __forceinline__ DF spow(DF a, float p) {
  float r = powf(a.v, p);
  return DF(r, a.v != 0.f ? p * r / a.v * a.d : 0.f);
}
__device__ __forceinline__ float spow(float a, float p) { return powf(a, p); }
__device__ __forceinline__ DF sexp(DF a) {
  const float e = expf(a.v);
  return DF(e, e * a.d);
}
__device__ __forceinline__ float sexp(float a) { return expf(a); }
__device__ __forceinline__ DF stanh(DF a) {
  const float t = tanhf(a.v);
  return DF(t, (1.f - t * t) * a.d);
}
__device__ __forceinline__ float stanh(float a) { return tanhf(a); }
template <class S> __device__ __forceinline__ S sabs(S a) { return a < S(0.f) ? -a : a; }
template <class S> __device__ __forceinline__ S smax(S a, S b) { return a > b ? a : b; }
template <class S> __device__ __forceinline__ S smin(S a, S b) { return a < b ? a : b; }
template <class S> __device__ __forceinline__ S sclamp(S a, S lo, S hi) { return a < lo ? lo : (a > hi ? hi : a); }

template <class S> struct V3 {
  S x, y, z;
};
template <class S> __device__ __forceinline__ V3<S> v3(S x, S y, S z) { return {x, y, z}; }
template <class S> __device__ __forceinline__ V3<S> v3f(const float* p) { return {S(p[0]), S(p[1]), S(p[2])}; }
template <class S> __device__ __forceinline__ V3<S> operator+(V3<S> a, V3<S> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class S> __device__ __forceinline__ V3<S> operator-(V3<S> a, V3<S> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S> __device__ __forceinline__ V3<S> operator-(V3<S> a) { return {-a.x, -a.y, -a.z}; }
template <class S> __device__ __forceinline__ V3<S> operator*(S s, V3<S> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class S> __device__ __forceinline__ S dot(V3<S> a, V3<S> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> __device__ __forceinline__ V3<S> cross(V3<S> a, V3<S> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class S> __device__ __forceinline__ S comp(V3<S> a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

template <class S> struct M3 {
  S m[9];
};
template <class S> __device__ __forceinline__ V3<S> mul(const M3<S>& R, V3<S> v) {
  return {R.m[0] * v.x + R.m[1] * v.y + R.m[2] * v.z, R.m[3] * v.x + R.m[4] * v.y + R.m[5] * v.z,
          R.m[6] * v.x + R.m[7] * v.y + R.m[8] * v.z};
}
template <class S> __device__ __forceinline__ V3<S> mulT(const M3<S>& R, V3<S> v) {
  return {R.m[0] * v.x + R.m[3] * v.y + R.m[6] * v.z, R.m[1] * v.x + R.m[4] * v.y + R.m[7] * v.z,
          R.m[2] * v.x + R.m[5] * v.y + R.m[8] * v.z};
}
template <class S> __device__ __forceinline__ V3<S> colv(const M3<S>& R, int j) { return {R.m[j], R.m[3 + j], R.m[6 + j]}; }
template <class S> __device__ __forceinline__ M3<S> mul33(const M3<S>& a, const M3<S>& b) {
  M3<S> r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[3 * i + j] = a.m[3 * i] * b.m[j] + a.m[3 * i + 1] * b.m[3 + j] + a.m[3 * i + 2] * b.m[6 + j];
  return r;
}
template <class S> __device__ __forceinline__ M3<S> qmat(S w, S x, S y, S z) {
  S n = ssqrt(w * w + x * x + y * y + z * z);
  S iw = S(1.f) / n;
  w = w * iw; x = x * iw; y = y * iw; z = z * iw;
  M3<S> r;
  S one(1.f), two(2.f);
  r.m[0] = one - two * (y * y + z * z); r.m[1] = two * (x * y - w * z); r.m[2] = two * (x * z + w * y);
  r.m[3] = two * (x * y + w * z); r.m[4] = one - two * (x * x + z * z); r.m[5] = two * (y * z - w * x);
  r.m[6] = two * (x * z - w * y); r.m[7] = two * (y * z + w * x); r.m[8] = one - two * (x * x + y * y);
  return r;
}
template <class S> __device__ __forceinline__ M3<S> arot(V3<S> a, S th) {
  S s, c;
  ssincos(th, s, c);
  S t = S(1.f) - c;
  M3<S> r;
  r.m[0] = t * a.x * a.x + c; r.m[1] = t * a.x * a.y - s * a.z; r.m[2] = t * a.x * a.z + s * a.y;
  r.m[3] = t * a.x * a.y + s * a.z; r.m[4] = t * a.y * a.y + c; r.m[5] = t * a.y * a.z - s * a.x;
  r.m[6] = t * a.x * a.z - s * a.y; r.m[7] = t * a.y * a.z + s * a.x; r.m[8] = t * a.z * a.z + c;
  return r;
}

// ---------------------------------------------------------------------------------------
// narrowphase (same geometry and conventions as the step kernel)
// ---------------------------------------------------------------------------------------
template <class S> struct RawS {
  S phi;
  V3<S> p, n;
};
template <class S> __device__ RawS<S> g_sphere_sphere(V3<S> ca, S ra, V3<S> cb, S rb) {
  V3<S> d = ca - cb;
  S dist = ssqrt(dot(d, d));
  V3<S> n = dist > S(0.f) ? (S(1.f) / dist) * d : v3(S(0.f), S(0.f), S(1.f));
  RawS<S> k;
  k.phi = dist - ra - rb;
  k.p = S(0.5f) * ((ca - ra * n) + (cb + rb * n));
  k.n = n;
  return k;
}
template <class S> __device__ RawS<S> g_sphere_plane(V3<S> c, S r, V3<S> o, V3<S> nz) {
  S dist = dot(nz, c - o);
  RawS<S> k;
  k.phi = dist - r;
  k.p = S(0.5f) * ((c - r * nz) + (c - dist * nz));
  k.n = nz;
  return k;
}
template <class S> __device__ void g_segments(V3<S> p1, V3<S> q1, V3<S> p2, V3<S> q2, S& s, S& t) {
  V3<S> d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
  S a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r), c = dot(d1, r), b = dot(d1, d2);
  S denom = a * e - b * b;
  S zero(0.f), one(1.f);
  if (val(denom) > 1e-3f * val(a * e)) {
    s = sclamp((b * f - c * e) / denom, zero, one);
    t = (b * s + f) / e;
    if (t < zero) { t = zero; s = sclamp(-c / a, zero, one); }
    else if (t > one) { t = one; s = sclamp((b - c) / a, zero, one); }
  } else {
    S sp = dot(p2 - p1, d1) / a, sq = dot(q2 - p1, d1) / a;
    S lo = smax(zero, smin(sp, sq)), hi = smin(one, smax(sp, sq));
    if (lo <= hi) s = S(0.5f) * (lo + hi);
    else s = smax(sp, sq) < zero ? zero : one;
    t = sclamp((b * s + f) / e, zero, one);
  }
}
template <class S> __device__ RawS<S> g_sphere_box(V3<S> c, S r, V3<S> bc, const M3<S>& R, V3<S> hs, bool sphere_is_a) {
  V3<S> l = mulT(R, c - bc);
  S lc[3] = {l.x, l.y, l.z}, h[3] = {hs.x, hs.y, hs.z}, cl[3];
  bool inside = true;
  for (int i = 0; i < 3; ++i) {
    cl[i] = sclamp(lc[i], -h[i], h[i]);
    if (lc[i] < -h[i] || lc[i] > h[i]) inside = false;
  }
  V3<S> nb, sbox;
  S dist;
  if (!inside) {
    V3<S> qb = bc + mul(R, v3(cl[0], cl[1], cl[2]));
    V3<S> d = c - qb;
    dist = ssqrt(dot(d, d));
    nb = (S(1.f) / dist) * d;
    sbox = qb;
  } else {
    int k = 0;
    S best = h[0] - sabs(lc[0]);
    for (int i = 1; i < 3; ++i) {
      S g = h[i] - sabs(lc[i]);
      if (g < best) { best = g; k = i; }
    }
    S sg = lc[k] >= S(0.f) ? S(1.f) : S(-1.f);
    nb = sg * colv(R, k);
    dist = -best;
    S sl[3] = {lc[0], lc[1], lc[2]};
    sl[k] = sg * h[k];
    sbox = bc + mul(R, v3(sl[0], sl[1], sl[2]));
  }
  RawS<S> o;
  o.phi = dist - r;
  o.p = S(0.5f) * ((c - r * nb) + sbox);
  o.n = sphere_is_a ? nb : -nb;
  return o;
}
template <class S> __device__ S g_box_sdf_along(const S* x0, const S* w, const S* s, S t) {
  S out2(0.f), inmax(-3.0e38f);
  bool outside = false;
  for (int k = 0; k < 3; ++k) {
    S e = sabs(x0[k] + t * w[k]) - s[k];
    if (e > S(0.f)) { outside = true; out2 += e * e; }
    inmax = smax(inmax, e);
  }
  return outside ? ssqrt(out2) : inmax;
}
template <class S> __device__ S g_box_dG(const S* x0, const S* w, const S* s, S t) {
  S g(0.f);
  for (int k = 0; k < 3; ++k) {
    S xk = x0[k] + t * w[k];
    S e = sabs(xk) - s[k];
    if (e > S(0.f)) g += e * (xk >= S(0.f) ? w[k] : -w[k]);
  }
  return g;
}
template <class S> __device__ S g_capsule_box_param(V3<S> x0v, V3<S> wv, S h, V3<S> sv) {
  S x0[3] = {x0v.x, x0v.y, x0v.z}, w[3] = {wv.x, wv.y, wv.z}, s[3] = {sv.x, sv.y, sv.z};
  S lo = -h, hi = h;
  bool hits = true;
  for (int k = 0; k < 3 && hits; ++k) {
    if (val(w[k]) == 0.f) {
      if (sabs(x0[k]) > s[k]) hits = false;
    } else {
      S ta = (-s[k] - x0[k]) / w[k], tb = (s[k] - x0[k]) / w[k];
      if (ta > tb) { S tt = ta; ta = tb; tb = tt; }
      lo = smax(lo, ta);
      hi = smin(hi, tb);
      if (lo > hi) hits = false;
    }
  }
  if (!hits) {
    if (g_box_dG(x0, w, s, -h) >= S(0.f)) return -h;
    if (g_box_dG(x0, w, s, h) <= S(0.f)) return h;
    S bp[8];
    int nb = 0;
    bp[nb++] = -h;
    bp[nb++] = h;
    for (int k = 0; k < 3; ++k)
      if (val(w[k]) != 0.f)
        for (int sg = -1; sg <= 1; sg += 2) {
          S tb = (S((float)sg) * s[k] - x0[k]) / w[k];
          if (tb > -h && tb < h) bp[nb++] = tb;
        }
    for (int i = 1; i < nb; ++i) {
      S v = bp[i];
      int j = i - 1;
      while (j >= 0 && bp[j] > v) { bp[j + 1] = bp[j]; --j; }
      bp[j + 1] = v;
    }
    for (int i = 0; i + 1 < nb; ++i) {
      S ta = bp[i], tb = bp[i + 1];
      S ga = g_box_dG(x0, w, s, ta), gb = g_box_dG(x0, w, s, tb);
      if (ga <= S(0.f) && gb >= S(0.f)) {
        if (val(ga) == 0.f && val(gb) == 0.f) return S(0.5f) * (ta + tb);
        if (val(ga) == 0.f) return ta;
        if (val(gb) == 0.f) return tb;
        S tm = S(0.5f) * (ta + tb), num(0.f), den(0.f);
        for (int k = 0; k < 3; ++k) {
          S xk = x0[k] + tm * w[k];
          if (sabs(xk) - s[k] > S(0.f)) {
            S sg = xk >= S(0.f) ? S(1.f) : S(-1.f);
            num += w[k] * (sg * s[k] - x0[k]);
            den += w[k] * w[k];
          }
        }
        return num / den;
      }
    }
    return S(0.f);
  }
  S la[6], lb[6];
  for (int k = 0; k < 3; ++k) {
    la[2 * k] = w[k];
    lb[2 * k] = x0[k] - s[k];
    la[2 * k + 1] = -w[k];
    lb[2 * k + 1] = -x0[k] - s[k];
  }
  S best = -h, fbest = g_box_sdf_along(x0, w, s, -h);
  S fh = g_box_sdf_along(x0, w, s, h);
  if (fh < fbest) { fbest = fh; best = h; }
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      S da = la[i] - la[j];
      if (fabsf(val(da)) > 1e-12f) {
        S tc = (lb[j] - lb[i]) / da;
        if (tc > -h && tc < h) {
          S fc = g_box_sdf_along(x0, w, s, tc);
          if (fc < fbest || (val(fc) == val(fbest) && tc < best)) { fbest = fc; best = tc; }
        }
      }
    }
  return best;
}

// Ellipsoid (centre c, rotation R, semi-axes e) against a plane (point o, normal n): the
// support point against n, c - R D^2 R^T n / |D R^T n| (D = diag(e)), is the lowest point
template <class S> __device__ RawS<S> g_ellipsoid_plane(V3<S> c, const M3<S>& R, V3<S> e, V3<S> o, V3<S> n) {
  const V3<S> nl = mulT(R, n);
  const V3<S> dn = v3(e.x * nl.x, e.y * nl.y, e.z * nl.z);
  const S il = S(1.f) / ssqrt(dot(dn, dn));
  const V3<S> p = c - mul(R, v3(e.x * dn.x * il, e.y * dn.y * il, e.z * dn.z * il));
  RawS<S> k;
  k.phi = dot(n, p - o);
  k.p = p - (S(0.5f) * k.phi) * n;
  k.n = n;
  return k;
}

// Cylinder (centre c, rotation R, radius r, half length h along body z) against a plane: rim
// point `sub` = 3 cap + j, cap 0 at -h and cap 1 at +h, at 120 j degrees from the rim's lowest
// direction u x (u x n) normalised (the body x axis when the caps are parallel to the plane)
template <class S>
__device__ RawS<S> g_cylinder_plane(V3<S> c, const M3<S>& R, float r, float h, V3<S> o, V3<S> n, int sub) {
  const V3<S> u = colv(R, 2);
  V3<S> w = cross(u, cross(u, n));
  const S wl2 = dot(w, w);
  w = val(wl2) > 1e-12f ? (S(1.f) / ssqrt(wl2)) * w : colv(R, 0);
  const V3<S> w2 = cross(u, w);
  const int j = sub % 3;
  const float cs = j == 0 ? 1.f : -0.5f, sn = j == 0 ? 0.f : (j == 1 ? 0.8660254f : -0.8660254f);
  const V3<S> p = c + S(sub >= 3 ? h : -h) * u + S(r * cs) * w + S(r * sn) * w2;
  RawS<S> k;
  k.phi = dot(n, p - o);
  k.p = p - (S(0.5f) * k.phi) * n;
  k.n = n;
  return k;
}

// Sphere (centre sc, radius rs) against a solid cylinder: a centre outside meets the closest
// point of the cylinder, one inside leaves through the nearer of the side and the cap; the
// normal points from B to A (sphere_is_a: the sphere is A)
template <class S>
__device__ RawS<S> g_sphere_cylinder(V3<S> sc, S rs, V3<S> c, const M3<S>& R, float r, float h, bool sphere_is_a) {
  const V3<S> u = colv(R, 2);
  const V3<S> rel = sc - c;
  const S t = dot(u, rel);
  const V3<S> d = rel - t * u;
  const S rho = ssqrt(dot(d, d));
  const V3<S> dr = val(rho) > 1e-12f ? (S(1.f) / rho) * d : colv(R, 0);
  V3<S> nb, q;
  S dist;
  if (fabsf(val(t)) <= h && val(rho) <= r) {
    const S side = S(r) - rho, cap = S(h) - sabs(t);
    if (val(side) <= val(cap)) {
      nb = dr;
      dist = -side;
      q = c + t * u + S(r) * dr;
    } else {
      const S sg(val(t) >= 0.f ? 1.f : -1.f);
      nb = sg * u;
      dist = -cap;
      q = c + (sg * S(h)) * u + d;
    }
  } else {
    const S tc = sclamp(t, S(-h), S(h)), rc = smin(rho, S(r));
    q = c + tc * u + rc * dr;
    const V3<S> g = sc - q;
    dist = ssqrt(dot(g, g));
    nb = (S(1.f) / dist) * g;
  }
  RawS<S> k;
  k.phi = dist - rs;
  k.p = S(0.5f) * ((sc - rs * nb) + q);
  k.n = sphere_is_a ? nb : -nb;
  return k;
}

// Box-box contact `sub` (0..7): the separating-axis test over the six face axes (A's first,
// the least overlap wins) picks the reference face; the incident box's face most anti-parallel
// to it is clipped by the reference face's four side planes; clipped vertex `sub` gives the
// gap (its distance to the reference plane), the point (midway to its projection) and the
// normal (the reference normal, from B to A).  phi = 3e38 when the polygon has fewer vertices.
// Every choice (axis, face, side of a plane) is taken on the values.
template <class S>
__device__ RawS<S> g_box_box(V3<S> ca, const M3<S>& Ra, V3<S> ha, V3<S> cb, const M3<S>& Rb, V3<S> hb, int sub) {
  RawS<S> o;
  o.phi = S(3.0e38f);
  o.p = ca;
  o.n = v3(S(0.f), S(0.f), S(1.f));
  const V3<S> d = cb - ca;
  const S hav[3] = {ha.x, ha.y, ha.z}, hbv[3] = {hb.x, hb.y, hb.z};
  int best = 0;
  float best_sep = 0.f;
  for (int k = 0; k < 6; ++k) {
    const V3<S> u = k < 3 ? colv(Ra, k) : colv(Rb, k - 3);
    S ra(0.f), rb(0.f);
    for (int i = 0; i < 3; ++i) {
      ra += hav[i] * sabs(dot(colv(Ra, i), u));
      rb += hbv[i] * sabs(dot(colv(Rb, i), u));
    }
    const float sep = val(sabs(dot(d, u)) - ra - rb);
    if (k == 0 || sep > best_sep) { best_sep = sep; best = k; }
  }
  const bool refA = best < 3;
  const int jr = best % 3;
  const V3<S> cR = refA ? ca : cb, cI = refA ? cb : ca;
  const M3<S>& RR = refA ? Ra : Rb;
  const M3<S>& RI = refA ? Rb : Ra;
  const S* hR = refA ? hav : hbv;
  const S* hI = refA ? hbv : hav;
  const V3<S> nR = S(val(dot(cI - cR, colv(RR, jr))) >= 0.f ? 1.f : -1.f) * colv(RR, jr);
  int ji = 0;
  float most = 0.f;
  for (int i = 0; i < 3; ++i) {
    const float c = fabsf(val(dot(colv(RI, i), nR)));
    if (i == 0 || c > most) { most = c; ji = i; }
  }
  const S si(val(dot(colv(RI, ji), nR)) > 0.f ? -1.f : 1.f);
  const int i1 = (ji + 1) % 3, i2 = (ji + 2) % 3;
  const V3<S> fc = cI + (si * hI[ji]) * colv(RI, ji);
  const V3<S> e1 = hI[i1] * colv(RI, i1), e2 = hI[i2] * colv(RI, i2);
  V3<S> poly[8], tmp[8];
  poly[0] = fc + e1 + e2; poly[1] = fc - e1 + e2; poly[2] = fc - e1 - e2; poly[3] = fc + e1 - e2;
  int n = 4;
  const int k1 = (jr + 1) % 3, k2 = (jr + 2) % 3;
  for (int pl = 0; pl < 4 && n > 0; ++pl) {
    const int ax = pl < 2 ? k1 : k2;
    const V3<S> u = S((pl & 1) ? -1.f : 1.f) * colv(RR, ax);
    const S hh = hR[ax];
    int m = 0;
    for (int v = 0; v < n; ++v) {
      const V3<S> Pv = poly[v], Qv = poly[v + 1 < n ? v + 1 : 0];
      const S dP = dot(Pv - cR, u) - hh, dQ = dot(Qv - cR, u) - hh;
      const bool inP = val(dP) <= 0.f, inQ = val(dQ) <= 0.f;
      if (inP && m < 8) tmp[m++] = Pv;
      if (inP != inQ && m < 8) tmp[m++] = Pv + (dP / (dP - dQ)) * (Qv - Pv);
    }
    for (int v = 0; v < m; ++v) poly[v] = tmp[v];
    n = m;
  }
  if (sub < n) {
    const V3<S> v = poly[sub];
    const S dist = dot(v - cR, nR) - hR[jr];
    o.phi = dist;
    o.p = v - (S(0.5f) * dist) * nR;
    o.n = refA ? -nR : nR;
  }
  return o;
}

// ---------------------------------------------------------------------------------------
// one articulated world, one thread
// ---------------------------------------------------------------------------------------
template <class S> struct W1 {
  V3<S> bx[kG1Body], bax[kG1Body], com[kG1Body], om[kG1Body], vo[kG1Body];
  M3<S> bR[kG1Body];
  V3<S> gc[kG1Geom];
  M3<S> gR[kG1Geom];
  S minv[kG1Tree][kMaxTreeDof * kMaxTreeDof];
  S vs[kG1V], p[kG1V];
};

template <class S>
__device__ void w1_tree(const StepParams& P, const DScene& sc, int t, const S* q, const S* v, const S* tau, W1<S>& w) {
  const DBody* B = P.bodies + sc.body0;
  const DTree& tr = P.trees[sc.tree0 + t];
  const S dt(P.dt);
  if (tr.free) {
    const int b = tr.body0;
    const DBody& bd = B[b];
    const S* qb = q + bd.qoff;
    w.bR[b] = qmat(qb[3], qb[4], qb[5], qb[6]);
    w.bx[b] = v3(qb[0], qb[1], qb[2]);
    w.com[b] = w.bx[b];
    w.bax[b] = v3(S(0.f), S(0.f), S(0.f));
    const S* vb = v + bd.voff;
    V3<S> om = v3(vb[3], vb[4], vb[5]);
    V3<S> I = v3f<S>(bd.inertia);
    V3<S> gy = cross(om, v3(I.x * om.x, I.y * om.y, I.z * om.z));
    S* vs = w.vs + bd.voff;
    vs[0] = vb[0] + S(P.gravity[0]) * dt;
    vs[1] = vb[1] + S(P.gravity[1]) * dt;
    vs[2] = vb[2] + S(P.gravity[2]) * dt;
    vs[3] = om.x - dt * gy.x / I.x;
    vs[4] = om.y - dt * gy.y / I.y;
    vs[5] = om.z - dt * gy.z / I.z;
    w.om[b] = mul(w.bR[b], v3(vs[3], vs[4], vs[5]));
    w.vo[b] = v3(vs[0], vs[1], vs[2]);
    return;
  }
  const int n = tr.nv, b0 = tr.body0, v0 = tr.voff;
  for (int j = 0; j < n; ++j) {
    const int b = b0 + j;
    const DBody& bd = B[b];
    M3<S> Rp;
    V3<S> xp = v3(S(0.f), S(0.f), S(0.f));
    if (bd.parent >= 0) {
      Rp = w.bR[bd.parent];
      xp = w.bx[bd.parent];
    } else {
      for (int k = 0; k < 9; ++k) Rp.m[k] = S((k % 4 == 0) ? 1.f : 0.f);
    }
    M3<S> Rfix = mul33(Rp, qmat(S(bd.quat[0]), S(bd.quat[1]), S(bd.quat[2]), S(bd.quat[3])));
    V3<S> ax = v3f<S>(bd.axis);
    ax = (S(1.f) / ssqrt(dot(ax, ax))) * ax;
    w.bR[b] = mul33(Rfix, arot(ax, q[bd.qoff]));
    w.bx[b] = xp + mul(Rp, v3f<S>(bd.pos));
    w.bax[b] = mul(Rfix, ax);
    w.com[b] = w.bx[b] + mul(w.bR[b], v3f<S>(bd.ipos));
  }
  // composite rigid bodies (mass, first moment, inertia about the world origin)
  S mc[kMaxTreeDof];
  V3<S> hc[kMaxTreeDof];
  S Io[kMaxTreeDof][6];
  for (int j = 0; j < n; ++j) {
    const DBody& bd = B[b0 + j];
    const M3<S>& R = w.bR[b0 + j];
    S m(bd.mass);
    V3<S> c = w.com[b0 + j];
    S I0(bd.inertia[0]), I1(bd.inertia[1]), I2(bd.inertia[2]);
    const S* r = R.m;
    S Iw[6] = {r[0] * r[0] * I0 + r[1] * r[1] * I1 + r[2] * r[2] * I2,
               r[3] * r[3] * I0 + r[4] * r[4] * I1 + r[5] * r[5] * I2,
               r[6] * r[6] * I0 + r[7] * r[7] * I1 + r[8] * r[8] * I2,
               r[0] * r[3] * I0 + r[1] * r[4] * I1 + r[2] * r[5] * I2,
               r[0] * r[6] * I0 + r[1] * r[7] * I1 + r[2] * r[8] * I2,
               r[3] * r[6] * I0 + r[4] * r[7] * I1 + r[5] * r[8] * I2};
    S cc = dot(c, c);
    Io[j][0] = Iw[0] + m * (cc - c.x * c.x);
    Io[j][1] = Iw[1] + m * (cc - c.y * c.y);
    Io[j][2] = Iw[2] + m * (cc - c.z * c.z);
    Io[j][3] = Iw[3] - m * c.x * c.y;
    Io[j][4] = Iw[4] - m * c.x * c.z;
    Io[j][5] = Iw[5] - m * c.y * c.z;
    mc[j] = m;
    hc[j] = m * c;
  }
  for (int j = n - 1; j >= 0; --j) {
    int p = B[b0 + j].parent;
    if (p >= 0) {
      int jp = p - b0;
      mc[jp] += mc[j];
      hc[jp] = hc[jp] + hc[j];
      for (int k = 0; k < 6; ++k) Io[jp][k] += Io[j][k];
    }
  }
  S M[kMaxTreeDof][kMaxTreeDof];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[i][j] = S(0.f);
  for (int j = 0; j < n; ++j) {
    V3<S> aj = w.bax[b0 + j], oj = w.bx[b0 + j];
    V3<S> cC = (S(1.f) / mc[j]) * hc[j];
    S cc = dot(cC, cC);
    S I6[6] = {Io[j][0] - mc[j] * (cc - cC.x * cC.x), Io[j][1] - mc[j] * (cc - cC.y * cC.y),
               Io[j][2] - mc[j] * (cc - cC.z * cC.z), Io[j][3] + mc[j] * cC.x * cC.y,
               Io[j][4] + mc[j] * cC.x * cC.z, Io[j][5] + mc[j] * cC.y * cC.z};
    V3<S> Ia = v3(I6[0] * aj.x + I6[3] * aj.y + I6[4] * aj.z, I6[3] * aj.x + I6[1] * aj.y + I6[5] * aj.z,
                  I6[4] * aj.x + I6[5] * aj.y + I6[2] * aj.z);
    V3<S> lin = mc[j] * cross(aj, cC - oj);
    for (int i = j; i >= 0; i = (B[b0 + i].parent >= 0 ? B[b0 + i].parent - b0 : -1)) {
      V3<S> ai = w.bax[b0 + i], oi = w.bx[b0 + i];
      S mij = dot(ai, Ia + cross(cC - oi, lin));
      M[i][j] = mij;
      M[j][i] = mij;
    }
  }
  // Newton-Euler bias
  V3<S> om[kMaxTreeDof], omd[kMaxTreeDof], ac[kMaxTreeDof], F[kMaxTreeDof], Nn[kMaxTreeDof];
  const V3<S> gv = v3f<S>(P.gravity);
  for (int j = 0; j < n; ++j) {
    const DBody& bd = B[b0 + j];
    int p = bd.parent >= 0 ? bd.parent - b0 : -1;
    V3<S> a = w.bax[b0 + j], x = w.bx[b0 + j];
    S qd = v[v0 + j];
    V3<S> zero = v3(S(0.f), S(0.f), S(0.f));
    V3<S> omp = p >= 0 ? om[p] : zero, omdp = p >= 0 ? omd[p] : zero;
    om[j] = omp + qd * a;
    omd[j] = omdp + cross(omp, qd * a);
    V3<S> aanc;
    if (p >= 0) {
      V3<S> ro = x - w.com[b0 + p];
      aanc = ac[p] + cross(omdp, ro) + cross(omp, cross(omp, ro));
    } else {
      aanc = -gv;
    }
    V3<S> rc = w.com[b0 + j] - x;
    ac[j] = aanc + cross(omd[j], rc) + cross(om[j], cross(om[j], rc));
    const M3<S>& R = w.bR[b0 + j];
    auto Iw = [&](V3<S> u) {
      V3<S> l = mulT(R, u);
      return mul(R, v3(S(bd.inertia[0]) * l.x, S(bd.inertia[1]) * l.y, S(bd.inertia[2]) * l.z));
    };
    F[j] = S(bd.mass) * ac[j];
    Nn[j] = Iw(omd[j]) + cross(om[j], Iw(om[j]));
  }
  V3<S> ft[kMaxTreeDof], nt[kMaxTreeDof];
  for (int j = 0; j < n; ++j) { ft[j] = v3(S(0.f), S(0.f), S(0.f)); nt[j] = ft[j]; }
  S rhs[kMaxTreeDof];
  for (int j = n - 1; j >= 0; --j) {
    const DBody& bd = B[b0 + j];
    ft[j] = ft[j] + F[j];
    nt[j] = nt[j] + Nn[j] + cross(w.com[b0 + j], F[j]);
    V3<S> a = w.bax[b0 + j], x = w.bx[b0 + j];
    S c = dot(a, nt[j] - cross(x, ft[j]));
    S u = bd.uoff >= 0 ? tau[bd.uoff] : S(0.f);
    rhs[j] = u - c - S(bd.damping) * v[v0 + j];
    int p = bd.parent >= 0 ? bd.parent - b0 : -1;
    if (p >= 0) { ft[p] = ft[p] + ft[j]; nt[p] = nt[p] + nt[j]; }
    M[j][j] += dt * S(bd.damping);
  }
  // Cholesky and explicit inverse
  S L[kMaxTreeDof][kMaxTreeDof];
  for (int j = 0; j < n; ++j) {
    S d = M[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    d = ssqrt(smax(d, S(1e-30f)));
    L[j][j] = d;
    for (int i = j + 1; i < n; ++i) {
      S tt = M[i][j];
      for (int k = 0; k < j; ++k) tt -= L[i][k] * L[j][k];
      L[i][j] = tt / d;
    }
  }
  S Li[kMaxTreeDof][kMaxTreeDof];
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) Li[i][j] = S(0.f);
    Li[j][j] = S(1.f) / L[j][j];
    for (int i = j + 1; i < n; ++i) {
      S tt(0.f);
      for (int k = j; k < i; ++k) tt += L[i][k] * Li[k][j];
      Li[i][j] = -tt / L[i][i];
    }
  }
  S* mi = w.minv[t];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      S tt(0.f);
      for (int k = (i > j ? i : j); k < n; ++k) tt += Li[k][i] * Li[k][j];
      mi[i * kMaxTreeDof + j] = tt;
    }
  for (int i = 0; i < n; ++i) {
    S tt(0.f);
    for (int j = 0; j < n; ++j) tt += mi[i * kMaxTreeDof + j] * rhs[j];
    w.vs[v0 + i] = v[v0 + i] + dt * tt;
  }
  for (int j = 0; j < n; ++j) {
    const DBody& bd = B[b0 + j];
    V3<S> a = w.bax[b0 + j], x = w.bx[b0 + j];
    V3<S> zero = v3(S(0.f), S(0.f), S(0.f));
    V3<S> omp = zero, vop = zero, xp = zero;
    if (bd.parent >= 0) { omp = w.om[bd.parent]; vop = w.vo[bd.parent]; xp = w.bx[bd.parent]; }
    w.om[b0 + j] = omp + w.vs[v0 + j] * a;
    w.vo[b0 + j] = vop + cross(omp, x - xp);
  }
}

template <class S>
__device__ S w1_trace(const StepParams& P, const DScene& sc, const W1<S>& w, int b, V3<S> p) {
  const DBody* B = P.bodies + sc.body0;
  const DBody& bd = B[b];
  if (P.trace_mode == 1) return S(1.f / bd.mass);
  const DTree& tr = P.trees[sc.tree0 + bd.tree];
  if (tr.free) {
    V3<S> r = p - w.bx[b];
    V3<S> l = mulT(w.bR[b], r);
    S i0(1.f / bd.inertia[0]), i1(1.f / bd.inertia[1]), i2(1.f / bd.inertia[2]);
    return S(3.f / bd.mass) + dot(r, r) * (i0 + i1 + i2) - (l.x * l.x * i0 + l.y * l.y * i1 + l.z * l.z * i2);
  }
  const S* mi = w.minv[bd.tree];
  int idx[kMaxTreeDof];
  V3<S> cc[kMaxTreeDof];
  int n = 0;
  for (int a = b; a >= 0; a = B[a].parent) {
    idx[n] = B[a].voff - tr.voff;
    cc[n] = cross(w.bax[a], p - w.bx[a]);
    ++n;
  }
  S t(0.f);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) t += mi[idx[i] * kMaxTreeDof + idx[j]] * dot(cc[i], cc[j]);
  return t;
}

template <class S>
__device__ void w1_apply(const StepParams& P, const DScene& sc, W1<S>& w, int b, V3<S> p, V3<S> f, V3<S> m) {
  const DBody* B = P.bodies + sc.body0;
  const DBody& bd = B[b];
  const DTree& tr = P.trees[sc.tree0 + bd.tree];
  if (tr.free) {
    V3<S> ang = mulT(w.bR[b], cross(p - w.bx[b], f) + m);
    S* a = w.p + bd.voff;
    a[0] += f.x; a[1] += f.y; a[2] += f.z;
    a[3] += ang.x; a[4] += ang.y; a[5] += ang.z;
    return;
  }
  for (int a = b; a >= 0; a = B[a].parent) w.p[B[a].voff] += dot(w.bax[a], cross(p - w.bx[a], f) + m);
}

template <class S>
__device__ S w1_solimp(const StepParams& P, S aphi) {
  S x = sclamp(aphi / S(P.solimp[2]), S(0.f), S(1.f));
  S m(P.solimp[3]);
  S g = x < m ? m * spow(x / m, P.solimp[4])
              : S(1.f) - (S(1.f) - m) * spow((S(1.f) - x) / (S(1.f) - m), P.solimp[4]);
  return S(P.solimp[0]) + (S(P.solimp[1]) - S(P.solimp[0])) * g;
}

// Gram blocks of a contact's six basis rows (n, t1, t2 linear; n, t1, t2 angular) through
// M~^-1, as the exact diagonal impedance of Sec. III-B needs them
template <class S> struct GramS {
  S nn, n1, n2, t11, t12, t22;  // translational block
  S n3, r33;                    // torsional
  S n4, n5, r44, r45, r55;      // rolling
};

// free body: inverse mass im, inverse principal inertia ii, rotation R, lever r
template <class S>
__device__ void w1_gram_free(GramS<S>& g, S im, V3<S> ii, const M3<S>& R, V3<S> r, V3<S> n, V3<S> t1, V3<S> t2) {
  const V3<S> a0 = mulT(R, cross(r, n)), a1 = mulT(R, cross(r, t1)), a2 = mulT(R, cross(r, t2));
  const V3<S> e0 = mulT(R, n), e1 = mulT(R, t1), e2 = mulT(R, t2);
  auto q = [&](V3<S> x, V3<S> y) { return x.x * y.x * ii.x + x.y * y.y * ii.y + x.z * y.z * ii.z; };
  g.nn += im + q(a0, a0); g.n1 += q(a0, a1); g.n2 += q(a0, a2);
  g.t11 += im + q(a1, a1); g.t12 += q(a1, a2); g.t22 += im + q(a2, a2);
  g.n3 += q(a0, e0); g.r33 += q(e0, e0);
  g.n4 += q(a0, e1); g.n5 += q(a0, e2); g.r44 += q(e1, e1); g.r45 += q(e1, e2); g.r55 += q(e2, e2);
}

// Gram of the contact between bodies ba and bb (bb < 0: static): free bodies in closed form,
// hinge chains through their joint-space rows and the tree's M~^-1, the rows of two bodies of
// one tree combined first (J = J_A - J_B)
template <class S>
__device__ void w1_gram(const StepParams& P, const DScene& sc, const W1<S>& w, int ba, int bb, V3<S> p, V3<S> n,
                        V3<S> t1, V3<S> t2, GramS<S>& g) {
  const DBody* B = P.bodies + sc.body0;
  S G[2][6][kMaxTreeDof];
  int gtree[2] = {-1, -1}, gnv[2] = {0, 0};
  int ng = 0;
  g.nn = g.n1 = g.n2 = g.t11 = g.t12 = g.t22 = g.n3 = g.r33 = g.n4 = g.n5 = g.r44 = g.r45 = g.r55 = S(0.f);
  for (int side = 0; side < 2; ++side) {
    const int b = side ? bb : ba;
    if (b < 0) continue;
    const S sg(side ? -1.f : 1.f);
    const DBody& bd = B[b];
    const DTree& tr = P.trees[sc.tree0 + bd.tree];
    if (tr.free) {
      w1_gram_free(g, S(1.f / bd.mass), v3(S(1.f / bd.inertia[0]), S(1.f / bd.inertia[1]), S(1.f / bd.inertia[2])),
                   w.bR[b], p - w.bx[b], n, t1, t2);
      continue;
    }
    const int slot = (ng > 0 && gtree[0] == bd.tree) ? 0 : ng;
    if (slot == ng) {
      gtree[slot] = bd.tree;
      gnv[slot] = tr.nv;
      for (int x = 0; x < 6; ++x)
        for (int i = 0; i < kMaxTreeDof; ++i) G[slot][x][i] = S(0.f);
      ++ng;
    }
    for (int a = b; a >= 0; a = B[a].parent) {
      const int k = B[a].voff - tr.voff;
      const V3<S> ax = w.bax[a];
      const V3<S> lin = cross(ax, p - w.bx[a]);  // point velocity per unit joint rate
      G[slot][0][k] += sg * dot(n, lin); G[slot][1][k] += sg * dot(t1, lin); G[slot][2][k] += sg * dot(t2, lin);
      G[slot][3][k] += sg * dot(n, ax); G[slot][4][k] += sg * dot(t1, ax); G[slot][5][k] += sg * dot(t2, ax);
    }
  }
  for (int slot = 0; slot < ng; ++slot) {
    const S* mi = w.minv[gtree[slot]];
    const int nv = gnv[slot];
    auto q = [&](int x, int y) {  // G_x^T M~^-1 G_y
      S acc(0.f);
      for (int i = 0; i < nv; ++i) {
        S h(0.f);
        for (int j = 0; j < nv; ++j) h += mi[i * kMaxTreeDof + j] * G[slot][y][j];
        acc += G[slot][x][i] * h;
      }
      return acc;
    };
    g.nn += q(0, 0); g.n1 += q(0, 1); g.n2 += q(0, 2); g.t11 += q(1, 1); g.t12 += q(1, 2); g.t22 += q(2, 2);
    g.n3 += q(0, 3); g.r33 += q(3, 3);
    g.n4 += q(0, 4); g.n5 += q(0, 5); g.r44 += q(4, 4); g.r45 += q(4, 5); g.r55 += q(5, 5);
  }
}

// J~_j M~^-1 J~_j^T of a facet row n_row - mu (c x + s y) from the Gram entries of its rows
template <class S>
__device__ S w1_gram_facet(S nn, S nx, S ny, S xx, S xy, S yy, S mu, float c, float s) {
  return nn - S(2.f) * mu * (S(c) * nx + S(s) * ny) +
         mu * mu * (S(c * c) * xx + S(2.f * c * s) * xy + S(s * s) * yy);
}

// Facet impulses with the exact diagonal impedance of Sec. III-B: M(phi) replaced per facet j
// by M_j = 1 / ((k dt + d) J~_j M~^-1 J~_j^T); outputs the resultant (normal, t1, t2, torsion,
// rolling t1, rolling t2) on A
template <class S>
__device__ void w1_facets_exact(const StepParams& P, S vn, S vt1, S vt2, S wn, S wr1, S wr2, S phi, S mu_t, S mu_tor,
                                S mu_rol, const GramS<S>& g, S& N, S& F1, S& F2, S& Tq, S& R1, S& R2) {
  const S kd(fmaf(P.k_user, P.dt, P.d_user));
  const S a = -S(P.k_user) * phi - kd * vn;
  S f1(0.f), f2(0.f), t(0.f), r1(0.f), r2(0.f);
  for (int j = 0; j < P.n_t; ++j) {
    const float c = P.tcos[j], s = P.tsin[j];
    const S gj = a + kd * mu_t * (S(c) * vt1 + S(s) * vt2);
    if (val(gj) > 0.f) {
      const S lam = gj / (kd * w1_gram_facet(g.nn, g.n1, g.n2, g.t11, g.t12, g.t22, mu_t, c, s));
      N += lam; f1 += S(c) * lam; f2 += S(s) * lam;
    }
  }
  for (int j = 0; j < P.n_tor; ++j) {
    const S sg((j & 1) ? -1.f : 1.f);
    const S gj = a + kd * mu_tor * sg * wn;
    if (val(gj) > 0.f) {
      const S lam = gj / (kd * (g.nn - S(2.f) * mu_tor * sg * g.n3 + mu_tor * mu_tor * g.r33));
      N += lam; t += sg * lam;
    }
  }
  for (int j = 0; j < P.n_rol; ++j) {
    const float c = P.rcos[j], s = P.rsin[j];
    const S gj = a + kd * mu_rol * (S(c) * wr1 + S(s) * wr2);
    if (val(gj) > 0.f) {
      const S lam = gj / (kd * w1_gram_facet(g.nn, g.n4, g.n5, g.r44, g.r45, g.r55, mu_rol, c, s));
      N += lam; r1 += S(c) * lam; r2 += S(s) * lam;
    }
  }
  F1 = -mu_t * f1; F2 = -mu_t * f2; Tq = -mu_tor * t; R1 = -mu_rol * r1; R2 = -mu_rol * r2;
}

// The learned impedance's factor exp(clamp(g(x), -8, 8)) on M(phi) (Sec. III-B's learned
// K(q), D(q)): inputs x = (phi / width, 1 - 3 sum(1/m) / tr, w_n / tr, b static), with w_n the
// normal row's inverse mass of both links taken as free bodies about their centres of mass;
// g = b2 + sum_h w2_h tanh(b1_h + sum_i W1_hi x_i) with parameters th [W1 (8 x 4), b1, w2, b2]
template <class S>
__device__ S w1_impnet_scale(const StepParams& P, const DScene& sc, const W1<S>& w, const float* th, int ba, int bb,
                             V3<S> p, V3<S> n, S phi, S tr) {
  const DBody* B = P.bodies + sc.body0;
  auto side = [&](int b) {
    const DBody& bd = B[b];
    const M3<S>& R = w.bR[b];
    const V3<S> com = w.bx[b] + mul(R, v3f<S>(bd.ipos));
    const V3<S> u = mulT(R, cross(p - com, n));
    return S(1.f / bd.mass) + u.x * u.x * S(1.f / bd.inertia[0]) + u.y * u.y * S(1.f / bd.inertia[1]) +
           u.z * u.z * S(1.f / bd.inertia[2]);
  };
  const S im_sum(1.f / B[ba].mass + (bb >= 0 ? 1.f / B[bb].mass : 0.f));
  const S w_n = bb >= 0 ? side(ba) + side(bb) : side(ba);
  S x[kImpIn];
  x[0] = sclamp(phi / S(P.solimp[2]), S(-1.f), S(1.f));
  x[1] = sclamp(S(1.f) - S(3.f) * im_sum / tr, S(-1.f), S(1.f));
  x[2] = sclamp(w_n / tr, S(0.f), S(4.f));
  x[3] = S(bb < 0 ? 1.f : 0.f);
  S gsum(th[kImpParams - 1]);
  for (int h = 0; h < kImpHidden; ++h) {
    S a(th[kImpHidden * kImpIn + h]);
    for (int i = 0; i < kImpIn; ++i) a += S(th[h * kImpIn + i]) * x[i];
    gsum += S(th[kImpHidden * kImpIn + kImpHidden + h]) * stanh(a);
  }
  return sexp(sclamp(gsum, S(-kImpClamp), S(kImpClamp)));
}

template <class S, bool kExt>
__device__ void w1_contact(const StepParams& P, const DScene& sc, W1<S>& w, int world, int ga, int gb,
                           const RawS<S>& k, bool plane, V3<S> px) {
  const DGeom& GA = P.geoms[sc.geom0 + ga];
  const DGeom& GB = P.geoms[sc.geom0 + gb];
  const int ba = GA.body, bb = GB.body;
  V3<S> t1, t2;
  if (plane) {
    t1 = px;
  } else {
    V3<S> c = fabsf(val(k.n.z)) < 0.5f ? v3(-k.n.y, k.n.x, S(0.f)) : v3(S(0.f), -k.n.z, k.n.y);
    t1 = (S(1.f) / ssqrt(dot(c, c))) * c;
  }
  t2 = cross(k.n, t1);
  V3<S> vc = w.vo[ba] + cross(w.om[ba], k.p - w.bx[ba]);
  V3<S> wc = w.om[ba];
  S tr = w1_trace(P, sc, w, ba, k.p);
  if (bb >= 0) {
    vc = vc - (w.vo[bb] + cross(w.om[bb], k.p - w.bx[bb]));
    wc = wc - w.om[bb];
    tr += w1_trace(P, sc, w, bb, k.p);
  }
  S vn = dot(k.n, vc), vt1 = dot(t1, vc), vt2 = dot(t2, vc);
  S wn = dot(k.n, wc), wr1 = dot(t1, wc), wr2 = dot(t2, wc);
  S mut(fmaxf(GA.mu[0], GB.mu[0])), mutor(fmaxf(GA.mu[1], GB.mu[1])), murol(fmaxf(GA.mu[2], GB.mu[2]));
  S N(0.f), F1(0.f), F2(0.f), Tq(0.f), R1(0.f), R2(0.f);
  if (kExt && P.trace_mode == 2) {
    GramS<S> g;
    w1_gram(P, sc, w, ba, bb, k.p, k.n, t1, t2, g);
    w1_facets_exact(P, vn, vt1, vt2, wn, wr1, wr2, k.phi, mut, mutor, murol, g, N, F1, F2, Tq, R1, R2);
    V3<S> f = N * k.n + F1 * t1 + F2 * t2;
    V3<S> m = Tq * k.n + R1 * t1 + R2 * t2;
    w1_apply(P, sc, w, ba, k.p, f, m);
    if (bb >= 0) w1_apply(P, sc, w, bb, k.p, -f, -m);
    return;
  }
  S r = w1_solimp(P, sabs(k.phi));
  S mphi = r / (S(1.f) - r) / tr;
  if (kExt && P.trace_mode == 3)
    mphi = mphi * w1_impnet_scale(P, sc, w, P.impnet + (size_t)world * P.impnet_stride, ba, bb, k.p, k.n, k.phi, tr);
  S kM = S(P.k_user) * mphi, dM = S(P.d_user) * mphi;
  S A = -kM * k.phi, Bc = kM * S(P.dt) + dM;
  for (int j = 0; j < P.n_t; ++j) {
    S c(P.tcos[j]), s(P.tsin[j]);
    S lam = smax(A - Bc * (vn - mut * (c * vt1 + s * vt2)), S(0.f));
    N += lam;
    F1 -= mut * c * lam;
    F2 -= mut * s * lam;
  }
  if (P.n_tor == 2) {
    S lp = smax(A - Bc * (vn - mutor * wn), S(0.f));
    S lm = smax(A - Bc * (vn + mutor * wn), S(0.f));
    N += lp + lm;
    Tq = -mutor * (lp - lm);
  }
  for (int j = 0; j < P.n_rol; ++j) {
    S c(P.rcos[j]), s(P.rsin[j]);
    S lam = smax(A - Bc * (vn - murol * (c * wr1 + s * wr2)), S(0.f));
    N += lam;
    R1 -= murol * c * lam;
    R2 -= murol * s * lam;
  }
  V3<S> f = N * k.n + F1 * t1 + F2 * t2;
  V3<S> m = Tq * k.n + R1 * t1 + R2 * t2;
  w1_apply(P, sc, w, ba, k.p, f, m);
  if (bb >= 0) w1_apply(P, sc, w, bb, k.p, -f, -m);
}

template <class S, bool kExt>
__device__ void w1_pair(const StepParams& P, const DScene& sc, W1<S>& w, int world, int ga, int gb) {
  const DGeom* G = P.geoms + sc.geom0;
  int ta = G[ga].type, tb = G[gb].type;
  if (ta == CF_GEOM_PLANE) { int t = ga; ga = gb; gb = t; t = ta; ta = tb; tb = t; }
  const float* sa = G[ga].size;
  const float* sb = G[gb].size;
  V3<S> ca = w.gc[ga], cb = w.gc[gb];
  const M3<S>& Ra = w.gR[ga];
  const M3<S>& Rb = w.gR[gb];
  const S margin(P.margin);
  if (tb == CF_GEOM_PLANE) {
    V3<S> nz = colv(Rb, 2), px = colv(Rb, 0);
    if (ta == CF_GEOM_SPHERE) {
      RawS<S> k = g_sphere_plane(ca, S(sa[0]), cb, nz);
      if (k.phi < margin) w1_contact<S, kExt>(P, sc, w, world, ga, gb, k, true, px);
    } else if (ta == CF_GEOM_CAPSULE) {
      V3<S> ax = colv(Ra, 2);
      for (int e = 0; e < 2; ++e) {
        RawS<S> k = g_sphere_plane(ca + S(e ? sa[1] : -sa[1]) * ax, S(sa[0]), cb, nz);
        if (k.phi < margin) w1_contact<S, kExt>(P, sc, w, world, ga, gb, k, true, px);
      }
    } else if (ta == CF_GEOM_BOX) {
      for (int ci = 0; ci < 8; ++ci) {
        V3<S> corner = ca + mul(Ra, v3(S((ci & 4) ? sa[0] : -sa[0]), S((ci & 2) ? sa[1] : -sa[1]),
                                       S((ci & 1) ? sa[2] : -sa[2])));
        RawS<S> k = g_sphere_plane(corner, S(0.f), cb, nz);
        if (k.phi < margin) w1_contact<S, kExt>(P, sc, w, world, ga, gb, k, true, px);
      }
    } else if (kExt && ta == CF_GEOM_CYLINDER) {
      for (int sub = 0; sub < 6; ++sub) {
        RawS<S> k = g_cylinder_plane(ca, Ra, sa[0], sa[1], cb, nz, sub);
        if (k.phi < margin) w1_contact<S, kExt>(P, sc, w, world, ga, gb, k, true, px);
      }
    } else if (kExt && ta == CF_GEOM_ELLIPSOID) {
      RawS<S> k = g_ellipsoid_plane(ca, Ra, v3f<S>(sa), cb, nz);
      if (k.phi < margin) w1_contact<S, kExt>(P, sc, w, world, ga, gb, k, true, px);
    }
    return;
  }
  RawS<S> k;
  k.phi = S(3.0e38f);
  if (ta >= CF_GEOM_CYLINDER || tb >= CF_GEOM_CYLINDER) {  // cylinders touch spheres only
    if (kExt && ta == CF_GEOM_SPHERE && tb == CF_GEOM_CYLINDER)
      k = g_sphere_cylinder(ca, S(sa[0]), cb, Rb, sb[0], sb[1], true);
    else if (kExt && ta == CF_GEOM_CYLINDER && tb == CF_GEOM_SPHERE)
      k = g_sphere_cylinder(cb, S(sb[0]), ca, Ra, sa[0], sa[1], false);
  } else if (ta == CF_GEOM_SPHERE && tb == CF_GEOM_SPHERE) {
    k = g_sphere_sphere(ca, S(sa[0]), cb, S(sb[0]));
  } else if (ta == CF_GEOM_CAPSULE && tb == CF_GEOM_CAPSULE) {
    V3<S> ua = colv(Ra, 2), ub = colv(Rb, 2);
    V3<S> p1 = ca - S(sa[1]) * ua, q1 = ca + S(sa[1]) * ua, p2 = cb - S(sb[1]) * ub, q2 = cb + S(sb[1]) * ub;
    S ss(0.f), tt(0.f);
    g_segments(p1, q1, p2, q2, ss, tt);
    k = g_sphere_sphere(p1 + ss * (q1 - p1), S(sa[0]), p2 + tt * (q2 - p2), S(sb[0]));
  } else if (ta == CF_GEOM_CAPSULE && tb == CF_GEOM_SPHERE) {
    V3<S> u = colv(Ra, 2);
    S t = sclamp(dot(cb - ca, u), S(-sa[1]), S(sa[1]));
    k = g_sphere_sphere(ca + t * u, S(sa[0]), cb, S(sb[0]));
  } else if (ta == CF_GEOM_SPHERE && tb == CF_GEOM_CAPSULE) {
    V3<S> u = colv(Rb, 2);
    S t = sclamp(dot(ca - cb, u), S(-sb[1]), S(sb[1]));
    k = g_sphere_sphere(ca, S(sa[0]), cb + t * u, S(sb[0]));
  } else if (ta == CF_GEOM_BOX || tb == CF_GEOM_BOX) {
    if (ta == CF_GEOM_BOX && tb == CF_GEOM_BOX) {  // each clipped face vertex
      if (kExt)
        for (int sub = 0; sub < 8; ++sub) {
          RawS<S> kb = g_box_box(ca, Ra, v3f<S>(sa), cb, Rb, v3f<S>(sb), sub);
          if (kb.phi < margin) w1_contact<S, kExt>(P, sc, w, world, ga, gb, kb, false, v3(S(0.f), S(0.f), S(0.f)));
        }
      return;
    }
    bool boxA = ta == CF_GEOM_BOX;
    const M3<S>& Rbx = boxA ? Ra : Rb;
    V3<S> cbx = boxA ? ca : cb, co = boxA ? cb : ca;
    const float* bs = boxA ? sa : sb;
    const float* os = boxA ? sb : sa;
    int to = boxA ? tb : ta;
    V3<S> hs = v3f<S>(bs);
    if (to == CF_GEOM_SPHERE) {
      k = g_sphere_box(co, S(os[0]), cbx, Rbx, hs, !boxA);
    } else {
      V3<S> u = colv(boxA ? Rb : Ra, 2);
      S t = g_capsule_box_param(mulT(Rbx, co - cbx), mulT(Rbx, u), S(os[1]), hs);
      k = g_sphere_box(co + t * u, S(os[0]), cbx, Rbx, hs, !boxA);
    }
  }
  if (k.phi < margin) w1_contact<S, kExt>(P, sc, w, world, ga, gb, k, false, v3(S(0.f), S(0.f), S(0.f)));
}

// one step of an articulated world in scalar type S: q[nq], v[nv] updated in place, tau per
// actuated hinge (scene order)
template <class S, bool kExt>
__device__ void w1_step(const StepParams& P, const DScene& sc, int world, S* q, S* v, const S* tau, W1<S>& w) {
  const DBody* B = P.bodies + sc.body0;
  const DGeom* G = P.geoms + sc.geom0;
  for (int t = 0; t < sc.ntree; ++t) w1_tree(P, sc, t, q, v, tau, w);
  for (int i = 0; i < sc.nv; ++i) w.p[i] = S(0.f);
  for (int g = 0; g < sc.ngeom; ++g) {
    const DGeom& gd = G[g];
    M3<S> Rl = qmat(S(gd.quat[0]), S(gd.quat[1]), S(gd.quat[2]), S(gd.quat[3]));
    if (gd.body >= 0) {
      w.gc[g] = w.bx[gd.body] + mul(w.bR[gd.body], v3f<S>(gd.pos));
      w.gR[g] = mul33(w.bR[gd.body], Rl);
    } else {
      w.gc[g] = v3f<S>(gd.pos);
      w.gR[g] = Rl;
    }
  }
  for (int k = 0; k < sc.npair; ++k) {
    uint32_t pr = P.pairs[sc.pair0 + k];
    int ga = pr >> 16, gb = pr & 0xffff;
    // the same conservative bounding test as the step kernel (values only)
    auto bound = [&](int g) {
      const DGeom& gd = G[g];
      return gd.type == CF_GEOM_SPHERE ? gd.size[0]
             : gd.type == CF_GEOM_CAPSULE ? gd.size[0] + gd.size[1]
             : sqrtf(gd.size[0] * gd.size[0] + gd.size[1] * gd.size[1] + gd.size[2] * gd.size[2]);
    };
    bool pa = G[ga].type == CF_GEOM_PLANE, pb = G[gb].type == CF_GEOM_PLANE;
    bool cand;
    if (pa || pb) {
      int gp = pa ? ga : gb, go = pa ? gb : ga;
      V3<S> nz = colv(w.gR[gp], 2);
      cand = val(dot(nz, w.gc[go] - w.gc[gp])) < bound(go) + P.margin;
    } else {
      V3<S> d = w.gc[ga] - w.gc[gb];
      float rr = bound(ga) + bound(gb) + P.margin;
      cand = val(dot(d, d)) < rr * rr;
    }
    if (cand) w1_pair<S, kExt>(P, sc, w, world, ga, gb);
  }
  // joint limits and dry joint friction, the step kernel's per-hinge impulses on the smooth
  // prediction: a limit below the margin is a one-row constraint +-e_k with the facet law and
  // M = r(|gap|) / (1 - r(|gap|)) / (M~^-1)_kk; friction applies the stopping impulse
  // -v_s,k / (M~^-1)_kk clamped to +-frictionloss dt.  Derivatives follow the primal branch:
  // an inactive limit or a saturated friction impulse passes none.
  if (sc.joints) {
    for (int t = 0; t < sc.ntree; ++t) {
      const DTree& tr = P.trees[sc.tree0 + t];
      if (tr.free) continue;
      const S* mi = w.minv[t];
      for (int j = 0; j < tr.nbody; ++j) {
        const DBody& bd = B[tr.body0 + j];
        if (!bd.limited && !(bd.frictionloss > 0.f)) continue;
        const int k = bd.voff - tr.voff;
        const S wkk = mi[k * kMaxTreeDof + k];
        const S vsk = w.vs[bd.voff];
        S pk(0.f);
        if (bd.limited) {
          const S qk = q[bd.qoff];
          for (int side = 0; side < 2; ++side) {
            const S gap = side ? S(bd.range[1]) - qk : qk - S(bd.range[0]);
            if (!(val(gap) < P.margin)) continue;
            const S sg(side ? -1.f : 1.f);
            const S sv = sg * vsk;
            S Mk;
            if (kExt && P.trace_mode == 2) {  // the exact impedance of the one-row constraint
              Mk = S(1.f) / (S(fmaf(P.k_user, P.dt, P.d_user)) * wkk);
            } else {
              const S r = w1_solimp(P, sabs(gap));
              Mk = r / ((S(1.f) - r) * wkk);
            }
            const S lam = -S(P.k_user) * Mk * (sv * S(P.dt) + gap) - S(P.d_user) * Mk * sv;
            if (val(lam) > 0.f) pk += sg * lam;
          }
        }
        if (bd.frictionloss > 0.f) {
          const S cap(bd.frictionloss * P.dt);
          pk += sclamp(-vsk / wkk, -cap, cap);
        }
        w.p[bd.voff] += pk;
      }
    }
  }
  const S dt(P.dt);
  for (int t = 0; t < sc.ntree; ++t) {
    const DTree& tr = P.trees[sc.tree0 + t];
    if (tr.free) {
      const DBody& bd = B[tr.body0];
      S* vb = v + bd.voff;
      const S* vs = w.vs + bd.voff;
      const S* pb = w.p + bd.voff;
      for (int k = 0; k < 3; ++k) vb[k] = vs[k] + pb[k] / S(bd.mass);
      for (int k = 0; k < 3; ++k) vb[3 + k] = vs[3 + k] + pb[3 + k] / S(bd.inertia[k]);
      S* qb = q + bd.qoff;
      for (int k = 0; k < 3; ++k) qb[k] = qb[k] + vb[k] * dt;
      S w0 = vb[3], w1 = vb[4], w2 = vb[5];
      S wn = ssqrt(w0 * w0 + w1 * w1 + w2 * w2);
      S dq0(1.f), dq1(0.f), dq2(0.f), dq3(0.f);
      if (val(wn) > 0.f) {
        S sn, cs;
        ssincos(S(0.5f) * wn * dt, sn, cs);
        S sc_ = sn / wn;
        dq0 = cs; dq1 = sc_ * w0; dq2 = sc_ * w1; dq3 = sc_ * w2;
      }
      S a0 = qb[3], a1 = qb[4], a2 = qb[5], a3 = qb[6];
      S n0 = a0 * dq0 - a1 * dq1 - a2 * dq2 - a3 * dq3;
      S n1 = a0 * dq1 + a1 * dq0 + a2 * dq3 - a3 * dq2;
      S n2 = a0 * dq2 - a1 * dq3 + a2 * dq0 + a3 * dq1;
      S n3 = a0 * dq3 + a1 * dq2 - a2 * dq1 + a3 * dq0;
      S inv = S(1.f) / ssqrt(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
      qb[3] = n0 * inv; qb[4] = n1 * inv; qb[5] = n2 * inv; qb[6] = n3 * inv;
    } else {
      const S* mi = w.minv[t];
      for (int i = 0; i < tr.nv; ++i) {
        S acc(0.f);
        for (int j = 0; j < tr.nv; ++j) acc += mi[i * kMaxTreeDof + j] * w.p[tr.voff + j];
        v[tr.voff + i] = w.vs[tr.voff + i] + acc;
      }
      for (int j = 0; j < tr.nbody; ++j) {
        const DBody& bd = B[tr.body0 + j];
        q[bd.qoff] = q[bd.qoff] + v[bd.voff] * dt;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// vector-Jacobian product of one step: CTA per world, lane j = input coordinate j
// (q, then v, then actuated tau); a_in = adjoint of the step's output state
// ---------------------------------------------------------------------------------------
// kExt: the extended step compiled in: the exact and learned impedances (trace_mode 2, 3),
// box-box pairs, cylinders and ellipsoids.  At most 128 registers, so that 8 worlds of 64 lanes
// are resident per SM (1216 on 152 SMs): a batch of 1024 worlds then runs in one wave instead
// of a full wave and a tail (168 registers left room for 6 per SM).
template <bool kExt>
__global__ void __launch_bounds__(kG1Lanes, 8) vjp_kernel(StepParams P, const float* q, const float* v, int step,
                                                       const float* aq_in, const float* av_in, float* aq_out,
                                                       float* av_out, float* dtau, int64_t total_nu) {
  const int world = blockIdx.x;
  const DWorld Wd = P.worlds[world];
  const DScene sc = P.scenes[Wd.scene];
  const int nin = sc.nq + sc.nv + sc.nu;
  W1<DF> w;
  DF qs[kG1Q], vs[kG1V], tau[kG1V];
  for (int j = threadIdx.x; j < ((nin + kG1Lanes - 1) / kG1Lanes) * kG1Lanes; j += kG1Lanes) {
    for (int i = 0; i < sc.nq; ++i) qs[i] = DF(q[Wd.qadr + i], j == i ? 1.f : 0.f);
    for (int i = 0; i < sc.nv; ++i) vs[i] = DF(v[Wd.vadr + i], j == sc.nq + i ? 1.f : 0.f);
    int slice = P.nctrl > 0 ? (step < P.nctrl ? step : P.nctrl - 1) : -1;
    for (int i = 0; i < sc.nu; ++i)
      tau[i] = DF(slice >= 0 ? P.ctrl[(size_t)slice * P.total_nu + Wd.uadr + i] : 0.f, j == sc.nq + sc.nv + i ? 1.f : 0.f);
    w1_step<DF, kExt>(P, sc, world, qs, vs, tau, w);
    float acc = 0.f;
    for (int i = 0; i < sc.nq; ++i) acc = fmaf(qs[i].d, aq_in[Wd.qadr + i], acc);
    for (int i = 0; i < sc.nv; ++i) acc = fmaf(vs[i].d, av_in[Wd.vadr + i], acc);
    if (j < sc.nq) aq_out[Wd.qadr + j] = acc;
    else if (j < sc.nq + sc.nv) av_out[Wd.vadr + j - sc.nq] = acc;
    else if (j < nin && dtau) dtau[(size_t)step * total_nu + Wd.uadr + (j - sc.nq - sc.nv)] = acc;
  }
}

bool grad_scene_supported(const DScene& s, const char** why) {
  if (s.pile) { *why = "pile scenes are not differentiable here"; return false; }
  if (s.nbody > kG1Body || s.ngeom > kG1Geom || s.nq > kG1Q || s.nv > kG1V || s.ntree > kG1Tree) {
    *why = "scene exceeds the adjoint's per-world limits (24 bodies, 32 geoms, 48 q, 48 v, 8 trees)";
    return false;
  }
  return true;
}

size_t grad_workspace_bytes(int W, int64_t total_nq, int64_t total_nv, const cf_batch_opts& o) {
  (void)W;
  int ck = o.grad_ckpt < 1 ? 1 : o.grad_ckpt;
  int nseg = (o.grad_steps + ck - 1) / ck;
  size_t state = (size_t)(total_nq + total_nv) * sizeof(float);
  state = (state + 255) / 256 * 256;
  return state * (size_t)(nseg + 1 + ck + 2);
}

cudaError_t run_grad(const StepParams& p0, const GradArgs& g, int nctrl, cudaStream_t s) {
  const size_t nq = g.total_nq, nv = g.total_nv;
  size_t state = (nq + nv) * sizeof(float);
  state = (state + 255) / 256 * 256;
  const int ck = g.ckpt;
  const int nseg = (g.T + ck - 1) / ck;
  char* base = g.tape;
  auto ckpt = [&](int k) { return base + state * k; };
  auto seg = [&](int k) { return base + state * (nseg + 1 + k); };
  char* adjA = base + state * (nseg + 1 + ck);
  char* adjB = adjA + state;
  auto qptr = [&](char* c) { return reinterpret_cast<float*>(c); };
  auto vptr = [&](char* c) { return reinterpret_cast<float*>(c) + nq; };
  cudaError_t e;
  StepParams p = p0;
  auto step_on = [&](float* q, float* v, int first, int n) {
    StepParams ps = p;
    ps.q = q;
    ps.v = v;
    ps.ctrl_offset = first;
    ps.nsteps = n;
    ps.capture = nullptr;
    ps.capture_cap = 0;
    int per = step_max_blocks_per_sm(true, g.variant, g.smem);
    int grid = ps.nunits < g.num_sms * per ? ps.nunits : g.num_sms * per;
    return launch_step(ps, true, g.variant, grid, g.smem, s);
  };
  // forward pass with checkpoints (the batch state advances to step T)
  e = cudaMemcpyAsync(qptr(ckpt(0)), p.q, nq * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vptr(ckpt(0)), p.v, nv * sizeof(float), cudaMemcpyDeviceToDevice, s);
  for (int k = 0; k < nseg && e == cudaSuccess; ++k) {
    int len = (g.T - k * ck) < ck ? (g.T - k * ck) : ck;
    e = step_on(p.q, p.v, k * ck, len);
    if (e == cudaSuccess) e = cudaMemcpyAsync(qptr(ckpt(k + 1)), p.q, nq * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vptr(ckpt(k + 1)), p.v, nv * sizeof(float), cudaMemcpyDeviceToDevice, s);
  }
  if (e != cudaSuccess) return e;
  // adjoint of the final state
  e = cudaMemcpyAsync(qptr(adjA), g.dqT, nq * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vptr(adjA), g.dvT, nv * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && g.dtau && g.total_nu > 0)
    e = cudaMemsetAsync(g.dtau, 0, sizeof(float) * g.total_nu * g.T, s);
  char* ain = adjA;
  char* aout = adjB;
  for (int k = nseg - 1; k >= 0 && e == cudaSuccess; --k) {
    int first = k * ck;
    int len = (g.T - first) < ck ? (g.T - first) : ck;
    // recompute the segment's step-entry states
    e = cudaMemcpyAsync(seg(0), ckpt(k), state, cudaMemcpyDeviceToDevice, s);
    for (int i = 1; i < len && e == cudaSuccess; ++i) {
      e = cudaMemcpyAsync(seg(i), seg(i - 1), state, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = step_on(qptr(seg(i)), vptr(seg(i)), first + i - 1, 1);
    }
    for (int i = len - 1; i >= 0 && e == cudaSuccess; --i) {
      StepParams pv = p;
      pv.ctrl_offset = 0;
      if (g.variant == kExtVariant)
        vjp_kernel<true><<<g.W, kG1Lanes, 0, s>>>(pv, qptr(seg(i)), vptr(seg(i)), first + i, qptr(ain), vptr(ain),
                                                  qptr(aout), vptr(aout), g.dtau, g.total_nu);
      else
        vjp_kernel<false><<<g.W, kG1Lanes, 0, s>>>(pv, qptr(seg(i)), vptr(seg(i)), first + i, qptr(ain), vptr(ain),
                                                   qptr(aout), vptr(aout), g.dtau, g.total_nu);
      e = cudaGetLastError();
      char* t = ain;
      ain = aout;
      aout = t;
    }
  }
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(g.dq0, qptr(ain), nq * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g.dv0, vptr(ain), nv * sizeof(float), cudaMemcpyDeviceToDevice, s);
  (void)nctrl;
  return e;
}

}  // namespace cf
