// Host runtime of libcomfree: model validation, batch layout inside the caller's device
// workspace, work-unit scheduling, autotuning, and the C entry points of comfree.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "cf_internal.cuh"
#include "cf_grad.cuh"

using namespace cf;

namespace {

thread_local std::string g_err;

cf_status fail(cf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

cf_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CF_CUDA(call, what)                     \
  do {                                          \
    cudaError_t e__ = (call);                   \
    if (e__ != cudaSuccess) return cuda_fail(e__, what); \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

void cf::set_last_error(const char* msg) { g_err = msg; }

// ---------------------------------------------------------------------------------------
// model
// ---------------------------------------------------------------------------------------
struct cf_model {
  std::vector<DScene> scenes;
  std::vector<DBody> bodies;
  std::vector<DGeom> geoms;
  std::vector<DTree> trees;
  std::vector<uint32_t> pairs;
  std::vector<float> cost;  // relative per-world cost estimate of each scene
  float gravity[3], k_user, d_user, solimp[5], margin;
  int n_t, n_tor, n_rol, trace_mode;
};

static cf_status build_scene(const cf_scene_desc& d, int si, cf_model* m) {
  if (d.nbody < 0 || d.ngeom < 1 || d.nbody > 4096 || d.ngeom > 16000)
    return fail(CF_ERR_INVALID_ARGUMENT, "scene %d: bad body/geom counts (%d, %d)", si, d.nbody, d.ngeom);
  if ((d.nbody && (!d.body_parent || !d.body_jnt || !d.body_pos || !d.body_quat || !d.body_axis || !d.body_ipos ||
                   !d.body_mass || !d.body_inertia || !d.body_damping)) ||
      !d.geom_type || !d.geom_body || !d.geom_pos || !d.geom_quat || !d.geom_size || !d.geom_mu)
    return fail(CF_ERR_INVALID_ARGUMENT, "scene %d: null array", si);
  DScene sc{};
  sc.nbody = d.nbody;
  sc.ngeom = d.ngeom;
  sc.body0 = (int)m->bodies.size();
  sc.geom0 = (int)m->geoms.size();
  sc.tree0 = (int)m->trees.size();
  sc.pair0 = (int)m->pairs.size();
  sc.pile = d.pile ? 1 : 0;
  int nq = 0, nv = 0, nu = 0;
  std::vector<DBody> B(d.nbody);
  std::vector<int> tree_of(d.nbody, -1);
  std::vector<DTree> T;
  for (int b = 0; b < d.nbody; ++b) {
    int p = d.body_parent[b], j = d.body_jnt[b];
    if (p < -1 || p >= b) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: parent %d not topological", si, b, p);
    if (j != CF_JOINT_FREE && j != CF_JOINT_HINGE)
      return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: joint type %d", si, b, j);
    if (j == CF_JOINT_FREE && p != -1)
      return fail(CF_ERR_UNSUPPORTED, "scene %d body %d: free joint below another body", si, b);
    if (p >= 0 && d.body_jnt[p] == CF_JOINT_FREE)
      return fail(CF_ERR_UNSUPPORTED, "scene %d body %d: child of a free body", si, b);
    double mass = d.body_mass[b];
    if (!(mass > 0.0) || !std::isfinite(mass))
      return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: mass must be positive", si, b);
    for (int k = 0; k < 3; ++k)
      if (!(d.body_inertia[3 * b + k] > 0.0))
        return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: inertia must be positive", si, b);
    if (d.body_damping[b] < 0.0) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: negative damping", si, b);
    DBody& o = B[b];
    o.parent = p;
    o.jnt = j;
    o.qoff = nq;
    o.voff = nv;
    o.uoff = j == CF_JOINT_HINGE ? nu : -1;
    nq += j == CF_JOINT_FREE ? 7 : 1;
    nv += j == CF_JOINT_FREE ? 6 : 1;
    nu += j == CF_JOINT_HINGE ? 1 : 0;
    for (int k = 0; k < 3; ++k) {
      o.pos[k] = (float)d.body_pos[3 * b + k];
      o.axis[k] = (float)d.body_axis[3 * b + k];
      o.ipos[k] = (float)d.body_ipos[3 * b + k];
      o.inertia[k] = (float)d.body_inertia[3 * b + k];
    }
    for (int k = 0; k < 4; ++k) o.quat[k] = (float)d.body_quat[4 * b + k];
    o.mass = (float)mass;
    o.damping = (float)d.body_damping[b];
    o.limited = 0;
    o.range[0] = o.range[1] = 0.f;
    o.frictionloss = 0.f;
    if (j == CF_JOINT_HINGE && d.body_range && d.body_range[2 * b] < d.body_range[2 * b + 1]) {
      if (!std::isfinite(d.body_range[2 * b]) || !std::isfinite(d.body_range[2 * b + 1]))
        return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: joint range must be finite", si, b);
      o.limited = 1;
      o.range[0] = (float)d.body_range[2 * b];
      o.range[1] = (float)d.body_range[2 * b + 1];
    }
    if (d.body_frictionloss) {
      const double fl = d.body_frictionloss[b];
      if (!(fl >= 0.0) || !std::isfinite(fl))
        return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: frictionloss must be >= 0", si, b);
      if (j == CF_JOINT_HINGE) o.frictionloss = (float)fl;
    }
    if (o.limited || o.frictionloss > 0.f) sc.joints = 1;
    if (j == CF_JOINT_FREE) {
      for (int k = 0; k < 3; ++k)
        if (d.body_ipos[3 * b + k] != 0.0)
          return fail(CF_ERR_UNSUPPORTED, "scene %d body %d: free body frame must sit at its centre of mass", si, b);
    } else {
      double an = std::sqrt(d.body_axis[3 * b] * d.body_axis[3 * b] + d.body_axis[3 * b + 1] * d.body_axis[3 * b + 1] +
                            d.body_axis[3 * b + 2] * d.body_axis[3 * b + 2]);
      if (!(an > 0.0)) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d body %d: zero hinge axis", si, b);
    }
    if (p < 0) {
      tree_of[b] = (int)T.size();
      DTree t{};
      t.body0 = b;
      t.nbody = 1;
      t.voff = o.voff;
      t.nv = j == CF_JOINT_FREE ? 6 : 1;
      t.free = j == CF_JOINT_FREE ? 1 : 0;
      T.push_back(t);
    } else {
      int t = tree_of[p];
      if (T[t].body0 + T[t].nbody != b)
        return fail(CF_ERR_UNSUPPORTED, "scene %d body %d: bodies of a hinge tree must be contiguous", si, b);
      tree_of[b] = t;
      T[t].nbody += 1;
      T[t].nv += 1;
      if (T[t].nv > kMaxTreeDof)
        return fail(CF_ERR_UNSUPPORTED, "scene %d: hinge tree with more than %d DoFs", si, kMaxTreeDof);
    }
    o.tree = tree_of[b];
    const int local = b - T[tree_of[b]].body0;
    o.anc = (1 << local) | (p >= 0 ? B[p].anc : 0);
  }
  std::vector<DGeom> G(d.ngeom);
  int nplane = 0, plane0 = -1;
  for (int g = 0; g < d.ngeom; ++g) {
    int ty = d.geom_type[g], bd = d.geom_body[g];
    if (ty < CF_GEOM_PLANE || ty > CF_GEOM_ELLIPSOID)
      return fail(CF_ERR_INVALID_ARGUMENT, "scene %d geom %d: type %d", si, g, ty);
    if (bd < -1 || bd >= d.nbody) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d geom %d: body %d", si, g, bd);
    if (ty == CF_GEOM_PLANE && bd != -1)
      return fail(CF_ERR_UNSUPPORTED, "scene %d geom %d: planes must be static", si, g);
    if (ty != CF_GEOM_PLANE) {
      int need = ty == CF_GEOM_SPHERE ? 1 : (ty == CF_GEOM_CAPSULE || ty == CF_GEOM_CYLINDER ? 2 : 3);
      for (int k = 0; k < need; ++k)
        if (!(d.geom_size[3 * g + k] > 0.0))
          return fail(CF_ERR_INVALID_ARGUMENT, "scene %d geom %d: size must be positive", si, g);
    }
    for (int k = 0; k < 3; ++k)
      if (d.geom_mu[3 * g + k] < 0.0) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d geom %d: negative friction", si, g);
    DGeom& o = G[g];
    o.type = ty;
    o.body = bd;
    for (int k = 0; k < 3; ++k) {
      o.pos[k] = (float)d.geom_pos[3 * g + k];
      o.size[k] = (float)d.geom_size[3 * g + k];
      o.mu[k] = (float)d.geom_mu[3 * g + k];
    }
    double qn = 0;
    for (int k = 0; k < 4; ++k) qn += d.geom_quat[4 * g + k] * d.geom_quat[4 * g + k];
    if (!(qn > 0.0)) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d geom %d: zero quaternion", si, g);
    for (int k = 0; k < 4; ++k) o.quat[k] = (float)(d.geom_quat[4 * g + k] / std::sqrt(qn));
    if (ty == CF_GEOM_PLANE) {
      if (plane0 < 0) plane0 = g;
      ++nplane;
    }
  }
  if (sc.pile) {
    if (d.ngeom < d.nbody) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d: pile needs one geom per body", si);
    for (int b = 0; b < d.nbody; ++b) {
      if (d.body_jnt[b] != CF_JOINT_FREE) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d: pile bodies must be free", si);
      const DGeom& g = G[b];
      if (g.body != b || g.type == CF_GEOM_PLANE || g.pos[0] != 0.f || g.pos[1] != 0.f || g.pos[2] != 0.f ||
          g.quat[0] != 1.f || g.quat[1] != 0.f || g.quat[2] != 0.f || g.quat[3] != 0.f)
        return fail(CF_ERR_INVALID_ARGUMENT, "scene %d: pile geom %d must sit at the origin of body %d", si, b, b);
    }
    for (int g = d.nbody; g < d.ngeom; ++g)
      if (G[g].type != CF_GEOM_PLANE) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d: pile extra geoms must be planes", si);
    if (d.nbody > 4096 || d.ngeom - d.nbody > 4096)
      return fail(CF_ERR_UNSUPPORTED, "scene %d: pile too large (at most 4096 bodies and 4096 planes)", si);
    sc.plane0 = d.nbody;
    sc.nplane = d.ngeom - d.nbody;
  } else {
    sc.plane0 = plane0 < 0 ? 0 : plane0;
    sc.nplane = nplane;
    // explicit candidate pair list: not both static, not the same body, not parent/child
    for (int a = 0; a < d.ngeom; ++a)
      for (int b = a + 1; b < d.ngeom; ++b) {
        int ba = G[a].body, bb = G[b].body;
        if (ba < 0 && bb < 0) continue;
        if (ba == bb) continue;
        if (ba >= 0 && bb >= 0 && (B[ba].parent == bb || B[bb].parent == ba)) continue;
        m->pairs.push_back(((uint32_t)a << 16) | (uint32_t)b);
      }
    if (d.ngeom >= 32768) return fail(CF_ERR_UNSUPPORTED, "scene %d: too many geoms", si);
  }
  {
    int nbox = 0;
    int nextra = 0;
    for (int g = 0; g < d.ngeom; ++g) {
      nbox += G[g].type == CF_GEOM_BOX && G[g].body >= 0;
      nextra += G[g].type >= CF_GEOM_CYLINDER;
    }
    sc.boxbox = (nbox >= 2 || nextra > 0) ? 1 : 0;
  }
  // fingertips of the MPC cost: capsules carried by a hinge body that no body has as parent
  for (int g = 0; g < d.ngeom; ++g) {
    const int bd = G[g].body;
    bool leaf = bd >= 0 && d.body_jnt[bd] == CF_JOINT_HINGE && G[g].type == CF_GEOM_CAPSULE;
    for (int k = 0; leaf && k < d.nbody; ++k)
      if (d.body_parent[k] == bd) leaf = false;
    G[g].tip = leaf ? 1 : 0;
  }
  {
    // one friction triple for every geom: the pair friction (the larger of two equal values)
    // is that triple, and the kernels need not look the geoms up per contact
    sc.mu_uniform = d.ngeom > 0 ? 1 : 0;
    for (int g = 0; g < d.ngeom; ++g)
      for (int k = 0; k < 3; ++k)
        if (G[g].mu[k] != G[0].mu[k]) sc.mu_uniform = 0;
    for (int k = 0; k < 3; ++k) sc.mu[k] = d.ngeom > 0 ? G[0].mu[k] : 0.f;
  }
  sc.npair = (int)m->pairs.size() - sc.pair0;
  sc.nq = nq;
  sc.nv = nv;
  sc.nu = nu;
  sc.ntree = (int)T.size();
  for (auto& t : T) m->trees.push_back(t);
  for (auto& b : B) m->bodies.push_back(b);
  for (auto& g : G) m->geoms.push_back(g);
  m->scenes.push_back(sc);
  float npairs = sc.pile ? 0.5f * sc.nbody * (sc.nbody - 1) + sc.nbody * sc.nplane : (float)sc.npair;
  m->cost.push_back(1.0f + npairs + 4.0f * nv);
  return CF_OK;
}

extern "C" cf_status cf_model_create(const cf_model_desc* desc, cf_model** out) {
  if (!desc || !out) return fail(CF_ERR_INVALID_ARGUMENT, "null argument");
  *out = nullptr;
  if (desc->nscene < 1 || !desc->scenes) return fail(CF_ERR_INVALID_ARGUMENT, "no scenes");
  auto bad_dirs = [](int n) { return n != 0 && (n < 2 || n > kMaxFacetDirs || (n & 1)); };
  if (bad_dirs(desc->n_t) || bad_dirs(desc->n_rol) || (desc->n_tor != 0 && desc->n_tor != 2))
    return fail(CF_ERR_INVALID_ARGUMENT, "facet counts: n_t, n_rol must be 0 or even in [2, 16]; n_tor 0 or 2");
  if (desc->n_t + desc->n_tor + desc->n_rol < 1) return fail(CF_ERR_INVALID_ARGUMENT, "no facets");
  if (!(desc->k_user >= 0.0) || !(desc->d_user >= 0.0)) return fail(CF_ERR_INVALID_ARGUMENT, "negative impedance");
  const double* si = desc->solimp;
  if (!(si[0] > 0.0 && si[0] <= si[1] && si[1] < 1.0 && si[2] > 0.0 && si[3] > 0.0 && si[3] < 1.0 && si[4] >= 1.0))
    return fail(CF_ERR_INVALID_ARGUMENT, "solimp must satisfy 0 < r_min <= r_max < 1, width > 0, 0 < mid < 1, power >= 1");
  if (desc->trace_mode < 0 || desc->trace_mode > 3)
    return fail(CF_ERR_INVALID_ARGUMENT, "trace_mode must be 0, 1, 2 or 3");
  cf_model* m = new (std::nothrow) cf_model();
  if (!m) return fail(CF_ERR_OUT_OF_MEMORY, "model allocation");
  for (int s = 0; s < desc->nscene; ++s) {
    cf_status st = build_scene(desc->scenes[s], s, m);
    if (st != CF_OK) {
      delete m;
      return st;
    }
  }
  for (int k = 0; k < 3; ++k) m->gravity[k] = (float)desc->gravity[k];
  m->k_user = (float)desc->k_user;
  m->d_user = (float)desc->d_user;
  for (int k = 0; k < 5; ++k) m->solimp[k] = (float)desc->solimp[k];
  m->margin = (float)desc->margin;
  m->n_t = desc->n_t;
  m->n_tor = desc->n_tor;
  m->n_rol = desc->n_rol;
  m->trace_mode = desc->trace_mode;
  *out = m;
  return CF_OK;
}

extern "C" void cf_model_destroy(cf_model* model) { delete model; }

extern "C" cf_status cf_scene_sizes(const cf_model* m, int32_t scene, int32_t sizes[5]) {
  if (!m || !sizes || scene < 0 || scene >= (int)m->scenes.size()) return fail(CF_ERR_INVALID_ARGUMENT, "bad scene");
  const DScene& s = m->scenes[scene];
  sizes[0] = s.nq; sizes[1] = s.nv; sizes[2] = s.nu; sizes[3] = s.nbody; sizes[4] = s.ngeom;
  return CF_OK;
}

// ---------------------------------------------------------------------------------------
// batch
// ---------------------------------------------------------------------------------------
struct Layout {
  size_t scenes, bodies, geoms, trees, pairs, worlds, order, units, sub_order, sub_units;
  size_t q, v, wparam, ctrl, ncontact, flags, errword, queue, capture, backup, grad, total;
};

struct cf_batch {
  cf_model model;  // private copy: the caller may destroy its model
  int W = 0;
  std::vector<DWorld> worlds;
  std::vector<int> scene_of;
  int64_t total_nq = 0, total_nv = 0, total_nu = 0, total_param = 0;
  cf_batch_opts opts{};
  Layout L{};
  char* ws = nullptr;
  std::vector<int> warps;      // per scene
  std::vector<DUnit> units;    // all worlds
  int nunits = 0;
  int group_warps = 0;         // warps per world when every unit shares it and grouping is on, else 0
  bool allow_group = false;    // warp groups pull worlds by themselves (cf_batch_autotune decides)
  size_t smem_all = 0;
  bool artic_all = false;
  bool ext = false;  // needs the extended kernel: possible box-box contacts, cylinders or ellipsoids
  bool imp = false;  // exact or learned impedance (trace_mode 2, 3)
  const float* impnet = nullptr;  // learned impedance network (trace_mode 3)
  int impnet_stride = 0;
  int variant = 0;             // pile kernel occupancy variant (autotuned)
  // fused MPC cost (cf_set_cost)
  float* cost = nullptr;
  const float* goal = nullptr;
  const float* qref = nullptr;
  int cost_body = 0;
  float cw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int nctrl = 0;
  int num_sms = 0;
  template <class T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

static Layout make_layout(const cf_model& m, int W, int64_t tnq, int64_t tnv, int64_t tnu, int64_t tparam,
                          const cf_batch_opts& o, size_t grad_bytes) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return r;
  };
  L.scenes = take(sizeof(DScene) * m.scenes.size());
  L.bodies = take(sizeof(DBody) * std::max<size_t>(m.bodies.size(), 1));
  L.geoms = take(sizeof(DGeom) * m.geoms.size());
  L.trees = take(sizeof(DTree) * std::max<size_t>(m.trees.size(), 1));
  L.pairs = take(sizeof(uint32_t) * std::max<size_t>(m.pairs.size(), 1));
  L.worlds = take(sizeof(DWorld) * W);
  L.order = take(sizeof(int) * W);
  L.units = take(sizeof(DUnit) * W);
  L.sub_order = take(sizeof(int) * W);
  L.sub_units = take(sizeof(DUnit) * W);
  L.q = take(sizeof(float) * tnq);
  L.v = take(sizeof(float) * tnv);
  L.wparam = take(sizeof(float) * std::max<int64_t>(tparam, 4));
  L.ctrl = take(sizeof(float) * std::max<int64_t>(tnu, 1) * std::max(o.max_ctrl_steps, 1));
  L.ncontact = take(sizeof(int) * W);
  L.flags = take(sizeof(int) * W);
  L.errword = take(sizeof(int) * 4);
  L.queue = take(sizeof(int) * 4);
  L.capture = take(sizeof(cf_contact) * (size_t)W * std::max(o.contact_capture, 0));
  L.backup = take(sizeof(float) * (tnq + tnv));
  L.grad = take(grad_bytes);
  L.total = off;
  return L;
}

static int default_warps(const DScene& s) {
  if (!s.pile) return 1;
  if (s.nbody <= 24) return 1;
  if (s.nbody <= 96) return 4;
  return 8;
}

static void fill_sizes(const cf_model& m, int W, const int32_t* scene_of, std::vector<DWorld>* worlds, int64_t& tnq,
                       int64_t& tnv, int64_t& tnu, int64_t& tparam) {
  tnq = tnv = tnu = tparam = 0;
  for (int w = 0; w < W; ++w) {
    const DScene& s = m.scenes[scene_of[w]];
    DWorld d{};
    d.scene = scene_of[w];
    d.qadr = (int)tnq;
    d.vadr = (int)tnv;
    d.uadr = (int)tnu;
    d.padr = s.pile ? (int)tparam : -1;
    tnq += s.nq;
    tnv += s.nv;
    tnu += s.nu;
    if (s.pile) tparam += 8 * (int64_t)s.nbody;
    if (worlds) worlds->push_back(d);
  }
}

extern "C" cf_status cf_batch_workspace_bytes(const cf_model* m, int32_t n_worlds, const int32_t* scene_of_world,
                                              const cf_batch_opts* opts, size_t* bytes) {
  if (!m || !scene_of_world || !bytes || n_worlds < 1) return fail(CF_ERR_INVALID_ARGUMENT, "bad arguments");
  cf_batch_opts o{1, 0, 0, 1};
  if (opts) o = *opts;
  if (o.max_ctrl_steps < 1) o.max_ctrl_steps = 1;
  for (int w = 0; w < n_worlds; ++w)
    if (scene_of_world[w] < 0 || scene_of_world[w] >= (int)m->scenes.size())
      return fail(CF_ERR_INVALID_ARGUMENT, "world %d: scene %d out of range", w, scene_of_world[w]);
  int64_t tnq, tnv, tnu, tp;
  fill_sizes(*m, n_worlds, scene_of_world, nullptr, tnq, tnv, tnu, tp);
  if (tnq >= INT32_MAX || tnv >= INT32_MAX || tp >= INT32_MAX) return fail(CF_ERR_UNSUPPORTED, "batch too large");
  size_t gb = o.grad_steps > 0 ? grad_workspace_bytes(n_worlds, tnq, tnv, o) : 0;
  *bytes = make_layout(*m, n_worlds, tnq, tnv, tnu, tp, o, gb).total;
  return CF_OK;
}

// worlds of `list` grouped by scene into units of kWarps / warps worlds, units sorted by cost
static void build_units(const cf_batch* b, const std::vector<int>& list, std::vector<int>& order,
                        std::vector<DUnit>& units, size_t& smem, bool& artic) {
  std::map<int, std::vector<int>> by_scene;
  for (int w : list) by_scene[b->worlds[w].scene].push_back(w);
  std::vector<std::pair<float, DUnit>> tmp;
  order.clear();
  smem = 0;
  artic = false;
  for (auto& kv : by_scene) {
    int sidx = kv.first;
    const DScene& sc = b->model.scenes[sidx];
    if (!sc.pile) artic = true;
    int wp = b->warps[sidx];
    int per = kWarps / wp;
    float cost = b->model.cost[sidx] / (float)wp;
    size_t need = world_smem_bytes(sc, wp) * per;
    smem = std::max(smem, need);
    const std::vector<int>& ws = kv.second;
    for (size_t i = 0; i < ws.size(); i += per) {
      DUnit u{};
      u.first = (int)order.size();
      u.count = (int)std::min<size_t>(per, ws.size() - i);
      u.warps = wp;
      for (int k = 0; k < u.count; ++k) order.push_back(ws[i + k]);
      tmp.push_back({cost, u});
    }
  }
  std::stable_sort(tmp.begin(), tmp.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
  // lay the worlds out in the units' (cost) order, so that order[] itself is that order
  std::vector<int> sorted;
  sorted.reserve(order.size());
  units.clear();
  for (auto& t : tmp) {
    DUnit u = t.second;
    const int first = (int)sorted.size();
    for (int k = 0; k < u.count; ++k) sorted.push_back(order[u.first + k]);
    u.first = first;
    units.push_back(u);
  }
  order.swap(sorted);
}

// warps per world shared by every unit (the launch can then let each warp group pull worlds
// by itself), else 0
static int uniform_warps(const std::vector<DUnit>& units) {
  if (units.empty()) return 0;
  for (const DUnit& u : units)
    if (u.warps != units[0].warps) return 0;
  return units[0].warps;
}

// the work list of a launch: units for CTAs, or (uniform warps, grouping on) the worlds for
// warp groups
static void set_work(StepParams& p, const std::vector<DUnit>& units, size_t nworld, bool allow_group) {
  p.group_warps = allow_group ? uniform_warps(units) : 0;
  p.nunits = p.group_warps > 0 ? (int)nworld : (int)units.size();
}

static cf_status upload_units(cf_batch* b, cudaStream_t st) {
  std::vector<int> all(b->W), order;
  for (int w = 0; w < b->W; ++w) all[w] = w;
  build_units(b, all, order, b->units, b->smem_all, b->artic_all);
  b->nunits = (int)b->units.size();
  b->group_warps = b->allow_group ? uniform_warps(b->units) : 0;
  if (b->smem_all > step_max_dynamic_smem())
    return fail(CF_ERR_UNSUPPORTED, "a work unit needs %zu bytes of shared memory", b->smem_all);
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, st),
          "upload order");
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.units, b->units.data(), sizeof(DUnit) * b->units.size(), cudaMemcpyHostToDevice,
                          st),
          "upload units");
  CF_CUDA(cudaStreamSynchronize(st), "upload units");
  return CF_OK;
}

extern "C" cf_status cf_batch_create(const cf_model* m, int32_t n_worlds, const int32_t* scene_of_world,
                                     const float* world_params, const cf_batch_opts* opts, void* device_workspace,
                                     size_t workspace_bytes, void* stream, cf_batch** out) {
  if (!out) return fail(CF_ERR_INVALID_ARGUMENT, "null out");
  *out = nullptr;
  size_t need = 0;
  cf_status st = cf_batch_workspace_bytes(m, n_worlds, scene_of_world, opts, &need);
  if (st != CF_OK) return st;
  if (!device_workspace || workspace_bytes < need)
    return fail(CF_ERR_OUT_OF_MEMORY, "workspace of %zu bytes given, %zu needed", workspace_bytes, need);
  if (reinterpret_cast<uintptr_t>(device_workspace) % 256)
    return fail(CF_ERR_INVALID_ARGUMENT, "workspace must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  cf_batch* b = new (std::nothrow) cf_batch();
  if (!b) return fail(CF_ERR_OUT_OF_MEMORY, "batch allocation");
  b->model = *m;
  b->W = n_worlds;
  b->opts = opts ? *opts : cf_batch_opts{1, 0, 0, 1};
  if (b->opts.max_ctrl_steps < 1) b->opts.max_ctrl_steps = 1;
  if (b->opts.grad_ckpt < 1) b->opts.grad_ckpt = 1;
  b->scene_of.assign(scene_of_world, scene_of_world + n_worlds);
  int64_t tp;
  fill_sizes(*m, n_worlds, scene_of_world, &b->worlds, b->total_nq, b->total_nv, b->total_nu, tp);
  b->total_param = tp;
  size_t gb = b->opts.grad_steps > 0 ? grad_workspace_bytes(n_worlds, b->total_nq, b->total_nv, b->opts) : 0;
  b->L = make_layout(*m, n_worlds, b->total_nq, b->total_nv, b->total_nu, tp, b->opts, gb);
  b->ws = static_cast<char*>(device_workspace);
  b->warps.resize(m->scenes.size());
  for (size_t i = 0; i < m->scenes.size(); ++i) b->warps[i] = default_warps(m->scenes[i]);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);

  // per-world parameters: validate overrides
  std::vector<float> params(std::max<int64_t>(tp, 4), 0.f);
  if (world_params) {
    std::memcpy(params.data(), world_params, sizeof(float) * tp);
    for (int w = 0; w < n_worlds; ++w) {
      const DWorld& d = b->worlds[w];
      if (d.padr < 0) continue;
      const DScene& sc = m->scenes[d.scene];
      for (int i = 0; i < sc.nbody; ++i) {
        const float* p = params.data() + d.padr + 8 * i;
        int ty = (int)p[4];
        bool ok = p[0] > 0.f && p[1] > 0.f && p[2] > 0.f && p[3] > 0.f &&
                  ty >= CF_GEOM_SPHERE && ty <= CF_GEOM_ELLIPSOID && p[5] > 0.f && (ty == CF_GEOM_SPHERE || p[6] > 0.f) &&
                  ((ty != CF_GEOM_BOX && ty != CF_GEOM_ELLIPSOID) || p[7] > 0.f) && (float)ty == p[4];
        if (!ok) {
          delete b;
          return fail(CF_ERR_INVALID_ARGUMENT, "world %d body %d: bad override block", w, i);
        }
      }
    }
  } else {
    // defaults from the template
    for (int w = 0; w < n_worlds; ++w) {
      const DWorld& d = b->worlds[w];
      if (d.padr < 0) continue;
      const DScene& sc = m->scenes[d.scene];
      for (int i = 0; i < sc.nbody; ++i) {
        const DBody& bd = m->bodies[sc.body0 + i];
        const DGeom& gd = m->geoms[sc.geom0 + i];
        float* p = params.data() + d.padr + 8 * i;
        p[0] = bd.mass; p[1] = bd.inertia[0]; p[2] = bd.inertia[1]; p[3] = bd.inertia[2];
        p[4] = (float)gd.type; p[5] = gd.size[0]; p[6] = gd.size[1]; p[7] = gd.size[2];
      }
    }
  }
  // the extended kernel serves worlds where two boxes may touch or that hold cylinders or
  // ellipsoids; the impedance modes have a lighter pile-only kernel of their own
  b->imp = m->trace_mode >= 2;
  b->ext = false;
  for (int w = 0; w < n_worlds && !b->ext; ++w) {
    const DWorld& d = b->worlds[w];
    const DScene& sc = m->scenes[d.scene];
    if (d.padr < 0) {
      if (sc.boxbox) b->ext = true;
      continue;
    }
    int nbox = 0;
    int nextra = 0;
    for (int i = 0; i < sc.nbody; ++i) {
      const int ty = (int)params[d.padr + 8 * i + 4];
      nbox += ty == CF_GEOM_BOX;
      nextra += ty >= CF_GEOM_CYLINDER;
    }
    if (nbox >= 2 || nextra > 0) b->ext = true;
  }
  // zero state with identity orientations
  std::vector<float> q0(b->total_nq, 0.f);
  for (int w = 0; w < n_worlds; ++w) {
    const DScene& sc = m->scenes[b->worlds[w].scene];
    for (int i = 0; i < sc.nbody; ++i) {
      const DBody& bd = m->bodies[sc.body0 + i];
      if (bd.jnt == CF_JOINT_FREE) q0[b->worlds[w].qadr + bd.qoff + 3] = 1.f;
    }
  }
  auto up = [&](size_t off, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(b->ws + off, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = up(b->L.scenes, m->scenes.data(), sizeof(DScene) * m->scenes.size());
  if (e == cudaSuccess) e = up(b->L.bodies, m->bodies.data(), sizeof(DBody) * m->bodies.size());
  if (e == cudaSuccess) e = up(b->L.geoms, m->geoms.data(), sizeof(DGeom) * m->geoms.size());
  if (e == cudaSuccess) e = up(b->L.trees, m->trees.data(), sizeof(DTree) * m->trees.size());
  if (e == cudaSuccess) e = up(b->L.pairs, m->pairs.data(), sizeof(uint32_t) * m->pairs.size());
  if (e == cudaSuccess) e = up(b->L.worlds, b->worlds.data(), sizeof(DWorld) * n_worlds);
  if (e == cudaSuccess) e = up(b->L.wparam, params.data(), sizeof(float) * tp);
  if (e == cudaSuccess) e = up(b->L.q, q0.data(), sizeof(float) * b->total_nq);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.v, 0, sizeof(float) * b->total_nv, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.ctrl, 0, sizeof(float) * std::max<int64_t>(b->total_nu, 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.ncontact, 0, sizeof(int) * n_worlds, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.flags, 0, sizeof(int) * n_worlds, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.errword, 0, sizeof(int) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.queue, 0, sizeof(int) * 4, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch upload");
  }
  b->nctrl = 0;
  st = upload_units(b, s);
  if (st != CF_OK) {
    delete b;
    return st;
  }
  *out = b;
  return CF_OK;
}

extern "C" void cf_batch_destroy(cf_batch* b) { delete b; }

extern "C" cf_status cf_batch_sizes(const cf_batch* b, int64_t* nq, int64_t* nv, int64_t* nu) {
  if (!b) return fail(CF_ERR_INVALID_ARGUMENT, "null batch");
  if (nq) *nq = b->total_nq;
  if (nv) *nv = b->total_nv;
  if (nu) *nu = b->total_nu;
  return CF_OK;
}

extern "C" cf_status cf_set_state(cf_batch* b, const float* q, const float* v, int32_t on_device, void* stream) {
  if (!b || (!q && !v)) return fail(CF_ERR_INVALID_ARGUMENT, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (on_device < 0 || on_device > 2) return fail(CF_ERR_INVALID_ARGUMENT, "on_device must be 0, 1 or 2");
  cudaMemcpyKind k = on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (q) CF_CUDA(cudaMemcpyAsync(b->ws + b->L.q, q, sizeof(float) * b->total_nq, k, s), "set q");
  if (v) CF_CUDA(cudaMemcpyAsync(b->ws + b->L.v, v, sizeof(float) * b->total_nv, k, s), "set v");
  if (on_device == 0) CF_CUDA(cudaStreamSynchronize(s), "set state");
  return CF_OK;
}

static cf_status read_errword(const cf_batch* b, cudaStream_t s, int* word) {
  CF_CUDA(cudaMemcpyAsync(word, b->ws + b->L.errword, sizeof(int), cudaMemcpyDeviceToHost, s), "read error word");
  CF_CUDA(cudaStreamSynchronize(s), "read error word");
  return CF_OK;
}

static cf_status status_of_word(int w) {
  if (w & CF_FLAG_NONFINITE) return fail(CF_ERR_NONFINITE, "a world produced a non-finite state");
  if (w & CF_FLAG_RANGE) return fail(CF_ERR_NONFINITE, "a contact velocity change left the scatter range");
  if (w & CF_FLAG_TIMEOUT) return fail(CF_ERR_TIMEOUT, "a bounded device wait gave up");
  if (w & CF_FLAG_CONTACT_OVERFLOW) return fail(CF_ERR_CONTACT_OVERFLOW, "contact capture overflow");
  return CF_OK;
}

extern "C" cf_status cf_get_state(const cf_batch* b, float* q, float* v, int32_t on_device, void* stream) {
  if (!b || (!q && !v)) return fail(CF_ERR_INVALID_ARGUMENT, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (on_device < 0 || on_device > 2) return fail(CF_ERR_INVALID_ARGUMENT, "on_device must be 0, 1 or 2");
  cudaMemcpyKind k = on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (q) CF_CUDA(cudaMemcpyAsync(q, b->ws + b->L.q, sizeof(float) * b->total_nq, k, s), "get q");
  if (v) CF_CUDA(cudaMemcpyAsync(v, b->ws + b->L.v, sizeof(float) * b->total_nv, k, s), "get v");
  if (on_device == 0) {
    int word = 0;
    cf_status st = read_errword(b, s, &word);
    if (st != CF_OK) return st;
    return status_of_word(word);
  }
  return CF_OK;
}

extern "C" cf_status cf_set_ctrl(cf_batch* b, const float* tau, int32_t T, int32_t on_device, void* stream) {
  if (!b || !tau || T < 1 || T > b->opts.max_ctrl_steps)
    return fail(CF_ERR_INVALID_ARGUMENT, "control sequence length %d outside [1, %d]", T, b ? b->opts.max_ctrl_steps : 0);
  cudaStream_t s = (cudaStream_t)stream;
  if (b->total_nu > 0)
    CF_CUDA(cudaMemcpyAsync(b->ws + b->L.ctrl, tau, sizeof(float) * b->total_nu * T,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
            "set ctrl");
  if (!on_device) CF_CUDA(cudaStreamSynchronize(s), "set ctrl");
  b->nctrl = T;
  return CF_OK;
}

static StepParams make_params(const cf_batch* b, float dt, int nsteps) {
  const cf_model& m = b->model;
  StepParams p{};
  p.scenes = b->at<DScene>(b->L.scenes);
  p.bodies = b->at<DBody>(b->L.bodies);
  p.geoms = b->at<DGeom>(b->L.geoms);
  p.trees = b->at<DTree>(b->L.trees);
  p.pairs = b->at<uint32_t>(b->L.pairs);
  p.worlds = b->at<DWorld>(b->L.worlds);
  p.units = b->at<DUnit>(b->L.units);
  p.order = b->at<int>(b->L.order);
  p.group_warps = b->group_warps;
  p.nunits = b->group_warps > 0 ? b->W : b->nunits;
  p.q = b->at<float>(b->L.q);
  p.v = b->at<float>(b->L.v);
  p.wparam = b->at<float>(b->L.wparam);
  p.ctrl = b->at<float>(b->L.ctrl);
  p.total_nu = (int)b->total_nu;
  p.nctrl = b->total_nu > 0 ? b->nctrl : 0;
  p.ncontact = b->at<int>(b->L.ncontact);
  p.flags = b->at<int>(b->L.flags);
  p.errword = b->at<int>(b->L.errword);
  p.queue = b->at<int>(b->L.queue);
  p.capture = b->opts.contact_capture > 0 ? b->at<cf_contact>(b->L.capture) : nullptr;
  p.capture_cap = std::max(b->opts.contact_capture, 0);
  p.dt = dt;
  p.nsteps = nsteps;
  for (int k = 0; k < 3; ++k) p.gravity[k] = m.gravity[k];
  p.k_user = m.k_user;
  p.d_user = m.d_user;
  for (int k = 0; k < 5; ++k) p.solimp[k] = m.solimp[k];
  p.margin = m.margin;
  p.n_t = m.n_t;
  p.n_tor = m.n_tor;
  p.n_rol = m.n_rol;
  p.trace_mode = m.trace_mode;
  p.impnet = b->impnet;
  p.impnet_stride = b->impnet_stride;
  for (int j = 0; j < m.n_t; ++j) {
    double th = 2.0 * M_PI * j / m.n_t;
    p.tcos[j] = (float)std::cos(th);
    p.tsin[j] = (float)std::sin(th);
  }
  for (int j = 0; j < m.n_rol; ++j) {
    double th = 2.0 * M_PI * j / m.n_rol;
    p.rcos[j] = (float)std::cos(th);
    p.rsin[j] = (float)std::sin(th);
  }
  p.cost = b->cost;
  p.goal = b->goal;
  p.qref = b->qref;
  p.cost_body = b->cost_body;
  for (int k = 0; k < 8; ++k) p.cw[k] = b->cw[k];
  return p;
}

static cf_status launch(const cf_batch* b, StepParams& p, bool artic, size_t smem, cudaStream_t s) {
  if (p.nunits <= 0) return CF_OK;
  if (p.trace_mode == 3 && !p.impnet)
    return fail(CF_ERR_INVALID_ARGUMENT, "trace_mode 3 needs an impedance network (cf_batch_set_impedance_net)");
  const int var = b->ext ? kExtVariant : (b->imp ? kImpVariant : b->variant);
  int per_sm = step_max_blocks_per_sm(artic, var, smem);
  const int per_block = p.group_warps > 0 ? kWarps / p.group_warps : 1;
  int grid = std::min((p.nunits + per_block - 1) / per_block, std::max(1, b->num_sms * per_sm));
  cudaError_t e = launch_step(p, artic, var, grid, smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "step launch");
  return CF_OK;
}

// The device address of page-locked host memory `p` (nullptr when it is not page-locked host
// memory)
static void* host_device_ptr(void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return a.devicePointer;
}

extern "C" cf_status cf_step_host(cf_batch* b, float* q, float* v, float dt, int32_t nsteps, void* stream) {
  if (!b) return fail(CF_ERR_INVALID_ARGUMENT, "null batch");
  if (!(dt > 0.f) || !std::isfinite(dt)) return fail(CF_ERR_INVALID_ARGUMENT, "dt must be positive");
  if (nsteps < 1) return fail(CF_ERR_INVALID_ARGUMENT, "nsteps must be >= 1");
  if ((reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(v)) & 3)
    return fail(CF_ERR_INVALID_ARGUMENT, "q and v must be 4-byte aligned");
  float* dq = static_cast<float*>(host_device_ptr(q));
  float* dv = static_cast<float*>(host_device_ptr(v));
  if (!dq || !dv) return fail(CF_ERR_INVALID_ARGUMENT, "q and v must be page-locked host memory");
  StepParams p = make_params(b, dt, nsteps);
  p.q = dq;
  p.v = dv;
  return launch(b, p, b->artic_all, b->smem_all, (cudaStream_t)stream);
}

extern "C" cf_status cf_step(cf_batch* b, const int32_t* worlds, int32_t n, float dt, int32_t nsteps, void* stream) {
  if (!b) return fail(CF_ERR_INVALID_ARGUMENT, "null batch");
  if (!(dt > 0.f) || !std::isfinite(dt)) return fail(CF_ERR_INVALID_ARGUMENT, "dt must be positive");
  if (nsteps < 1) return fail(CF_ERR_INVALID_ARGUMENT, "nsteps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  StepParams p = make_params(b, dt, nsteps);
  if (!worlds) return launch(b, p, b->artic_all, b->smem_all, s);
  if (n < 0 || n > b->W) return fail(CF_ERR_INVALID_ARGUMENT, "bad world count %d", n);
  std::vector<int> list(worlds, worlds + n), seen(b->W, 0);
  for (int w : list) {
    if (w < 0 || w >= b->W) return fail(CF_ERR_INVALID_ARGUMENT, "world index %d out of range", w);
    if (seen[w]++) return fail(CF_ERR_INVALID_ARGUMENT, "world index %d repeated", w);
  }
  std::vector<int> order;
  std::vector<DUnit> units;
  size_t smem = 0;
  bool artic = false;
  build_units(b, list, order, units, smem, artic);
  if (units.empty()) return CF_OK;
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.sub_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s),
          "upload subset");
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.sub_units, units.data(), sizeof(DUnit) * units.size(), cudaMemcpyHostToDevice, s),
          "upload subset");
  p.order = b->at<int>(b->L.sub_order);
  p.units = b->at<DUnit>(b->L.sub_units);
  set_work(p, units, order.size(), b->allow_group);
  cf_status st = launch(b, p, artic, smem, s);
  // the host lists above are pageable: the copies completed before cudaMemcpyAsync returned
  return st;
}

extern "C" cf_status cf_get_contact_counts(const cf_batch* b, int32_t* counts, int32_t on_device, void* stream) {
  if (!b || !counts) return fail(CF_ERR_INVALID_ARGUMENT, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  CF_CUDA(cudaMemcpyAsync(counts, b->ws + b->L.ncontact, sizeof(int) * b->W,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
          "contact counts");
  if (!on_device) CF_CUDA(cudaStreamSynchronize(s), "contact counts");
  return CF_OK;
}

extern "C" cf_status cf_get_contacts(const cf_batch* b, cf_contact* out, int32_t* counts, void* stream) {
  if (!b || !out || !counts) return fail(CF_ERR_INVALID_ARGUMENT, "null argument");
  if (b->opts.contact_capture <= 0) return fail(CF_ERR_UNSUPPORTED, "contact capture is off for this batch");
  cudaStream_t s = (cudaStream_t)stream;
  CF_CUDA(cudaMemcpyAsync(out, b->ws + b->L.capture, sizeof(cf_contact) * (size_t)b->W * b->opts.contact_capture,
                          cudaMemcpyDeviceToHost, s),
          "contacts");
  CF_CUDA(cudaMemcpyAsync(counts, b->ws + b->L.ncontact, sizeof(int) * b->W, cudaMemcpyDeviceToHost, s), "counts");
  CF_CUDA(cudaStreamSynchronize(s), "contacts");
  for (int w = 0; w < b->W; ++w)
    if (counts[w] > b->opts.contact_capture)
      return fail(CF_ERR_CONTACT_OVERFLOW, "world %d had %d contacts, capacity %d", w, counts[w], b->opts.contact_capture);
  return CF_OK;
}

extern "C" cf_status cf_batch_status(cf_batch* b, int32_t* flags, int32_t clear, void* stream) {
  if (!b) return fail(CF_ERR_INVALID_ARGUMENT, "null batch");
  cudaStream_t s = (cudaStream_t)stream;
  int word = 0;
  if (flags) CF_CUDA(cudaMemcpyAsync(flags, b->ws + b->L.flags, sizeof(int) * b->W, cudaMemcpyDeviceToHost, s), "flags");
  cf_status st = read_errword(b, s, &word);
  if (st != CF_OK) return st;
  if (clear) {
    CF_CUDA(cudaMemsetAsync(b->ws + b->L.flags, 0, sizeof(int) * b->W, s), "clear flags");
    CF_CUDA(cudaMemsetAsync(b->ws + b->L.errword, 0, sizeof(int) * 4, s), "clear flags");
    CF_CUDA(cudaStreamSynchronize(s), "clear flags");
  }
  return status_of_word(word);
}

extern "C" cf_status cf_batch_set_warps(cf_batch* b, int32_t scene, int32_t warps) {
  if (!b || scene < 0 || scene >= (int)b->model.scenes.size()) return fail(CF_ERR_INVALID_ARGUMENT, "bad scene");
  if (warps != 1 && warps != 2 && warps != 4 && warps != 8) return fail(CF_ERR_INVALID_ARGUMENT, "warps must be 1/2/4/8");
  int old = b->warps[scene];
  b->warps[scene] = warps;
  cf_status st = upload_units(b, 0);
  if (st != CF_OK) {
    b->warps[scene] = old;
    upload_units(b, 0);
  }
  return st;
}

extern "C" cf_status cf_batch_autotune(cf_batch* b, float dt, void* stream, int32_t* chosen) {
  if (!b || !(dt > 0.f)) return fail(CF_ERR_INVALID_ARGUMENT, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  // save the state, time each candidate on the worlds of one scene, restore
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.backup, b->ws + b->L.q, sizeof(float) * b->total_nq, cudaMemcpyDeviceToDevice, s),
          "autotune backup");
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.backup + sizeof(float) * b->total_nq, b->ws + b->L.v, sizeof(float) * b->total_nv,
                          cudaMemcpyDeviceToDevice, s),
          "autotune backup");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (size_t sc = 0; sc < b->model.scenes.size(); ++sc) {
    std::vector<int> list;
    for (int w = 0; w < b->W; ++w)
      if (b->worlds[w].scene == (int)sc) list.push_back(w);
    if (list.empty()) continue;
    const int cands_pile[] = {1, 2, 4, 8};
    const int cands_artic[] = {1, 2};
    const int* cands = b->model.scenes[sc].pile ? cands_pile : cands_artic;
    int nc = b->model.scenes[sc].pile ? 4 : 2;
    float best = 3e38f;
    int best_w = b->warps[sc];
    for (int c = 0; c < nc; ++c) {
      b->warps[sc] = cands[c];
      std::vector<int> order;
      std::vector<DUnit> units;
      size_t smem = 0;
      bool artic = false;
      build_units(b, list, order, units, smem, artic);
      if (smem > step_max_dynamic_smem()) continue;
      cudaMemcpyAsync(b->ws + b->L.sub_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(b->ws + b->L.sub_units, units.data(), sizeof(DUnit) * units.size(), cudaMemcpyHostToDevice, s);
      StepParams p = make_params(b, dt, 1);
      p.order = b->at<int>(b->L.sub_order);
      p.units = b->at<DUnit>(b->L.sub_units);
      set_work(p, units, order.size(), b->allow_group);
      cf_status st = launch(b, p, artic, smem, s);  // warm-up
      if (st != CF_OK) return st;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) launch(b, p, artic, smem, s);
      cudaEventRecord(e1, s);
      CF_CUDA(cudaEventSynchronize(e1), "autotune timing");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_w = cands[c];
      }
    }
    b->warps[sc] = best_w;
    if (chosen) chosen[sc] = best_w;
  }
  // occupancy variant of the pile kernel, timed on the whole batch with the chosen warps
  {
    cf_status st = upload_units(b, s);
    if (st != CF_OK) return st;
    if (!b->artic_all && !b->ext && !b->imp) {
      float best = 3e38f;
      int best_v = 0, prev_blocks = 0;
      for (int var = 0; var < kPileVariants; ++var) {
        // a variant built for more resident blocks only pays when the shared memory lets
        // those blocks in; otherwise it just spills
        const int blocks = step_max_blocks_per_sm(false, var, b->smem_all);
        if (blocks <= prev_blocks) continue;
        prev_blocks = blocks;
        b->variant = var;
        StepParams p = make_params(b, dt, 1);
        st = launch(b, p, false, b->smem_all, s);
        if (st != CF_OK) return st;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch(b, p, false, b->smem_all, s);
        cudaEventRecord(e1, s);
        CF_CUDA(cudaEventSynchronize(e1), "autotune timing");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_v = var; }
      }
      b->variant = best_v;
    }
    // CTAs pulling units of worlds, or (every world of the batch with the same warps) warp
    // groups pulling worlds by themselves: timed on the whole batch
    if (uniform_warps(b->units) > 0) {
      float best = 3e38f;
      bool best_g = false;
      for (int g = 0; g < 2; ++g) {
        b->allow_group = g == 1;
        st = upload_units(b, s);
        if (st != CF_OK) return st;
        StepParams p = make_params(b, dt, 1);
        st = launch(b, p, b->artic_all, b->smem_all, s);
        if (st != CF_OK) return st;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch(b, p, b->artic_all, b->smem_all, s);
        cudaEventRecord(e1, s);
        CF_CUDA(cudaEventSynchronize(e1), "autotune timing");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_g = g == 1; }
      }
      b->allow_group = best_g;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.q, b->ws + b->L.backup, sizeof(float) * b->total_nq, cudaMemcpyDeviceToDevice, s),
          "autotune restore");
  CF_CUDA(cudaMemcpyAsync(b->ws + b->L.v, b->ws + b->L.backup + sizeof(float) * b->total_nq, sizeof(float) * b->total_nv,
                          cudaMemcpyDeviceToDevice, s),
          "autotune restore");
  CF_CUDA(cudaStreamSynchronize(s), "autotune");
  return upload_units(b, s);
}

extern "C" cf_status cf_set_cost(cf_batch* b, const cf_cost_desc* desc, const float* goals, const float* qref,
                                 float* costs) {
  if (!b) return fail(CF_ERR_INVALID_ARGUMENT, "null batch");
  if (!desc) {
    b->cost = nullptr;
    return CF_OK;
  }
  if (!goals || !qref || !costs) return fail(CF_ERR_INVALID_ARGUMENT, "goals, qref and costs are required");
  for (int w = 0; w < b->W; ++w) {
    const DScene& sc = b->model.scenes[b->worlds[w].scene];
    if (sc.pile) return fail(CF_ERR_UNSUPPORTED, "the fused MPC cost covers articulated scenes only");
    if (desc->body < 0 || desc->body >= sc.nbody || b->model.bodies[sc.body0 + desc->body].jnt != CF_JOINT_FREE)
      return fail(CF_ERR_INVALID_ARGUMENT, "cost body %d is not a free body of world %d", desc->body, w);
  }
  b->cost = costs;
  b->goal = goals;
  b->qref = qref;
  b->cost_body = desc->body;
  b->cw[0] = desc->w_quat; b->cw[1] = desc->w_pos; b->cw[2] = desc->w_contact; b->cw[3] = desc->w_joint;
  b->cw[4] = desc->w_fallen; b->cw[5] = desc->fall_radius; b->cw[6] = desc->term_pos; b->cw[7] = desc->term_quat;
  return CF_OK;
}

extern "C" cf_status cf_batch_set_impedance_net(cf_batch* b, const float* theta, int32_t n_sets) {
  if (!b) return fail(CF_ERR_INVALID_ARGUMENT, "null batch");
  if (!theta) {
    b->impnet = nullptr;
    b->impnet_stride = 0;
    return CF_OK;
  }
  if (n_sets != 1 && n_sets != b->W)
    return fail(CF_ERR_INVALID_ARGUMENT, "n_sets must be 1 or the number of worlds (%d), got %d", b->W, n_sets);
  if (reinterpret_cast<uintptr_t>(theta) & 3u) return fail(CF_ERR_INVALID_ARGUMENT, "theta not 4-byte aligned");
  b->impnet = theta;
  b->impnet_stride = n_sets == 1 ? 0 : kImpParams;
  return CF_OK;
}

extern "C" cf_status cf_step_grad(cf_batch* b, int32_t T, float dt, const float* dL_dqT, const float* dL_dvT,
                                  float* dL_dq0, float* dL_dv0, float* dL_dtau, void* stream) {
  if (!b) return fail(CF_ERR_INVALID_ARGUMENT, "null batch");
  if (b->opts.grad_steps <= 0) return fail(CF_ERR_UNSUPPORTED, "batch created without an adjoint tape (grad_steps = 0)");
  if (b->model.trace_mode == 3 && !b->impnet)
    return fail(CF_ERR_INVALID_ARGUMENT, "trace_mode 3 needs an impedance network (cf_batch_set_impedance_net)");
  if (T < 1 || T > b->opts.grad_steps || T > b->opts.max_ctrl_steps)
    return fail(CF_ERR_INVALID_ARGUMENT, "T = %d outside [1, min(grad_steps, max_ctrl_steps)]", T);
  if (!(dt > 0.f)) return fail(CF_ERR_INVALID_ARGUMENT, "dt must be positive");
  if (!dL_dqT || !dL_dvT || !dL_dq0 || !dL_dv0) return fail(CF_ERR_INVALID_ARGUMENT, "null gradient buffer");
  for (int w = 0; w < b->W; ++w) {
    const char* why = nullptr;
    if (!grad_scene_supported(b->model.scenes[b->worlds[w].scene], &why))
      return fail(CF_ERR_UNSUPPORTED, "world %d: %s", w, why);
  }
  StepParams p = make_params(b, dt, 1);
  p.cost = nullptr;
  GradArgs g{};
  g.T = T;
  g.ckpt = b->opts.grad_ckpt;
  g.W = b->W;
  g.total_nq = b->total_nq;
  g.total_nv = b->total_nv;
  g.total_nu = b->total_nu;
  g.tape = b->ws + b->L.grad;
  g.dqT = dL_dqT;
  g.dvT = dL_dvT;
  g.dq0 = dL_dq0;
  g.dv0 = dL_dv0;
  g.dtau = b->total_nu > 0 ? dL_dtau : nullptr;
  g.num_sms = b->num_sms;
  g.smem = b->smem_all;
  // the impedance modes, box-box pairs, cylinders and ellipsoids live in the extended kernel
  g.variant = (b->imp || b->ext) ? kExtVariant : 0;
  cudaError_t e = run_grad(p, g, b->nctrl, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint");
  return CF_OK;
}

extern "C" const char* cf_status_string(cf_status s) {
  switch (s) {
    case CF_OK: return "CF_OK";
    case CF_ERR_INVALID_ARGUMENT: return "CF_ERR_INVALID_ARGUMENT";
    case CF_ERR_OUT_OF_MEMORY: return "CF_ERR_OUT_OF_MEMORY";
    case CF_ERR_CUDA: return "CF_ERR_CUDA";
    case CF_ERR_CONTACT_OVERFLOW: return "CF_ERR_CONTACT_OVERFLOW";
    case CF_ERR_NONFINITE: return "CF_ERR_NONFINITE";
    case CF_ERR_TIMEOUT: return "CF_ERR_TIMEOUT";
    case CF_ERR_UNSUPPORTED: return "CF_ERR_UNSUPPORTED";
  }
  return "CF_ERR_UNKNOWN";
}

extern "C" const char* cf_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------------------
// Stepping without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a memory pool whose
// allocations are fixed up front, plugins of hosts that own the CUDA context and forbid
// cudaMalloc, or real-time loops that must not touch the allocator.  cf_step_noalloc
// serves them: the caller passes its state and parameters, and every piece of scratch the
// step needs (scene templates, world records, work units, the work-queue counters, flags)
// lives in one file-scope device array of fixed size that each GPU loading the library keeps
// until the process exits.
// ---------------------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;  // 2 MiB per device
constexpr int kNoAllocMaxWorlds = 16384;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr int kNoAllocMaxDevices = 64;
std::atomic<char*> g_noalloc_ptr[kNoAllocMaxDevices];  // static storage: starts as null
}  // namespace

extern "C" cf_status cf_step_noalloc(const cf_model* m, int32_t scene, int32_t n_worlds, float* q, float* v,
                                     const float* world_params, float dt, int32_t nsteps, int32_t* contacts,
                                     void* stream) {
  if (!m || !q || !v) return fail(CF_ERR_INVALID_ARGUMENT, "null argument");
  if (scene < 0 || scene >= (int)m->scenes.size()) return fail(CF_ERR_INVALID_ARGUMENT, "scene %d out of range", scene);
  if (n_worlds < 1 || n_worlds > kNoAllocMaxWorlds)
    return fail(CF_ERR_INVALID_ARGUMENT, "cf_step_noalloc takes 1..%d worlds per call, got %d", kNoAllocMaxWorlds,
                n_worlds);
  if (!(dt > 0.f) || !std::isfinite(dt)) return fail(CF_ERR_INVALID_ARGUMENT, "dt must be positive");
  if (nsteps < 1) return fail(CF_ERR_INVALID_ARGUMENT, "nsteps must be >= 1");
  const DScene& sc = m->scenes[scene];
  if (!sc.pile && world_params) return fail(CF_ERR_INVALID_ARGUMENT, "per-world parameters need a pile scene");
  if (m->trace_mode == 3) return fail(CF_ERR_UNSUPPORTED, "cf_step_noalloc has no impedance network (trace_mode 3)");
  // the pile kernel reads the parameter blocks as float4
  if (reinterpret_cast<uintptr_t>(world_params) & 15)
    return fail(CF_ERR_INVALID_ARGUMENT, "world_params must be 16-byte aligned");
  // the uploads below come from host memory local to this call: a graph could not replay them
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)
      return fail(CF_ERR_UNSUPPORTED, "cf_step_noalloc does not run while its stream is being captured");
  }

  // layout of the static scratch for this call
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return r;
  };
  const size_t o_scenes = take(sizeof(DScene) * m->scenes.size());
  const size_t o_bodies = take(sizeof(DBody) * std::max<size_t>(m->bodies.size(), 1));
  const size_t o_geoms = take(sizeof(DGeom) * m->geoms.size());
  const size_t o_trees = take(sizeof(DTree) * std::max<size_t>(m->trees.size(), 1));
  const size_t o_pairs = take(sizeof(uint32_t) * std::max<size_t>(m->pairs.size(), 1));
  const size_t o_worlds = take(sizeof(DWorld) * n_worlds);
  const size_t o_order = take(sizeof(int) * n_worlds);
  const size_t o_units = take(sizeof(DUnit) * n_worlds);
  const size_t o_count = take(sizeof(int) * n_worlds);
  const size_t o_flags = take(sizeof(int) * n_worlds);
  const size_t o_words = take(sizeof(int) * 8);  // [0..3] error word, [4..7] work-queue counters
  if (off > kNoAllocScratchBytes)
    return fail(CF_ERR_INVALID_ARGUMENT, "model and %d worlds need %zu bytes, more than the %zu-byte static scratch",
                n_worlds, off, kNoAllocScratchBytes);

  // once per device, with that device current: the device address of the static array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(CF_ERR_UNSUPPORTED, "device ordinal %d", dev);
  char* base = g_noalloc_ptr[dev].load();
  if (!base) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    base = static_cast<char*>(ptr);
    g_noalloc_ptr[dev].store(base);  // every thread that looks it up finds the same address
  }

  // host-side records: worlds of one scene packed back to back, units of kWarps / warps worlds
  const int warps = default_warps(sc);
  const int per = kWarps / warps;
  std::vector<DWorld> worlds(n_worlds);
  std::vector<int> order(n_worlds);
  std::vector<DUnit> units;
  for (int w = 0; w < n_worlds; ++w) {
    DWorld d{};
    d.scene = scene;
    d.qadr = w * sc.nq;
    d.vadr = w * sc.nv;
    d.uadr = 0;
    d.padr = (sc.pile && world_params) ? w * 8 * sc.nbody : -1;
    worlds[w] = d;
    order[w] = w;
  }
  for (int w = 0; w < n_worlds; w += per) {
    DUnit u{};
    u.first = w;
    u.count = std::min(per, n_worlds - w);
    u.warps = warps;
    units.push_back(u);
  }
  cudaStream_t s = (cudaStream_t)stream;
  auto up = [&](size_t o, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  // the host vectors are pageable: each copy has been taken before cudaMemcpyAsync returns
  e = up(o_scenes, m->scenes.data(), sizeof(DScene) * m->scenes.size());
  if (e == cudaSuccess) e = up(o_bodies, m->bodies.data(), sizeof(DBody) * m->bodies.size());
  if (e == cudaSuccess) e = up(o_geoms, m->geoms.data(), sizeof(DGeom) * m->geoms.size());
  if (e == cudaSuccess) e = up(o_trees, m->trees.data(), sizeof(DTree) * m->trees.size());
  if (e == cudaSuccess) e = up(o_pairs, m->pairs.data(), sizeof(uint32_t) * m->pairs.size());
  if (e == cudaSuccess) e = up(o_worlds, worlds.data(), sizeof(DWorld) * n_worlds);
  if (e == cudaSuccess) e = up(o_order, order.data(), sizeof(int) * n_worlds);
  if (e == cudaSuccess) e = up(o_units, units.data(), sizeof(DUnit) * units.size());
  // the array keeps the previous call's contents: zero the error word, queue counters, flags
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_words, 0, sizeof(int) * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_flags, 0, sizeof(int) * n_worlds, s);
  if (e != cudaSuccess) return cuda_fail(e, "static scratch upload");

  StepParams p{};
  p.scenes = reinterpret_cast<const DScene*>(base + o_scenes);
  p.bodies = reinterpret_cast<const DBody*>(base + o_bodies);
  p.geoms = reinterpret_cast<const DGeom*>(base + o_geoms);
  p.trees = reinterpret_cast<const DTree*>(base + o_trees);
  p.pairs = reinterpret_cast<const uint32_t*>(base + o_pairs);
  p.worlds = reinterpret_cast<const DWorld*>(base + o_worlds);
  p.units = reinterpret_cast<const DUnit*>(base + o_units);
  p.order = reinterpret_cast<const int*>(base + o_order);
  p.nunits = (int)units.size();
  p.q = q;
  p.v = v;
  p.wparam = world_params;
  p.ctrl = nullptr;
  p.total_nu = 0;
  p.nctrl = 0;
  p.ctrl_offset = 0;
  p.ncontact = contacts ? contacts : reinterpret_cast<int*>(base + o_count);
  p.flags = reinterpret_cast<int*>(base + o_flags);
  p.errword = reinterpret_cast<int*>(base + o_words);
  p.queue = reinterpret_cast<int*>(base + o_words) + 4;
  p.capture = nullptr;
  p.capture_cap = 0;
  p.dt = dt;
  p.nsteps = nsteps;
  for (int k = 0; k < 3; ++k) p.gravity[k] = m->gravity[k];
  p.k_user = m->k_user;
  p.d_user = m->d_user;
  for (int k = 0; k < 5; ++k) p.solimp[k] = m->solimp[k];
  p.margin = m->margin;
  p.n_t = m->n_t;
  p.n_tor = m->n_tor;
  p.n_rol = m->n_rol;
  p.trace_mode = m->trace_mode;
  for (int j = 0; j < m->n_t; ++j) {
    double th = 2.0 * M_PI * j / m->n_t;
    p.tcos[j] = (float)std::cos(th);
    p.tsin[j] = (float)std::sin(th);
  }
  for (int j = 0; j < m->n_rol; ++j) {
    double th = 2.0 * M_PI * j / m->n_rol;
    p.rcos[j] = (float)std::cos(th);
    p.rsin[j] = (float)std::sin(th);
  }
  const bool artic = !sc.pile;
  // per-world override blocks live on the device here, so a pile with overrides may hold boxes
  const int var = (sc.boxbox || (sc.pile && world_params)) ? kExtVariant : (m->trace_mode == 2 ? kImpVariant : 0);
  const size_t smem = world_smem_bytes(sc, warps) * per;
  if (smem > step_max_dynamic_smem()) return fail(CF_ERR_UNSUPPORTED, "a world needs %zu bytes of shared memory", smem);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = step_max_blocks_per_sm(artic, var, smem);
  const int grid = std::min(p.nunits, std::max(1, nsm * per_sm));
  e = launch_step(p, artic, var, grid, smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "step launch");
  return CF_OK;
}
