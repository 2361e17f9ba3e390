// Internal device-side data layout of libcomfree (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "comfree.h"

namespace cf {

constexpr int kBlock = 256;           // threads per CTA of the step kernel
constexpr int kWarps = kBlock / 32;
constexpr int kQueue = 64;            // per-warp candidate queue (entries)
constexpr int kMaxFacetDirs = 16;     // n_t, n_rol <= 16
constexpr int kMaxTreeDof = 8;        // hinge DoFs per tree handled by the articulated path
constexpr float kFixScale = 1099511627776.0f;          // 2^40: fixed-point impulse quantum
constexpr float kFixInv = 9.094947017729282e-13f;      // 2^-40
constexpr float kFixClamp = 8.0e6f;                    // |impulse| clamp before conversion
// two-word velocity-change accumulators of pile worlds: x = hi 2^-16 + lo 2^-36
constexpr float kFix2Hi = 65536.0f;                    // 2^16
constexpr float kFix2Lo = 1048576.0f;                  // 2^20 (fraction bits of the low word)
constexpr float kFix2HiInv = 1.52587890625e-05f;       // 2^-16
constexpr float kFix2LoInv = 1.4551915228366852e-11f;  // 2^-36
constexpr float kFix2Range = 4096.0f;                  // |dv| per contribution; larger raises CF_FLAG_RANGE
// learned impedance network (trace_mode 3): inputs, tanh hidden units, parameters, output clamp
constexpr int kImpIn = 4;
constexpr int kImpHidden = 8;
constexpr int kImpParams = kImpHidden * kImpIn + 2 * kImpHidden + 1;
constexpr float kImpClamp = 8.0f;

// ---------------------------------------------------------------------------------------
// scene templates (uploaded once per batch into the workspace)
// ---------------------------------------------------------------------------------------
struct alignas(16) DScene {
  int nbody, ngeom, nq, nv;
  int nu, ntree, pile, nplane;
  int body0, geom0, tree0, pair0;
  int npair, plane0, maxdepth, joints;  // joints: some hinge is limited or has dry friction
  int boxbox, pad1, pad2, pad3;         // boxbox: needs the extended kernel (two boxes, cylinders, ellipsoids)
  float mu[3];                          // every geom's friction coefficients, when they are all equal:
  int mu_uniform;                       // then every pair's friction is mu (else 0)
};

struct alignas(16) DBody {
  int parent, jnt, qoff, voff;      // parent is scene-local, offsets world-local
  int uoff, tree, anc, pad1;        // uoff: actuator slot of a hinge, -1 otherwise; anc: bit i set
                                    // when the tree's i-th body is this body or one of its ancestors
  float pos[3], quat[4], axis[3], ipos[3], mass, inertia[3], damping, frictionloss;
  float range[2];                   // hinge limits (used when limited != 0)
  int limited, pad3[3];
};

struct alignas(16) DGeom {
  int type, body, tip, pad1;        // tip: a capsule on a hinge body with no child (a fingertip
                                    // of the MPC cost)
  float pos[3], quat[4], size[3], mu[3], pad2[3];
};

struct alignas(16) DTree {
  int body0, nbody, voff, nv;
  int free, pad0, pad1, pad2;
};

struct alignas(16) DWorld {
  int scene, qadr, vadr, padr;
  int uadr, pad0, pad1, pad2;
};

struct alignas(16) DUnit {
  int first, count, warps, pad;     // worlds order[first .. first+count) processed by groups
};

// ---------------------------------------------------------------------------------------
// launch parameters
// ---------------------------------------------------------------------------------------
struct StepParams {
  const DScene* scenes;
  const DBody* bodies;
  const DGeom* geoms;
  const DTree* trees;
  const uint32_t* pairs;     // (ga << 16) | gb, scene-local geom indices
  const DWorld* worlds;
  const DUnit* units;
  const int* order;
  int nunits;                // units (group_warps 0) or worlds in order (group_warps > 0)
  int group_warps;           // > 0: every world takes this many warps and each warp group
                             // pulls worlds from order[] by itself; 0: CTAs pull units
  float* q;
  float* v;
  const float* wparam;
  const float* ctrl;
  int total_nu;
  int nctrl;
  int ctrl_offset;           // control slice of the launch's first step
  int* ncontact;
  int* flags;
  int* errword;
  int* queue;                // [0] next unit, [1] finished CTAs (self-resetting)
  cf_contact* capture;
  int capture_cap;
  float dt;
  int nsteps;
  float gravity[3];
  float k_user, d_user;
  float solimp[5];
  float margin;
  int n_t, n_tor, n_rol, trace_mode;
  const float* impnet;       // trace_mode 3: [sets][kImpParams] network parameters
  int impnet_stride;         // floats between worlds' parameter sets (0: one shared set)
  float tcos[kMaxFacetDirs], tsin[kMaxFacetDirs];
  float rcos[kMaxFacetDirs], rsin[kMaxFacetDirs];
  // fused MPC cost of articulated worlds (cost == nullptr: off)
  float* cost;               // [W] += running cost of every step + terminal cost
  const float* goal;         // [W][7] target position and quaternion
  const float* qref;         // [total_nq] home pose (hinge coordinates used)
  int cost_body;             // the free body whose pose is scored
  float cw[8];               // quat, pos, contact, joint, fallen penalty, fall radius, terminal pos, terminal quat
};

// thread-local message returned by cf_last_error (set by every failing entry point)
void set_last_error(const char* msg);

// bytes of dynamic shared memory one world of a scene needs in the step kernel
size_t world_smem_bytes(const DScene& s, int warps);

// artic = the launch contains worlds of non-pile scenes (selects the kernel instantiation);
// variant 0..2 = pile-only kernel compiled for 2, 3 or 4 resident CTAs per SM
constexpr int kStepVariants = 6;
constexpr int kPileVariants = 3;
constexpr int kExtImp = 1;       // step-kernel feature: exact and learned impedances (trace_mode 2, 3)
constexpr int kExtGeo = 2;       // step-kernel feature: box-box contacts, cylinders, ellipsoids
constexpr int kExtVariant = 99;  // the extended kernel: articulated worlds and every feature
constexpr int kImpVariant = 98;  // the impedance modes without the extra geometry (pile-only
                                 // kernel unless the launch holds articulated worlds)
cudaError_t launch_step(const StepParams& p, bool artic, int variant, int grid, size_t smem, cudaStream_t stream);
int step_max_blocks_per_sm(bool artic, int variant, size_t smem);
size_t step_max_dynamic_smem();

}  // namespace cf
