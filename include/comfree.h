/*
 * comfree.h -- C ABI of libcomfree, the GB300 (sm_103a) batched ComFree contact step.
 *
 * The library advances thousands of independent rigid-body worlds with the
 * complementarity-free contact model of ComFree-Sim (arxiv 2603.12185): a contact-free
 * velocity prediction (Eq. smooth_vel), closed-form impulses on the facets of the polyhedral
 * dual friction cone (Eqs. dual_polyhedral, tilde_defs, cf_wrench) with the heuristic
 * impedance (Eqs. k_d_setting, r_scaling), the J~^T lambda scatter and M^-1 correction
 * (Eq. vel_correction, Algorithm 1 Kernels I-IV), followed by semi-implicit integration.
 *
 * Conventions
 *   - Ownership: model and batch handles belong to the library (create/destroy pairs).  All
 *     device memory belongs to the caller: cf_batch_create receives a caller-allocated device
 *     workspace (e.g. a torch uint8 tensor) and the library never calls cudaMalloc for it.
 *     Pointers passed to a call are borrowed for the duration of that call only.
 *   - Precision: state, controls and model quantities are FP32 on the device; the model
 *     description is read in FP64 on the host and rounded once.
 *   - State layout: world-major and contiguous.  World w owns nq(scene) floats of q and
 *     nv(scene) floats of v, in world order.  Per body: a free body holds q = (x, y, z, qw, qx,
 *     qy, qz) and v = (world linear velocity, body-frame angular velocity); a hinge holds its
 *     angle and rate.  Bodies appear in scene order.
 *   - Streams: every device operation is enqueued on the stream passed in (a cudaStream_t
 *     handed over as void*; NULL = legacy default stream).  Host-pointer variants synchronise
 *     that stream before returning.
 *   - Errors: no exception crosses the ABI; every call returns a cf_status.  cf_last_error()
 *     gives a thread-local human-readable message for the most recent failure.  Device-side
 *     conditions (non-finite state, contact-capture overflow, a bounded wait that gave up) are
 *     latched into per-world flags and an error word in the workspace and reported by the next
 *     call that synchronises (cf_batch_status, cf_get_state with host buffers).
 */
#ifndef COMFREE_H
#define COMFREE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CF_OK = 0,
  CF_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, index or description            */
  CF_ERR_OUT_OF_MEMORY = 2,    /* host allocation failed / workspace too small        */
  CF_ERR_CUDA = 3,             /* a CUDA runtime call failed (message in cf_last_error) */
  CF_ERR_CONTACT_OVERFLOW = 4, /* contact capture buffer full for some world          */
  CF_ERR_NONFINITE = 5,        /* a world produced a NaN/Inf state or left the range   */
  CF_ERR_TIMEOUT = 6,          /* a bounded device wait gave up                       */
  CF_ERR_UNSUPPORTED = 7       /* a valid but unsupported request                     */
} cf_status;

/* per-world flag bits (cf_batch_status) */
#define CF_FLAG_NONFINITE 1
#define CF_FLAG_CONTACT_OVERFLOW 2
#define CF_FLAG_TIMEOUT 4
#define CF_FLAG_RANGE 8  /* a contact's velocity change left the pile scatter's range (|dv| > 4096 per step) */

/* geom and joint kinds */
#define CF_GEOM_PLANE 0   /* static only; the plane through pos with normal = local +z   */
#define CF_GEOM_SPHERE 1  /* size[0] = radius                                           */
#define CF_GEOM_CAPSULE 2 /* size[0] = radius, size[1] = half length along local z      */
#define CF_GEOM_BOX 3     /* size = half extents                                        */
#define CF_GEOM_CYLINDER 4  /* size[0] = radius, size[1] = half length along local z; touches
                               planes and spheres only                                      */
#define CF_GEOM_ELLIPSOID 5 /* size = semi-axes; touches planes only                        */
#define CF_JOINT_FREE 0
#define CF_JOINT_HINGE 1

typedef struct cf_model cf_model;
typedef struct cf_batch cf_batch;

/* One scene template.  Bodies form a forest in topological order (parent < child): either a
 * free body with no children (its body frame at its centre of mass), or a fixed-base tree of
 * hinges whose bodies are contiguous.  Arrays are host pointers, FP64, read during
 * cf_model_create only.  `pile` != 0 declares the layout "body i is free and carries geom i at
 * its origin; geoms nbody.. are static planes" (at most 4096 bodies and 4096 planes, else
 * CF_ERR_UNSUPPORTED); only such scenes accept per-world overrides. */
typedef struct {
  int32_t nbody, ngeom;
  const int32_t* body_parent;   /* [nbody] parent body or -1                              */
  const int32_t* body_jnt;      /* [nbody] CF_JOINT_*                                     */
  const double* body_pos;       /* [nbody][3] hinge frame origin in the parent frame      */
  const double* body_quat;      /* [nbody][4] hinge frame orientation in the parent frame */
  const double* body_axis;      /* [nbody][3] hinge axis in the body frame                */
  const double* body_ipos;      /* [nbody][3] centre of mass in the body frame            */
  const double* body_mass;      /* [nbody]                                                */
  const double* body_inertia;   /* [nbody][3] principal inertia about the centre of mass  */
  const double* body_damping;   /* [nbody] hinge damping (implicit)                       */
  const int32_t* geom_type;     /* [ngeom] CF_GEOM_*                                      */
  const int32_t* geom_body;     /* [ngeom] body or -1 (static)                            */
  const double* geom_pos;       /* [ngeom][3] in the body frame (world if static)         */
  const double* geom_quat;      /* [ngeom][4]                                             */
  const double* geom_size;      /* [ngeom][3]                                             */
  const double* geom_mu;        /* [ngeom][3] tangential, torsional, rolling coefficients */
  int32_t pile;
  const double* body_range;     /* [nbody][2] hinge limits (lower, upper), nullable; a hinge
                                   with lower < upper is limited (Sec. III-A)             */
  const double* body_frictionloss; /* [nbody] hinge dry friction (N m, >= 0), nullable     */
} cf_scene_desc;

/* Global model parameters (one set per model). */
typedef struct {
  int32_t nscene;
  const cf_scene_desc* scenes;
  double gravity[3];
  double k_user, d_user;   /* Eq. k_d_setting global impedance                           */
  double solimp[5];        /* Eq. r_scaling (r_min, r_max, width, midpoint, power)        */
  double margin;           /* contact when the signed gap phi < margin                   */
  int32_t n_t, n_tor, n_rol; /* facets per subspace (Eq. tilde_defs); n_tor in {0, 2},
                                n_t and n_rol in {0, 2..16} (symmetric unit directions)  */
  int32_t trace_mode;      /* 0: M(phi) with tr(J_i M~^-1 J_i^T) of body i's translational
                              point Jacobian; 1: 1/m_i per body; 2: the exact diagonal
                              impedance of Sec. III-B instead of M(phi): per facet j,
                              M_j = 1 / ((k_user dt + d_user) J~_j M~^-1 J~_j^T) (solimp
                              unused); 3: the learned impedance of Sec. III-B's
                              learning-based K(q), D(q): mode 0's M(phi) times
                              exp(clamp(g(x), -8, 8)), g the network of
                              cf_batch_set_impedance_net (joint limits keep mode 0;
                              cf_step_noalloc answers CF_ERR_UNSUPPORTED).  cf_step_grad
                              differentiates all four modes */
} cf_model_desc;

/* Validate a description and build the host model.  Errors: CF_ERR_INVALID_ARGUMENT for a
 * malformed description (index out of range, non-topological parents, non-positive mass or
 * inertia, a plane attached to a body, bad facet counts), CF_ERR_UNSUPPORTED for structures
 * outside the forest rules above, CF_ERR_OUT_OF_MEMORY. */
cf_status cf_model_create(const cf_model_desc* desc, cf_model** out);
void cf_model_destroy(cf_model* model);

/* per-model sizes of one scene: nq, nv, nu (actuated hinge DoFs), nbody, ngeom */
cf_status cf_scene_sizes(const cf_model* model, int32_t scene, int32_t sizes[5]);

/* Batch options. */
typedef struct {
  int32_t max_ctrl_steps;  /* capacity T of the control sequence [T][sum nu] (>= 1)       */
  int32_t contact_capture; /* per-world capacity of the contact record buffer (0 = off)   */
  int32_t grad_steps;      /* capacity (steps) of the adjoint tape; 0 = no cf_step_grad    */
  int32_t grad_ckpt;       /* checkpoint interval of the adjoint (>= 1)                   */
} cf_batch_opts;

/* Device bytes the caller must provide for a batch of n_worlds worlds whose scene indices are
 * scene_of_world[n_worlds] (host).  world_params may be NULL for the size query. */
cf_status cf_batch_workspace_bytes(const cf_model* model, int32_t n_worlds, const int32_t* scene_of_world,
                                   const cf_batch_opts* opts, size_t* bytes);

/* Create a batch inside the caller's device workspace (at least cf_batch_workspace_bytes,
 * 256-byte aligned).  world_params (host, nullable) holds, in world order, one block of 8
 * floats per body for every world of a pile scene: mass, I1, I2, I3, geom type (sphere,
 * capsule, box, cylinder or ellipsoid), size0, size1, size2; worlds of other scenes contribute
 * nothing.  NULL keeps the
 * scene defaults.  The initial state is the scene's zero state (identity poses) until
 * cf_set_state.  The workspace must outlive the batch.  Synchronises `stream`. */
cf_status cf_batch_create(const cf_model* model, int32_t n_worlds, const int32_t* scene_of_world,
                          const float* world_params, const cf_batch_opts* opts, void* device_workspace,
                          size_t workspace_bytes, void* stream, cf_batch** out);
void cf_batch_destroy(cf_batch* batch);

/* total floats of q, v and actuated controls over all worlds */
cf_status cf_batch_sizes(const cf_batch* batch, int64_t* total_nq, int64_t* total_nv, int64_t* total_nu);

/* Copy the full state in (set) or out (get).  q[total_nq], v[total_nv]; on_device: 1 = device
 * pointers (asynchronous on `stream`); 0 = host pointers (the call synchronises and, for get,
 * reports latched device errors); 2 = pinned host pointers, asynchronous: the copy is only
 * enqueued on `stream`, the buffers must stay valid until the stream passes it, and device
 * errors wait for the next synchronising call (cf_batch_status). */
cf_status cf_set_state(cf_batch* batch, const float* q, const float* v, int32_t on_device, void* stream);
cf_status cf_get_state(const cf_batch* batch, float* q, float* v, int32_t on_device, void* stream);

/* Control sequence: tau[T][total_nu] generalised forces of the actuated hinges (world order,
 * then hinge order), 1 <= T <= max_ctrl_steps.  Step s of a cf_step call uses slice
 * min(s, T - 1); free bodies are unactuated. */
cf_status cf_set_ctrl(cf_batch* batch, const float* tau, int32_t T, int32_t on_device, void* stream);

/* Advance worlds nsteps steps of length dt (one launch; the state stays on chip across the
 * nsteps).  worlds: NULL = all, else a host list of n distinct world indices.  Errors:
 * CF_ERR_INVALID_ARGUMENT (dt <= 0, nsteps < 1, bad index), CF_ERR_CUDA (launch failure).
 * With worlds == NULL the call enqueues exactly one kernel launch and nothing else, so it may
 * be captured into a CUDA graph (replays then re-run the same dt, nsteps and launch shape);
 * make one uncaptured call first, which sets the kernel's attributes.  The subset form copies
 * its world list from pageable host memory and cannot be captured. */
cf_status cf_step(cf_batch* batch, const int32_t* worlds, int32_t n, float dt, int32_t nsteps, void* stream);

/* cf_step of every world with the state in the caller's host memory: q[total_nq] and
 * v[total_nv] are page-locked host buffers (cudaHostAlloc, cudaHostRegister or a pinned torch
 * tensor), 4-byte aligned, that the step kernel itself reads at the start of the launch and
 * overwrites with the new state at its end, over the host-device link; the batch's device
 * state is neither read nor changed.  No separate copy is enqueued: on a coherent host link
 * (NVLink-C2C) the transfers overlap the other worlds' compute.  Asynchronous on `stream`; the
 * buffers must stay valid until the stream reaches this point.  Errors: CF_ERR_INVALID_ARGUMENT
 * (null batch, a buffer that is not page-locked host memory, bad dt or nsteps), CF_ERR_CUDA. */
cf_status cf_step_host(cf_batch* batch, float* q, float* v, float dt, int32_t nsteps, void* stream);

/* Per-world number of contacts (phi < margin) detected in the last step of the last cf_step,
 * counts[n_worlds] (device or host per on_device). */
cf_status cf_get_contact_counts(const cf_batch* batch, int32_t* counts, int32_t on_device, void* stream);

/* One captured contact (contact_capture > 0): geoms (a, b) with a the geom the normal points
 * to, sub = contact index within the pair (capsule end / box corner), phi, point, normal,
 * the summed facet impulse (lambda dt) and M(phi) (trace_mode 3: the learned impedance;
 * trace_mode 2: 0). */
typedef struct {
  int32_t geom_a, geom_b, sub, flags;  /* flags: CF_CONTACT_B_STATIC when geom_b has no body   */
  float phi, pos[3], normal[3], lam_sum, mphi;
  float rho;      /* trace_mode 2 and 3: the learned impedance's input x1 (below), else 0      */
  float wn;       /* trace_mode 2 and 3: the learned impedance's input x2 (below), else 0      */
  float target;   /* trace_mode 2: ln(M_exact / M(phi)), the learned impedance's regression
                     target, M_exact the mean over the facets of the exact diagonal impedance
                     1 / ((k_user dt + d_user) J~_j M~^-1 J~_j^T), M(phi) the mode-0 heuristic;
                     else 0                                                                    */
} cf_contact;
#define CF_CONTACT_B_STATIC 1

/* Copy the contacts captured in the last step: out[n_worlds][capacity], counts[n_worlds]
 * (host).  Order within a world is unspecified.  CF_ERR_CONTACT_OVERFLOW if a world had more
 * contacts than the capacity (the first `capacity` are kept).  Synchronises. */
cf_status cf_get_contacts(const cf_batch* batch, cf_contact* out, int32_t* counts, void* stream);

/* Synchronise and report the latched device error word; flags[n_worlds] (host, nullable)
 * receives the per-world CF_FLAG_* bits.  clear != 0 resets them. */
cf_status cf_batch_status(cf_batch* batch, int32_t* flags, int32_t clear, void* stream);

/* Pick warps-per-world for every scene class of the batch by timing candidate launch shapes
 * on the batch itself (the state is saved and restored).  chosen[nscene] (host, nullable)
 * receives the warps per world.  Synchronises. */
cf_status cf_batch_autotune(cf_batch* batch, float dt, void* stream, int32_t* chosen);
/* Set warps-per-world of one scene class explicitly (1, 2, 4 or 8). */
cf_status cf_batch_set_warps(cf_batch* batch, int32_t scene, int32_t warps);

/* Reverse-mode gradient of a T-step rollout from the current state with the current control
 * sequence (T <= min(grad_steps, max_ctrl_steps); step s uses control slice s).  Given the
 * cotangents of the final state dL_dqT[total_nq], dL_dvT[total_nv] (device), writes
 * dL_dq0[total_nq], dL_dv0[total_nv] and dL_dtau[T][total_nu] (device).  The forward state is
 * recomputed from checkpoints every grad_ckpt steps.  The batch state is left at the rollout's
 * final state.  The differentiable set: hinge trees (with joint limits and dry joint friction)
 * and free bodies with every geom type (sphere, capsule, box, cylinder, ellipsoid, plane;
 * box-box pairs through their clipped face vertices), under every impedance mode (the
 * heuristic ones, trace_mode 0 and 1; the exact, 2, through each facet's J~_j M~^-1 J~_j^T;
 * the learned, 3, through the network's inputs); at a kink (a facet or a limit turning on,
 * friction saturating, a narrowphase branch, a clamp of the network's inputs or output) the
 * derivative is that of the branch the state selects (a separating axis, a reference face or
 * a clipped vertex included).  Errors: CF_ERR_UNSUPPORTED for pile scenes and for worlds past
 * the per-world limits (24 bodies, 32 geoms, 48 q, 48 v, 8 trees), CF_ERR_INVALID_ARGUMENT
 * (also trace_mode 3 without an impedance network). */
cf_status cf_step_grad(cf_batch* batch, int32_t T, float dt, const float* dL_dqT, const float* dL_dvT,
                       float* dL_dq0, float* dL_dv0, float* dL_dtau, void* stream);

/* ---------------------------------------------------------------------------------------
 * Sampling MPC (MPPI) around the step, for the in-hand reorientation task of Sec. V.
 * ------------------------------------------------------------------------------------- */
/* Weights of the fused MPC cost (Sec. V, Eq. mpc and the running/terminal costs after it;
 * the paper tunes its weights per object and does not print them).  With the cost set,
 * every cf_step of an articulated world adds, per step, the running cost of the state at the
 * start of the step:
 *   w_quat (1 - (q*^T q)^2) + w_pos (|dx| + |dy| + |dz|) + w_contact sum_tips |p - p_tip|^2
 *   + w_joint |q_hinge - q_ref|^2 + w_fallen [|p_xy - p*_xy| > fall_radius]
 * and, after the last step, the terminal cost term_pos |p - p*|^2 + term_quat (1 - (q*^T q)^2).
 * p, q: position and quaternion of free body `body`; tips: the +z ends of the capsules of leaf
 * hinge bodies. */
typedef struct {
  int32_t body;
  float w_quat, w_pos, w_contact, w_joint, w_fallen, fall_radius, term_pos, term_quat;
} cf_cost_desc;
/* goals[W][7] (target position, quaternion), qref[total_nq] (home pose) and costs[W] are device
 * pointers borrowed until the cost is switched off (desc = NULL).  costs accumulate (+=). */
cf_status cf_set_cost(cf_batch* batch, const cf_cost_desc* desc, const float* goals, const float* qref,
                      float* costs);
/* controls of N rollouts over H steps: sample k < n_prop ~ N(prop_mean, exp(prop_logstd)^2),
 * the others ~ N(mean, sigma^2), clipped to [-limit, limit].  noise[N][H][nu] standard normals
 * (caller-drawn); ctrl[H][N * nu] (the cf_set_ctrl layout for N worlds of nu actuators);
 * samples[N][H][nu].  All device pointers. */
cf_status cf_mppi_sample(int32_t N, int32_t H, int32_t nu, const float* mean, const float* noise, float sigma,
                         float limit, const float* prop_mean, const float* prop_logstd, int32_t n_prop, float* ctrl,
                         float* samples, void* stream);
/* MPPI update: w_k = exp(-(J_k - min J) / lambda), mean = sum w_k U_k / sum w_k (N <= 16384);
 * stats[3] (nullable) = min cost, mean cost, effective sample size. */
cf_status cf_mppi_update(int32_t N, int32_t H, int32_t nu, const float* costs, const float* samples, float lambda,
                         float* mean, float* stats, void* stream);
/* receding horizon: mean[h] <- mean[h + 1] for h < H - 1 */
cf_status cf_mppi_shift(int32_t H, int32_t nu, float* mean, void* stream);
/* out[n] = base[n] + scale * delta[n] (device; out may alias base): a plan corrected by the
 * learned proposal's output (the learned warm start).  n = 0 does nothing. */
cf_status cf_mppi_blend(int32_t n, const float* base, const float* delta, float scale, float* out, void* stream);
/* copy one world's state into W back-to-back worlds */
cf_status cf_broadcast_state(const float* q0, const float* v0, int32_t nq, int32_t nv, int32_t W, float* q, float* v,
                             void* stream);
/* out = clamp(concat(q[nq], v_scale * v[nv], goal[ngoal]), -clamp, clamp): the proposal's
 * input features (velocities scaled to the range of the pose coordinates) */
cf_status cf_mppi_features(const float* q, int32_t nq, const float* v, int32_t nv, float v_scale, const float* goal,
                           int32_t ngoal, float clamp, float* out, void* stream);

/* ---------------------------------------------------------------------------------------
 * Learned proposal for sampling MPC: a 3-layer perceptron in -> hidden -> hidden -> out with
 * GELU, BF16 operands and FP32 accumulation on the tensor cores (the paper's MPPI controller,
 * Sec. V, samples around a warm start only; the learned proposal is this library's addition).
 * Output = Gaussian over an action sequence: out/2 means followed by out/2 log-stds.
 * Parameters are FP32, flat: W1[hidden][kin] b1[hidden] W2[hidden][hidden] b2[hidden]
 * W3[out][hidden] b3[out], kin = in rounded up to a multiple of 64 (padding columns unused).
 * Limits: 1 <= in <= 256, hidden % 128 == 0 (<= 1024), out % 256 == 0 (<= 4096).
 * ------------------------------------------------------------------------------------- */
typedef struct cf_mlp cf_mlp;
cf_status cf_mlp_workspace_bytes(int32_t fin, int32_t hidden, int32_t fout, int32_t max_batch, size_t* bytes);
/* params: device FP32 initial parameters (copied); workspace: caller-owned, 256-byte aligned */
cf_status cf_mlp_create(int32_t fin, int32_t hidden, int32_t fout, int32_t max_batch, const float* params,
                        void* device_workspace, size_t bytes, void* stream, cf_mlp** out);
void cf_mlp_destroy(cf_mlp* mlp);
cf_status cf_mlp_param_count(const cf_mlp* mlp, int64_t* n);
/* y[B][out] = MLP(x[B][in]) (device pointers, FP32 in and out) */
cf_status cf_mlp_forward(cf_mlp* mlp, const float* x, int32_t B, float* y, void* stream);
/* Gradient of the mean Gaussian negative log-likelihood of target[B][out/2] under the output
 * (log-stds clamped to [lo, hi]); grads[n_params] and loss[1] are device pointers (nullable).
 * The gradients are bitwise reproducible: every sum runs in a fixed order (split-K slices and
 * the bias gradients' partial sums are added in order).  The loss adds one partial per block
 * with an atomic, so its last bits may vary from call to call. */
cf_status cf_mlp_gradients(cf_mlp* mlp, const float* x, const float* target, int32_t B, float logstd_lo,
                           float logstd_hi, float* grads, float* loss, void* stream);
/* one Adam step (beta 0.9/0.999, eps 1e-8) on that loss */
cf_status cf_mlp_train_step(cf_mlp* mlp, const float* x, const float* target, int32_t B, float lr, float logstd_lo,
                            float logstd_hi, float* loss, void* stream);
cf_status cf_mlp_get_params(const cf_mlp* mlp, float* params, void* stream);
/* synchronise; CF_ERR_TIMEOUT if a tensor-core pipeline wait gave up */
cf_status cf_mlp_status(cf_mlp* mlp, void* stream);

/* Step n_worlds worlds of one scene with no device allocation at all, for callers that cannot
 * allocate device memory (a host that owns the CUDA context and forbids cudaMalloc, a fixed
 * memory pool, a real-time loop that must not touch the allocator).  The paper has no
 * counterpart: this is a deployment convenience around the same step kernel.
 *   q[n_worlds * nq], v[n_worlds * nv]  device, the worlds' states back to back (in/out);
 *   world_params                        device, nullable, 16-byte aligned (the kernel reads it
 *                                       as float4; a misaligned pointer is refused with
 *                                       CF_ERR_INVALID_ARGUMENT before any launch); pile scenes
 *                                       only: one 8-float block per body per world, as in
 *                                       cf_batch_create.  The blocks are not validated (a zero
 *                                       mass or an unknown geom type gives undefined results).
 *                                       A pile call with world_params always runs the kernel
 *                                       instantiation with every optional feature compiled in
 *                                       (the blocks may hold boxes), which is slower than the
 *                                       batch path's pile kernel; without world_params the
 *                                       scene's own bodies and geoms are used;
 *   contacts                            device, nullable; per-world contact counts (out).
 * Controls are zero.  All scratch (scene templates, world records, work units, work-queue
 * counters, flags) lives in a file-scope 2 MiB device array that every GPU loading the library
 * holds until the process exits; at most 16384 worlds per call, and the model plus the worlds'
 * records must fit the array (CF_ERR_INVALID_ARGUMENT otherwise).  The first call on a device
 * looks up the array's device address (make that first call before any stream capture).
 * CF_ERR_UNSUPPORTED while `stream` is being captured: each call uploads its records from host
 * memory that lives only for the call.  Each call clears the counters it needs; every call
 * shares the one array, so calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Device-side flags are not reported by this entry
 * point: neither CF_FLAG_NONFINITE (a non-finite state) nor CF_FLAG_RANGE (a velocity change
 * beyond the scatter's fixed-point range, after which the velocities are wrong); a caller that
 * needs them uses the batch path (cf_batch_status). */
cf_status cf_step_noalloc(const cf_model* model, int32_t scene, int32_t n_worlds, float* q, float* v,
                          const float* world_params, float dt, int32_t nsteps, int32_t* contacts, void* stream);

/* ---- learned impedance (trace_mode 3) -------------------------------------------------------
 * Sec. III-B lets K(q) and D(q) be learned instead of set by the heuristic and fixes no model.
 * Here K = k_user M_theta / dt and D = d_user M_theta / dt as in Eq. k_d_setting, with
 * M_theta = M(phi) exp(clamp(g(x), -8, 8)) per contact and
 *   g(x) = b2 + sum_h w2_h tanh(b1_h + sum_i W1_hi x_i),  h < 8,  i < 4,
 *   theta = [W1 (8 x 4, row-major), b1[8], w2[8], b2]  (CF_IMPNET_PARAMS floats),
 *   x = (clamp(phi / solimp width, -1, 1), clamp(1 - 3 (1/m_A + 1/m_B) / (tr_A + tr_B), -1, 1),
 *        clamp(w_n / (tr_A + tr_B), 0, 4), 1 if side B is static else 0),
 * tr the mode-0 point-Jacobian trace, 1/m of a static side 0, and w_n = sum over the dynamic
 * sides of 1/m_b + (l_b x n)^T I_b^-1 (l_b x n), l_b the lever from body b's centre of mass and
 * I_b its world inertia (the normal row of J M^-1 J^T with every body taken as free).  g = 0 is
 * the heuristic. */
#define CF_IMPNET_INPUTS 4
#define CF_IMPNET_PARAMS 49

/* Use the network theta (device, [n_sets][CF_IMPNET_PARAMS]; n_sets = 1: every world, n_sets =
 * n_worlds: world w uses set w) in trace_mode 3 steps of this batch.  The batch keeps the
 * pointer: theta must stay valid while steps (or graphs captured after this call) run; the
 * values may change between steps.  theta = NULL detaches it.  CF_ERR_INVALID_ARGUMENT for
 * another n_sets.  A trace_mode 3 step without a network answers CF_ERR_INVALID_ARGUMENT. */
cf_status cf_batch_set_impedance_net(cf_batch* batch, const float* theta, int32_t n_sets);

/* g(x) (unclamped) at x[n][CF_IMPNET_INPUTS] (device, 16-byte aligned) into g[n] (device).
 * n = 0 does nothing (the pointers are then not read); CF_ERR_INVALID_ARGUMENT for a null
 * pointer, n < 0 or a misaligned x. */
cf_status cf_impnet_eval(const float* theta, const float* x, int32_t n, float* g, void* stream);

/* Device floats of the fitting state: Adam's two moments and the reduction scratch.  Zero it
 * before the first cf_impnet_fit of a run. */
size_t cf_impnet_state_floats(void);

/* Mean squared error L = (1/n) sum_i (g(x_i) - y_i)^2 and its gradient grad[CF_IMPNET_PARAMS]
 * (device; either may be NULL) at x[n][4] (16-byte aligned), y[n], all device.  Uses state's
 * scratch.  Deterministic: the sums run in a fixed order. */
cf_status cf_impnet_loss_grad(const float* theta, const float* x, const float* y, int32_t n, float* state,
                              float* grad, float* loss, void* stream);

/* iters steps of full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments) on
 * that loss, updating theta (device) in place; step0 = Adam steps already taken with this
 * state.  losses[iters] (device, nullable) receives the loss before each step.  Enqueued on
 * `stream`, no synchronisation. */
cf_status cf_impnet_fit(float* theta, float* state, int32_t step0, const float* x, const float* y, int32_t n,
                        int32_t iters, float lr, float* losses, void* stream);

const char* cf_status_string(cf_status status);
const char* cf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* COMFREE_H */
