/*
 * ipc.h — C ABI of the B300-native multi-environment IPC stepper.
 *
 * The library advances a batch of independent grasp environments with Incremental Potential
 * Contact (GRIP, arXiv 2503.05020, Sec. II-C: barrier augmentation, CCD and a projected Newton
 * solver with a step-size filter; Sec. III-A: the environments are isolated in collision
 * detection and step-size filtering, each one stops on its own criterion and is frozen, and a
 * failed environment is detected and excluded; Sec. III-D: dt, kappa, dhat, eps_v, FP64 and at
 * most 100 Newton iterations). Soft bodies are Neo-Hookean tet meshes; rigid parts are 12-DOF
 * affine bodies (Sec. I, IPC coupled with affine body dynamics).
 *
 * Conventions
 *  - Every function returns an ipc_status; on error, ipc_last_error() returns a message that
 *    stays valid until the next call on the same host thread.
 *  - All descriptor arrays are HOST pointers. They are copied during the call; the caller keeps
 *    ownership and may free them on return.
 *  - Output buffers are HOST pointers owned by the caller. When a buffer is too small the call
 *    returns IPC_ERR_ARG and *written (if not NULL) gets the required byte count.
 *  - Device memory is allocated by the library (cudaMalloc on the scene's device) and released
 *    by ipc_scene_destroy. Work is issued on the scene's stream (borrowed, or created when the
 *    descriptor passes NULL). ipc_step returns after the step's work has completed.
 *  - A scene is not thread-safe: use one scene per host thread.
 *  - Layout of an environment's DOF vector ("DOFs"): the vertices of its soft bodies in the
 *    order they were given (x, y, z each, metres), then for each affine body its 12 affine
 *    coordinates q = (p, a1, a2, a3) where a rest point xb sits at p + xb0*a1 + xb1*a2 + xb2*a3.
 */
#ifndef IPC_B300_H
#define IPC_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipc_scene ipc_scene;

typedef enum {
  IPC_OK = 0,
  IPC_ERR_ARG = 1,            /* bad argument, unknown env id, output buffer too small */
  IPC_ERR_OOM = 2,            /* device allocation failed */
  IPC_ERR_BUDGET = 3,         /* the env would exceed the scene's HBM budget (admission) */
  IPC_ERR_CUDA = 4,           /* a CUDA call failed; the message names it */
  IPC_ERR_INIT_INTERSECT = 5, /* initial state has a touching or intersecting pair: IPC needs an
                                 intersection-free start (Sec. III-C) */
  IPC_ERR_INIT_INVERTED = 6,  /* a tet has non-positive rest or initial volume */
  IPC_ERR_NO_ENV = 7,         /* the scene holds no environment */
  IPC_ERR_INTERNAL = 8        /* an internal capacity or traversal limit was hit */
} ipc_status;

typedef enum { IPC_FP64 = 0, IPC_MIXED = 1 } ipc_precision;

/* Solver parameters shared by every environment of a scene (Sec. III-D gives dt = 0.01 s,
 * kappa = 3e6 kg/s^2, dhat = 1e-3 m, eps_v = 1e-3 m/s, 100 Newton iterations, FP64). */
typedef struct {
  double dt;             /* time step h (s) */
  double dhat;           /* barrier activation distance (m) */
  double kappa;          /* barrier stiffness (kg/s^2) */
  double eps_v;          /* friction static/dynamic transition speed (m/s) */
  double newton_tol;     /* converged when ||p||_inf / h < newton_tol (m/s) */
  double pcg_rel_tol;    /* PCG stops at ||r|| <= pcg_rel_tol ||b|| */
  double kappa_affine;   /* affine-body orthogonality stiffness (Pa) */
  double gravity[3];     /* m/s^2 */
  int32_t max_newton;    /* Newton iterations per step before the env is marked FAILED */
  int32_t max_ls_halvings; /* line-search halvings before the env is marked FAILED */
  int32_t max_pcg_iters; /* PCG iteration cap per solve */
  int32_t precision;     /* ipc_precision */
  uint64_t hbm_budget_bytes; /* 0 = no admission limit */
  int32_t device;        /* CUDA device ordinal */
  int32_t pcg_cluster;   /* PCG launch shape: 0 = automatic, 1/2/4/8/16 = one persistent cluster of
                            that many CTAs per environment, -1 = one launch per PCG phase over
                            tiles of all environments */
  int32_t fresh_broad_phase; /* 0: inside a time step, the line-search trials and the later Newton
                            iterations take their contact sets from the step filter's swept
                            candidates (boxes swept over [x, x + p] and grown by dhat/2, which
                            hold every pair that can come within dhat on the segment); 1: a BVH
                            traversal at every evaluation. Both give the same contacts in the
                            same order. */
  int32_t kappa_adapt;   /* 0: the barrier stiffness is kappa throughout (Sec. III-D). 1: adapted
                            per env: at each step start the least-squares balance of the barrier
                            gradient against the other terms' gradient over the free DOFs,
                            -(g_E . G) / (G . G), clamped to [kappa, 1000 kappa], and held for
                            the rest of the step */
  void* cuda_stream;     /* cudaStream_t to borrow, or NULL for a library-owned stream */
  int32_t collect_slots; /* partners a collect traversal keeps per query (0 = 128; 1..4096); a
                            query with more sends the pass to a count-then-fill traversal, with the
                            same candidates in the same order */
} ipc_scene_desc;

/* Soft body: a Neo-Hookean tet mesh. verts: n_verts*3 doubles (rest = initial positions);
 * tets: n_tets*4 int32 with positive rest orientation; tris: n_tris*3 int32 outward surface
 * triangles (vertex indices of this body); kinematic: n_verts bytes, 1 = the vertex follows the
 * schedule (may be NULL). */
typedef struct {
  int32_t n_verts, n_tets, n_tris, pad;
  const double* verts;
  const int32_t* tets;
  const int32_t* tris;
  const uint8_t* kinematic;
  double youngs, poisson, density;
} ipc_soft_body_desc;

/* Affine body: closed outward rest surface (n_verts*3 doubles, n_tris*3 int32), density,
 * initial coordinates q0 and rates qdot0 (12 each). A kinematic body follows the schedule; a free
 * body with pd_stiffness > 0 is pulled toward it. */
typedef struct {
  int32_t n_verts, n_tris, kinematic, pad;
  const double* verts;
  const int32_t* tris;
  double density;
  double q0[12];
  double qdot0[12];
  double pd_stiffness; /* k_pd (1/s^2) of a free body driven toward its scheduled coordinates by
                          1/2 h^2 k_pd (q - q^)^T (M4 x I3) (q - q^) = 1/2 h^2 k_pd int rho |x - x^|^2
                          (rigid links of a hand following joint targets); 0 = none */
} ipc_affine_body_desc;

/* Point joint between two affine bodies of one environment (Sec. I: IPC coupled with affine body
 * dynamics for articulated multibodies). The anchor of body a and the anchor of body b (each in
 * its body's rest frame, x = p + A xbar) are held together by the potential 1/2 k |x_a - x_b|^2
 * (k in N/m, scaled by h^2 like every potential of the incremental potential). Two joints
 * between the same bodies on one axis make a hinge. */
typedef struct {
  int32_t body_a, body_b; /* indices among the env's affine bodies; distinct */
  double anchor_a[3];     /* rest-frame anchor on body a (m) */
  double anchor_b[3];     /* rest-frame anchor on body b (m) */
  double stiffness;       /* k > 0 (N/m) */
} ipc_joint_desc;

/* One environment. gravity_on: n_steps bytes, the gravity of step s: 0 none, 1 the scene's
 * gravity vector, 2..7 its magnitude along +x, -x, +y, -y, +z, -z (the axis-aligned phases of the
 * grasp evaluation protocol, Sec. III-D); other values are rejected (IPC_ERR_ARG).
 * targets: n_steps * (n_soft + n_affine) * 12 doubles: for step s and body b (soft bodies
 * first) the affine map the body's kinematic vertices (soft, applied to their initial
 * positions) or the kinematic affine body itself must reach at the end of step s. */
typedef struct {
  int32_t n_soft, n_affine, n_steps, pad;
  const ipc_soft_body_desc* soft;
  const ipc_affine_body_desc* affine;
  double friction_mu;
  const uint8_t* gravity_on;
  const double* targets;
  int32_t n_joints, pad2;       /* point joints of the env (0: none) */
  const ipc_joint_desc* joints; /* n_joints entries (may be NULL when n_joints = 0) */
  int32_t grasped_object;       /* 1 + the handle of the grasped object (soft bodies first, then
                                   affine bodies), for IPC_Q_GRASP_RESULT; 0 = none */
  int32_t pad3;
} ipc_env_desc;

typedef enum {
  IPC_Q_DOFS = 0,        /* double[ndof]: current DOFs */
  IPC_Q_VELOCITIES = 1,  /* double[ndof]: current DOF rates */
  IPC_Q_STATUS = 2,      /* int32[4]: status (0 ACTIVE, 1 DONE, 2 FAILED), reason (0 none,
                            1 Newton cap, 2 line search, 3 non-finite), steps done, next step */
  IPC_Q_STATS = 3,       /* int64[5]: Newton iterations, PCG iterations, line-search halvings,
                            steps, ACCD iterations (cumulative) */
  IPC_Q_CANDIDATES = 4,  /* int32[n][3]: (kind 0 = point-triangle / 1 = edge-edge, i, j) of the
                            dhat/2-inflated box candidates at the current DOFs, env-local
                            surface-vertex / triangle / edge indices, sorted */
  IPC_Q_CONTACTS = 5,    /* int32[n][4]: (kind, i, j, distance type) of candidates closer than
                            dhat, sorted like CANDIDATES */
  IPC_Q_POINTS = 6,      /* double[n_points][3]: world positions of all surface-capable points
                            (soft vertices, then affine rest vertices mapped by q; joint anchors
                            are not among them) */
  IPC_Q_SIZES = 7,       /* int64[8]: ndof, points (those of IPC_Q_POINTS), surface vertices,
                            edges, triangles, tets, bodies, steps */
  IPC_Q_INTERSECTIONS = 8, /* int64[2]: segment-triangle intersections, inverted tets */
  IPC_Q_SCENE_COUNTERS = 9, /* int64[12] for the whole scene (env_id ignored), from the last Newton
                              iteration: contacts, point-triangle contacts, friction stencils,
                              stencil-node incidence entries, longest node incidence list,
                              candidates, BSR blocks, sliced-ELL padded blocks; then the PCG
                              cluster size in use (0 = tiled multi-launch PCG), the most 32-row
                              slices of one environment, the point joints of the batch and the
                              collect traversal passes that spilled since the scene was made */
  IPC_Q_ALL_STATUS = 10,   /* int32[4 * n_env] for the whole scene (env_id ignored): env id,
                              status, failure reason, next step of every environment, in one
                              read-back (a serving loop polls this once per step) */
  IPC_Q_KAPPA = 11,        /* double[1]: the env's barrier stiffness in its current (or last) step */
  IPC_Q_TET_STRESS = 12,   /* double[n_tets]: von Mises stress (Pa) of the Neo-Hookean Cauchy
                              stress of each of the env's tets at its current DOFs */
  IPC_Q_CONTACT_FORCES = 13, /* double[n]: normal force kappa e |b'(d)| (N) of each contact at
                              the env's current DOFs, in the order of IPC_Q_CONTACTS */
  IPC_Q_FRICTION_FORCES = 14, /* double[n]: tangential force mu lambda f1(|u|) (N) of each lagged
                              friction stencil of the env's current (or last) step at its
                              current DOFs (u: tangential relative displacement since the step
                              start); point-triangle stencils first */
  IPC_Q_CONTACT_HANDLES = 15, /* int32[n][2]: the bodies of the two sides of each contact (env-local
                              handles: soft bodies first, then affine bodies), in the order of
                              IPC_Q_CONTACTS */
  IPC_Q_ENERGY_TRACE = 16, /* double[n]: the incremental potential (J) at each Newton iterate of the
                              env's current (or last) step, in iteration order, n <= max_newton
                              (Sec. II-C projected Newton: a diagnostic trace for parity checks) */
  IPC_Q_GRASP_RESULT = 17  /* double[4] for an env that names its grasped object: in contact with
                              another body at the current DOFs (0/1); the motion of the object's
                              centre of mass (the mean of its points) over the last step, dt times
                              its velocity (m); the stability label of Sec. III-D (1 when in contact
                              and that motion is below eps_v dt); the rise of the centre since the
                              env's initial state (m). IPC_ERR_ARG when the env names no object */
} ipc_query_kind;

/* Create / destroy a scene on desc->device. */
ipc_status ipc_scene_create(const ipc_scene_desc* desc, ipc_scene** out);
ipc_status ipc_scene_destroy(ipc_scene* scene);

/* Add an environment (copied). Rejects inverted tets (IPC_ERR_INIT_INVERTED), an initial
 * state with a touching or crossing pair (IPC_ERR_INIT_INTERSECT; checked when the batch is
 * next laid out on the device, i.e. at the next ipc_step / query), and an env whose estimated
 * device bytes do not fit the remaining HBM budget (IPC_ERR_BUDGET). */
ipc_status ipc_env_add(ipc_scene* scene, const ipc_env_desc* env, int32_t* env_id);
/* Remove an environment; its slot and memory are reused. */
ipc_status ipc_env_remove(ipc_scene* scene, int32_t env_id);

/* Advance every ACTIVE environment by up to n_steps time steps (Sec. III-A: each env has its
 * own step size, stopping test and failure state; a failure never fails the call). Inside the
 * call the envs step at their own pace: an env whose Newton loop has stopped starts its next
 * step while slower envs still iterate. Each env's results are those of stepping it alone, one
 * step per call. Returns when every env has done its steps (or stopped: DONE, FAILED). */
ipc_status ipc_step(ipc_scene* scene, int32_t n_steps);

/* Copy one result of one environment into out (host). */
ipc_status ipc_query(ipc_scene* scene, int32_t env_id, int32_t kind, void* out, size_t out_bytes,
                     size_t* written);

/* Overwrite an environment's state: DOFs x and rates v (ndof doubles each, host) and the index
 * of its next step. Used for checkpoint/resume and for parity checks. */
ipc_status ipc_env_set_state(ipc_scene* scene, int32_t env_id, const double* x, const double* v,
                             int32_t step);

/* Incremental potential and its gradient at DOFs q (host, ndof doubles) for the env's next
 * step, taking its current state as x^t (predicted positions and friction lagged at x^t).
 * grad may be NULL. Diagnostic entry point (parity checks); it recomputes the step set-up. */
ipc_status ipc_eval(ipc_scene* scene, int32_t env_id, const double* q, double* energy,
                    double* grad);

/* Newton direction p of the first Newton iteration of the env's next step, taken at its current
 * state (host, ndof doubles): kinematic DOFs get target - x, free DOFs the PCG solution of the
 * projected-Hessian system H p = -g - H pbar (Sec. II-C projected Newton). Diagnostic entry
 * point for parity checks of the Hessian and the linear solve; the env's state is unchanged. */
ipc_status ipc_newton_direction(ipc_scene* scene, int32_t env_id, double* p);

/* y = H d with H the PSD-projected Hessian of the env's incremental potential at its current
 * state, as the PCG applies it (kinematic rows give 0). d and y are host arrays of ndof doubles.
 * Diagnostic entry point for parity checks of the Hessian assembly. */
ipc_status ipc_hessian_apply(ipc_scene* scene, int32_t env_id, const double* d, double* y);

/* Streaming schedule: overwrite, for every ACTIVE env (in env-id order of the ids returned by
 * ipc_env_add), the kinematic targets of its next step from a host array laid out as
 * [env][body][12]. bytes must equal 12*8*sum over active envs of their body counts. */
ipc_status ipc_set_next_targets(ipc_scene* scene, const double* targets, size_t bytes);
/* Rewrite rows first_step .. first_step + n_steps - 1 of one env's schedule (targets: host array
 * [n_steps][body][12], soft bodies first); kept across relayouts. IPC_ERR_ARG outside the
 * schedule. */
ipc_status ipc_env_set_targets(ipc_scene* scene, int32_t env_id, int32_t first_step, int32_t n_steps,
                               const double* targets);

/* Copy the DOFs of every ACTIVE-or-finished env, in env-id order, into one host array. */
ipc_status ipc_get_all_dofs(ipc_scene* scene, double* out, size_t out_bytes, size_t* written);

/* Estimated device bytes an env would hold (used for admission control). */
ipc_status ipc_env_estimate_bytes(const ipc_env_desc* env, int32_t precision, uint64_t* bytes);

/* Allocation-free Neo-Hookean energy (the paper has no counterpart; this is a deployment
 * convenience). For callers that cannot call cudaMalloc: real-time control loops where an
 * allocation's latency or failure is not acceptable, or hosts whose memory manager owns every
 * device allocation and forbids others. It computes, for each group g of tets
 * [group_offsets[g], group_offsets[g+1]), h2 * sum V Psi(F) over the group with the same per-tet
 * energy code and the same fixed-order reduction as the scene path, and sets inverted[g] = 1 when
 * a tet of the group has J <= 0 (its energy then counts as 0).
 * All pointers are DEVICE pointers on the current device, owned by the caller, each aligned to
 * its element type (4 bytes for int32, 8 for double; IPC_ERR_ARG otherwise):
 *   tets: n_tets*4 int32 node indices into x; tet_params: n_tets*12 doubles per tet (row-major
 *   Dm^-1, rest volume, mu, lambda); x: node positions (3 doubles each); group_offsets:
 *   n_groups+1 int32, non-decreasing, with group_offsets[0] = 0 and group_offsets[n_groups] =
 *   n_tets; energy: n_groups doubles (written); inverted: n_groups int32 (written).
 *   stream: cudaStream_t or NULL for the legacy default stream.
 * The offsets are device data and are not read back: the kernels clamp each one to [0, n_tets],
 * so every access stays in bounds whatever they hold, and tets outside [group_offsets[0],
 * group_offsets[n_groups]) belong to no group (neither summed nor flagged); offsets that break
 * the rules above give unspecified sums. Node indices must lie inside x.
 * Scratch lives in a file-scope device array of IPC_NOALLOC_MAX_TETS doubles (2 MiB), held by
 * every device that loads the library until the process exits. Calls with n_tets above that
 * maximum, or more than IPC_NOALLOC_MAX_GROUPS groups, return IPC_ERR_ARG. The first call on a
 * device looks the array up (cudaGetSymbolAddress, with that device current) and keeps its
 * address for the life of the process; make that first call before any stream capture, and do
 * not call this entry point on a device after cudaDeviceReset (or any other destruction of its
 * primary context) in the same process. All calls share the array: calls that overlap on the
 * GPU (different streams, or different host threads) race on it. The call enqueues its work and
 * returns without synchronising; it performs no allocation of any kind. */
#define IPC_NOALLOC_MAX_TETS 262144
#define IPC_NOALLOC_MAX_GROUPS 65536
ipc_status ipc_elastic_energy_noalloc(int32_t n_tets, const int32_t* tets, const double* tet_params, const double* x,
                                      int32_t n_groups, const int32_t* group_offsets, double h2, double* energy,
                                      int32_t* inverted, void* stream);

/* Number of kernel launches issued by this scene since creation (instrumentation). */
ipc_status ipc_launch_count(ipc_scene* scene, int64_t* count);

/* Kernel-family profiling on the scene's stream (CUDA events around each launch of the family;
 * a few microseconds of overhead per launch). Families: */
typedef enum {
  IPC_PROF_SPMV = 0,        /* PCG / Newton matrix-vector product (BSR rows + stencil gathers) */
  IPC_PROF_ELASTIC = 1,     /* Neo-Hookean energy, gradient and projected Hessian per tet */
  IPC_PROF_CONTACT = 2,     /* barrier + friction stencils with projected Hessians */
  IPC_PROF_CCD = 3,         /* swept-box traversal with additive CCD */
  IPC_PROF_PCG_VECTOR = 4,  /* PCG vector updates, preconditioner and dot products */
  IPC_PROF_BROAD = 5,       /* constraint-set traversal, narrow phase */
  IPC_PROF_ASSEMBLY = 6,    /* gradient / BSR gather, preconditioner blocks, stencil incidence */
  IPC_PROF_LS_ENERGY = 7,   /* energy-only evaluation of line-search trials */
  IPC_PROF_PCG_SOLVE = 8,   /* persistent per-environment PCG (work: algorithmic bytes) */
  IPC_PROF_PCG_FLOPS = 9,   /* work only: floating-point operations of the persistent PCG (an FMA
                               counts 2); its launches and time are those of IPC_PROF_PCG_SOLVE */
  IPC_PROF_HOST_IDLE = 10,  /* host round trips inside ipc_step (a count or flag read back before
                               the next launch): "launches" counts them and the time is the GPU's
                               idle time from the end of the work before each wait to the next
                               kernel launch (events on the scene's stream) */
  IPC_PROF_COUNT = 11
} ipc_prof_family;
/* Turn profiling on (1) or off (0); turning it on clears the counters. */
ipc_status ipc_profile_enable(ipc_scene* scene, int32_t on);
/* Launches, summed event time (ms) and algorithmic work of one family since profiling was
 * turned on. work: SPMV = algorithmic bytes (BSR blocks 76 B, node vectors 56 B, stencil
 * entries 28 B, body blocks 1344 B); PCG_SOLVE = algorithmic bytes and PCG_FLOPS = operations,
 * both counted on the device; ELASTIC = tets processed by the Hessian evaluations; CONTACT,
 * CCD, BROAD, ASSEMBLY = algorithmic bytes counted on the host from the sizes of each launch
 * (records, gathered points and outputs once each, over the launch's whole extent); others 0.
 * Synchronises. */
ipc_status ipc_profile_read(ipc_scene* scene, int32_t family, int64_t* launches, double* ms, double* work);

const char* ipc_last_error(void);
const char* ipc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IPC_B300_H */
