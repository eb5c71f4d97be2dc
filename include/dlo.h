/*
 * dlo.h -- C ABI of the GB300 batched differentiable discrete-elastic-rod stepper.
 *
 * The library steps many independent rods ("DLOs") forward in time and differentiates
 * whole rollouts back through time.  The model is the one of DLO-Lab (arXiv 2606.04206):
 * discrete elastic rods with stretching, bending and twisting energies and symplectic-Euler
 * time stepping (Sec. 3.1, App. A.1), position-based inextensibility and self-collision
 * projections with friction (App. A.1), bending plasticity with a yield threshold and a
 * creep rate (App. A.1), soft SDF coupling to rigid planes, boxes and kinematic capsule
 * grippers (Sec. 3.2), closed-loop holonomy frame initialisation (App. A.1) and gradient
 * checkpointing over long horizons (Sec. 3.3).  Frame time and substeps follow App. B.1.
 *
 * Conventions
 *   B          number of rods ("batch"); rod b has Nv[b] vertices and Ne[b] edges,
 *              Ne = Nv-1 for open rods, Ne = Nv for closed loops.
 *   V = sum Nv, Etot = sum Ne; rods are packed back to back (rod 0 first).
 *   x   [V][4] float   positions (x, y, z, unused on input / inverse mass on output)
 *   v   [V][4] float   velocities (vx, vy, vz, twist rate of the edge that starts at this
 *                      vertex; unused for the last vertex of an open rod)
 *   theta [Etot] float twist angle of each edge's material frame about its reference frame
 *   actions [F][B][2][6] float  per frame, per rod, per gripper: translation increment
 *                      (m) then rotation-vector increment (rad), both in world coordinates.
 *   All device pointers must be 16-byte aligned where they hold float4 data.
 *
 * Ownership and ordering
 *   The caller owns every pointer it passes.  Host arrays are read during the call only.
 *   Device arrays must stay valid until the work enqueued on the context's stream has run.
 *   The library's own workspace (state mirror, checkpoints, segment buffers, scratch) is
 *   allocated through the caller's allocator (or cudaMalloc when none is given) and freed
 *   by dlo_destroy.  All work is enqueued on the stream given at dlo_create and is
 *   asynchronous; argument errors are returned at once, device-side errors (non-finite
 *   state, pair-list overflow) are reported by the next call that synchronises
 *   (dlo_get_state, dlo_backward, dlo_query).  No call throws or exits; a context is not
 *   thread-safe.
 */
#ifndef DLO_H
#define DLO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dlo_ctx dlo_ctx;

typedef enum {
    DLO_OK = 0,
    DLO_ERR_INVALID_ARG = 1,   /* bad size, pointer, option or alignment */
    DLO_ERR_CUDA = 2,          /* a CUDA call failed; dlo_last_error has the CUDA message */
    DLO_ERR_OOM = 3,           /* the allocator returned NULL */
    DLO_ERR_NONFINITE = 4,     /* a rod's state became NaN/Inf; dlo_last_error names the rod */
    DLO_ERR_CAPACITY = 5,      /* self-contact pair list or checkpoint ring too small */
    DLO_ERR_TIMEOUT = 6,       /* reserved: no device-side wait exists in this library */
    DLO_ERR_STATE = 7,         /* call out of order, e.g. dlo_backward without a rollout */
    DLO_ERR_BOUNDS = 8         /* debug builds only (-DDLO_DEBUG_BOUNDS): an index a kernel took
                                  from data failed its bounds check; dlo_last_error names the rod */
} dlo_status;

/* Per-rod material (App. A.1 energies; App. B Table "sim_params" gives the task values). */
typedef struct {
    float density;        /* kg/m^3 */
    float radius;         /* m (uniform along the rod) */
    float K_stretch;      /* stretching modulus K, Pa (k_s = K A); ignored if inextensible */
    float E_bend;         /* bending modulus E, Pa (B = E A r^2 / 4) */
    float G_twist;        /* twisting modulus G, Pa (beta = G A r^2 / 2); 0 = no twist energy
                             and no twist dynamics (the twist angles keep their values) */
    int   inextensible;   /* 1: stretching energy off, edges projected to rest length */
    float strain_limit;   /* >0: elastic stretching plus projection back into [1-s, 1+s] */
    int   plastic;        /* 1: bending plasticity on */
    float yield_curv;     /* sigma_y, 1/m (compared with |kappa_el| / lbar) */
    float creep_rate;     /* r_c; 1 = return to the yield surface in one substep */
    float damping;        /* c_d, 1/s: force -c_d m v and torque -c_d I omega */
    int   closed;         /* 1: closed loop (edge Nv-1 joins vertex Nv-1 to vertex 0) */
} dlo_material;

/* Rigid scene shared by every rod (each rod is its own environment), plus per-rod grippers
 * and, optionally, the strands of rods that hold several DLOs of one environment. */
typedef struct {
    int          n_planes;      /* <= 4 */
    const float* planes;        /* host [n_planes][4]: unit normal n, offset o (n.x = o) */
    int          n_boxes;       /* <= 4 */
    const float* boxes;         /* host [n_boxes][6]: centre, half extents (axis aligned) */
    const int*   n_grippers;    /* host [B] in 0..2, or NULL for none */
    const float* grip_pose;     /* host [B][2][12]: position (3) then rotation matrix (3x3,
                                   row major; column 2 is the capsule axis) at grasp time */
    float        grip_radius;   /* capsule radius, m */
    float        grip_half_len; /* capsule half length, m */
    const unsigned char* pinned;/* host [V] 1 = vertex fixed in space, or NULL */
    const unsigned char* strand_start; /* host [V] 1 = the vertex begins another DLO of the same
                                   environment, or NULL.  A rod with strand starts holds several
                                   DLOs back to back ("strands", e.g. the two ropes of the
                                   Separation task, Sec. 4): they share its material, substeps
                                   and grippers, interact only through self-collision and friction
                                   (App. A.1), and nothing joins them; the edge between two
                                   strands has no force, no length constraint, keeps its frame
                                   (tangent z, d1 = x) and is no contact segment.  Only open rods;
                                   every strand has >= 2 vertices (else DLO_ERR_INVALID_ARG) */
} dlo_scene;

typedef struct {
    float  dt;              /* frame time, s (App. B.1: 1e-3) */
    int    n_iter_pbd;      /* N_C projection iterations per substep (default 10) */
    int    substeps_min;    /* minimum substeps per frame (App. B.1: 5) */
    float  gravity;         /* m/s^2 along -z */
    float  mu_self;         /* self-contact Coulomb coefficient */
    float  mu_rigid;        /* rigid-contact Coulomb coefficient */
    float  restitution;     /* rigid-contact restitution */
    float  eps_soft;        /* softness eps_s as a multiple of the rod radius */
    float  contact_margin;  /* self-contact candidate margin as a multiple of the radius */
    int    self_contact;    /* 1: self-collision projections and friction on (needs
                               n_iter_pbd >= 1: friction uses the first iteration's contacts) */
    int    checkpoint_every;/* frames between rollout checkpoints; 0 = chosen by the library */
    size_t hbm_budget;      /* bytes for checkpoints + backward buffers; 0 = 80 GiB */
    int    warps_per_cta;   /* rods per CTA of the persistent kernels; 0 = autotune */
    int    reaction;        /* 1: dlo_step accumulates the impulse every rigid contact gives each
                               vertex (read with dlo_reaction); 0: off, no cost */
    int    broad_phase;     /* self-contact candidates, once per frame: 0 every edge pair of the rod
                               behind a bounding-sphere filter; 1 a per-rod spatial hash of the
                               edge midpoints (cells of the candidate distance plus the frame's
                               longest edge).  Both give the same candidate set */
} dlo_options;

typedef struct {
    void* (*alloc)(size_t bytes, void* user);  /* device memory, 256-byte aligned */
    void  (*free)(void* ptr, void* user);
    void* user;
} dlo_allocator;

/* Create a context for 1 <= B <= 2^24 rods (an empty batch is an argument error).
 * n_verts[B] >= 2 and <= 256, mat[B], x_rest [V][3] host: the rest shape
 * (rest lengths, masses and grasped vertices are taken from it; open rods rest straight,
 * loops rest as a planar circle of the same length).  The state is set to the rest shape
 * at rest.  cuda_stream may be NULL (legacy default stream).  alloc may be NULL.
 * Defined by: the rod discretisation, masses and reference frames of App. A.1, the
 * kinematic grasp of Sec. 3.2, frame time and substeps of App. B.1.  With
 * opt->warps_per_cta == 0 the rods-per-CTA setting is measured here (a few frames run from
 * the rest state, which is then set again).
 * Errors: DLO_ERR_INVALID_ARG for sizes, options or scene out of range (self-contact needs
 * n_iter_pbd >= 1) or a zero-length rest edge; DLO_ERR_OOM / DLO_ERR_CUDA; *out is NULL on
 * any error. */
dlo_status dlo_create(dlo_ctx** out, int batch, const int* n_verts, const dlo_material* mat,
                      const float* x_rest, const dlo_scene* scene, const dlo_options* opt,
                      const dlo_allocator* alloc, void* cuda_stream);

/* Set a fresh state (device x [V][4], v [V][4], theta [Etot]).  Reference frames are rebuilt
 * from x by space-parallel transport (loops: holonomy spread over the edges, App. A.1), rest
 * curvatures and gripper poses are reset to their create-time values.  Ends any armed
 * recording.  Defined by: the state variables and frame initialisation of App. A.1.
 * Errors: DLO_ERR_INVALID_ARG for a NULL x or a pointer that is not 16-byte aligned. */
dlo_status dlo_set_state(dlo_ctx* ctx, const float* x, const float* v, const float* theta);

/* Replace the per-rod material (host mat[B]) after create: the moduli K_stretch, E_bend and
 * G_twist, the yield curvature, the creep rate and the damping, with which the next dlo_step
 * runs.  Each rod's substep count is recomputed from the new moduli (as at dlo_create).
 * Density, radius, inextensibility, strain limit, plasticity, topology and whether G_twist
 * is zero are fixed at create (they set masses, inertias and the rod's constraints; a rod
 * with G_twist = 0 has no twist dynamics) and must be unchanged.  Ends
 * any armed recording (a recorded rollout ran with the previous material).  Synchronises.
 * Defined by: the material parameters of the energies and the plasticity rule of App. A.1
 * (the quantities the system identification of Sec. 5 fits).
 * Errors: DLO_ERR_INVALID_ARG for a NULL mat, a value out of range or a change of a
 * create-time quantity (dlo_last_error names the rod); the context is unchanged then. */
dlo_status dlo_set_material(dlo_ctx* ctx, const dlo_material* mat);

/* Copy the state into caller-owned device buffers (any may be NULL).  Synchronises the
 * stream and reports device-side errors. */
dlo_status dlo_get_state(dlo_ctx* ctx, float* x, float* v, float* theta);

/* Copy the full internal state into caller-owned device buffers (any may be NULL):
 * ref [Etot][4] = (reference d1 xyz, theta), tan [Etot][4] = (tangent the reference frame
 * is adapted to, unused), hinge [V][4] = (rest curvature 2, rest twist, reference twist)
 * indexed by the hinge's vertex, grip [B][2][12] = current gripper poses. Synchronises. */
dlo_status dlo_get_internal(dlo_ctx* ctx, float* ref, float* tan, float* hinge, float* grip);

/* Arm recording of the next n_frames frames: checkpoints every K frames into the HBM ring
 * and a copy of the actions, so that dlo_backward can differentiate the rollout.  K is
 * opt.checkpoint_every, or when that is 0 the shortest interval whose ring, action record
 * and backward workspace fit opt.hbm_budget (80 GiB by default).  It also sets how many
 * frames the backward reverses per launch pair: its chunk records may take half of what the
 * ring and the action record leave of the budget (at most 24 GiB).
 * Defined by: the gradient checkpointing of Sec. 3.3 (checkpoints kept in HBM here).
 * Errors: DLO_ERR_INVALID_ARG for n_frames <= 0; DLO_ERR_OOM when the ring cannot be
 * allocated. */
dlo_status dlo_begin_rollout(dlo_ctx* ctx, int n_frames);

/* Advance every rod by `frames` frames of dt with actions (device, [frames][B][2][6]; may be
 * NULL = no gripper motion).  substeps > 0 forces that many substeps per frame for every rod;
 * 0 uses each rod's own count (max(substeps_min, ceil(dt * omega_max))).  x_frames (device,
 * [frames][V][4]) optionally receives the positions after every frame (may be NULL).
 * One persistent launch per rod size class; only stream-ordered work, no synchronisation,
 * so the call can be captured in a CUDA graph on the context's stream.
 * Defined by: symplectic-Euler time stepping of the energies of Sec. 3.1 / App. A.1
 * (stretching, bending, twisting), bending plasticity, the inextensibility and self-collision
 * projections with friction (App. A.1), soft coupling to rigid primitives and grippers
 * (Sec. 3.2), frame time and substeps of App. B.1.
 * Errors: DLO_ERR_INVALID_ARG for negative frames or substeps or an unaligned x_frames;
 * DLO_ERR_STATE when a recorded rollout would run past its armed frames or change its
 * substeps.  Non-finite states and pair-list overflow are reported by the next
 * synchronising call. */
dlo_status dlo_step(dlo_ctx* ctx, const float* actions, int frames, int substeps, float* x_frames);

/* The same rollout computed by the plain per-phase kernels (one launch per phase per
 * substep, state in HBM, one thread per element): the speed comparator.  Same arguments and
 * errors as dlo_step (without x_frames).  Armed by dlo_begin_rollout it records checkpoints
 * and actions as dlo_step does (the rollout can then be differentiated by dlo_backward or
 * dlo_backward_plain).  Defined by: the same passages as dlo_step. */
dlo_status dlo_step_plain(dlo_ctx* ctx, const float* actions, int frames, int substeps);

/* The adjoint of dlo_backward computed the plain way, the comparator of the fused adjoint:
 * per frame, last first, the frame's start state is restored from its checkpoint (and the
 * frames before it in its segment re-run), the frame is re-run by the plain per-phase
 * kernels storing every substep's intermediates in HBM, and each substep is reversed by one
 * kernel launch per phase, one thread per element, every cotangent in HBM.  Same arguments,
 * outputs and errors as dlo_backward.  Defined by: the gradient through time of Sec. 3.3. */
dlo_status dlo_backward_plain(dlo_ctx* ctx, const float* dL_dx_T, const float* dL_dv_T,
                              const float* dL_dtheta_T, float* dL_dactions, float* dL_dmaterial,
                              float* dL_dx0, float* dL_dv0, float* dL_dtheta0);

/* Differentiate the recorded rollout (the gradient through time of Sec. 3.3, computed by a
 * hand-written adjoint that replays each frame from its checkpoint).  Inputs (device, may be
 * NULL = zero): dL/dx_T [V][4]
 * (w ignored), dL/dv_T [V][4] (w = dL/d twist rate), dL/dtheta_T [Etot].  Outputs (device,
 * may be NULL = not wanted): dL/dactions [F][B][2][6], dL/dmaterial [B][5] for
 * (K_stretch, E_bend, G_twist, yield_curv, damping), dL/dx0 [V][4], dL/dv0 [V][4],
 * dL/dtheta0 [Etot].  Gradients are with respect to the state set by dlo_set_state when the
 * rollout started from it (reference frames rebuilt from x0), else with respect to the state
 * at dlo_begin_rollout holding its reference frames fixed.  Synchronises.
 * Errors: DLO_ERR_STATE without a completed recorded rollout; DLO_ERR_INVALID_ARG for
 * unaligned float4 arrays or self-contact with no projection iteration; DLO_ERR_OOM when
 * the workspace cannot be allocated; DLO_ERR_NONFINITE / DLO_ERR_CAPACITY as recorded by the
 * rollout. */
dlo_status dlo_backward(dlo_ctx* ctx, const float* dL_dx_T, const float* dL_dv_T,
                        const float* dL_dtheta_T, float* dL_dactions, float* dL_dmaterial,
                        float* dL_dx0, float* dL_dv0, float* dL_dtheta0);

/* The same adjoint with no memory allocation.  The paper has no counterpart: this is an
 * interface for callers that cannot allocate during the call, such as an optimisation loop
 * whose device memory budget is already handed out (an allocator pool at capacity, or memory
 * partitioned between simulation workers), where a workspace allocation would fail with
 * out-of-memory in the middle of a run.  Arguments, outputs and results are those of
 * dlo_backward.  Every temporary comes from one static device array of
 * DLO_NOALLOC_SCRATCH_BYTES inside the library; the call makes no cudaMalloc, cudaFree or
 * other allocating call on the device and no heap allocation on its success path.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before any
 *   stream capture begins.
 *   Zero state: nothing in the array needs to start at zero (every scratch word is written
 *   before it is read); the per-launch work-queue heads, which live in context memory from
 *   dlo_create, are reset with cudaMemsetAsync on the context's stream.
 *   Capacity: the rods run with as many in flight as the array holds (fewer than
 *   dlo_backward uses, so it can be slower).  When one rod's recompute buffers plus the
 *   batch-wide frame cotangents (32 bytes per edge, plus 96 per vertex when dL_dx0 is asked
 *   for after dlo_set_state) exceed the array, the call returns DLO_ERR_CAPACITY and
 *   dlo_last_error states the sizes.
 *   Concurrency: the array is shared by every context on the device, so calls must not
 *   overlap (two calls in flight from different threads or streams race on it).  Each call
 *   synchronises its stream before returning.
 *   Footprint: the array is device memory of the library's own module, reserved on a device
 *   when that module is loaded there.  With CUDA's lazy module loading (the default) that is
 *   the first call of this function on the device; with CUDA_MODULE_LOADING=EAGER it is every
 *   context that loads the library, whether or not it ever calls this function. */
#define DLO_NOALLOC_SCRATCH_BYTES ((size_t)256 << 20)
dlo_status dlo_backward_noalloc(dlo_ctx* ctx, const float* dL_dx_T, const float* dL_dv_T,
                                const float* dL_dtheta_T, float* dL_dactions, float* dL_dmaterial,
                                float* dL_dx0, float* dL_dv0, float* dL_dtheta0);

/* Task losses of App. B ("Reward design"), per rod, on the device. */
enum {
    DLO_LOSS_TARGET = 1,    /* (1/N) sum_i |x_i - t_i|^2; aux = targets [V][4] (trajectory optimisation) */
    DLO_LOSS_CHAMFER = 2,   /* (1/N) sum_i min_j |x_i - y_j|^2 + (1/M) sum_j min_i |x_i - y_j|^2;
                               aux = points [B][m][4], 1 <= m <= 1024 (Separation, Wiring-post) */
    DLO_LOSS_WINDING = 3,   /* (1/2pi) sum over segments of the signed angle each subtends at a
                               vertical post in the xy-plane; aux = post [B][4] (x, y, -, -) (Wrapping) */
    DLO_LOSS_CROSSING = 4,  /* sum over ordered pairs of non-adjacent edges of Omega / (4 pi), Omega
                               the exact Gauss double integral of the two segments: the signed
                               crossing sum of Unknotting's crossing number; aux unused */
    DLO_LOSS_MINDIST = 5,   /* min_i |x_i - o|: distance from the rod to an object's centre (the
                               rope-object contact terms of Gathering, Lifting, Wrapping);
                               aux = o [B][4] (x, y, z, -); the gradient goes to the nearest
                               vertex (the lowest index on an exact tie) */
    DLO_LOSS_REPULSION = 6  /* sum over unordered edge pairs more than k apart along the rod
                               (cyclically for loops) of max(0, delta - d_ab)^2, d_ab the distance
                               between the closest points of the two segments (Unknotting's
                               self-repulsion penalty); aux = [B][4] (delta, k, -, -), k >= 1 */
};

/* Loss Q_b of every rod and, when dL_dx is given, dL/dx for L = sum_b g_b Q_b: the cotangent
 * dlo_backward takes as dL/dx_T.  x [V][4] device positions (w ignored); aux as the kind
 * says (device float4, 16-byte aligned); g [B] device dL/dQ_b (NULL = 1); q [B] device out (may
 * be NULL); dL_dx [V][4] device out (NULL = not wanted; every vertex is written).  Enqueued on
 * the context's stream, deterministic, no synchronisation.  The paper defines these task
 * terms in App. B; the crossing sum's pair term is the standard closed form of the Gauss
 * integral for straight segments (a reading of "signed crossing contributions").
 * Errors: DLO_ERR_INVALID_ARG for an unknown kind, a missing or unaligned array, m out of
 * range, rods of more than 256 vertices, or a loss over edges (winding, crossing,
 * repulsion) on a context with strands (dlo_scene.strand_start).  A repulsion window k < 1
 * (read on the device) is taken as 1. */
dlo_status dlo_loss(dlo_ctx* ctx, int kind, const float* x, const float* aux, int m, const float* g, float* q,
                    float* dL_dx);

/* System-identification loss (Sec. 5, "System Identification": the pixel-wise projection error
 * between the simulated rope and a camera's binary mask, back-propagated to the material).
 * Reading: a soft silhouette.  Each edge is a capsule of radius rho_e = (rho_a + rho_b) / 2,
 * rho = fx r / Z the projected rod radius at an endpoint; a pixel centre p at signed distance
 * s_e(p) = dist(p, projected segment) - rho_e from it is covered with sigma(-s_e / tau), and
 * its occupancy is o(p) = 1 - prod_e (1 - sigma(-s_e(p) / tau)).  Q_b = mean over cameras and
 * pixels of (o - mask)^2.  Edges with an endpoint at Z <= 1e-3 (at or behind the camera plane)
 * are not drawn.
 *   x       [V][4] device positions
 *   cams    [n_cams][16] device floats per pinhole camera: fx, fy, cx, cy (pixels), then the
 *           world-to-camera rotation R (row major) and translation t: X_cam = R x + t,
 *           u = fx X/Z + cx, v = fy Y/Z + cy; pixel (i, j) is column i, row j, centre
 *           (i + 0.5, j + 0.5)
 *   masks   [B][n_cams][height][width] device bytes, nonzero = rope
 *   tau     edge softness in pixels (> 0)
 *   g, q, dL_dx as for dlo_loss (L = sum_b g_b Q_b)
 *   render  [B][n_cams][height][width] device floats: the soft silhouettes o (NULL = not wanted)
 * Grows a context workspace of B * height * width floats.  Enqueued on the context's stream,
 * deterministic.  Errors: DLO_ERR_INVALID_ARG for a missing or unaligned array, no camera,
 * more than 2^24 pixels, tau <= 0, rods of more than 256 vertices or a context with strands
 * (dlo_scene.strand_start); DLO_ERR_OOM when the workspace cannot grow. */
dlo_status dlo_loss_silhouette(dlo_ctx* ctx, const float* x, const float* cams, int n_cams, int height, int width,
                               const unsigned char* masks, float tau, const float* g, float* q, float* dL_dx,
                               float* render);

/* Contact impulses of the rigid coupling (Sec. 3.2; the two-way coupling hands the rigid
 * body the equal and opposite momentum): for every rod, the impulse sum_substeps m (v' - v)
 * that each response of the soft rigid contact gave its vertices since the last reset, in
 * four slots: all planes, all boxes, gripper 0, gripper 1 (N s, world frame).  The rigid
 * bodies received the opposite impulses.  Only dlo_step accumulates (not dlo_step_plain, not
 * the backward's recomputation); the context must be created with opt.reaction = 1.
 *   per_rod    [B][4][4] device floats out (x, y, z, 0 per slot), or NULL; summed over the
 *              rod's vertices in a fixed order
 *   per_vertex [V][4][4] device floats out, or NULL: where along the rod the impulses acted
 *   reset      1: zero the accumulators after reading
 * Enqueued on the context's stream.  Errors: DLO_ERR_STATE if the context was created without
 * opt.reaction; DLO_ERR_INVALID_ARG for unaligned outputs. */
dlo_status dlo_reaction(dlo_ctx* ctx, float* per_rod, float* per_vertex, int reset);

enum {
    DLO_Q_SUBSTEPS = 1,      /* int [B]: substeps per frame of each rod */
    DLO_Q_STATUS = 2,        /* unsigned [B]: status bits since the last dlo_set_state: 1 non-finite
                                state, 2 pair-list overflow (both errors), 4 a warning: some vertex
                                moved, within one frame, at least half of the candidate margin
                                (contact_margin x radius), so the candidates found at the frame's
                                start may miss a pair that came into contact during it; 8 (debug
                                builds) an index failed its bounds check (an error) */
    DLO_Q_BYTES = 3,         /* size_t: device bytes held by the context */
    DLO_Q_CONFIG = 4,        /* int [4]: warps per CTA, checkpoint interval, CTAs, smem/CTA */
    DLO_Q_RESIDUAL = 5,      /* double [B]: sum |C_j| of the inextensibility constraints
                                after the last frame, accumulated in FP64 */
    DLO_Q_PAIRS = 6,         /* int [B]: largest self-contact candidate count of any frame of the
                                last dlo_step (capacity: 4 per vertex of the rod's size class) */
    DLO_Q_LAUNCHES = 7,      /* long long: kernels launched by this context so far */
    DLO_Q_MASS = 8,          /* float [V][4]: (mass, inverse mass, kind, 0); kind 0 free,
                                1 pinned, 2/3 grasped by gripper 0/1 (host out) */
    DLO_Q_PAIR_LIST = 9      /* unsigned [B][1 + 1024]: per rod, the number n of self-contact
                                candidates found at the start of the last frame of the last
                                dlo_step, then n entries (a | b << 16), edge a < edge b, in no
                                particular order; the rest of the row is 0xffffffff.  All counts
                                are 0 when self-contact is off */
};

/* Query (host `out`).  Synchronises. */
dlo_status dlo_query(dlo_ctx* ctx, int what, void* out);

/* Measurement utility, not part of the method (the paper has no counterpart): the device's
 * FP32 throughput in TFLOP/s (an FMA counted as 2), measured by a kernel of independent
 * register-only FMA chains on every SM, run for about `seconds` (0 < seconds <= 60) on the
 * given stream (NULL = legacy default stream) after a short warm-up launch.  It is the
 * denominator of the FP32 roofline fraction the benchmark reports for the rod kernels.
 * Synchronises the stream; allocates and frees a few bytes of device memory.
 * Errors: DLO_ERR_INVALID_ARG for a NULL result or seconds out of range; DLO_ERR_CUDA. */
dlo_status dlo_measure_fp32_peak(double seconds, void* cuda_stream, double* tflops);

/* How this library was built: bit 1 set when the kernels check every index they take from data
 * (compiled with -DDLO_DEBUG_BOUNDS; a failed check gives DLO_ERR_BOUNDS).  No device work. */
int dlo_build_flags(void);

const char* dlo_status_string(dlo_status s);
const char* dlo_last_error(const dlo_ctx* ctx);
void dlo_destroy(dlo_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DLO_H */
