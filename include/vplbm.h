/*
 * vplbm.h - C ABI of the GB300 volume-penalization lattice Boltzmann library.
 *
 * The library advances a D2Q9 multiple-relaxation-time (or BGK) lattice
 * Boltzmann fluid in which a rigid body (disk, ellipse or rectangle; up to
 * VPLBM_MAX_BODIES of them) is represented by a characteristic function chi
 * and enters the fluid as a penalization force (Liberge & Beghein,
 * "Fluid Structure Interaction modelling using Lattice Boltzmann and Volume
 * Penalization method", Sec. 2).  One time step is Algorithm 1 of Sec. 2.3:
 * collide and stream (Eqs. 17-18), macroscopic moments with the penalized
 * velocity (Eqs. 19-22), the force and torque on the body (Eqs. 25-27), the
 * rigid-body update (Eqs. 23-24, fourth-order Runge-Kutta).
 *
 * Conventions shared by every entry point:
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3.  Node (i, j), 0 <= i < nx,
 *    0 <= j < ny, sits at x = i, y = j.  Walls are half-way: x = -1/2,
 *    x = nx - 1/2, y = -1/2, y = ny - 1/2.
 *  - Host arrays of a field are row-major [ny][nx] (i fastest); population
 *    arrays are [9][ny][nx] with the velocity order of Eq. (10):
 *    c0 = (0,0), c1..c4 = (1,0),(0,1),(-1,0),(0,-1),
 *    c5..c8 = (1,1),(-1,1),(-1,-1),(1,-1).
 *  - The state after n steps is the post-collision population field of
 *    step n - 1 (for n = 0 the field set by vplbm_init_equilibrium or
 *    vplbm_set_populations).  Populations cross the ABI as full f in FP64,
 *    whatever the storage precision.
 *  - Every pointer argument is a HOST pointer unless its name ends in _dev.
 *    Host inputs are copied before the call returns; the caller keeps
 *    ownership of everything it passes.
 *  - Work is queued on the stream given at creation.  Calls that return
 *    data to the host synchronize that stream.  Errors detected on the
 *    device (non-finite density) are latched and returned by the next
 *    vplbm_sync or host read.
 *  - No call aborts or throws: every failure returns a status, and
 *    vplbm_last_error() gives a message (per calling thread).
 */
#ifndef VPLBM_H
#define VPLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Most bodies one lattice can hold (vplbm_create_bodies). */
#define VPLBM_MAX_BODIES 4

typedef enum {
    VPLBM_OK = 0,
    VPLBM_EINVAL = 1,        /* invalid argument or descriptor */
    VPLBM_ENOMEM = 2,        /* device or host allocation failed */
    VPLBM_ECUDA = 3,         /* a CUDA runtime call failed */
    VPLBM_ENONFINITE = 4,    /* a density became non-positive or non-finite */
    VPLBM_ETIMEOUT = 5,      /* a bounded device wait gave up */
    VPLBM_EUNSUPPORTED = 6,  /* valid request the library does not support */
    VPLBM_ERANGE = 7,        /* history record no longer (or not yet) stored */
    VPLBM_EIO = 8            /* file read or write failed */
} vplbm_status;

/* Storage precision of the populations.  Arithmetic is FP64 for VPLBM_F64
 * and FP32 otherwise.  The force/torque sums are FP64 for VPLBM_F64 and
 * float-float (about 44 bits, converted exactly to FP64) otherwise; the body
 * update is always FP64.  The _DEV variants store f_a - w_a rho0 (deviation
 * from rest). */
typedef enum { VPLBM_F64 = 0, VPLBM_F32_DEV = 1, VPLBM_F16_DEV = 2 } vplbm_precision;

/* Boundary kinds of one lattice edge (Sec. 3.1 / 3.2):
 *  PERIODIC  wrap around (must be set on both opposite edges);
 *  NOSLIP    half-way bounce-back, f_a(x) = f~_abar(x);
 *  VELOCITY  half-way bounce-back of a moving wall,
 *            f_a(x) = f~_abar(x) + 6 w_a rho0 (c_a . u_w);
 *  ZEROGRAD  west/east only: f_a(x) = f~_a(i, j - c_ay) from the edge column;
 *  SYMMETRY  south/north only: specular reflection at the half-way wall
 *            (u.n = 0, no shear stress), f_a(i, j) = f~_a*(i - c_ax, j) with
 *            a* the mirror image of a (c_ay -> -c_ay); where i - c_ax lies
 *            outside a non-periodic x edge, f~_a*(i, j);
 *  CONVECTIVE east only: outflow advected at the speed U = ux of this edge
 *            (>= 0), df/dt + U df/dx = 0 implicit in time and upwind in
 *            space: f_a(N, n+1) = (f_a(N, n) + U f_a(N-1, n+1)) / (1 + U),
 *            where f_a(N-1, n+1) is the zero-gradient value and f_a(N, n)
 *            the value the rule gave at the previous step (at the first
 *            step after the populations are set: their outlet column).
 *            The previous values are part of the state (checkpoints keep
 *            them).  Not with vplbm_step_noalloc or the adjoint.
 * When the source node of a pull lies outside in y, the south/north rule
 * applies, otherwise the west/east rule. */
typedef enum {
    VPLBM_BC_PERIODIC = 0, VPLBM_BC_NOSLIP = 1, VPLBM_BC_VELOCITY = 2, VPLBM_BC_ZEROGRAD = 3,
    VPLBM_BC_SYMMETRY = 4, VPLBM_BC_CONVECTIVE = 5
} vplbm_bc_kind;

enum { VPLBM_WEST = 0, VPLBM_EAST = 1, VPLBM_SOUTH = 2, VPLBM_NORTH = 3 };

typedef struct {
    int kind;                 /* vplbm_bc_kind */
    double ux, uy;            /* uniform wall velocity (VELOCITY) */
    const double *ux_profile; /* optional per-node wall velocity along the */
    const double *uy_profile; /* edge (ny values west/east, nx south/north) */
} vplbm_bc;

/* Collision operator.  MRT: Eq. (17) with the rates s[0..8].  BGK: the
 * single-relaxation-time operator of Sec. 2.1, f~ = f - (f - f_eq)/tau +
 * (1 - 1/(2 tau)) F with the equilibrium of Eq. (11) and the forcing of
 * Eq. (12); it relaxes at 1/tau = s[7] and ignores the other rates.  BGK
 * runs on the scalar step kernels only (no TMA kernel, no adjoint). */
typedef enum { VPLBM_COLLISION_MRT = 0, VPLBM_COLLISION_BGK = 1 } vplbm_collision;

/* Lattice and fluid.  s: diagonal of S (Eq. 16) in the moment order of
 * Eq. (15), each in (0, 2); eta > 0: penalization factor (Eq. 2);
 * rho0 > 0: reference density; (gx, gy): uniform body acceleration of the
 * fluid, added to the penalization force in the forcing term. */
typedef struct {
    int nx, ny;               /* >= 3 each */
    double s[9];
    double eta;
    double rho0;
    double gx, gy;
    vplbm_bc bc[4];           /* indexed by VPLBM_WEST .. VPLBM_NORTH */
    int precision;            /* vplbm_precision */
    int collision;            /* vplbm_collision (0: MRT) */
} vplbm_lattice_desc;

typedef enum {
    VPLBM_MOTION_FIXED = 0,   /* pose and velocity held at their initial values */
    VPLBM_MOTION_IMPOSED = 1, /* q_axis(t) = q_c + amp sin(2 pi freq t + phase) */
    VPLBM_MOTION_FREE = 2     /* Eqs. (23)-(24) for the DOFs in dof_mask, RK4 */
} vplbm_motion;

/* Body shapes.  DISK: chi(x) = 1 iff (i - x_G)^2 + (j - y_G)^2 <= radius^2.
 * ELLIPSE: semi-axis `radius` along the body's x axis, at the angle theta
 * of the pose, and `radius_b` across it: with u = dx cos(theta) + dy
 * sin(theta), v = dy cos(theta) - dx sin(theta), chi = 1 iff
 * radius_b^2 u^2 + radius^2 v^2 <= radius^2 radius_b^2.  RECTANGLE: half-
 * sides `radius` and `radius_b` along the same axes, chi = 1 iff |u| <=
 * radius and |v| <= radius_b.  All in FP64 without fused multiply-add; the
 * cos / sin of theta come from the host's math library for a pose set on
 * the host and from CUDA's for a pose the GPU advanced (they may differ in
 * the last bit).  The adjoint takes the disk only. */
typedef enum { VPLBM_SHAPE_DISK = 0, VPLBM_SHAPE_ELLIPSE = 1, VPLBM_SHAPE_RECTANGLE = 2 } vplbm_shape;

/* Rigid body (disk, ellipse or rectangle, see vplbm_shape).  The rigid velocity at a node is
 * u_s = (vx - omega (y - y_G), vy + omega (x - x_G)).
 * Imposed motion: q_c is chosen so that q_axis(0) equals the initial pose.
 * Free motion: m q'' + damp q' + stiff (q - q0) = F_h + f_ext per DOF
 * (x, y with mass, theta with inertia); F_h is held over the step. */
typedef struct {
    double radius;
    double x, y, theta, vx, vy, omega;
    int motion;               /* vplbm_motion */
    int axis;                 /* imposed coordinate: 0 x, 1 y, 2 theta */
    double amp, freq, phase;
    double mass, inertia;
    double damp[3], stiff[3], q0[3], f_ext[3];
    unsigned dof_mask;        /* bit0 x, bit1 y, bit2 theta */
    double u_ref, d_ref;      /* C_D = F_x / (rho0 d_ref u_ref^2 / 2), C_L alike */
    int shape;                /* vplbm_shape (0: disk) */
    double radius_b;          /* ellipse: semi-axis along the body's y axis */
} vplbm_body_desc;

/* One record per time step n.  (fx, fy, torque) is the momentum exchanged
 * through the links between the solid nodes and the rest of the lattice
 * during the streaming into step n (Eqs. 25-27 with u_Gamma = 0), the force
 * that drives a free body; (fpen_x, fpen_y, tpen) is the reaction of the
 * penalization force, sum over solid nodes of rho chi (u - u_s) / eta, and
 * its torque about x_G.  Pose and velocity are those used by step n. */
typedef struct {
    double t, fx, fy, torque, cd, cl, x, y, theta, vx, vy, omega;
    double fpen_x, fpen_y, tpen, n_solid;
} vplbm_record;

typedef struct vplbm_ctx vplbm_ctx;

/* Device memory a context needs, for callers that allocate it themselves. */
typedef struct {
    size_t populations;   /* bytes of EACH of the two population buffers */
    size_t body_state;    /* bytes of the body-state pair */
    size_t partials;      /* bytes of the per-block reduction scratch */
    size_t history;       /* bytes of the history ring */
    size_t profiles;      /* bytes of the wall-velocity profiles and the outlet state */
    size_t control;       /* bytes of the ticket / error words */
} vplbm_buffer_sizes;

typedef struct {
    void *populations_dev[2];
    void *body_state_dev;
    void *partials_dev;
    void *history_dev;
    void *profiles_dev;
    void *control_dev;
} vplbm_buffers;

/* Size of each device buffer for this lattice, body and history capacity.
 * Every buffer must be 256-byte aligned. */
vplbm_status vplbm_buffer_sizes_for(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                                    long long history_capacity, vplbm_buffer_sizes *out);

/* Create a simulation.  body may be NULL (no solid).  history_capacity
 * (>= 1) records are kept in a ring.  cuda_stream is a cudaStream_t (NULL:
 * the legacy default stream).  The library allocates its device memory.
 * The populations are left at rest (rho0, u = 0). */
vplbm_status vplbm_create(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                          long long history_capacity, void *cuda_stream, vplbm_ctx **out);

/* Same, on device buffers owned by the caller (sizes from
 * vplbm_buffer_sizes_for); the caller keeps them alive until destroy. */
vplbm_status vplbm_create_with_buffers(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                                       long long history_capacity, void *cuda_stream,
                                       const vplbm_buffers *buffers, vplbm_ctx **out);

/* Several bodies in one lattice (1 <= nbodies <= VPLBM_MAX_BODIES; bodies
 * is an array of nbodies descriptors).  Each body has its own chi, force
 * and torque sums (Eqs. 25-27 over its own solid nodes), history ring and
 * motion.  A node belongs to the first body in the array whose chi holds
 * there; bodies are meant not to overlap (Eq. 2 gives each node at most one
 * solid velocity).  The library allocates its device memory.  The scalar
 * kernels run it (VPLBM_KERNEL_TMA, the adjoint and the allocation-free
 * entry point take one body).  nbodies == 1 is the same as vplbm_create. */
vplbm_status vplbm_create_bodies(const vplbm_lattice_desc *lat, const vplbm_body_desc *bodies, int nbodies,
                                 long long history_capacity, void *cuda_stream, vplbm_ctx **out);

void vplbm_destroy(vplbm_ctx *ctx);

/* State := equilibrium (Eq. 11) of the host fields rho, ux, uy ([ny][nx]);
 * a NULL field means rho0 (for rho) or 0 (for a velocity).  Resets the
 * step counter, the history and the body to its initial pose.  A
 * page-locked (pinned, device-mapped) field is read in place by the
 * initialisation kernel over the CPU-GPU link; a pageable one is copied to
 * device memory first. */
vplbm_status vplbm_init_equilibrium(vplbm_ctx *ctx, const double *rho, const double *ux,
                                    const double *uy);

/* State := the host populations f[9][ny][nx] (full f; rounded to the
 * storage precision).  Resets step counter, history and body like init. */
vplbm_status vplbm_set_populations(vplbm_ctx *ctx, const double *f);

/* Queue nsteps >= 0 time steps on the context's stream (asynchronous). */
vplbm_status vplbm_step(vplbm_ctx *ctx, long long nsteps);

/* Wait for queued work; returns a latched device error if any. */
vplbm_status vplbm_sync(vplbm_ctx *ctx);

/* Current state, full f in FP64 [9][ny][nx] (host). */
vplbm_status vplbm_get_populations(vplbm_ctx *ctx, double *f);

/* rho, u_x, u_y of the current step (Eqs. 19-22, with chi of the current
 * pose), host arrays [ny][nx]; any pointer may be NULL.  If every given
 * array is page-locked (pinned, device-mapped) the fields kernel writes
 * them in place over the CPU-GPU link; otherwise they are staged through
 * device memory.  Returns when the arrays hold the fields. */
vplbm_status vplbm_get_fields(vplbm_ctx *ctx, double *rho, double *ux, double *uy);

/* Same into device arrays (asynchronous, on the context's stream). */
vplbm_status vplbm_get_fields_dev(vplbm_ctx *ctx, double *rho_dev, double *ux_dev, double *uy_dev);

/* Records first .. first + count - 1; VPLBM_ERANGE if any of them is not
 * yet written or already overwritten in the ring. */
vplbm_status vplbm_get_history(vplbm_ctx *ctx, long long first, long long count, vplbm_record *dst);

/* Pose (x, y, theta), velocity (vx, vy, omega) and step counter. */
vplbm_status vplbm_get_body(vplbm_ctx *ctx, double q[3], double v[3], long long *step);

/* Number of bodies of the context (0 when it was created without one). */
vplbm_status vplbm_get_num_bodies(vplbm_ctx *ctx, int *nbodies);

/* vplbm_get_history and vplbm_get_body for body k (0 <= k < the number
 * of bodies; k = 0 also for a context without a body). */
vplbm_status vplbm_get_history_body(vplbm_ctx *ctx, int k, long long first, long long count, vplbm_record *dst);
vplbm_status vplbm_get_body_k(vplbm_ctx *ctx, int k, double q[3], double v[3], long long *step);

/* Step kernels.  Both compute the same method; they differ in data movement:
 *  VPLBM_KERNEL_SCALAR     one node per thread, its nine pulls loaded straight
 *                          into registers (every precision), register budget
 *                          of 4 blocks of 256 threads per SM (64 registers):
 *                          the default for FP64 storage;
 *  VPLBM_KERNEL_SCALAR_48  the same sized for 5 blocks (48 registers);
 *  VPLBM_KERNEL_SCALAR_40  the same sized for 6 blocks (40 registers): the
 *                          default for FP32 / FP16 storage (256 x 1 blocks);
 *  VPLBM_KERNEL_TMA        persistent blocks fed by tensor-memory-accelerator
 *                          copies into a shared-memory ring (FP32/FP16
 *                          storage, nx * element size a multiple of 16 bytes,
 *                          nx >= 136 (FP32) / 144 (FP16), ny >= 4).
 *  VPLBM_KERNEL_FUSED2     two time steps per launch (FP32/FP16 storage,
 *                          a body on a prescribed path or none, one
 *                          body): a block computes
 *                          step n on its 64 x 8 tile and a one-node ring
 *                          around it into shared memory, then step n + 1
 *                          from there, so HBM is read and written once per
 *                          two steps.  A launch advances the state by
 *                          two steps but the two population buffers by
 *                          one, so vplbm_step issues them in pairs: every
 *                          call of 4 or more steps runs as pairs of
 *                          two-step launches (in 32-step graphs from an
 *                          even step, as direct launches otherwise), except
 *                          for the last nsteps mod 4 steps and, in a call
 *                          of more than 32 steps from an odd step, its
 *                          first step; those single steps run the
 *                          40-register scalar kernel on the (block_x,
 *                          block_y) given to vplbm_set_launch (0 x 0: the
 *                          current blocks).  Its populations equal the
 *                          scalar kernel's bit for bit.
 *  VPLBM_KERNEL_PAIR       two x-adjacent nodes per thread (FP32 or FP16
 *                          storage, MRT collision, one body, even nx): a block of
 *                          block_x x block_y threads updates a tile of
 *                          2 block_x x block_y nodes, loading the pulls of
 *                          both nodes, running the update on paired FP32
 *                          instructions and storing 32-bit pairs; tiles on
 *                          a lattice edge or near the body take the
 *                          one-node code.  Its populations equal the
 *                          scalar kernel's bit for bit.
 * Nodes on the lattice edges and near the body always take the same code.
 * The results of different kernels agree to the rounding of the storage
 * precision. */
typedef enum {
    VPLBM_KERNEL_SCALAR = 0, VPLBM_KERNEL_SCALAR_48 = 1, VPLBM_KERNEL_SCALAR_40 = 2, VPLBM_KERNEL_TMA = 3,
    VPLBM_KERNEL_FUSED2 = 4, VPLBM_KERNEL_PAIR = 5
} vplbm_kernel;

/* Kernel and block shape: block_x * block_y threads, block_x a multiple of
 * 32, block_x * block_y in {128, 256} (ignored for VPLBM_KERNEL_TMA).
 * VPLBM_EUNSUPPORTED if the kernel cannot run this lattice. */
vplbm_status vplbm_set_launch(vplbm_ctx *ctx, int kernel, int block_x, int block_y);
vplbm_status vplbm_get_launch(vplbm_ctx *ctx, int *kernel, int *block_x, int *block_y);

/* Time every candidate kernel and block shape on the current state (the
 * state is saved and restored around the trials) and keep the fastest. */
vplbm_status vplbm_autotune(vplbm_ctx *ctx, int steps_per_trial);

/* Test hook for the bounded waits of the TMA-staged kernel: when enabled,
 * the first shared-memory stage of every block waits for 16 bytes more than
 * its tensor copies deliver, so the wait gives up after about one second,
 * the block leaves once its copies have landed, and the next vplbm_sync
 * returns VPLBM_ETIMEOUT; the context stays usable.  Disable to resume.
 * VPLBM_EUNSUPPORTED unless the TMA-staged kernel is selected. */
vplbm_status vplbm_inject_wait_timeout(vplbm_ctx *ctx, int enable);

/* Number of step-kernel launches made by vplbm_step since creation
 * (vplbm_load restores the count saved in the checkpoint). */
vplbm_status vplbm_get_launch_count(vplbm_ctx *ctx, long long *launches);

/* Kinds of kernel launches vplbm_step makes (an index into the counts of
 * vplbm_get_kernel_launches):
 *  VPLBM_LAUNCH_ONE_STEP   one time step on a scalar step kernel (any
 *                          register budget, shape, or several bodies) or
 *                          on the node-pair kernel;
 *  VPLBM_LAUNCH_TWO_STEP   two time steps on the two-step kernel;
 *  VPLBM_LAUNCH_LOOKAHEAD  the one-thread launch that computes pose n + 1
 *                          of a prescribed path ahead of a run of two-step
 *                          launches (no lattice work);
 *  VPLBM_LAUNCH_TMA        one time step on the TMA-staged kernel. */
typedef enum {
    VPLBM_LAUNCH_ONE_STEP = 0, VPLBM_LAUNCH_TWO_STEP = 1, VPLBM_LAUNCH_LOOKAHEAD = 2, VPLBM_LAUNCH_TMA = 3,
    VPLBM_LAUNCH_KINDS = 4
} vplbm_launch_kind;

/* counts[k] := launches of kind k that vplbm_step made on this context
 * since its creation (not saved in checkpoints).  Their sum equals the
 * vplbm_get_launch_count increase over the same calls; a caller that reads
 * the counts around a call learns which kernels ran it. */
vplbm_status vplbm_get_kernel_launches(vplbm_ctx *ctx, long long counts[VPLBM_LAUNCH_KINDS]);

/* Write / read a checkpoint: populations (storage precision), body state,
 * step counter and history ring.  vplbm_load requires a context created
 * with the same lattice size, precision and history capacity. */
vplbm_status vplbm_save(vplbm_ctx *ctx, const char *path);
vplbm_status vplbm_load(vplbm_ctx *ctx, const char *path);

/* ---- discrete adjoint --------------------------------------------------------
 * Gradients of J = w_cd * mean C_D + w_cl * RMS C_L, both over the steps
 * [window_start, nsteps) of a run of nsteps steps from the current state,
 * with respect to the inlet u_x profile of the west wall (a VELOCITY wall
 * with a ux_profile), eta (Eq. 2), s_nu (= s_7 = s_8, Eq. 16) and s_e (= s_1).
 * C_D, C_L use the momentum-exchange force of each step (Eqs. 25-27).  The
 * body must move on a prescribed path (fixed or imposed; chi is the binary
 * mask of each step).  The run is the exact discrete reverse of the
 * forward steps: forward with a checkpoint every checkpoint_interval steps
 * (0: ceil(sqrt(nsteps))), then, segment by segment from the end, the
 * segment's states are recomputed and the adjoint stepped back through it.
 * The context ends at the state after the forward run (advanced by nsteps).
 * FP64 storage: FP64 adjoint; FP32 deviation storage: FP32 adjoint with
 * FP64 parameter sums.  history_capacity must be >= nsteps.
 * grad (host, ny + 3 values): dJ/du_in(j) for j < ny, then dJ/deta,
 * dJ/ds_nu, dJ/ds_e.  j_out (host, 2 values, may be NULL): J1, J2.
 * Device memory: the first call allocates a workspace of about
 * (ceil(nsteps / K) + 2 K + 3) population buffers (K the checkpoint
 * interval) and the context keeps it for later calls (a call that needs
 * more replaces it) until vplbm_destroy. */
typedef struct {
    long long nsteps;
    long long window_start;
    double w_cd, w_cl;
    long long checkpoint_interval;
} vplbm_adjoint_desc;

vplbm_status vplbm_adjoint(vplbm_ctx *ctx, const vplbm_adjoint_desc *desc, double *grad, double *j_out);

/* ---- batched sweep ---------------------------------------------------------
 * Many independent simulations of uneven lattice sizes (a parameter sweep:
 * stiffness, reduced velocity, ... as in the vortex-induced-vibration study
 * of Sec. 3.3) advanced together, each member keeping its own body, force
 * reduction, tail and history (three ways to launch them: vplbm_batch_mode).  Members are ordinary contexts (vplbm_batch_member): every
 * per-simulation call (init, fields, history, body, checkpoints) works on
 * them; vplbm_step on a single member would take it out of step with the
 * others, which vplbm_batch_step then rejects with VPLBM_EINVAL.
 * All members: the same precision. */
typedef struct vplbm_batch vplbm_batch;

/* lats[0..n-1] describe the members; bodies is NULL (no body anywhere) or an
 * array of n pointers (NULL entries: that member has no body). */
vplbm_status vplbm_batch_create(const vplbm_lattice_desc *lats, const vplbm_body_desc *const *bodies, int n,
                                long long history_capacity, void *cuda_stream, vplbm_batch **out);
void vplbm_batch_destroy(vplbm_batch *batch);   /* destroys the members too */
vplbm_status vplbm_batch_member(vplbm_batch *batch, int k, vplbm_ctx **member);
/* nsteps time steps of every member (asynchronous on the batch's stream). */
vplbm_status vplbm_batch_step(vplbm_batch *batch, long long nsteps);
/* Wait; returns VPLBM_ETIMEOUT if a barrier wait of the persistent kernel
 * gave up (reported once), else the first member's latched device error,
 * if any. */
vplbm_status vplbm_batch_sync(vplbm_batch *batch);
/* How a batch steps its members.  BRANCHES (default): each member's own step
 * kernel (its launch shape is set through vplbm_batch_member +
 * vplbm_set_launch), one CUDA-graph branch per member so the members run
 * concurrently.  TILES: one launch per time step over the concatenated
 * tiles of every member, shaped by vplbm_batch_set_launch.  PERSISTENT
 * (FP32 or FP16 storage, MRT collision; VPLBM_EUNSUPPORTED otherwise): one
 * cooperative launch runs up to 1024 time steps of every member (a CUDA
 * graph of that launch from an even step), its blocks resident for the
 * whole launch, taking work items (each member's body tiles, then node-pair
 * tiles of two x-adjacent nodes per thread, one-node tiles for an odd nx)
 * from a queue and meeting at a grid-wide barrier after every step; shaped
 * by vplbm_batch_set_persistent.  In every mode a member's populations,
 * forces and trajectory are those of its own step kernel at the same
 * block shape. */
typedef enum { VPLBM_BATCH_BRANCHES = 0, VPLBM_BATCH_TILES = 1, VPLBM_BATCH_PERSISTENT = 2 } vplbm_batch_mode;
vplbm_status vplbm_batch_set_mode(vplbm_batch *batch, int mode);
vplbm_status vplbm_batch_get_mode(vplbm_batch *batch, int *mode);
/* Launch shape of the batched kernel (TILES mode): blocks of block_x x block_y threads
 * (block_x a multiple of 32, block_x * block_y in {128, 256}), each running
 * tiles_per_block (1..64) tiles of that shape stacked in y, so the member
 * lookup and parameter staging of a block are shared by that many tiles.
 * get_launch also returns the number of batched step launches made so far.
 * EINVAL for a shape outside these limits or one that needs more reduction
 * slots than a member allocated (the previous shape is kept). */
vplbm_status vplbm_batch_set_launch(vplbm_batch *batch, int block_x, int block_y, int tiles_per_block);
vplbm_status vplbm_batch_get_launch(vplbm_batch *batch, int *block_x, int *block_y, int *tiles_per_block,
                                   long long *launches);
/* Shape of the persistent kernel: blocks of block_x x block_y = 256 threads
 * (block_x a multiple of 32); node-pair tiles of 2 block_x x block_y nodes,
 * body and one-node tiles of block_x x block_y; a block takes chunk (1..16)
 * work items from the queue at a time; params_in_shared != 0 copies a
 * member's parameters to shared memory when a block's member changes
 * (otherwise they are read from device memory where they are used).
 * EINVAL for a shape outside these limits or one that needs more reduction
 * slots than a member allocated (the previous shape is kept);
 * VPLBM_EUNSUPPORTED for FP64 storage or BGK collision. */
vplbm_status vplbm_batch_set_persistent(vplbm_batch *batch, int block_x, int block_y, int chunk,
                                       int params_in_shared);
/* The persistent shape, the grid (blocks kept resident on the device) and
 * the number of persistent launches made so far.  Any pointer may be NULL. */
vplbm_status vplbm_batch_get_persistent(vplbm_batch *batch, int *block_x, int *block_y, int *chunk,
                                       int *params_in_shared, int *grid, long long *kernel_launches);
/* Test hook for the bounded barrier waits of the persistent kernel: when
 * enabled, every grid-wide barrier waits for one arrival more than the grid
 * makes and gives up after 20 ms; the launch's blocks then leave, and the
 * next vplbm_batch_sync returns VPLBM_ETIMEOUT once (the members hold the
 * state of an unfinished step: initialise or load them again).  Disable to
 * resume. */
vplbm_status vplbm_batch_inject_barrier_timeout(vplbm_batch *batch, int enable);
/* Time the branch mode with six member launch choices (every member set to
 * one scalar or node-pair kernel and block shape), six tile-mode launch
 * shapes and (FP32/FP16, MRT) six persistent variants over 2 x
 * steps_per_trial steps each (rounded up to whole 32-step graphs) and keep
 * the fastest (members keep the winning launch choice; the tile-mode and
 * persistent shapes are the fastest of their mode whichever mode won, so
 * that vplbm_batch_set_mode afterwards runs at them); the trial steps
 * advance the members (they are real steps). */
vplbm_status vplbm_batch_autotune(vplbm_batch *batch, int steps_per_trial);

/* ---- allocation-free stepping --------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory while they run: a host application whose
 * device memory belongs to another framework's caching allocator (an extra
 * cudaMalloc would fail or fragment that pool), or a control loop with a
 * fixed memory budget that forbids allocation after start-up, since
 * cudaMalloc and cudaFree can synchronize the device and take unbounded time.
 *
 * vplbm_step_noalloc queues nsteps time steps -- the same fused step kernel
 * as vplbm_step -- on buffers the caller owns, and allocates nothing: the
 * kernel's scratch (block force partials, tail ticket, error word, internal
 * pose records) is one static device array of about 260 KB that every GPU
 * loading this library holds until the process exits.  Its device address is
 * looked up on the first call on each device (with that device current), so
 * make that first call before any stream capture.  The address is kept for
 * the life of the process and belongs to the context that was current at
 * that first call: do not use this entry point on a device after
 * cudaDeviceReset (or from another context on it).  All calls share the
 * array: calls whose work overlaps on the GPU (other streams, other threads)
 * race on it and must be serialized by the caller.
 *
 *  populations_dev[0]  device buffer holding the state in storage layout:
 *                      9 planes, plane stride = nx*ny rounded up to a
 *                      multiple of 128 elements, element (a, j, i) at
 *                      a*stride + j*nx + i; FP64 full f for VPLBM_F64,
 *                      FP32 / FP16 of f_a - w_a rho0 for the _DEV kinds.
 *  populations_dev[1]  second buffer of the same size; after the call the
 *                      state is in populations_dev[nsteps & 1].
 *  state_dev           device vplbm_body_state, read at the start, written at
 *                      the end (pose and velocity after the steps, step
 *                      counter advanced by nsteps, error != 0 if a density
 *                      became non-positive or non-finite).
 *  history_dev         NULL, or a device ring of history_capacity records;
 *                      the record of step n goes to slot n % capacity.
 * Buffers must be aligned: the population buffers to the storage element
 * size, state_dev and history_dev to 8 bytes (VPLBM_EINVAL otherwise, before
 * any device work).
 * Walls take uniform velocities only (bc[].ux_profile/uy_profile must be
 * NULL: VPLBM_EUNSUPPORTED).  A disk too large for the fixed scratch (radius
 * above about 450 lattice units) is rejected with VPLBM_ERANGE before any
 * device work.  Asynchronous on cuda_stream; read state_dev after
 * synchronizing. */
typedef struct {
    double q[3];      /* x_G, y_G, theta */
    double v[3];      /* vx, vy, omega */
    long long step;   /* step counter: time of q and v */
    int error;        /* output: non-zero if the call saw a non-finite density */
    int pad;
} vplbm_body_state;

vplbm_status vplbm_step_noalloc(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                                void *const populations_dev[2], vplbm_body_state *state_dev,
                                vplbm_record *history_dev, long long history_capacity,
                                long long nsteps, void *cuda_stream);

/* ---- diagnostics ---------------------------------------------------------
 * y_dev[k] := the FP32 reciprocal the FP32 / FP16 step kernels use for
 * 1/rho in u = j / rho (Eq. 22): the hardware reciprocal estimate refined
 * by one Newton-Raphson step, r0 + r0 (1 - x r0) with fused multiply-adds.
 * Subnormal inputs and outputs are flushed to zero.  x_dev and y_dev are
 * device arrays of n floats (4-byte aligned; VPLBM_EINVAL otherwise);
 * asynchronous on cuda_stream.  For tests of the reciprocal's error bound. */
vplbm_status vplbm_eval_recip_f32(const float *x_dev, float *y_dev, long long n, void *cuda_stream);

/* Message of the last failed call on this thread (never NULL). */
const char *vplbm_last_error(void);

/* Library version string. */
const char *vplbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VPLBM_H */
