/*
 * lbsph — lattice Boltzmann for moving rigid spheroids on NVIDIA GB300 (sm_103a).
 *
 * C ABI of the CUDA library.  The method is the one of Thampi, Stratford and
 * Henrich, "Simulating dynamics of ellipsoidal particles using lattice
 * Boltzmann method": a D3Q19 lattice Boltzmann fluid (Sec. II.A, Eq. 1-4)
 * coupled to rigid ellipsoids by link bounce-back on moving boundaries
 * (Sec. II.B, Eq. fb and Eq. ub), momentum-exchange forces split into
 * velocity-independent parts and drag matrices (Eq. Fsplit-Eq. drag4), and an
 * implicit update of translational / angular velocity with a quaternion
 * orientation (Sec. II.C-D, Eq. Fdiscrete, Eq. Tdiscrete, Eq. posupdate,
 * Eq. qnplus0-1, Eq. Irot, Eq. Irotdiff), one iteration being the ten steps of
 * the paper's Appendix.
 *
 * Conventions for every entry point:
 *  - Every call returns lb_status; nothing throws or aborts across the ABI.
 *    lb_last_error() gives a message for the last failing call on a context.
 *  - The caller owns every buffer it passes; the library copies inputs and
 *    never keeps a caller pointer after the call returns.
 *  - The library owns its device memory.  It allocates through
 *    lb_options.alloc / lb_options.release when given (e.g. the PyTorch caching
 *    allocator), else with cudaMalloc / cudaFree.
 *  - Calls taking a stream enqueue work on it (NULL = the context's own
 *    stream) and return without waiting, except the getters, which wait for
 *    the work they need.  Device-side errors (a NaN in a particle state, a
 *    particle too large for the configured scratch, particles that come too
 *    close) are recorded in a device status word and returned by the next call
 *    that synchronises (the getters, lb_synchronize).
 *  - A context is not thread safe.  Units are lattice units (dx = dt = 1).
 *  - Quaternions are (q0, q1, q2, q3), unit, Hamilton product, rotating body
 *    axes into the lab frame (Eq. vectrotn); the body x axis is the axis of
 *    semi-axis a (the spheroid's long axis e).
 */
#ifndef LBSPH_H
#define LBSPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBSPH_ABI_VERSION 5

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,      /* bad argument; nothing was changed                  */
    LB_ENOMEM = 2,      /* device allocation failed                           */
    LB_ECUDA = 3,       /* a CUDA call failed (no device, launch error, ...)  */
    LB_ETIMEOUT = 4,    /* a bounded device-side wait gave up                 */
    LB_ENAN = 5,        /* a particle state became NaN or Inf                 */
    LB_EOVERLAP = 6,    /* particles (or a particle and a wall) came too close */
    LB_ECAPACITY = 7,   /* a particle outgrew the scratch sized at lb_create  */
    LB_ESTATE = 8       /* call not allowed in the context's current state    */
} lb_status;

/* storage of the distributions, always as deviations f_i - w_i rho0 */
enum { LB_FP32 = 0, LB_FP16 = 1, LB_BF16 = 2 };

/* field selectors for lb_get_fields */
enum {
    LB_FIELD_F = 1u,      /* f_i, float32, [Q][nz][ny][nx] (Q = 19 or 27); 0 on solid nodes */
    LB_FIELD_DF = 2u,     /* f_i - w_i rho0, float32, same layout                  */
    LB_FIELD_RHO = 4u,    /* rho - rho0, float32, [nz][ny][nx]; 0 on solid nodes  */
    LB_FIELD_U = 8u,      /* u = (sum f c + g/2)/rho, float32, [3][nz][ny][nx]     */
    LB_FIELD_SOLID = 16u  /* owner, int32, [nz][ny][nx]: 0 fluid, -1 wall, p+1     */
};

/* option flags */
enum {
    LB_FLAG_SEPARATE_KERNELS = 1u  /* run each step as four kernel launches instead of the
                                      persistent step kernel (the same arithmetic; the two
                                      compilations may contract a*b+c differently, so the
                                      results agree to FP32 round-off) */
};

/* One periodic box (x, y, z periodic) or a channel (walls != 0: the planes
 * y = 0 and y = ny-1 are solid and move with wall_u_lo / wall_u_hi).
 * nx must be a multiple of 4 (8 for 16-bit storage). */
typedef struct {
    int32_t nx, ny, nz;
    double tau;                 /* BGK relaxation time, nu = (tau - 1/2)/3 (Sec. II.A) */
    double rho0;                /* mean density; rho_0 of Eq. fb                       */
    double body_force[3];       /* uniform force density on every fluid node           */
    int32_t counter_force;      /* 1: fluid also gets -sum(F_ext)/N_fluid (zero net)   */
    int32_t walls;
    double wall_u_lo[3], wall_u_hi[3];
    /* Lubrication correction between particles of the box (0: none).  Below
     * this gap h_c (lattice units, at most 4; 2/3 is the usual choice) the
     * squeeze force of two spheres that the lattice does not resolve is added
     * along the line of centres (the Nguyen-Ladd correction of the
     * moving-boundary method of Sec. II.B; the paper itself does not use it):
     * F_a = -6 pi mu R^2 (1/h - 1/h_c) (n . (U_a - U_b)) n = -F_b, n the unit
     * vector from a to b, h = |x_b - x_a| - R_a - R_b with R = (n^T A n)^(-1/2)
     * each body's centre-to-surface distance along n (A of
     * Eq. ellipsoidsurface), R = R_a R_b / (R_a + R_b), mu = rho0 (tau - 1/2)/3,
     * h >= 0.1, velocities of time t, the coefficient at most the reduced mass
     * M_a M_b / (M_a + M_b).  It is part of the reported F and enters the
     * right-hand side of Eq. Fdiscrete. */
    double lub_cut;
} lb_box_desc;

typedef struct {
    int32_t precision;          /* LB_FP32 | LB_FP16 | LB_BF16                        */
    int32_t didt_mode;          /* I(t+1) in Eq. Tdiscrete: 0 I + dI/dt (Eq. Irotdiff);
                                   1 I + (I(t) - I(t-1)); 2 predictor-corrector: the mode-0
                                   solution predicts q(t+1) and the system is solved again
                                   with I(q(t+1)) (Eq. Irot; Sec. II.D names it)      */
    int32_t device;             /* CUDA device ordinal                               */
    uint32_t flags;             /* LB_FLAG_*                                          */
    int32_t max_semi;           /* largest semi-axis any particle will have (<= 29)  */
    int32_t max_particles;      /* total particles over all boxes (sizes the state)  */
    double fp16_scale;          /* LB_FP16: stored value = deviation * scale; 0 = 2^14 */
    void* (*alloc)(size_t bytes, void* user);   /* optional device allocator          */
    void (*release)(void* ptr, void* user);
    void* alloc_user;
    /* Collision: 0 BGK (Eq. 3-4); 1 the paper's scheme (Sec. II.A): one
     * relaxation time for the non-conserved hydrodynamic modes, the
     * non-hydrodynamic (ghost) modes set to equilibrium in every collision,
     * i.e. f_i' = feq_i + (1 - 1/tau) w_i [c_i.j_neq / c_s^2 + (c_i c_i -
     * c_s^2 I) : Pi_neq / (2 c_s^4)] + the Guo source; the same as BGK at
     * tau = 1.  1 needs LB_FP32 storage. */
    int32_t collision;
    /* Lattice: 0 or 19 D3Q19; 27 D3Q27, the lattice the paper compares D3Q19
     * with (Sec. III.A: all 27 velocities of {-1,0,1}^3, weights 8/27, 2/27,
     * 1/54, 1/216, c_s^2 = 1/3).  27 takes LB_FP32 storage, either collision,
     * periodic boxes (walls 0) and at most one passive particle per box (B1 =
     * B2 = 0); its distributions and fields have 27 planes in the order of
     * lb_lattice_q(27, ...).  With 27, lb_step_io, lb_get_force_torque_async,
     * lb_profile_step, lb_autotune, lb_init_fluid and lb_stokes_field return
     * LB_ESTATE. */
    int32_t lattice;
} lb_options;

typedef struct {
    double semi[3];             /* a (body x, long axis e), b (body y), c (body z)     */
    double x[3];                /* centre                                             */
    double q[4];                /* orientation, unit; divided by its norm on input     */
    double U[3], Omega[3];      /* initial velocity and angular velocity              */
    double density;             /* particle density; M = density * 4/3 pi a b c      */
    double F_ext[3], T_ext[3];  /* external force and torque                          */
    double B1, B2;              /* squirmer slip modes (Eq. squirmer); 0 = passive    */
} lb_particle;

/* Number of doubles per particle written by lb_get_force_torque. */
#define LB_RECORD_DOUBLES 25

/* Creates a context holding nbox boxes, all fluid at rest (f_i = w_i rho0).
 * Validates every descriptor (sizes >= 4, nx a multiple of 4 or 8, tau > 1/2,
 * rho0 > 0) and allocates: two distribution buffers (2*19*N*s bytes, s = 4 or
 * 2), per particle a ring of two occupancy bitmasks and its state.
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA.  *out is NULL on error. */
lb_status lb_create(const lb_box_desc* boxes, int32_t nbox, const lb_options* opt, lb_ctx** out);

/* Frees every allocation of the context (after waiting for its work). */
lb_status lb_destroy(lb_ctx* ctx);

/* Places n particles in box `box` (replacing any set before) and builds their
 * solid nodes (Eq. ellipsoidsurface), boundary links and drag matrices
 * (Eq. drag1-drag4).  Allowed only before the first lb_step.  Particles may
 * come as close as the lattice allows: where the bounding cubes of two
 * particles reach each other (partners, at most 8 per particle), the nodes
 * between them are updated once with the links of both surfaces, and the
 * critical parts of such a cluster run after all of its boundary work.
 * Errors: LB_EINVAL (bad semi-axes, semi-axis > max_semi, too many particles,
 * more than 64 particles in the box, a box too small for two nearby cubes,
 * a particle touching a wall), LB_ECAPACITY (more than 8 partners), LB_EOVERLAP
 * (two bodies share a node), LB_ESTATE (after a step).  During a run, two
 * bodies that come to share a node stop it with LB_EOVERLAP. */
lb_status lb_set_particles(lb_ctx* ctx, int32_t box, const lb_particle* p, int32_t n);

/* Sets F_ext and T_ext of the n particles of `box` (box = -1: all particles of
 * all boxes, in box order) from a host array ft[n][6] = (F_ext, T_ext); one
 * copy on `stream`, in effect from the next iteration.  Pinned host memory
 * makes the copy asynchronous; the caller keeps ft valid until it completes. */
lb_status lb_set_external(lb_ctx* ctx, int32_t box, const double* ft, int32_t n, void* stream);

/* Advances every box by nsteps iterations of the Appendix algorithm (collide,
 * stream with link bounce-back, F0/T0, inertia, implicit solve, position and
 * quaternion update, remap with covered/uncovered nodes, drag matrices).
 * Asynchronous on `stream` (a cudaStream_t, NULL = the context's stream).
 * After the first collision the steps run in a persistent cooperative kernel
 * that occupies every SM, up to 256 iterations per launch; its grid barriers
 * give up after about two seconds and then report LB_ECUDA.  On a stream that
 * is being captured into a CUDA graph the launches are recorded instead of run:
 * after the first step, a graph of an even number of steps (the two
 * distribution buffers return to the same parity) can be replayed any number of
 * times to continue the run; wait for the replays (e.g. lb_synchronize) before
 * the getters. */
lb_status lb_step(lb_ctx* ctx, int32_t nsteps, void* stream);

/* Writes the fields `what` (one LB_FIELD_* bit) of box `box` at the current
 * time t: f(x, t) is the pre-collision distribution at the start of
 * iteration t.  dst gets dst_bytes bytes (must equal the field's size); it is
 * device memory when dst_is_device != 0.  Waits for completion. */
lb_status lb_get_fields(lb_ctx* ctx, int32_t box, uint32_t what, void* dst, size_t dst_bytes,
                        int32_t dst_is_device, void* stream);

/* Copies, for the n particles of box `box` (box = -1: all particles of all
 * boxes, in box order), LB_RECORD_DOUBLES doubles each:
 * F0[3], T0[3] (Eq. F0, Eq. T0 of the last iteration), F[3], T[3] (Eq. Fsplit /
 * Eq. Tsplit with the new velocities), U[3], Omega[3], x[3], q[4] at the
 * current time.  out is host memory (one device-to-host copy).  Waits for the
 * context's work on `stream` (NULL = its own stream). */
lb_status lb_get_force_torque(lb_ctx* ctx, int32_t box, double* out, int32_t n);

/* Like lb_get_force_torque, but only enqueues the copy of the records on
 * `stream` (NULL = the context's stream), behind the work already queued there
 * and behind the last lb_step, and returns at once.  out (n * LB_RECORD_DOUBLES
 * doubles) must be pinned host memory or device memory and stay valid; it holds
 * the records once the stream (or lb_synchronize) has been waited for.  Meant
 * for pipelined loops that queue inputs, steps and record copies for many
 * steps and wait once.  Not part of the paper.
 * Errors: LB_EINVAL (bad box, buffer or count), LB_ECUDA; device errors of the
 * steps surface at the next call that waits. */
lb_status lb_get_force_torque_async(lb_ctx* ctx, int32_t box, double* out, int32_t n, void* stream);

/* nsteps iterations with per-step input and output, queued on `stream` by the
 * library (one call instead of three per step): before iteration k the
 * external forces and torques of all particles come from ft + k*np*6 (the
 * layout of lb_set_external over all boxes; ft may be NULL: unchanged), after it
 * all particle records go to rec + k*np*LB_RECORD_DOUBLES (the layout of
 * lb_get_force_torque over all boxes; rec may be NULL: not copied).  np is the
 * total number of particles.  ft and rec stay valid until the stream has been
 * waited for; returns without waiting.  When the GPU can address them
 * (page-locked host memory, reached over the coherent CPU-GPU link of a Grace
 * system, or device or managed memory) the persistent step kernel reads each
 * step's forces and writes each step's records itself, so a long run records
 * its whole trajectory (forces, torques, velocities, poses of every step) at
 * the speed of lb_step; pageable memory falls back to three queued copies and
 * launches per step.  Not part of the paper.
 * Errors: those of lb_step, lb_set_external and lb_get_force_torque_async. */
lb_status lb_step_io(lb_ctx* ctx, int32_t nsteps, const double* ft, double* rec, void* stream);

/* Boundary links (x fluid, x + c_b solid) of particle `particle` of box `box`
 * at the current time, compacted on the device: pairs[2k] = node index
 * (z*ny + y)*nx + x of the fluid node, pairs[2k+1] = direction index b in the
 * library's order of the context's lattice (lb_lattice_q).  *count = number of links (all of them
 * are written only if count <= cap).  Waits for completion. */
lb_status lb_get_links(lb_ctx* ctx, int32_t box, int32_t particle, int32_t* pairs, int32_t cap,
                       int32_t* count);

/* The 6x6 drag matrix [[zeta_FU, zeta_FOmega], [zeta_TU, zeta_TOmega]] of
 * Eq. drag1-drag4 for the current links of a particle, row-major. */
lb_status lb_get_drag(lb_ctx* ctx, int32_t box, int32_t particle, double* out36);

/* Runs nsteps iterations like lb_step but launches every kernel directly, in
 * sequence on `stream`, with a CUDA event between consecutive kernels, and
 * returns the summed device time in milliseconds of the bulk lattice kernels
 * (ms_out[0]), the boundary kernels (ms_out[1]), the critical particle kernels
 * (ms_out[2]) and the auxiliary particle kernels (ms_out[3]).  Waits for
 * completion.  For measurement only. */
lb_status lb_profile_step(lb_ctx* ctx, int32_t nsteps, void* stream, double* ms_out);

/* Autotuner of the time-step kernel's launch shape for this context's boxes:
 * runs, each for 2 + steps_per_candidate iterations timed with CUDA events,
 * (1) the number of blocks that share one particle's boundary nodes (1, 2, 3,
 * the size-based default d, 2d and 3d: those below d whose node lists fit
 * 100 KB of shared memory and whose threads still cover every row of the
 * largest bounding cube, those above d while every particle item still gets a
 * block of its own), then (2) the number of consecutive 128-node bulk
 * units a warp takes per fetch from the work counter (1, 2, 4, 8), and keeps the
 * fastest of each for later lb_step calls.  The candidates compute the same
 * values bit for bit, so tuning advances the simulation exactly as lb_step
 * would.  out3 (may be NULL): units per fetch kept, blocks per particle kept,
 * iterations advanced (including the first collision if none ran yet).
 * ms_per_step (may be NULL, 10 doubles): time per iteration of each candidate,
 * blocks per particle 1, 2, 3, d, 2d, 3d then units per fetch 1, 2, 4, 8 (0
 * where a candidate was skipped).  Not part of the paper.  Waits for
 * completion.  Errors: LB_EINVAL, LB_ESTATE (separate-kernels mode), LB_ECUDA. */
lb_status lb_autotune(lb_ctx* ctx, int32_t steps_per_candidate, void* stream, int32_t* out3, double* ms_per_step);

/* Waits for all work of the context and returns the device status word's error. */
lb_status lb_synchronize(lb_ctx* ctx);

/* Boundary links of one spheroid, for callers that cannot allocate device
 * memory: a plug-in running inside a host program that owns the device's
 * memory pool and forbids raw allocations, or a real-time loop that cannot take
 * the implicit synchronisation of cudaMalloc.  The paper has no counterpart of
 * this entry point; it computes what lb_get_links returns for a particle with
 * this pose in a box of nx x ny x nz nodes (walls != 0: solid planes y = 0 and
 * y = ny-1), without a context.
 *
 * Inputs: semi[3], q[4] (unit), x[3] in host memory.  Outputs, in caller-owned
 * device memory: pairs_dev[2k] = node index (z*ny + y)*nx + x of the fluid node,
 * pairs_dev[2k+1] = direction b (lb_lattice order), for k < min(count, cap), in
 * no particular order, and *count_dev = the number of links.  Asynchronous on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).
 *
 * Allocates nothing: the occupancy bitmap and the counter are kept in one
 * file-scope device array of 32 KiB + 256 B, held by every GPU that loads the
 * library until the process exits.  The maximum is a bounding cube of 64 nodes
 * a side, i.e. semi-axes up to 29 lattice units; larger particles (or a cube
 * larger than the box) return LB_ECAPACITY.  Every call looks up the array's
 * address in the current device's context (cudaGetSymbolAddress, no allocation
 * and no synchronisation), so a context that was reset and created again is
 * served at its new address; the first call on a device may load the module,
 * so make it before any stream capture.  Every call shares the array and
 * clears it first; calls whose work overlaps on the GPU race on it, so
 * serialise them (one stream, or events).
 * Errors: LB_EINVAL (bad pose, sizes or pointers), LB_ECAPACITY, LB_ECUDA. */
lb_status lb_links_noalloc(const double* semi, const double* q, const double* x, int32_t nx, int32_t ny,
                           int32_t nz, int32_t walls, int32_t* pairs_dev, int32_t cap, int32_t* count_dev,
                           void* stream);

/* Sets the initial fluid of box `box` (before the first lb_step, after
 * lb_set_particles) to the local equilibrium f_i = f_eq_i(rho0 + drho(x), u(x))
 * of the velocity field u (FP32 [3][nz][ny][nx], u_bytes = 3*N*4) and the
 * density deviation drho (FP32 [nz][ny][nx], NULL = uniform rho0) on every fluid
 * node; solid and wall nodes keep no distributions.  u and drho are host memory,
 * or device memory if is_device.  with_stress != 0 adds the first-order
 * (Chapman-Enskog) non-equilibrium part of a viscous flow,
 *   f_i += -3 tau rho w_i (c_ia c_ib - delta_ab / 3) d_a u_b,
 * rho = rho0 + drho, d_a the periodic central difference of u, so that the
 * populations start with the flow's viscous stress (second moment
 * -tau rho c_s^2 (grad u + grad u^T)) instead of none, which otherwise relaxes
 * in the first steps and launches shear and sound waves through the box.  The
 * first iteration then collides these distributions in place (the Appendix's
 * step 1 at t = 0) instead of the rest state.  Not part of the paper: this is
 * the fluid half of the learned warm start (lbsurrogate.h).  Waits for
 * completion.
 * Errors: LB_EINVAL (bad box or size), LB_ESTATE (after a step), LB_ECUDA. */
lb_status lb_init_fluid(lb_ctx* ctx, int32_t box, const float* u, size_t u_bytes, const float* drho,
                        int32_t is_device, int32_t with_stress, void* stream);

/* The periodic steady flow that the particles of box `box` drive in the lattice
 * fluid, with its density: g puts each particle's F_ext uniformly on the fluid
 * nodes next to it (a face neighbour is its solid node: a uniform traction
 * just outside the surface) and the box's body force plus, with counter_force,
 * the balancing -sum F_ext / N_fluid on the fluid nodes; a net mean force is
 * dropped.  The flow is the exact steady state of the linear lattice dynamics
 * itself (D3Q19 BGK with Guo forcing at the box's tau and rho0), solved mode by
 * mode in Fourier space (DFTs on the device, a 4 x 4 system in the conserved
 * moments per mode in FP64): at the scales of a few nodes the lattice's own
 * viscous and pressure operators differ from a Stokes stencil by several per
 * cent, and only a start on the lattice's own steady state avoids the slow
 * relaxation of that difference.  Then a uniform velocity is added on the
 * fluid nodes so that rho0 sum_fluid u + sum_p M_p U_p = 0 with the particles'
 * current (initial) velocities, the total momentum of a run that starts from
 * rest under balanced forces.  u_dev: device FP32 [3][nz][ny][nx]; drho_dev
 * (device FP32 [nz][ny][nx], may be NULL): the density deviation of the steady
 * state (zero mean over the fluid nodes).  Fully periodic boxes only, before
 * the first step (it reads the particles' initial solid nodes).  This is the
 * fluid half of a warm start (feed both to lb_init_fluid).  Not part of the
 * paper.  Waits for completion.
 * Errors: LB_EINVAL (walls, edge > 4096), LB_ESTATE, LB_ENOMEM, LB_ECUDA. */
lb_status lb_stokes_field(lb_ctx* ctx, int32_t box, float* u_dev, float* drho_dev, void* stream);

/* The library's D3Q19 table: c[19][3] and w[19] (1/3, 1/18, 1/36). */
void lb_lattice(int32_t* c57, double* w19);

/* The library's table of lattice q (19 or 27): c[q][3] and w[q], either may
 * be NULL.  The D3Q27 order is the D3Q19 one followed by the eight corners in
 * +/- pairs (+++, ---, ++-, --+, +-+, -+-, -++, +--); for every direction b > 0
 * the opposite one is b + 1 (b odd) or b - 1 (b even).  Weights for |c|^2 = 0,
 * 1, 2, 3: 8/27, 2/27, 1/54, 1/216 (Sec. III.A names the lattice; these are
 * its standard weights, c_s^2 = 1/3).  Errors: LB_EINVAL for another q. */
lb_status lb_lattice_q(int32_t q, int32_t* c, double* w);

const char* lb_status_string(lb_status s);
const char* lb_last_error(const lb_ctx* ctx);
int32_t lb_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
