/*
 * lbsq.h -- C ABI of a GB300-native (sm_103a) lattice Boltzmann library for
 * squirmers, after Kuron, Staerk, Burkard, de Graaf & Holm, "A Lattice
 * Boltzmann Model for Squirmers" (arXiv:1903.04799).
 *
 * One context = one periodic D3Q19 lattice resident on one GPU, with
 * spherical bodies (squirmers, fixed obstacles) and plane walls.  One time
 * step does, on the GPU:
 *   - the fused stream-collide of every cell with the TRT (or BGK) operator
 *     of Sec. III, Eq. "lb" (in-place AA pattern, populations stored as FP64,
 *     or as FP32 / FP16 / BF16 deviations from w_i rho0 collided in FP32);
 *   - shifted link bounce-back on every boundary link (Sec. III), with the
 *     wall velocity v + omega x r of Eq. "vb" plus the squirmer slip of
 *     Eq. "squirmer";
 *   - the momentum-exchange force and torque of Eqs. "bbforce", "bbtorque"
 *     summed per body in FP64 in a fixed order;
 *   - a symplectic Euler update of every mobile sphere (Sec. III, last
 *     paragraph), including the optional WCA contact force of Eq. "wca";
 *   - the fluid/solid conversion of cells a moving sphere covers or
 *     uncovers, with the conversion force of Eq. "consforce", and the
 *     rebuild of the boundary-link lists.
 *
 * Conventions
 *   - Units are lattice units (a_grid = tau_grid = 1).
 *   - Cells are indexed x-fastest: n = x + nx*(y + ny*z), 0 <= x < nx ...
 *   - The lattice is periodic on all three axes; confinement is built from
 *     wall cells (lb_add_wall).
 *   - Every call returns an lb_status; out-parameters are written only on
 *     LB_OK.  No C++ exception crosses this boundary.
 *   - lb_step is stream-ordered: it enqueues work on the context's stream
 *     and returns.  Errors found on the device (overlap, capacity, a
 *     diverged body) are reported by the next synchronising call (lb_sync
 *     and every getter).  An error found on the device is sticky: the
 *     context then refuses lb_step with LB_ERR_STATE.
 *   - A context must not be used from two host threads at once.
 *   - Host buffers passed in are read or written before the call returns;
 *     the library keeps no pointer to them.  Device memory is owned by the
 *     context and freed by lb_destroy.
 *
 * D3Q19 velocity order (the layout of population arrays in this API):
 *   i = 0 rest; 1,2 = (+-1,0,0); 3,4 = (0,+-1,0); 5,6 = (0,0,+-1);
 *   7,8 = +-(1,1,0); 9,10 = +-(1,-1,0); 11,12 = +-(1,0,1); 13,14 = +-(1,0,-1);
 *   15,16 = +-(0,1,1); 17,18 = +-(0,1,-1).  The opposite of i >= 1 is
 *   i+1 for odd i and i-1 for even i.
 */
#ifndef LBSQ_H
#define LBSQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID = 1,  /* bad argument; nothing changed */
    LB_ERR_OOM = 2,      /* device allocation failed */
    LB_ERR_CUDA = 3,     /* a CUDA runtime call failed (message in lb_last_error) */
    LB_ERR_OVERLAP = 4,  /* a body overlaps another body or a wall */
    LB_ERR_DIVERGED = 5, /* a body reached |v| >= 1/2 (the scheme needs |v| << 1); it is held in place */
    LB_ERR_TIMEOUT = 6,  /* a bounded device wait ran out */
    LB_ERR_STATE = 7,    /* the context holds an earlier device error */
    LB_ERR_CAPACITY = 8  /* a boundary-link list outgrew its capacity */
} lb_status;

typedef enum { LB_BGK = 0, LB_TRT = 1 } lb_collision;

/* Population storage.  LB_F64 stores f_i; the others store the deviation
 * d_i = f_i - w_i rho0 (FP16 scaled by 2^dev_scale_log2), decoded to FP32,
 * collided in FP32 and rounded to nearest even on store.  Bodies, forces and
 * the Newton-Euler update are FP64 for every storage. */
typedef enum { LB_F64 = 0, LB_F32 = 1, LB_F16DEV = 2, LB_BF16DEV = 3 } lb_storage;

/* Equilibrium (Sec. III).  LB_EQ_COMPRESSIBLE: f_i^eq = w_i rho (1 + 3 c.u +
 * 9/2 (c.u)^2 - 3/2 u.u) with u = j / rho, the reading of the paper used for
 * every result here.  LB_EQ_INCOMPRESSIBLE: the model in which the printed
 * u = sum f_i c_i holds as written (for rho0 = 1), f_i^eq = w_i (rho + rho0
 * (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)) with u = j / rho0; it applies to the
 * collision, the refill of uncovered cells, lb_set_fields and the exported
 * velocity. */
typedef enum { LB_EQ_COMPRESSIBLE = 0, LB_EQ_INCOMPRESSIBLE = 1 } lb_equilibrium;

/* Rounding of the populations the stream-collide step stores in BF16 storage
 * (a property of the storage format, not of the paper's method).
 * LB_ROUND_NEAREST: round to nearest even.  LB_ROUND_STOCHASTIC: round up
 * with probability equal to the fraction of the BF16 unit that the value
 * carries, from a counter-based hash of (step, cell, population): the
 * rounding errors are then independent from step to step and average out
 * instead of repeating in a steady flow.  The hash makes the result a
 * function of the inputs alone (the same bits alone, in a serving mix, or
 * resumed from a checkpoint).  LB_ROUND_DEFAULT: stochastic for BF16.  Other
 * storages always round to nearest. */
typedef enum { LB_ROUND_DEFAULT = -1, LB_ROUND_NEAREST = 0, LB_ROUND_STOCHASTIC = 1 } lb_rounding;

/* Optional device allocator (for example a caching allocator of the host
 * framework).  alloc returns a device pointer of at least `bytes` bytes on
 * the context's device, or NULL; free receives the same pointer and size. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, size_t bytes, void* user);
    void* user;
} lb_allocator;

typedef struct {
    int32_t nx, ny, nz;  /* lattice size, each >= 1; nx*ny*nz < 2^27 (a boundary link is
                            coded in 32 bits as cell << 5 | direction); else
                            lb_create returns LB_ERR_INVALID */
    int32_t collision;   /* lb_collision */
    double lambda_e;     /* even (viscous) relaxation rate, 0 < lambda_e < 2;
                            kinematic viscosity (1/lambda_e - 1/2)/3 (Sec. III) */
    double magic;        /* TRT magic parameter (1/le - 1/2)(1/lo - 1/2),
                            3/16 in the paper; ignored for BGK (lo = le) */
    double rho0;         /* rest density, > 0 */
    int32_t storage;     /* lb_storage */
    int32_t dev_scale_log2; /* FP16 deviation scale exponent k (store d * 2^k);
                               -1 = default 14: deviations up to 4 fit, and the
                               usual 1e-5..1e-2 stay in FP16's normal range */
    int32_t device;      /* CUDA device ordinal */
    void* stream;        /* cudaStream_t to run on; NULL = a stream the context creates */
    const lb_allocator* allocator; /* NULL = cudaMalloc / cudaFree */
    int32_t equilibrium; /* lb_equilibrium */
    int32_t rounding;    /* lb_rounding */
} lb_params;

/* Fill *p with: 32^3, BGK, lambda_e = 1, magic = 3/16, rho0 = 1, FP64,
 * default FP16 scale, device 0, own stream, cudaMalloc, compressible
 * equilibrium, default rounding. */
void lb_params_default(lb_params* p);

/* Create a lattice with every population at rest equilibrium w_i rho0 and
 * every cell fluid (Sec. III).  *out receives the context.  Errors:
 * LB_ERR_INVALID (sizes, rates, storage), LB_ERR_OOM, LB_ERR_CUDA. */
lb_status lb_create(const lb_params* p, lb_ctx** out);

/* End a simulation: free all device memory of the context (the paper's
 * method has no counterpart; the context is this library's container for
 * the lattice of Sec. III).  Synchronises the context's stream first.  NULL
 * is accepted.  Errors: LB_ERR_CUDA. */
lb_status lb_destroy(lb_ctx* c);

/* Add a sphere of radius R centred at pos (wrapped into the box) with unit
 * orientation e (normalised here) and squirmer modes B1, B2 = beta*B1
 * (Sec. II, Eq. "squirmer"; B1 = 0 gives a passive sphere).  mobile = 0
 * holds it fixed (force and torque still measured), mobile = 1 lets the
 * Newton-Euler update move it.  density: body density (mass
 * density * 4/3 pi R^3, moment of inertia 2/5 M R^2).  Cells whose node
 * lies strictly inside (|d| < R, minimum image) become solid.  *id
 * receives the body id (>= 1).  Errors: LB_ERR_INVALID (R <= 0,
 * 2R + 6 >= min(n), |e| = 0, density <= 0), LB_ERR_OVERLAP (a covered
 * cell is already solid; nothing changed). */
lb_status lb_add_squirmer(lb_ctx* c, const double pos[3], const double e[3], double R, double B1,
                          double beta, int32_t mobile, double density, int32_t* id);

/* Add a wall (static boundary, Sec. III shifted bounce-back).
 *   kind 0, plane wall:  params = {axis, index [, vx, vy, vz]} -- one layer
 *           of solid cells at coordinate `index` along `axis` (0,1,2),
 *           moving with velocity v (default 0, a no-slip wall);
 *   kind 1, square tube along z: params = {} -- plane walls at x = 0,
 *           x = nx-1, y = 0, y = ny-1 (four ids; *id receives the first);
 *   kind 2, fixed sphere obstacle: params = {x, y, z, radius} -- a body that
 *           never moves and has no slip (Sec. V B obstacle);
 *   kind 3, round tube along z: params = {cx, cy, r} -- every node with
 *           (x - cx)^2 + (y - cy)^2 >= r^2 (in FP64) is a wall at rest, for
 *           the paper's tube flow (Sec. V; r > 1, the axis inside the box).
 *           Squirmers meet it in the contact force (lb_set_contact) at the
 *           surface r - 1/2 from the axis.
 * Errors: LB_ERR_INVALID, LB_ERR_OVERLAP. */
lb_status lb_add_wall(lb_ctx* c, int32_t kind, const double* params, int32_t nparams, int32_t* id);

/* WCA contact force (Eq. "wca") between mobile spheres and every other body
 * and wall, as a function of the surface gap r: -dU/dr of
 * U = 4 eps((sigma/r)^12 - (sigma/r)^6) + eps for r < 2^(1/6) sigma (gap
 * clamped below at 0.05 sigma).  eps = 0 (default) switches it off. */
lb_status lb_set_contact(lb_ctx* c, double sigma, double eps);

/* Readings of the moving-wall bounce-back of Sec. III that the paper leaves
 * open (Eq. "vb" and the shift 6 w_i rho c_i.v_b):
 *   density_of_node = 0 (default): the shift takes the rest density rho0, as
 *     in Ladd's original scheme; 1: the density of the fluid node the link
 *     leaves (the sum of its post-collision populations);
 *   velocity_at_node = 0 (default): the wall velocity v_b and the lever arm
 *     of the torque and stresslet are taken at the link midpoint x + c_i/2,
 *     where halfway bounce-back places the wall; 1: at the boundary node
 *     x + c_i, as the text of Sec. III words it.
 * The defaults reproduce the swim speeds printed in Fig. "resolution"; the
 * node reading swims about 14 % too fast at R = 4.  Both options apply to
 * every body of the context.  Errors: LB_ERR_INVALID (a value not 0 or 1). */
lb_status lb_set_link_options(lb_ctx* c, int32_t density_of_node, int32_t velocity_at_node);

/* Coupling of the spheres to the fluid.
 *   LB_COUPLE_LINKS (default): Sec. III -- the cells a sphere covers are
 *     solid, the links between them and the fluid bounce back from the moving
 *     surface, and cells the surface sweeps over are converted.
 *   LB_COUPLE_PSM: partially saturated cells (Noble and Torczynski, the
 *     remedy Sec. IV A names for the fluctuating swim speed of the link
 *     coupling).  Every cell stays fluid.  At the start of each step each
 *     sphere's solid fraction eps of every cell (its share of 8^3 sample
 *     points of the unit cube about the node, exact multiples of 1/512) is
 *     found; a covered cell collides with
 *       f_i + (1 - B) Omega_i + B Omega^s_i,
 *       Omega^s_i = [f_ib - f_ib^eq(rho, u)] - [f_i - f_i^eq(rho, u_s)],
 *       B = eps (tau - 1/2) / ((1 - eps) + tau - 1/2),  tau = 1 / lambda_e,
 *     Omega_i the fluid collision, u_s the surface velocity at the node
 *     (rigid motion plus the squirmer slip of Eq. "squirmer" by direction);
 *     the sphere receives -B sum_i Omega^s_i c_i from each covered cell
 *     (force, torque about its centre and stresslet), computed from the
 *     populations the step starts from.  The blended collision is FP64
 *     arithmetic for every storage; stores round to nearest.  Walls keep their
 *     links; a covered wall cell stays a wall cell.  A cell covered by two
 *     spheres sets LB_ERR_OVERLAP.  Spheres claim no cells (lb_get_owner
 *     shows none) and have no links.
 * Set it before the first sphere (obstacles of lb_add_wall kind 2 are
 * spheres).  Errors: LB_ERR_INVALID (another value, or spheres exist),
 * LB_ERR_OOM. */
typedef enum { LB_COUPLE_LINKS = 0, LB_COUPLE_PSM = 1 } lb_coupling;
lb_status lb_set_coupling(lb_ctx* c, int32_t coupling);

/* Solid fraction of every cell found at the start of the last step
 * (eps[N], x-fastest), all zero under link coupling.  Errors: LB_ERR_INVALID,
 * LB_ERR_CUDA and the device error word. */
lb_status lb_get_solid_fraction(lb_ctx* c, double* eps);

/* Ladd's two-step force average (Sec. III): with on = 1, every body's update
 * applies (F_bb(t) + F_bb(t-1)) / 2 and (T_bb(t) + T_bb(t-1)) / 2 instead of
 * this step's momentum exchange, F_bb(t-1) = 0 before a body's first step;
 * the conversion force is not averaged.  The paper leaves the average off
 * (on = 0, the default) and names it a remedy for forces that oscillate
 * between consecutive steps.  The fluid still gives up F_bb(t) each step, so
 * fluid plus body momentum plus F_bb(t)/2 is what stays constant.
 * lb_get_force_torque reports the force that entered the update.
 * Errors: LB_ERR_INVALID (on not 0 or 1). */
lb_status lb_set_force_average(lb_ctx* c, int32_t on);

/* Set every cell's populations to the equilibrium of host fields rho[N] and
 * u[3][N] (SoA, x-fastest).  Solid cells are overwritten too (harmless). */
lb_status lb_set_fields(lb_ctx* c, const double* rho, const double* u);

/* Copy all populations from / to a host buffer f[19][N] (absolute values
 * f_i, velocity order above).  Reduced storages round on set. */
lb_status lb_set_populations(lb_ctx* c, const double* f);
lb_status lb_get_populations(lb_ctx* c, double* f);

/* Enqueue nsteps >= 0 time steps.  One step is the update of Sec. III in
 * this order: stream and collide every cell (Eq. "lb"); bounce back every
 * boundary link with the moving-wall shift of the squirmer surface velocity
 * (Eq. "vb" with the slip of Eq. "squirmer"), summing the momentum exchange
 * force and torque (Eqs. "bbforce", "bbtorque"); advance each mobile body by
 * the symplectic Euler step that closes Sec. III with that force plus the
 * conversion force of Eq. "consforce" (and the WCA force of Eq. "wca" when
 * contact is on); re-classify the cells the moved bodies cover or uncover,
 * booking their momentum and refilling uncovered cells; rebuild the link
 * lists.  When the bodies occupy a thin box of
 * rows, a step's body kernels run beside the sweep of the cells away from
 * the bodies in the next step; the body kernels of the last step enqueued
 * are then issued by the next call that steps, reads or changes the context
 * (every lb_get_*, lb_set_*, lb_add_*, lb_profile_begin), so that
 * consecutive lb_step calls keep that overlap.  Results never depend on it.
 * Errors: LB_ERR_INVALID, LB_ERR_STATE, LB_ERR_CUDA. */
lb_status lb_step(lb_ctx* c, int64_t nsteps);

/* Wait for the work issued on the context's stream and report the device
 * error word (it issues no pending body kernels: see lb_step). */
lb_status lb_sync(lb_ctx* c);

/* Steps taken so far. */
int64_t lb_step_count(const lb_ctx* c);

/* Macroscopic fields (Sec. III): rho[N] and u[3][N] with u = j / rho, into
 * caller-owned HOST buffers; solid cells report 0.  Either pointer may be
 * NULL.  Synchronises. */
lb_status lb_get_fields(lb_ctx* c, double* rho, double* u);

/* As lb_get_fields, into caller-owned DEVICE buffers on the context's
 * device; stream-ordered (does not synchronise). */
lb_status lb_get_fields_device(lb_ctx* c, double* rho_dev, double* u_dev);

/* Cell owners into a host buffer owner[N]: 0 = fluid, else the body or wall id. */
lb_status lb_get_owner(lb_ctx* c, int32_t* owner);

/* Hydrodynamic force and torque on body `id` that entered the last update:
 * momentum exchange of the last step (Eqs. "bbforce", "bbtorque") plus the
 * conversion force booked by the step before (Eq. "consforce"); FP64.  For
 * walls the momentum exchange of the last step.  Synchronises. */
lb_status lb_get_force_torque(lb_ctx* c, int32_t id, double F[3], double T[3]);

/* Position, velocity, orientation and angular velocity of body `id`: the
 * state the symplectic Euler step at the end of Sec. III advances (r, v, the
 * unit swimming direction e of Eq. "squirmer", omega), after the last step
 * enqueued.  FP64, host buffers of 3 doubles each.  Synchronises.  Any
 * pointer may be NULL.  Errors: LB_ERR_INVALID (id), LB_ERR_CUDA and the
 * device errors of the steps (see above). */
lb_status lb_get_object_state(lb_ctx* c, int32_t id, double pos[3], double vel[3], double e[3],
                              double omega[3]);

/* Force dipole the surface tractions of body `id` exert on the fluid in the
 * last step: S = -sum_links symtraceless(d (x) dF), d the link midpoint
 * relative to the centre and dF the momentum given to the body on that link;
 * order xx, yy, zz, xy, xz, yz.  The paper defines no stresslet; this is the
 * traction part of Batchelor's stresslet with the sign flipped (it leaves out
 * the surface-velocity term -eta int(u n + n u) dA).  For the squirmer of
 * Eq. "squirmerflow" in unbounded Stokes flow it is
 * -(12 pi / 5) eta R^2 B2 (e e - I/3), eta = (1/lambda_e - 1/2) rho0 / 3.
 * Synchronises. */
lb_status lb_get_stresslet(lb_ctx* c, int32_t id, double S[6]);

/* Mass sum(rho) and momentum sum(j) over fluid cells, FP64, summed in a
 * fixed order (conserved to roundoff, Sec. I).  Either pointer may be NULL.
 * Synchronises. */
lb_status lb_get_mass(lb_ctx* c, double* mass, double mom[3]);

/* Boundary links of body `id` (0 = all bodies, by id), each as
 * cell_index * 32 + direction i, where cell_index is the fluid node and
 * node + c_i the solid one.  Writes at most cap entries; *count receives
 * the number of links.  Synchronises. */
lb_status lb_get_links(lb_ctx* c, int32_t id, int64_t* out, int64_t cap, int64_t* count);

/* Checkpoint and resume.  The paper's method has no counterpart: this saves a
 * run so that it can continue later, bit for bit.
 *
 * lb_checkpoint_size writes the bytes a checkpoint of the context takes now.
 * lb_checkpoint writes the checkpoint into the caller's host buffer buf of
 * `bytes` bytes (at least lb_checkpoint_size).  It holds:
 *   - the populations in the lattice's own storage;
 *   - both owner fields;
 *   - per body, its two state buffers, its accumulators (force, torque,
 *     stresslet, conversion force, averages) and its link list;
 *   - the near-body windows and the step count.
 * Pending body kernels are issued first (see lb_step).
 *
 * lb_restore loads a checkpoint into a context set up the same way: the
 * same lb_params and the same bodies, added in the same order (their
 * positions may differ: the checkpoint's replace them), and the same
 * lb_set_contact and lb_set_force_average settings (not checked).  Stepping it then
 * gives the bits the checkpointed context would have given.  The caller's
 * buffer is not kept.  The format is that of the library version that wrote it
 * (host byte order, the library's structure layouts).
 *
 * Errors: LB_ERR_INVALID (NULL, buffer too small, not a checkpoint, or one of
 * another lattice, other bodies, or a link list larger than this context
 * holds; nothing is changed then), LB_ERR_STATE (the context holds a device
 * error), LB_ERR_CUDA. */
lb_status lb_checkpoint_size(lb_ctx* c, size_t* bytes);
lb_status lb_checkpoint(lb_ctx* c, void* buf, size_t bytes);
lb_status lb_restore(lb_ctx* c, const void* buf, size_t bytes);

/* Message of the last failing call on c, or "" -- valid until the next call on c. */
const char* lb_last_error(const lb_ctx* c);

/* Number of kernel launches the context has enqueued so far (all kinds). */
int64_t lb_kernel_launches(const lb_ctx* c);

/* Tuning: the form of the stream-collide kernel (Sec. III, Eq. "lb").
 * 0 = default: FP64 storage collided in double-float arithmetic (pairs of
 * FP32 numbers, about 47 significant bits), one cell per thread; FP32 with
 * even nx: two cells per thread with paired loads; FP16 / BF16: even steps
 * as 3, odd steps as 2, except in the split steps of a lattice whose bodies
 * occupy a thin slab, where odd steps take four cells per thread without
 * shared memory (nx a multiple of 4).
 * 1 = one cell per thread; for FP64 storage, FP64 arithmetic.
 * 2 = two cells per thread where nx is even (not FP64).
 * 3 = FP16 / BF16: four cells per thread in blocks of whole rows, the
 *     odd-step x-shifts through shared memory (nx a multiple of 4 up to 768;
 *     else as 2).
 * For FP32, FP16 and BF16 the forms give identical bits; for FP64 the two
 * arithmetics agree to about 1e-14 relative per step.  LB_ERR_INVALID for
 * another value. */
lb_status lb_set_sweep_variant(lb_ctx* c, int32_t variant);

/* Kernel tracing.  Between lb_profile_begin and lb_profile_end, lb_step
 * launches each kernel of a step directly (no graph) with a CUDA event
 * recorded on the context's stream before and after it.  lb_profile_end
 * synchronises and writes, per kernel kind in launch order
 *   0 sweep, 1 links (bounce-back, force reduction, Newton-Euler; with
 *   partially saturated cells also the solid fractions and the spheres'
 *   forces and updates), 2 classify, 3 convert, 4 rebuild, 5 tick (end of step),
 * the summed device time in ms (total_ms[6]) and the launch count
 * (launches[6]).  Either pointer may be NULL. */
lb_status lb_profile_begin(lb_ctx* c);
lb_status lb_profile_end(lb_ctx* c, double total_ms[6], int64_t launches[6]);

/* ---- Serving: many independent simulations resident at once ------------
 * A server keeps many squirmer simulations (requests) resident on one GPU and
 * advances them together: each step is one launch per storage type of a
 * persistent sweep over a packed list of tiles (fixed-size chunks of cells)
 * of every resident lattice, whatever their
 * sizes and storages, followed by the body kernels of all their bodies; the
 * steps of a round are replayed from one CUDA graph.  Requests are admitted in
 * arrival order as lattice slots and device memory (a fixed HBM budget,
 * allocated once and carved per request) free up; later requests that fit
 * may start before an earlier one that does not (at most 4 times).  A
 * request stops after its own number of steps; its results stay until
 * polled.  Every request evolves exactly as it would alone: kernels never mix
 * data of two lattices and every reduction has a fixed order per body. */
typedef struct lb_server lb_server;

typedef struct {
    int32_t device;
    void* stream;            /* cudaStream_t, or NULL: the server creates one */
    size_t hbm_budget_bytes; /* device memory for resident lattices (populations,
                                owners, boundary links); allocated at creation */
    int32_t max_resident;    /* lattice slots, 1..256 */
    int32_t round_steps;     /* steps per scheduling round (even, >= 2) */
    int32_t tile_units;      /* cells (or cell pairs) per sweep tile; 0 = pick by timing at creation */
    const lb_allocator* allocator; /* NULL = cudaMalloc / cudaFree */
} lb_server_params;

/* One simulation (a configuration of the paper's Secs. II-III):
 *   geometry 0: periodic box with one squirmer;
 *   geometry 1: square tube along z (plane walls at x, y = 0 and n-1, as
 *               lb_add_wall kind 1) with one squirmer;
 *   geometry 2: periodic box with one squirmer and a fixed obstacle sphere
 *               (obstacle = x, y, z, radius; as lb_add_wall kind 2). */
typedef struct {
    int32_t geometry;
    int32_t nx, ny, nz;
    int32_t storage;           /* lb_storage */
    int32_t collision;         /* lb_collision */
    double lambda_e, magic, rho0;
    double pos[3], e[3];       /* squirmer centre and orientation */
    double R, B1, beta;        /* squirmer radius and modes (mobile, density rho0) */
    double obstacle[4];
    double wca_sigma, wca_eps; /* contact force (Eq. "wca"), eps = 0: none */
    int64_t steps;
} lb_request;

typedef enum { LB_REQ_QUEUED = 0, LB_REQ_RUNNING = 1, LB_REQ_DONE = 2, LB_REQ_FAILED = 3 } lb_request_state;

typedef struct {
    int32_t state;       /* lb_request_state */
    int32_t status;      /* lb_status of a failed request */
    int64_t steps_done;
    double pos[3], vel[3], e[3], omega[3]; /* squirmer state at the end */
    double F[3], T[3];   /* as lb_get_force_torque, last step */
    double mean_speed;   /* mean of v.e over the updates after the half-way round */
    double mean_vel[3];  /* mean velocity over all updates */
} lb_result;

void lb_server_params_default(lb_server_params* p);
/* Errors: LB_ERR_INVALID, LB_ERR_OOM (budget not allocatable), LB_ERR_CUDA. */
lb_status lb_server_create(const lb_server_params* p, lb_server** out);
lb_status lb_server_destroy(lb_server* s);
/* Queue a request; *ticket identifies it.  Errors: LB_ERR_INVALID (sizes,
 * radius, storage, a request larger than the whole budget). */
lb_status lb_server_submit(lb_server* s, const lb_request* r, int64_t* ticket);
/* One scheduling round: retire finished requests, admit queued ones that
 * fit, advance every resident request by round_steps steps (or fewer, to its
 * end), wait for the GPU.  *running and *queued receive the counts after the
 * round (either may be NULL). */
lb_status lb_server_advance(lb_server* s, int32_t* running, int32_t* queued);
/* State and (when done) results of a request; a done request is forgotten
 * after it has been polled once.  LB_ERR_INVALID for an unknown ticket. */
lb_status lb_server_poll(lb_server* s, int64_t ticket, lb_result* out);
/* Sweep tile size in use (picked by timing when tile_units = 0), persistent
 * blocks per SM, device memory in use and total cell updates done. */
lb_status lb_server_info(const lb_server* s, int32_t* tile_units, int32_t* blocks_per_sm, size_t* bytes_used,
                         double* cell_updates);
const char* lb_server_last_error(const lb_server* s);

/* ---- Allocation-free entry point (the paper has no counterpart) ----------
 * For callers that must not allocate device memory: code that runs while a
 * host framework owns all device memory through its own pool, code inside a
 * latency-critical loop where a cudaMalloc would synchronise the device, or a
 * monitoring hook that must not change the memory footprint of the program
 * it watches.  Such callers cannot create an lb_ctx either (lb_create
 * allocates), so this call works on buffers the caller already owns.
 *
 * lb_fluid_totals_static sums mass (sum of f_i) and momentum (sum of
 * f_i c_i) over the fluid cells of a population field, like lb_get_mass,
 * and writes out[4] = {mass, jx, jy, jz}.  It calls no cudaMalloc, cudaFree
 * or allocating library routine: its per-block partial sums live in a
 * file-scope device array of LB_STATIC_PARTIALS x 4 doubles (32 KiB), which
 * every GPU that loads the library holds until the process exits.
 *   f       device, FP64 [19][n_cells] absolute populations in the velocity
 *           order of this header, cells x-fastest (the layout of
 *           lb_get_populations);
 *   owner   device int32 [n_cells], 0 = fluid (the layout of lb_get_owner),
 *           or NULL to count every cell;
 *   out     device, 4 doubles;
 *   stream  cudaStream_t, or NULL for the legacy default stream.
 * Runs on the current device, stream-ordered; it does not synchronise.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  Under CUDA's default lazy module loading that
 * first lookup also loads this entry point's device code and array onto the
 * device, which takes device memory and may synchronise; so make the first
 * call on each device during set-up, before the caller's own pool takes the
 * device memory and before any stream capture.  Later calls allocate
 * nothing.  A call made while the calling thread already holds a CUDA error
 * returns LB_ERR_CUDA, launches nothing and leaves that error in place.
 * Every call shares the one array: calls that overlap on the GPU race, so
 * issue them on one stream.  Each call writes every partial it reads, so
 * nothing needs clearing between calls.  Errors: LB_ERR_INVALID (f or out
 * NULL, n_cells outside [1, LB_STATIC_MAX_CELLS]), LB_ERR_CUDA. */
#define LB_STATIC_PARTIALS 1024
#define LB_STATIC_MAX_CELLS (1LL << 27)
lb_status lb_fluid_totals_static(const double* f, const int32_t* owner, int64_t n_cells, double* out,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBSQ_H */
