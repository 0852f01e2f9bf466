/*
 * lbm.h -- C ABI of the GB300 (sm_103a) coupled lattice Boltzmann /
 * rigid-body swimmer step.
 *
 * One call of lbm_step advances a D3Q19 fluid with moving rigid bodies by
 * the coupled step of Pickl et al., "All good things come in threes" (arXiv
 * 1108.0786), Algorithm 2: map the bodies onto the lattice (Sec. 2.3), fused
 * stream + velocity-corrected bounce-back + reconstruction of uncovered
 * cells + LBGK collision (Eq. 1-4 and the moving-wall rule of Sec. 2.3),
 * momentum-exchange force and torque per body (Eq. hydroF), drive
 * (Eq. FB1-FB3), damped springs (Eq. osci_i, osci_j) and the rigid-body
 * time step (Algorithm 1, Eq. totalFSwimmer).  Everything runs on the
 * device; the host never synchronises inside lbm_step.
 *
 * Units: lattice units, dx = dt = 1, rest density 1.  Cell (x, y, z) has its
 * centre at the integer point (x, y, z) and linear index
 * c = (z * ny + y) * nx + x.  A non-periodic axis has halfway no-slip walls
 * half a cell outside its first and last cell centres.
 *
 * Population order (19 directions e_a):
 *    0:( 0, 0, 0)
 *    1:(+1, 0, 0)  2:(-1, 0, 0)  3:( 0,+1, 0)  4:( 0,-1, 0)  5:( 0, 0,+1)  6:( 0, 0,-1)
 *    7:(+1,+1, 0)  8:(-1,-1, 0)  9:(+1,-1, 0) 10:(-1,+1, 0)
 *   11:(+1, 0,+1) 12:(-1, 0,-1) 13:(+1, 0,-1) 14:(-1, 0,+1)
 *   15:( 0,+1,+1) 16:( 0,-1,-1) 17:( 0,+1,-1) 18:( 0,-1,+1)
 *
 * Body state (13 doubles): position[3], unit quaternion (w, x, y, z)[4],
 * velocity[3], angular velocity[3], all in the world frame.  The body-frame
 * x axis is the capsule axis and the drive direction.
 *
 * Ownership: a handle owns every byte of device memory it uses.  It
 * allocates lazily, at the first call that needs the device (lbm_step,
 * lbm_set_fields, lbm_get_*), through the allocator installed with
 * lbm_set_allocator or, if none, cudaMalloc.  Host pointers passed in are
 * read during the call only; host output buffers are owned by the caller.
 *
 * Errors: every int-returning call returns LBM_OK (0) or a negative
 * LBM_E_* code and stores a message for lbm_last_error.  Errors found on
 * the device (a bounded wait that ran out, a full link or cell list,
 * overlapping bodies, a body crossing a wall, a non-finite body state or
 * link term, a body faster than LBM_MAX_BODY_STEP per step) are latched in
 * a device status word and returned by the next synchronising call
 * (lbm_sync, lbm_get_*, lbm_save), in that order of precedence when several
 * are latched; the state after such an error is unspecified.
 * Nothing is thrown across the ABI.  A handle is not thread safe.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK            0
#define LBM_E_ARG        -1   /* bad argument */
#define LBM_E_OOM        -2   /* device or host allocation failed */
#define LBM_E_OVERLAP    -3   /* a cell lies inside two bodies */
#define LBM_E_OUTSIDE    -4   /* a body crosses a wall of the domain */
#define LBM_E_NAN        -5   /* non-finite body state */
#define LBM_E_LINKS      -6   /* link list capacity exceeded */
#define LBM_E_TIMEOUT    -7   /* a bounded device wait expired */
#define LBM_E_CUDA       -8   /* CUDA runtime error */
#define LBM_E_STATE      -9   /* call not allowed in the current state */
#define LBM_E_UNSTABLE  -10   /* a body moved more than LBM_MAX_BODY_STEP in one step */

/* bc bitmask: periodic axes; the other axes get halfway no-slip walls */
#define LBM_BC_PERIODIC_X 1
#define LBM_BC_PERIODIC_Y 2
#define LBM_BC_PERIODIC_Z 4

#define LBM_SHAPE_SPHERE  0
#define LBM_SHAPE_CAPSULE 1   /* cylinder of `length` along body x + two caps */

/* population storage; the collision runs in FP64 for LBM_PREC_F64 and in
 * FP32 otherwise.  Populations are stored as deviations f_a - w_a from the
 * rest equilibrium. */
#define LBM_PREC_F64  0
#define LBM_PREC_F32  1
#define LBM_PREC_F16  2   /* deviations scaled by 2^LBM_F16_SCALE_EXP */
#define LBM_F16_SCALE_EXP 10
#define LBM_PREC_BF16 3

#define LBM_OPT_NO_FLUID  1   /* bodies only: no mapping, no hydrodynamic force */
#define LBM_OPT_AVERAGE_FORCE 2   /* rigid-body step with the mean hydrodynamic load of steps n and n-1
                                     (not in the paper: a stabiliser of the explicit coupling for
                                     light bodies; lbm_get_forces still reports step n's load) */
#define LBM_OPT_OVERLAP   4       /* overlapped steps (the same bits): the bulk kernel of step n leaves
                                     the tiles near a body to a near-cell kernel after the remap and
                                     runs beside the force and remap of the neighbouring steps */

#define LBM_FIELD_RHO   0     /* density, cells */
#define LBM_FIELD_U     1     /* velocity, [3][cells] */
#define LBM_FIELD_FLAGS 2     /* uint8 per cell: 0 fluid, 1 + body id if solid */
#define LBM_FIELD_POP   3     /* post-collision populations, [19][cells] */

#define LBM_DTYPE_F64 0
#define LBM_DTYPE_F32 1
#define LBM_DTYPE_U8  2

#define LBM_MAX_BODIES     254
#define LBM_MAX_BODY_STEP  0.5   /* largest displacement of a body per step */

/* kernel slots reported by lbm_time_kernels */
#define LBM_KERNEL_REMAP          0   /* body geometry and remap candidates, then map bodies to the lattice */
#define LBM_KERNEL_STREAM_COLLIDE 1   /* bulk pull + LBGK over all cells */
#define LBM_KERNEL_BOUNDARY       2   /* refill / bounce-back cells near bodies and walls */
#define LBM_KERNEL_LINKS          3   /* per-body link lists, then the step's drive and spring loads */
#define LBM_KERNEL_FORCE          4   /* momentum exchange; with fluid it also runs the rigid-body step */
#define LBM_KERNEL_INTEGRATE      5   /* drive, springs, rigid-body step when there is no fluid */
#define LBM_NUM_KERNELS           6

typedef struct lbm_s lbm_t;

/* Device allocator hook: return `bytes` of device memory (256-byte aligned)
 * usable on the handle's stream, or NULL; free_fn releases it. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, void *ctx);

/* Create a lattice of nx*ny*nz cells with LBGK relaxation time tau > 1/2
 * (Eq. 1-2; viscosity (tau - 1/2)/3), FP32 storage, no body force.
 * Allocates no device memory.  Errors: LBM_E_ARG, LBM_E_OOM (host). */
int lbm_create(int nx, int ny, int nz, double tau, int bc, lbm_t **out);

/* As lbm_create with a storage precision (LBM_PREC_*), a body-force density
 * g[3] acting on the fluid through Guo's forcing term and on each body as
 * g times its volume (g may be NULL for zero), and LBM_OPT_* options. */
int lbm_create_ex(int nx, int ny, int nz, double tau, int bc, int precision,
                  const double g[3], int options, lbm_t **out);

/* Release the handle and all device memory it owns (synchronises). */
int lbm_destroy(lbm_t *h);

/* Install the device allocator; only before the first device allocation. */
int lbm_set_allocator(lbm_t *h, lbm_alloc_fn alloc_fn, lbm_free_fn free_fn, void *ctx);

/* CUDA stream (a cudaStream_t) on which all work is enqueued; NULL is the
 * legacy default stream.  The device is the current device at the first
 * device allocation. */
int lbm_set_stream(lbm_t *h, void *stream);

/* Add a rigid body (Sec. 2.2, 3.1-3.2): sphere of `radius` (length 0) or
 * capsule of cylinder `length` and cap `radius` along the body x axis, of
 * `mass`, centre pos[3] and orientation orient[4] (unit quaternion w,x,y,z,
 * normalised here; NULL for identity).  Inertia is that of a uniform solid.
 * Only before the first step.  Returns the body id (>= 0).  With the fluid on,
 * every periodic extent must be at least the side of the body's remap cube,
 * 2 (ceil(radius + length/2) + 4) + 1 cells (the per-step scans around a body
 * wrap on periodic axes and would otherwise visit cells twice); a shorter
 * periodic axis is LBM_E_ARG. */
int lbm_add_body(lbm_t *h, int shape, double radius, double length, double mass,
                 const double pos[3], const double orient[4]);

/* Volume and body-frame principal moments of inertia of a uniform solid
 * sphere or capsule (Sec. 2.2, 3.1-3.2; the values lbm_add_body uses), and
 * their derivatives: out[4] = V, I1, I2, I3 (I1 about the capsule axis);
 * d_mass[4] and d_length[4] (either may be NULL) the derivatives of the same
 * four with respect to the mass and to the cylinder length (zero for a
 * sphere).  For the chain rule of gradients with respect to mass and
 * capsule length.  Host only, no handle; LBM_E_ARG for bad dimensions. */
int lbm_body_properties(int shape, double radius, double length, double mass, double out[4],
                        double d_mass[4], double d_length[4]);

/* Damped harmonic spring between bodies i and j (Eq. spring_i, damp_i,
 * osci_i, osci_j): F_i = -k (|d| - rest) d/|d| - damping (V_i - V_j),
 * d = X_i - X_j, F_j = -F_i; rest is the centre-to-centre rest length.
 * Only before the first step.  Returns the spring id. */
int lbm_add_spring(lbm_t *h, int i, int j, double k, double rest, double damping);

/* Add a drive term on `body` (Eq. FB1-FB3): the force
 * amp * sin(2 pi freq t - phase) along the body x axis (or the axis set by
 * lbm_set_drive_axis) for t >= phase / (2 pi freq), zero before; t is the
 * step index.  Terms on one body add up, so the middle body's -(F2 + F3) is
 * two terms.  Only before the first step.  Returns the term id. */
int lbm_set_drive(lbm_t *h, int body, double amp, double freq, double phase);

/* Direction of drive term `term` as a body-frame vector (used as given, not
 * normalised; default 1, 0, 0): the world-frame force is amp sin(...) R(q) a.
 * The paper's perpendicular capsules (Sec. 5.1) are driven along the
 * swimming direction, across their own axis.  Only before the first step. */
int lbm_set_drive_axis(lbm_t *h, int term, const double axis[3]);

/* Switch drive term `term` off for t >= t_off (the paper's protocol stops
 * the drives at t1 and t2, Sec. 5.1). */
int lbm_set_drive_window(lbm_t *h, int term, double t_off);

/* Overwrite the current state (13 doubles) of a body.  After the first
 * step the position may change by less than LBM_MAX_BODY_STEP per axis
 * (else LBM_E_STATE).  Synchronous. */
int lbm_set_body_state(lbm_t *h, int body, const double state[13]);

/* Overwrite the post-collision populations of the last completed step
 * (before the first step: the populations the first step streams from).
 * Only LBM_FIELD_POP with LBM_DTYPE_F64 host data [19][cells].  Synchronous. */
int lbm_set_fields(lbm_t *h, int what, const void *host_in, int dtype);

/* Enqueue n coupled steps on the handle's stream (CUDA graphs; no host
 * synchronisation).  Returns launch errors only. */
int lbm_step(lbm_t *h, int n);

/* Wait for all enqueued work and return any latched device error. */
int lbm_sync(lbm_t *h);

/* Time average of the velocity field (Sec. 6, Fig. 13: the flow around one
 * and three swimmers averaged over five swimming cycles).
 * lbm_average_begin starts the average, or restarts it from zero: from then
 * on every step adds the velocity of the populations it wrote,
 * u = (sum_a e_a f~_a - g/2) / rho (0 in obstacle cells, the LBM_FIELD_U
 * value), to an FP64 sum of 3 doubles per cell on the device (allocated at
 * the first call through the handle's allocator; one extra kernel a step).
 * lbm_average_stop stops adding and keeps the sum.  lbm_average_get
 * synchronises and writes the mean, FP64 [3][cells] in the field layout, to
 * host memory `out` and the number of steps averaged to *steps (optional);
 * LBM_E_STATE if no average was begun.  The moments are FP64 for FP64
 * storage and FP32 for 32/16-bit storage. */
int lbm_average_begin(lbm_t *h);
int lbm_average_stop(lbm_t *h);
int lbm_average_get(lbm_t *h, double *out, long long *steps);

/* Number of completed (enqueued) steps. */
long long lbm_steps_done(lbm_t *h);

/* Body states after the last step, out[bodies][13] (synchronises). */
int lbm_get_bodies(lbm_t *h, double *out);

/* The same read without waiting: enqueues on the handle's stream a copy of
 * the body states after the steps enqueued so far into host memory
 * out[bodies][13] (page-locked memory lets the copy run asynchronously;
 * `out` must stay valid until the read completes), and the status word
 * beside it, and returns a ticket (>= 0; -1 before the first step, when the
 * initial states are copied at once).  lbm_wait_ticket(h, ticket) waits for
 * that read and returns the first error the status word held then (as
 * lbm_sync; the word is copied beside the next step, so it may also hold
 * that step's errors).  The copy runs on a stream of its own after the
 * steps enqueued before it and beside the step enqueued next; the step
 * after that, which overwrites the buffer read, waits for it.  So a caller
 * can keep the GPU stepping while reading each step's states one step late.
 * LBM_E_ARG for a ticket never issued. */
int lbm_get_bodies_async(lbm_t *h, double *out, long long *ticket);
int lbm_wait_ticket(lbm_t *h, long long ticket);

/* Hydrodynamic force and torque of the last step, out[bodies][6]: F[3],
 * T[3]; the torque is about the body centre (synchronises). */
int lbm_get_forces(lbm_t *h, double *out);

/* Copy a field of the last completed step to host memory (synchronises):
 * RHO = sum f~, U = (sum e f~ - g/2)/rho, solid cells report rho = 1 and
 * u = 0; FLAGS as LBM_FIELD_FLAGS; POP = f~ as [19][cells].  dtype
 * LBM_DTYPE_F64 or LBM_DTYPE_F32 for RHO, U, POP; LBM_DTYPE_U8 for FLAGS. */
int lbm_get_fields(lbm_t *h, int what, void *out, int dtype);

/* As lbm_get_fields into caller-owned device memory (enqueued, no sync). */
int lbm_get_fields_device(lbm_t *h, int what, void *dev_out, int dtype);

/* Record every step's body states in a device ring buffer of `capacity`
 * steps (0 disables).  Only before the first step. */
int lbm_enable_history(lbm_t *h, int capacity);

/* Copy the recorded states, oldest first, out[n][bodies][13] with
 * n = min(steps done, capacity, max_steps); *n_out = n (synchronises). */
int lbm_get_history(lbm_t *h, double *out, int max_steps, int *n_out);

/* Checkpoint / restore the full state (populations, both flag epochs, both
 * body states, forces, step counter) to / from a file (synchronises).  The
 * handle given to lbm_load must have the same lattice, bodies and
 * precision. */
int lbm_save(lbm_t *h, const char *path);
int lbm_load(lbm_t *h, const char *path);

/* Diagnostic timing: run n steps launching each kernel separately with CUDA
 * events around it on the handle's stream, and write the average duration
 * in milliseconds of each kernel slot (LBM_KERNEL_*) to ms_out[slots]; a
 * slot that does not run is reported as 0.  The state advances by n steps. */
int lbm_time_kernels(lbm_t *h, int n, double *ms_out, int slots);

/* Launch shape of the bulk stream-collide kernel: cells_per_thread
 * consecutive x cells per thread (1, 2, 4; 8 for 16-bit storage; nx must be
 * a multiple) and min_blocks_per_sm, a register cap that lets that many
 * 256-thread blocks share an SM (0 for each: the defaults).  16-bit storage
 * with an even cells_per_thread keeps the populations packed two to a
 * 32-bit word between load and store.
 * cells_per_thread = -1 selects the row-staged kernel: persistent blocks
 * (min_blocks_per_sm of them per SM: 1 or 2 for FP64 / FP32 storage, 2, 3
 * or 4 for 16-bit storage) copy each x-row's 19 source rows
 * and flags into shared memory with bulk asynchronous copies (TMA) and
 * collide from there; it needs nx a multiple of 16 and the stages within the
 * shared memory of an SM (FP32: nx <= 1472 for 2 blocks per SM).  Only the
 * compiled combinations are accepted (LBM_E_ARG otherwise).  Only before the
 * first step.  Results do not depend on the shape. */
int lbm_tune(lbm_t *h, int cells_per_thread, int min_blocks_per_sm);

/* Autotuner: time every compiled shape of the bulk kernel on this handle's
 * lattice (`trials` launches each, on the populations of the next step,
 * which that step rewrites) and keep the fastest for the following steps.
 * Reports the choice through the optional outputs (synchronises). */
int lbm_autotune(lbm_t *h, int trials, int *cells_per_thread, int *min_blocks_per_sm);

/* Checks of the failure paths (failure detection; the paper has no
 * counterpart) and of the reverse sweep's schedule.  The first two make the
 * device latch an error from the host side, without faulting or hanging
 * anything:
 *   LBM_DEBUG_EXPIRE_WAITS, value 1: the first wait of every block of the
 *     row-staged bulk kernel (lbm_tune with cells_per_thread = -1) is on a
 *     barrier that no copy completes, bounded by about 2^16 SM cycles.  It
 *     runs out as a real stall would: the block latches LBM_E_TIMEOUT, waits
 *     (bounded) for its copies in flight and returns.  Value 0 (default):
 *     the normal bound of about 1 s.
 *   LBM_DEBUG_CELL_LIST_CAP, value k >= 1: the list of cells the boundary
 *     kernel handles (fluid cells next to a body or uncovered) holds at most
 *     k entries instead of its sized capacity; a step that finds more
 *     latches LBM_E_LINKS, stores none past the capacity and handles only
 *     those listed.  Value 0: the sized capacity.
 *   LBM_DEBUG_ADJOINT_SERIAL, value 1: lbm_adjoint_backward recomputes and
 *     reverses its segments in turn with one set of recomputation slots.
 *     Value 0 (default): where the device has room for a second set, the
 *     recomputation of segment k - 1 runs on its own stream beside the
 *     reverse steps of segment k.  Both give the same bits.  Any time; it
 *     holds for the following calls of lbm_adjoint_backward.
 *   LBM_DEBUG_NO_PDL, value 1 (default): every kernel of a step graph is
 *     launched only after the kernel before it has completed.  Value 0: the
 *     force kernel and the next step's remap in serial steps are launched
 *     with programmatic dependent launch, so that their blocks become
 *     resident while the bulk kernel and the force kernel drain, and wait,
 *     before touching memory, until those have completed (on the capsule
 *     swarm within 0.5 us a step of the default either way, so it stays
 *     off).  Both give the same bits.  Any time (it synchronises and
 *     rebuilds the step graphs).
 * The steps after such an error are not valid.  The first two only before
 * the first step (LBM_E_STATE after it); LBM_E_ARG for an unknown knob or
 * value. */
#define LBM_DEBUG_EXPIRE_WAITS  1
#define LBM_DEBUG_CELL_LIST_CAP 2
#define LBM_DEBUG_ADJOINT_SERIAL 3
#define LBM_DEBUG_NO_PDL 4
int lbm_debug_set(lbm_t *h, int knob, long long value);

/* ---- reverse mode ---------------------------------------------------------
 *
 * Gradients of J = sum_b seed[b] . state_b(n0 + n), a linear function of the
 * body states (the layout of lbm_get_bodies) after n steps, with respect to
 * the parameters of the swimmers: drive terms (Eq. FB1-FB3), springs
 * (Eq. osci_i, osci_j), body mass, inertia and volume (Algorithm 1), and the
 * state the run starts from.  The obstacle maps of the recorded run are held
 * fixed: the cell-centre test of Sec. 2.3 is piecewise constant in the body
 * positions, so J is the smooth function of the parameters that the recorded
 * map sequence defines.  A gradient with respect to a capsule length is the
 * chain rule through mass, inertia and volume (the cell map held fixed).
 * The paper has no reverse mode; it is the differentiation path of the
 * swimmer design study.
 *
 * lbm_adjoint_record advances the handle by n steps from its current step n0
 * (like lbm_step, through the same kernels) and keeps: the body state and the
 * hydrodynamic force and torque of every step (13 + 6 doubles per body and
 * step), and every `segment` steps a checkpoint of the populations and the
 * flags entering the step (19 populations + 2 bytes per cell).  Device memory
 * comes from the handle's allocator and is held until the next recording or
 * lbm_destroy.  FP64 and FP32 storage only (LBM_E_ARG otherwise); at least
 * one body.  Synchronises.
 *
 * lbm_adjoint_backward runs the reverse sweep over the recording: segment by
 * segment, last first, it recomputes the segment's populations and flags from
 * its checkpoint (segment + 1 population and flag slots), then applies the
 * transposed step in reverse order.  The adjoint populations are kept in the
 * storage precision (FP64, or FP32 for FP32 storage); body adjoints and
 * parameter gradients in FP64.  It does not change the handle's state.
 * Outputs (host, caller-owned, each may be NULL):
 *   grad_state   [nb][13]  dJ/d state n0
 *   grad_prev    [nb][13]  dJ/d state n0 - 1 (the moving-wall velocities of
 *                          the first stream); when n0 = 0 these two are one
 *                          state: the sum is reported in grad_state and
 *                          grad_prev is zero
 *   grad_drive   [nd][2]   dJ/d amp, dJ/d phase of each drive term (the
 *                          switch-on step phase / (2 pi freq) held fixed)
 *   grad_spring  [ns][3]   dJ/d k, dJ/d rest, dJ/d damping
 *   grad_body    [nb][5]   dJ/d mass, dJ/d I_1, I_2, I_3 (body-frame
 *                          principal moments), dJ/d volume (body force g)
 *   grad_pop     [19][C]   dJ/d populations entering step n0 (FP64)
 * Allocates and frees its own working buffers (through the allocator hook);
 * LBM_E_STATE without a recording.  Synchronises. */
int lbm_adjoint_record(lbm_t *h, int n, int segment);
int lbm_adjoint_backward(lbm_t *h, const double *seed, double *grad_state, double *grad_prev,
                         double *grad_drive, double *grad_spring, double *grad_body, double *grad_pop);

/* ---- ensembles ------------------------------------------------------------
 *
 * Many independent lattices (ensemble members, e.g. one swimmer design per
 * member on its own periodic box, of uneven sizes and step counts) stepped
 * together.  One CUDA graph advances every member of a set by CHUNK (16)
 * steps; members whose step budget runs out drop out of the set (a graph
 * per set is built on first use and kept).
 *   LBM_ENSEMBLE_BATCHED (default): each step is one launch of each per-step
 *     kernel (body preparation, remap, boundary cells, links, loads, bulk
 *     stream-collide, force) over the members of a storage precision: the
 *     members' grids are flattened into one grid, and each block finds its
 *     member's record in a device table.  A set of two or more members is
 *     split into two halves of about equal cell counts, each its own chain
 *     of launches; the second starts one remap behind the first, and the
 *     latency-bound kernels run at a higher stream priority than the bulk
 *     kernels, so one half's prep, remap and force run beside the other
 *     half's bulk kernel.  ~16 launches a step for the whole set, however
 *     many members.  Every member needs the fluid; the bulk kernel runs in
 *     one shape for all members (lbm_ensemble_autotune), not in the
 *     members' own.
 *   LBM_ENSEMBLE_BRANCHES: the members' own step kernels as parallel graph
 *     branches (6 launches a step per member).
 * Both give the bits of the members stepped alone.  There is no dependency
 * between members: no kernel waits on another.  The paper runs one
 * simulation per design study point; the ensemble is the throughput path
 * for a set of such points.
 *
 * lbm_ensemble_create: members (n handles, not owned) must share one stream
 * (lbm_set_stream); each keeps its own buffers, bodies and status word.
 * lbm_ensemble_step advances member i by steps[i] steps (host array of n
 * counts, >= 0): whole chunks through the ensemble graphs, the rest through
 * the member's own step graphs.  Asynchronous, like lbm_step.
 * lbm_ensemble_sync synchronises and returns the first member error.
 * lbm_ensemble_destroy releases the graphs and tables, not the members.
 * lbm_ensemble_set_mode selects the mode (LBM_E_ARG for another value).
 * lbm_ensemble_autotune times every batched bulk shape that fits all members
 * of a precision (`trials` launches each, on the populations of the members'
 * next step, which that step rewrites; the members must be at steps of the
 * same parity, else LBM_E_STATE) and keeps the fastest; *cells_per_thread
 * (optional) reports the choice for the first member's precision. */
typedef struct lbm_ensemble_s lbm_ensemble_t;
#define LBM_ENSEMBLE_BATCHED  0
#define LBM_ENSEMBLE_BRANCHES 1
int lbm_ensemble_create(lbm_t *const *members, int n, lbm_ensemble_t **out);
int lbm_ensemble_set_mode(lbm_ensemble_t *e, int mode);
int lbm_ensemble_autotune(lbm_ensemble_t *e, int trials, int *cells_per_thread);
int lbm_ensemble_step(lbm_ensemble_t *e, const int *steps);
int lbm_ensemble_sync(lbm_ensemble_t *e);
int lbm_ensemble_destroy(lbm_ensemble_t *e);
const char *lbm_ensemble_last_error(lbm_ensemble_t *e);

/* Kernel launches one step makes (for launch accounting): with bodies and
 * fluid, remap, bulk stream-collide, boundary cells (one more launch with
 * walls), link lists, drive and spring loads, and the momentum exchange
 * with the rigid-body step.  A body preparation kernel (geometry records of
 * states the rigid-body step did not make) runs once before the first step
 * after the host wrote a body state, and in every overlapped step. */
int lbm_kernels_per_step(lbm_t *h);

/* Algorithmic bytes per cell the stream-collide kernel moves:
 * 2 * 19 * sizeof(population) + 1 flag byte. */
int lbm_bytes_per_cell(lbm_t *h);

/* ---- momentum exchange without device allocation -------------------------
 *
 * The paper has no counterpart to this call; it serves callers that cannot
 * call cudaMalloc: programs that keep every byte of device memory in a pool
 * of their own under a fixed budget, or loops that must not pay the implicit
 * device-wide synchronisation of cudaMalloc / cudaFree.  Such a caller owns
 * all inputs and outputs and asks the library for the hydrodynamic force and
 * torque of each body (the values lbm_get_forces reports for a step).
 *
 * Inputs (device pointers, read only):
 *   pop     post-collision populations f~ as FP64, [19][nx*ny*nz] in the
 *           population order above (as LBM_FIELD_POP / LBM_DTYPE_F64);
 *   flags   uint8 per cell: 0 fluid, 1 + body id for a cell of that body
 *           (as LBM_FIELD_FLAGS);
 *   bodies  [nb][13] FP64 body states (as lbm_get_bodies) of the same step.
 * Output (device pointer): out[nb][6] = F[3], T[3] per body, torque about
 * the body centre.  half_width bounds the links of every body: all its
 * solid cells lie within half_width - 1 cells of floor(X) on each axis.
 * The scan covers the cube of side 2 half_width + 1 around floor(X), cut to
 * one period on each periodic axis shorter than that side, so every cell and
 * link is counted once.
 * Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default).
 *
 * Scratch: per-block partial sums live in one file-scope device array of
 * LBM_STATIC_SCRATCH_RECORDS records of 48 bytes (3 MiB), which every GPU
 * that loads the library holds until the process exits.  The first call on
 * a device looks up that array's device address, with the device current,
 * and looks it up again when the device's context has changed (after
 * cudaDeviceReset); make that first call, and the first call after a reset,
 * before any stream capture.  Every call shares the
 * array and leaves its last contents there; calls that overlap on the GPU
 * (for example on two streams) race and give wrong results.
 *
 * Errors: LBM_E_ARG for a null pointer, nb outside [1, LBM_MAX_BODIES], bad
 * sizes or bc, half_width outside [1, LBM_STATIC_SCRATCH_MAX_HALF_WIDTH], or
 * nb * ceil(sx sy sz / 256) > LBM_STATIC_SCRATCH_RECORDS, with s the scan's
 * extent per axis (2 half_width + 1, or the axis length where it is cut);
 * LBM_E_CUDA for a CUDA error.  Nothing is allocated in any case. */
#define LBM_STATIC_SCRATCH_RECORDS        65536
#define LBM_STATIC_SCRATCH_MAX_HALF_WIDTH 64
int lbm_momentum_exchange_static(const double *pop, const unsigned char *flags, const double *bodies,
                                 int nb, int nx, int ny, int nz, int bc, int half_width, double *out,
                                 void *stream);

/* Message of the last error on this handle (never NULL). */
const char *lbm_last_error(lbm_t *h);

#ifdef __cplusplus
}
#endif
#endif
