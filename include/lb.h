/*
 * lb.h -- C ABI of the GB300 (sm_103a) immersed-boundary / lattice-Boltzmann solver for a
 * tensorial viscoelastic fluid (Floyd, Vaikuntanathan, Dinner, arXiv 2209.14889).
 *
 * One time step (Fig. 2; every field is updated from the state at t):
 *   node forces f_a = -grad U (App. A, Eq. Const, plus a constant pull and/or the harmonic trap
 *   of Eq. Utrap with its pulling protocol),
 *   spreading f_IB = sum_a f_a K(R_a - r) (App. A), polymer force f^p = div sigma^p (Sec. II B),
 *   Ericksen force f^E = div sigma^E (Sec. II C 1), D2Q9 BGK collide + stream with the Guo
 *   body force (Sec. II A, Eq. LB, Eq. BGK), predictor-corrector updates of sigma^p
 *   (Eq. StiffCons with C~(P) of App. B) and of P (Eq. BE), and overdamped advection of the
 *   nodes by the interpolated velocity (App. A).
 *
 * Units: lattice units (dx = dt = 1, c_s^2 = 1/3).  Periodic in x and y unless walls are set
 * (App. C; see "Walls" below).
 * Fields are [y][x] planes, x fastest, FP32 on the device.
 *
 * Ownership: the handle owns every device buffer it allocates (cudaMalloc in lb_create and
 * lb_set_body) and frees them in lb_destroy.  Pointers passed in are only read or written
 * during the call.  Every launch and copy goes on the stream given to lb_create; calls that
 * return data to the host synchronise that stream.  A handle is not thread-safe.
 *
 * Errors: every int-returning call returns LB_OK (0) or a negative LB_E* code;
 * lb_last_error() describes the last failure.  Numerical trouble detected on the device
 * (non-finite readouts, a ring leaving its work box, node displacement >= 1 cell per step)
 * is reported by lb_sync().
 */
#ifndef VLB_LB_H
#define VLB_LB_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define LB_OK 0
#define LB_EINVAL (-1)      /* bad argument or parameter                                */
#define LB_ENOMEM (-2)      /* device allocation failed                                 */
#define LB_ECUDA (-3)       /* CUDA runtime error (message in lb_last_error)             */
#define LB_ENONFINITE (-4)  /* a readout (mass, momentum, force, node) became NaN/Inf    */
#define LB_EUNSTABLE (-5)   /* parameters outside the explicit stability bounds          */
#define LB_EBODY (-6)       /* a ring left its work box or moved >= 1 cell in one step   */
#define LB_ESTATE (-7)      /* call out of order (e.g. lb_step before lb_init_fields)    */
#define LB_ETIMEOUT (-8)    /* a bounded wait inside a kernel gave up (results invalid)  */

/* Storage precision of the lattice state (arithmetic is FP32 in both). */
#define LB_FP32 0           /* 14 FP32 planes: 112 B per cell and step                          */
#define LB_FP16_BF16 1      /* populations FP16 as (h_n - w_n rho0) 2^12 / w_n, sigma^p BF16,
                               P - P_ref FP16; stochastic rounding on store: 56 B per cell-step  */

/* Field identifiers for lb_readout / lb_write_field. */
#define LB_FIELD_DRHO 0     /* rho - rho0 of the current state (readout only)           */
#define LB_FIELD_UX 1       /* u_x = (sum c h + F/2)_x / rho (readout only)              */
#define LB_FIELD_UY 2
#define LB_FIELD_SXX 3      /* polymer stress sigma^p_xx                                 */
#define LB_FIELD_SYY 4
#define LB_FIELD_SXY 5
#define LB_FIELD_PX 6       /* polarisation P_x                                          */
#define LB_FIELD_PY 7
#define LB_FIELD_POP0 8     /* LB_FIELD_POP0 + n: h_n - w_n rho0 (stored form), n = 0..8 */
#define LB_FIELD_NODES 17   /* node positions, FP64 [n_total][2], wrapped into the box   */

typedef struct lb_params {
    int32_t nx, ny;                 /* lattice size, each >= 8                                */
    double tau, rho0;               /* BGK relaxation time (Eq. BGK), rest density            */
    double K1111, K1122, K2222, K1212; /* K^x of Eq. Kmatrix (prefactor absorbed, App. B)    */
    double eta_p;                   /* polymer viscosity (Eq. StiffCons); if <= 0, taken as   */
    double lambda_steps;            /*   lambda_steps * C~11(k = 0) (relaxation time in steps)*/
    double Dp;                      /* stress diffusion D_p (Eq. MaxDiff)                      */
    double alpha, beta, xi, Gamma, kappa; /* Beris-Edwards (Eq. BE, Eq. Ffunctional)          */
    double P_cap;                   /* cap on |P| when solving Eq. Pk (0.99)                  */
    double director_angle;          /* initial director angle theta_d (radians)               */
    int32_t ericksen;               /* 1: include f^E in the body force                        */
    int32_t precision;              /* LB_FP32 or LB_FP16_BF16                                 */
    int32_t readout_every;          /* record readouts when t % readout_every == 0 (10)       */
    int32_t max_samples;            /* capacity of the readout ring buffer (rows)             */
    int32_t diffusion_substeps;     /* 0: D_p inside the Heun step (needs 8 D_p <= 2); s > 0:  */
                                    /*   the Heun step without diffusion, then s Heun sub-steps */
                                    /*   of D_p / s on sigma (needs 8 D_p / s <= 2; FP32 only)  */
    int32_t model;                  /* LB_MODEL_TENSORIAL (0) or LB_MODEL_SCALAR (1), below    */
    int32_t walls_y;                /* 1: walls in y (App. C), below; 0: periodic in y         */
    int32_t walls_x;                /* 1: walls in x, the same; both: the closed box of App. C  */
} lb_params;

/*
 * Walls (App. C; walls_y = 1 and/or walls_x = 1): no-slip walls half-way between nodes at
 * y = -1/2 and y = ny - 1/2 (x = -1/2, nx - 1/2), half-way bounce-back of the populations, zero
 * gradient of sigma^p and P across them (a cell beyond a wall mirrors the cell inside), zero
 * velocity and zero Ericksen stress at the wall (their mirrored values are negated, so the
 * Ericksen force moves no momentum into the walls); an axis without walls stays periodic.
 * Needs at least 4 cells across each walled axis (else LB_EINVAL at lb_create), the FP32 state,
 * no diffusion sub-steps and the one-cell tile kernel; ring nodes must stay
 * 5 cells from the walls at lb_set_body (else LB_EINVAL) and 4 cells while stepping (else
 * LB_EBODY at lb_sync); the learned stepper takes periodic lattices only.
 */

/*
 * Viscoelastic model.  LB_MODEL_TENSORIAL: Eq. StiffCons with C~(P) (App. B) and the
 * Beris-Edwards P field (Eq. BE).  LB_MODEL_SCALAR: the scalar diffusive Johnson-Segalman model
 * of Eq. MaxDiff (Sec. II B), D sigma / Dt = C Psi - (C / eta_p) sigma + D_p lap sigma with one
 * modulus C, and no orientation field: the state moves 12 planes (96 B per cell and step in
 * FP32).  It needs K2222 = K1111, K1122 = 0, K1212 = K1111 / 2 (C = K1111: the isotropic K^x, for
 * which the tensorial C~ is C times the identity at every P, so both models then compute the same
 * fluid and stress), ericksen = 0, the FP32 state and the one-cell tile kernel (lb_set_kernel
 * AUTO or TILE); P stays at its initial field and is not writable.  Else LB_EINVAL.
 */
#define LB_MODEL_TENSORIAL 0
#define LB_MODEL_SCALAR 1

typedef struct lb_ring {
    int32_t n_nodes;                /* 3 <= n_nodes <= 1024                                    */
    int32_t pad_;
    double k_spring, eps_angle;     /* Eq. Const: spring and angle stiffness                   */
    double l_eq;                    /* spring rest length                                      */
    double pull_force, pull_angle;  /* constant total pull on the ring, split over its nodes  */
    /* Harmonic trap of Eq. Utrap, k(t)/2 |R_ext(t) - R_com|^2, off when trap_k = 0.  Protocol
     * (App. C: sigmoid transitions of trap_width steps): with s(t; c) = 1 / (1 + exp(-8 (t - c) /
     * trap_width)), k(t) = trap_k s(t; trap_width / 2) (1 - s(t; trap_t_eq + trap_pull +
     * trap_width / 2)); the trap starts at the initial centre of mass R0 and moves to
     * R0 + (trap_dx, trap_dy) with a speed proportional to s(t; trap_t_eq) - s(t; trap_t_eq +
     * trap_pull) (t in steps).  Its force k (R_ext - R_com) / N acts on every node. */
    double trap_k, trap_dx, trap_dy, trap_t_eq, trap_pull, trap_width;
} lb_ring;

typedef struct lb_handle lb_handle;

/*
 * Create a solver.  Validates the parameters (stability: 0.5 < tau, 8 D_p <= 2 for the Heun
 * step of the diffusion term (8 D_p / s <= 2 with s diffusion sub-steps), Gamma*|alpha| linear
 * rate <= 2, else LB_EUNSTABLE), allocates
 * the double-buffered state (2 x 14 FP32 planes of nx*ny) and builds the C~(P) table on the
 * host (FP64, Eq. Pk inverted numerically, App. B).  stream: a cudaStream_t (NULL = default).
 */
int lb_create(const lb_params* p, void* stream, lb_handle** out);

/*
 * Initial state: h_n = w_n rho0 (fluid at rest), sigma^p = 0,
 * P = P_eq (cos theta_d, sin theta_d) + noise with P_eq = sqrt(-alpha/beta) (Sec. III B)
 * (0 if alpha >= 0).  noise: host FP64 [2][ny][nx] added to P, or NULL.
 * Resets the step counter to 0 and clears the readout series; rings already set keep their
 * positions, and their forces and work boxes are recomputed for the restart.
 */
int lb_init_fields(lb_handle* h, const double* noise);

/*
 * Immersed rings (App. A).  xy: host FP64 positions [n_total][2], ring after ring, in lattice
 * coordinates (cell (i, j) sits at (i, j)); copied.  Replaces any previous rings and computes
 * the forces of the initial configuration.  Each ring, widened by 8 cells, must span at most
 * half the lattice in x and in y (else LB_EINVAL).
 */
int lb_set_body(lb_handle* h, int32_t n_rings, const lb_ring* rings, const double* xy);

/* Advance n time steps, asynchronously on the handle's stream (one kernel launch per step with
 * the default settings: see lb_set_node_tail and lb_launches_per_step). */
int lb_step(lb_handle* h, int64_t n);

/* Synchronise the stream and return LB_OK or the first device-side error (LB_ENONFINITE,
 * LB_EBODY) raised since the last lb_sync. */
int lb_sync(lb_handle* h);

/* Current step counter t (host copy). */
int64_t lb_time(const lb_handle* h);

/*
 * Copy one field of the current state to dst (FP32 [ny][nx], or FP64 [n_total][2] for
 * LB_FIELD_NODES).  bytes must equal the field size.  dst_is_device: 1 if dst is device
 * memory, 0 for host memory.  DRHO/UX/UY run the force + moment part of the step on the
 * current state.  Synchronises the stream.
 */
int lb_readout(lb_handle* h, int32_t field, void* dst, size_t bytes, int32_t dst_is_device);

/*
 * lb_readout without any device allocation (the paper has no counterpart: this serves callers,
 * not the method).  lb_readout creates its intermediate buffer for rho and u with cudaMalloc on
 * first use; callers whose device memory is owned by another allocator, or who must not
 * allocate after set-up, use this call instead.  It accepts LB_FIELD_DRHO, UX, UY, PX and PY
 * and returns the same values as lb_readout.  The intermediate planes live in one scratch
 * array compiled into the library: 3 x 2^20 FP32 (12 MiB), held on every GPU that loads the
 * library until the process exits.  Lattices above 2^20 cells return LB_EINVAL.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before capturing the stream into a graph; threads making their first calls on a
 * device at the same time may each look it up and store the same value, which is harmless.
 * The call itself allocates nothing on any call.  All calls share the array: calls whose
 * work overlaps on the GPU (several handles, streams or threads at once) race on it.
 * Synchronises the stream.
 */
int lb_readout_noalloc(lb_handle* h, int32_t field, void* dst, size_t bytes, int32_t dst_is_device);

/* Overwrite one stored field (SXX..PY, POP0..POP8) of the current state from FP32 [ny][nx]. */
int lb_write_field(lb_handle* h, int32_t field, const void* src, size_t bytes, int32_t src_is_device);

/*
 * Readout series, one row per recorded step, oldest first:
 *   [t, sum(rho - rho0), sum c h (x, y), sum F (x, y),
 *    then per ring: F_rest (x, y), centre of mass (x, y)]
 * F_rest = sum_a sum_r f^p(r) K(R_a - r), the polymer force density (div sigma^p, called the
 * restoring force in Sec. III A) interpolated to the nodes and summed over the ring.
 * Sums are FP64 over FP32 values in a fixed order.  Row length: 6 + 4 n_rings.
 * dst: host FP64 [max_rows][row length].  *rows_written gets the number of rows copied.
 */
int lb_series(lb_handle* h, double* dst, int32_t max_rows, int32_t* rows_written);
int32_t lb_series_row_len(const lb_handle* h);
/* The most recent n rows of the same series (oldest first), copying only those rows; host FP64
 * [n][row length]; *rows_written gets the number copied (fewer while fewer are recorded).
 * Synchronises the stream. */
int lb_series_latest(lb_handle* h, double* dst, int32_t n, int32_t* rows_written);
/* lb_series_latest without the synchronisation (the paper has no counterpart; this serves callers
 * that keep the GPU busy with the next steps while the rows come back): the copies of the newest
 * n rows, as of the steps enqueued so far, are enqueued on the handle's stream behind those steps,
 * and the call returns.  dst must stay valid until lb_series_wait returns (pinned host memory for
 * a copy that does not block the caller).  lb_series_wait blocks until the copies of the last
 * lb_series_latest_async are done (at once if none is pending).  LB_EINVAL / LB_ECUDA. */
int lb_series_latest_async(lb_handle* h, double* dst, int32_t n, int32_t* rows_written);
int lb_series_wait(lb_handle* h);

/*
 * Bulk transfer of the stored state (the paper has no counterpart; it exists so that a caller
 * can move a whole state between host and device in one copy).  The layout is the stored one:
 * N_PLANES planes of nx*ny values in the handle's storage form (LB_FP32: FP32; LB_FP16_BF16: the
 * 2-byte encodings above), x fastest: the 9 shifted populations h_n - w_n rho0 (scaled as above in
 * the 2-byte form), sigma^p (xx, yy, xy), P - P_ref (x, y); lb_state_bytes gives the size.
 * lb_read_state copies the current state into dst and synchronises the stream.  lb_write_state
 * replaces the current state with src (node positions, forces and work boxes are unchanged, as
 * with lb_write_field); the copy is enqueued on the handle's stream: host memory that is not
 * pinned is staged before the call returns, pinned host or device memory must stay unchanged
 * until the stream has passed the copy (lb_sync).  LB_EINVAL (null pointer or wrong size),
 * LB_ESTATE (before lb_init_fields).
 */
int64_t lb_state_bytes(const lb_handle* h);
int lb_read_state(lb_handle* h, void* dst, size_t bytes, int32_t dst_is_device);
int lb_write_state(lb_handle* h, const void* src, size_t bytes, int32_t src_is_device);

/*
 * lb_write_state in two halves, so that the upload of the next state overlaps the steps running
 * on the current one (the paper has no counterpart; this serves callers that feed a new state
 * every few steps).  lb_stage_state enqueues the copy of a whole stored state (layout and size as
 * for lb_write_state) into a staging buffer of the handle on a copy stream of its own and returns;
 * lb_commit_state makes the handle's stream wait for that upload and makes the staged state
 * current, in stream order with the steps before and after it: the handle takes the staging
 * buffer as its current state buffer and keeps its former current buffer for the next stage (no
 * copy), or, while the handle belongs to a batch (whose captured launches hold its buffers),
 * copies the staged state device to device into its current buffer.  The staging buffer (one state) and the copy stream are created on the
 * first lb_stage_state.  A second lb_stage_state before a commit replaces the staged state; a
 * stage after a commit waits on the GPU until that commit's copy has read the buffer.  src must
 * stay unchanged until the upload is done (pinned host memory overlaps; host memory that is not
 * pinned is staged before the call returns).  LB_EINVAL (null pointer or wrong size), LB_ESTATE
 * (before lb_init_fields; lb_commit_state with nothing staged), LB_ENOMEM / LB_ECUDA.
 */
int lb_stage_state(lb_handle* h, const void* src, size_t bytes, int32_t src_is_device);
int lb_commit_state(lb_handle* h);

/*
 * Checkpoint and resume (the paper has no counterpart: its runs are single jobs).  lb_save
 * finishes the handle's queued work and writes to the file `path` a raw snapshot of everything
 * a step carries over to the next: both state buffers and which one is current, the step
 * counter, the control block, the readout partials and series ring buffer and, with rings, the
 * ring records (parameters, trap protocol and its origin, work-box extents), both node position
 * buffers, the per-node cell, fraction and force, the work boxes, the tail's tickets and claims
 * and the node partial sums.  Native byte order; a file is read only by this library version.
 * lb_load reads such a file into a handle that was created with equal lb_params (every field)
 * and given the same rings by lb_set_body (the same number of rings and nodes per ring, and
 * equal spring constant, angle constant, rest length, pull and trap protocol per ring; the node
 * positions and the trap's origin then come from the file) and replaces its state, so
 * that stepping on continues exactly (bitwise) as the saved run would have.  Kernel choice and
 * node-tail setting stay the handle's own.  Neither call may run while the handle is stepped
 * by an lb_batch (sync the batch first).  Errors: LB_EINVAL (null argument, a file that cannot
 * be written or read, or that belongs to another version, parameter set, ring layout or ring
 * parameters; the handle is then unchanged), LB_ESTATE (lb_save before lb_init_fields), LB_ECUDA.  Synchronises
 * the stream.
 */
int lb_save(lb_handle* h, const char* path);
int lb_load(lb_handle* h, const char* path);

/* Restoring force of ring `ring` for the recorded rows: host FP64 [max_k][2]. */
int lb_restoring_force(lb_handle* h, int32_t ring, double* dst, int32_t max_k, int32_t* k_written);

/*
 * Kernel timing for throughput and roofline reports.  enable = 1 brackets every launch of
 * the fused lattice kernel with CUDA events on the handle's stream; lb_kernel_time returns
 * the summed device time (ms) and the launch count since timing was enabled.
 */
int lb_timing(lb_handle* h, int32_t enable);
int lb_kernel_time(lb_handle* h, double* fused_ms, int64_t* fused_launches, double* node_ms,
                   int64_t* node_launches);

/*
 * Lattice kernel used by lb_step.  All compute the same step with the same per-cell
 * arithmetic.  LB_KERNEL_TILE: 32 x 16 tiles with their halo recomputed, one cell per thread
 * (any lattice).  LB_KERNEL_PAIR: the same tiles with two neighbouring cells per thread on
 * paired FP32 instructions (any lattice).  LB_KERNEL_SWEEP: column strips swept row by row,
 * rows streamed by asynchronous bulk copies (needs nx % 4 == 0, nx >= 256, ny >= 16, FP32 state,
 * else LB_EINVAL).  LB_KERNEL_STRIP: one warp per strip of 32 columns (24 stored) swept along y,
 * stencil neighbours from registers and warp shuffles, no shared-memory staging; the node step
 * in the separate node kernel (periodic lattices with nx >= 64, ny >= 32, either precision,
 * either model, else LB_EINVAL); its fields and nodes equal the tile kernel's bit for bit.
 * LB_KERNEL_AUTO (default): the kernel measured fastest on GB300 for the lattice: the strip
 * kernel where it applies and the lattice fills at least four waves of its CTAs (4096^2 and
 * larger), else the one-cell tile kernel (with the node step in its tail).
 */
#define LB_KERNEL_AUTO 0
#define LB_KERNEL_TILE 1
#define LB_KERNEL_SWEEP 2
#define LB_KERNEL_PAIR 3
#define LB_KERNEL_STRIP 4
int lb_set_kernel(lb_handle* h, int32_t kernel);
/* The lattice kernel lb_step launches for this handle: LB_KERNEL_TILE, _PAIR, _SWEEP or _STRIP
 * (LB_KERNEL_AUTO resolved), or LB_EINVAL for a null handle. */
int32_t lb_lattice_kernel(const lb_handle* h);

/*
 * Where lb_step runs the node step (App. A: interpolation of u onto the nodes, their advection
 * and forces, the ring readouts) relative to the lattice step of the same time step.
 * enable = 1 (default): in the tail of the tile kernels (LB_KERNEL_TILE, _PAIR, _AUTO), one launch
 * per step: once the last tile whose region meets a ring's work box is done, that ring's node
 * blocks run in tiles that finish later while the other tiles still run.  enable = 0: a separate
 * node kernel after each lattice kernel.  Both compute the same values bit for bit;
 * LB_KERNEL_SWEEP and LB_KERNEL_STRIP always take the separate kernel.  LB_EINVAL for other
 * values.
 */
int lb_set_node_tail(lb_handle* h, int32_t enable);

/*
 * Number of kernels launched per lb_step(1) call: 1 (tile kernel with the node tail) or 2
 * (lattice + node kernel), plus, with s > 0 diffusion sub-steps, s sub-step launches and one
 * copy when s is odd.
 */
int32_t lb_launches_per_step(const lb_handle* h);

/* Bytes of lattice state per cell moved by one step (read + write, the algorithmic minimum). */
double lb_bytes_per_cell(const lb_handle* h);

/*
 * The host-built table behind C~(P) (App. B), for inspection: entry i (i = 0 .. n-1) holds
 * (a2, a4) = (r2 / q, r4 / q^2) at q = |P|^2 = P_cap^2 i / (n - 1), with r_n = I_n(k) / I_0(k) and
 * k solving I1(k) / I0(k) = |P| (Eq. Pk); a2(0) = 1/2, a4(0) = 1/24.  dst: host FP32 [n][2], or
 * NULL to query n.  Returns n, or a negative LB_E* code.  Needs no GPU.
 */
int32_t lb_stiffness_table(double P_cap, float* dst, int32_t max_entries);

const char* lb_last_error(const lb_handle* h);
void lb_destroy(lb_handle* h);

/*
 * Batched form.  Many independent lattices (each with its own size, parameters, rings and
 * diffusion sub-steps; Sec. II with the parameters of Tables I-IV varied per instance) advanced
 * together, a chunk of readout_every steps at a time, the chunk captured once as a CUDA graph and
 * replayed.  By default every step is three launches per tile-shape group: all instances'
 * lattice tiles, then their diffusion sub-steps, then their node blocks.  With
 * lb_batch_set_persistent(b, 1) one persistent cooperative kernel per group runs the whole chunk
 * instead, with a grid barrier between the phases.
 * Each instance computes exactly what lb_step computes for its handle (fields and nodes bitwise
 * equal; the readout sums of the lattice may differ in the last bits with the tile shape).
 *
 * lb_batch_create: handles[0..n-1] (n >= 1) must be distinct, have their fields and bodies set
 *   (lb_init_fields, lb_set_body), use the FP32 state and one model (all tensorial or all scalar), share one stream and be at the same
 *   buffer parity (an equal step count mod 2).  The batch keeps the pointers: the handles must
 *   outlive it and must not be stepped with lb_step while it exists.  Readouts (lb_readout,
 *   lb_series, ...) on the handles stay valid and are ordered after the batch's steps.
 *   Returns LB_ESTATE for a handle not ready, LB_EINVAL for a mismatch.
 * lb_batch_step: queue n >= 0 steps of every instance (asynchronous, on the handles' stream
 *   order).  lb_batch_sync: wait, then report LB_ETIMEOUT if a grid barrier gave up (the
 *   states are then undefined) or the first instance error of lb_sync.
 * lb_batch_set_shape: tile shape of instance inst (-1: all): 0 = 32x16, 1 = 32x8, 2 = 64x8,
 *   3 = 16x16 cells, 4 = the warp-strip kernel (LB_KERNEL_STRIP's step; periodic instances with
 *   nx >= 64 even and ny >= 32, phase launches only, else LB_EINVAL).  lb_batch_shape returns
 *   it (-1 for a bad index).
 * lb_batch_autotune: time `steps` steps with each shape that applies, first for the whole batch
 *   (one shape for all untuned sizes), then per distinct lattice size from the best of those,
 *   and keep the fastest; the states are saved and restored, so the simulation does not advance.  cache_path
 *   (or NULL) is a flat JSON object "<gpu name>|<nx>x<ny>": shape, read first and rewritten.
 * lb_batch_set_persistent: 1 = the persistent cooperative kernel, 0 = phase launches (default;
 *   measured faster on GB300: the tile phase keeps the tile kernel's three CTAs per SM and no
 *   CTA waits at a grid barrier).  Both compute the same values bit for bit.  LB_EINVAL for
 *   other values.
 * lb_batch_set_wait_limit: limit of one barrier wait of the persistent kernel in ms (default
 *   2000) and an arrival-count offset that is 0 in normal use; a positive offset makes every
 *   barrier wait run out, which exercises the LB_ETIMEOUT path.
 * lb_batch_grid: CTAs of the persistent launch of the first group, or the lattice-tile CTAs of
 *   one step over all groups with phase launches; lb_batch_uses_graph: 1 if chunks are replayed
 *   from a captured graph.
 */
typedef struct lb_batch lb_batch;
int lb_batch_create(lb_handle* const* handles, int32_t n, lb_batch** out);
int lb_batch_step(lb_batch* b, int64_t n);
int lb_batch_sync(lb_batch* b);
int lb_batch_set_shape(lb_batch* b, int32_t inst, int32_t shape);
int32_t lb_batch_shape(const lb_batch* b, int32_t inst);
int lb_batch_autotune(lb_batch* b, const char* cache_path, int32_t steps);
int lb_batch_set_persistent(lb_batch* b, int32_t enable);
int lb_batch_set_wait_limit(lb_batch* b, double wait_ms, int32_t extra_arrivals);
int32_t lb_batch_grid(const lb_batch* b);
int32_t lb_batch_uses_graph(const lb_batch* b);
const char* lb_batch_last_error(const lb_batch* b);
void lb_batch_destroy(lb_batch* b);

/*
 * The network of the learned stepper (no counterpart in the paper's method: a convolutional
 * surrogate trained on the method's own trajectories).  A 4-level U-Net on NHWC activations:
 * per level two 3x3 convolutions + LeakyReLU (slope 0.1) with 32, 64, 96, 128 channels at full,
 * 1/2, 1/4, 1/8 resolution, 2x2 average pooling down, nearest 2x upsampling + concatenation
 * with the skip up, and a final 3x3 convolution to 16 channels.  Input x: BF16 [B][H][W][16]
 * (H, W multiples of 8); output: FP32 [B][H][W][16].  BF16 weights and activations on the tensor
 * cores, FP32 accumulation, FP32 master weights and Adam.
 *
 * Parameters are one flat FP32 array, layer by layer in execution order (e0a, e0b, e1a, e1b,
 * e2a, e2b, bta, btb, d2a, d2b, d1a, d1b, d0a, d0b, head), each as w[9][Co][Ci] (tap
 * t = (dy + 1) * 3 + (dx + 1)) then b[Co].
 * lb_net_create: initialises He-normal weights from seed; all work on `stream`.
 * lb_net_forward: x is a device pointer; the output stays on the device (lb_net_output, owned by
 *   the network) and is copied to y (device FP32, or NULL); the activations are kept for
 *   lb_net_backward.
 * lb_net_backward: gradients of sum(g * output) for every parameter (overwritten, FP32;
 *   lb_net_get_grads), g a device FP32 [B][H][W][16].
 * lb_net_mse: loss = mean over pixels and the channels with mask16[c] != 0 of
 *   (mask (output - target))^2 (target device FP32 [B][H][W][16], mask16 host), its gradient kept
 *   for lb_net_train_step; *loss on the host (synchronises).
 * lb_net_adam: one Adam step with the last gradients.  lb_net_train_step: forward, mse,
 *   backward, Adam (lr, 0.9, 0.999, 1e-8).
 * lb_conv3x3 / lb_conv3x3_dgrad / lb_conv3x3_wgrad: the single-layer kernels (device pointers,
 *   BF16 activations and weights w[9][Co][Ci]), exposed to test them alone: forward with optional
 *   bias and LeakyReLU into BF16 y or FP32 yf; the data gradient gx[B][H][W][Ci] from
 *   gz[B][H][W][Co]; the weight and bias gradients gw[9][Co][Ci], gb[Co] (FP32) from x and gz.
 */
typedef struct lb_net lb_net;
int lb_net_create(int32_t batch, int32_t height, int32_t width, uint64_t seed, void* stream, lb_net** out);
int64_t lb_net_num_params(const lb_net* n);
int lb_net_set_params(lb_net* n, const float* host, int64_t count);
int lb_net_get_params(lb_net* n, float* host, int64_t count);
int lb_net_get_grads(lb_net* n, float* host, int64_t count);
int lb_net_forward(lb_net* n, const void* x, float* y);
const float* lb_net_output(const lb_net* n);
int lb_net_backward(lb_net* n, const float* grad_out);
int lb_net_mse(lb_net* n, const float* target, const float* mask16, double* loss);
const float* lb_net_loss_grad(const lb_net* n);
int lb_net_adam(lb_net* n, float lr, float beta1, float beta2, float eps);
int lb_net_train_step(lb_net* n, const void* x, const float* target, const float* mask16, float lr, double* loss);
int lb_net_shape(const lb_net* n, int32_t* batch, int32_t* height, int32_t* width);
/* Copy one stored BF16 activation of the last forward to the host (a test hook): which = 0 x,
 * 1 e0a, 2 cat0 [up(d1) | e0b], 3 pool(e0), 4 e1a, 5 cat1 [up(d2) | e1b], 6 pool(e1), 7 e2a,
 * 8 cat2 [up(bt) | e2b], 9 pool(e2), 10 bta, 11 btb, 12 d2a, 13 d2b, 14 d1a, 15 d1b, 16 d0a,
 * 17 d0b; bytes must equal the activation's size. */
int lb_net_activation(lb_net* n, int32_t which, void* host, int64_t bytes);
const char* lb_net_last_error(const lb_net* n);
void lb_net_destroy(lb_net* n);
/* Convolution kernel of the forward passes and data gradients (process-wide): 0 mma.sync
 * m16n8k16 tiles, 1 tcgen05.mma with tensor-memory accumulators (default).  lb_conv_status returns
 * LB_ETIMEOUT (once) if a tcgen05 convolution's bounded wait for its MMAs gave up. */
int lb_conv_kernel(int32_t kernel);
int lb_conv_status(void);
int lb_conv3x3(const void* x, int64_t ldx, int32_t xoff, const void* w, const float* bias, void* y, float* yf,
               int64_t ldy, int32_t yoff, int32_t B, int32_t H, int32_t W, int32_t Ci, int32_t Co, int32_t act,
               void* stream);
int lb_conv3x3_dgrad(const void* gz, const void* w, void* gx, int32_t B, int32_t H, int32_t W, int32_t Ci, int32_t Co,
                     void* stream);
int lb_conv3x3_wgrad(const void* x, const void* gz, float* gw, float* gb, int32_t B, int32_t H, int32_t W, int32_t Ci,
                     int32_t Co, void* stream);

/*
 * The learned stepper (no counterpart in the paper: a surrogate of 16 steps of its method, used
 * only where a residual check against the method passes).  Network channels: 0 ux, 1 uy,
 * 2 sigma_xx, 3 sigma_xy, 4 sigma_yy, 5 dP_x, 6 dP_y (dP = P - P_ref), 7 body indicator (sum of
 * the IB kernel weights phi phi of the ring nodes), 8..15 zero.  norm (host, 23 floats):
 * shift[8], scale[8] of the inputs x_c = (f_c - shift_c) scale_c, then oscale[7]: the network
 * outputs the change of channel c over 16 steps times oscale_c.
 *
 * lb_learned_pack: the handle's current fields as the network input x (device BF16 [ny][nx][16],
 *   or NULL) and the raw fields raw (device FP32 [ny][nx][8], or NULL); FP32 state only.
 * lb_learned_target: the training target (device FP32 [cells][16]) of a pair of raw fields 16
 *   steps apart.  lb_learned_normalize: the network input (BF16 [cells][16]) of raw fields.
 * lb_learned_create: a stepper for handle h (FP32 state, tensorial model, readout_every a multiple of 16) with a
 *   network of batch 1 and the lattice's size.  eps_momentum bounds the momentum-balance
 *   residual |sum u_net - sum u(t) - 16 F_pull| / (16 |F_pull|) (an accepted velocity is then
 *   shifted uniformly so that the balance holds exactly); eps_tendency bounds the relative
 *   mismatch between the network's per-step change of sigma and P and one plain step, in the
 *   scaled channel norm.
 * lb_learned_step: `calls` calls of 16 steps each.  Per call: one plain step, then either the
 *   network's state at t + 16 (both residuals within bounds; populations rebuilt as the
 *   equilibrium plus the regularised BGK non-equilibrium part, ring nodes advanced 15 steps
 *   with the mean velocity) or 15 more plain steps (*n_fallbacks counts these).  The restoring
 *   force series (lb_series) holds the rows of the plain steps at multiples of 16.
 * lb_learned_stats: out4 = (momentum residual, tendency residual of the last call, calls,
 *   accepted calls).
 */
typedef struct lb_learned lb_learned;
int lb_learned_pack(lb_handle* h, const float* norm, void* x, float* raw);
int lb_learned_target(const float* raw0, const float* raw1, const float* norm, float* target, int64_t cells,
                      void* stream);
int lb_learned_normalize(const float* raw, const float* norm, void* x, int64_t cells, void* stream);
int lb_learned_create(lb_handle* h, lb_net* net, const float* norm, double eps_momentum, double eps_tendency,
                      lb_learned** out);
int lb_learned_step(lb_learned* L, int64_t calls, int64_t* n_fallbacks);
int lb_learned_stats(const lb_learned* L, double* out4);
const char* lb_learned_last_error(const lb_learned* L);
void lb_learned_destroy(lb_learned* L);

#ifdef __cplusplus
}
#endif
#endif
