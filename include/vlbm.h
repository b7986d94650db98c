/*
 * vlbm.h -- C ABI of the GB300 (sm_103a) blended D2Q5 vectorial lattice
 * Boltzmann library for the 2D compressible Euler equations.
 *
 * Method: Wissocq, Liu & Abgrall, "A positive- and bound-preserving vectorial
 * lattice Boltzmann method in two dimensions", arXiv 2411.15001.
 *   - problem: Sec. 1, eq. (hyperbolic_PDE) with the ideal-gas Euler fluxes and
 *     the admissible set G of eq. (convex_G);
 *   - D2Q5 velocity set and Maxwellians: Sec. 2, Example "Five-wave (D2Q5) model";
 *   - blended collide-and-stream update: Sec. 3.2, eq. (blending_u1) and
 *     eq. (blending_u) (u_5 eliminated, 20 values per cell);
 *   - per-face blending theta = min(1, theta_rho, theta_p): Sec. 3.2-3.4
 *     (PP / LMP / RLMP density bounds, GQL internal-energy bound);
 *   - kinetic speed a^n = 4 lambda^n and Delta t^n = dx / a^n: Sec. 4 preamble.
 *
 * Conventions shared by every call
 *   - Return value: VLBM_OK (0) or a negative VLBM_E_* code; vlbm_strerror()
 *     names it. Nothing is thrown, nothing aborts.
 *   - Device memory: the library never allocates device memory. The caller
 *     passes one device workspace (vlbm_workspace_bytes) that must stay alive
 *     and unmoved until vlbm_destroy; every other device pointer is borrowed for
 *     the duration of the call's stream work only.
 *   - Host memory: the opaque vlbm_state is allocated by vlbm_init and freed by
 *     vlbm_destroy.
 *   - Streams: every call enqueues its work on the stream given to vlbm_init
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream) and
 *     returns without waiting, except the calls documented as synchronising.
 *   - Field layout: a "plane" is nx*ny values, cell (i, j) at j*nx + i (x
 *     fastest), in the state's precision (double for VLBM_FP64, float for
 *     VLBM_FP32). Momentum arguments hold two planes back to back: m1 then m2.
 *   - Sticky errors: a state that leaves G (rho <= 0 or E - |m|^2/(2 rho) <= 0)
 *     or becomes non-finite is recorded on the device and reported by the next
 *     synchronising call (vlbm_sync, vlbm_monitors, vlbm_time).
 */
#ifndef VLBM_H
#define VLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported symbols (the library is built with hidden default visibility). */
#if defined(__GNUC__)
#define VLBM_API __attribute__((visibility("default")))
#else
#define VLBM_API
#endif

/* ------------------------------------------------------------------ codes */
#define VLBM_OK 0
#define VLBM_E_INVAL (-1)        /* bad argument or inadmissible initial state */
#define VLBM_E_CUDA (-2)         /* a CUDA runtime call failed (no device, launch error) */
#define VLBM_E_POSITIVITY (-3)   /* a cell left the admissible set G */
#define VLBM_E_NONFINITE (-4)    /* a cell became NaN or infinite */
#define VLBM_E_TIMEOUT (-5)      /* a bounded device wait gave up */
#define VLBM_E_UNSUPPORTED (-6)  /* valid request this build does not implement */
#define VLBM_E_NOMEM (-7)        /* workspace too small or misaligned */

/* Density bound used by the convex limiter (Sec. 3.3). FIRST_ORDER forces
 * theta = 0 (the first-order scheme of eq. 1st-order_kinetic), NONE forces
 * theta = 1 (the second-order scheme of eq. 2nd-order_kinetic). PP, LMP and
 * RLMP all add the internal-energy bound theta_p of Sec. 3.4. */
#define VLBM_LIM_FIRST_ORDER 0
#define VLBM_LIM_NONE 1
#define VLBM_LIM_PP 2
#define VLBM_LIM_LMP 3
#define VLBM_LIM_RLMP 4

/* Boundary rule per side (Sec. 4: periodic; zero gradient of all
 * distributions; reflective (symmetry) wall; a prescribed state whose
 * distributions are its Maxwellians, as the double Mach reflection of Sec. 4.7
 * and the jets of Sec. 4.8 use at their boundaries). A periodic side must face
 * a periodic side. VLBM_BC_DIRICHLET needs a vlbm_boundary (vlbm_opts) for its
 * field. */
#define VLBM_BC_PERIODIC 0
#define VLBM_BC_TRANSMISSIVE 1
#define VLBM_BC_REFLECTIVE 2
#define VLBM_BC_DIRICHLET 3

/* Arithmetic of the state. FP32: populations, collision and density bounds
 * in float; the internal-energy bound theta_p is settled per face by a float
 * screen (theta_p >= min(1, theta_rho) proved with rigorous error bounds), else
 * by a tight float interval (a certified lower bound), else by a solve whose
 * cancelling quantities are formed in double -- theta never exceeds the exact
 * theta_p; conservation sums in double. FP64: every formula in double. */
#define VLBM_FP64 0
#define VLBM_FP32 1

/* Kernel choice. VLBM_KERNEL_AUTO takes the row-marching kernel for FP32 grids of at
 * least 2^19 cells and FP64 grids of at least 2^22 cells, the one-thread-per-cell
 * kernel otherwise (where it is faster). */
#define VLBM_KERNEL_AUTO 0
#define VLBM_KERNEL_SIMPLE 1    /* one thread per cell, radius-2 gather from L2 */
#define VLBM_KERNEL_FUSED 2     /* row-marching TMA kernel, one pass per step */

typedef struct vlbm_state vlbm_state;

/* Uniform Cartesian grid: nx * ny cells of side dx. bc = {west, east, south, north}. */
typedef struct {
    int32_t nx, ny;
    double dx;
    int32_t bc[4];
} vlbm_grid;

/* Field of the prescribed (VLBM_BC_DIRICHLET) parts of the boundary. At the
 * start time t of a step, the ghost cell with centre (x, y) holds the conserved
 * state `in` if nx[k] x + ny[k] y >= c0[k] + c1[k] t for every k < nplanes, and
 * `out` otherwise (each side of the test evaluated in double, products first);
 * its populations are the Maxwellians M_1..M_4 of that state at the step's
 * kinetic speed. Both states must lie in G. The kinetic speed lambda^n also
 * covers both states (so that Bouchut's condition holds on the boundary faces). */
typedef struct {
    double in[4], out[4];            /* conserved (rho, m1, m2, E) */
    int32_t nplanes;                 /* 0, 1 or 2 half-planes (0: `in` everywhere) */
    double nx[2], ny[2], c0[2], c1[2];
} vlbm_field;

/* Boundary beyond vlbm_grid.bc: sides that switch type once along their length
 * (a partial wall, Sec. 4.7) and the prescribed field. The ghost cells of side s
 * (0 west, 1 east, 2 south, 3 north) whose index along the side -- column i for
 * south/north, row j for west/east, ghost indices included -- is below split[s]
 * follow grid.bc[s], the others bc_hi[s]. split[s] = 0: a uniform side (bc_hi[s]
 * must equal bc[s]); otherwise 2 <= split[s] <= n - 2 along that side, so that
 * the two cells at either end, and the corner ghosts beyond them, share a type.
 * A periodic side does not switch. Cell (i, j) has centre
 * (x0 + (i + 1/2) dx, y0 + (j + 1/2) dx). */
typedef struct {
    int32_t bc_hi[4];
    int32_t split[4];
    double x0, y0;
    vlbm_field field;
} vlbm_boundary;

/* Optional settings; pass NULL for the defaults. */
typedef struct {
    double alpha;     /* D2Q5 rest weight M_5 = alpha u; 1/2 <= alpha < 1 (Prop. convex
                         preservation); default 0.5 as in Sec. 4 */
    double eps;       /* epsilon subtracted in the PP and pressure bounds; default 1e-16 */
    int32_t kernel;   /* VLBM_KERNEL_*; default AUTO */
    int32_t sponge;   /* sponge layer of Sec. 4.2: theta = 0 on every face of the cells within
                         `sponge` cells of a zero-gradient side (the paper uses 5 with its
                         zero-gradient boundaries); 0 = none; at most n / 2 along every axis
                         that has a zero-gradient side. A side counts as zero-gradient when
                         it is so along its whole length */
    const vlbm_boundary *boundary;   /* NULL: uniform sides, no prescribed state. Copied by
                                        vlbm_init; the batch applies it to every grid */
} vlbm_opts;

/* Host copy of the device-side step state and monitors. */
typedef struct {
    int64_t n;                 /* time steps taken since vlbm_set_conserved / vlbm_load */
    double t;                  /* simulated time */
    double a;                  /* kinetic speed the next step will use */
    double dt;                 /* time step the next step will use */
    double lambda;             /* max_cells |v| + sqrt(gamma p / rho) of the current state */
    int64_t bad_cells;         /* cells outside G in the last step's output */
    int64_t nonfinite_cells;   /* non-finite cells in the last step's output */
    int64_t first_bad_step;    /* first step whose output left G (or went non-finite); -1 if none */
    double min_rho;            /* min density of the current state */
    double sum[4];             /* FP64 sums of rho, m1, m2, E over the cells of the current state */
    int64_t theta_p_fp64_faces; /* faces of the last step whose theta_p needed the FP64 solve: FP32
                                   state, where neither the float screen nor a tight float interval
                                   settled it; FP64 state, every face */
    int32_t done;              /* 1 once vlbm_step_to has reached its final time */
    int32_t status;            /* sticky VLBM_OK / VLBM_E_* of the device */
    double min_internal_energy; /* min of E - |m|^2 / (2 rho) over the cells of the current state,
                                   evaluated in the state's precision (membership of G is decided
                                   by an exact test: bad_cells) */
} vlbm_monitor_t;

/* Bytes of device workspace for a grid and precision (two padded 20-plane
 * states with a two-cell ghost frame, plus the device control block).
 * Returns 0 for an invalid grid or precision. */
VLBM_API size_t vlbm_workspace_bytes(const vlbm_grid *grid, int32_t precision);

/* Create a solver on `d_workspace` (caller-owned device memory, >= the size
 * above, 256-byte aligned) for the Euler system with heat capacity ratio
 * gamma > 1. lambda > 0 holds the kinetic speed fixed at a = 2 lambda/(1-alpha)
 * (= 4 lambda at alpha = 1/2; Sec. 4.1 runs a = 10.7); lambda <= 0 updates it
 * every step from the current state (Sec. 4 preamble). `stream` is a
 * cudaStream_t. Allocates only the host object; enqueues nothing.
 * Errors: VLBM_E_INVAL (any argument out of range), VLBM_E_NOMEM (workspace too
 * small or misaligned), VLBM_E_CUDA (no usable device). */
VLBM_API int vlbm_init(const vlbm_grid *grid, double gamma, double lambda, int32_t limiter,
              int32_t precision, const vlbm_opts *opts, void *d_workspace,
              size_t workspace_bytes, void *stream, vlbm_state **out);

/* Load initial conserved fields u_0 = (rho, m1, m2, E) from device planes and
 * initialise the populations at equilibrium, u_k^0 = M_k(u_0) (Sec. 4
 * preamble), with a^0 from u_0. Resets n and t to 0 and clears sticky errors.
 * Synchronises the stream: returns VLBM_E_INVAL if a cell of u_0 is outside G
 * or not finite. */
VLBM_API int vlbm_set_conserved(vlbm_state *s, const void *d_rho, const void *d_mom, const void *d_E);

/* Advance `nsteps` >= 0 time steps (one fused collide + limit + stream pass
 * each, eq. blending_u1 / blending_u). Asynchronous. */
VLBM_API int vlbm_step(vlbm_state *s, int64_t nsteps);

/* Advance until t = t_end (the last step is shortened so that t lands on t_end,
 * with a = dx / Delta t, still above the Bouchut speed of eq. Bouchut_D2Q5) or
 * until max_steps steps, whichever comes first. Synchronises the stream once per
 * chunk of steps to learn whether t_end was reached. */
VLBM_API int vlbm_step_to(vlbm_state *s, double t_end, int64_t max_steps);

/* Copy the conserved fields of the current state into caller-owned device
 * planes (any pointer may be NULL to skip it). Asynchronous. */
VLBM_API int vlbm_moments(const vlbm_state *s, void *d_rho, void *d_mom, void *d_E);

/* Wait for the stream, then fill *out (host) with the step state and monitors.
 * Returns the sticky device status (VLBM_OK, VLBM_E_POSITIVITY, ...). */
VLBM_API int vlbm_monitors(vlbm_state *s, vlbm_monitor_t *out);

/* Monitors without waiting for the stream (for a loop that checks every step's
 * monitors while the next step runs): vlbm_monitors_async enqueues on the state's
 * stream a copy of the raw step-state record, as the work enqueued so far leaves
 * it, into h_dst (caller-owned host memory of vlbm_monitors_raw_bytes() bytes;
 * pinned, or the copy is not asynchronous). Once that copy has completed (the
 * caller records an event after it, or synchronises), vlbm_monitors_decode turns
 * the record into *out and returns its sticky status, as vlbm_monitors does. */
VLBM_API size_t vlbm_monitors_raw_bytes(void);
VLBM_API int vlbm_monitors_async(vlbm_state *s, void *h_dst);
VLBM_API int vlbm_monitors_decode(const void *h_src, vlbm_monitor_t *out);

/* Wait for the stream and return the sticky device status. */
VLBM_API int vlbm_sync(vlbm_state *s);

/* Wait for the stream; *t and *n (either may be NULL) get the simulated time
 * and step count. Returns the sticky device status. */
VLBM_API int vlbm_time(vlbm_state *s, double *t, int64_t *n);

/* Bytes of a checkpoint: a 64-byte header (n, t, a, dt, done) followed by the
 * 20 planes of the current state (u, then u_1..u_4, 4 planes each). */
VLBM_API size_t vlbm_checkpoint_bytes(const vlbm_state *s);

/* Write the current state into caller-owned device memory d_dst (>=
 * vlbm_checkpoint_bytes). Asynchronous. */
VLBM_API int vlbm_save(const vlbm_state *s, void *d_dst);

/* Restore a checkpoint written by vlbm_save for the same grid and precision;
 * stepping on from it reproduces the uninterrupted run bit for bit.
 * Asynchronous. */
VLBM_API int vlbm_load(vlbm_state *s, const void *d_src);

/* Kernel timing. While enabled, every step records a CUDA event pair around its
 * collide + limit + stream kernel (not the pass that writes prescribed ghosts
 * before it, on grids with a prescribed part) on the state's
 * stream. vlbm_profile_read waits for the stream and returns the summed kernel
 * time in milliseconds and the number of timed launches since the last enable. */
VLBM_API int vlbm_profile(vlbm_state *s, int32_t enable);
VLBM_API int vlbm_profile_read(vlbm_state *s, double *kernel_ms, int64_t *launches);

/* ---------------------------------------------------------------- batches */

/* Many independent grids of uneven sizes (one gamma, limiter and precision)
 * advanced together: every time step is one launch of the row-marching kernel
 * over the work items (grid, strip of 120 columns, band of rows) of all grids,
 * persistent CTAs taking items from a shared counter; steps are replayed from
 * a CUDA graph of 64 launches. Each grid keeps its own dynamic kinetic speed
 * a^n = 4 lambda^n (Sec. 4 preamble), time, monitors and ghost frame. */
typedef struct vlbm_batch vlbm_batch;

#define VLBM_ORDER_LPT 0     /* work items of the grids with most cells first */
#define VLBM_ORDER_INDEX 1   /* work items in grid index order */
#define VLBM_ORDER_GUIDED 2  /* as LPT, rows cut into bands of decreasing height: each
                                band's height is the rows x strips left in all grids over
                                the CTA count, within [4, chunk] (guided self-scheduling;
                                a single vlbm_state always uses it, with chunk 128) */

/* Work decomposition: rows per work item (the largest band under GUIDED; 4 to 1024),
 * CTAs per SM (1 to 4), item order; items and CTAs of the resulting launch (outputs). A new
 * batch starts with GUIDED bands of at most 128 rows and as many CTAs per SM as
 * the kernel's occupancy allows. */
typedef struct {
    int32_t chunk, ctas_per_sm, order;
    int32_t items, ctas;
} vlbm_batch_tuning;

/* Bytes of device workspace for n grids (0 if an argument is invalid). */
VLBM_API size_t vlbm_batch_workspace_bytes(int32_t n, const vlbm_grid *grids, int32_t precision);

/* Create a batch over caller-owned d_workspace (>= the size above, 256-byte
 * aligned). Enqueues nothing. Errors as vlbm_init. */
VLBM_API int vlbm_batch_init(int32_t n, const vlbm_grid *grids, double gamma, int32_t limiter,
                             int32_t precision, const vlbm_opts *opts, void *d_workspace,
                             size_t workspace_bytes, void *stream, vlbm_batch **out);

/* Initial conserved planes of grid i (layout as vlbm_set_conserved), populations
 * at equilibrium (Sec. 4 preamble). Synchronises; VLBM_E_INVAL for a state
 * outside G. Every grid must be set before the first vlbm_batch_step. */
VLBM_API int vlbm_batch_set_conserved(vlbm_batch *b, int32_t i, const void *d_rho, const void *d_mom,
                                      const void *d_E);

/* Advance every grid by nsteps time steps. Asynchronous. */
VLBM_API int vlbm_batch_step(vlbm_batch *b, int64_t nsteps);

/* Conserved planes of grid i into caller-owned device memory (NULL skips). */
VLBM_API int vlbm_batch_moments(const vlbm_batch *b, int32_t i, void *d_rho, void *d_mom, void *d_E);

/* Checkpoint of grid i, format of vlbm_save. Asynchronous. */
VLBM_API int vlbm_batch_save(const vlbm_batch *b, int32_t i, void *d_dst);

/* Monitors of grid i (synchronises); returns the grid's sticky status. */
VLBM_API int vlbm_batch_monitors(vlbm_batch *b, int32_t i, vlbm_monitor_t *out);

/* Current work decomposition, or set one explicitly. */
VLBM_API int vlbm_batch_get_tuning(const vlbm_batch *b, vlbm_batch_tuning *t);
VLBM_API int vlbm_batch_set_tuning(vlbm_batch *b, const vlbm_batch_tuning *t);

/* Autotuner: times every decomposition (chunk 32/128/512/1024 rows x 1..max CTAs per SM
 * x the three item orders) over trial_steps steps each with CUDA events, keeps the
 * fastest and returns it with its time per step. The decomposition does not
 * change any cell's arithmetic, so the trial steps are real steps: the grids
 * advance by (1 + trial_steps) x candidates steps. Synchronises. */
VLBM_API int vlbm_batch_autotune(vlbm_batch *b, int32_t trial_steps, vlbm_batch_tuning *best,
                                 double *best_ms_per_step);

VLBM_API void vlbm_batch_destroy(vlbm_batch *b);

/* Last error message of a batch call: that batch's, or with b = NULL the calling
 * thread's last failed call that had no batch object (vlbm_batch_init). */
VLBM_API const char *vlbm_batch_last_error(const vlbm_batch *b);

/* ---------------------------------------------------------------- adjoint */

/* Gradient of a loss L(u^N) of the final conserved fields with respect to the
 * initial conserved fields u_0 (rho, m1, m2, E), through N steps of the blended
 * scheme (Sec. 3.2, eq. blending_u1 / blending_u, theta of Sec. 3.2-3.4) and the
 * equilibrium initialisation u_k^0 = M_k(u_0) (Sec. 4 preamble). The transpose
 * of each step is differentiated piecewise: theta on the branch the forward step
 * took (1, the density bound, the internal-energy bound, or the clamp at 0). The
 * kinetic speeds a^n: with a fixed speed (a state made with lambda > 0) they are
 * constants; with the dynamic speed a^n = 2 lambda^n / (1 - alpha) of Sec. 4,
 * lambda^n = max over the cells of |v| + sqrt(gamma p / rho), they are held as
 * the forward run produced them (VLBM_ADJOINT_HOLD_A, the default) or
 * differentiated too (VLBM_ADJOINT_DIFF_A: the subgradient of the max taken at
 * the first cell, in index order j nx + i, where it is reached). Covered: the
 * first-order, unlimited and PP schemes, on periodic grids and on grids with a
 * boundary (zero gradient, mirror walls, prescribed states, sides that switch
 * type, the sponge layer): there the transpose of the ghost fill carries each
 * ghost's cotangent to the cell it was filled from, and a prescribed ghost holds
 * no state. LMP / RLMP (Sec. 3.3.1-3.3.2: theta^rho through the local bounds, each
 * the min / max of five candidates, the cotangent going to the first that attains
 * it) are covered on every grid (with a boundary the bounds of the first ghost
 * layer reach the second, and both layers are folded back), a^n held or
 * differentiated (d theta / da then includes the bound's dependence on a through
 * rho* of the face where it was taken). With VLBM_ADJOINT_DIFF_A and a prescribed
 * boundary state, the prescribed ghosts' populations M_k(u_field; a^n) add their
 * dL/da^n (the field itself is piecewise constant in time: no time derivative),
 * and a step whose lambda^n is set by the prescribed states hands nothing to the
 * cells.
 *
 * Memory: checkpoints of the state every ckpt_every steps, two segment buffers of
 * ckpt_every + 1 states for the recomputation (the recomputation of one segment
 * runs on a second stream of the library's, overlapping the adjoint steps of the
 * segment after it), and two cotangent buffers, all in caller-owned d_scratch of
 * vlbm_adjoint_scratch_bytes (256-byte aligned). Cost: one forward run, one
 * recomputation of every step but the last of each segment, and one adjoint kernel
 * per step. */
VLBM_API size_t vlbm_adjoint_scratch_bytes(const vlbm_state *s, int64_t nsteps, int32_t ckpt_every);

/* How vlbm_adjoint treats a dynamic kinetic speed (see above); the mode applies
 * to later calls. With a fixed speed both modes give the same gradient. Cost of
 * VLBM_ADJOINT_DIFF_A: two reads of the conserved planes per step (the argmax of
 * lambda) and one reduction. VLBM_E_INVAL for an unknown mode. */
#define VLBM_ADJOINT_HOLD_A 0
#define VLBM_ADJOINT_DIFF_A 1
VLBM_API int vlbm_adjoint_set_mode(vlbm_state *s, int32_t mode);

/* Forward run with checkpoints: from the state vlbm_set_conserved left (n = 0),
 * advance nsteps steps with the state's kernel, storing a checkpoint before
 * every ckpt_every-th step into d_scratch. Afterwards the state holds u^N as
 * after vlbm_step. Asynchronous. */
VLBM_API int vlbm_rollout(vlbm_state *s, int64_t nsteps, int32_t ckpt_every, void *d_scratch,
                          size_t scratch_bytes);

/* Reverse sweep. d_dLduN: dL/du^N as 4 planes (rho, m1, m2, E) back to back;
 * d_dLdu0 (output): dL/du_0 in the same layout; both in the state's precision.
 * With d_u0 (4 planes, same layout) the call first runs vlbm_set_conserved(u_0)
 * and vlbm_rollout itself; with d_u0 = NULL it uses the checkpoints of the
 * preceding vlbm_rollout, which must have had the same nsteps, ckpt_every and
 * d_scratch (VLBM_E_INVAL otherwise). The state is left at u^N. Asynchronous
 * (the d_u0 form synchronises once, in vlbm_set_conserved). */
VLBM_API int vlbm_adjoint(vlbm_state *s, const void *d_u0, int64_t nsteps, int32_t ckpt_every,
                          const void *d_dLduN, void *d_dLdu0, void *d_scratch, size_t scratch_bytes);

/* ---------------------------------------------------------- no workspace */

/* Result of vlbm_step_noalloc, in host memory. */
typedef struct {
    double lambda;               /* max |v| + sqrt(gamma p / rho) of the new state */
    double a_next;               /* 2 lambda / (1 - alpha): the kinetic speed for a following step */
    double min_rho;              /* min density of the new state */
    double sum[4];               /* FP64 sums of rho, m1, m2, E of the new state */
    int64_t bad_cells;           /* cells of the new state outside G */
    int64_t nonfinite_cells;
    int64_t theta_p_fp64_faces;
} vlbm_step_result;

/* One time step that allocates nothing and needs no workspace. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory at all -- a plugin whose host application's memory pool already owns
 * the device, a real-time loop that may not pay the implicit device-wide
 * synchronisation of cudaMalloc, a sandbox without access to the allocator.
 * Such a caller holds its state and passes it in and out.
 *   d_in, d_out: caller-owned device buffers of 20 compact planes each (u, then
 *     u_1..u_4, 4 planes each, plane q at q * nx * ny, cell (i, j) at j * nx + i)
 *     in the given precision; they must not overlap. Boundaries are applied on
 *     the fly from grid->bc; opts->boundary must be NULL (a prescribed field
 *     needs the time, which this call does not keep: VLBM_E_UNSUPPORTED).
 *   a: the kinetic speed of this step (Delta t = dx / a); result->a_next is the
 *     dynamic speed for the next one.
 * The only scratch, one reduction record per CTA of 32 x 8 cells, lives in a
 * fixed array of about 0.5 MB inside the library that every GPU loading it keeps
 * until the process exits; grids of more than 8192 such CTAs (about two million
 * cells, e.g. 2048 x 1024) are rejected with VLBM_E_INVAL. Every call shares that
 * array and overwrites it, so calls whose work overlaps on the GPU (other
 * streams, other host threads on the same device) race; serialise them. The
 * first call on a device looks up the array's device address once, with that
 * device current; make that first call before any stream capture. Runs on
 * `stream` (a cudaStream_t) on the current device and synchronises it to fill
 * *result. Returns VLBM_OK, VLBM_E_POSITIVITY / VLBM_E_NONFINITE for a new state
 * outside G, VLBM_E_INVAL or VLBM_E_CUDA. Calls no cudaMalloc or cudaFree. */
VLBM_API int vlbm_step_noalloc(const vlbm_grid *grid, double gamma, double a, int32_t limiter,
                               int32_t precision, const vlbm_opts *opts, const void *d_in, void *d_out,
                               vlbm_step_result *result, void *stream);

/* Free the host object. Enqueues nothing and does not touch the workspace. */
VLBM_API void vlbm_destroy(vlbm_state *s);

/* Static, NUL-terminated name of a return code. */
VLBM_API const char *vlbm_strerror(int code);

/* Copy the last error message recorded for `s` (or for the thread if s is NULL)
 * into buf (n bytes, always NUL-terminated). Returns the message length. */
VLBM_API int vlbm_last_error_detail(const vlbm_state *s, char *buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif
