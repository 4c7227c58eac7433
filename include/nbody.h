/*
 * nbody.h -- C ABI of the GB300 direct particle-particle (PP) N-body library.
 *
 * The library computes the O(N^2) softened gravitational accelerations and
 * potentials of Khrapov, Khoperskov & Khoperskov (2018), "New features of
 * parallel implementation of N-body problems on GPU", and advances them with
 * the paper's KDK leapfrog or a fourth-order scheme, on one NVIDIA GB300
 * (sm_103a) GPU.  Every call is plain C: pointers, sizes and codes, no C++ or
 * framework types.
 *
 * Conventions for every function below
 *   - Return value: NBODY_OK (0) or a negative NBODY_E* code; nothing throws.
 *     nbody_strerror() turns a code into text; nbody_last_error() gives the
 *     detail of the most recent failure on the calling thread.
 *   - Arrays of 3-vectors are n x 3 row-major doubles (x, y, z of particle i
 *     at [3i], [3i+1], [3i+2]); scalar arrays are n doubles.
 *   - on_device = 0: the pointers are host memory; on_device = 1: they are
 *     device memory of the context's GPU.  The caller owns every pointer it
 *     passes and keeps it valid until the call returns (host pointers) or
 *     until the context's stream has reached the call (device pointers).
 *   - A context owns its resident device state and issues all its work on the
 *     CUDA stream given at creation (NULL = the legacy default stream).
 *     Calls that return host values synchronise that stream; the others are
 *     stream-ordered and return before the GPU finishes.
 *   - A context is not thread-safe; use one per thread or lock around it.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define NBODY_OK        0
#define NBODY_EINVAL   -1  /* bad argument: n < 1, eps < 0, eps == 0 with mode that needs eps > 0,
                              non-finite input, dt <= 0 or non-finite, unknown mode or scheme,
                              NULL pointer */
#define NBODY_ENOMEM   -2  /* device or host allocation failed */
#define NBODY_ECUDA    -3  /* a CUDA runtime call or kernel launch failed */
#define NBODY_ETIMEOUT -4  /* a bounded wait on the GPU expired */
#define NBODY_ESTATE   -5  /* the call needs state that was never set (nbody_set_state) */
#define NBODY_ENOSPC   -6  /* a batch has no free slot or not enough reserved memory */

/* ---- precision modes (Eq. 2 evaluated in...) ---------------------------- */
#define NBODY_FP64  0  /* binary64 throughout: the paper's double precision (DP) */
#define NBODY_MIXED 1  /* binary32 pair arithmetic on coordinates re-centred per j-tile from
                          binary64 storage; tile partial sums accumulated with compensation
                          and returned in binary64; state and update in binary64 */
#define NBODY_FP32  2  /* binary32 throughout, state included: the paper's single precision (SP) */
#define NBODY_F64E  3  /* binary64-class accuracy from float-float (about 48-bit) arithmetic on
                          the binary32 pipes, on coordinates re-centred per j-tile; tile partial
                          sums folded into binary64; state and update in binary64. */

/* ---- time integration schemes ------------------------------------------ */
#define NBODY_KDK 0    /* Eq. 5-7 (section 1): predictor, drift, one force evaluation, corrector */
#define NBODY_RK4 1    /* the paper's fourth-order scheme (abstract), read as classical
                          Runge-Kutta on (r, v): four force evaluations per step */
#define NBODY_FR4 2    /* the other reading of that scheme: the fourth-order symplectic
                          composition of the KDK step (Yoshida 1990; Forest and Ruth 1990),
                          three KDK steps of w1 dt, w0 dt, w1 dt with w1 = 1/(2 - 2^(1/3)),
                          w0 = 1 - 2 w1 (binary64 roundings of the exact values): three
                          force evaluations per step */

typedef struct nbody_ctx nbody_ctx;

/* Library version as 10000*major + 100*minor + patch. */
int nbody_version(void);

/* Text for an error code (static storage, never NULL). */
const char *nbody_strerror(int code);

/* Detail of the last failure on this thread (static per-thread storage). */
const char *nbody_last_error(void);

/*
 * Create a simulation context for n particles (Eq. 1: i = 1..n) with
 * softening eps (the paper's delta, Eq. 2: |r_i - r_j + delta| =
 * sqrt(|r_i - r_j|^2 + delta^2)) and gravitational constant G, in precision
 * `mode`, on the current CUDA device, issuing work on `cuda_stream`
 * (a cudaStream_t, or NULL).  Allocates the resident device state.
 * eps == 0 is allowed (the self pair j == i is excluded explicitly, Eq. 1);
 * coincident particles then give non-finite results, as Eq. 2 does.
 * Errors: EINVAL (n < 1, eps < 0 or non-finite, G non-finite, unknown mode,
 * out == NULL), ENOMEM, ECUDA.
 */
int nbody_create(nbody_ctx **out, int64_t n, int mode, double eps, double G, void *cuda_stream);

/* Free a context and its device memory (synchronises its stream).  NULL is a no-op. */
int nbody_destroy(nbody_ctx *ctx);

/*
 * Bound, in seconds, on every host wait of this context (the calls that
 * synchronise).  0 (the default) waits without limit.  When a wait exceeds
 * the bound the call returns NBODY_ETIMEOUT; the queued GPU work is not
 * cancelled, and the context may be used again once it has finished.
 */
int nbody_set_timeout(nbody_ctx *ctx, double seconds);

/*
 * Set positions pos (n x 3), velocities vel (n x 3) and masses mass (n) and
 * reset the time to 0 and the step counter to 0.  vel may be NULL (zero
 * velocities).  Inputs are checked: any non-finite value or a negative mass
 * gives EINVAL and leaves the previous state in place.  Synchronises.
 */
int nbody_set_state(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                    int on_device);

/*
 * Set the model time and step counter reported by nbody_get_state, e.g. after
 * nbody_set_state from a checkpoint.  Resuming from a checkpoint (set_state
 * with the saved positions, velocities and masses, then set_clock) continues
 * the trajectory bit for bit: a(t) is recomputed from the same positions by
 * the same deterministic kernels.  EINVAL for non-finite t or step < 0.
 */
int nbody_set_clock(nbody_ctx *ctx, double t, int64_t step);

/*
 * Read the state at the current step boundary: pos (n x 3), vel (n x 3),
 * the model time *t and the step counter *step.  Any output may be NULL.
 * Synchronises.  ESTATE before nbody_set_state.
 */
int nbody_get_state(nbody_ctx *ctx, double *pos, double *vel, double *t, int64_t *step,
                    int on_device);

/*
 * Eq. 1-2 for an arbitrary particle set of the context's size n, in the
 * context's mode and with its eps and G; does not touch the simulation state:
 *   acc_i = -G sum_{j != i} m_j (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^{3/2}   (n x 3)
 *   pot_i = -G sum_{j != i} m_j / (|r_i - r_j|^2 + eps^2)^{1/2}               (n)
 * pot may be NULL.  Synchronises.  Errors: EINVAL (NULL pos/mass/acc),
 * ECUDA.  Inputs are not scanned for non-finite values (use set_state for
 * checked input); a NaN input gives NaN outputs.
 */
int nbody_accel(nbody_ctx *ctx, const double *pos, const double *mass, double *acc, double *pot,
                int on_device);

/*
 * Eq. 1-2 for the rows i in [i0, i0 + ni) only, against all n particles of
 * pos (n x 3) and mass (n): acc (ni x 3) and pot (ni, may be NULL) for those
 * rows, row k holding particle i0 + k.  This is the per-GPU share of the
 * paper's i-partition of the force sum over k GPUs (section 2, Figs. 1-3:
 * every GPU holds all positions and sums N/k particles).  It always uses the
 * one-sided kernels in input order with the context's launch shape, so the
 * rows equal, bit for bit, the same rows of nbody_accel on a context with the
 * each-pair-once path off (nbody_set_symmetric 0) and NBODY_ORDER_INPUT.
 * Does not touch the simulation state.  Synchronises.  Errors: EINVAL (NULL
 * pos/mass/acc, i0 < 0, ni < 1, i0 + ni > n), ENOMEM, ECUDA.
 */
int nbody_accel_rows(nbody_ctx *ctx, int64_t i0, int64_t ni, const double *pos, const double *mass,
                     double *acc, double *pot, int on_device);

/*
 * Accelerations and potentials of the current state (those of the last force
 * evaluation at the state's positions, computed now if stale).  acc (n x 3),
 * pot (n); either may be NULL.  Synchronises.
 */
int nbody_get_accel(nbody_ctx *ctx, double *acc, double *pot, int on_device);

/*
 * Advance the state nsteps steps of size dt with `scheme` (NBODY_KDK: Eq. 5-7;
 * NBODY_RK4: classical Runge-Kutta; NBODY_FR4: the fourth-order composition of
 * Eq. 5-7).  KDK and FR4 need a(t) before their first step (Eq. 5): it is
 * evaluated once when stale, so nsteps KDK steps cost nsteps + 1 force
 * evaluations the first time and nsteps afterwards (FR4: 3 nsteps + 1, 3 nsteps).
 * Stream-ordered: returns once the work is queued.
 * Errors: EINVAL (unknown scheme, dt <= 0 or non-finite, nsteps < 0),
 * ESTATE, ECUDA.
 */
int nbody_step(nbody_ctx *ctx, int scheme, double dt, int64_t nsteps);

/*
 * Eq. 8-10 at the current state, reduced on the GPU in binary64 in a fixed
 * order (deterministic):
 *   *E  = sum_i m_i |v_i|^2 / 2 - 1/2 sum_i sum_{j != i} G m_i m_j / |r_i - r_j + eps|
 *         (Eq. 8 prints the potential term with a + sign; a bound system has
 *          negative potential energy, so it is taken with a - sign here)
 *   P   = sum_i m_i v_i                            (Eq. 9; 3 doubles)
 *   L   = sum_i m_i r_i x v_i                      (3 doubles; L[2] is Eq. 10)
 * Any output may be NULL.  K and W separately: nbody_diagnostics_ext.
 * Synchronises.
 */
int nbody_diagnostics(nbody_ctx *ctx, double *E, double *P, double *L);

/* As nbody_diagnostics, plus kinetic energy *K and potential energy *W (E = K + W). */
int nbody_diagnostics_ext(nbody_ctx *ctx, double *E, double *K, double *W, double *P, double *L);

/*
 * Force-kernel launch shape (for tuning; 0 = library default for that field):
 *   ipt    -- i-particles held in registers per thread (1, 2, 4 or 8; NBODY_F64E uses
 *             at most 4)
 *   jsplit -- number of j-segments evaluated by separate thread blocks and
 *             summed afterwards in a fixed order (1..64)
 * The shape changes rounding order only.  EINVAL for unsupported values.
 */
int nbody_set_launch(nbody_ctx *ctx, int ipt, int jsplit);

/* Current launch shape actually used for this context's n (outputs may be NULL). */
int nbody_get_launch(nbody_ctx *ctx, int *ipt, int *jsplit, int *threads, int *tile);

/*
 * FP64 and F64E modes: evaluate each unordered pair once and apply it to both
 * particles (Newton's third law; the same terms with opposite signs, summed in
 * a different fixed order than the one-sided kernels, so results differ from
 * them by rounding only and stay deterministic).  Particles are cut into
 * blocks of 384 (FP64) or 256 (F64E).  mode = -1 (default): automatic, used
 * when n spans at least 64 blocks; 0: never; 1: whenever n spans at least 2
 * blocks.  The launch shape of nbody_set_launch does not apply to this path.
 * Memory: the first force evaluation on this path allocates the context's
 * per-diagonal row and column buffers (2 x D x n x 32 bytes, at most 1 GiB;
 * D = 8 at n = 2^20 in FP64) and P + 2 slices of partial sums (P <= 4);
 * mode 0 avoids both.
 * Errors: EINVAL (NULL context, mode outside -1..1, mode 1 in MIXED or FP32).
 */
int nbody_set_symmetric(nbody_ctx *ctx, int mode);
/* The setting (-1, 0, 1) and whether the next force evaluation uses the path. */
int nbody_get_symmetric(const nbody_ctx *ctx, int *mode, int *active);

/*
 * Particle order of the force sum (a project addition; the paper sums in input
 * order).  NBODY_ORDER_SPATIAL sorts the particles along a Morton (Z-order)
 * curve of their positions before each force evaluation (bounding box,
 * 21-bit cells per coordinate, stable sort on the 63-bit keys) and runs the
 * force kernels on the sorted copy; results come back in input order.  The
 * order is a deterministic function of the positions, so results stay
 * reproducible bit for bit.  It matters for NBODY_MIXED: the binary32
 * coordinates relative to a j-tile's anchor keep their digits only when the
 * tile is spatially compact (force error at eps = 1e-3 several times
 * smaller); NBODY_F64E gains less (its float-float coordinates lose digits
 * only far from the anchor).  It is the default in both; NBODY_ORDER_INPUT in
 * NBODY_FP64 (which accepts either: the order changes only its summation
 * order).  NBODY_FP32 keeps input order (the paper's SP).
 * Memory: the first force evaluation with the spatial order allocates about
 * 70 + 32 S bytes per particle (keys, indices, permutation, sort scratch and
 * sorted copies of the positions and of the S partial-sum slices).
 * Errors: EINVAL (NULL context, unknown order, NBODY_ORDER_SPATIAL in FP32).
 */
#define NBODY_ORDER_INPUT   0
#define NBODY_ORDER_SPATIAL 1
int nbody_set_order(nbody_ctx *ctx, int order);
int nbody_get_order(const nbody_ctx *ctx, int *order);

/* Number of kernel launches this context has issued since creation. */
int64_t nbody_launch_count(const nbody_ctx *ctx);

/*
 * Opt-in timing of the force kernel (Eq. 1-2 sum, the O(N^2) part): when
 * enabled, every force-kernel launch is bracketed by two CUDA events recorded
 * on the context's stream.  nbody_profile_read synchronises, returns the
 * summed event time in milliseconds and the number of timed launches since
 * the last read (or since enabling), and resets both.  Either output may be
 * NULL.  Disabled by default.
 */
int nbody_profile(nbody_ctx *ctx, int enable);
int nbody_profile_read(nbody_ctx *ctx, double *force_ms, int64_t *force_launches);

/*
 * Measured issue rates of the pipes that bound the force kernels, on the
 * current device (the denominators of their rooflines; the paper reports no
 * such figures).  Each rate is timed with CUDA events over a kernel that runs
 * one full wave of resident blocks issuing only independent chains of one
 * instruction; the SM clock is read from the cycle counter of one block of
 * the binary64 kernel.  Runs about 0.2 s on the legacy default stream and
 * synchronises the device.  out[0..NBODY_PIPE_FIELDS-1] receives:
 *   0 SM count            1 SM clock [MHz] during the run
 *   2 DFMA  [G instr/s]   3 FFMA lane-ops [G/s]   4 FFMA2 (packed) lane-ops [G/s]
 *   5 MUFU.RSQ [G/s]      6 DFMA per clock per SM  7 FFMA2 lane-ops per clock per SM
 *   8 MUFU.RSQ per clock per SM
 * Allocates 16 bytes of device memory for the duration of the call.
 * Errors: EINVAL (out NULL or nout < NBODY_PIPE_FIELDS), ENOMEM, ECUDA.
 */
#define NBODY_PIPE_FIELDS 9
int nbody_measure_pipes(double *out, int nout);

/* ======================================================================
 * Batched execution of many independent simulations (serving).
 *
 * A batch is a device pool of `capacity` particles shared by up to
 * `max_sims` resident simulations of uneven size.  Each simulation runs the
 * KDK leapfrog of Eq. 5-7 over the Eq. 1-2 force sum with its own n, eps, G,
 * dt and mode (NBODY_FP64, NBODY_MIXED or NBODY_F64E; NBODY_FP32 is not
 * offered here).
 * One tick (nbody_batch_step) advances every resident simulation by one
 * step in a few launches whose thread blocks are work units of single
 * simulations, so small and large simulations share the GPU.  A simulation's
 * first tick after admission evaluates a(t0) (Eq. 5 needs it) and does not
 * count as a step.  Results of one simulation do not depend on which others
 * share its ticks beyond the summation-order effect of the launch shape.
 * All work is ordered on the stream given at creation; calls that return
 * host values synchronise it.  The paper runs one system at a time; this
 * interface is the library's own.
 * ====================================================================== */
typedef struct nbody_batch nbody_batch;

/* Device bytes the pool reserves per particle of capacity. */
int64_t nbody_batch_bytes_per_particle(void);

/* Text of the last batch failure on this thread. */
const char *nbody_batch_last_error(void);

/* Create a pool (allocates capacity x nbody_batch_bytes_per_particle() bytes).
 * Errors: EINVAL (capacity < 1, max_sims < 1), ENOMEM, ECUDA. */
int nbody_batch_create(nbody_batch **out, int64_t capacity, int max_sims, void *cuda_stream);
int nbody_batch_destroy(nbody_batch *b);

/* Admit a simulation: pos (n x 3), vel (n x 3, NULL = at rest), mass (n),
 * host (on_device = 0; checked for non-finite values and negative masses,
 * copied before the call returns) or device pointers (on_device = 1; read in
 * stream order).  *slot receives its handle.  Errors: ENOSPC when no slot
 * or no contiguous free range of n particles is left (retry after an
 * eviction), EINVAL, ECUDA.  Does not synchronise. */
int nbody_batch_admit(nbody_batch *b, int64_t n, int mode, double eps, double G, double dt,
                      const double *pos, const double *vel, const double *mass, int on_device,
                      int *slot);

/* Remove a simulation and return its slot and range (stream-ordered). */
int nbody_batch_evict(nbody_batch *b, int slot);

/* Queue nticks ticks (each: one KDK step of every resident simulation). */
int nbody_batch_step(nbody_batch *b, int64_t nticks);

/* Wait for all queued work of the pool. */
int nbody_batch_sync(nbody_batch *b);

/* Non-blocking: 1 when all queued work of the pool has finished, 0 when some
 * is still running, a negative code on error. */
int nbody_batch_query(nbody_batch *b);

/* State (n x 3 each; either may be NULL), time and step count of one
 * simulation at its current step boundary.  Synchronises. */
int nbody_batch_get_state(nbody_batch *b, int slot, double *pos, double *vel, double *t,
                          int64_t *step, int on_device);

/* a(t) and pot at the current positions of one simulation (after its first
 * tick; ESTATE before).  Synchronises. */
int nbody_batch_get_accel(nbody_batch *b, int slot, double *acc, double *pot, int on_device);

/* Eq. 8-10 for one simulation (as nbody_diagnostics_ext).  Synchronises. */
int nbody_batch_diagnostics(nbody_batch *b, int slot, double *E, double *K, double *W, double *P,
                            double *L);

/* Occupancy: resident simulations, particles in use (rounded to the pool
 * alignment) and the largest free contiguous range. */
int nbody_batch_info(nbody_batch *b, int *active, int64_t *used, int64_t *largest_free);
int nbody_batch_slot_info(nbody_batch *b, int slot, int64_t *n, int *mode, int64_t *steps);

/* Launch shape for one mode's force launches: i-particles per thread (1, 2,
 * 4, 8) and target j-segment length (rounded up to the tile; a simulation
 * is split into at most 16 segments).  Changes rounding order only. */
int nbody_batch_set_launch(nbody_batch *b, int mode, int ipt, int64_t seg);

/* FP64 force launches of this pool run as a persistent grid of at most
 * blocks_per_sm thread blocks per SM (default 2; 0 = one block per work unit).
 * FP64 work keeps the FP64 pipe busy with few warps; capping its residency
 * leaves the rest of each SM to FP32-bound work of other streams (for
 * instance a MIXED pool ticking at the same time). */
int nbody_batch_set_fp64_residency(nbody_batch *b, int blocks_per_sm);

/* Per-tick CUDA-event timing (see nbody_batch_profile_read). */
int nbody_batch_profile(nbody_batch *b, int enable);

/* Synchronise and return, for up to `cap` ticks recorded since the last
 * read: tick_ms[k] (whole tick), force_ms[3k..3k+2] (the FP64, MIXED and
 * F64E force launches, 0 when absent), inter[3k..3k+2] (their interactions,
 * n^2 summed over simulations); *nticks = ticks recorded.  Any array may be
 * NULL; the record is cleared. */
int nbody_batch_profile_read(nbody_batch *b, int64_t cap, double *tick_ms, double *force_ms,
                             double *inter, int64_t *nticks);

/* Kernel launches issued by the pool since creation. */
int64_t nbody_batch_launch_count(const nbody_batch *b);

/*
 * Allocation-free variant of the binary64 force evaluation: the same Eq. 1-2
 * result as nbody_accel on an NBODY_FP64 context (acc n x 3, pot n, same
 * kernel), but with no context and no device allocation by the library, for
 * callers that cannot let it call cudaMalloc: an application that owns all GPU
 * memory through its own allocator (or has reserved it), or a timing-critical
 * loop where an allocation or free would stall the device.  The paper has no
 * counterpart of this entry point.
 *   pos (n x 3), mass (n), acc (n x 3), pot (n, may be NULL): device pointers
 *   owned by the caller; work is queued on cuda_stream (NULL = default stream)
 *   and the call returns before it finishes.
 * Scratch: one file-scope device array of NBODY_STATIC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits; it limits n to
 * NBODY_STATIC_MAX_N, and a larger n returns NBODY_EINVAL before any launch.
 * All calls share that array (nothing in it needs clearing between calls), so
 * calls whose work overlaps on the GPU (several streams or host threads) race
 * and give wrong results: order them on one stream.  The array's device
 * address is looked up once per CUDA context with that context current (the
 * first call in a device's primary context, again after cudaDeviceReset, and
 * in any other context the caller makes current); make that first call before
 * any stream capture begins.  Inputs are not scanned for non-finite values
 * (as in nbody_accel): a NaN input gives NaN outputs.
 * Errors (detail in nbody_last_error): EINVAL (n < 1, n > NBODY_STATIC_MAX_N,
 * NULL pos/mass/acc, eps < 0 or non-finite, G non-finite), ECUDA.
 */
#define NBODY_STATIC_MAX_N 32768
#define NBODY_STATIC_SCRATCH_BYTES (16 * 1024 * 1024)
int nbody_accel_f64_static(int64_t n, const double *pos, const double *mass, double eps, double G,
                           double *acc, double *pot, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
