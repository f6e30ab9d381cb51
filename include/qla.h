/*
 * qla.h - C ABI of the GB300 qubit lattice algorithm (QLA) library, libqla.so.
 *
 * The library advances the 2D curl Maxwell equations in a diagonal-tensor
 * dielectric with the QLA of arXiv 2301.13601 (Vahala et al.): at every site
 * of a periodic Nx x Ny lattice the 6-qubit state
 *     Q = (q0..q5) = (n_x E_x, n_y E_y, n_z E_z, B_x, B_y, B_z)        (Eq. 15)
 * is advanced by collision rotations C_X, C_Y (Eq. 17, Eq. 19), one-cell
 * streaming shifts (Eq. 18, Eq. 20) and the external potential operators V_X,
 * V_Y (Eq. 21, Eq. 22), in the plain order of Eq. 23 or the interleaved order
 * of Eq. 28, with collision angles from Eq. 24 and potential angles from Eq. 25.
 *
 * Conventions shared by every entry point:
 *  - Host arrays are row-major [Ny][Nx] planes (x fastest); a state is 6 such
 *    planes [6][Ny][Nx] in the component order of Eq. 15. Lattice units: sites
 *    at integer (x, y), spacing delta in the physical units of Eq. 25.
 *  - Streaming direction: S^{+x} sets q(x) <- q(x+1) and S^{-x} sets
 *    q(x) <- q(x-1); operator products act right to left.
 *  - Host buffers are owned by the caller and only read or written during the
 *    call (copies are synchronous unless stated). Device buffers are owned by
 *    the context unless the caller passes its own (qla_device_buffers).
 *  - Every call returns a qla_status. QLA_EINVAL (bad argument) leaves the
 *    context usable. Any CUDA failure is sticky: the context records the first
 *    one, returns it from every later call and keeps its text for
 *    qla_last_error() until qla_destroy().
 *  - Calls on one context are not thread-safe; different contexts are
 *    independent. Work runs on the context's stream, in call order.
 */
#ifndef QLA_H
#define QLA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qla_ctx qla_ctx;

typedef enum {
    QLA_OK = 0,
    QLA_EINVAL = 1,        /* invalid argument (sizes, delta, non-finite or non-positive n, NULL) */
    QLA_ENOMEM = 2,        /* device or host allocation failed */
    QLA_ECUDA = 3,         /* a CUDA runtime call failed (sticky) */
    QLA_ETIMEOUT = 4,      /* a bounded device-side wait gave up (sticky) */
    QLA_ENONFINITE = 5,    /* the state holds NaN or Inf (reported by the diagnostics) */
    QLA_EUNSUPPORTED = 6,  /* option combination not built (e.g. unsupported steps_per_pass) */
    QLA_ESTATE = 7         /* call out of order (e.g. step before any state was set) */
} qla_status;

enum { QLA_FP32 = 0, QLA_FP64 = 1 };                        /* state / arithmetic precision */
enum { QLA_SEQ_INTERLEAVED = 0, QLA_SEQ_PLAIN = 1 };        /* Eq. 28 / Eq. 23 */
enum { QLA_POT_PAPER = 0, QLA_POT_UNITARY = 1 };            /* V as printed / unitary variant */
enum { QLA_POL_EZ = 0, QLA_POL_EY = 1 };                    /* pulse polarisation */
/* Polarisation families advanced (qla_options.families). The six components
 * split into two families that no operator of Eq. 17-22 couples (C_X pairs
 * (q1,q5), (q2,q4); C_Y (q0,q5), (q2,q3); the potential rows 5<-1, 4<-2,
 * 3<-2, 5<-0): TM = (q2, q3, q4) = (n_z E_z, B_x, B_y), the E_z polarisation;
 * TE = (q0, q1, q5) = (n_x E_x, n_y E_y, B_z), the E_y polarisation. A field
 * with only one family's components nonzero keeps the other family at exactly
 * zero, so advancing one family gives the same result at half the work. */
enum { QLA_FAMILIES_BOTH = 0, QLA_FAMILY_TM = 1, QLA_FAMILY_TE = 2 };
/* How qla_step launches the passes of the balanced split (qla_options.launch).
 * QLA_LAUNCH_PER_PASS: one kernel launch per pass of steps_per_pass steps.
 * QLA_LAUNCH_PERSISTENT: all the full passes of one qla_step call in one
 *   cooperative launch, one CTA per resident slot; CTA b sweeps share b of each
 *   advanced family in every pass and, before a pass, waits only for the shares
 *   whose previous pass wrote what it reads or read what it overwrites (see
 *   qla_sweep_dependencies), not for the whole lattice. Bit-identical results.
 *   Applies to FP32 contexts with the balanced split (chunk_rows = 0), 2 steps
 *   per pass, Nx a multiple of 8 and at least 256; other contexts, and a launch
 *   the device refuses, use one launch per pass.
 * QLA_LAUNCH_AUTO: one launch per pass (the faster form where measured). */
enum { QLA_LAUNCH_AUTO = 0, QLA_LAUNCH_PER_PASS = 1, QLA_LAUNCH_PERSISTENT = 2 };

/* Options for qla_create. Obtain defaults with qla_default_options().
 * potential: QLA_POT_PAPER applies V_X, V_Y as printed (Eq. 21-22, with
 *   row 3 of V_Y read as (0,0,sin b3,cos b3,0,0) and the "o" of its row 0 as
 *   zero). QLA_POT_UNITARY rotates each coupled pair by half the angle instead,
 *   so that every operator of the step is orthogonal (the fully unitary QLA
 *   the paper's summary calls for). */
typedef struct {
    int precision;       /* QLA_FP32 (default) or QLA_FP64 (correctness mode) */
    int sequence;        /* QLA_SEQ_INTERLEAVED (default, Eq. 28) or QLA_SEQ_PLAIN (Eq. 23) */
    int potential;       /* QLA_POT_PAPER (default) or QLA_POT_UNITARY */
    int steps_per_pass;  /* full time steps fused per HBM pass: 0 = automatic (2; FP32 with chunk_rows
                            set: 2 from 2^25 sites up, else 4), else 1, 2 or 4 */
    int chunk_rows;      /* rows of one sweep tile, else 0 = automatic: each family's rows are
                            split into one share of equal estimated cost per resident CTA
                            (see qla_sweep_split) */
    int device;          /* CUDA device ordinal; -1 = the calling thread's current device */
    void *stream;        /* cudaStream_t to run on; NULL = a non-blocking stream owned by the context */
    int families;        /* QLA_FAMILIES_BOTH (default), or QLA_FAMILY_TM / QLA_FAMILY_TE: only that
                            family is stored and advanced; the other family's components are
                            held at zero (qla_set_fields* ignore them, qla_get_fields* return
                            zeros, qla_init_pulse requires the matching polarisation) */
    int launch;          /* QLA_LAUNCH_AUTO (default), QLA_LAUNCH_PER_PASS or QLA_LAUNCH_PERSISTENT */
} qla_options;

/* Fill *opt with the defaults listed above. */
void qla_default_options(qla_options *opt);

/* Device memory one context needs (bytes; each buffer 256-byte aligned). */
typedef struct {
    size_t state_bytes;    /* one state buffer (6 planes); two are needed (ping-pong) */
    size_t coeff_bytes;    /* rotation and potential coefficient planes */
    size_t index_bytes;    /* n_x, n_y, n_z (double) */
    size_t scratch_bytes;  /* reduction scratch for the diagnostics */
} qla_buffer_sizes;

/* Report the buffer sizes qla_create needs for an Nx x Ny lattice with these
 * options (opt may be NULL for defaults). Errors: QLA_EINVAL for bad sizes. */
qla_status qla_query_buffer_sizes(int Nx, int Ny, const qla_options *opt, qla_buffer_sizes *out);

/* Caller-provided device buffers (each of the sizes above, on opt->device,
 * 256-byte aligned). They must outlive the context; the context never frees
 * them. */
typedef struct {
    void *state[2];
    void *coeff;
    void *index;
    void *scratch;
} qla_device_buffers;

/* Create a context for an Nx x Ny periodic lattice (Nx, Ny >= 1, Nx*Ny <= 2^31).
 * n_x, n_y, n_z: host [Ny][Nx] principal refractive indices (Eq. 15), copied.
 * delta: the perturbation parameter (Eq. 24-25), 0 < delta <= 0.5.
 * The collision angles theta_i = delta/(4 n_i) (Eq. 24) and potential angles
 * beta from central differences of n (Eq. 25, lattice spacing delta) are
 * computed once on the device in FP64 and stored as (cos-1, sin) pairs in the
 * state precision; in FP32 each rotation pair is rounded so that
 * (1 + m)^2 + s^2 is as close to 1 as FP32 allows.
 * buffers: NULL = the library allocates with cudaMalloc and frees on destroy.
 * The state is zero after creation. Errors: QLA_EINVAL (n <= 0, non-finite n or
 * delta, bad sizes), QLA_ENOMEM, QLA_ECUDA. On error *out is NULL. */
qla_status qla_create(int Nx, int Ny, const double *n_x, const double *n_y, const double *n_z,
                      double delta, const qla_options *opt, const qla_device_buffers *buffers,
                      qla_ctx **out);

/* Set the state to a 1D Gaussian pulse travelling in +x, uniform in y
 * (Sec. 2.2 and Sec. 4: a 1D pulse propagating in x):
 *   g(x) = amplitude * exp(-d^2 / (2 sigma^2)),  d = periodic minimum-image x - x0,
 *   QLA_POL_EZ: q2 = g, q4 = -g;  QLA_POL_EY: q1 = g, q5 = +g;  others 0.
 * (the pairings follow the +x travelling solution of Eq. 16 in a uniform medium).
 * Resets the step counter. Errors: QLA_EINVAL (sigma <= 0, bad polarisation,
 * or a polarisation whose family the context does not advance). */
qla_status qla_init_pulse(qla_ctx *ctx, int polarization, double x0, double sigma, double amplitude);

/* Copy a host state [6][Ny][Nx] (double) into the context (rounded to the
 * context precision). Resets the step counter. Synchronous. With a single
 * family (qla_options.families) only that family's three planes are copied. */
qla_status qla_set_fields(qla_ctx *ctx, const double *q);

/* Same with a float host state [6][Ny][Nx]; no rounding in FP32 mode.
 * Asynchronous with respect to the host if q is pinned (page-locked) memory. */
qla_status qla_set_fields_f32(qla_ctx *ctx, const float *q);

/* Advance nsteps >= 0 time steps (Eq. 28 or Eq. 23). Asynchronous on the
 * context stream; nsteps is split into fused passes of steps_per_pass steps
 * plus shorter passes for the remainder. */
qla_status qla_step(qla_ctx *ctx, long long nsteps);

/* Energy (Eq. 27): the mean over sites of Q.Q, reduced in FP64 with
 * compensated summation in a fixed order (deterministic). Synchronises the
 * context stream. */
qla_status qla_energy(qla_ctx *ctx, double *energy);

/* div B with central differences in lattice units,
 *   div = (B_x[x+1] - B_x[x-1])/2 + (B_y[y+1] - B_y[y-1])/2,  B = (q3, q4, q5),
 * the diagnostic behind the paper's max div B/|B| < 1e-3 (Sec. 4.1):
 * *l2_sq_sum = sum over sites of div^2, *max_abs = max |div|,
 * *max_absB = max |B|. FP64, deterministic. Synchronises. */
qla_status qla_divB(qla_ctx *ctx, double *l2_sq_sum, double *max_abs, double *max_absB);

/* Divergence of D (Sec. 4.2: for the E_y polarisation the QLA generates E_x so
 * that div D = 0). The dielectric tensor is diagonal with eps_i = n_i^2, so
 * D = (n_x q0, n_y q1, n_z q2) (Eq. 15); div D = (D_x[x+1] - D_x[x-1])/2 +
 * (D_y[y+1] - D_y[y-1])/2 in lattice units at the sites, periodic. Outputs:
 * sum over sites of div^2, max |div|, max |D|; FP64 with compensated sums,
 * deterministic. Synchronous. QLA_ENONFINITE if q0, q1 or q2 holds NaN/Inf. */
qla_status qla_divD(qla_ctx *ctx, double *l2_sq_sum, double *max_abs, double *max_absD);

/* All diagnostics from one reduction pass. nonfinite = number of non-finite
 * state values; when it is non-zero the call returns QLA_ENONFINITE (not
 * sticky) with the other fields still filled in. */
typedef struct {
    double energy;       /* Eq. 27 */
    double div_l2_sq;    /* sum div^2 */
    double div_max;      /* max |div| */
    double b_max;        /* max |B| */
    long long nonfinite; /* NaN/Inf count */
} qla_diag;

qla_status qla_diagnostics(qla_ctx *ctx, qla_diag *out);

/* The same diagnostics for a state the caller holds in device memory, with no
 * context and no device allocation. The paper has no counterpart: this exists
 * for callers that may not call cudaMalloc when they need the diagnostics (an
 * application whose device memory all belongs to its own allocator, or a loop
 * that must not block on or fail in the allocator). Its scratch is a fixed
 * 256 KB array in device memory that the library reserves on every GPU that
 * loads it, for the life of the process.
 * q: device pointer to [6][Ny][Nx] float (precision QLA_FP32) or double
 *    (QLA_FP64) on the current device; read only. out: host struct, written.
 * stream: cudaStream_t to run on (NULL = the legacy default stream); the call
 *    synchronises it before returning.
 * Limit: Ny <= 16384 (4 rows per partial record, 4096 records); a taller
 * lattice, Nx*Ny > 2^31-1, a NULL pointer or a bad precision returns
 * QLA_EINVAL without touching the GPU. CUDA failures return QLA_ECUDA.
 * Non-finite values return QLA_ENONFINITE with *out filled in.
 * Each call looks up the array's device address on the current device (so a
 * device reset or a re-created context is followed); the first call on a
 * device may also load the module: make it before any stream capture begins.
 * All calls share
 * the one array and it keeps the last call's contents (each call writes every
 * record it reads, so nothing needs clearing); calls whose kernels overlap on
 * the GPU (other streams, other host threads) race on it and must be
 * serialised by the caller. Sums are taken in a fixed order that differs from
 * qla_diagnostics, so the two agree to rounding (~1e-15 relative), not bitwise. */
qla_status qla_diagnostics_noalloc(const void *q, int precision, int Nx, int Ny, void *stream, qla_diag *out);

/* Copy the state to a caller-owned host array [6][Ny][Nx] of double
 * (or float). Synchronous. */
qla_status qla_get_fields(qla_ctx *ctx, double *q);
qla_status qla_get_fields_f32(qla_ctx *ctx, float *q);

/* Single operators of one step, for operator-level tests (Sec. 3):
 *   QLA_OP_CX, QLA_OP_CX_T: collision C_X (Eq. 17) on (q1,q5) by theta_1 and
 *     (q2,q4) by theta_2, or its transpose;
 *   QLA_OP_CY, QLA_OP_CY_T: C_Y (Eq. 19, row 2 read as (0,0,c2,s2,0,0)) on
 *     (q0,q5) by theta_0 and (q2,q3) by theta_2, or its transpose;
 *   QLA_OP_S14_XP .. QLA_OP_S25_YM: streaming S^{+x}_{14}, S^{-x}_{14},
 *     S^{+x}_{25}, S^{-x}_{25}, S^{+y}_{03}, S^{-y}_{03}, S^{+y}_{25},
 *     S^{-y}_{25} (Eq. 18, Eq. 20), with S^{+} q(r) <- q(r + e) and S^{-}
 *     q(r) <- q(r - e), periodic;
 *   QLA_OP_VX, QLA_OP_VY: the potentials (Eq. 21-22, the context's variant)
 *     with the angles of one application in the context's step (beta for
 *     Eq. 23, beta/2 for Eq. 28).
 * The same per-site arithmetic and coefficients as qla_step. */
enum {
    QLA_OP_CX = 0, QLA_OP_CX_T = 1, QLA_OP_CY = 2, QLA_OP_CY_T = 3,
    QLA_OP_S14_XP = 4, QLA_OP_S14_XM = 5, QLA_OP_S25_XP = 6, QLA_OP_S25_XM = 7,
    QLA_OP_S03_YP = 8, QLA_OP_S03_YM = 9, QLA_OP_S25_YP = 10, QLA_OP_S25_YM = 11,
    QLA_OP_VX = 12, QLA_OP_VY = 13
};

/* Apply operator `op` to the state `count` >= 0 times (asynchronous, on the
 * context stream; the step counter is unchanged). Errors: QLA_EINVAL (unknown
 * op, count < 0), QLA_ESTATE (no state), QLA_ECUDA. */
qla_status qla_debug_apply(qla_ctx *ctx, int op, int count);

/* Device pointer to the current state (6 planes [6][Ny][Nx] of float or
 * double, per the precision). Valid until the next qla_step. With a single
 * family, writes through it must leave the other family's planes zero. */
void *qla_state_device_ptr(qla_ctx *ctx);

/* Block the host until all queued work of the context has finished.
 * QLA_ETIMEOUT (sticky) if a sweep's bounded wait for its TMA row copies ran
 * out since creation; the state is then invalid. qla_diagnostics reports the
 * same condition. */
qla_status qla_synchronize(qla_ctx *ctx);

/* Steps taken since the last state reset; -1 for a NULL context. */
long long qla_step_count(const qla_ctx *ctx);

/* Resolved configuration: steps per pass and rows per tile used by qla_step
 * (0: the balanced split), and the precision. Any pointer may be NULL. */
qla_status qla_get_config(const qla_ctx *ctx, int *steps_per_pass, int *chunk_rows, int *precision);

/* The launch form qla_step uses for the context's passes of steps_per_pass
 * steps: QLA_LAUNCH_PERSISTENT or QLA_LAUNCH_PER_PASS (the option resolved
 * against what the context allows; PER_PASS after the device refused a
 * cooperative launch). QLA_EINVAL on NULL. */
qla_status qla_get_launch(const qla_ctx *ctx, int *launch);

/* Test hook of the persistent launch form: the limit in nanoseconds of the
 * waits of one pass for the shares it depends on (default 2 s), and a number
 * of extra passes every such wait demands (0 normally; a positive value makes
 * the first wait run out, which must end the call with QLA_ETIMEOUT at the
 * next synchronisation instead of hanging; the context then stays in that
 * error). Takes effect at the next qla_step. QLA_EINVAL on NULL, a limit
 * <= 0 or a negative withhold. */
qla_status qla_set_wait_limit(qla_ctx *ctx, long long timeout_ns, int withhold);

/* The balanced split of one fused pass of steps_per_pass steps (the sweep of
 * Eq. 28 / Eq. 23 over the lattice, one CTA grid layer per family). The
 * lattice is cut into strips of 256 - 8K output columns (K = steps_per_pass;
 * a strip reads 256 columns, its halo included); in FP32 with K >= 2 and Nx a
 * multiple of 8, at least 256, strip 0 straddles the periodic seam x = 0 and
 * strips 1.. cover the columns between. Row unit u = strip * Ny + y. The
 * `ctas` CTAs of a family's layer sweep the units [bounds[b], bounds[b + 1])
 * (share b). Shares are sized by estimated cost: one per row (the seam
 * strip's rows a little more), plus the 8K + R (K - 1) warm-up rows, R = 4
 * (8 for FP32 at K = 1), at each strip start, and weighted by the CTAs' start
 * (with one layer, or in the first of two: the first ctas/2 CTAs, the first
 * resident on their SMs, a few percent more; in the second of two layers,
 * where the CTAs start as the first layer's finish, decreasing with the order
 * of start, share b going to the b-th CTA to start).
 * family: QLA_FAMILY_TM or QLA_FAMILY_TE; layers: 1 (one family advanced) or
 * 2 (both: TM is the first layer). bounds: caller-owned, capacity >= ctas + 1
 * entries; bounds[0] = 0 and bounds[ctas] = strips * Ny. Host arithmetic only:
 * needs no GPU. QLA_EINVAL on a bad size, precision, family, layer count, CTA
 * count or capacity; QLA_EUNSUPPORTED if steps_per_pass is not instantiated
 * for the precision. */
qla_status qla_sweep_split(int Nx, int Ny, int precision, int steps_per_pass, int ctas, int family, int layers,
                           long long *bounds, int capacity);

/* The shares that share `share` of the persistent launch form waits for
 * before each of its passes after the first (QLA_LAUNCH_PERSISTENT): the other
 * shares of the same family (split as qla_sweep_split with layers = 1, FP32)
 * whose previous pass wrote a cell that it reads or read a cell that it
 * overwrites. A segment of rows [y0, y1) of a strip writes those rows of the
 * strip's output columns and reads rows [y0 - 4K, y1 + 4K + R - 1) of its 256
 * input columns (a pass of K steps has dependency radius 4K along each axis,
 * Eq. 18 and Eq. 20; R = 4 rows per iteration); the test takes rows
 * [y0 - 4K - R, y1 + 4K + R) against the other share's rows, either way, so
 * the list may hold a few more shares than strictly needed, never fewer.
 * Writes the share indices in increasing order to deps (caller-owned,
 * capacity entries) and their number to *count. Host arithmetic only (the
 * same function the kernel evaluates): needs no GPU. QLA_EINVAL on a bad
 * size, family, CTA count, share or capacity; QLA_EUNSUPPORTED if the
 * persistent form is not built for steps_per_pass or the lattice has no seam
 * layout (Nx not a multiple of 8, or below 256). */
qla_status qla_sweep_dependencies(int Nx, int Ny, int steps_per_pass, int ctas, int family, int share, int *deps,
                                  int capacity, int *count);

/* The split the context's passes of steps_per_pass steps use for `family`
 * (with the persistent launch form, one layer's split per family):
 * *ctas = CTAs of the family's layer (0 when the context sweeps tiles of
 * chunk_rows rows instead, or does not advance the family), and, if bounds is
 * not NULL and *ctas > 0, the share bounds as qla_sweep_split writes them
 * (capacity >= *ctas + 1). */
qla_status qla_get_sweep_split(const qla_ctx *ctx, int steps_per_pass, int family, int *ctas, long long *bounds,
                               int capacity);

/* Text of the last error on the context (empty string if none). */
const char *qla_last_error(const qla_ctx *ctx);

/* Name of a status code. */
const char *qla_status_string(qla_status s);

/* Release the context and any device memory it allocated. NULL is a no-op. */
void qla_destroy(qla_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Batched lattices: many independent scattering problems (each its own
 * periodic lattice, medium, delta and pulse, Sec. 4 setting) advanced by one
 * persistent kernel launch that is captured once into a CUDA graph and
 * replayed by every qla_batch_run. The kernel takes work items
 * (instance, pass of steps_per_pass fused steps, family, tile) from a queue
 * ordered by pass; before a pass it waits, with a time limit, for the
 * previous pass of the same lattice to complete. FP32 only.
 * ------------------------------------------------------------------------- */
typedef struct qla_batch qla_batch;

typedef struct {
    int Nx, Ny;                      /* lattice; Nx a multiple of 4, Nx*Ny <= 2^31 - 1 */
    const double *n_x, *n_y, *n_z;   /* host [Ny][Nx] refractive indices, copied */
    double delta;                    /* 0 < delta <= 0.5 (Eq. 24-25) */
    long long nsteps;                /* steps per qla_batch_run; a multiple of steps_per_pass */
    int pulse_polarization;          /* QLA_POL_EZ or QLA_POL_EY: initial pulse as qla_init_pulse; -1: zero state */
    double pulse_x0, pulse_sigma, pulse_amplitude;
    int chunk_rows;                  /* rows per tile; 0 = automatic */
} qla_instance_desc;

/* Create a batch of `count` lattices (descs copied; the host arrays are only
 * read during the call). opt: precision must be QLA_FP32; steps_per_pass 2 or 4
 * (0 = 4); sequence and potential apply to every lattice; opt->stream is
 * ignored (the batch owns a stream). Errors: QLA_EINVAL (bad descriptor),
 * QLA_EUNSUPPORTED (precision, steps_per_pass, or opt->families other than
 * QLA_FAMILIES_BOTH), QLA_ENOMEM, QLA_ECUDA. */
qla_status qla_batch_create(int count, const qla_instance_desc *descs, const qla_options *opt, qla_batch **out);

/* Advance every lattice by its nsteps (one graph launch; blocks until done).
 * QLA_ETIMEOUT if a dependency wait or a tile's wait for its TMA copies
 * exceeded its limit (the states are then partially advanced and should be
 * discarded). */
qla_status qla_batch_run(qla_batch *b);

/* State of lattice i (creation order) as a host float array [6][Ny][Nx]. */
qla_status qla_batch_get_fields_f32(qla_batch *b, int i, float *q);

/* Diagnostics of lattice i (as qla_diagnostics). */
qla_status qla_batch_diagnostics(qla_batch *b, int i, qla_diag *out);

/* Work items per run, steps per pass, and site-updates per run. */
qla_status qla_batch_info(const qla_batch *b, long long *total_items, int *steps_per_pass, long long *site_updates);

/* Test hook: limit of each dependency wait in nanoseconds (default 4 s), and a
 * number of extra tile completions every dependency waits for (0 normally; a
 * positive value makes the first wait run out, which must end the run with
 * QLA_ETIMEOUT instead of hanging). Takes effect at the next qla_batch_run. */
qla_status qla_batch_set_wait_limit(qla_batch *b, long long timeout_ns, int withhold);

const char *qla_batch_last_error(const qla_batch *b);
void qla_batch_destroy(qla_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* QLA_H */
