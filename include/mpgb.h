/*
 * mpgb.h — C ABI of the GB300 (sm_103a) Matching Pursuit decoder.
 *
 * The library recovers a sparse x in R^M from y = Psi x (Sec. 2, Eq. 2),
 * Psi an N x M dictionary with unit-L2 columns (Eq. 4), by the Matching
 * Pursuit iteration of Sec. 3 (Eqs. 8-12):
 *
 *     r <- y, x~ <- 0, t <- 0
 *     while ||r||_2 > eps ||y||_2 and t < T:
 *         i <- argmax_m |<r, psi_m>|     (smallest index on ties, Sec. 4)
 *         x~_i <- x~_i + <r, psi_i>
 *         r <- r - <r, psi_i> psi_i
 *         t <- t + 1
 *
 * Conventions shared by every entry point:
 *  - Indices are 0-based.  All sizes are element counts.
 *  - "device pointer" means memory of the current CUDA device (for example a
 *    torch tensor's data_ptr()); "host pointer" means ordinary CPU memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device-pointer entry points are stream-ordered: they enqueue
 *    work and return; buffers must stay valid until the stream reaches it.
 *  - Errors are returned as mp_status codes, never thrown or aborted; a
 *    human-readable reason for the last failure on the calling thread is
 *    given by mp_last_error_message().
 *  - The loop test is evaluated in the squared form
 *        e > eps^2 * e0,  e = sum_n r_n^2,  e0 = sum_n y_n^2
 *    with e and e0 accumulated in FP64 on the device.  In exact arithmetic
 *    it is Sec. 3's test ||r|| > eps ||y||.
 *  - A plan is not thread-safe: calls on one plan must be serialised by the
 *    caller (one host thread, one stream at a time).  Different plans are
 *    independent.
 */
#ifndef MPGB_H
#define MPGB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MPGB_API __attribute__((visibility("default")))
#else
#define MPGB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Status codes, precisions, layouts                                   */
/* ------------------------------------------------------------------ */

typedef enum {
    MP_OK = 0,
    MP_PENDING = 1,            /* server: request not finished yet            */
    MP_ERR_INVALID = -1,       /* bad argument or size, or non-unit atom      */
    MP_ERR_NOMEM = -2,         /* device or host allocation failed            */
    MP_ERR_BUSY = -3,          /* server: over its HBM or queue budget        */
    MP_ERR_TIMEOUT = -4,       /* a device-side wait ran past its limit       */
    MP_ERR_NONFINITE = -5,     /* non-finite input (y or Psi)                 */
    MP_ERR_CUDA = -6,          /* a CUDA runtime call failed                  */
    MP_ERR_UNSUPPORTED = -7,   /* size or precision the library cannot run    */
    MP_ERR_NOT_FOUND = -8      /* server: unknown ticket or dictionary        */
} mp_status;

typedef enum {
    MP_PREC_FP32 = 0,          /* FP32 correlations (CUDA cores)                    */
    MP_PREC_BF16 = 1,          /* BF16 correlations on tcgen05, FP32 top-8 rescore  */
    MP_PREC_FP8E4M3 = 2,       /* FP8-E4M3 per-atom-scaled correlations, FP32 rescore */
    MP_PREC_FP64 = 3           /* FP64 atoms, residual and correlations (CUDA cores): */
                               /* the double-precision decode of Sec. 5              */
} mp_precision;

typedef enum {
    MP_LAYOUT_ATOM_MAJOR = 0,  /* M rows of N floats: row m is psi_m (column m of Psi) */
    MP_LAYOUT_ROW_MAJOR = 1    /* Psi itself, N rows of M floats                       */
} mp_layout;

typedef enum {
    MP_STOP_CONVERGED = 0,     /* ||r|| <= eps ||y||                          */
    MP_STOP_MAX_ITERS = 1,     /* t reached T                                 */
    MP_STOP_ZERO_Y = 2,        /* y == 0                                      */
    MP_STOP_RANK = 3           /* OMP: the selected atom lies in the span of  */
                               /* the atoms already selected                  */
} mp_stop_reason;

typedef struct mp_plan_s* mp_plan_t;
typedef struct mp_server_s* mp_server_t;

/* Dictionary description for mp_plan_create. */
typedef struct {
    int N;                     /* measurement length, rows of Psi (>= 1)             */
    int M;                     /* number of atoms, columns of Psi (>= 1)             */
    int layout;                /* mp_layout of the psi pointer                       */
    unsigned prec_mask;        /* bit (1u << p) builds the copy for precision p;     */
                               /* FP32 is always built                               */
    int normalize;             /* nonzero: scale atoms to unit norm (Eq. 4);         */
                               /* zero: reject atoms with | ||psi_m|| - 1 | > 1e-5   */
    int reserved;              /* must be 0                                          */
} mp_plan_desc;

/* Stopping parameters of Sec. 3's loop (eps, T). */
typedef struct {
    double eps;                /* relative residual target, >= 0                     */
    int max_iters;             /* T, >= 0                                            */
    int reserved;              /* must be 0                                          */
} mp_stop;

/* Per-signal result. */
typedef struct {
    int iters;                 /* t at exit: number of completed updates             */
    int stop_reason;           /* mp_stop_reason                                     */
    int status;                /* mp_status of this signal                           */
    int reserved;
    double rel_residual;       /* ||r|| / ||y|| at exit (0 when y == 0)               */
    double energy_audit_max;   /* max_k |e_k - (e_{k-1} - c_k^2)| / e_0, where c_k is */
                               /* the committed coefficient (energy conservation,     */
                               /* Eq. 11 with Eq. 4)                                  */
} mp_result;

/* Optional per-iteration trace, device pointers (any may be NULL).
 * Entry k (k < capacity) records step k: the selected atom, the
 * coefficient added to x~ (Eq. 10) and the FP64 energy after the step.
 * `residual` (N floats) receives the final residual r. */
typedef struct {
    int* atoms;
    float* coefs;
    double* energies;
    float* residual;
    int capacity;
    int reserved;
} mp_trace;

/* The same trace for mp_recover_f64: coefficients and residual in FP64. */
typedef struct {
    int* atoms;
    double* coefs;
    double* energies;
    double* residual;
    int capacity;
    int reserved;
} mp_trace_f64;

/* Plan options for mp_plan_set_option. */
typedef enum {
    MP_OPT_PLAIN_MODE = 1,     /* 0 auto, 1 one-cluster resident, 2 grid resident,   */
                               /* 3 grid streaming (TMA ring)                        */
    MP_OPT_WATCHDOG_NS = 2,    /* limit of every device-side wait, ns (default 2e9)  */
    MP_OPT_DEBUG_SKIP_ARRIVE = 3, /* grid modes: this CTA never arrives at the first */
                               /* grid barrier (watchdog test), -1 = off             */
    MP_OPT_GRID_CTAS = 4,      /* grid modes: CTA count (0 = one per SM)             */
    MP_OPT_BATCH_TILE_N = 5,   /* batched: atoms per GEMM tile, 128..256 in steps of */
                               /* 32 (0 = autotuned)                                 */
    MP_OPT_PLAIN_PREFETCH = 6, /* grid streaming: stages pulled into L2 ahead of the */
                               /* shared-memory ring (0 = off, the default)          */
                               /* (7: no longer used)                                */
    MP_OPT_PLAIN_STAGE_BYTES = 8, /* grid streaming: target bytes per ring stage     */
                               /* (whole atoms, at least one; default 32768)         */
    MP_OPT_PLAIN_EVICT_FIRST = 9, /* grid streaming: 1 = evict-first L2 hint on the  */
                               /* streamed atoms (default), 0 = no hint              */
    MP_OPT_BATCH_AUTOTUNE = 10,/* batched: 1 = time the GEMM tile shapes on the first */
                               /* batch of each size bucket (default), 0 = heuristic */
    MP_OPT_PLAIN_GRAM = 11,    /* FP32 decode with Gram-updated correlations, period */
                               /* R >= 1 (0 = off, the default).  Not in the paper:   */
                               /* from Eqs. 9 and 11, <r - c psi_k, psi_m> =          */
                               /* c_m - c G[k][m] with G = Psi^T Psi, so step t reads */
                               /* one row of G (M floats) instead of Psi (N M), and   */
                               /* every R-th step recomputes c = Psi^T r directly to  */
                               /* bound the drift of the recurrence.  The plan builds */
                               /* G (M x M FP32, 4 M^2 bytes) on the first such       */
                               /* decode.  R = 1 gives the direct decode's bits.      */
    MP_OPT_PLAIN_L2_KEEP_BYTES = 12, /* grid streaming: bytes of the dictionary (the   */
                               /* first atoms of every CTA's slice) loaded with an   */
                               /* evict-last L2 hint so they stay in L2 from one     */
                               /* iteration to the next; the rest streams evict-first */
    MP_OPT_BATCH_TILE_M = 13,  /* batched GEMM: signals per tile, 128 or 256 (two    */
                               /* 128-row MMAs sharing each staged atom slice;       */
                               /* taken while the batch has more 128-row tiles than  */
                               /* the GPU has SMs, 128 after); 0 = auto              */
    MP_OPT_BATCH_GRAM = 14,    /* batched decodes (either precision: Gram steps use  */
                               /* the FP32 atoms only) and served decodes (BF16      */
                               /* dictionaries) with                                 */
                               /* Gram-updated correlations; the value is the        */
                               /* refresh period R, a multiple of 16 (0 = off, the   */
                               /* default).  Not in the paper: each signal keeps its */
                               /* FP32 correlations c = Psi^T r, computed directly   */
                               /* from the FP32 atoms when it is admitted and again  */
                               /* every R of its own steps; a step takes the 8       */
                               /* largest |c|, rescores them in FP32 exactly as the  */
                               /* direct batched step does, commits the best, and    */
                               /* updates c_j -= c G[m][j] (G = Psi^T Psi, FP32,     */
                               /* M x M, built on first use).  A step reads one row  */
                               /* of G per signal and no GEMM runs.  Whenever the    */
                               /* FP32 argmax is among the 8 candidates the result   */
                               /* equals the plain FP32 decode's bit for bit.        */
    MP_OPT_BATCH_PAIR = 15,    /* batched GEMM on two-SM tiles: a cluster of two     */
                               /* CTAs takes 256 signals x TILE_N atoms with M = 256 */
                               /* MMAs (tcgen05 cta_group::2), each SM holding a     */
                               /* 128 x TILE_N accumulator twice so the top-8 of one */
                               /* tile runs under the MMAs of the next.  0 = the     */
                               /* autotuner decides (default), 1 = off, 2 = on.  The */
                               /* candidates (and so the results) do not depend on   */
                               /* the tile shape.                                    */
    MP_OPT_BATCH_GRAM_BELOW = 16 /* mp_recover_batched with MP_OPT_BATCH_GRAM = R > 0: */
                               /* a threshold S >= 1 switches the decode from direct */
                               /* steps (BF16 tcgen05 GEMM + FP32 rescore) to        */
                               /* Gram-updated steps once at most S signals are      */
                               /* still active (0 = off, the default: every step is  */
                               /* a Gram step).  Not in the paper: a direct step     */
                               /* costs a GEMM whose time barely falls as the batch  */
                               /* drains (every tile reads the whole K extent of its */
                               /* atoms and signals), a Gram step one row of G per   */
                               /* active signal.  At the switch the correlations of  */
                               /* every active signal are computed directly from the */
                               /* FP32 atoms; after it they are refreshed every R of */
                               /* the signal's own steps.  The switch comes between  */
                               /* graph replays (16 steps), the first replay after   */
                               /* the count is seen at or below S; a batch of at     */
                               /* most S signals starts with Gram steps.  Selections */
                               /* are the FP32 rescore's in both kinds of step, so   */
                               /* whenever the FP32 argmax is among the 8 candidates */
                               /* the result equals the direct decode's bit for bit. */
                               /* The server ignores this option.                    */
} mp_option;

/* Read-only plan properties for mp_plan_query. */
typedef enum {
    MP_Q_PLAIN_MODE = 1,       /* mode the next mp_recover will use (1, 2 or 3; 4 =  */
                               /* grid with Gram-updated correlations)               */
    MP_Q_PLAIN_CTAS = 2,       /* CTAs it will launch                                */
    MP_Q_PLAIN_THREADS = 3,    /* threads per CTA                                    */
    MP_Q_PLAIN_SMEM = 4,       /* dynamic shared memory per CTA, bytes               */
    MP_Q_PLAIN_STAGE_ATOMS = 5,/* streaming mode: atoms per ring stage               */
    MP_Q_PLAIN_STAGES = 6,     /* streaming mode: ring depth                         */
    MP_Q_LD_FP32 = 7,          /* padded row length of the FP32 atom copy, floats    */
    MP_Q_DEVICE_BYTES = 8,     /* device memory owned by the plan, bytes             */
    MP_Q_KERNEL_LAUNCHES = 9,  /* kernels this library launched for the plan so far  */
    MP_Q_BATCH_TILE_N = 10,    /* atoms per GEMM tile of the current batch state     */
                               /* (11: no longer used)                               */
    MP_Q_PLAIN64_MODE = 12,    /* mode the next mp_recover_f64 will use (0: none)    */
    MP_Q_PLAIN64_STAGES = 13,  /* its streaming ring depth                           */
    MP_Q_GRAM_BYTES = 14,      /* device bytes of the Gram matrix (0 until built)     */
    MP_Q_PLAN_N = 15,          /* N of the plan                                      */
    MP_Q_PLAN_M = 16,          /* M of the plan                                      */
    MP_Q_BATCH_TILE_M = 17,    /* signals per GEMM tile of the current batch state   */
    MP_Q_PLAIN64_PIECES = 18,  /* FP64 streaming with the 4 warps sharing every      */
                               /* stage: ring stages per atom (an atom streams as    */
                               /* that many pieces); 0 when warps own whole atoms    */
    MP_Q_BATCH_GRAM = 19,      /* Gram period of the current batch state (0: off)    */
    MP_Q_BATCH_PAIR = 20,      /* 1 if the current batch state uses two-SM tiles     */
    MP_Q_BATCH_GRAM_BELOW = 21 /* switch threshold of the current batch state (0:   */
                               /* no switch)                                          */
} mp_query;

/* ------------------------------------------------------------------ */
/* Errors                                                              */
/* ------------------------------------------------------------------ */

/* Static string naming a status code.  Never NULL. */
MPGB_API const char* mp_status_string(mp_status s);

/* Reason for the most recent failure on the calling thread ("" if none).
 * The pointer stays valid until the thread's next mpgb call. */
MPGB_API const char* mp_last_error_message(void);

/* ------------------------------------------------------------------ */
/* Plans (Sec. 2: the dictionary shared by encoder and decoder)        */
/* ------------------------------------------------------------------ */

/* Create a plan for one dictionary.
 *  out    : receives the plan handle (set to NULL on failure).
 *  desc   : sizes, layout of `psi`, copies to build, normalisation policy.
 *  psi    : device pointer to N*M floats in desc->layout; it is copied, the
 *           caller keeps ownership and may free it after return.
 *  stream : stream on which the copy and checks run; the call synchronises
 *           it before returning.
 * The plan owns an FP32 atom-major copy padded to a multiple of 32 floats
 * per atom, plus the BF16 copy and/or the FP8-E4M3 copy with per-atom FP32
 * scale max|psi_m|/448 that prec_mask asks for.
 * Errors: MP_ERR_INVALID (sizes, layout, reserved field, non-unit atom
 * without normalize, zero atom with normalize), MP_ERR_NONFINITE (a
 * non-finite entry), MP_ERR_NOMEM, MP_ERR_CUDA. */
MPGB_API mp_status mp_plan_create(mp_plan_t* out, const mp_plan_desc* desc, const float* psi,
                         void* stream);

/* Create a plan from an FP64 dictionary (the paper's double-precision runs
 * draw Psi in FP64, Eq. 13).  Same contract as mp_plan_create, with psi a
 * device pointer to N*M doubles.  prec_mask must include MP_PREC_FP64; the
 * FP64 copy holds the input atoms (scaled to unit norm in FP64 when
 * desc->normalize), and the FP32 copy (always built) and any BF16/FP8 copy
 * are those atoms rounded to FP32 first.  The norm check of Eq. 4 runs on
 * the FP64 atoms.  A plan created by mp_plan_create with MP_PREC_FP64 in
 * prec_mask instead widens its FP32 atoms exactly, so both decodes read the
 * same dictionary. */
MPGB_API mp_status mp_plan_create_f64(mp_plan_t* out, const mp_plan_desc* desc, const double* psi,
                             void* stream);

/* Release a plan and everything it owns (synchronises the device first).
 * NULL is accepted and ignored. */
MPGB_API mp_status mp_plan_destroy(mp_plan_t plan);

/* Set an mp_option.  MP_ERR_INVALID for an unknown option or value. */
MPGB_API mp_status mp_plan_set_option(mp_plan_t plan, int option, long long value);

/* Read an mp_query value into *value.  MP_ERR_INVALID if unknown. */
MPGB_API mp_status mp_plan_query(mp_plan_t plan, int what, long long* value);

/* ------------------------------------------------------------------ */
/* Single-signal decode, FP32 (Sec. 3, Eqs. 8-12)                      */
/* ------------------------------------------------------------------ */

/* Decode one signal with the persistent FP32 kernel: correlations, the
 * argmax, the x~ and r updates and the FP64 stop test all run in one
 * launch with no host round-trip per iteration.
 *  y        : device pointer, N floats (read only).
 *  x        : device pointer, M floats; overwritten with x~ (zeroed first).
 *  stop     : eps and T.
 *  trace    : optional per-step record (NULL for none).
 *  host_out : if non-NULL, the call synchronises `stream` and fills it;
 *             the return value then reflects device-side errors too
 *             (MP_ERR_TIMEOUT, MP_ERR_NONFINITE for non-finite y).
 *             If NULL the call returns after enqueueing; fetch the result
 *             later with mp_plan_last_result.
 * Errors: MP_ERR_INVALID (NULL pointers, eps < 0, T < 0),
 * MP_ERR_UNSUPPORTED (N too large for the on-chip residual), MP_ERR_CUDA. */
MPGB_API mp_status mp_recover(mp_plan_t plan, const float* y, float* x, const mp_stop* stop,
                     const mp_trace* trace, mp_result* host_out, void* stream);

/* Orthogonal Matching Pursuit, the method Sec. 5 names as the next one to
 * port: MP's selection (Eq. 9, ties to the smallest index), then x~ on the
 * selected set S is the least-squares fit argmin ||y - Psi_S z|| and
 * r = y - Psi_S x~_S (replacing Eqs. 10-11).  One persistent FP32 launch on
 * the grid shapes (modes 5 and 6 of mp_plan_query's numbering): each step
 * streams the dictionary for the correlations, orthonormalises the new atom
 * against the selected ones (classical Gram-Schmidt applied twice, FP32,
 * norms in FP64), and updates r by its projection on the new direction;
 * after the loop x~_S solves R x = Q^T y by back substitution on the device.
 * Stops as mp_recover, plus MP_STOP_RANK when the new atom's component
 * orthogonal to the selected span is below 1e-4 (or N atoms are selected).
 *  y, x, stop, trace, host_out, stream : as mp_recover (trace coefs record
 *  <r, psi_m> at selection; x~ is written after the last step).
 * Scratch of about 4 (k N + k^2/2) bytes, k = min(T, N), is allocated on
 * first use and kept by the plan.  Errors: as mp_recover, plus MP_ERR_NOMEM
 * for the scratch and MP_ERR_UNSUPPORTED when MP_OPT_PLAIN_MODE forces the
 * one-cluster shape. */
MPGB_API mp_status mp_recover_omp(mp_plan_t plan, const float* y, float* x, const mp_stop* stop,
                         const mp_trace* trace, mp_result* host_out, void* stream);

/* Synchronise the stream of the plan's last mp_recover and return its
 * result (and its device-side status as the return value). */
MPGB_API mp_status mp_plan_last_result(mp_plan_t plan, mp_result* out);

/* The same decode entirely in FP64 (Sec. 3, Eqs. 8-12 in double precision,
 * the precision of the paper's reference CPU code): FP64 atoms, residual,
 * correlations, argmax (ties to the smallest index, compared on all 64 bits
 * of |c|) and x~.  Launch shapes as for mp_recover with 8-byte elements.
 *  y : device pointer, N doubles.  x : device pointer, M doubles.
 *  trace, host_out, stream : as for mp_recover (mp_trace_f64 records FP64
 *  coefficients and residual).
 * Errors: as mp_recover, plus MP_ERR_UNSUPPORTED when the plan holds no
 * FP64 copy (prec_mask without MP_PREC_FP64). */
MPGB_API mp_status mp_recover_f64(mp_plan_t plan, const double* y, double* x, const mp_stop* stop,
                         const mp_trace_f64* trace, mp_result* host_out, void* stream);

/* mp_recover with HOST buffers: copies y to the device, decodes, copies x~
 * back, and fills *out.  Blocking.  y_host: N floats; x_host: M floats.
 * Uses plan-owned device and pinned staging buffers. */
MPGB_API mp_status mp_recover_host(mp_plan_t plan, const float* y_host, float* x_host,
                          const mp_stop* stop, mp_result* out);

/* ------------------------------------------------------------------ */
/* Batched decode of B signals sharing the plan's dictionary           */
/* ------------------------------------------------------------------ */

/* Decode B independent signals.  Each step computes the correlations of
 * every still-active signal as one GEMM C = R Psi (tcgen05, BF16 or FP8
 * operands, FP32 accumulation) that keeps only the top-8 |c| per signal,
 * rescores those 8 atoms in FP32 from the FP32 atoms and commits the best
 * (ties to the smallest index), updates x~ and r in FP32 and evaluates the
 * FP64 stop test per signal.  Signals stop independently; finished ones
 * leave the GEMM.
 *  prec     : MP_PREC_BF16 or MP_PREC_FP8E4M3 (the plan must hold that
 *             copy) or MP_PREC_FP32 (runs mp_recover per signal).
 *  Y        : device pointer, B x N floats, row b is y_b.
 *  X        : device pointer, B x M floats, row b receives x~_b.
 *  stops    : n_stops entries, 1 (shared) or B (per signal).
 *  trace    : optional; atoms, coefs and energies each hold B rows of
 *             `capacity` entries (row b records signal b's steps);
 *             `residual`, when set, holds B rows of N floats and row b
 *             receives signal b's final FP32 residual.
 *  host_out : B results (required); the call synchronises `stream`.
 * The plan keeps the batch state (residuals, quantised GEMM operand, slot
 * table, candidate buffer) between calls and grows it to the largest B.
 * Errors: MP_ERR_INVALID, MP_ERR_UNSUPPORTED (precision not built),
 * MP_ERR_NOMEM, MP_ERR_CUDA, MP_ERR_TIMEOUT, MP_ERR_NONFINITE (a signal). */
MPGB_API mp_status mp_recover_batched(mp_plan_t plan, int prec, const float* Y, float* X, int B,
                             const mp_stop* stops, int n_stops, const mp_trace* trace,
                             mp_result* host_out, void* stream);

/* Autotuner of the batched correlation GEMM: times each tile shape (128 or
 * 256 signals per tile; 128, 224 or 256 atoms per tile) on B synthetic rows
 * and on B/4 (a batch drains as its signals stop) at precision `prec`, keeps
 * the fastest sum for B's size bucket (the next power
 * of two, at least 128) and returns it.  With the default
 * MP_OPT_BATCH_AUTOTUNE = 1, mp_recover_batched runs the same timing on its
 * own first batch of a new bucket.  Options MP_OPT_BATCH_TILE_N /
 * MP_OPT_BATCH_TILE_M, when set, override the result.  Synchronises the
 * legacy default stream.  tile_n, tile_m: may be NULL. */
MPGB_API mp_status mp_plan_autotune(mp_plan_t plan, int prec, int B, int* tile_n, int* tile_m);
/* The same, also timing two-SM tiles (MP_OPT_BATCH_PAIR) for B > 128 unless
 * that option is 1; *pair (may be NULL) receives 1 if the chosen shape is a
 * two-SM tile (tile_m is then 256). */
MPGB_API mp_status mp_plan_autotune_shape(mp_plan_t plan, int prec, int B, int* tile_n, int* tile_m, int* pair);

/* Diagnostic: the tensor-core correlations of the batched path, written out
 * in full.  R (device, B x N floats) is quantised as the batched step does
 * (BF16, or E4M3 with per-row scale max|r|/448) and C (device, B x M floats)
 * receives the FP32-accumulated correlations of R with the plan's BF16 or
 * FP8 atoms, rescaled by the FP8 per-atom and per-row scales.  Synchronises
 * `stream`.  For tests of the GEMM; the decode paths never write C. */
MPGB_API mp_status mp_debug_correlations(mp_plan_t plan, int prec, const float* R, int B, float* C,
                                void* stream);

/* Diagnostic: device time of the batched correlation GEMM (GEMM + top-8
 * epilogue, one launch per step) on B synthetic rows at precision `prec`:
 * the autotuner's timing routine, mean of `reps` launches after 2 warm-up
 * launches, written to *us in microseconds per launch.  Tile shape
 * (tile_m signals x tile_n atoms): tile_m 128 or 256, tile_n 128..256 in steps of 32; both 0 = the shape
 * mp_recover_batched would use for B signals (options, else autotuned).
 * Allocates its own buffers; synchronises the legacy default stream.
 * Errors: MP_ERR_INVALID (bad shape or argument), MP_ERR_UNSUPPORTED
 * (precision not built), MP_ERR_CUDA. */
MPGB_API mp_status mp_debug_time_gemm(mp_plan_t plan, int prec, int B, int tile_m, int tile_n, int reps,
                                      double* us);
/* The same with pair = 1 for a two-SM tile (tile_m 256, tile_n 128..256 in
 * steps of 32); pair = 0 is mp_debug_time_gemm. */
MPGB_API mp_status mp_debug_time_gemm_pair(mp_plan_t plan, int prec, int B, int tile_m, int tile_n, int pair,
                                           int reps, double* us);

/* ------------------------------------------------------------------ */
/* One decode with the atoms split across ranks (one GPU each)         */
/* ------------------------------------------------------------------ */

/* Each rank's plan holds a contiguous shard of Psi: global atoms
 * [atom_offset, atom_offset + M) (its desc->M), all ranks the same N.  Per
 * MP iteration (Sec. 3, Eqs. 9-12) a rank computes its shard's best
 * candidate as a record (mp_shard_step_local), the caller all-gathers the
 * records of all ranks (one exchange of mp_shard_record_bytes per rank, e.g.
 * NCCL all-gather), and every rank applies the step (mp_shard_step_apply):
 * the largest |c| wins, ties to the smallest global atom index (Sec. 4);
 * every rank updates its copy of r with the winner's atom row carried in
 * the record, the FP64 energy and the stop test; the owning rank adds c to
 * its x~ slice (Eq. 10).  All ranks apply identical arithmetic, so their r
 * copies and states stay bit-identical.  The correlation and energy orders
 * are the persistent kernel's: with one rank (or with the records of
 * several shards of one dictionary gathered by hand) the atoms, x~ and
 * energies equal mp_recover's bit for bit.  The calls are stream-ordered
 * and never synchronise; once the state says stopped, apply is a no-op, so
 * the caller may check `stopped` every few iterations. */
typedef struct {
    double e0;                 /* ||y||^2                                         */
    double e;                  /* ||r||^2 after the last step (FP64)              */
    double thr2;               /* eps^2 e0                                        */
    double audit;              /* max |e_k - (e_{k-1} - c_k^2)| / e0              */
    int t;                     /* completed steps                                 */
    int T;                     /* cap                                             */
    int stopped;               /* nonzero once the loop test of Eq. 8 fails       */
    int stop_reason;           /* mp_stop_reason                                  */
    int status;                /* mp_status (MP_ERR_NONFINITE for non-finite y)   */
    int reserved;
} mp_shard_state;

/* Bytes of one rank's record: a 16-byte head (key, global atom, c) followed
 * by the atom's FP32 row (ld floats, the plan's MP_Q_LD_FP32). 0 for NULL. */
MPGB_API size_t mp_shard_record_bytes(mp_plan_t plan);

/* r <- y (device, N floats; r has room for MP_Q_LD_FP32 floats), x~ slice
 * (device, M floats) <- 0, and the state (device) for eps, T.
 * Errors: MP_ERR_INVALID (NULL, bad stop), MP_ERR_CUDA. */
MPGB_API mp_status mp_shard_init(mp_plan_t plan, const float* y, float* r, float* x, const mp_stop* stop,
                        mp_shard_state* state, void* stream);

/* This rank's candidate for the current r: correlations of its shard,
 * the best packed key, and the winner's row, written to `record` (device,
 * mp_shard_record_bytes, 16-byte aligned).  atom_offset: global index of the
 * shard's first atom.  Errors: MP_ERR_INVALID, MP_ERR_CUDA. */
MPGB_API mp_status mp_shard_step_local(mp_plan_t plan, int atom_offset, const float* r, void* record,
                              void* stream);

/* Apply one step from the n_records gathered records (device, contiguous,
 * mp_shard_record_bytes each): update r, x~ (owner only), state, and the
 * optional trace (atoms, coefs by step; energies and residual unused).
 * Errors: MP_ERR_INVALID, MP_ERR_CUDA. */
MPGB_API mp_status mp_shard_step_apply(mp_plan_t plan, int atom_offset, const void* records, int n_records,
                              float* r, float* x, mp_shard_state* state, const mp_trace* trace,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPGB_H */
