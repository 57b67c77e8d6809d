/*
 * madmap.h -- C ABI of libmadmap, a GB300 (sm_103a) library for the
 * maximum-likelihood map-making solve of MADmap (Cantalupo et al.,
 * arXiv:0906.1775).
 *
 * The library solves  H m = b,  H = A^T N^-1 A,  b = A^T N^-1 d
 * (Section 4, Eq. 10; the maximum-likelihood map of Section 3, Eq. 8) with
 * preconditioned conjugate gradients, where
 *   A     is the sparse pointing matrix: one unit weight per sample for
 *         temperature (Section 3, Eq. 3), or the weights (1, cos 2psi, sin 2psi)
 *         on (I, Q, U) for polarisation (Section 3, Eq. 4, relabelled as
 *         (I, Q, U) = (i/2, u/2, q/2) of the paper's Stokes vector);
 *   N^-1  is block diagonal with one banded symmetric Toeplitz block per
 *         stationary interval, N^-1_{t,t'} = f(|t-t'|) for |t-t'| < n_c
 *         (Section 5.2, Eq. 15), applied by FFT convolution of circulant
 *         embeddings over overlapping windows (Section 5.2, Eqs. 16-22).
 *
 * Conventions (all entry points):
 *   - Every call returns a madmap_status; nothing aborts or exits.  On an
 *     error, madmap_last_error() returns a message (thread local).
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are ordinary host memory, read during the call only.
 *   - Calls that take a cudaStream_t (passed as void*, NULL = legacy default
 *     stream) are ordered on that stream and may return before the GPU work
 *     finishes, except where stated.
 *   - A plan keeps the caller's pix/psi device pointers by reference only
 *     during madmap_plan_create (it copies what it needs into derived buffers
 *     it owns); after creation the caller may free them.
 *   - Maps exchanged with the caller are laid out [n_rhs][n_obs][n_stokes]
 *     over the plan's observed pixels (ascending global index, Section 5.4).
 *   - A plan is not thread safe: calls on one plan must be serialised.
 */
#ifndef MADMAP_H_
#define MADMAP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct madmap_plan_s* madmap_plan_t;

/* autotuner candidates reported in madmap_plan_stats */
#define MADMAP_MAX_TUNED 12

typedef enum {
  MADMAP_OK = 0,
  MADMAP_WARN_MAXITER = 1,      /* result valid: lowest-residual iterate returned */
  MADMAP_STOPPED = 2,           /* result valid: a checkpoint callback stopped the solve */
  MADMAP_ERR_INVALID_ARG = -1,  /* bad sizes, pointers, indices, offsets or filters */
  MADMAP_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  MADMAP_ERR_OOM = -3,          /* device allocation failed (or was injected to fail) */
  MADMAP_ERR_NOT_PD = -4,       /* a filter's Toeplitz symbol is not positive, or p^T H p <= 0 */
  MADMAP_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
  MADMAP_ERR_INTERNAL = -6
} madmap_status;

/* Sums `count` elements of a device buffer, in place, over all ranks of a
 * sharded solve (see madmap_plan_desc.allreduce).  dtype: MADMAP_REDUCE_F64
 * (double), MADMAP_REDUCE_F32 (float) or MADMAP_REDUCE_I32 (int32).  The
 * library calls it on the host, from the thread that made the library call,
 * with work on `stream` (a cudaStream_t) producing the buffer; the sum must be
 * complete, or ordered on `stream`, before the callback returns.  Every rank
 * makes the same calls in the same order.  Returns 0 on success; any other
 * value makes the library call fail with MADMAP_ERR_INTERNAL. */
typedef int32_t (*madmap_reduce_fn)(void* buf, int64_t count, int32_t dtype, void* stream, void* user);
enum { MADMAP_REDUCE_F64 = 0, MADMAP_REDUCE_F32 = 1, MADMAP_REDUCE_I32 = 2 };

typedef enum {
  MADMAP_FP64 = 0,   /* operator, vectors and scalars in float64 */
  MADMAP_MIXED = 1,  /* float32 operator and vectors inside float64 iterative refinement */
  MADMAP_FP32 = 2,   /* float32 operator (madmap_apply_ATNA / madmap_apply_ninv / madmap_rhs only) */
  MADMAP_DF64 = 3    /* double-float operator: every product and sum on pairs of float32 numbers
                        (about 48 significant bits), float64 maps in and out.  Accepted by
                        madmap_apply_ATNA, madmap_rhs and madmap_time_operator, and as
                        madmap_solve_opts.refine_precision.  Not in the paper: GB300 runs float32
                        arithmetic many times faster than float64. */
} madmap_precision;

/* Description of the data a plan is built over.  Section 3 (data model),
 * Section 5.2 (stationary intervals and filters), Section 5.4 (indexing). */
typedef struct {
  int32_t n_stokes;                 /* 1 (T) or 3 (IQU) */
  int64_t n_samples;                /* n_t, all detectors concatenated; 0 allowed (empty plan) */
  int32_t n_pix;                    /* global pixel count n_z (> 0) */
  const int32_t* pix;               /* device [n_samples]: global pixel of each sample,
                                       -1 = flagged sample (zero row of A, Section 4 gap filling);
                                       any other value outside [0, n_pix) is INVALID_ARG */
  const float* psi;                 /* device [n_samples]: polarisation angle in radians;
                                       must be NULL when n_stokes == 1 and non-NULL when 3 */
  int32_t n_intervals;              /* stationary intervals (Toeplitz blocks of N^-1), >= 0 */
  const int64_t* interval_offsets;  /* host [n_intervals + 1]: non-decreasing, [0] = 0,
                                       [n_intervals] = n_samples; interval i = [off[i], off[i+1]) */
  const int32_t* interval_filter;   /* host [n_intervals]: filter index of each interval */
  int32_t n_filters;                /* >= 1 */
  int32_t n_lags;                   /* n_c >= 1: lags tau = 0 .. n_c-1 of Eq. 15 */
  const double* filter_lags;        /* host [n_filters][n_lags]: f(tau) of each filter; each
                                       filter's Toeplitz symbol must be > 0 (else NOT_PD) */
  double rcond_excise;              /* IQU: excise pixels with hits < 3 or
                                       rcond(A^T A block) < this (<= 0: default 1e-6) */
  double rcond_fp64;                /* IQU: keep float64 preconditioner blocks for pixels with
                                       rcond below this in MIXED solves (<= 0: default 1e-2) */
  int32_t fft_len;                  /* complex FFT length M per window (power of two in
                                       [256, 2^20], > 2 (n_lags-1)); 0 = chosen by the plan */
  int32_t tiles_per_chunk;          /* windows pairs per operator launch chunk; 0 = chosen */
  /* Multi-resolution maps (Section 6): Q and U on their own pixelisation.
   * IQU only; NULL (default) puts all three Stokes parameters on pix. */
  const int32_t* pix_pol;           /* device [n_samples]: Q/U pixel of each sample in [0, n_pix_pol),
                                       or -1 (flagged: the sample's row is zero) */
  int32_t n_pix_pol;                /* global Q/U pixel count (> 0 when pix_pol is set) */
  /* Pointing expanded on the fly from compressed boresight pointing
   * (Section 5.3).  When boresight is set, pix, psi and pix_pol must be NULL,
   * and the plan stores no per-sample pointing: every pass over the samples
   * (the operator's gather and scatter, the preconditioner, the backward pass)
   * recomputes each sample's pixel and weights.  Sample t = d * n_per_det + j
   * of detector d (n_per_det = n_samples / n_det): with u = j / bore_step and
   * f = (j mod bore_step) / bore_step, each node quantity q is interpolated as
   * q_u + f (q_{u+1} - q_u); the detector sits at X = x + (c dx - s dy),
   * Y = y + (s dx + c dy) and observes pixel floor(Y) * grid_width + floor(X)
   * when 0 <= X < grid_width and 0 <= Y < grid_height (else the sample is
   * flagged).  IQU weights: (C, S) = (c cd - s sd, s cd + c sd), n = C^2 + S^2,
   * cos 2psi = (C^2 - S^2) / n, sin 2psi = 2 C S / n; n = 0 flags the sample.
   * Every step is one float32 operation rounded to nearest, in this order
   * (no contraction), so pixel decisions are reproducible bit for bit. */
  const float* boresight;           /* device [n_bore][4]: node u = detector sample u * bore_step:
                                       x, y (pixel units of the grid), cos and sin of the
                                       boresight orientation; finite */
  int32_t n_bore;                   /* >= (n_per_det - 1) / bore_step + 2 */
  int32_t bore_step;                /* detector samples per node interval, >= 1 */
  const float* det_pointing;        /* host [n_det][4]: dx, dy (focal-plane offset, pixel units),
                                       cos and sin of the polariser orientation; finite */
  int32_t n_det;                    /* detectors (>= 1; must divide n_samples); no interval
                                       may span two detectors */
  int32_t grid_width, grid_height;  /* flat pixel grid; n_pix must equal their product */
  /* Extended pointing (Section 6, Eqs. 39-40): extra unknowns o with A -> [A B],
   * B one unit entry per sample, for destriping offsets (with a white-noise
   * filter of one lag) or binned synchronous templates.  Stored pointing
   * only (pix_pol and boresight NULL).  Maps then have the observed sky
   * pixels' rows followed by one row per extra column with its
   * amplitude in column 0 (other columns 0).  A sample that is flagged or
   * whose sky pixel is excised has a zero row in both blocks; an extra
   * column without samples is excised; its preconditioner block is
   * 1 / (B^T W^-1 B).  The caller keeps the system non-singular (offsets on
   * every sample are degenerate with a constant I map: leave one baseline
   * without a column). */
  const int32_t* extra_index;       /* device [n_samples]: extra column of each sample in
                                       [0, n_extra), or -1 (none); NULL: no extra columns */
  int32_t n_extra;                  /* extra columns (>= 1 when extra_index is set) */
  /* Parametric half-wave-plate signal (Section 6, Eqs. 41-42), with or without
   * extra_index, stored single-resolution pointing only: 32 unknowns per group
   * of intervals, b_1..b_32 with the sample's columns cos k w, tau cos k w,
   * sin k w, tau sin k w (k = 1..8, in that order), w = hwp_angle, tau =
   * hwp_tau.  Their rows follow the extra columns' rows (32 per group, the
   * parameter in column 0).  Each parameter's preconditioner block is
   * 1 / sum_t f(0) C_{t,i}^2; a parameter with a zero sum is excised. */
  const float* hwp_angle;           /* device [n_samples]: polariser angle w (radians); NULL: none */
  const float* hwp_tau;             /* device [n_samples]: the model's time variable (caller's units) */
  const int32_t* interval_hwp_group;/* host [n_intervals]: group of each interval in [0, n_hwp_groups)
                                       or -1 (no half-wave-plate term) */
  int32_t n_hwp_groups;             /* >= 1 when hwp_angle is set */
  /* Sharded solves over several processes, one GPU each (Section 5.1: each
   * process holds a share of the time-ordered data made of whole stationary
   * intervals, balanced by sample count, see madmap_partition_intervals;
   * Section 5.5: the map-domain sum across processes once per operator
   * application, the role of MM_SomeReduce).  With allreduce set, this plan
   * holds one rank's samples and intervals; the observed-pixel set, the hit
   * counts and the preconditioner blocks are summed across ranks at
   * plan_create (so every rank has the same map rows and excisions), and every
   * map that madmap_apply_ATNA, madmap_rhs, the solves and the backward pass
   * produce (H x, b, the refinement residuals, grad_lags) is summed across ranks
   * before it is used.  The PCG vector work and dot products then run
   * redundantly on the identical maps of every rank, so the ranks take the
   * same decisions with no further exchange.  Every rank must make the same
   * calls on its plan in the same order.  Stored single-resolution pointing
   * only; solves run with direct launches (use_graph is treated as 0).
   * NULL: an ordinary single-process plan. */
  madmap_reduce_fn allreduce;
  void* allreduce_user;             /* passed to allreduce */
  /* Bit-reproducible maps (the paper fixes no summation order): nonzero makes
   * every map-domain sum of the operator (A^T w in madmap_apply_ATNA,
   * madmap_rhs and every solve) a sum over each observed pixel's samples in
   * ascending sample order, instead of floating-point atomics whose order
   * varies run to run, so repeated calls on this plan give identical bits.
   * The operator writes its weighted timestream (n_samples values per
   * right-hand side, kept by the plan) and a second pass sums each pixel's
   * samples.  Stored single-resolution pointing without extended pointing;
   * n_samples < 2^31.  The preconditioner blocks are still summed with atomics
   * at plan creation (plans built twice may differ in their last bits). */
  int32_t deterministic;
  /* Measuring autotuner (the paper picks n_f by its cost model, Section 5.2;
   * on a GPU the fastest FFT length and launch batching depend on the
   * kernels): nonzero times one float32 operator application, with CUDA events
   * after one warm-up application, for each candidate FFT length (fft_len if
   * given, else the plan's cost-model choice and the lengths twice and half
   * it) and tiles per launch chunk (tiles_per_chunk if given, else the default
   * rule and half and twice it), and keeps the fastest.  The candidates and
   * their times are in madmap_plan_stats.  Adds a few operator applications
   * to plan creation; ignored for white-noise plans. */
  int32_t autotune;
  /* Scatter of the float32 operator (stored T or IQU pointing, one
   * pixelisation, atomic map sums, FFT lengths 2^13 .. 2^20): lanes holding
   * consecutive samples that hit one pixel add their sum with one atomic per
   * run instead of one per sample.  0 (default): on when at least a quarter
   * of the samples repeat their predecessor's pixel, or as the autotuner
   * measures; 1: on; -1: off.  The two differ only in the order of the
   * rounded additions.  Must be -1, 0 or 1. */
  int32_t scatter_runs;
  /* Split of the FFT length into column and row transforms (the four-step
   * FFT, M = N1 N2): 0 (default) N2 = 2^ceil(log2(M) / 2), or as the
   * autotuner measures; 1: columns half as long, rows twice (N1 at most
   * 1024).  Any split gives the same product up to rounding.  Must be 0 or 1. */
  int32_t fft_split;
} madmap_plan_desc;

typedef struct {
  int32_t n_obs;           /* map rows: observed pixels (slots for multi-resolution plans; plus the
                              extra and half-wave-plate rows of extended pointing) */
  int32_t n_excised;       /* observed pixels excised (IQU, Section 4) */
  int32_t n_fp64_pixels;   /* pixels keeping float64 preconditioner blocks */
  int32_t n_stokes;
  int32_t fft_len;         /* M */
  int32_t n1, n2;          /* M = n1 * n2 (four-step factorisation) */
  int32_t n_segments;      /* overlap-save windows over all intervals */
  int32_t n_tiles;         /* window pairs (two real windows per complex FFT) */
  int32_t tiles_per_chunk;
  int32_t n_lags;
  int32_t n_filters;
  int64_t n_samples;
  int64_t device_bytes;    /* device memory owned by the plan */
  int32_t n_obs_pol;       /* multi-resolution plans: observed Q/U pixels (else 0) */
  int32_t n_excised_pol;   /* multi-resolution plans: excised Q/U pixels */
  int32_t n_extra;         /* extended pointing: extra columns (rows n_obs - n_extra .. n_obs - 1 of
                              the map), else 0 */
  int32_t n_excised_extra; /* extended pointing: extra columns without samples */
  int32_t n_hwp_params;    /* half-wave-plate parameters (32 per group; the last rows of the map) */
  int32_t n_excised_hwp;   /* half-wave-plate parameters without weight */
  int32_t n_map_replicas;  /* copies of the map the operator scatters into (8 for small maps under
                              more than 1024 samples per row, else 1) */
  int32_t deterministic;   /* 1 when map sums run in a fixed order (madmap_plan_desc.deterministic) */
  int32_t sharded;         /* 1 for a sharded plan (madmap_plan_desc.allreduce set) */
  int32_t n_tuned;         /* candidates the autotuner timed (0: not tuned), at most MADMAP_MAX_TUNED reported */
  int32_t tuned_fft_len[MADMAP_MAX_TUNED];
  int32_t tuned_tiles_per_chunk[MADMAP_MAX_TUNED];
  float tuned_ms[MADMAP_MAX_TUNED];       /* float32 operator application time of each candidate */
  int32_t tuned_runs[MADMAP_MAX_TUNED];   /* 1 when the candidate summed runs of one pixel before its atomics */
  int32_t tuned_n2[MADMAP_MAX_TUNED];     /* the candidate's column transform length N2 (fft_len = n1 n2) */
  int32_t scatter_runs;    /* 1 when the operator's scatter adds each run of consecutive samples in
                              one pixel with one atomic (madmap_plan_desc.scatter_runs), else 0 */
  double repeat_frac;      /* fraction of samples whose successor hits the same observed pixel */
} madmap_plan_stats;

typedef struct {
  int32_t max_iter;        /* PCG iterations (mixed: total inner iterations); default 50 (Section 5) */
  double rel_tol;          /* stop at ||r_k|| / ||b|| <= rel_tol; default 1e-6 (Section 5) */
  int32_t precision;       /* madmap_precision: FP64 or MIXED */
  int32_t max_outer;       /* MIXED: refinement steps, default 10 */
  double inner_rel_tol;    /* MIXED: inner float32 PCG stops at this reduction of its residual,
                              default 1e-4 (and, with inner_restart = 0, not below rel_tol / 2) */
  int32_t use_graph;       /* 2 (default): one CUDA graph runs all iterations on the device (a
                              conditional WHILE node, capped at max_iter + 2 passes); 1: chunks of
                              iters_per_sync iterations replayed as graphs with host checks
                              between them; 0: direct launches with host checks */
  int32_t iters_per_sync;  /* iterations enqueued between host checks (modes 0 and 1), default 8 */
  int32_t refine_precision; /* MIXED: arithmetic of the right-hand side b = A^T N^-1 d and of the
                              refinement residuals b - H x: MADMAP_DF64 (default) or MADMAP_FP64.
                              Vectors, dot products and the refinement update stay float64. */
  /* Checkpoints (Section 5: the solver state is saved every 20 PCG iterations by
   * default, as five map vectors and six scalars, and a run can restart from any
   * of them).  FP64 solves of one right-hand side only. */
  int32_t checkpoint_every;              /* write the state every this many iterations; 0 (default): never */
  struct madmap_checkpoint_s* checkpoint; /* host: where the state is written (caller-owned buffers) */
  int32_t (*on_checkpoint)(const struct madmap_checkpoint_s* state, void* user);
                                         /* called after each checkpoint, may be NULL; a nonzero return
                                            stops the solve with MADMAP_STOPPED (m = best iterate so far) */
  void* checkpoint_user;                 /* passed to on_checkpoint */
  /* Residual history (Section 5 monitors the relative residual of every
   * iteration; the paper keeps no record of it).  Host [n_rhs][history_capacity]
   * or NULL.  Entry k is the relative residual ||r_k|| / ||b|| after PCG
   * iteration k (entry 0 = 1): FP64 the recursively updated residual; MIXED
   * the inner float32 PCG's recursive residual relative to ||b|| (continued
   * steps: at each refinement step's first entry the refined iterate's
   * residual that replaced it; restarted steps: scaled by the relative residual
   * of the float64 iterate the step started from), inner iterations of all
   * refinement steps in order.  The solve records at
   * most 4096 iterations; madmap_solve_info.history_len tells how many entries
   * were written.  A resumed solve writes NaN for the iterations done before
   * the checkpoint. */
  double* residual_history;
  int32_t history_capacity;
  /* MIXED (not in the paper): 0 (default) continues the inner float32 PCG
   * across refinement steps by residual replacement: the refined iterate's
   * residual replaces the recursive one, the correction restarts from zero and
   * the search direction is kept, so the Krylov progress of earlier steps is
   * not lost.  1: each refinement step solves H e = r from e = 0 (classic
   * iterative refinement). */
  int32_t inner_restart;
  /* MIXED, continued PCG: 0 (default) a step whose float32 recursive residual
   * reaches rel_tol, after a full-precision residual has replaced it at least
   * once, ends the solve without one more full-precision residual (the paper
   * stops on the recursively updated residual, Section 5; the replacement
   * bounds its drift); final_rel_res is then that recursive residual.  1:
   * every stop is confirmed by a full-precision residual. */
  int32_t final_residual;
} madmap_solve_opts;

/* Solver state at a checkpoint, independent of the launch configuration (a
 * different plan over the same pointing and filters can resume it).  The five
 * maps are host [n_obs][n_stokes] float64 arrays owned by the caller: the
 * iterate x, the residual r, the preconditioned residual z = P r, the next
 * search direction p, and the iterate with the lowest residual so far. */
typedef struct madmap_checkpoint_s {
  int32_t n_obs, n_stokes;   /* layout of the maps (checked on resume) */
  int32_t iters;             /* PCG iterations done */
  int32_t best_iter;         /* iteration of x_best */
  double rz;                 /* <r, z> */
  double bnorm;              /* ||b|| */
  double rel_res;            /* ||r|| / ||b|| */
  double best_rel_res;       /* relative residual of x_best */
  double *x, *r, *z, *p, *x_best;
} madmap_checkpoint;

typedef struct {
  int32_t status;          /* madmap_status of the solve */
  int32_t iters;           /* PCG iterations performed (sum of inner iterations for MIXED) */
  int32_t outer_iters;     /* MIXED inner steps, each ended by a refinement (FP64: 1) */
  int32_t best_iter;       /* iteration count at which the returned iterate was produced */
  int32_t fp64_applies;    /* full-precision operator applications (float64, or double-float per
                              refine_precision), including the right-hand side; MIXED solves of
                              single-resolution stored pointing form the right-hand side in float32
                              (it only starts the first inner solve; each refinement residual
                              b - H x is formed from the data as A^T N^-1 (d - A x) in full precision)
                              and count it in fp32_applies; a continued solve that stops on its
                              recursive residual (final_residual = 0) forms no residual for its
                              last step */
  int32_t fp32_applies;    /* float32 operator applications */
  double final_rel_res;    /* last relative residual ||b - H x_k|| / ||b|| (recursive for FP64, and
                              for a MIXED solve that stopped on its recursive residual) */
  double best_rel_res;     /* relative residual of the returned map */
  double t_rhs_ms;         /* right-hand side time */
  double t_solve_ms;       /* total call time (right-hand side included) */
  int32_t history_len;     /* entries written to madmap_solve_opts.residual_history */
  int32_t pad_;
  double t_pcg_ms;         /* host time spent in PCG iterations (MIXED: the inner float32 solves) */
  double t_refine_ms;      /* MIXED: host time of the refinement steps (x += e, b - H x, best iterate) */
} madmap_solve_info;

/* ------------------------------------------------------------------ plans */

/* Build a plan: observed-pixel compaction (Section 5.4), pixel classification
 * and preconditioner blocks (Sections 4-5), overlap-save windows, filter
 * spectra and work buffers.  Synchronises `stream` before returning.
 * out: receives the plan (NULL on error). */
madmap_status madmap_plan_create(const madmap_plan_desc* desc, void* stream, madmap_plan_t* out);

/* The concatenated data distribution of Section 5.1: the intervals, in
 * order, are cut into n_ranks contiguous runs of whole intervals whose sample
 * counts are as equal as the interval boundaries allow: rank r's run ends at
 * the boundary (an index j into interval_offsets) nearest to
 * (r + 1) n_samples / n_ranks, the lowest such j on ties, and never before the
 * previous rank's end.  interval_offsets: host
 * [n_intervals + 1] as in madmap_plan_desc; first_interval_out: host
 * [n_ranks + 1], rank r gets intervals [first[r], first[r + 1]).  Host only. */
madmap_status madmap_partition_intervals(int32_t n_intervals, const int64_t* interval_offsets, int32_t n_ranks,
                                         int32_t* first_interval_out);

/* Free all device memory of a plan.  NULL is accepted. */
madmap_status madmap_plan_destroy(madmap_plan_t plan);

madmap_status madmap_plan_get_stats(madmap_plan_t plan, madmap_plan_stats* out);

/* Observed pixels (Section 5.4).  *n_obs receives their count.  When
 * non-NULL, obs2glob (device int32 [n_obs], caller-owned) receives the global
 * index of each observed pixel in ascending order, and excised (device uint8
 * [n_obs]) receives 1 for pixels excised as poorly conditioned (Section 4; their
 * map value is 0).  Copies are ordered on `stream`.  Call with NULL buffers
 * first to learn n_obs. */
madmap_status madmap_plan_observed(madmap_plan_t plan, int32_t* n_obs, int32_t* obs2glob, uint8_t* excised,
                                   void* stream);

/* Multi-resolution plans (pix_pol set): maps are [n_slots][3] with n_slots =
 * madmap_plan_stats.n_obs = max(observed I pixels, observed Q/U pixels).
 * Column 0 of row k is I of observed I pixel k (madmap_plan_observed lists the
 * I pixels and their excision flags), columns 1-2 of row k are Q, U of
 * observed Q/U pixel k (listed here).  Entries past either count are 0.  The
 * preconditioner blocks are the 1 x 1 I blocks and 2 x 2 (Q, U) blocks of
 * A^T W^-1 A; a Q/U pixel with fewer than 2 hits or rcond of its 2 x 2 A^T A
 * block below rcond_excise is excised with the rows of its samples, and an I
 * pixel left without rows is excised too.  Arguments as madmap_plan_observed;
 * *n_obs_pol = 0 for single-resolution plans. */
madmap_status madmap_plan_observed_pol(madmap_plan_t plan, int32_t* n_obs_pol, int32_t* obs2glob_pol,
                                       uint8_t* excised_pol, void* stream);

/* Plans over compressed pointing (madmap_plan_desc.boresight): the expanded
 * pointing of every sample, as the operator computes it (Section 5.3).
 * pix: device int32 [n_samples], the global pixel or -1 (flagged); cos2psi,
 * sin2psi: device float [n_samples] (IQU; may be NULL; 0 at flagged samples).
 * Any output may be NULL.  INVALID_ARG for plans over stored pointing.
 * Asynchronous on `stream`. */
madmap_status madmap_plan_expand_pointing(madmap_plan_t plan, int32_t* pix, float* cos2psi, float* sin2psi,
                                          void* stream);

/* Replace the filter lags (host [n_filters][n_lags]) without re-planning:
 * recomputes spectra and preconditioner blocks.  Synchronises `stream`. */
madmap_status madmap_plan_set_filters(madmap_plan_t plan, const double* filter_lags, void* stream);

/* ------------------------------------------------------------------ operators */

/* y = H x = A^T N^-1 A x (Eq. 10) for n_rhs maps.  x, y: device
 * [n_rhs][n_obs][n_stokes], double for MADMAP_FP64, float for MADMAP_FP32.
 * y is overwritten.  n_rhs >= 1.  Excised pixels give 0. */
madmap_status madmap_apply_ATNA(madmap_plan_t plan, int32_t precision, int32_t n_rhs,
                                const void* x, void* y, void* stream);

/* b = A^T N^-1 d (Eq. 10), the right-hand side.  d: device float [n_rhs][n_samples];
 * b: device [n_rhs][n_obs][n_stokes] (double for FP64, float for FP32). */
madmap_status madmap_rhs(madmap_plan_t plan, int32_t precision, int32_t n_rhs, const float* d,
                         void* b, void* stream);

/* w = N^-1 y on timestreams (Section 5.2, Eq. 15), interval by interval.
 * y, w: device [n_rhs][n_samples], double for FP64, float for FP32. */
madmap_status madmap_apply_ninv(madmap_plan_t plan, int32_t precision, int32_t n_rhs,
                                const void* y, void* w, void* stream);

/* ------------------------------------------------------------------ solves */

void madmap_solve_opts_default(madmap_solve_opts* opts);

/* PCG solve of H m = A^T N^-1 d (Section 4, Eq. 10; Section 5: x_0 = 0,
 * stop at max_iter or relative residual rel_tol, return the iterate with the
 * lowest relative residual).  d: device float [n_samples]; m: device double
 * [n_obs][n_stokes].  opts/info may be NULL (defaults / not reported).
 * Synchronises `stream` before returning.  Returns MADMAP_WARN_MAXITER when
 * rel_tol was not reached (m is still the best iterate). */
madmap_status madmap_solve(madmap_plan_t plan, const float* d, double* m, const madmap_solve_opts* opts,
                           madmap_solve_info* info, void* stream);

/* Continue an FP64 PCG solve from a checkpoint written by madmap_solve (or a
 * previous resume) with the same pointing and filters: the iteration counts,
 * lowest-residual rule and stopping tests carry on from the saved state
 * (opts->rel_tol and opts->max_iter apply to the total), and further
 * checkpoints may be written.  The right-hand side is not needed.  m: device
 * double [n_obs][n_stokes], the best iterate.  state: host, read during the
 * call.  MADMAP_ERR_INVALID_ARG when the state's layout does not match the
 * plan or opts->precision is not FP64. */
madmap_status madmap_solve_resume(madmap_plan_t plan, const madmap_checkpoint* state, double* m,
                                  const madmap_solve_opts* opts, madmap_solve_info* info, void* stream);

/* ------------------------------------------------------------------ allocation-free weighting */

/* Size of the fixed device array used by madmap_apply_ninv_noalloc, and the
 * largest n_lags it accepts. */
#define MADMAP_NOALLOC_SCRATCH_BYTES (32u << 20)
#define MADMAP_NOALLOC_MAX_LAGS (1 << 15)

/* w = N^-1 y on timestreams, like madmap_apply_ninv, for callers that cannot
 * allocate device memory (an allocator that forbids new allocations after
 * start-up, a real-time loop that must not stall in cudaMalloc, or host code
 * without its own CUDA memory management).  There is no counterpart in the
 * paper: it is an interface convenience, not part of the method.
 *
 * No plan is needed and nothing is allocated: the derived tables and the FFT
 * intermediate live in a fixed device array of MADMAP_NOALLOC_SCRATCH_BYTES
 * that every GPU loading the library holds until the process exits.  The
 * caller passes the inputs and outputs: precision FP64 (y, w double) or FP32
 * (float); y, w: device [n_samples]; interval_offsets (host [n_intervals+1]),
 * interval_filter (host [n_intervals]) and filter_lags (host
 * [n_filters][n_lags]) as in madmap_plan_desc.  Sizes that do not fit the
 * array (n_lags > MADMAP_NOALLOC_MAX_LAGS, or too many filters or windows)
 * return MADMAP_ERR_INVALID_ARG with a message; a filter that is not positive
 * definite returns MADMAP_ERR_NOT_PD.
 *
 * The array is shared by all calls and keeps the last call's contents; calls
 * that overlap on the GPU race on it.  Every call looks up the array's device
 * address for the device that is current.  Ordered on `stream`.  The derived
 * tables are uploaded from host memory that lives only during the call: the
 * upload may hold the host until `stream` reaches it, and a call made while
 * `stream` is being captured into a CUDA graph returns MADMAP_ERR_INVALID_ARG
 * (a replay would read freed host memory).  Returns once the work is
 * enqueued. */
madmap_status madmap_apply_ninv_noalloc(int32_t precision, int64_t n_samples, int32_t n_intervals,
                                        const int64_t* interval_offsets, const int32_t* interval_filter,
                                        int32_t n_filters, int32_t n_lags, const double* filter_lags,
                                        const void* y, void* w, void* stream);

/* ------------------------------------------------------------------ diagnostics */

/* Number of kernels this library has launched in the process (each kernel
 * node of a replayed CUDA graph counts once per replay; kernels that return
 * at once because a solve already finished still count). */
int64_t madmap_kernel_launch_count(void);

/* The polarisation weights (cos 2psi, sin 2psi) of Section 3, Eq. 4 (as
 * relabelled above) for n angles, formed exactly as the operator kernels of
 * `precision` form them: FP32 reduces 2 psi to [-pi, pi] (Cody-Waite, two
 * parts of 2 pi) and uses the hardware sine and cosine approximations (absolute
 * error below 1e-6 against the exact weights of the float32 angle); FP64
 * uses correctly rounded float64 sincos of 2 (double) psi.  psi: device float
 * [n] radians; cos2psi, sin2psi: device [n], float for FP32, double for FP64.
 * A diagnostic of the weights alone.  Asynchronous on `stream`. */
madmap_status madmap_polarisation_weights(int32_t precision, int64_t n, const float* psi, void* cos2psi,
                                          void* sin2psi, void* stream);

/* Times the operator H = A^T N^-1 A in the plan's launch configuration:
 * `reps` applications to the plan's current search-direction buffer.  First
 * with CUDA events recorded on `stream` around every launch of each of the
 * three operator kernels (gather + column FFTs; row FFTs x filter spectrum;
 * inverse column FFTs + scatter), the chunks run one after another; then
 * `reps` applications as the solver launches them (chunks of one application
 * overlapped on two plan streams) between two events on `stream`.
 * ms_out (host [4]): [0..2] mean duration of one launch of each kernel, [3]
 * mean duration of one application.  launches_out (host [3], may be NULL):
 * launches of each kernel per application.  Synchronises `stream`.
 * precision: FP64, FP32 or DF64. */
madmap_status madmap_time_operator(madmap_plan_t plan, int32_t precision, int32_t reps, double* ms_out,
                                   int32_t* launches_out, void* stream);

/* Batched solve: n_rhs right-hand sides sharing the plan's pointing (e.g.
 * noise Monte Carlo realisations), each solved as madmap_solve would, in one
 * pass of work: every kernel launch covers all unfinished right-hand sides,
 * the noise weighting pairs right-hand sides of the same window in one
 * complex FFT (so the pointing is read once per pair), and each right-hand
 * side stops on its own (MIXED: each keeps its own float64 refinement).
 * d: device float [n_rhs][n_samples]; m: device double [n_rhs][n_obs][n_stokes];
 * info: host [n_rhs] or NULL.  Returns the most severe per-rhs status.
 * Synchronises `stream`. */
madmap_status madmap_solve_batched(madmap_plan_t plan, int32_t n_rhs, const float* d, double* m,
                                   const madmap_solve_opts* opts, madmap_solve_info* info, void* stream);

/* Gradients of a loss L(m) through the solve, by the implicit adjoint (the
 * paper does not differentiate the solve; with lambda = H^-1 dL/dm, one more
 * solve with the self-adjoint H, perturbing N^-1 and d in m = H^-1 A^T N^-1 d
 * gives):
 *   grad_d         = dL/dd = N^-1 A lambda                  (float32 operator)
 *   grad_lags[k,t] = dL/df_k(t) = sum over intervals of filter k of
 *                    sum_{|t1 - t2| = t} (A lambda)_t1 (d - A m)_t2
 * (both orders of each pair for t > 0; direct sums, float32 products with
 * float64 totals).  d: device float [n_samples]; m and grad_m: device double
 * [n_obs][n_stokes] (m the solution for d; grad_m is ignored at excised
 * pixels and at the unused columns of extended pointing's extra rows);
 * grad_d: device float [n_samples] or NULL; grad_lags: device double
 * [n_filters][n_lags] or NULL.  opts/info as in madmap_solve, for the
 * adjoint solve.  Gradients with respect to PSD parameters follow by the
 * chain rule through madmap_noise_filter's dlags_out.  Synchronises `stream`. */
madmap_status madmap_solve_backward(madmap_plan_t plan, const float* d, const double* m, const double* grad_m,
                                    float* grad_d, double* grad_lags, const madmap_solve_opts* opts,
                                    madmap_solve_info* info, void* stream);

/* ------------------------------------------------------------------ host helpers */

/* Inverse-noise filter lags from the PSD p(f) = sigma^2 (1 + (fknee/f)^alpha)
 * (Section 4, Eq. 13).  The paper leaves the PSD-to-lag map unstated; this
 * library samples 1/p on L = 4 n_lags frequencies nu_j = min(j, L-j) fs / L
 * (the j = 0 bin takes the value of j = 1), inverse-DFTs, and applies a
 * Bartlett taper 1 - tau/n_lags, which keeps every Toeplitz block positive
 * definite.  lags_out: host [n_lags].  dlags_out: host [3][n_lags]
 * (d/dsigma, d/dfknee, d/dalpha) or NULL.  Host only, synchronous. */
madmap_status madmap_noise_filter(int32_t n_lags, double fs, double sigma, double fknee, double alpha,
                                  double* lags_out, double* dlags_out);

/* Chain rule through madmap_noise_filter: given grad_lags = dL/df (host
 * [n_lags]) for the filter built from (sigma, fknee, alpha), writes
 * grad_params_out (host [3]) = dL/d(sigma, fknee, alpha).  Host only. */
madmap_status madmap_noise_filter_vjp(int32_t n_lags, double fs, double sigma, double fknee, double alpha,
                                      const double* grad_lags, double* grad_params_out);

/* FFT length of Section 5.2: the smallest power of two above the longest
 * interval, halved while h'(n_f) (Eq. 24) stays positive and n_f/2 > 2 n_c. */
int64_t madmap_paper_fft_length(int64_t n_lags, int64_t longest_interval);

/* Message of the last error on this thread ("" if none). */
const char* madmap_last_error(void);

/* Library version string. */
const char* madmap_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MADMAP_H_ */
