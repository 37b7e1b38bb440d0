/*
 * srm.h -- C ABI of libsrm, a GB300 (sm_103a) implementation of the EM
 * iteration of the probabilistic Shared Response Model.
 *
 * Method: Anderson et al., "Enabling Factor Analysis on Thousand-Subject
 * Neuroimaging Datasets" (arXiv 1608.04647), Sec. II and Algorithm 1 (D-SRM).
 *
 *   model (Sec. II-A, Eq. 1):  x_it = W_i s_t + mu_i + eps_it,
 *       W_i (v_i x k) with W_i^T W_i = I,  s_t ~ N(0, Sigma_s),
 *       eps_it ~ N(0, rho_i^2 I),  i = 1..N subjects,  t = 1..T samples.
 *   E-step (eq:srm_inversion_opt, eq:srm_wt_psi_w, eq:srm_mean_distributed):
 *       rho_0 = sum_i rho_i^-2,  Phi = (Sigma_s^-1 + rho_0 I)^-1,
 *       E[S] = Phi * sum_i rho_i^-2 W_i^T X^_i         (k x T)
 *   M-step (eq:srm_variance_update_optimized, eq:srm_mapping_update,
 *           eq:srm_rho_update):
 *       Sigma_s = Phi + E[S] E[S]^T / T,
 *       A_i = X^_i E[S]^T,  W_i = A_i (A_i^T A_i)^-1/2,
 *       rho_i^2 = (||X^_i||_F^2 - 2 tr(W_i^T A_i) + T tr Sigma_s) / (T v_i)
 *   X^_i is subject i's data demeaned over time (Algorithm 1, initialisation).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major.  X_i is v_i x T (T contiguous), W_i is v_i x k
 *     (k contiguous), E[S] is k x T (T contiguous), Sigma_s is k x k.
 *   - "_dev" pointers are device (HBM) pointers on the context's device; all
 *     other pointers are host pointers.  The caller owns every pointer it
 *     passes; the library owns the context and everything it allocates.
 *   - Compute calls are asynchronous on the context's stream.  Calls that
 *     return host data synchronise that stream.  Numerical failures detected
 *     on the device (non-finite values, a non-positive-definite matrix, an
 *     eigen-solver that did not converge) are raised by the next
 *     synchronising call as SRM_ERR_NUMERIC.
 *   - No exception crosses the ABI.  On failure the call returns a non-zero
 *     srm_status and srm_last_error() describes it; the context is left
 *     usable unless the status is SRM_ERR_CUDA.
 *   - One context must not be used from two host threads at once.
 */
#ifndef SRM_H
#define SRM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SRM_API __attribute__((visibility("default")))
#else
#define SRM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SRM_OK = 0,
    SRM_ERR_ARG = 1,      /* invalid argument (null pointer, bad size, bad flag) */
    SRM_ERR_CUDA = 2,     /* a CUDA runtime/driver call failed */
    SRM_ERR_NOMEM = 3,    /* device or host allocation failed */
    SRM_ERR_NUMERIC = 4,  /* device-side numerical failure (see above) */
    SRM_ERR_STATE = 5,    /* call out of order (e.g. srm_get_s before any E-step) */
    SRM_ERR_UNSUPPORTED = 6 /* valid request this build does not support */
} srm_status;

typedef enum { SRM_F32 = 0, SRM_BF16 = 1 } srm_dtype;

/* srm_config.flags */
#define SRM_BATCHED    (1u << 0) /* grouped persistent tensor-core contractions over all
                                    subjects (requires store_dtype == SRM_BF16); without it
                                    the plain per-subject FP32 SIMT form runs (requires
                                    store_dtype == SRM_F32) */
#define SRM_GRAPH      (1u << 1) /* srm_fit replays one EM iteration as a CUDA graph */
#define SRM_FINAL_LL   (1u << 3) /* srm_fit also evaluates the log-likelihood of the final
                                    parameters (one extra E-step, E[S] not replaced) */
#define SRM_HOST_INPUT (1u << 4) /* X pointers given to srm_init are host pointers; the
                                    library streams them to the device subject by subject */
#define SRM_PROFILE    (1u << 5) /* time every kernel with CUDA events on the context stream
                                    (srm_get_kernel_times); disables SRM_GRAPH */
#define SRM_SINGLE_PASS (1u << 6) /* with SRM_BATCHED, k <= 64 and T <= 1024: each M-step
                                    streams X^ once, producing A_i, its Gram and, for the
                                    next E-step, A_i^T X^_i (W_i^T X^_i = M_i A_i^T X^_i,
                                    Sec. II-B); E-steps that follow an M-step then read no
                                    X^.  Ignored where unsupported (srm_layout out[5]
                                    reports whether it is active) */

typedef struct {
    int32_t n_subjects;      /* N >= 1 */
    const int64_t* voxels;   /* host array of N voxel counts v_i >= k (may differ) */
    int32_t T;               /* samples per subject, T >= 2 */
    int32_t k;               /* features, 1 <= k <= 128, k <= T */
    srm_dtype in_dtype;      /* element type of the X_i given to srm_init */
    srm_dtype store_dtype;   /* element type of the library's resident copy of X^_i */
    uint32_t flags;          /* SRM_* flags above */
    int32_t max_iter;        /* capacity of the log-likelihood trace (>= total iterations
                                run over the context's life; 0 -> 1024) */
    uint64_t seed;           /* seed of the random orthogonal W^0 that srm_init draws when
                                it is given no W0 (see srm_init) */
} srm_config;

typedef struct srm_ctx srm_ctx;  /* opaque; created by srm_init, freed by srm_destroy */

/*
 * srm_init -- create a context, copy and demean the data (Algorithm 1,
 * initialisation: mu_i = (1/T) sum_t x_it, x^_it = x_it - mu_i), compute
 * ||X^_i||_F^2, and set rho_i^2 = 1, Sigma_s = I_k, W_i = W0_i.
 *
 *   cfg       configuration (read during the call only).
 *   X         N pointers; X[i] is v_i x T row-major, element type cfg->in_dtype,
 *             device pointers unless SRM_HOST_INPUT.  Read during the call only:
 *             the library keeps its own demeaned copy in cfg->store_dtype.
 *   W0_dev    N device pointers; W0_dev[i] is v_i x k row-major FP32 with
 *             orthonormal columns (Algorithm 1: "a random orthogonal matrix").
 *             Read during the call only.  NULL: the library draws W^0 itself
 *             from the Haar distribution, as the Q factor (with a positive-
 *             diagonal R) of a v_i x k matrix G_i of standard normals from the
 *             counter-based generator Philox4x64-10 (Salmon et al., SC 2011):
 *             key (cfg->seed, 0), counter (b, i, 0, 0) for block b of subject
 *             i; each output word w gives u = ((w >> 12) + 1/2) 2^-52; the
 *             word pairs (w0, w1), (w2, w3) of block b give entries 4b..4b+3
 *             of G_i (row-major) by Box-Muller, sqrt(-2 ln u_a) cos(2 pi u_b)
 *             and sqrt(-2 ln u_a) sin(2 pi u_b).  Any implementation of this
 *             definition draws the same W^0 (to rounding).  Q is formed by two
 *             Cholesky-QR passes in FP64 in a temporary workspace
 *             (about 20 v_max k bytes).
 *   stream    cudaStream_t the context runs on, or NULL for a library-owned
 *             non-blocking stream.  The device is the current CUDA device.
 *   out       receives the context.
 * Returns SRM_ERR_ARG for N < 1, k outside [1, 128], k > T, k > v_i, a null
 * pointer, or an unsupported dtype/flag combination; SRM_ERR_NOMEM if the
 * resident copy does not fit.  The call synchronises the stream.
 */
SRM_API srm_status srm_init(const srm_config* cfg, const void* const* X, const float* const* W0_dev,
                    void* stream, srm_ctx** out);

/*
 * srm_estep -- one E-step at the current parameters (Algorithm 1, E-step):
 * the reduction y = sum_i rho_i^-2 W_i^T X^_i, rho_0, Phi, E[S]
 * (eq:srm_mean_distributed), the log-likelihood of the current parameters
 * (appended to the trace) and the pending Sigma_s^new
 * (eq:srm_variance_update_optimized).  Asynchronous.
 */
SRM_API srm_status srm_estep(srm_ctx* ctx);

/*
 * srm_mstep -- the M-step that follows an E-step (Algorithm 1, M-step):
 * commit Sigma_s^new, form A_i = X^_i E[S]^T and its Gram matrix, set
 * W_i = A_i (A_i^T A_i)^-1/2 (eq:srm_mapping_update) and rho_i^2
 * (eq:srm_rho_update).  SRM_ERR_STATE if no E-step preceded it.  Asynchronous.
 */
SRM_API srm_status srm_mstep(srm_ctx* ctx);

/*
 * srm_fit -- n_iter EM iterations (E-step then M-step each).  If ll_host is
 * not NULL it receives the n_iter log-likelihoods of the parameters each
 * E-step used (n_iter + 1 values with SRM_FINAL_LL) and the call synchronises;
 * otherwise the call is asynchronous.
 */
SRM_API srm_status srm_fit(srm_ctx* ctx, int32_t n_iter, double* ll_host);

/*
 * Sharded E-step (Algorithm 1, D-SRM: subjects are spread over processes and
 * the E-step's one exchange is the Reduce of eq:srm_mean_distributed).  Each
 * process holds a context over its own subjects.  Per iteration:
 *   srm_estep_partial(ctx, y, sums)   this context's share;
 *   the caller sums y and sums over all contexts (an all-reduce, e.g. NCCL);
 *   srm_estep_finish(ctx, y, sums)    the rest of the E-step from the totals;
 *   srm_mstep(ctx)                    W_i and rho_i^2 of this context's subjects.
 * Every context then holds the same Sigma_s, E[S] and log-likelihood trace,
 * equal (to rounding) to one context over all subjects.  Sigma_s and E[S]
 * are formed redundantly in every context, so no broadcast follows.
 *
 * srm_estep_partial -- the pending M-step tail, the E-pass and the reduction
 * over this context's subjects, stopped before Phi:
 *   y     k x T row-major FP64, device pointer (written):
 *         y = sum over this context's subjects of rho_i^-2 W_i^T X^_i.
 *   sums  4 FP64, device pointer (written): { sum rho_i^-2 (eq:srm_wt_psi_w),
 *         sum v_i ln rho_i^2, sum ||X^_i||_F^2 / rho_i^2, sum v_i } over this
 *         context's subjects (the log-likelihood's sums over subjects).
 * Asynchronous on the context's stream; the caller must order its reduction
 * after it (e.g. on the same stream).  SRM_ERR_STATE while a partial E-step
 * awaits its finish; until srm_estep_finish, srm_estep, srm_mstep, srm_fit,
 * srm_set_plan, srm_autotune and the state calls return SRM_ERR_STATE.
 *
 * srm_estep_finish -- Phi = (Sigma_s^-1 + rho_0 I)^-1 with rho_0 = sums[0]
 * (eq:srm_inversion_opt), E[S] = Phi y (eq:srm_mean_distributed), and, with
 * the next M-step, Sigma_s^new (eq:srm_variance_update_optimized) and the
 * log-likelihood of the parameters this E-step used, over all subjects.
 *   y, sums  the totals over every context, laid out as above (device
 *            pointers, read by launches on the context's stream).
 * SRM_ERR_STATE without a preceding srm_estep_partial.  Asynchronous.
 */
SRM_API srm_status srm_estep_partial(srm_ctx* ctx, double* y_dev, double* sums_dev);
SRM_API srm_status srm_estep_finish(srm_ctx* ctx, const double* y_dev, const double* sums_dev);

/*
 * srm_transform -- map new data of one subject to the shared space
 * (Sec. II-A: W_i^T x): S_out = W_i^T (X_new - mean_t X_new).
 *   subject    0 <= subject < N
 *   X_new_dev  v_i x T_new row-major, cfg->in_dtype, device pointer
 *   T_new      >= 1 columns
 *   S_out_dev  k x T_new row-major FP32, device pointer (written)
 * Asynchronous.
 */
SRM_API srm_status srm_transform(srm_ctx* ctx, int32_t subject, const void* X_new_dev, int32_t T_new,
                         float* S_out_dev);

/*
 * srm_map -- map new data of subject `from` into the voxel space of subject
 * `to` through the shared space (Sec. II-A, the orthogonality of the mappings
 * gives the subject-to-subject map W_j W_i^T):
 *   Y_out = W_to W_from^T (X_new - mean_t X_new).
 *   from, to   0 <= from, to < N (equal: the projection onto span W_from)
 *   X_new_dev  v_from x T_new row-major, cfg->in_dtype, device pointer
 *   T_new      >= 1 columns
 *   Y_out_dev  v_to x T_new row-major FP32, device pointer (written)
 * Uses the mappings of the last M-step (W^0 before any).  Keeps a scratch
 * buffer of 2 k T_new floats in the context (grown on demand; SRM_ERR_NOMEM
 * if that allocation fails).  Asynchronous.
 */
SRM_API srm_status srm_map(srm_ctx* ctx, int32_t from, int32_t to, const void* X_new_dev, int32_t T_new,
                           float* Y_out_dev);

/*
 * srm_transform_noalloc -- the same result as srm_transform, for callers that
 * must not allocate device memory: real-time or latency-bound loops, where a
 * cudaMalloc or cudaFree would synchronise the whole device and stall them,
 * and hosts whose device memory is handed out by a pool or by another
 * framework, so that an allocation from outside that pool fails or breaks
 * its accounting.  srm_transform allocates (and grows) its scratch on first
 * use; this entry point allocates nothing: no cudaMalloc, no cudaFree and no
 * allocating library routine.  The paper has no counterpart.
 *
 * Scratch lives in one fixed device array of 16 MiB compiled into the
 * library (every GPU that loads the library holds it until the process
 * exits).  A call needs 4 * v_i bytes (rounded up to 256) for the row means
 * plus 64 * kld * 4 bytes per 64 columns of X_new for one v-split (kld = k
 * padded: to 64 or 128 in the batched form, to a multiple of 16 in the plain
 * form); larger requests return SRM_ERR_ARG with the sizes in
 * srm_last_error().  Arguments, layout and result are those of srm_transform.
 *
 * The context's device must be the current device (SRM_ERR_ARG otherwise).
 * The first call on a device looks up the device address of the array once,
 * with that device current; make that first call before any stream capture.
 * Every call uses the same array and overwrites what it reads, so nothing
 * needs clearing, but calls whose work overlaps on the GPU (on different
 * streams, or from different contexts of one process on one device) race on
 * the array: order them on one stream.  Asynchronous.
 */
SRM_API srm_status srm_transform_noalloc(srm_ctx* ctx, int32_t subject, const void* X_new_dev, int32_t T_new,
                                         float* S_out_dev);

/* srm_get_w -- W_i = A_i (A_i^T A_i)^-1/2 (eq:srm_mapping_update) materialised as
 * v_i x k row-major FP32 into W_dev (device, caller-owned).  Asynchronous. */
SRM_API srm_status srm_get_w(srm_ctx* ctx, int32_t subject, float* W_dev);

/* srm_get_s -- E[S] of the last E-step, k x T row-major FP32, into S_dev (device).
 * SRM_ERR_STATE before the first E-step.  Asynchronous. */
SRM_API srm_status srm_get_s(srm_ctx* ctx, float* S_dev);

/* srm_get_params -- current rho_i^2 (N doubles) and Sigma_s (k x k doubles) to the
 * host; either pointer may be NULL.  Synchronises. */
SRM_API srm_status srm_get_params(srm_ctx* ctx, double* rho2_host, double* sigma_host);

/* srm_get_ll -- the whole log-likelihood trace so far: writes min(*n, count) values
 * to ll_host and sets *n = count.  Synchronises. */
SRM_API srm_status srm_get_ll(srm_ctx* ctx, double* ll_host, int32_t* n);

/* srm_synchronize -- wait for the context's stream and report device-side status. */
SRM_API srm_status srm_synchronize(srm_ctx* ctx);

/*
 * srm_get_state / srm_set_state -- checkpoint of the EM state (rho^2, Sigma_s,
 * the per-subject mapping factors, the log-likelihood trace and the iteration
 * count) to a host buffer.  With buf == NULL, srm_get_state only sets *bytes to
 * the size needed.  srm_set_state requires a context created with the same
 * configuration; SRM_ERR_ARG on a size or header mismatch.  Both synchronise.
 */
SRM_API srm_status srm_get_state(srm_ctx* ctx, void* buf, size_t* bytes);
SRM_API srm_status srm_set_state(srm_ctx* ctx, const void* buf, size_t bytes);

/*
 * srm_get_kernel_times -- with SRM_PROFILE: for each kernel kind, its name,
 * launch count and total CUDA-event time (ms) since the last reset.  Writes up
 * to *n entries; sets *n to the number of kinds.  names[j] points to static
 * strings.  reset != 0 clears the counters after reading.  Synchronises.
 */
SRM_API srm_status srm_get_kernel_times(srm_ctx* ctx, const char** names, int64_t* launches, double* ms,
                                int32_t* n, int32_t reset);

/*
 * srm_layout -- sizes the library chose for this context (for reporting):
 * out[0] = padded row stride of the resident X^ (elements), out[1] = padded k
 * of the tensor-core operands, out[2] = total resident rows (all subjects, padded),
 * out[3] = bytes of the resident X^, out[4] = bytes of the per-subject
 * mapping factors A_i, out[5] = 1 if the single-pass form (SRM_SINGLE_PASS) is
 * active, else 0.  n = number of entries the caller's array holds.
 */
SRM_API srm_status srm_layout(srm_ctx* ctx, int64_t* out, int32_t n);

/*
 * Launch plan of the batched form (SRM_BATCHED).  How the two contractions
 * of Algorithm 1 (the E-step reduction sum_i W_i^T X^_i and the M-step's
 * A_i = X^_i E[S]^T with its Gram) are cut into tiles and pipelined.  The
 * mathematics is the same under every plan.  e_reserve and single_pass
 * change the order of the FP32 partial sums, so results differ between such
 * plans by rounding only.  Results under one fixed plan are bitwise
 * reproducible.
 */
typedef struct {
    int32_t single_pass;    /* 1: one stream of X^ per iteration (the SRM_SINGLE_PASS form;
                               needs k <= 64 and T <= 1024), 0: two passes */
    int32_t e_reserve;      /* SMs the E-pass leaves to the M-step tail that runs beside it;
                               the E-pass runs (SMs - e_reserve) persistent CTAs, which
                               split the voxel dimension (the split-v depth) */
    int32_t m_stages;       /* M-pass shared-memory pipeline stages, 2..8 */
    int32_t m_gram_bufs;    /* M-pass Gram operand buffers, 1 or 2 */
    int32_t m_resident_es;  /* 1: E[S] stays resident in shared memory during the M-pass */
    int32_t m_prefetch;     /* M-pass L2 prefetch distance in 64-column X^ chunks (0 = off) */
    int32_t f_prefetch;     /* single-pass L2 prefetch distance in 128-row tiles (0 = off) */
    int32_t f_l2_hints;     /* single-pass L2 eviction hints, bits: 1 = a tile's first read
                               evicts last, 2 = its second read (last use) evicts first,
                               4 = A_i stores evict first */
    int32_t f_first_stages; /* single pass: stages of the ring that streams each tile from HBM
                               for A_i; the rest re-read it for A_i^T X^_i.  With f_slots = 0,
                               32 KB stages of 4: 1..3, or 4 = one shared ring serving both
                               reads in turn.  With f_slots = 8 or 9, 16 KB slots: 2..f_slots - 2 */
    int32_t f_reserve;      /* SMs the single pass leaves to the Sigma_s chain that runs
                               beside it (the pass runs on the rest, in whole clusters) */
    int32_t m_boxes;        /* M-pass: consecutive 64-column boxes of the same 128 rows of X^
                               per stage, 1, 2 or 4 (longer contiguous reads per row) */
    int32_t f_lead;         /* single pass with two rings: tiles the first read of X^ may run
                               ahead of the second (which then finds the tile in L2), 1..4;
                               0 = no limit */
    int32_t f_slots;        /* single pass, T <= 512 only: 0 = four 32 KB stages and two
                               A_tile buffers; 8 = eight 16 KB slots and two A_tile buffers;
                               9 = nine 16 KB slots and one A_tile buffer (the phase-1
                               epilogue of a tile then waits for phase 2 of the one before) */
} srm_plan;

/* srm_get_plan -- the plan the context runs.  SRM_ERR_UNSUPPORTED for the plain
 * FP32 form, which has no plan. */
SRM_API srm_status srm_get_plan(srm_ctx* ctx, srm_plan* plan);

/*
 * srm_set_plan -- run later iterations under `plan`.  Allowed between
 * iterations only, so SRM_ERR_STATE if an E-step awaits its M-step.  A pending
 * M-step tail is finished first under the old plan.  SRM_ERR_ARG if the
 * M-pass plan does not fit in shared memory or a field is out of range.
 * SRM_ERR_UNSUPPORTED for single_pass = 1 where that form is unsupported.
 * SRM_ERR_NOMEM if the single-pass buffers, allocated on first use, do not
 * fit.  Synchronises.
 */
SRM_API srm_status srm_set_plan(srm_ctx* ctx, const srm_plan* plan);

/*
 * srm_autotune -- choose the plan for this context's shapes (v_i, T, k) on
 * this device by timing, then leave the context as srm_init left it.  The
 * search has four stages:
 *   1. every M-pass plan that fits in shared memory, timed launch by launch;
 *   2. the single-pass prefetch distances, where that form is supported;
 *   3. E-pass reserves (split-v depths), timed as whole EM iterations;
 *   4. the two forms, timed as whole EM iterations.
 * Iterations run through srm_fit's own path, with CUDA events on the
 * context's stream.  Call it right after srm_init, before any E-step;
 * otherwise SRM_ERR_STATE.  The W0 given to srm_init and the initial
 * parameters are restored afterwards, so the fit that follows is the one an
 * untuned context would run under the chosen plan.
 *
 *   cache_path    NULL, or a text file of tuned plans keyed by the device name,
 *                 SM count, N, T, k and a hash of the v_i.  A matching line is
 *                 applied without timing anything.  Otherwise the result is
 *                 added to the file, written through a temporary file and a
 *                 rename.  Concurrent tuners of one file may drop each
 *                 other's lines.
 *   iters         EM iterations timed per whole-iteration candidate (>= 1;
 *                 2 more run untimed before each).  The log-likelihood trace
 *                 must hold iters + 3 entries (srm_config.max_iter).
 *   chosen        receives the chosen plan (may be NULL).
 *   ms_per_iter   receives its milliseconds per EM iteration (may be NULL).
 *   report        NULL, or a host buffer for a text table of every timing.
 *                 It is truncated to report_bytes and NUL-terminated.
 * Temporarily allocates one copy of the A_i (W0).  SRM_ERR_NOMEM if that
 * copy does not fit.  SRM_ERR_UNSUPPORTED for the plain FP32 form.
 * Synchronises.
 */
SRM_API srm_status srm_autotune(srm_ctx* ctx, const char* cache_path, int32_t iters, srm_plan* chosen,
                                double* ms_per_iter, char* report, size_t report_bytes);

/* Thread-local description of the last failure in this thread ("" if none). */
SRM_API const char* srm_last_error(void);

/* Free the context and everything it owns.  NULL is a no-op.  Synchronises. */
SRM_API void srm_destroy(srm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SRM_H */
