/*
 * gabp_svm.h -- C ABI of the GB300 GaBP SVM solver.
 *
 * The solver follows Bickson, Yom-Tov and Dolev, "A Gaussian Belief
 * Propagation Solver for Large Scale Support Vector Machines":
 *
 *   - the SVM dual (Section 1.1) with D_ij = y_i y_j K(x_i, x_j) and the RBF
 *     kernel K(a, b) = exp(-gamma ||a - b||^2);
 *   - the bias as an extra constant feature lambda (Section 3), which for the
 *     RBF kernel adds lambda^2 to every kernel value; default lambda = 1/n;
 *   - a weighted main diagonal that makes the matrix diagonally dominant
 *     (Section 3.1), giving the matrix Q that the solver works on;
 *   - the unconstrained Gaussian p(h) ~ exp(-h'Qh/2 + h'1) (Section 3), whose
 *     mean Q^-1 1 is found by the broadcast form of Gaussian belief
 *     propagation (Algorithm 2, Section 4) in synchronous rounds (Section 5);
 *   - the weights alpha = clip(mean, 0, C) and the decision function
 *     f(x) = sum_i alpha_i y_i K'(x_i, x) (Section 1.1).
 *
 * Options extend it along the paper's own directions: BF16 tensor-core Q and
 * BF16 messages with defect correction (the precision forms), a block
 * Gauss-Seidel message schedule (Section 3.2), kernel ridge regression on
 * the same solver (Section 1.2), a tile-sparse kernel (Section 6), and the
 * batched and served forms for many instances.
 *
 * Everything after create() runs on one CUDA device in hand-written kernels.
 * There is no CPU fallback: every call that needs the GPU fails with
 * GABP_ECUDA when there is none.
 *
 * Conventions
 *   - Every call returns a gabp_status; no exception or signal crosses the ABI.
 *     On failure gabp_last_error() returns a message (thread-local).
 *   - Inputs are read-only and stay owned by the caller; outputs are
 *     caller-allocated.  In device-pointer mode (opts.ptr_mode = 1) the library
 *     reads and writes the caller's device buffers during the call only and
 *     never frees them.
 *   - A handle owns every device buffer it allocates and frees them in
 *     gabp_svm_destroy().  A handle is not thread-safe: one thread at a time.
 *   - All work is issued on the handle's stream (opts.stream, or a stream the
 *     handle creates).  Every call returns after its work has completed.
 *   - Non-convergence is not an error: gabp_svm_solve() returns GABP_OK with
 *     *iters_done == iters and the residual of the last round.
 */
#ifndef GABP_SVM_H
#define GABP_SVM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GABP_SVM_VERSION 3

#if defined(__GNUC__)
#define GABP_API __attribute__((visibility("default")))
#else
#define GABP_API
#endif

typedef enum {
    GABP_OK = 0,
    GABP_EINVAL = 1,    /* bad argument (size, pointer, label not +-1, non-finite input ...) */
    GABP_ENOMEM = 2,    /* device memory for the handle does not fit; nothing was launched */
    GABP_ECUDA = 3,     /* a CUDA runtime call failed (no device, launch error ...) */
    GABP_ENUMERIC = 4,  /* a cavity precision Ptilde_i - P_ji went nonpositive or non-finite */
    GABP_ETIMEOUT = 5,  /* a bounded device-side wait ran out (batched/serving forms) */
    GABP_ESTATE = 6     /* call not valid in the handle's current state */
} gabp_status;

/* How Q is held during the sweeps. */
typedef enum {
    GABP_Q_F32 = 0,        /* upper triangle stored in FP32, formed by an FP32 Gram kernel */
    GABP_Q_BF16 = 1,       /* upper triangle stored in BF16, formed by the tensor-core Gram kernel */
    GABP_Q_RECOMPUTE = 2   /* not stored: every sweep recomputes Q tiles on the tensor cores (BF16 Gram, FP32 accumulate) */
} gabp_q_mode;

/* The problem solved on the same sweep.  SVM (Section 1.1, 3): y are labels
 * +-1, Q_ij = y_i y_j (K + lambda^2), right-hand side 1, alpha = clip(mu, 0,
 * C).  KRR, kernel ridge regression (Section 1.2): y are real targets, the
 * C argument is the ridge lambda_r, Q = K + lambda_r I (under the soft2 rule;
 * the dominant rule raises the diagonal as for the SVM), right-hand side y,
 * alpha = c = Q^-1 y unclipped, the bias term off unless bias_mode = 1, and
 * f(x) = sum_i c_i K(x_i, x). */
typedef enum {
    GABP_TASK_SVM = 0,
    GABP_TASK_KRR = 1
} gabp_task;

typedef enum {
    GABP_DIAG_DOMINANT = 0, /* Q_ii = max(1 + lambda^2 + 1/C, (1 + delta) sum_{j!=i} |Q_ij|) */
    GABP_DIAG_SOFT2 = 1     /* Q_ii = 1 + lambda^2 + 1/C (2-norm soft margin only) */
} gabp_diag_rule;

/* Options.  gabp_svm_opts_default() fills the defaults; a zero-initialised
 * struct also means the defaults except where noted. */
typedef struct {
    int32_t x_dtype;       /* layout of X and Xtest: 0 = float32 (default), 1 = float64 (converted to FP32
                              on the device), 2 = bfloat16 (widened to FP32 on the device, exactly) */
    int32_t ptr_mode;      /* 0 = host pointers (copied in/out, default), 1 = device pointers */
    void*   stream;        /* cudaStream_t to run on; NULL = the handle creates its own */
    int32_t diag_rule;     /* gabp_diag_rule, default GABP_DIAG_DOMINANT */
    double  diag_delta;    /* delta of the dominant rule; 0 selects the default 0.1 */
    int32_t bias_mode;     /* 0 = lambda = 1/n (default), 1 = lambda = bias_lambda (may be 0;
                              lambda^2 must not exceed FLT_MAX, else GABP_EINVAL) */
    double  bias_lambda;
    int32_t q_mode;        /* gabp_q_mode, default GABP_Q_F32 */
    int32_t refine;        /* precision form only: up to this many defect-correction passes with the
                              FP32-Gram residual (FP64 sums); 0 = plain BF16 solve */
    double  sv_threshold;  /* support vectors are the i with alpha_i > sv_threshold (default 0) */
    int32_t chunk;         /* sweeps per captured CUDA graph replay between convergence checks; 0 = 16 */
    int32_t msg_bf16;      /* precision forms only: store the messages in BF16 (arithmetic stays FP32);
                              use with refine > 0, which removes the rounding error */
    float   refine_handover; /* refinement only: the first solve hands over to the defect correction
                                once its in-sweep ||r||_inf < refine_handover (never below tol);
                                0 = 1e-3 with BF16 messages, 1e-4 with FP32 messages */
    float   refine_inner;  /* refinement only: each correction pass stops once its residual is below
                              refine_inner * ||r||_inf of its right-hand side (never below tol / 2);
                              0 = 3e-2 with BF16 messages, 1e-2 with FP32 messages */
    int32_t task;          /* gabp_task, default GABP_TASK_SVM */
    int32_t stages;        /* message schedule: 0 or 1 = synchronous (Algorithm 2 as in Section 5's
                              experiments, default); S = 2..16 = block Gauss-Seidel: a round updates
                              every pair once, in S stages over bands of tile columns, and later stages
                              use the aggregates of the earlier ones (Section 3.2: GaBP also converges
                              under non-synchronous schedules).  Same fixed point, fewer rounds */
    float   sparse_tau;    /* tile-sparse kernel (Section 6's sparsified kernel, at the granularity of the
                              128 x 128 tiles): every off-diagonal tile whose largest |Q_ij| <= sparse_tau
                              is dropped, i.e. solved as 0 (its messages stay 0 and are never swept);
                              the diagonal keeps the row sums of the whole matrix, so the matrix stays
                              diagonally dominant and only the dropped entries change.  Device memory:
                              the messages, Q and per-node partial sums of the kept tiles only, plus
                              bookkeeping of 48 B per tile and 8 B per node for the whole matrix's row
                              sums.  Effective when rows are ordered so that near points
                              share tiles.  0 = dense (default).  Single-instance API only (not the
                              batched or served forms) */
    int32_t reserved[1];
} gabp_svm_opts;

typedef struct gabp_svm_s* gabp_svm_t;

/* Per-handle results of the last solve. */
typedef struct {
    int64_t n, m;
    int64_t sweeps_total;      /* message updates applied to the state since the last create/refit */
    int32_t kstar;             /* round whose means were returned (counted since create/refit) */
    int32_t converged;         /* 1 if the last solve stopped on its tolerance; then residual_inf < tol
                                  (except an unrefined BF16 / recompute solve, which stops on its BF16
                                  matrix while residual_inf is that of the FP32-Gram matrix) */
    double  residual_inf;      /* ||1 - Q mu(kstar)||_inf, FP64 sums */
    double  dual_objective;    /* sum_i alpha_i - 1/2 alpha' Q alpha for alpha = clip(mu(kstar), 0, C), FP64 */
    int64_t n_support;         /* #{i : alpha_i > sv_threshold} */
    double  lambda, gamma, C, diag_delta;
    int64_t device_bytes;      /* device memory held by the handle */
    int32_t q_mode, diag_rule;
    int32_t refine_passes;     /* defect-correction passes done by the last solve */
    int64_t tiles_total;       /* upper-triangle 128 x 128 tiles of Q */
    int64_t tiles_kept;        /* tiles swept (all of them unless sparse_tau > 0) */
    double  margin;            /* min_i (Q_ii - sum_{j != i} |Q_ij|) of the FP32-Gram matrix, FP64 sums
                                  (whole-matrix row sums, so also a lower bound for the tile-sparse
                                  matrix); <= 0 when Q is not strictly diagonally dominant */
    double  err_bound;         /* Varah's bound on ||mu(kstar) - Q^-1 b||_inf for that matrix:
                                  residual_inf / margin (+inf when margin <= 0); alpha = clip(mu, 0, C)
                                  is within the same distance of clip(Q^-1 b, 0, C) */
} gabp_svm_stats;

/* Default options. */
GABP_API void gabp_svm_opts_default(gabp_svm_opts* opts);

/*
 * Create a solver for the n x m training set X (row-major) with labels y
 * (n floats, each +1 or -1), RBF width gamma > 0 and box constant C > 0
 * (with opts->task = GABP_TASK_KRR: y are finite real targets and C > 0 is
 * the ridge lambda_r).
 * Forms Q on the device (Gram kernel fused with exp, bias and labels), weights
 * its diagonal (Section 3.1) and sets the GaBP state to Algorithm 2's Step 1
 * (all messages 0).  Requires n >= 2, m >= 1.
 * gamma and lambda^2 enter the kernels in FP32: gamma > FLT_MAX or a non-finite
 * C is GABP_EINVAL (so are the same values in the batched and served forms).
 * Device memory: about 8 n^2 bytes of message state plus the stored Q
 * (2 n^2 bytes for FP32, n^2 for BF16, 0 for recompute); GABP_ENOMEM if that
 * does not fit in free device memory, before anything is allocated.
 * X may be host or device memory per opts->ptr_mode and is not retained.
 */
GABP_API gabp_status gabp_svm_create(const void* X, const float* y, int64_t n, int64_t m,
                            double gamma, double C, gabp_svm_t* out);
GABP_API gabp_status gabp_svm_create_ex(const void* X, const float* y, int64_t n, int64_t m,
                               double gamma, double C, const gabp_svm_opts* opts,
                               gabp_svm_t* out);

/*
 * Replace the training set of an existing handle with a new one of the same
 * n and m (new X, y, gamma, C), reusing its device memory: forms Q and resets
 * the state as create() does.
 */
GABP_API gabp_status gabp_svm_refit(gabp_svm_t h, const void* X, const float* y, double gamma,
                           double C);

/*
 * Run synchronous broadcast-GaBP rounds (Algorithm 2, Steps 2-3) from the
 * handle's current state.  Round t forms the aggregates Ptilde_i, mutilde_i of
 * the current messages and the residual r(t) = b - Q mutilde(t) (b = 1 for
 * the SVM, the targets for KRR); it stops at
 * the first t with ||r(t)||_inf < tol (tol <= 0: never), or after `iters`
 * message updates.  The stop test runs inside the rounds on compensated FP32
 * tile sums; a stop is confirmed by the final residual (FP64 sums of FP32
 * tile partials, the residual_inf reported), and while that one is still
 * >= tol the rounds go on (within the `iters` limit), so a converged solve
 * reports residual_inf < tol.  (An unrefined BF16 or recompute solve stops on
 * the BF16 matrix it sweeps; its residual_inf is that of the FP32-Gram
 * matrix.  With refine > 0 the stop is on the FP32-Gram residual.)  Writes alpha = clip(mutilde(kstar), 0, C) (KRR: the
 * unclipped mutilde(kstar)) (n floats) and,
 * when non-NULL, ||r(kstar)||_inf (FP64) and the number of updates done in
 * this call.  Calling again continues from the current messages.
 * GABP_ENUMERIC if a cavity precision went nonpositive (the matrix is then
 * outside GaBP's convergence conditions); the state is then undefined until
 * the next refit.
 */
GABP_API gabp_status gabp_svm_solve(gabp_svm_t h, int32_t iters, double tol, float* alpha,
                           double* residual_inf, int32_t* iters_done);

/* Unclipped means mutilde(kstar) of the last solve (n floats; before any solve,
 * the Step-1 means b_i / Q_ii). */
GABP_API gabp_status gabp_svm_get_mean(gabp_svm_t h, float* mu);

/* Decision values f(x) = sum_i alpha_i y_i (K(x_i, x) + lambda^2) for t test
 * rows Xtest (t x m, same dtype and pointer mode as X) with the alpha of the
 * last solve; the predicted label is sign(f).  KRR: the prediction
 * f(x) = sum_i c_i K(x_i, x) (+ lambda^2 sum_i c_i with the bias on).
 * out: t floats. */
GABP_API gabp_status gabp_svm_decision(gabp_svm_t h, const void* Xtest, int64_t t, float* out);

/* Indices i with alpha_i > sv_threshold (KRR: |c_i| > sv_threshold),
 * ascending (host memory). Writes up to cap indices and the total count. */
GABP_API gabp_status gabp_svm_support(gabp_svm_t h, int32_t* idx, int64_t cap, int64_t* count);

GABP_API gabp_status gabp_svm_get_stats(gabp_svm_t h, gabp_svm_stats* stats);

/*
 * Inspection, for tests and diagnostics (host memory, small sizes):
 *   get_q:     the dense n x n matrix Q as the sweeps see it (FP32; BF16 values
 *              widened), mirrored from the stored upper triangle.  Not
 *              available in recompute mode (GABP_ESTATE).
 *   get_pairs: for cnt index pairs (i[k] < j[k]) the current messages
 *              {P_ij, P_ji, H_ij, H_ji} with H = P mu (information form);
 *              out: 4*cnt floats.
 *   get_aggregates: Ptilde, htilde = Ptilde*mutilde and mutilde of the
 *              current message state (n floats each; any may be NULL).
 */
GABP_API gabp_status gabp_svm_get_q(gabp_svm_t h, float* Q);
GABP_API gabp_status gabp_svm_get_pairs(gabp_svm_t h, const int64_t* i, const int64_t* j, int64_t cnt,
                               float* out);
GABP_API gabp_status gabp_svm_get_aggregates(gabp_svm_t h, float* Pt, float* ht, float* mu);

/* ------------------------------------------------------------------------
 * Batched and served forms.  Many instances of uneven size are swept
 * together: every synchronous round is one persistent launch over the tiles
 * of all live instances, and each instance keeps its own round count,
 * limit, tolerance and stop test (Algorithm 2, Step 3, per instance).
 * ------------------------------------------------------------------------ */
typedef struct {
    const void* X;        /* n x m features (dtype and pointer mode from the options) */
    const float* y;       /* n labels +-1 */
    int64_t n, m;
    double gamma, C;
} gabp_problem;

typedef struct {
    float*  alpha;          /* caller buffer for n weights (host or device per ptr_mode), may be NULL */
    double  residual_inf;   /* ||1 - Q mu||_inf of the answer, FP32-Gram Q, FP64 sums */
    double  dual_objective;
    int64_t n_support;
    int32_t iters_done;     /* synchronous rounds run (refinement passes included) */
    int32_t converged;      /* residual_inf < tol */
    int32_t status;         /* gabp_status of this problem */
    int32_t refine_passes;
    float*  mu;             /* caller buffer for the n unclipped means (same memory kind as alpha), may be NULL */
    double  margin;         /* min_i (Q_ii - sum_{j != i} |Q_ij|), as in gabp_svm_stats */
    double  err_bound;      /* residual_inf / margin: Varah's bound on ||mu - Q^-1 b||_inf (+inf if margin <= 0) */
} gabp_result;

/*
 * Solves `count` independent problems together.  opts (may be NULL) applies
 * to all: q_mode (BF16 store / recompute run the tensor-core Gram), refine
 * (precision forms: defect-correction passes until residual_inf < tol),
 * ptr_mode / x_dtype / stream.  opts->chunk = 0 lets the solver choose the
 * schedule (persistent sweep CTAs per SM, rounds per convergence check) by
 * timing candidates on this set; results are cached per shape signature.
 * results[k].alpha must point to the caller's buffer (or NULL).  Returns
 * GABP_OK, or the status of the first problem that failed (each result
 * carries its own status).
 */
GABP_API gabp_status gabp_batch_solve(const gabp_problem* probs, int64_t count, const gabp_svm_opts* opts,
                                      int32_t iters, double tol, gabp_result* results);

/* Host wall time (ms) of the phases of this thread's last gabp_batch_solve:
 * out7 = {formation, schedule tuning, rounds, stop handling (final residuals,
 * refinement set-up, result copies), total, number of round chunks, the host
 * part of formation (allocating and enqueuing the instances)}. */
GABP_API gabp_status gabp_batch_last_phases(double* out7);

/* gabp_batch_solve keeps its engine (instance table, tile and node lists,
 * control blocks, pinned mirrors, streams, captured round graphs: a few MB,
 * growing with the largest batch) per calling thread for the next call with
 * compatible sizes and options; instance memory is returned to the CUDA
 * stream-ordered pool at the end of every call.  This frees the calling
 * thread's kept engine (a thread that exits without calling it leaves it
 * allocated until the process ends).  Always GABP_OK. */
GABP_API gabp_status gabp_batch_release(void);

/*
 * Continuous-batching server.  Requests queue in arrival order; each
 * gabp_server_step() launches one chunk of rounds over every live instance,
 * and while it runs finishes the instances that stopped in the previous
 * chunk (their final passes ran on a stop stream meanwhile: results recorded,
 * alpha copied to the caller's buffer, or the next refinement pass started)
 * and admits queued requests (free slots and the device memory budget
 * permitting; their Q is formed on a side stream while the other instances
 * keep sweeping); after the chunk it takes the instances that stopped out of
 * the sweeps and queues their final passes, and lets instances whose
 * formation has finished join from the next chunk.  A ticket therefore
 * completes one step after its instance stopped.  The problem's X and y must
 * stay valid until its ticket completes.
 */
typedef struct gabp_server_s* gabp_server_t;
typedef struct {
    int64_t hbm_budget_bytes;  /* device memory for instances; 0 = 80% of free memory */
    int32_t max_members;       /* concurrent instances; 0 = 64 */
    int32_t iters;             /* round limit per request */
    double  tol;               /* residual tolerance per request */
    gabp_svm_opts opts;        /* q_mode, refine, diag rule, pointer mode, stream, chunk (0 = 8) */
} gabp_server_cfg;

GABP_API gabp_status gabp_server_create(const gabp_server_cfg* cfg, gabp_server_t* out);
GABP_API gabp_status gabp_server_submit(gabp_server_t s, const gabp_problem* p, float* alpha_out, int64_t* ticket);
/* As gabp_server_submit; mu_out (may be NULL) also receives the n unclipped
 * means of the answer (host or device memory like alpha_out). */
GABP_API gabp_status gabp_server_submit_ex(gabp_server_t s, const gabp_problem* p, float* alpha_out,
                                           float* mu_out, int64_t* ticket);
GABP_API gabp_status gabp_server_step(gabp_server_t s, int32_t* active, int32_t* queued, int32_t* completed);
/* done = 1 once the ticket finished; then *res holds its result. */
GABP_API gabp_status gabp_server_poll(gabp_server_t s, int64_t ticket, gabp_result* res, int32_t* done);
/* Tickets finished since the previous call, in completion order: up to `cap`
 * of them are written to tickets[] and *count says how many; the rest stay for
 * the next call.  Lets a caller with many requests in flight poll only the
 * finished ones. */
GABP_API gabp_status gabp_server_completed(gabp_server_t s, int64_t* tickets, int32_t cap, int32_t* count);
/* Host wall time (ms) spent in the phases of gabp_server_step since the
 * server was created: out8 = {admission (device allocation, input copies,
 * formation launches), activation, round-list rebuilds, rounds (the chunk and
 * its wait), stop handling (final residuals, refinement, retiring), total,
 * number of steps, number of list rebuilds}. */
GABP_API gabp_status gabp_server_phases(gabp_server_t s, double* out8);
GABP_API gabp_status gabp_server_destroy(gabp_server_t s);

/*
 * Instrumentation.  gabp_svm_set_profiling(h, k): k = 0 off; k >= 1 brackets
 * the pair-sweep kernel of every k-th round (rounds k-1, 2k-1, ... of each
 * captured chunk; k = 1: every round) by CUDA events recorded on the handle's
 * stream inside the captured graphs, and sums their device time here (the
 * counts below are of the bracketed sweeps).  Each event pair costs the graph
 * a few microseconds, so a stride above 1 keeps the timed solve close to an
 * unprofiled one.  k < 0 is GABP_EINVAL.  kernel_launches counts every kernel
 * the handle has launched since create (always on).
 */
typedef struct {
    int64_t sweep_launches;            /* pair sweeps timed */
    int64_t sweep_launches_zero_state; /* of which the first round (messages all 0, not read) */
    int64_t sweep_launches_p_frozen;   /* of which rounds after the P messages reached their fixed
                                          point (P read, not written) */
    double  sweep_ms;                  /* their summed device time */
    int64_t kernel_launches;           /* all kernels launched by this handle */
} gabp_svm_profile;

GABP_API gabp_status gabp_svm_set_profiling(gabp_svm_t h, int32_t on);
/* Copies the counters; reset != 0 zeroes the timing counters afterwards. */
GABP_API gabp_status gabp_svm_get_profile(gabp_svm_t h, gabp_svm_profile* out, int32_t reset);

/*
 * Decision values with no device allocation (the paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * e.g. plugins inside a host framework that owns all device memory through
 * its own allocator, or serving loops that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree imply).
 *
 * Computes out[s] = sum_i alpha_i y_i (exp(-gamma ||x_i - xt_s||^2) + lambda^2)
 * for s < t, like gabp_svm_decision, but without a handle.  All pointers are
 * DEVICE memory owned by the caller: X (n x m FP32, row-major), y and alpha
 * (n FP32), Xtest (t x m FP32), out (t FP32).  stream is a cudaStream_t (NULL =
 * legacy default stream); the call returns after its work has completed.
 *
 * Temporaries live in one fixed 4 MiB array in device memory that every GPU
 * which loads this library holds until the process exits; the call calls no
 * cudaMalloc, cudaFree or allocating library routine.  Sizes must satisfy
 * n + t + ceil(n/128) * t <= 1048576 floats, else GABP_EINVAL (split the test
 * rows into smaller calls).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current.  Every
 * call shares the array and keeps the last call's contents: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.
 */
GABP_API gabp_status gabp_decision_noalloc(const float* X, const float* y, const float* alpha,
                                           int64_t n, int64_t m, const float* Xtest, int64_t t,
                                           double gamma, double lambda, float* out, void* stream);

/*
 * Failure-detection self test (no counterpart in the paper): launches one
 * kernel whose thread waits, with the bounded wait that the pair sweep uses
 * for its shared-memory pipeline, on a barrier that nothing ever completes.
 * Returns GABP_ETIMEOUT after about limit_ns nanoseconds (0 < limit_ns <= 1e10)
 * with the CUDA context still usable; any other result means the bounded
 * wait is broken.
 */
GABP_API gabp_status gabp_selftest_bounded_wait(int64_t limit_ns);

/*
 * Numerics self test (no counterpart in the paper): out[i] = the reciprocal
 * the pair sweep uses for the cavity precisions (hardware approximation
 * refined by one Newton-Raphson step), for cnt positive FP32 inputs (host
 * arrays).  Tests compare it with IEEE division.
 */
GABP_API gabp_status gabp_selftest_reciprocal(const float* d, float* out, int64_t cnt);

/* Frees everything the handle owns. NULL is accepted. */
GABP_API gabp_status gabp_svm_destroy(gabp_svm_t h);

/* Message of the last failing call on this thread ("" if none). */
GABP_API const char* gabp_last_error(void);

/* GABP_SVM_VERSION of the loaded library. */
GABP_API int32_t gabp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GABP_SVM_H */
