/*
 * fth.h -- C ABI of the GB300 f-thermostat (FTH) library (libfth.so).
 *
 * The f-thermostat (Nava, Ceriotti, Dryzun, Parrinello, "Evaluating functions of
 * positive-definite matrices using colored noise thermostats") estimates elements of
 * f(M) for a symmetric positive-definite M.  M is the Hessian of the harmonic
 * potential V(q) = q^T M q / 2 (Eq. 5); every Cartesian degree of freedom carries the
 * same Markovian generalized-Langevin thermostat (Eq. 2) with drift A_p and
 * free-particle covariance C_p (Eq. 4), fitted so that a normal mode of frequency w
 * has momentum fluctuations <p^2>(w) = f(w^2).  Then <p_i p_j> = f(M)_ij (Eq. 6), and
 * averaging over time and over R independent replicas gives the estimate.
 *
 * Integrator: the modified velocity Verlet scheme the paper cites; per step
 *   O(dt/2) B(dt/2) A(dt) [F = -M q] B(dt/2) O(dt/2)
 * with O: (p, s) <- T (p, s) + S xi,  T = exp(-A_p dt/2),  S S^T = C_p - T C_p T^T,
 * S lower triangular (a pivot at or below 1e-14 of the largest diagonal entry is an
 * exact zero), xi standard normals from Philox4x32-10 (counter (kappa, i, r, k), key
 * = seed) through Box-Muller.  Samples of p (or q) are taken at the end of each step.
 * The two O half-steps around a sample (end of step kappa-1, start of step kappa) are
 * drawn jointly from their exact joint law with s + 2 normals of kappa (same Markov
 * chain as two independent half-steps); the first step's start half uses s + 1.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an fth_status; none aborts.  After an error,
 *    fth_last_error(ctx) describes it (ctx may be NULL for create-time errors, then
 *    the message is thread-local).
 *  - Host buffers belong to the caller and are only read during the call.
 *  - Device memory: the library allocates none.  The caller provides one device
 *    workspace of fth_workspace_size() bytes (e.g. a torch uint8 tensor) that must
 *    outlive the context; all state, copies of M, samples and accumulators live there.
 *  - Work is enqueued on opt.stream (a cudaStream_t, NULL = legacy default stream);
 *    fth_run returns once enqueued.  Calls that return data synchronise that stream.
 *  - Results are FP64.  (i, j) and (j, i) name the same element.
 *  - A context is not thread-safe: use one per host thread.
 *  - State planes exchanged with the host use the replica-major layout [R][N]
 *    (s: [R][s][N]) in FP64.
 */
#ifndef FTH_H
#define FTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fth_ctx fth_ctx;

typedef enum {
    FTH_OK = 0,
    FTH_E_INVALID_ARG = 1,   /* bad size, pointer, enum value or GLE               */
    FTH_E_NOT_SPD = 2,       /* M fails the positive-definiteness precondition     */
    FTH_E_UNSUPPORTED = 3,   /* valid request with no kernel here (e.g. s > 4)     */
    FTH_E_WORKSPACE = 4,     /* workspace NULL, misaligned or too small            */
    FTH_E_CUDA = 5,          /* a CUDA runtime call failed                         */
    FTH_E_TIMEOUT = 6,       /* a device wait gave up (bounded spin)               */
    FTH_E_NONFINITE = 7,     /* NaN/Inf found in the accumulators at a block flush */
    FTH_E_NOT_TRACKED = 8    /* fth_elements asked for an unregistered element     */
} fth_status;

enum fth_matrix_kind { FTH_DENSE = 0, FTH_CSR = 1 };
enum fth_dtype { FTH_F32 = 0, FTH_F64 = 1 };

/* Arithmetic of the force F = -M Q (all forms accumulate in FP32 except FP64):
 *   FP32    plain FP32 FFMA GEMM / SpMM;
 *   TF32    tcgen05 kind::tf32 tensor-core GEMM (dense only);
 *   BF16X3  tcgen05 kind::f16 with split BF16 operands, hi*hi + hi*lo + lo*hi (dense only);
 *   FP64    FP64 state and arithmetic, one CTA per replica (dense, N <= 1024).
 * With FTH_TRACK_ALL the TF32 and BF16X3 forms also accumulate every element on the
 * tensor cores: the samples are staged rounded to nearest BF16 (8 significant bits) and
 * their products summed in FP32.  A product's rounding error is at most 2^-7 of it and
 * averages out over samples up to a bias of order 1e-5 of the element (Gaussian
 * samples: about -4.5e-6); FP32 accumulates in FFMA, FP64 in FP64.     */
enum fth_precision { FTH_PREC_FP32 = 0, FTH_PREC_TF32 = 1, FTH_PREC_BF16X3 = 2, FTH_PREC_FP64 = 3 };

/* Which elements of <x x^T> are accumulated (sized at create, paper's "2A" reals):
 *   LIST  the opt.pairs list;  DIAG  all (i, i);  ALL  every element (dense only).  */
enum fth_track { FTH_TRACK_LIST = 0, FTH_TRACK_DIAG = 1, FTH_TRACK_ALL = 2 };

/* Sampled variable: p (Eq. 6, default) or q. */
enum fth_observable { FTH_OBS_P = 0, FTH_OBS_Q = 1 };

enum fth_plane { FTH_PLANE_Q = 0, FTH_PLANE_P = 1, FTH_PLANE_S = 2 };

typedef struct {
    int kind;               /* FTH_DENSE or FTH_CSR                                       */
    int dtype;              /* FTH_F32 or FTH_F64: element type of `values`               */
    int on_device;          /* 0: host pointers; 1: device pointers                       */
    int64_t n;              /* order N >= 1                                               */
    int64_t nnz;            /* CSR: number of stored entries                              */
    const void* values;     /* dense: N*N row-major; CSR: nnz values                      */
    const int32_t* rowptr;  /* CSR: N+1 offsets, rowptr[0] = 0, non-decreasing            */
    const int32_t* colind;  /* CSR: nnz column indices in [0, N)                          */
} fth_matrix;

typedef struct {
    int s;                  /* auxiliary momenta per dof, 0 <= s <= 4                      */
    double a_p[25];         /* drift A_p, (s+1)x(s+1) row-major in the leading entries     */
    double c_p[25];         /* free-particle covariance C_p, (s+1)x(s+1) row-major         */
} fth_gle;

typedef struct {
    int64_t replicas;       /* R >= 1 independent replicas                                 */
    uint64_t seed;          /* Philox key                                                  */
    double dt;              /* time step > 0                                               */
    int64_t burnin;         /* samples discarded before accumulation starts                */
    int64_t block;          /* samples per block for the error bars (>= 1)                */
    int observable;         /* enum fth_observable                                        */
    int precision;          /* enum fth_precision                                         */
    int track;              /* enum fth_track                                             */
    const int64_t* pairs;   /* LIST: host array of 2*npairs indices (i, j)                */
    int64_t npairs;
    int64_t stack;          /* samples staged before one accumulation pass (0 = auto: 4096
                             * BF16 columns / Rp on the tensor-core all-elements paths, 2048 /
                             * Rp on the FFMA one, 4 for element lists)                   */
    void* stream;           /* cudaStream_t                                               */
    int64_t replica_offset; /* global index of replica 0 in the noise counter: a run split
                               across processes with offsets 0, R, 2R, ... draws exactly the
                               noise of one run with all replicas                          */
} fth_options;

typedef struct {
    int64_t steps;          /* completed steps                                             */
    int64_t samples;        /* samples taken (burn-in included)                            */
    int64_t accumulated;    /* samples accumulated                                         */
    int64_t blocks;         /* completed blocks                                            */
    int64_t launches;       /* kernels launched by this context so far                     */
    int primed;             /* 1 if the start half of the next step is already applied     */
    int precision;          /* precision actually used                                     */
    int64_t n, replicas, tracked;
    size_t workspace_bytes;
} fth_info_t;

/* Bytes of device workspace fth_create needs for this problem (no device access).
 * Passage: none (device memory of this library; the paper's program ran on CPUs). */
fth_status fth_workspace_size(const fth_matrix* M, const fth_gle* gle, const fth_options* opt,
                              size_t* bytes);

/* Validate the problem, build T and S in FP64 on the host, copy M into the workspace
 * (converted/rounded for the chosen precision) and zero the state: q = p = s = 0 at a
 * step boundary.  `workspace` must be 256-byte aligned device memory of at least
 * fth_workspace_size() bytes.  Enqueues its copies on opt->stream and returns after they
 * completed.  A dense M is checked and converted on the device: read in place when
 * M->on_device (it must stay valid until fth_create returns), else copied in row chunks
 * through the part of the workspace that the state will occupy.  A host M is read and
 * not kept.
 * Errors: INVALID_ARG (also non-finite entries), NOT_SPD (a diagonal entry <= 0),
 * UNSUPPORTED, WORKSPACE, CUDA.
 * Passage: Eq. 5 (M is the Hessian of the harmonic potential), Eq. 2 and Eq. 4 (the GLE
 * fixed by A_p and C_p), and the velocity Verlet GLE integrator Sec. "The f-thermostat"
 * cites. */
fth_status fth_create(const fth_matrix* M, const fth_gle* gle, const fth_options* opt,
                      void* workspace, size_t workspace_bytes, fth_ctx** out);

/* Advance the dynamics by `steps` steps, taking one sample per step (the hot path:
 * force, B, O, sample, O, B, A per step, plus one accumulation pass per `stack`
 * samples and one FP64 block flush per completed block).  Asynchronous.  Each launch
 * carries per-step values that the context tracks on the host (kick index, stack slot),
 * so the launches of a call are not meant to be
 * captured into a CUDA graph and replayed; fth_dense_step_noalloc is the entry point for
 * capture.
 * Passage: Eq. 2 integrated for every degree of freedom of every replica under the force
 * of Eq. 5; the samples are the ones Eq. 6 averages. */
fth_status fth_run(fth_ctx* ctx, int64_t steps);

/* Estimates of <x_i x_j> for k pairs (2k indices): values[e] = mean over every
 * accumulated sample and replica; errbars[e] = standard error of the mean of the
 * completed block means (NaN with fewer than 2 blocks).  Synchronises the stream.
 * Errors: NOT_TRACKED if a pair is not accumulated, NONFINITE, CUDA.
 * Passage: Eq. 6, averaged over time and replicas; the block error bar estimates the
 * statistical error whose sqrt(tau / t) scaling Sec. "Results and benchmarks" discusses. */
fth_status fth_elements(fth_ctx* ctx, const int64_t* pairs, int64_t k, double* values,
                        double* errbars);

/* Copy one state plane to / from the host in FP64, layout [R][N] ([R][s][N] for s).
 * Passage: none (state access for checks and restarts). */
fth_status fth_get_state(fth_ctx* ctx, int plane, double* host);

/* Linear functionals of tracked elements, L = sum_k w_k <x_{i_k} x_{j_k}>: the trace
 * estimators of Sec. "The f-thermostat" -- Tr f(M) = <p^T p> (unit weights on the
 * diagonal) and Tr O f(M) = <p^T O p> (w = O_ii on (i, i), 2 O_ij on (i < j) for a
 * symmetric O) -- with their own block error bar: at every block flush the block value
 * of L is folded into FP64 Welford sums, so correlations between the terms are kept.
 * Every (i, j) must be tracked (NOT_TRACKED otherwise).  Add before the first sample is
 * accumulated.  Device storage: `device_buffer` (caller-owned, 256-byte aligned, at
 * least fth_functional_bytes(nterms) bytes, kept until the context is destroyed). */
size_t fth_functional_bytes(int64_t nterms);
fth_status fth_functional_add(fth_ctx* ctx, const int64_t* pairs, const double* weights,
                              int64_t nterms, void* device_buffer, size_t bytes, int64_t* id);
/* Value (all accumulated samples, as fth_elements) and block error bar (NaN before two
 * complete blocks).  Synchronises the stream. */
fth_status fth_functional(fth_ctx* ctx, int64_t id, double* value, double* errbar);

/* The trace estimators with their weights built by the library: Tr O f(M) = <p^T O p>
 * for a symmetric O of the context's order (dense or CSR, host or device buffers, FP32
 * or FP64; entries on and above the diagonal are read, w = O_ii on (i, i) and 2 O_ij on
 * (i < j), zero entries dropped), or Tr f(M) when O is NULL.  _terms gives the number of
 * terms, so the caller can size the device buffer with fth_functional_bytes; _add then
 * registers the functional as fth_functional_add does (same rules and errors, plus
 * INVALID_ARG for an O that does not fit the context or has non-finite entries). */
fth_status fth_functional_operator_terms(fth_ctx* ctx, const fth_matrix* O, int64_t* nterms);
fth_status fth_functional_add_operator(fth_ctx* ctx, const fth_matrix* O, void* device_buffer,
                                       size_t bytes, int64_t* id);

/* Reusing one fitted GLE for other spectra (Sec. "The f-thermostat"): with
 * A_p -> alpha A_p and C_p -> gamma C_p, the estimate for the input r M + m I is
 * gamma f((r M + m I) / alpha^2).  fth_spectral_map gives (r, m) with r lo + m = lo_target
 * and r hi + m = hi_target (the shift printed in the paper has its sign flipped; this is
 * the corrected form).  fth_gle_scale writes (alpha A_p, gamma C_p); in and out may be the
 * same struct.  Errors: INVALID_ARG. */
fth_status fth_spectral_map(double lo, double hi, double lo_target, double hi_target, double* r,
                            double* m);
fth_status fth_gle_scale(const fth_gle* in, double alpha, double gamma, fth_gle* out);

/* Inverse transforms of the paper's benchmarks, from the sampled elements (or trace) to
 * the wanted ones:
 *   LOG_SCALED    params {r}:    ln M = ln(r M) - I ln r (diagonal elements lose ln r;
 *                                the trace loses n ln r; error bars unchanged);
 *   EXP_SHIFTED   params {a, m}: exp(-a M) = exp(-a (M + m I)) e^{a m} (values and error
 *                                bars times e^{a m});
 *   POWER_SCALED  params {r, k}: f(M) = f(r M) r^-k for f(x) = x^k (values and error bars
 *                                times r^-k).
 * Elements: `pairs` (2k indices, as fth_elements) name the elements of values / errbars
 * (errbars may be NULL), transformed in place.  Trace: n is the order.  Errors:
 * INVALID_ARG. */
enum fth_untransform_kind { FTH_U_LOG_SCALED = 0, FTH_U_EXP_SHIFTED = 1, FTH_U_POWER_SCALED = 2 };
fth_status fth_untransform(int kind, const double* params, const int64_t* pairs, int64_t k,
                           double* values, double* errbars);
fth_status fth_untransform_trace(int kind, const double* params, int64_t n, double* value,
                                 double* errbar);
fth_status fth_set_state(fth_ctx* ctx, int plane, const double* host);

/* Context housekeeping (info, error word, messages, release).  Passage: none. */

/* Counters and configuration of a context. */
fth_status fth_info(const fth_ctx* ctx, fth_info_t* info);

/* Synchronise and report the device error word (TIMEOUT, NONFINITE) or FTH_OK. */
fth_status fth_status_poll(fth_ctx* ctx);

/* Last error message of ctx (or of this thread when ctx is NULL). */
const char* fth_last_error(const fth_ctx* ctx);

/* Release host resources; the caller then frees the workspace. */
void fth_destroy(fth_ctx* ctx);

/* The library's own O half-step constants in FP64: T = exp(-A_p dt/2) (Pade scaling
 * and squaring) and lower-triangular S with S S^T = C_p - T C_p T^T; (s+1)^2 each.
 * Passage: the thermostat part of Eq. 2 for A_p and C_p (Eq. 4), as the exact
 * Ornstein-Uhlenbeck half-step of the integrator Sec. "The f-thermostat" cites. */
fth_status fth_gle_propagator(const fth_gle* gle, double dt, double* T, double* S);

/* ----------------------------------------------------------------------------------
 * GLE fitting (host, FP64; no device work).  The paper fits the drift A_p and the
 * free-particle covariance C_p so that a normal mode of eigenvalue lambda = w^2 has
 * <p^2>(w) = f(lambda) over the spectrum of M (Sec. "The f-thermostat", the fitting
 * paragraph; Eq. 2, Eq. 4), starting from delta-like memory kernels and then refining the
 * general form, under the requirements of Sec. "Results and benchmarks": follow f over
 * the range, treat f below delta * max f as an upper bound only (the exponential-tail
 * rule), and keep correlation times short.  The fitted response is that of this
 * library's integrator at the given dt (stationary covariance of the sample-to-sample
 * map of each mode), so it carries no finite-dt error.
 * ---------------------------------------------------------------------------------- */
enum fth_function {
    FTH_F_INV_SQRT = 0,     /* x^(-1/2)                                      (no params) */
    FTH_F_FERMI = 1,        /* 1 / (1 + exp(beta (x - mu)))         params: beta, mu     */
    FTH_F_LOG = 2,          /* ln x (the range must have lambda_min > 1) (no params)     */
    FTH_F_EXP = 3,          /* exp(-alpha x)                        params: alpha        */
    FTH_F_POWER = 4         /* x^k                                  params: k            */
};

enum fth_fit_objective {
    FTH_FIT_AUTO = 0,       /* ABS for FERMI, LOG otherwise                              */
    FTH_FIT_LOG = 1,        /* residuals ln(gamma g / f): relative error                 */
    FTH_FIT_ABS = 2         /* residuals (gamma g - f) / max f: absolute error           */
};

/* Options of fth_fit_gle.  A zeroed struct means: observable P, 120 grid points, 6
 * starts, 400 iterations, delta 1e-3, no correlation-time penalty, seed 0, all host
 * threads, objective AUTO.  Passing NULL gives the same with w_tau = 0.2. */
typedef struct {
    int observable;         /* enum fth_observable: the moment fitted                      */
    int npts;               /* log-spaced grid points over [lambda_min, lambda_max]        */
    int starts;             /* seeded delta-like starts                                    */
    int max_iter;           /* Levenberg-Marquardt iterations per start                    */
    double delta;           /* tail threshold, relative to max f over the grid             */
    double w_tau;           /* weight of the penalty ln(max(1, tau_max / tau_ref)), tau_ref =
                               2.5 / (sqrt(lambda_min) dt) samples (>= 0)                  */
    uint64_t seed;          /* seed of the starts                                          */
    int threads;            /* host threads running the starts (0: all)                    */
    int objective;          /* enum fth_fit_objective                                      */
} fth_fit_options;

typedef struct {
    double max_rel_err;     /* max |gamma g / f - 1| over grid points with f >= delta max f */
    double rms_rel_err;     /* rms of the same                                             */
    double max_abs_err;     /* max |gamma g - f| / max f over the whole grid               */
    double tail_max;        /* max gamma g / max f where f < delta max f (0 if none)       */
    double tau_max;         /* largest integrated correlation time of the sampled x^2 over
                               the grid, in samples (steps)                                */
    double lambda_tau_max;  /* eigenvalue where tau_max is reached                         */
    double cost;            /* final least-squares cost                                    */
    int64_t evaluations;    /* response evaluations over all starts                        */
    int grid;               /* grid points                                                 */
    int objective;          /* FTH_FIT_LOG or FTH_FIT_ABS, as used                         */
} fth_fit_report;

/* Fit a GLE with s auxiliary momenta (1 <= s <= 4) to f over [lambda_min, lambda_max]
 * for time step dt; writes out (s, A_p, C_p, with the overall scale gamma folded into
 * C_p) and, if report is not NULL, the fit's quality.  Deterministic for a given seed
 * and option set.  Errors: INVALID_ARG (bad range, lambda_max dt^2 >= 4, parameters or
 * options, f not finite or negative on the grid), UNSUPPORTED (no start gave a valid GLE). */
fth_status fth_fit_gle(int f_kind, const double* f_params, double lambda_min, double lambda_max,
                       int s, double dt, const fth_fit_options* opt, fth_gle* out,
                       fth_fit_report* report);

/* The exact per-mode response of this library's integrator for a GLE at time step dt:
 * for each eigenvalue lambda[e] > 0, g[e] = stationary <x^2> of the sampled observable
 * (x = p or q) and, if tau is not NULL, tau[e] = its integrated correlation time of x^2
 * in samples, 1 + 2 sum_{l >= 1} corr(x^2(0), x^2(l)).  With U diag(g) U^T (M = U diag
 * (lambda) U^T) this is the value the estimate converges to (Eq. 6 for the fitted GLE),
 * and tau sets the block length the error bars need (blocks much longer than tau).
 * Errors: INVALID_ARG (bad arguments, lambda dt^2 >= 4 where velocity Verlet has no
 * stationary state, or a GLE whose chain has none). */
fth_status fth_gle_response(const fth_gle* gle, double dt, int observable, const double* lambda,
                            int64_t n, double* g, double* tau);

/* Kernel classes reported by fth_profile_read. */
enum fth_kernel_class {
    FTH_K_FORCE_FP32 = 0,   /* FFMA force GEMM                                  */
    FTH_K_FORCE_TC = 1,     /* tcgen05 force GEMM (TF32 or split BF16)          */
    FTH_K_GLE_DENSE = 2,    /* element-wise fused GLE step, dense path           */
    FTH_K_CSR_STEP = 3,     /* fused CSR SpMM + GLE step                         */
    FTH_K_PAIR_ACCUM = 4,   /* pair-list accumulation pass                       */
    FTH_K_SYRK_FP32 = 5,    /* FFMA all-elements accumulation pass               */
    FTH_K_SYRK_TC = 6,      /* tcgen05 all-elements accumulation pass            */
    FTH_K_FLUSH = 7,        /* FP64 block flush                                  */
    FTH_K_FP64_DENSE = 8,   /* FP64 one-CTA-per-replica segment                  */
    FTH_K_FP64_NOISE = 9,   /* FP64 normals of a segment, generated ahead        */
    FTH_K_CLASSES = 10
};

/* Enable (1) or disable (0) CUDA-event timing of every kernel the context launches:
 * one event pair around each launch on the context's stream (off by default).
 * Passage: none (measurement), as for fth_profile_read and fth_test_stall. */
fth_status fth_profile_enable(fth_ctx* ctx, int enable);

/* Synchronise, then return per kernel class the summed device milliseconds and the
 * launch counts recorded since the last read (arrays of FTH_K_CLASSES entries). */
fth_status fth_profile_read(fth_ctx* ctx, double* ms, int64_t* launches);

/* Test hook for the device timeout path (tensor-core dense contexts only).  With
 * limit_ns > 0 the context's next force launches issue no operand copies, so the waits
 * of their main loop, which nothing completes, give up after limit_ns: each CTA sets
 * FTH_E_TIMEOUT in the context's error word, issues nothing more, frees its tensor
 * memory and returns (nothing is in flight, so no GPU fault is possible).  The error
 * word is sticky: fth_status_poll and fth_elements report FTH_E_TIMEOUT from then on,
 * because the steps that ran without a force are not valid.  0 restores normal
 * launches.  Errors: INVALID_ARG (limit above the 1 s bound), UNSUPPORTED (no
 * tensor-core force in this context). */
fth_status fth_test_stall(fth_ctx* ctx, uint64_t limit_ns);

/* One dense FP32 fused launch that allocates nothing, for callers that cannot allocate
 * device memory: a plugin whose host framework owns all device memory through its own
 * pool, a real-time loop that must never enter an allocator, or code that can only pass
 * pointers it already owns.  No workspace is taken; the intermediate force M q lives in
 * a library-owned static device array of 4,194,304 floats (16 MiB) per device, kept
 * until the process exits.  The paper has no counterpart: this is only an allocation
 * policy of the library.
 *
 * Computes, on device buffers the caller owns (all FP32, 16-byte aligned):
 *   mode 0: MQ = M q; end of the current step (B, O, sample) and start of the next
 *           (O, B, A) with kick index kappa, exactly as one step of fth_run;
 *   mode 1: MQ = M q; only the start half (the prologue of a fresh run).
 * M: [n][ldm] row-major.  q, p: [n][ldr], replica fastest, ldr >= replicas, ldr % 4 == 0.
 * s: s_aux planes of [n][ldr], contiguous.  sample (mode 0, may be NULL): [n][ldr] gets p
 * at the end of the step.  T, S: (s_aux+1)^2 FP64 from fth_gle_propagator.  Noise is the
 * same Philox stream as fth_run with the same seed (replica offset 0).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress
 * with that device current); make that first call before any stream capture.  Every
 * call shares the one array and leaves its last contents there; each call overwrites
 * every entry it reads, so nothing needs clearing.  Calls that overlap on the GPU (two
 * streams, or two host threads on one device) race on the array: serialise them.
 * Errors: INVALID_ARG (pointers, sizes, alignment), UNSUPPORTED when n * ldr exceeds the
 * array (4,194,304 floats) or ldr exceeds 2,097,120 (65,535 tiles of 32 replicas), both
 * checked before any device work, CUDA. */
fth_status fth_dense_step_noalloc(const float* M, int64_t n, int64_t ldm, float* q, float* p,
                                  float* s, int64_t replicas, int64_t ldr, int s_aux,
                                  const double* T, const double* S, double dt, uint64_t seed,
                                  uint32_t kappa, int mode, float* sample, void* stream);

/* ----------------------------------------------------------------------------------
 * Passage: Sec. "Final discussion" (independent simulations that run side by side); the
 * arithmetic per problem is that of fth_create / fth_run.
 * Problem pools: many independent problems resident on one device and stepped together
 * (ragged batches, continuous batching).  Problems of different order and kind (dense
 * or CSR) share one set of launches per step: a persistent tensor-core force kernel
 * over a work list of (problem, 128-row block) items for the dense ones, one
 * element-wise GLE kernel, one fused CSR kernel, one accumulate/flush kernel with a CTA
 * per problem.  Every launch reads its inputs from a device descriptor table, so a
 * chunk of steps is replayed from a captured CUDA graph.  Problems are added and
 * removed between runs; admission fails with FTH_E_WORKSPACE when the problem's
 * footprint does not fit the free part of the pool's workspace.  A problem's noise
 * (key = its seed, replicas from its replica_offset) and arithmetic do not depend on
 * the other problems: its results are identical alone and in any mix.  Its first
 * pool step is its prologue (start half only), as on a fresh fth_ctx.
 * ---------------------------------------------------------------------------------- */
typedef struct fth_pool fth_pool;

typedef struct {
    int64_t replicas;       /* R of every problem: 32, 64 or 128                          */
    int precision;          /* dense force: FTH_PREC_BF16X3 or FTH_PREC_TF32 (CSR: FP32)   */
    int64_t max_problems;   /* capacity of the problem table                              */
    int64_t graph_steps;    /* steps per captured CUDA graph (0: direct launches)         */
    void* stream;           /* cudaStream_t                                               */
} fth_pool_options;

typedef struct {
    uint64_t seed;          /* Philox key of this problem                                 */
    double dt;
    int64_t burnin;         /* samples discarded                                          */
    int64_t block;          /* samples per block                                          */
    int observable;         /* enum fth_observable                                        */
    const int64_t* pairs;   /* tracked elements (2 * npairs indices, host)                */
    int64_t npairs;
    int64_t replica_offset; /* global index of replica 0 in the noise counter              */
} fth_problem_options;

typedef struct {
    int64_t live;           /* problems in the pool                                        */
    size_t slab_bytes;      /* workspace available to problems                            */
    size_t used_bytes;      /* of which allocated                                          */
    int64_t force_items, gle_items, csr_items;
    int tuned_variant;      /* force-kernel configuration chosen by the autotuner          */
    int tuned_grid;
    double tuned_us;        /* its measured time per force launch                          */
    int gle_variant;        /* dense GLE kernel configuration chosen by the autotuner      */
    double gle_us;          /* its measured time per launch                                */
    int64_t graphs;         /* CUDA graphs captured so far                                 */
} fth_pool_stats_t;

/* Create an empty pool on `workspace` (256-byte aligned device memory the caller owns
 * for the pool's lifetime).  Errors: INVALID_ARG, WORKSPACE, UNSUPPORTED, CUDA. */
fth_status fth_pool_create(const fth_pool_options* opt, void* workspace, size_t bytes,
                           fth_pool** out);

/* Device bytes a problem would take in this pool (admission by footprint). */
fth_status fth_pool_footprint(const fth_pool* pool, const fth_matrix* M, const fth_gle* gle,
                              const fth_problem_options* po, size_t* bytes);

/* Validate and add a problem (copies M, zero state); *handle identifies it.
 * Errors: INVALID_ARG, NOT_SPD, UNSUPPORTED, WORKSPACE (does not fit: not admitted), CUDA. */
fth_status fth_pool_add(fth_pool* pool, const fth_matrix* M, const fth_gle* gle,
                        const fth_problem_options* po, int64_t* handle);

/* Remove a problem and free its memory (between runs). */
fth_status fth_pool_remove(fth_pool* pool, int64_t handle);

/* Advance every problem by `steps` launches (asynchronous on the pool's stream). */
fth_status fth_pool_run(fth_pool* pool, int64_t steps);

/* As fth_elements, for one problem of the pool.  Synchronises the stream. */
fth_status fth_pool_elements(fth_pool* pool, int64_t handle, const int64_t* pairs, int64_t k,
                             double* values, double* errbars);

/* Copy one state plane of a problem to host FP64, laid out as fth_get_state: q and p
 * [R][n], s [R][s][n].  Synchronises the stream. */
fth_status fth_pool_get_state(fth_pool* pool, int64_t handle, int plane, double* host);

/* Convergence of every problem in one device pass: for each handle slot h
 * (0 <= h < max_problems), rel_err[h] = sqrt(sum_e sigma_e^2) / sqrt(sum_e mean_e^2)
 * over the problem's tracked elements (sigma_e the block error bar, mean_e the mean of
 * the complete blocks; NaN before 2 blocks, and for empty slots) and blocks[h] = its
 * number of complete blocks (-1 for empty slots; may be NULL).  Synchronises. */
fth_status fth_pool_progress(fth_pool* pool, double* rel_err, int64_t* blocks);

/* Counters of one problem (steps, samples, blocks ...).  Synchronises the stream. */
fth_status fth_pool_problem_info(fth_pool* pool, int64_t handle, fth_info_t* info);

fth_status fth_pool_stats(const fth_pool* pool, fth_pool_stats_t* stats);

/* Kernel classes of a pool step, for fth_pool_profile. */
enum fth_pool_kernel { FTH_PK_FORCE = 0, FTH_PK_GLE = 1, FTH_PK_CSR = 2, FTH_PK_ACCUM = 3,
                       FTH_PK_CLASSES = 4 };

/* Advance every problem by `steps` steps as direct launches with a CUDA event pair
 * around each launch (on the pool's stream), and return per kernel class the summed
 * device time in ms (`ms[FTH_PK_CLASSES]`) and the number of launches
 * (`launches[FTH_PK_CLASSES]`, may be NULL).  The steps are real steps.  Synchronises. */
fth_status fth_pool_profile(fth_pool* pool, int64_t steps, double* ms, int64_t* launches);
const char* fth_pool_last_error(const fth_pool* pool);
void fth_pool_destroy(fth_pool* pool);

/* ----------------------------------------------------------------------------------
 * Passage: none beyond the pool's (a scheduling policy over independent problems; the
 * retirement rule is the block error bar of fth_elements).
 * Serving loop over a pool: requests are queued on submit, admitted into the pool when
 * a slot and enough workspace are free (arrival order; a request that does not fit is
 * passed by later ones at most max_bypass times), stepped together with all others
 * (continuous batching), and retired when the normwise relative error bar of their
 * tracked elements (fth_pool_progress) is <= their target with at least min_blocks
 * complete blocks, or when their step budget is spent.  Host code only; the GPU work
 * is the pool's.  Results are those the same problem gives alone in a pool.
 * ---------------------------------------------------------------------------------- */
typedef struct fth_server fth_server;

enum fth_request_state { FTH_REQ_QUEUED = 0, FTH_REQ_RUNNING = 1, FTH_REQ_DONE = 2,
                         FTH_REQ_BUDGET = 3 /* retired at max_steps above target */,
                         FTH_REQ_FAILED = 4 /* rejected by validation */ };

typedef struct {
    fth_pool_options pool;
    int64_t chunk_steps;    /* steps between admission / retirement checks (>= 1)          */
    int64_t min_blocks;     /* complete blocks needed before a target counts (>= 2)        */
    int64_t max_bypass;     /* times a waiting request may be passed by later ones         */
} fth_server_options;

typedef struct {
    int64_t admitted, retired, running, queued;  /* this step; now                      */
    int64_t steps;                               /* server steps so far                 */
    size_t used_bytes, slab_bytes;               /* pool workspace occupancy            */
} fth_server_counts;

typedef struct {
    int state;              /* enum fth_request_state                                      */
    int64_t steps;          /* steps run (so far)                                          */
    double rel_err;         /* normwise relative error bar at the last check               */
    double t_submit, t_admit, t_done;   /* seconds on the server clock                      */
    int64_t npairs;
} fth_request_info;

/* Create a server and its pool on `workspace` (as fth_pool_create). */
fth_status fth_server_create(const fth_server_options* opt, void* workspace, size_t bytes,
                             fth_server** out);

/* Queue a request (copies M and the pairs; po->npairs >= 1).  target > 0: relative
 * accuracy wanted; max_steps: step budget (0 = none).  *id numbers requests from 0. */
fth_status fth_server_submit(fth_server* srv, const fth_matrix* M, const fth_gle* gle,
                             const fth_problem_options* po, double target, int64_t max_steps,
                             int64_t* id);

/* One serving iteration: admit, run chunk_steps steps, retire.  Synchronises. */
fth_status fth_server_step(fth_server* srv, fth_server_counts* counts);

/* State of a request; when retired, its tracked elements (in its pair order) and their
 * error bars are copied to values / errbars (npairs each, may be NULL). */
fth_status fth_server_result(fth_server* srv, int64_t id, fth_request_info* info,
                             double* values, double* errbars);

double fth_server_clock(const fth_server* srv);     /* seconds since creation           */
fth_pool* fth_server_pool(fth_server* srv);         /* the server's pool (stats)        */
const char* fth_server_last_error(const fth_server* srv);
void fth_server_destroy(fth_server* srv);

/* Library version string. */
const char* fth_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FTH_H */
