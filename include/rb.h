/*
 * rb.h -- C ABI of the GB300 (sm_103a) greedy reduced-basis library.
 *
 * Method: Antil, Chen, Field, "A Note on QR-Based Model Reduction: Algorithm,
 * Software, and Gravitational Wave Applications", arXiv 1805.06124.
 *   - RB-greedy, Alg. 3 (Sec. 5.2.1), equivalent to MGS with column pivoting,
 *     Alg. 2 (Prop. 5.3): a column-pivoted QR of the snapshot matrix S.
 *   - pivot search with the incremental residual bookkeeping of Eq. (Residual)
 *     (Sec. 6.1.2): err_j = ||s_j||^2 - sum_l |c_lj|^2, c_lj = q_l^H s_j,
 *     norms and sums stored separately, no square roots in the argmax.
 *   - orthogonalisation of each pivot column by Hoffmann's iterated
 *     Gram-Schmidt (MGSCI, kappa = 2; Sec. 6.1.2 and the remark after
 *     Prop. 5.3).
 *   - stopping rule of Cor. 5.4: the max error equals R(k+1,k+1).
 *
 * Conventions shared by every entry point:
 *   - complex128 = two doubles (re, im) interleaved; complex64 = two floats.
 *   - S (the paper's N x M snapshot matrix) is column-major: snapshot j
 *     occupies S + j*ldS (in complex elements), N entries, ldS >= N.
 *   - Q is column-major N x kmax: basis vector q_l at Q + l*ldQ, ldQ >= N.
 *   - C is row-major kmax x M: C[l*ldC + j] = q_l^H s_j, ldC >= M.
 *   - c = q^H s (conjugate on the basis vector); |c|^2 = c c^*.
 *   - tol is a tolerance on the SQUARED error: a vector is appended only while
 *     max_j err_j >= tol, so every column ends with err_j < tol unless kmax
 *     or min(N, M) is reached first.
 *   - ties in the argmax go to the lowest column index; picked columns are
 *     excluded.
 *   - Pointers are DEVICE pointers unless an entry point says otherwise.  They
 *     are borrowed: the caller allocates them (outputs at capacity kmax) and
 *     keeps them valid until the call returns.  Inputs are never modified.
 *   - Calls are issued on the context's stream.  The greedy entry points
 *     synchronise that stream before returning (they return k and a status),
 *     as does rb_project; rb_generate and rb_split are asynchronous.
 *   - Return value: 0 = success, > 0 = warning (outputs valid), < 0 = error
 *     (outputs unspecified).  rb_last_error() describes the last failure.
 *     No call aborts the process or traps on the device; device-side waits
 *     are bounded and report RB_ETIMEOUT.
 *   - One context per host thread; a context is not thread-safe.
 */
#ifndef RB_GB300_H
#define RB_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rb_ctx rb_ctx;

typedef enum rb_status {
    RB_OK = 0,
    RB_KMAX_REACHED = 1,   /* warning: kmax vectors built, max err still >= tol */
    RB_EINVAL = -1,        /* bad argument (size, leading dimension, alignment, option) */
    RB_ENOMEM = -2,        /* device workspace could not be allocated */
    RB_ECUDA = -3,         /* a CUDA runtime call failed */
    RB_ENONFINITE = -4,    /* NaN or Inf in the input */
    RB_EORTHO = -5,        /* IMGS did not meet the kappa test within imgs_max_passes */
    RB_ETIMEOUT = -6,      /* a bounded device-side wait ran out */
    RB_ESTATE = -7         /* inconsistent device state */
} rb_status;

/* Sweep arithmetic of the FP64 form. */
enum {
    RB_SWEEP_DF32 = 0,  /* FP64-accurate double-float products on the FP32 pipe over a hi/lo copy of S */
    RB_SWEEP_FP64 = 1   /* plain FP64 (DFMA) products read straight from complex128 S */
};

/* rb_options.flags */
#define RB_FLAG_TIMING 1u        /* time every sweep launch with CUDA events (fills rb_result.ms_sweep) */
#define RB_FLAG_PROJECT_FP64 2u  /* rb_project on the plain-FP64 CUDA-core kernel instead of the tensor cores */
#define RB_FLAG_SPLIT_NO_SWITCH 4u /* rb_greedy_split never switches to hi + lo sweeps on the candidate count
                                      (it re-checks however many candidates the bounds admit) */

typedef struct rb_options {
    int device;            /* CUDA device ordinal */
    int sweep;             /* RB_SWEEP_DF32 (default) or RB_SWEEP_FP64 */
    double imgs_kappa;     /* MGSCI kappa, > 1 (default 2.0) */
    int imgs_max_passes;   /* cap on IMGS passes per vector, >= 1 (default 4) */
    double switch_err;     /* rb_greedy_split: switch to hi + lo sweeps once every error is certified below
                              switch_err * max_j ||s_j||^2 (the largest upper bound of the hi-only phase);
                              0 (default) = switch on the candidate count only.  Finite, >= 0 */
    int iters_per_sync;    /* iterations queued between host checks of the stop flag (default 8) */
    void *stream;          /* cudaStream_t; NULL = the context creates its own stream */
    unsigned flags;        /* RB_FLAG_* */
    int recompute_period;  /* FP64 form (rb_greedy, rb_greedy_host): every recompute_period iterations
                              acc_j = sum_l |C[l, j]|^2 is rebuilt from the stored coefficients with
                              compensated summation before the sweep (the periodic exact recompute of the
                              bookkeeping); 0 = off.  >= 0 (default 16) */
    int batched_variant;   /* rb_greedy_batched sweep: -1 (default) = chosen by the autotuner; otherwise
                              2 * v + c forces sweep variant v (0..5: complex128 read and split in
                              registers, 6..11: pre-split hi/lo copy; unroll 2 << (v % 3), block width
                              by v / 3 within each half) and c (0: 32, 1: 128 columns per chunk).
                              Forcing a pre-split variant when the copy does not fit in free device memory
                              returns RB_EINVAL.  In [-1, 23]. */
    unsigned long long timeout_cycles; /* budget of every device-side wait of the tensor-core kernels
                              (mbarrier waits), in SM clock cycles; a wait that runs out sets an error
                              flag, the kernel returns and the call reports RB_ETIMEOUT.  0 (default) =
                              2^31 cycles, about one second at 2 GHz; otherwise >= 2^20 (a shorter budget
                              could end a wait that is only slow) */
} rb_options;

/* Fills *opt with the defaults listed above. */
void rb_default_options(rb_options *opt);

typedef struct rb_result {
    /* ---- outputs: caller-allocated device buffers ---- */
    void *Q;               /* complex128 N x kmax, column-major, ldQ >= N (required) */
    long long ldQ;
    long long *pivots;     /* kmax entries: 0-based column indices in pick order (required) */
    double *err_curve;     /* kmax+1 entries: err_curve[l] = max err over unpicked columns after l
                              vectors; err_curve[0] = max_j ||s_j||^2; err_curve[l] = R(l+1,l+1)^2
                              (Cor. 5.4) (required) */
    void *C;               /* optional complex128 kmax x M row-major, ldC >= M: C = Q^H S */
    long long ldC;
    double *final_err;     /* optional, M entries: err_j after the last vector */
    double *rdiag;         /* optional, kmax entries: R(l,l) = ||v|| before normalisation */
    /* ---- filled by the call (host scalars) ---- */
    int k;                 /* number of basis vectors built */
    int imgs_passes;       /* total IMGS passes over all vectors */
    int switch_iter;       /* split form: basis size when C was completed on lo (-1 = not reached) */
    int n_launches;        /* kernels this call launched */
    int n_sweeps;          /* sweep launches that did work */
    double ms_total;       /* CUDA-event time of the call on its stream */
    double ms_sweep;       /* summed CUDA-event time of the sweep launches (RB_FLAG_TIMING) */
    double sweep_bytes;    /* algorithmic bytes read and written by those sweeps */
    int status;            /* this problem's rb_status (the batched call returns the most severe) */
} rb_result;

/* Creates a context on opt->device (NULL opt = defaults).  The context owns
 * its device workspace and, when opt->stream is NULL, a stream.
 * Errors: RB_EINVAL (bad option), RB_ECUDA. */
rb_status rb_create(const rb_options *opt, rb_ctx **out);

/* Releases the context's workspace and stream.  NULL is a no-op. */
void rb_destroy(rb_ctx *ctx);

/* Text of the last error on this context (never NULL). */
const char *rb_last_error(const rb_ctx *ctx);

/* Seeded synthetic snapshots (a stand-in for the paper's waveform model,
 * Sec. 6.1.1): for j < M, i < N, with t_i = i/N, t_c = 1.05,
 *   s_j(t_i) = (t_c - t_i)^(-1/4) exp(-i omega_j (t_c - t_i)^(5/8)),
 *   omega_j = 200 eta_j^(-3/8) m_j^(-5/8), eta_j = q_j/(1+q_j)^2,
 * each column then divided by its 2-norm.  q, m: device doubles, M entries
 * (the random draws are the caller's).  S: device complex128, ldS >= N.
 * Errors: RB_EINVAL, RB_ECUDA. */
rb_status rb_generate(rb_ctx *ctx, const double *q, const double *m, long long N, long long M,
                      void *S, long long ldS);

/* hi/lo split storage of the split-precision form: per real component
 * hi = fl32(x) and lo = fl32(x - hi), both rounded to nearest, so that
 * |x - hi - lo| <= 2^-48 |x| for x in the normal FP32 range.  S: complex128
 * (ldS >= N); hi, lo: complex64 with leading dimension ldH >= N.
 * Errors: RB_EINVAL, RB_ECUDA. */
rb_status rb_split(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS,
                   void *hi, void *lo, long long ldH);

/* RB-greedy (Alg. 3) on complex128 S in the FP64 form: FP64 bookkeeping of
 * Eq. (Residual), FP64 IMGS, FP64-accurate sweep products (see
 * rb_options.sweep).  Builds k <= kmax basis vectors; fills out->Q, pivots,
 * err_curve (k+1 entries used), C (k rows), final_err, rdiag and the host
 * scalars.  Returns RB_OK, RB_KMAX_REACHED, or an error (RB_EINVAL,
 * RB_ENOMEM, RB_ECUDA, RB_ENONFINITE, RB_EORTHO, RB_ETIMEOUT). */
rb_status rb_greedy(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS,
                    double tol, int kmax, rb_result *out);

/* rb_greedy resumed from a checkpoint: the first k0 entries of out->Q (rows),
 * out->pivots, out->C (rows, columns 0..Mc-1), out->err_curve and out->rdiag
 * hold an earlier call's results (a saved checkpoint, or the same buffers
 * after a call that stopped at kmax = k0), and the loop continues from basis
 * size k0 with the same outputs, status and stopping rule as rb_greedy.
 * Columns Mc..M-1 of S are new (the iterative enrichment of the paper's
 * software, Sec. 6.1: snapshots added after a validation pass): their first
 * k0 coefficients are computed with rb_project before the loop.  The error
 * bookkeeping of Eq. (Residual) is rebuilt from C with error-free squares and
 * a compensated sum, so a resumed run may differ from an uninterrupted one
 * in the last bits of the errors (and hence at exact pivot ties).  Requires
 * out->C; 0 <= k0 <= min(kmax, N, M); the pivots must be distinct columns of
 * S.  k0 = 0 is rb_greedy.  Returns as rb_greedy. */
rb_status rb_greedy_resume(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol, int kmax,
                           int k0, long long Mc, rb_result *out);

/* Split-precision RB-greedy on S stored as complex64 hi + lo (see rb_split;
 * column j at hi + j*ld and lo + j*ld, ld even, both 16-byte aligned; N <= 2^22).
 * Two phases.  Hi-only phase: every sweep reads hi only: c~ = q^H hi with
 * FP32 FMAs summed against a fixed power-of-two offset per lane chain
 * (rounding about 2^-42 ||hi_j|| at N = 16384), FP64 bookkeeping of the error
 * of hi_j, and the certified bounds
 * |err(hi_j) - bookkeeping| <= 2 eta ||hi_j|| sum_l |c~_lj| (eta = 2^-46 sqrt(N))
 * and |sqrt(err_j) - sqrt(err(hi_j))| <= ||lo_j||.  The columns whose upper
 * bound reaches the best lower bound are re-checked exactly (hi and lo,
 * compensated) and the exact argmax is the pivot.  The switch: once more
 * than max(M/8, 256) columns are candidates (unless opt.flags has
 * RB_FLAG_SPLIT_NO_SWITCH), or once every upper bound is below
 * opt.switch_err * max_j ||s_j||^2, the basis so far is projected onto lo on
 * the tensor cores (C becomes exact), the errors are rebuilt from C, and every
 * later sweep reads hi + lo with double-float products (the FP64 form's
 * sweep, 16 bytes per element).  The loop ends when every upper bound, or
 * the exact pivot error, is below tol (or at kmax); if that happens in the
 * hi-only phase, one projection of the basis onto lo then completes C and the
 * errors.  IMGS, norms, the bookkeeping and the re-check stay FP64(-accurate).
 * Outputs and returns as rb_greedy; the rows of C before the switch are
 * accurate to (2^-48 sqrt(N) + 2^-42) ||s_j|| beyond the FP64 form's (the
 * hi-only sweep's rounding and the FP16 pieces of the projection onto lo),
 * later rows as the FP64 form's; out->switch_iter is the basis size at the
 * switch (-1: the loop ended in the hi-only phase). */
rb_status rb_greedy_split(rb_ctx *ctx, const void *hi, const void *lo, long long N, long long M, long long ld,
                          double tol, int kmax, rb_result *out);

/* One problem of a batch: complex128 snapshots, column-major, ldS >= N (device). */
typedef struct rb_problem {
    const void *S;
    long long N, M, ldS;
} rb_problem;

/* nprob independent RB-greedy problems of uneven N and M (Alg. 3 on each), in
 * the FP64 form's arithmetic.  Every iteration runs each active problem's IMGS
 * and ONE persistent sweep launch over the columns of all active problems
 * (chunks of columns numbered across problems); each problem keeps its own
 * state and stops on its own.  The iteration is captured once as a CUDA graph
 * and replayed.  The sweep reads complex128 directly (hi/lo split in
 * registers), so the batch needs no copy of its data.  The sweep's unroll
 * depth, block width and columns per chunk are chosen by timing every variant
 * on a dry sweep of the batch (cached per batch shape in the context).
 * outs[b] as for rb_greedy.  Returns the most severe status over the
 * problems (an error if any failed, RB_KMAX_REACHED if any stopped at kmax). */
rb_status rb_greedy_batched(rb_ctx *ctx, int nprob, const rb_problem *probs, double tol, int kmax,
                            rb_result *outs);

/* Reconstruction (Alg. 4, Sec. 5.2.2): from a greedy basis Q_j and its
 * coefficients C = Q_j^H S (= R(1:j, 1:M) up to the column order), the SVD
 * C = V Sigma W^H (left factor only) and the enriched basis X_k = Q_j V(:, 1:k)
 * with k = #{i : sigma_i > tau2} (sigma_{k+1} < tau2 < sigma_k).  By Theorem
 * 5.6 / 5.8, ||S - X_i X_i^H S||_2 lies between sigma_{i+1}(S) (equal for an
 * exact-rank S) and sigma_{i+1}(C) + ||S - Q_j C||_2.
 *   Q: device complex128 N x j, column-major (ldQ >= N) -- rb_result.Q;
 *   C: device complex128 j x M, row l at C + l*ldC (ldC >= M) -- rb_result.C;
 *   X: device complex128 N x j capacity, column-major (ldX >= N); the first k
 *      columns are written;
 *   sigma: device double[j], the singular values of C in decreasing order;
 *   V: device complex128 j x j row-major (V[l*j + c] = component l of vector c),
 *      or NULL; each column's entry of largest magnitude (lowest row among
 *      equals) is made real and positive;
 *   *k_out: host.
 * The SVD is taken through the Gram matrix in two Jacobi passes (FP64;
 * singular values to about 1e-11 relative down to 1e-6 sigma_1).  j <=
 * RB_RECON_MAX_J.  Synchronises the stream.  Errors: RB_EINVAL, RB_ENOMEM,
 * RB_ECUDA. */
#define RB_RECON_MAX_J 112
rb_status rb_reconstruct(rb_ctx *ctx, const void *Q, long long N, int j, long long ldQ, const void *C, long long M,
                         long long ldC, double tau2, void *X, long long ldX, double *sigma, void *V, int *k_out);

/* What the last rb_reconstruct on ctx did (host arrays, either may be NULL):
 *   ms[7]     CUDA-event times in ms of its phases (zeros unless the context
 *             was created with RB_FLAG_TIMING): pass-1 Gram (FP32), pass-1
 *             Jacobi (FP32), Newton-Schulz steps, transform B = V1^H C,
 *             pass-2 Gram, pass-2 Jacobi (FP64) + ordering, basis X_k;
 *   counts[4] Jacobi sweeps and rotations applied in pass 1 and in pass 2.
 * Errors: RB_EINVAL (ctx NULL). */
rb_status rb_reconstruct_stats(const rb_ctx *ctx, double *ms, int *counts);

/* Empirical interpolation (EI) nodes of a basis: the greedy EIM / DEIM rule
 * that the paper's software applies after the greedy (Sec. 6.1; the algorithm
 * is the cited one, not printed in the paper).  p_1 = argmax_x |q_1(x)|; for
 * i > 1, p_i = argmax over the grid points not yet chosen of the residual of
 * q_i after interpolating it on p_1..p_{i-1} with q_1..q_{i-1} (lowest index
 * among equal maxima).  Computed as Gaussian elimination with partial
 * pivoting on the N x k basis matrix, FP64.
 *   Q: device complex128 N x k column-major (ldQ >= N) -- rb_result.Q, 1 <= k <= N;
 *   nodes: device int64[k] (grid indices p_1..p_k);
 *   V: device complex128 k x k row-major, V[m*k + l] = q_l(p_m), or NULL;
 *   B: device complex128 N x k column-major (ldB >= N), or NULL: the
 *      interpolant I[f](x) = sum_m B[x + m*ldB] f(p_m), with B V = Q;
 *   Vinv: device complex128 k x k row-major, V^{-1} (= Q^H B, valid for an
 *      orthonormal Q), or NULL -- the input of rb_validate.
 * Synchronises the stream.  Errors: RB_EINVAL, RB_ENOMEM, RB_ECUDA, RB_ESTATE
 * (a residual vanished on every free grid point: the basis is dependent). */
rb_status rb_eim(rb_ctx *ctx, const void *Q, long long N, int k, long long ldQ, long long *nodes, void *V, void *B,
                 long long ldB, void *Vinv);

/* Out-of-sample validation of a basis and its interpolant (Sec. 6.1) on Mt
 * snapshots T (device complex128, N x Mt column-major, ldT >= N):
 *   err_proj[j] = ||t_j - Q Q^H t_j||^2, formed as ||t_j||^2 - ||Q^H t_j||^2
 *                 (Eq. (Residual)) with Q^H T from rb_project;
 *   err_eim[j]  = ||t_j - I[t_j]||^2 for the EI nodes and V^{-1} of rb_eim,
 *                 formed as err_proj[j] + ||V^{-1} t_j(P) - Q^H t_j||^2 (exact
 *                 for an orthonormal Q: I reproduces span(Q) and t - Q Q^H t
 *                 is orthogonal to it), or NULL for projection errors only.
 * Outputs are device double[Mt].  k <= RB_VALIDATE_MAX_K when err_eim is
 * requested.  Synchronises the stream.  Errors: RB_EINVAL, RB_ENOMEM,
 * RB_ECUDA, RB_ETIMEOUT (tensor-core wait, from the projection). */
#define RB_VALIDATE_MAX_K 3000
rb_status rb_validate(rb_ctx *ctx, const void *Q, long long N, int k, long long ldQ, const long long *nodes,
                      const void *Vinv, const void *T, long long Mt, long long ldT, double *err_proj, double *err_eim);

/* Per-iteration trace of the last rb_greedy / rb_greedy_host / rb_greedy_resume
 * on ctx (FP64 form; host arrays of capacity cap, any may be NULL):
 *   imgs_passes[i]  IMGS passes of the i-th vector built by the call (the
 *                   paper reports fewer than three, Sec. 6.1.2);
 *   sweep_ms[i], imgs_ms[i]  CUDA-event times of that iteration's sweep and
 *                   IMGS steps (zeros unless the context has RB_FLAG_TIMING).
 * *n receives the number of iterations (entries beyond cap are not written).
 * Errors: RB_EINVAL. */
rb_status rb_trace(const rb_ctx *ctx, int *imgs_passes, double *sweep_ms, double *imgs_ms, int cap, int *n);

/* Same as rb_greedy, but S, every output array of *out, and the result are in
 * HOST memory (pinned or pageable).  Pinned S under RB_SWEEP_DF32 is read in
 * place over the host link (rb_greedy_streamed with resident = -1: no device
 * copy of S; identical results); otherwise the call copies S to the device.
 * The outputs are copied back inside the call; device workspace is owned by
 * the context. */
rb_status rb_greedy_host(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS,
                         double tol, int kmax, rb_result *out);

/* The FP64-form greedy (Alg. 3, Eq. (Residual) bookkeeping, the same
 * double-float sweep and IMGS as rb_greedy) on a snapshot matrix S that stays
 * in HOST memory: the paper's largest runs hold S of about half a terabyte
 * (Sec. 1, Sec. 6), beyond one GPU's memory.
 *   S: host complex128 N x M column-major (ldS >= N), 16-byte aligned; pinned
 *      memory is used in place, pageable memory is registered (mapped) for
 *      the duration of the call.  Device memory is rejected (RB_EINVAL).
 *   resident: columns 0..resident-1 keep a hi/lo split copy (16 ldH bytes per
 *      column, ldH = N rounded up to 64) on the device; < 0 = as many as the
 *      free device memory holds (after 4 GB of headroom).  The other columns
 *      are read from host memory in chunks of chunk_cols (0 = 1) columns.
 *   out: as for rb_greedy (DEVICE arrays).
 * A chunk is read only when its errors, as of its last read plus a bound on
 * their rounding drift, may reach the best error of the iteration; it then
 * applies every basis vector it has not seen, in order and with the
 * arithmetic of the in-core sweep.  Pivots, Q, C, err_curve, rdiag and
 * final_err equal those of rb_greedy bit for bit.  Needs RB_SWEEP_DF32.
 * Errors: as rb_greedy; RB_EINVAL for device S or chunk_cols outside
 * [0, 2^20]; RB_ECUDA when the host memory cannot be mapped. */
rb_status rb_greedy_streamed(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol,
                             int kmax, long long resident, long long chunk_cols, rb_result *out);

/* Statistics of the last rb_greedy_streamed on ctx: counts[0..3] = resident
 * columns, chunks, columns per chunk, chunk reads (each applies one or more
 * basis vectors); *host_bytes = bytes read from host memory (the first pass
 * over all of S, the IMGS pivot columns and every chunk read); *ms_init = the
 * CUDA-event time of the first pass (RB_FLAG_TIMING only, else 0).  Any
 * pointer may be NULL.  Errors: RB_EINVAL. */
rb_status rb_streamed_stats(const rb_ctx *ctx, long long *counts, double *host_bytes, double *ms_init);

/* ---------------------------------------------------------------------------
 * One rank's part of the column-sharded greedy: the paper's parallel scheme
 * (Sec. 6.1.4, Sec. 6.2).  Rank r owns columns col0 .. col0 + M - 1 of the
 * global snapshot matrix; per iteration the ranks reduce their local
 * candidates (error, global index) to the global pivot with a max-loc (ties
 * to the lowest global index), the owner sends the pivot column, and every
 * rank orthogonalises it against its own copy of the basis with the same
 * deterministic kernels, so all ranks hold bit-identical bases.  The
 * exchange and the stopping rule (max error < tol, k = kmax, k = min(N, M_total))
 * belong to the caller (paper_1805_06124_gb300/sharded.py drives them over
 * torch.distributed).  Arithmetic as rb_greedy with RB_SWEEP_DF32: the
 * ranks' local sweeps are the in-core sweep on their columns.
 * ------------------------------------------------------------------------- */
typedef struct rb_shard rb_shard;

/* S: this rank's columns (device complex128, N x M column-major, ldS >= N),
 * global indices col0 ..; out: Q (N x kmax, every rank), pivots (kmax,
 * global indices), optional C (kmax x M, this rank's columns; needed for the
 * periodic recompute, off without it) and rdiag; err_curve is the caller's.
 * The shard keeps pointers to S and *out's arrays.  Errors: RB_EINVAL,
 * RB_ENOMEM. */
rb_status rb_shard_create(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, long long col0,
                          int kmax, rb_result *out, rb_shard **sh);
void rb_shard_destroy(rb_shard *sh);
/* Norms (Alg. 3 before the loop) and the local candidate: *best_err = the
 * largest ||s_j||^2 of the rank's columns, *best_idx its global index (-1:
 * none).  Returns RB_ENONFINITE for NaN/Inf in S. */
rb_status rb_shard_init(rb_shard *sh, double *best_err, long long *best_idx);
/* The owner's side of the send: column j (global index, owned by this rank)
 * copied to dst (device, 16-byte aligned) and its stored norm ||s_j||^2 to
 * *norm2 (host; synchronises the stream), or, when norm2 is NULL, into the
 * real part of dst[N] on the device (dst then holds N + 1 complex128 entries;
 * asynchronous on the stream). */
rb_status rb_shard_column(rb_shard *sh, long long j, void *dst, double *norm2);
/* Every rank: IMGS of the received pivot column v (device, N complex128) with
 * norm2 from its owner (a negative norm2: taken from the real part of v[N]
 * on the device, v then holding N + 1 entries) against the current basis
 * (MGSCI, Sec. 6.1.2), the new
 * basis vector appended (pivots[k] = j), then the sweep of this rank's
 * columns; returns the next local candidate.  *appended = 0 when v lay in the
 * span of the basis (exact rank: the caller stops).  Errors: RB_EORTHO,
 * RB_EINVAL (kmax vectors built, bad arguments), RB_ECUDA. */
rb_status rb_shard_append(rb_shard *sh, const void *v, double norm2, long long j, double *best_err,
                          long long *best_idx, int *appended);
/* final_err (device, M doubles, optional): err_j of this rank's columns; *k:
 * vectors built. */
rb_status rb_shard_finish(rb_shard *sh, double *final_err, int *k);

/* Projection onto a basis: C[l*ldC + j] = q_l^H x_j for l < k, j < Mx
 * (Sec. 2: a column is represented by its orthogonal projection onto the
 * span of the basis).  Q: complex128 N x k (ldQ >= N); X: complex128 N x Mx
 * (ldX >= N); C: complex128 row-major k x Mx (ldC >= Mx).  FP64-accurate on
 * the BF16 tensor cores: every value is split into seven 7-bit slices under a
 * per-row power-of-two scale, the 28 leading slice products accumulate per
 * level in TMEM (exact in FP32 over 512-term chunks) and are summed in
 * double-float; error a few 2^-48 max|q_l| max|x_j| N.  Synchronises the
 * stream (RB_FLAG_PROJECT_FP64 selects a plain FP64 kernel, asynchronous).
 * Errors: RB_EINVAL, RB_ECUDA, RB_ENOMEM, RB_ETIMEOUT. */
rb_status rb_project(rb_ctx *ctx, const void *Q, long long N, int k, long long ldQ,
                     const void *X, long long Mx, long long ldX, void *C, long long ldC);

/* ---------------------------------------------------------------------------
 * Learned surrogate (no counterpart in the paper): an MLP mapping a snapshot's
 * parameters (q, m), scaled by the caller, to its n_out = 2k basis
 * coefficients (Re/Im of c = Q^H s, interleaved), widths 2-256-256-256-n_out,
 * exact-erf GELU, BF16 weights with FP32 master copies and FP32 accumulation
 * on the tensor cores, Adam (beta 0.9/0.999, eps 1e-8) with cosine
 * learning-rate decay.  Parameters are one FP32 vector: W1 (256x2), b1, W2
 * (256x256), b2, W3 (256x256), b3, W4 (n_out x 256), b4, row-major.  Work is
 * issued on the context's stream; rb_mlp_train synchronises it.
 * ------------------------------------------------------------------------- */
typedef struct rb_mlp rb_mlp;

/* Weights and biases of each layer uniform on +-1/sqrt(fan_in) from
 * splitmix64(seed); batch_cap bounds
 * the rows of one rb_mlp_grad call and the chunk of rb_mlp_infer. */
rb_status rb_mlp_create(rb_ctx *ctx, int n_out, int batch_cap, unsigned long long seed, rb_mlp **out);

/* rb_mlp_create_ex flags */
#define RB_MLP_FOURIER 1u  /* input rows are the physical (q, m); the first layer is the fixed encoding
                              h1 = (cos(omega tau_f), sin(omega tau_f)), f < 128, tau_f uniform on
                              [tau_lo, tau_hi], omega = 200 eta^(-3/8) m^(-5/8), eta = q/(1+q)^2 (the
                              snapshot family's phase rate; a coefficient c_l = q_l^H s(omega) is a sum of
                              exp(-i omega tau_i) over the samples, tau_i = (t_c - t_i)^(5/8)); W1 and b1
                              are unused and their gradient is zero */
#define RB_MLP_SPLIT 2u    /* forward GEMMs on FP32 activations and master weights, each as BF16
                              hi + lo pieces, hi*hi + hi*lo + lo*hi accumulated in FP32 (about 16-bit
                              operands instead of 8-bit); the backward pass stays single BF16 */
/* As rb_mlp_create with the flags above (tau_lo, tau_hi used with
 * RB_MLP_FOURIER: 0 <= tau_lo < tau_hi).  Errors: RB_EINVAL, RB_ENOMEM,
 * RB_ECUDA. */
rb_status rb_mlp_create_ex(rb_ctx *ctx, int n_out, int batch_cap, unsigned long long seed, unsigned flags,
                           double tau_lo, double tau_hi, rb_mlp **out);
void rb_mlp_destroy(rb_mlp *mlp);
long long rb_mlp_num_params(const rb_mlp *mlp);
/* dst / src: device FP32, rb_mlp_num_params entries.  set_params also resets
 * the Adam moments and the step counter. */
rb_status rb_mlp_get_params(rb_mlp *mlp, float *dst);
rb_status rb_mlp_set_params(rb_mlp *mlp, const float *src);
/* Y (rows x n_out, FP32) = MLP(X (rows x 2, FP32)); device pointers. */
rb_status rb_mlp_infer(rb_mlp *mlp, const float *X, long long rows, float *Y);
/* One forward + backward on rows <= batch_cap: grad (num_params) = d loss /
 * d params for loss = (1/rows) sum_r ||MLP(x_r) - t_r||^2, *loss = that loss. */
rb_status rb_mlp_grad(rb_mlp *mlp, const float *X, const float *T, long long rows, float *grad, float *loss);
/* epochs x floor(rows/batch) Adam steps over (X, T); batch b of epoch e takes
 * rows (a_e (b*batch + r) + c_e) mod rows (a seeded bijection per
 * epoch); loss_curve (optional, device, epochs entries) receives each epoch's
 * mean batch loss.  Returns RB_ETIMEOUT if a tensor-core wait ran out. */
rb_status rb_mlp_train(rb_mlp *mlp, const float *X, const float *T, long long rows, int epochs, int batch, double lr,
                       unsigned long long seed, float *loss_curve);

/* Greedy without any memory allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code whose
 * device memory is owned by a framework's pool, services that must not grow
 * their footprint after start-up, hosts where an allocation could block or
 * fail at an unpredictable moment.  It runs the rb_greedy kernels with the
 * plain-FP64 sweep (RB_SWEEP_FP64, which needs no N x M copy of S) and keeps
 * all scratch in one fixed array in device memory (about 4.7 MB, present on
 * every GPU that loads this library until the process exits), so it needs
 * no rb_ctx and allocates nothing, host or device.
 *   - Sizes must satisfy N <= RB_NOALLOC_MAX_N, M <= RB_NOALLOC_MAX_M and
 *     kmax <= RB_NOALLOC_MAX_KMAX; larger sizes return RB_EINVAL with a message.
 *   - S and *out as for rb_greedy (device pointers, caller-allocated).
 *   - opt may be NULL: current device, the legacy default stream, default
 *     IMGS options, no periodic recompute.  opt->sweep and opt->flags are
 *     ignored; the timing fields of *out are left at zero.
 *   - opt->recompute_period is honoured as in rb_greedy when out->C is given
 *     (the recompute reads the stored coefficients); without out->C the
 *     fixed array has no room for them and the recompute is off.  With the
 *     same options the results equal rb_greedy's with RB_SWEEP_FP64 bit for
 *     bit.
 *   - The calling thread's current device is the same after the call as
 *     before it, on every return path.
 *   - errbuf (may be NULL, errlen bytes) receives a message on failure.
 *   - The first call for a device looks up the array's device address with
 *     that device current (one runtime call per device and process).
 *   - Every call shares the array; calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and must be serialised by the
 *     caller.
 * Returns as rb_greedy. */
#define RB_NOALLOC_MAX_N 16384
#define RB_NOALLOC_MAX_M 262144
#define RB_NOALLOC_MAX_KMAX 1024
rb_status rb_greedy_noalloc(const void *S, long long N, long long M, long long ldS, double tol, int kmax,
                            const rb_options *opt, rb_result *out, char *errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif
#endif /* RB_GB300_H */
