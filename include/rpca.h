/*
 * rpca.h -- C-ABI of the GB300 randomized block-Lanczos PCA library.
 *
 * Computes the rank-k approximation A ~ U diag(S) V^T of Halko, Martinsson,
 * Shkolnisky and Tygert, "An algorithm for the principal component analysis
 * of large data sets" (Section 1, eq. svd_approx; Section 3, Steps 1-6):
 *
 *   Step 1  G (n x l) standard Gaussian; H^(0) = A G; H^(j) = A (A^T H^(j-1))
 *           for j = 1..i (eqs. first_prod .. last_prod), H = [H^(0) .. H^(i)]
 *   Step 2  H = Q R with Q m x (i+1)l orthonormal (eq. good_approx23)
 *   Step 3  T = A^T Q (eq. product_t3)
 *   Step 4  T = V~ Sigma~ W^T, singular values descending (eq. svd_small3)
 *   Step 5  U~ = Q W (eq. product33)
 *   Step 6  U = U~[:, :k], V = V~[:, :k], S = diag(Sigma~)[:k]
 *
 * Every streamed pass over A (Step 1's products and Step 3) reads each row
 * tile of A once: pass j forms H^(j)_b = A_b X and accumulates
 * F += A_b^T H^(j)_b in the same kernel, where X = G for j = 0 and the
 * orthonormalised F of the previous pass otherwise (the normalised iteration
 * suggested by the Remark on over/underflow at the end of Section 3; same
 * span(H) in exact arithmetic).  A row-major A is the layout of Section 4.2.
 *
 * Conventions for every function below
 *   - Matrices are row-major with an explicit leading dimension (elements).
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary host memory.  Pointers marked
 *     "host or device" are copied with cudaMemcpyDefault.
 *   - The caller owns every buffer it passes; the library owns its
 *     workspace, allocated in rpca_init and freed by rpca_destroy /
 *     rpca_finish.
 *   - No exception or longjmp crosses this boundary: every call returns an
 *     rpca_status.  After an error the context stays valid for
 *     rpca_last_error and rpca_destroy.
 *   - Without a usable CUDA device every call that would compute returns
 *     RPCA_ENODEV; there is no CPU fallback.
 *   - One context per host thread; calls on one context are not reentrant.
 */
#ifndef RPCA_H
#define RPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RPCA_OK = 0,
  RPCA_MORE = 1,          /* rpca_pass: more passes remain */
  RPCA_EINVAL = -1,       /* invalid argument (sizes, pointers, dtype) */
  RPCA_ENOMEM = -2,       /* device or pinned-host allocation failed */
  RPCA_ECUDA = -3,        /* a CUDA runtime/driver call failed */
  RPCA_ENODEV = -4,       /* no usable CUDA device */
  RPCA_EBREAKDOWN = -5,   /* QR could not orthonormalise: a block still
                             needed a shifted Cholesky in its last pass, or
                             the shifted factorisation failed (numerical
                             rank loss is otherwise handled) */
  RPCA_ETIMEOUT = -6,     /* a bounded device-side wait gave up */
  RPCA_ESTATE = -7        /* call out of order (e.g. finish before passes) */
} rpca_status;

/* Storage type of A.  Compute precision: FP64 for RPCA_F64, otherwise FP32
 * accumulation on BF16 tensor-core operands (FP32 data through exact BF16
 * hi/lo splits, FP8 bytes widened exactly to BF16 by converter warps). */
typedef enum {
  RPCA_F64 = 0,
  RPCA_F32 = 1,
  RPCA_BF16 = 2,
  RPCA_FP8E4M3 = 3        /* OCP e4m3 bytes, with per-column FP32 scales */
} rpca_dtype;

/* rpca_problem.flags */
#define RPCA_CENTER     0x1u  /* subtract column means first (Section 1) */
#define RPCA_HOST_A     0x2u  /* A lives in host memory (pinned recommended);
                                 each pass streams it to the device in tiles
                                 of tile_rows rows, double-buffered (the
                                 out-of-core form of Section 4.2) */
#define RPCA_SIMT       0x4u  /* force the CUDA-core pass kernels (testing) */
#define RPCA_TIMING     0x8u  /* record per-phase CUDA-event times */
#define RPCA_ADJOINT    0x10u /* keep what rpca_backward needs (m >= n, no
                                 centring, device A) */
#define RPCA_HOST_RESIDENT 0x20u /* with RPCA_HOST_A: the first pass of each
                                 run copies A's tiles once into a device copy
                                 the context owns (m x n, allocated at init;
                                 each tile's pass-0 kernel runs as soon as its
                                 copy lands), and the later passes read that
                                 copy.  For A in host memory that fits in
                                 device memory: one host-to-device transfer
                                 per run instead of one per pass.  Not part of
                                 the paper (no device memory there). */

#define RPCA_KEEP_T_PASS 0x40u /* always run Step 3 as its own pass over A.
                                 Without it, FP32 and FP8 problems whose
                                 Step 2 ran as one Cholesky QR of H with a
                                 well-conditioned factor (max/min diagonal of
                                 R <= 8) form T = A^T Q = [F^(0) .. F^(i)] R^-1
                                 from the blocks F^(j) = A^T H^(j) their
                                 passes accumulate (Section 3: Q = H R^-1),
                                 and read A i+1 times instead of i+2 */
#define RPCA_NO_GROUPED  0x80u /* rpca_batch_init: give this batch one
                                 context per problem even when its problems
                                 fit the grouped kernels (see rpca_batch_init) */

typedef struct {
  int64_t m, n;           /* A is m x n; 1 <= k < min(m, n) */
  int32_t k, l, i;        /* rank, block width (l >= k), power steps (i >= 0);
                             (i+1) l <= min(m, n) (Sections 2-3) */
  uint64_t seed;          /* G drawn from Philox4x32-10, key = seed, domain 0,
                             Box-Muller, row-major, when G == NULL */
  const double* G;        /* optional host FP64 test matrix, row-major:
                             n x l when n <= m, else m x l (the method
                             runs on A^T when n > m, Section 3) */
  rpca_dtype dtype;       /* storage type of A */
  uint32_t flags;         /* RPCA_* flags above */
  int64_t tile_rows;      /* RPCA_HOST_A: rows per streamed tile (0: 1 GiB) */
  void* stream;           /* cudaStream_t for all work; NULL: the default
                             (legacy) stream, ordered after the caller's
                             default-stream work */
} rpca_problem;

typedef struct {
  const void* data;       /* m x n row-major, type = problem dtype; device
                             memory, or host memory with RPCA_HOST_A */
  int64_t ld;             /* leading dimension in elements, >= n */
  const float* col_scale; /* device FP32[n]: value = stored * col_scale[j];
                             required for RPCA_FP8E4M3, optional otherwise
                             (NULL = 1) */
} rpca_matrix;

typedef struct rpca_ctx rpca_ctx;

/* Validate *p, allocate the workspace on the current device and draw G.
 * Errors: RPCA_EINVAL (bad sizes/flags), RPCA_ENODEV, RPCA_ENOMEM. */
rpca_status rpca_init(rpca_ctx** out, const rpca_problem* p);

/* One streamed pass over A (Section 4.2).  Passes 0..i are the fused
 * Step-1 passes; pass i+1 runs Step 2 (QR of H) and then Step 3 (T = A^T Q).
 * Returns RPCA_MORE while passes remain, RPCA_OK after the last.  A must be
 * the same matrix on every call.  Work is queued on the context stream. */
rpca_status rpca_pass(rpca_ctx* c, const rpca_matrix* A);

/* Steps 4-6 and copy-out.  U: m x k (ldu >= k), V: n x k (ldv >= k), element
 * type FP64 for RPCA_F64 problems and FP32 otherwise; S: k FP64 values,
 * descending.  U, S, V are host or device pointers (NULL skips that output).
 * Synchronises the stream and reports any device-side error.  Does not free
 * the context. */
rpca_status rpca_finish(rpca_ctx* c, void* U, int64_t ldu, double* S,
                        void* V, int64_t ldv);

/* Free the context and its workspace.  NULL is a no-op. */
void rpca_destroy(rpca_ctx* c);

/* init + all passes + finish + destroy in one call. */
rpca_status rpca_run(const rpca_problem* p, const rpca_matrix* A, void* U,
                     int64_t ldu, double* S, void* V, int64_t ldv);

/* Re-run all passes and Steps 2-6 on a new A of the same shape and type,
 * reusing the context's workspace and G (no allocation). */
rpca_status rpca_rerun(rpca_ctx* c, const rpca_matrix* A, void* U,
                       int64_t ldu, double* S, void* V, int64_t ldv);

const char* rpca_strerror(rpca_status s);
/* Last error message of a context (never NULL). */
const char* rpca_last_error(const rpca_ctx* c);

/* ---------------------------------------------------------------------- */
/* Single operations (used by the tests to check one pass at a time).     */
/* All pointers device memory unless noted; FP32 compute unless dtype is   */
/* RPCA_F64 (then FP64 buffers).  Work runs on `stream` (NULL = default).  */
/* ---------------------------------------------------------------------- */

/* One fused pass of Step 1 (eqs. first_prod..last_prod, Section 4.2):
 *   H[:, 0:p] = A_c X        (m x p, ldh)
 *   F         = A_c^T H      (n x p, ldf; overwritten; skipped if F NULL)
 * with A_c = A diag(col_scale) - 1 shift^T (shift NULL = 0, FP32/FP64 as
 * compute).  X: n x p, ldx.  p <= 256.  kernel: 0 auto, 1 CUDA cores,
 * 2 tensor cores (RPCA_EINVAL where unsupported).  Synchronises `stream`;
 * RPCA_ETIMEOUT if a bounded wait inside a tensor-core kernel expired. */
rpca_status rpca_op_fused_pass(rpca_dtype dtype, int64_t m, int64_t n,
                               int32_t p, const void* A, int64_t lda,
                               const float* col_scale, const void* shift,
                               const void* X, int64_t ldx, void* H,
                               int64_t ldh, void* F, int64_t ldf,
                               int32_t kernel, void* stream);

/* Step 3 (eq. product_t3): T = A_c^T Q, T n x w (ldt), Q m x w (ldq).
 * Synchronises `stream`; RPCA_ETIMEOUT as for rpca_op_fused_pass. */
rpca_status rpca_op_t_pass(rpca_dtype dtype, int64_t m, int64_t n, int32_t w,
                           const void* A, int64_t lda, const float* col_scale,
                           const void* shift, const void* Q, int64_t ldq,
                           void* T, int64_t ldt, int32_t kernel, void* stream);

/* Step 2 on a block-structured H (m x (nblk*l), ld): replaces H by Q with
 * orthonormal columns spanning the same space (block Gram-Schmidt twice +
 * Cholesky QR twice, Gram matrices and Cholesky in FP64). */
rpca_status rpca_op_qr(int32_t f64, int64_t m, int32_t nblk, int32_t l,
                       void* H, int64_t ld, void* stream);

/* C (p x q, FP64, ldc) = X^T Y over m rows; X (m x p, ldx) and Y (m x q,
 * ldy) FP32 device matrices.  kernel: 0 auto, 1 CUDA cores, 2 tensor cores
 * (FP32-accurate TF32 x3).  p, q <= 256.  Synchronises `stream`. */
rpca_status rpca_op_gram(int64_t m, int32_t p, int32_t q, const float* X,
                         int64_t ldx, const float* Y, int64_t ldy, double* C,
                         int64_t ldc, int32_t kernel, void* stream);

/* Y (m x q, ldy) = beta Y + alpha X M; X (m x p, ldx) FP32, M (p x q, ldm)
 * FP64, all device memory.  kernel as for rpca_op_gram.  p, q <= 256.
 * Synchronises `stream`. */
rpca_status rpca_op_apply(int64_t m, int32_t p, int32_t q, const float* X,
                          int64_t ldx, const double* M, int64_t ldm,
                          double alpha, double beta, float* Y, int64_t ldy,
                          int32_t kernel, void* stream);

/* Step 4 on T (n x w, ldt, FP32 or FP64 per f64): S[w] (FP64, device),
 * Vt (n x w, ldv, same type as T) and W (w x w FP64 row-major, device). */
rpca_status rpca_op_small_svd(int32_t f64, int64_t n, int32_t w,
                              const void* T, int64_t ldt, double* S, void* Vt,
                              int64_t ldv, double* W, void* stream);

/* Library-side test-matrix stream: `count` standard normals (FP64, host)
 * from Philox4x32-10 (key = seed, counter = (p, 0, domain, 0)) and
 * Box-Muller, element 2p and 2p+1 from counter p. */
rpca_status rpca_gaussian(uint64_t seed, uint32_t domain, int64_t count,
                          double* out);

/* Number of the library's own kernels launched since load (all devices).
 * A replay of a batch's captured CUDA graph adds the number of kernels the
 * graph holds. */
uint64_t rpca_kernel_launches(void);

/* Passes over A of the last completed run of c: i+2 (Step 1's i+1 and
 * Step 3's), or i+1 when T was formed from the F blocks (RPCA_KEEP_T_PASS
 * above); 0 before a run completed. */
int32_t rpca_last_run_passes(const rpca_ctx* c);

/* Per-phase device times of a context created with RPCA_TIMING, summed
 * over the runs finished since the previous call (then reset).  Phases:
 * 0..i the streaming kernels of the Step-1 passes, i+1 the QR of H (Step 2),
 * i+2 the T pass (Step 3), i+3 Step 4 (QR of T and the small SVD), i+4 the
 * products forming U and V (Steps 5-6).  Writes min(cap, i+5) values (ms)
 * to ms (host), the run count to *runs (may be NULL); returns i+5, or 0
 * without RPCA_TIMING. */
int32_t rpca_phase_times(rpca_ctx* c, double* ms, int32_t cap, int32_t* runs);

/* ---------------------------------------------------------------------- */
/* Adjoint.  The paper has no gradient; this differentiates the computed    */
/* singular values with respect to A (G fixed).                             */
/* ---------------------------------------------------------------------- */

/* dA (m x n, ldda, device, FP64 for RPCA_F64 else FP32) = sum_j dS[j]
 * d sigma_j / dA for the k singular values of the last completed run of a
 * context created with RPCA_ADJOINT (A the same matrix, device memory).
 * dS: k FP64 values in device memory.  Re-streams A 2 + 2i times (the
 * blocks H^(j) are recomputed from the saved n x l blocks X^(j), not
 * stored) and writes dA once as the product of two thin factors.  The
 * losses sum_j sigma_j and ||A - U S V^T||_F^2 = ||A||_F^2 - sum_j sigma_j^2
 * take dS = 1 and dS = -2 sigma (plus 2A).  RPCA_EBREAKDOWN if a small
 * factor is singular. */
rpca_status rpca_backward(rpca_ctx* c, const rpca_matrix* A, const double* dS,
                          void* dA, int64_t ldda);

/* ---------------------------------------------------------------------- */
/* Error estimate (Appendix) and adaptive rank (Remark after Section 3).    */
/* ---------------------------------------------------------------------- */

/* p_{j,q}(D), the Appendix's power-method estimate of ||D||_2 for
 * D = A - U diag(S) V^T:
 *   p = max_c sqrt(||(D^T D)^j w_c|| / ||(D^T D)^(j-1) w_c||),
 * j steps from q start vectors w_c (n x q, row-major FP64, host: `omega`;
 * NULL: the Philox4x32-10 Gaussian stream of p->seed, domain 1).  D is
 * applied only through products with A and A^T, D then D^T in turn: each
 * step is an H pass and a T pass over A plus the rank-kd corrections, with
 * the columns renormalised between steps.  p (problem) gives m, n, dtype and stream of A
 * (device, no RPCA_CENTER / RPCA_HOST_A); U (m x kd, ldu), V (n x kd, ldv):
 * device, compute type (FP64 for RPCA_F64, else FP32); S: kd FP64 values
 * (host or device).  *est (host) receives p; col_est (host, q values, may be
 * NULL) each column's estimate.  p <= ||D||_2 always; p >= ||D||_2 / 2 with
 * probability at least 1 - (2n / ((2j - 1) 16^j))^(q/2) (eq. high_prob).
 * The paper uses j = 6 and q = the rank.  Synchronises the stream. */
rpca_status rpca_estimate_error(const rpca_problem* p, const rpca_matrix* A,
                                const void* U, int64_t ldu, const double* S,
                                const void* V, int64_t ldv, int32_t kd,
                                int32_t j, int32_t q, const double* omega,
                                double* est, double* col_est);

/* Adaptive rank: runs the method (rpca_run) at k = p->k, then 2k, 4k, ...
 * (at most kmax; oversampling l - k and power steps i kept from p) until
 * the estimate of ||A - U S V^T||_2 (rpca_estimate_error, j steps, q = k
 * start vectors) is at most tol.  U (m x kmax capacity, ldu >= kmax), S
 * (kmax), V (n x kmax, ldv >= kmax) hold the last run's rank-k result;
 * *k_out its rank and *eps_out its estimate (> tol only when kmax or the
 * limits of the method stopped the doubling).  The Remark after Section 3
 * refers the choice of k to the literature; this is the doubling rule with
 * the paper's own estimator.  A is a device matrix: RPCA_CENTER and
 * RPCA_HOST_A give RPCA_EINVAL before anything runs.  Synchronises
 * p->stream. */
rpca_status rpca_run_adaptive(const rpca_problem* p, const rpca_matrix* A,
                              double tol, int32_t kmax, int32_t j, void* U,
                              int64_t ldu, double* S, void* V, int64_t ldv,
                              int32_t* k_out, double* eps_out);

/* ---------------------------------------------------------------------- */
/* Batches of independent problems (uneven shapes).                        */
/* ---------------------------------------------------------------------- */
typedef struct rpca_batch rpca_batch;

/* A batch of independent problems (problems[p] as for rpca_init; device
 * matrices only, no RPCA_TIMING).  Two forms:
 *   grouped   when every problem is BF16 with no flags (RPCA_KEEP_T_PASS
 *             aside), m >= n, n <= 1024, l <= 32, (i+1) l <= 64,
 *             n (i+1) l <= 45056, and all share k, l and i: each step of
 *             Section 3 runs as one launch over all problems (about
 *             3 i + 8 kernels per run; rpca_batch_grouped says so).  Step 1
 *             is the block Lanczos form, Step 2 a twice-repeated Cholesky
 *             QR, Step 4 a Householder QR plus one-sided Jacobi in FP32 on
 *             the n side.  A numerically rank-deficient H is reported as
 *             RPCA_EBREAKDOWN for its problem (the per-problem form handles
 *             it).  X^(0) = orth(G) is formed here.
 *   per-problem otherwise (or with RPCA_NO_GROUPED on any problem): one
 *             context per problem, spread over nstreams streams of the
 *             library that fork from and join to problems[0].stream.
 * All workspace of the chosen form is allocated here. */
rpca_status rpca_batch_init(rpca_batch** out, int32_t count,
                            const rpca_problem* problems, int32_t nstreams);

/* 1 if the batch's last run (before any run: the batch as created) used
 * the grouped kernels, 0 otherwise or for NULL. */
int32_t rpca_batch_grouped(const rpca_batch* b);

/* Launch parameters of the grouped kernels: tuning[0] H-pass TMA stages
 * (2..4), [1] T-pass stages (2..5), [2] rows per T-pass work item,
 * [3] rows per row-kernel item (multiples of 64), [4] distance in ring
 * stages of the H and T passes' L2 prefetches (0..64, 0: none).  Get and
 * set copy 5 int32 values (host); set clamps them to their ranges.
 * RPCA_EINVAL for a per-problem batch or NULL arguments. */
rpca_status rpca_batch_get_tuning(const rpca_batch* b, int32_t* tuning);
rpca_status rpca_batch_set_tuning(rpca_batch* b, const int32_t* tuning);

/* Autotuner of the grouped kernels: times rpca_batch_run on these
 * arguments for a set of launch parameters (coordinate search over the
 * five values above, each candidate run twice and timed once with CUDA
 * events), keeps the fastest, and records it in the JSON file cache_path
 * (host path; NULL: no cache) under a key made of the storage type, the
 * power-of-two buckets of the largest n and of the mean m, k, l and i.  A
 * key already in the file is applied without timing.  The outputs are
 * written as by rpca_batch_run.  *chosen (5 values, may be NULL) receives
 * the parameters in use.  RPCA_EINVAL for a per-problem batch. */
rpca_status rpca_batch_tune(rpca_batch* b, const rpca_matrix* A, void* const* U,
                            const int64_t* ldu, double* const* S, void* const* V,
                            const int64_t* ldv, const char* cache_path,
                            int32_t* chosen);

/* All problems: A[p] as for rpca_pass, outputs as for rpca_finish (arrays
 * of count pointers / leading dimensions; U, S, V or their entries may be
 * NULL).  The first run, and the first run after any pointer in the
 * arguments changed, executes directly and then records the whole batch as
 * one CUDA graph; later runs with the same pointers replay that graph (one
 * launch).  Synchronises problems[0].stream and reports the first problem
 * whose device-side checks failed (rpca_batch_last_error names it).  The
 * batch runs on streams of its own, ordered after the work queued on
 * problems[0].stream, which in turn waits for the batch. */
rpca_status rpca_batch_run(rpca_batch* b, const rpca_matrix* A, void* const* U,
                           const int64_t* ldu, double* const* S, void* const* V,
                           const int64_t* ldv);

/* The adjoint of rpca_backward for every problem of a batch whose problems
 * were all created with RPCA_ADJOINT, after a completed rpca_batch_run:
 * dA[p] (m_p x n_p, ldda[p], device) = sum_j dS[p][j] d sigma_j / dA for
 * problem p, dS[p] its k FP64 values in device memory, A[p] the same
 * matrices as in the run.  The problems' backward passes run concurrently
 * on the batch's streams, ordered after the work queued on
 * problems[0].stream; synchronises and reports the first failing problem
 * (rpca_batch_last_error).  RPCA_EINVAL if a problem lacks RPCA_ADJOINT.
 * (The paper has no gradient; see rpca_backward.) */
rpca_status rpca_batch_backward(rpca_batch* b, const rpca_matrix* A, const double* const* dS, void* const* dA,
                                const int64_t* ldda);

/* Frees the batch (NULL is a no-op). */
void rpca_batch_destroy(rpca_batch* b);

/* Last error message of a batch, or of the last failed rpca_batch_init when
 * b is NULL (never NULL). */
const char* rpca_batch_last_error(const rpca_batch* b);

/* ---------------------------------------------------------------------- */
/* Allocation-free fused pass.  The paper has no counterpart to this call: */
/* it exists for callers that must not allocate device memory per call.   */
/* ---------------------------------------------------------------------- */

/* Limits of the fixed scratch: X^T in BF16 for up to RPCA_NOALLOC_MAX_P
 * columns and RPCA_NOALLOC_MAX_N rows, then 64 error words (512 KiB + 256 B
 * per device in total).  (The allocating entry's tensor-core pass takes n
 * up to 8192.) */
#define RPCA_NOALLOC_MAX_N 4096
#define RPCA_NOALLOC_MAX_P 64
#define RPCA_NOALLOC_SCRATCH_BYTES (64 * 4096 * 2 + 256)

/* The tensor-core fused pass of rpca_op_fused_pass (dtype RPCA_BF16,
 * kernel 2, no shift or column scale) with its scratch in a fixed device
 * array of RPCA_NOALLOC_SCRATCH_BYTES instead of a per-call allocation;
 * the call allocates no device memory.
 *   H[:, 0:p] = A X  (m x p FP32, ldh),  F = A^T bf16(H)  (n x p FP32, ldf;
 *   overwritten; skipped if F is NULL)
 * A: m x n BF16 row-major (lda elements; base 16-byte aligned, lda*2 a
 * multiple of 16).  X: n x p FP32 (ldx).  All device memory, owned by the
 * caller.  Returns RPCA_EINVAL for n > RPCA_NOALLOC_MAX_N,
 * p > RPCA_NOALLOC_MAX_P, bad sizes, NULL A/X/H or a layout the tensor-core
 * pass does not take; RPCA_ENODEV without a GPU; RPCA_ETIMEOUT if a bounded
 * wait inside the kernel expired.  Synchronises `stream`.
 * The scratch address is looked up (cudaGetSymbolAddress) on the first
 * call on each device, with that device current: make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset on a device this entry must not be called
 * on it again.  The error words are cleared on `stream` at the start of
 * every call.  Calls that overlap in time on one device (other streams or
 * host threads) share the scratch and race: serialise them. */
rpca_status rpca_op_fused_pass_noalloc(int64_t m, int64_t n, int32_t p,
                                       const void* A, int64_t lda,
                                       const float* X, int64_t ldx, float* H,
                                       int64_t ldh, float* F, int64_t ldf,
                                       void* stream);

/* ---------------------------------------------------------------------- */
/* Test hook of the bounded device-side waits.  The paper has no           */
/* counterpart: it exists so that a test can make a wait expire and check  */
/* that the call reports RPCA_ETIMEOUT and the device stays usable.        */
/* ---------------------------------------------------------------------- */

/* Arms the next tensor-core launch of one kernel (0: the fused pass of
 * Step 1, 1: the T pass of Step 3), whichever call makes it: that launch's
 * first CTA leaves its TMA stage `withhold_stage` unissued (nothing is in
 * flight for it, so the wait on it can only expire) and every mbarrier wait
 * of the launch gives up after limit_ns (100 us .. 2 s; the default is 2 s).
 * The launch then returns early and the call that made it reports
 * RPCA_ETIMEOUT.  withhold_stage = -1 only shortens the limit.  The arming
 * is consumed by that one launch.  RPCA_EINVAL for an unknown kernel or a
 * limit out of range. */
rpca_status rpca_test_arm_wait_expiry(int32_t kernel, uint64_t limit_ns, int64_t withhold_stage);

#ifdef __cplusplus
}
#endif
#endif /* RPCA_H */
