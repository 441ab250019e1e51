// Internal launcher interface between the host orchestration and kernels.
#pragma once
#include "common.cuh"

namespace rpca {

enum PassMode { MODE_FUSED = 0, MODE_H = 1, MODE_T = 2 };

// One streamed pass over A (see k_stream_simt.cu / k_stream_tc.cu).
struct PassArgs {
  rpca_dtype dtype = RPCA_F32;
  int mode = MODE_FUSED;
  const void* A = nullptr;
  int64_t lda = 0, m = 0, n = 0;
  const float* scale = nullptr;  // per-column scale (FP8), may be null
  const void* shift = nullptr;   // per-column shift (compute type), may be null
  const void* X = nullptr;       // n x p right factor (compute type)
  int64_t ldx = 0;
  int p = 0;                     // columns of X / H / F
  void* H = nullptr;             // m x p output (MODE_FUSED/H) or input Q (MODE_T)
  int64_t ldh = 0;
  const void* corr = nullptr;    // p-vector subtracted from each H row, may be null
  int ones_col = -1;             // >= 0: F column `ones_col` accumulates A~^T 1
  void* F = nullptr;             // n x (p [+1]) accumulator (zeroed by the launcher)
  int64_t ldf = 0;
  bool accumulate_f = false;     // true: add into F (caller zeroed it)
  bool f_f64 = false;            // MODE_T: F is an FP64 accumulator
  void* work = nullptr;          // device scratch for the tensor-core path
  size_t work_bytes = 0;
  // MODE_T on tensor cores: Q already in BF16 (q16, ld q16_ld), block-padded
  // (block b of q_blk columns at columns [64b, 64b + q_blk)); T columns are
  // written in compact numbering.
  const void* q16 = nullptr;
  int64_t q16_ld = 0;
  int q_blk = 0;
  int64_t q16_plane = 0;         // elements between BF16 slice planes of Q (0: one slice)
};

// Test hook of the bounded-wait path (rpca_test_arm_wait_expiry): the next
// tensor-core launch of kernel `kind` (0: fused pass, 1: T pass) leaves
// TMA stage `withhold` of its first CTA unissued and bounds every wait by
// limit_ns.  Returns {2 s, -1} when nothing is armed; disarms what it returns.
struct WaitTest {
  uint64_t limit_ns;
  int64_t withhold;
};
WaitTest take_wait_test(int kind);

void launch_pass_simt(const PassArgs& a, cudaStream_t st);
// Tensor-core pass; returns false when the shape/dtype is not supported.
bool launch_pass_tc(const PassArgs& a, cudaStream_t st, uint32_t* dev_err);
// Fused Step-1 pass on tensor cores (k_fused_rr.cu); false if unsupported.
bool fused_pass_tc(const PassArgs& a, cudaStream_t st, uint32_t* dev_err);
// Passes over FP32 A on tensor cores through converter warps (BF16 hi/lo
// slices of A and of the small operand; k_stream_cvt.cu); false if unsupported.
bool pass_cvt(const PassArgs& a, cudaStream_t st, uint32_t* dev_err);

// ---------------------------------------------------------------- linalg
// C (p x q, FP64, ldc) (+)= X^T Y over rows [0, m); X m x p (ldx), Y m x q.
// Compute type TC: FP32 sums over short row chunks, FP64 accumulation.
void gram(bool f64, int64_t m, int p, int q, const void* X, int64_t ldx, const void* Y,
          int64_t ldy, double* C, int64_t ldc, bool accumulate, cudaStream_t st,
          const uint32_t* active = nullptr);
// C (p x p, FP64, both triangles) = X^T X for X m x p FP64, FP64-class, in
// FP32 arithmetic (hi/lo split, exact products, compensated sums).
void gram_sym_comp(int64_t m, int p, const double* X, int64_t ldx, double* C, int64_t ldc, cudaStream_t st);
// Y[:, 0:q] = beta * Y + alpha * X M, X m x p, M p x q FP64 (ldm).  In-place
// safe when Y aliases X (rows are staged before they are overwritten).
// `active` (device word, may be null): the kernel does nothing when it is 0.
void gemm_xm(bool f64, int64_t m, int p, int q, const void* X, int64_t ldx, const double* M,
             int64_t ldm, double alpha, double beta, void* Y, int64_t ldy, cudaStream_t st,
             const uint32_t* active = nullptr);
// Pass `pass` (0..3) of a Cholesky-QR sequence on one block: factor the
// FP64 Gram G = R^T R (R upper), write R and Rinv (p x p, ld p).  A pivot
// below piv_rel * max diag retries with a diagonal shift shift_rel * max
// diag.  Passes 2 and 3 run only after a shifted pass (else identities).
// A pass >= 1 whose G is within 2e-3 of I (p <= 64) writes instead the
// symmetric M = I - E/2 + 3/8 E^2 (E = G - I) as Rinv and its inverse as R:
// the same span, orthonormal to O(E^3).
// qf: 4 device words private to the block; the word qf + pass gates the
// Gram/gemm of passes 2-3 (qf[2], qf[3]).
// Cholesky-QR passes per block (passes >= 2 run only after a shifted pass)
// and device words of flags per block (qf).
constexpr int kCholPasses = 6;
constexpr int kQfWords = 8;
// inv_f32: Rinv may be formed in FP32 (it then only feeds FP32 products).
// gate (device word, may be null): the kernel does nothing when it is 0.
void chol_small(int p, const double* G, int64_t ldg, double* R, double* Rinv, int pass,
                double piv_rel, double shift_rel, uint32_t* qf, uint32_t* dev_err, cudaStream_t st,
                bool inv_f32 = false, const uint32_t* gate = nullptr);

// Racc = Rk * Racc (p x p FP64)
void left_mul(int p, const double* Rk, double* Racc, cudaStream_t st);
// M -= I (p x p FP64, ld p)
void sub_identity(int p, double* M, cudaStream_t st);
// M = I (p x p FP64)
void set_identity(int p, double* M, cudaStream_t st);
// dst += src (rows x cols FP64)
void mat_add(int rows, int cols, const double* src, int64_t lds, double* dst, int64_t ldd,
             cudaStream_t st);
// One-sided Jacobi SVD of a w x w FP64 matrix B (row-major): B = Ub S W^T,
// S descending.  FP32 sweeps with an FP64 finish (f64 = false) or FP64.
// Singular triplets of B (w x w FP64 row-major): S descending, Ub, W
// (row-major w x w, ld w); callers use the leading kk.  work: 4 w^2 doubles.
// Step 4's one-sided Jacobi (FP32) on a thread-block cluster: J (w x w,
// column-major FP32) with B J having orthogonal columns.  False when the
// shape or the device does not admit the cluster.
bool jacobi_cluster_f32(int w, const double* B, float* Jc, double tol, int max_sweeps, uint32_t* dev_err,
                        cudaStream_t st);
// ---------------------------------------------- H in three BF16 slices
// (k_qr_slices.cu): planes of plane_rows x (nblk*64) BF16, block-padded.
void slice_blocks(int64_t m, int64_t plane_rows, int nblk, int l, const float* H, int64_t ld, void* S,
                  cudaStream_t st);
void unslice_blocks(int64_t m, int64_t plane_rows, int nblk, int l, const void* S, float* H, int64_t ld,
                    cudaStream_t st);
void col_sums_slices(int64_t m, int64_t plane_rows, int nblk, int l, const void* S, double* out, cudaStream_t st);
// E (w x w, compact) from the symmetric C with block-padded indices (ld
// ldc), read from C's upper block triangle (block row <= block column)
void compact_sq(int nblk, int l, const double* C, int64_t ldc, double* E, cudaStream_t st);
// C (p x q FP64, ldc) = X^T Y, X = columns [x0, x0+p), Y = [y0, y0+q) of the
// slices (x0, y0 multiples of 64).  upper (X = Y only): only the 64-wide
// block rows at or above each block column are formed (and read: column
// group g reads the first g + 1 boxes), the rest of C stays zero.
bool gram_slices(int64_t m, int64_t plane_rows, const void* S, int lds, int x0, int p, int y0, int q, double* C,
                 int64_t ldc, cudaStream_t st, uint32_t* dev_err, const uint32_t* active, bool upper = false);
// Y = beta Y + X (alpha M): X = nkb 64-column boxes at x0, Y = the 64 columns
// at y0 (slices, rewritten when write_slices), M krows x q FP64 (ldm) with
// row remap rl (block-padded K when rl > 0); optional FP32 copy Yf
// (columns < qf, ldf).  mt: scratch of 3 * 64 * 192 BF16.
bool apply_slices(int64_t m, int64_t plane_rows, void* S, int lds, int x0, int nkb, int y0, const double* M,
                  int krows, int q, int64_t ldm, double alpha, int rl, bool beta, bool write_slices, float* Yf,
                  int64_t ldf, int qf, void* mt, cudaStream_t st, uint32_t* dev_err, const uint32_t* active);

// ---------------------------------------------------------- adjoint
// (k_adjoint.cu)  out = (M^-1)^T (p x p FP64, ld p), aug: p x 2p scratch.
void small_inv_t(int p, const double* M, int64_t ldm, double* aug, double* out, uint32_t* dev_err, cudaStream_t st);
// Mk (k x w) = diag(c) W[:, :k]^T, W w x w row-major FP64
void make_mk(int k, int w, const double* c, const double* W, double* Mk, cudaStream_t st);
// out = V diag(c) (rows x k, compute type)
void scale_cols(bool f64, int64_t rows, int k, const void* V, int64_t ldv, const double* c, void* out, int64_t ldo,
                cudaStream_t st);
// dst += src (compute type)
void add_matrix(bool f64, int64_t rows, int cols, const void* src, int64_t lds, void* dst, int64_t ldd,
                cudaStream_t st);
// G (m x n) = P Z^T, P m x r, Z n x r (compute type)
void lowrank_out(bool f64, int64_t m, int64_t n, int r, const void* P, int64_t ldp, const void* Z, int64_t ldz,
                 void* G, int64_t ldg, cudaStream_t st);

// work: 5 w^2 doubles.  FP32 paths: FP32 Jacobi sweeps, then FP64
// refinement of the right singular vectors (k_small64.cu); FP64: FP64 Jacobi.
void jacobi_svd(bool f64, int w, int kk, const double* B, double* S, double* Ub, double* W,
                double* work, uint32_t* dev_err, cudaStream_t st);
// C = alpha op(A) op(B) + beta D for small FP64 row-major matrices (D may
// alias C).
void gemm64_small(int M, int N, int K, double alpha, const double* A, int64_t lda, bool ta, const double* B,
                  int64_t ldb, bool tb, double beta, const double* D, int64_t ldd, double* C, int64_t ldc,
                  cudaStream_t st);
// `steps` FP64 refinement steps of the eigenvectors X (w x w) of B^T B, or
// of B itself when gram_given (B = a symmetric Gram G) (k_small64.cu); Xn,
// P, S, E: w x w scratch.  On return S holds X^T M X of the last step's
// input only when steps > 0.
void refine_eigvecs64(int w, const double* B, double* X, double* Xn, double* P, double* S, double* E, int steps,
                      cudaStream_t st, bool gram_given = false);
// B (upper triangular FP64 container) with B^T B = G + 1e-6 max diag(G) I,
// FP32 Cholesky (a preconditioner only; w <= 224).
void chol32_shift(int w, const double* G, double* B, cudaStream_t st);

// sigma_j = sqrt(S_jj) sorted descending, W = X reordered, Vs = W Sigma^-1.
void eig_finish(int w, const double* Sm, const double* X, double* S, double* Vs, double* W, cudaStream_t st);
// Step 4 from the Gram of T (FP32-class paths): S, W (right singular
// vectors of T) and Vs = W Sigma^-1 with V = T Vs; work: 6 w^2 doubles.
void svd_from_gram(int w, const double* G, double* S, double* Vs, double* W, double* work, uint32_t* dev_err,
                   cudaStream_t st);

// ------------------------------------------- tensor-core tall products
// FP32-accurate (TF32 x3) products on FP32 data carried with a remainder
// array (x_lo = x - trunc_tf32(x), same layout and ld).  Return false when
// the shape or alignment does not suit the tensor-core kernels.
void split_lo(int64_t rows, int cols, const float* X, int64_t ldx, float* Xlo, int64_t ldl, cudaStream_t st);
// C = X^T Y (FP64, overwritten); slices: device scratch of at least
// 6 m (round_up(p,64) + round_up(q,64)) bytes.
// reslice_x = false reuses the X slices of the previous call (same X).
bool gram_tc(int64_t m, int p, int q, const float* X, int64_t ldx, const float* Y, int64_t ldy, double* C,
             int64_t ldc, void* slices, size_t slice_bytes, cudaStream_t st, uint32_t* dev_err,
             const uint32_t* active = nullptr, bool reslice_x = true);
// Y = beta Y + alpha X M (and Ylo); scratch: 2 p q floats of device memory.
bool apply_tc(int64_t m, int p, int q, const float* X, const float* Xlo, int64_t ldx, const double* M,
              int64_t ldm, double alpha, double beta, float* Y, float* Ylo, int64_t ldy, float* scratch,
              cudaStream_t st, uint32_t* dev_err, const uint32_t* active = nullptr);

// Y (m x q) = beta Y + alpha X M for small FP64 matrices, FP32 arithmetic
// (for corrections whose own relative accuracy needs only FP32).
void small_gemm_f32(int m, int p, int q, const double* X, int64_t ldx, const double* M, int64_t ldm,
                    double alpha, double beta, double* Y, int64_t ldy, cudaStream_t st);

// ----------------------------------------------------------------- small ops
// s[j] = mean of (scaled) A[0:rows, j] in the compute type.
void panel_mean(rpca_dtype dt, const void* A, int64_t lda, int64_t rows, int64_t n,
                const float* scale, void* s, cudaStream_t st);
// out[c] = sum_j x[j] * M[j, c] (x length n FP64, M n x p compute type).
void vec_mat(bool f64, int64_t n, int p, const double* x, const void* M, int64_t ldm,
             double* out, cudaStream_t st);
// v (compute type, p) = out (FP64) cast.
void cast_f64_to(bool f64, int64_t count, const double* src, void* dst, cudaStream_t st);
void cast_to_f64(bool f64, int64_t count, const void* src, double* dst, cudaStream_t st);
// M[j, c] -= alpha * x[j] * y[c] for j < n, c < p (M compute type).
void rank1_sub(bool f64, int64_t n, int p, double alpha, const double* x, const double* y,
               void* M, int64_t ldm, cudaStream_t st);
// d[j] = F[j, col] / m  (F compute type, d FP64)
void column_to_vec(bool f64, int64_t n, const void* F, int64_t ldf, int col, double scale,
                   double* d, cudaStream_t st);
// colsum[c] = sum_r Q[r, c]  (FP64 out)
void col_sums(bool f64, int64_t m, int p, const void* Q, int64_t ldq, double* out,
              cudaStream_t st);
// H[r, c] -= v[c]
void sub_rowvec(bool f64, int64_t m, int p, const double* v, void* H, int64_t ldh,
                cudaStream_t st);
// out (rows x cols, ld_out) = in^T (cols x rows, ld_in), storage type dt
void transpose(rpca_dtype dt, int64_t rows, int64_t cols, const void* in, int64_t ld_in,
               void* out, int64_t ld_out, cudaStream_t st);
// 2-D strided copy of compute-type matrix with optional type change to out_f64
void copy_matrix(bool in_f64, bool out_f64, int64_t rows, int64_t cols, const void* in,
                 int64_t ld_in, void* out, int64_t ld_out, cudaStream_t st);

}  // namespace rpca
