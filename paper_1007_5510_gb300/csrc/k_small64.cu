// FP64 small dense kernels for Step 4 (Section 3, eq. svd_small3): the SVD
// of the (i+1)l x (i+1)l factor B = R_T of T is finished in FP64.
//
// The one-sided Jacobi sweeps run in FP32 (k_jacobi_cl.cu), which gives
// right singular vectors W0 of B to FP32 accuracy.  They are then refined in
// FP64 by the iterative refinement of Ogita and Aishima ("Iterative
// refinement for symmetric eigenvalue decomposition", Japan J. Indust. Appl.
// Math. 35 (2018)) applied to M = B^T B through products with B only.
// Derivation, for a current X (approximately orthonormal eigenvectors of M):
// seek X' = X (I + E) with X'^T X' = I and X'^T M X' diagonal.  With
// R = I - X^T X and S = X^T M X = (B X)^T (B X), first order gives
//   E + E^T = R,   S_ij + lambda_j E_ji + lambda_i E_ij = 0  (i != j),
// so E_ii = R_ii / 2 and, eliminating E_ji = R_ij - E_ij,
//   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i),
// lambda_i = S_ii / (1 - R_ii).  Pairs whose lambdas are closer than the
// size of the first-order terms are only orthonormalised (E_ij = R_ij / 2):
// inside a cluster of nearly equal singular values the basis of the cluster
// is kept, not its individual vectors.  Each step squares the error of X
// (relative to the gaps), so two steps take the FP32 start to FP64
// rounding.  S_ij is a dot product of two columns of B X, so its error is
// relative to those columns' norms: the refinement keeps the relative
// accuracy of one-sided Jacobi and never forms B^T B on its own.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rpca {
namespace {

constexpr int T64 = 16;

// C = alpha op(A) op(B) + beta D (FP64, row-major; op = transpose when the
// flag is set).  16 x 16 output tile per CTA, K staged through shared
// memory in steps of 16, two independent accumulators per thread.
__global__ void __launch_bounds__(256)
k_gemm64_small(int M, int N, int K, double alpha, const double* __restrict__ A, int64_t lda, int ta,
               const double* __restrict__ B, int64_t ldb, int tb, double beta, const double* D, int64_t ldd,
               double* C, int64_t ldc) {
  __shared__ double As[T64][T64 + 1];
  __shared__ double Bs[T64][T64 + 1];
  const int tx = threadIdx.x & (T64 - 1), ty = threadIdx.x / T64;
  const int i0 = blockIdx.y * T64, j0 = blockIdx.x * T64;
  double acc0 = 0.0, acc1 = 0.0;
  for (int k0 = 0; k0 < K; k0 += T64) {
    {
      const int ai = i0 + ty, ak = k0 + tx;
      As[ty][tx] = (ai < M && ak < K) ? (ta ? A[(int64_t)ak * lda + ai] : A[(int64_t)ai * lda + ak]) : 0.0;
      const int bk = k0 + ty, bj = j0 + tx;
      Bs[ty][tx] = (bk < K && bj < N) ? (tb ? B[(int64_t)bj * ldb + bk] : B[(int64_t)bk * ldb + bj]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < T64; kk += 2) {
      acc0 = fma(As[ty][kk], Bs[kk][tx], acc0);
      acc1 = fma(As[ty][kk + 1], Bs[kk + 1][tx], acc1);
    }
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  if (i < M && j < N) {
    double v = alpha * (acc0 + acc1);
    if (beta != 0.0) v += beta * D[(int64_t)i * ldd + j];
    C[(int64_t)i * ldc + j] = v;
  }
}

// One refinement step's correction E (w x w) from S = X^T M X and
// Gx = X^T X (R = I - Gx), as derived at the top of this file.  First the
// eigenvalue estimates lambda_i and the threshold delta (one CTA), then E
// elementwise (many CTAs; E may alias Gx: each element is read, then
// written, by the same thread).
__global__ void __launch_bounds__(1024)
k_refine_stats(int w, const double* __restrict__ S, const double* __restrict__ Gx, double* __restrict__ lam_out) {
  __shared__ double red_s[32], red_r[32], lmax_s[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double off_s = 0.0, off_r = 0.0, lmax = 0.0;
  for (int i = tid; i < w; i += blockDim.x) {
    const double g = Gx[(int64_t)i * w + i];
    const double lam = g > 0.0 ? S[(int64_t)i * w + i] / g : 0.0;     // S_ii / (1 - R_ii)
    lam_out[i] = lam;
    lmax = fmax(lmax, fabs(lam));
  }
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e % w;
    const double r = (i == j ? 1.0 : 0.0) - Gx[e];
    off_r += r * r;
    if (i != j) off_s += S[e] * S[e];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    off_s += __shfl_xor_sync(0xffffffffu, off_s, o);
    off_r += __shfl_xor_sync(0xffffffffu, off_r, o);
    lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  }
  if (lane == 0) {
    red_s[warp] = off_s;
    red_r[warp] = off_r;
    lmax_s[warp] = lmax;
  }
  __syncthreads();
  if (warp == 0) {
    double a = lane < nw ? red_s[lane] : 0.0, b = lane < nw ? red_r[lane] : 0.0,
           c = lane < nw ? lmax_s[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c = fmax(c, __shfl_xor_sync(0xffffffffu, c, o));
    }
    // first-order terms are reliable only for gaps well above their size
    if (lane == 0) lam_out[w] = 2.0 * (sqrt(a) + c * sqrt(b));
  }
}

__global__ void k_refine_apply(int w, const double* __restrict__ S, const double* Gx,
                               const double* __restrict__ lam, double* E) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= w * w) return;
  const int i = e / w, j = e % w;
  const double delta = lam[w];
  const double r = (i == j ? 1.0 : 0.0) - Gx[e];
  double v;
  if (i == j) {
    v = 0.5 * r;
  } else {
    const double gap = lam[j] - lam[i];
    v = fabs(gap) > delta ? (S[e] + lam[j] * r) / gap : 0.5 * r;
  }
  E[e] = v;
}

// B (upper triangular, w x w, FP64 container) with B^T B = G + delta I to
// FP32 accuracy: right-looking Cholesky in FP32 in shared memory, one CTA
// of 32 x 32 threads (thread (ty, tx) updates rows ty + 32 a, columns
// tx + 32 b of the trailing matrix, no index division in the loop).  Row k
// of the trailing matrix is left unscaled (c_kj = r_kk r_kj) and the update
// is c_ij -= c_ki c_kj / c_kk, so each pivot needs one barrier; the rows
// are scaled by 1 / r_kk on the way out.
// It only preconditions Step 4 (its output seeds the FP32 Jacobi sweeps,
// whose vectors are then refined in FP64 against G itself), so a shift
// delta = 1e-6 max diag(G) keeps it defined whatever G's conditioning: the
// shift moves every eigenvalue by delta and no eigenvector.
__global__ void __launch_bounds__(1024) k_chol32_shift(int w, const double* __restrict__ G, double* __restrict__ B) {
  extern __shared__ float cm[];                 // w x ws
  const int ws = w | 1;
  __shared__ float dmax, rowk[256];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  if (tid == 0) dmax = 0.f;
  __syncthreads();
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e % w;
    cm[i * ws + j] = (float)G[e];
    if (i == j) atomicMax(reinterpret_cast<int*>(&dmax), __float_as_int(fmaxf((float)G[e], 0.f)));
  }
  __syncthreads();
  const float delta = 1e-6f * dmax;
  for (int i = tid; i < w; i += blockDim.x) cm[i * ws + i] += delta;
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    // pivot c_kk (floored at the shift: rounding cannot make it vanish)
    const float ck = fmaxf(cm[k * ws + k], delta);
    const float inv = __fdividef(1.f, ck);
    if (tid == 0) rowk[k] = ck;
    // trailing update c_ij -= c_ki c_kj / c_kk for k < i <= j (row k unchanged)
    for (int i = k + 1 + ty; i < w; i += 32) {
      const float a = cm[k * ws + i] * inv;
      for (int j = i + tx; j < w; j += 32) cm[i * ws + j] = fmaf(-a, cm[k * ws + j], cm[i * ws + j]);
    }
    __syncthreads();
  }
  // r_kk = sqrt(c_kk), r_kj = c_kj / r_kk
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e % w;
    const float rs = rsqrtf(rowk[i]);
    B[e] = j > i ? (double)(cm[i * ws + j] * rs) : (j == i ? (double)(rowk[i] * rs) : 0.0);
  }
}

// Eigenvalues lambda_j = S_jj of the refined S = X^T G X, sorted
// descending: sigma_j = sqrt(lambda_j) (S_out), W = X with its columns in
// that order, and Vs = W diag(1/sigma) (the factor that takes T to its left
// singular vectors, V = T W Sigma^-1).  CTA c moves column c.
__global__ void k_eig_finish(int w, const double* __restrict__ Sm, const double* __restrict__ X,
                             double* __restrict__ S_out, double* __restrict__ Vs, double* __restrict__ W) {
  const int c = blockIdx.x;
  __shared__ int rank;
  __shared__ double sc;
  if (threadIdx.x == 0) {
    rank = 0;
    sc = sqrt(fmax(Sm[(int64_t)c * w + c], 0.0));
  }
  __syncthreads();
  int r = 0;
  for (int o = threadIdx.x; o < w; o += blockDim.x) {
    const double so = sqrt(fmax(Sm[(int64_t)o * w + o], 0.0));
    r += (so > sc) || (so == sc && o < c);
  }
  atomicAdd(&rank, r);
  __syncthreads();
  const int d = rank;
  const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
  for (int row = threadIdx.x; row < w; row += blockDim.x) {
    const double x = X[(int64_t)row * w + c];
    W[(int64_t)row * w + d] = x;
    Vs[(int64_t)row * w + d] = x * inv;
  }
  if (threadIdx.x == 0) S_out[d] = sc;
}

}  // namespace

void chol32_shift(int w, const double* G, double* B, cudaStream_t st) {
  const size_t smem = (size_t)w * (w | 1) * sizeof(float);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_chol32_shift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_chol32_shift<<<1, 1024, smem, st>>>(w, G, B);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void eig_finish(int w, const double* Sm, const double* X, double* S, double* Vs, double* W, cudaStream_t st) {
  k_eig_finish<<<w, 128, 0, st>>>(w, Sm, X, S, Vs, W);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void gemm64_small(int M, int N, int K, double alpha, const double* A, int64_t lda, bool ta, const double* B,
                  int64_t ldb, bool tb, double beta, const double* D, int64_t ldd, double* C, int64_t ldc,
                  cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)cdiv(N, T64), (unsigned)cdiv(M, T64));
  k_gemm64_small<<<grid, T64 * T64, 0, st>>>(M, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, D, ldd,
                                            C, ldc);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void refine_eigvecs64(int w, const double* B, double* X, double* Xn, double* P, double* S, double* E, int steps,
                      cudaStream_t st, bool gram_given) {
  double* cur = X;
  double* nxt = Xn;
  for (int it = 0; it < steps; ++it) {
    gemm64_small(w, w, w, 1.0, B, w, false, cur, w, false, 0.0, nullptr, 0, P, w, st);   // P = B X (or G X)
    if (gram_given)
      gemm64_small(w, w, w, 1.0, cur, w, true, P, w, false, 0.0, nullptr, 0, S, w, st);  // S = X^T G X
    else
      gemm64_small(w, w, w, 1.0, P, w, true, P, w, false, 0.0, nullptr, 0, S, w, st);   // S = P^T P
    gemm64_small(w, w, w, 1.0, cur, w, true, cur, w, false, 0.0, nullptr, 0, E, w, st); // X^T X
    // lambda (w values) and delta in the first row of Xn, free until the update
    k_refine_stats<<<1, 1024, 0, st>>>(w, S, E, nxt);
    RPCA_CUDA_TRY(cudaGetLastError());
    k_refine_apply<<<(unsigned)cdiv((int64_t)w * w, 256), 256, 0, st>>>(w, S, E, nxt, E);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch(2);
    gemm64_small(w, w, w, 1.0, cur, w, false, E, w, false, 1.0, cur, w, nxt, w, st);    // X (I + E)
    std::swap(cur, nxt);
  }
  if (cur != X) RPCA_CUDA_TRY(cudaMemcpyAsync(X, cur, (size_t)w * w * sizeof(double), cudaMemcpyDeviceToDevice, st));
}

}  // namespace rpca
