// Kernels of the adjoint (gradient of a function of the k computed singular
// values with respect to A): small FP64 algebra, column scalings, and the
// streamed write of the gradient, which is a low-rank product P Z^T.
#include "common.cuh"
#include "kernels.h"

namespace rpca {
namespace {

template <typename T> __device__ __forceinline__ double ld64(const T* p) { return (double)*p; }

// out = (M^-1)^T, M p x p FP64 (ldm), by Gauss-Jordan elimination with
// partial pivoting on [M | I] (aug: p x 2p FP64 scratch).  One CTA.  A pivot
// that is zero or not finite sets DEV_ERR_BREAKDOWN and leaves out = 0.
__global__ void k_small_inv_t(int p, const double* __restrict__ M, int64_t ldm, double* __restrict__ aug,
                              double* __restrict__ out, uint32_t* __restrict__ dev_err) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int w2 = 2 * p;
  for (int e = tid; e < p * w2; e += nt) {
    const int i = e / w2, j = e % w2;
    aug[e] = j < p ? M[(int64_t)i * ldm + j] : (j - p == i ? 1.0 : 0.0);
  }
  __shared__ int piv;
  __shared__ double amax;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < p; ++c) {
    if (tid == 0) {
      // pivot row: largest |aug[r][c]|, r >= c (serial: p <= 256)
      int best = c;
      double bv = fabs(aug[(int64_t)c * w2 + c]);
      for (int r = c + 1; r < p; ++r) {
        const double v = fabs(aug[(int64_t)r * w2 + c]);
        if (v > bv) { bv = v; best = r; }
      }
      piv = best;
      amax = bv;
      if (!(bv > 0.0) || !isfinite(bv)) bad = 1;
    }
    __syncthreads();
    if (bad) break;
    if (piv != c)
      for (int j = tid; j < w2; j += nt) {
        const double t = aug[(int64_t)c * w2 + j];
        aug[(int64_t)c * w2 + j] = aug[(int64_t)piv * w2 + j];
        aug[(int64_t)piv * w2 + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / aug[(int64_t)c * w2 + c];
    for (int j = tid; j < w2; j += nt) aug[(int64_t)c * w2 + j] *= inv;
    __syncthreads();
    for (int e = tid; e < p * w2; e += nt) {
      const int r = e / w2, j = e % w2;
      if (r != c) {
        const double f = aug[(int64_t)r * w2 + c];
        if (j != c) aug[e] -= f * aug[(int64_t)c * w2 + j];
      }
    }
    __syncthreads();
    for (int r = tid; r < p; r += nt)
      if (r != c) aug[(int64_t)r * w2 + c] = 0.0;
    __syncthreads();
  }
  (void)amax;
  for (int e = tid; e < p * p; e += nt) {
    const int i = e / p, j = e % p;
    out[e] = bad ? 0.0 : aug[(int64_t)j * w2 + p + i];   // transpose of the inverse
  }
  if (tid == 0 && bad) atomicOr(dev_err, DEV_ERR_BREAKDOWN);
}

// Mk (k x w FP64) = diag(c) W[:, :k]^T, W w x w row-major.
__global__ void k_make_mk(int k, int w, const double* __restrict__ c, const double* __restrict__ W,
                          double* __restrict__ Mk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * w) return;
  const int j = e / w, q = e % w;
  Mk[e] = c[j] * W[(int64_t)q * w + j];
}

// out[r, j] = V[r, j] * c[j]  (rows x k, compute type)
template <typename T>
__global__ void k_scale_cols(int64_t rows, int k, const T* __restrict__ V, int64_t ldv, const double* __restrict__ c,
                             T* __restrict__ out, int64_t ldo) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * k) return;
  const int64_t r = e / k;
  const int j = (int)(e % k);
  out[r * ldo + j] = (T)((double)V[r * ldv + j] * c[j]);
}

// dst += src (rows x cols, compute type)
template <typename T>
__global__ void k_add_matrix(int64_t rows, int cols, const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                             int64_t ldd) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e / cols;
  const int c = (int)(e % cols);
  dst[r * ldd + c] += src[r * lds + c];
}

// G (m x n, ldg) = P Z^T with P m x r, Z n x r (compute type): 64 x 64 output
// tiles, 256 threads (4 x 4 outputs each), K = r in chunks of 16 through
// shared memory; accumulation in the compute type.
template <typename T>
__global__ void __launch_bounds__(256) k_lowrank_out(int64_t m, int64_t n, int r, const T* __restrict__ P,
                                                     int64_t ldp, const T* __restrict__ Z, int64_t ldz,
                                                     T* __restrict__ G, int64_t ldg) {
  __shared__ T ps[16][65];
  __shared__ T zs[16][65];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.y * 64, col0 = (int64_t)blockIdx.x * 64;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < r; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, ii = e % 64;
      const int64_t pr = row0 + ii, zr = col0 + ii;
      ps[kk][ii] = (pr < m && k0 + kk < r) ? P[pr * ldp + k0 + kk] : T(0);
      zs[kk][ii] = (zr < n && k0 + kk < r) ? Z[zr * ldz + k0 + kk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = ps[kk][ty * 4 + q];
        b[q] = zs[kk][tx * 4 + q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += a[x] * b[y];
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t gr = row0 + ty * 4 + x;
    if (gr >= m) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t gc = col0 + tx * 4 + y;
      if (gc < n) G[gr * ldg + gc] = acc[x][y];
    }
  }
}

unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void small_inv_t(int p, const double* M, int64_t ldm, double* aug, double* out, uint32_t* dev_err, cudaStream_t st) {
  k_small_inv_t<<<1, 256, 0, st>>>(p, M, ldm, aug, out, dev_err);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void make_mk(int k, int w, const double* c, const double* W, double* Mk, cudaStream_t st) {
  k_make_mk<<<blocks((int64_t)k * w), 256, 0, st>>>(k, w, c, W, Mk);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void scale_cols(bool f64, int64_t rows, int k, const void* V, int64_t ldv, const double* c, void* out, int64_t ldo,
                cudaStream_t st) {
  if (f64)
    k_scale_cols<double><<<blocks(rows * k), 256, 0, st>>>(rows, k, (const double*)V, ldv, c, (double*)out, ldo);
  else
    k_scale_cols<float><<<blocks(rows * k), 256, 0, st>>>(rows, k, (const float*)V, ldv, c, (float*)out, ldo);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void add_matrix(bool f64, int64_t rows, int cols, const void* src, int64_t lds, void* dst, int64_t ldd,
                cudaStream_t st) {
  if (f64)
    k_add_matrix<double><<<blocks(rows * cols), 256, 0, st>>>(rows, cols, (const double*)src, lds, (double*)dst, ldd);
  else
    k_add_matrix<float><<<blocks(rows * cols), 256, 0, st>>>(rows, cols, (const float*)src, lds, (float*)dst, ldd);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void lowrank_out(bool f64, int64_t m, int64_t n, int r, const void* P, int64_t ldp, const void* Z, int64_t ldz,
                 void* G, int64_t ldg, cudaStream_t st) {
  dim3 grid((unsigned)((n + 63) / 64), (unsigned)((m + 63) / 64));
  if (f64)
    k_lowrank_out<double><<<grid, 256, 0, st>>>(m, n, r, (const double*)P, ldp, (const double*)Z, ldz, (double*)G, ldg);
  else
    k_lowrank_out<float><<<grid, 256, 0, st>>>(m, n, r, (const float*)P, ldp, (const float*)Z, ldz, (float*)G, ldg);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

}  // namespace rpca
