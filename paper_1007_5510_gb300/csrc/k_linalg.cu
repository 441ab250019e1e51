// Small and tall-skinny linear algebra around the streamed passes:
//   Step 2 (QR of H): block Gram-Schmidt twice + Cholesky QR twice, Gram
//           matrices accumulated in FP64, Cholesky in FP64;
//   Step 4 (SVD of T): QR of T the same way, then one-sided Jacobi on its
//           triangular factor;
//   Steps 5-6 and the centring corrections: tall x small products.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "kernels.h"

namespace rpca {

namespace {

template <typename TC>
__device__ __forceinline__ TC ld_or0(const TC* p, bool ok) { return ok ? *p : TC(0); }

// ------------------------------------------------------------------- Gram
// C[p0.., q0..] += X^T Y over this block's rows.  256 threads, 64 x 64 tile.
// Products summed in the compute type over SUB rows, then in FP64.
template <typename TC>
__global__ void __launch_bounds__(256)
k_gram(int64_t m, int p, int q, const TC* __restrict__ X, int64_t ldx, const TC* __restrict__ Y,
       int64_t ldy, double* __restrict__ C, int64_t ldc, int64_t rows_per_block,
       const uint32_t* __restrict__ active) {
  if (active && *active == 0u) return;
  constexpr int RC = 32;                       // rows per smem chunk
  constexpr int SUB = 256;                     // rows per FP64 flush
  __shared__ TC Xs[RC][64 + 1];
  __shared__ TC Ys[RC][64 + 1];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int p0 = blockIdx.y * 64, q0 = blockIdx.z * 64;
  const int64_t rbeg = (int64_t)blockIdx.x * rows_per_block;
  const int64_t rend = min(m, rbeg + rows_per_block);
  TC acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = TC(0); dacc[a][b] = 0.0; }
  int since = 0;
  for (int64_t r0 = rbeg; r0 < rend; r0 += RC) {
    for (int e = tid; e < RC * 64; e += 256) {
      int rr = e / 64, cc = e % 64;
      int64_t r = r0 + rr;
      bool rok = r < rend;
      Xs[rr][cc] = ld_or0(X + r * ldx + p0 + cc, rok && p0 + cc < p);
      Ys[rr][cc] = ld_or0(Y + r * ldy + q0 + cc, rok && q0 + cc < q);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < RC; ++rr) {
      TC xv[4], yv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = Xs[rr][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yv[b] = Ys[rr][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xv[a], yv[b], acc[a][b]);
    }
    __syncthreads();
    since += RC;
    if (since >= SUB) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { dacc[a][b] += (double)acc[a][b]; acc[a][b] = TC(0); }
      since = 0;
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = p0 + ty * 4 + a, j = q0 + tx * 4 + b;
      if (i < p && j < q) atomicAdd(&C[(int64_t)i * ldc + j], dacc[a][b] + (double)acc[a][b]);
    }
}

// ------------------------------------------------------------------ X * M
template <typename TC, int BM>
__global__ void __launch_bounds__(256)
k_gemm_xm(int64_t m, int p, int q, const TC* __restrict__ X, int64_t ldx,
          const double* __restrict__ M, int64_t ldm, double alpha, double beta, TC* Y, int64_t ldy,
          const uint32_t* __restrict__ active) {
  if (active && *active == 0u) return;
  constexpr int RPT = BM / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* Xs = reinterpret_cast<TC*>(smem_raw);          // [BM][p]
  TC* Ms = Xs + BM * p;                               // [p][64]
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t nblk = (m + BM - 1) / BM;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t r0 = blk * BM;
    for (int e = tid; e < BM * p; e += 256) {
      int rr = e / p, kk = e % p;
      int64_t r = r0 + rr;
      Xs[e] = (r < m) ? X[r * ldx + kk] : TC(0);
    }
    __syncthreads();                                  // rows staged before any write
    for (int c0 = 0; c0 < q; c0 += 64) {
      for (int e = tid; e < p * 64; e += 256) {
        int kk = e / 64, cc = e % 64;
        Ms[e] = (c0 + cc < q) ? TC(alpha * M[(int64_t)kk * ldm + c0 + cc]) : TC(0);
      }
      __syncthreads();
      TC acc[RPT][4];
#pragma unroll
      for (int a = 0; a < RPT; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TC(0);
      for (int kk = 0; kk < p; ++kk) {
        TC mv[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) mv[b] = Ms[kk * 64 + tx * 4 + b];
#pragma unroll
        for (int a = 0; a < RPT; ++a) {
          TC xv = Xs[(ty * RPT + a) * p + kk];
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(xv, mv[b], acc[a][b]);
        }
      }
#pragma unroll
      for (int a = 0; a < RPT; ++a) {
        int64_t r = r0 + ty * RPT + a;
        if (r >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int c = c0 + tx * 4 + b;
          if (c < q) {
            TC* y = Y + r * ldy + c;
            *y = (beta == 0.0) ? acc[a][b] : TC(beta) * (*y) + acc[a][b];
          }
        }
      }
      __syncthreads();
    }
  }
}

// --------------------------------------------------------------- Cholesky
// One CTA.  G = R^T R (R upper), then Rinv by back substitution, both in
// shared memory (p <= 64) or global memory (larger p).
// Pass `pass` (0..kCholPasses-1) of a Cholesky-QR sequence on one block (qf:
// kQfWords words private to the block: qf[0] = which passes needed a shift,
// qf[1] = some pass needed one (gates the re-orthogonalisation against the
// earlier blocks), qf[p] (p >= 2) = whether pass p runs).
// A pivot below piv_rel * max(diag G) retries with G + shift_rel * max(diag G) I
// (shifted Cholesky QR); pass p >= 2 runs only if pass p-1 or p-2 needed a
// shift, and otherwise leaves identities (exact no-ops).  Each shifted pass
// multiplies the directions a numerically rank-deficient block is missing by
// about 1/sqrt(shift_rel), so a block whose missing directions start at the
// rounding level needs a few of them before an unshifted pass.
// 1 / sqrt(d) for d > 0 in FP64: an FP32 seed refined by Newton-Raphson
// steps y <- y (3 - d y^2) / 2 (quadratic convergence: ~2^-22 -> 2^-44 ->
// below FP64 rounding).  A short chain of multiplies instead of a division
// and a square root; one step (2^-44) when the factor only feeds FP32 work.
__device__ __forceinline__ double rsqrt_newton(double d, bool two_steps) {
  double y = (double)rsqrtf((float)d);
  y = y * (1.5 - 0.5 * d * y * y);
  if (two_steps) y = y * (1.5 - 0.5 * d * y * y);
  return y;
}

// p <= 64, in shared memory.  FP64 Cholesky by 16-column blocks: warp 0
// factors the diagonal block (warp-synchronous), then the whole CTA solves
// the block row (one column per thread) and updates the trailing triangle.
// Rinv = R^-1 = U^-1 D^-1 with R = D U (U unit upper triangular): U^-1 by
// right-looking elimination, one barrier per step (U^-1's row k is final at
// step k), then scaled by columns; in FP32 when inv_f32 (the factor then
// only feeds FP32 / BF16-slice products, whose own rounding is of the same
// order), else FP64.
__global__ void __launch_bounds__(256)
k_chol(int p, const double* __restrict__ G, int64_t ldg, double* __restrict__ Rout,
       double* __restrict__ Rinvout, int pass, double piv_rel, double shift_rel, uint32_t* qf,
       uint32_t* dev_err, int inv_f32, const uint32_t* __restrict__ gate) {
  if (gate && *gate == 0u) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int fail;
  __shared__ double dmax;
  __shared__ double dinv[64];
  extern __shared__ double sm_chol[];
  const int ps = p | 1;                                  // odd row stride (banks)
  double* R = sm_chol;                                   // p x ps
  double* X64 = sm_chol + p * ps;                        // p x ps (FP64 inverse)
  float* X32 = reinterpret_cast<float*>(X64);            // p x ps (FP32 inverse)
  const bool active = (pass < 2) || (qf[pass] != 0u);
  if (!active) {
    for (int e = tid; e < p * p; e += blockDim.x) {
      double v = (e / p == e % p) ? 1.0 : 0.0;
      Rout[e] = v;
      Rinvout[e] = v;
    }
    if (tid == 0 && pass + 1 < kCholPasses) qf[pass + 1] = 0u;
    return;
  }
  if (tid == 0) {
    dmax = 0.0;
    if (pass == 0) {
      qf[0] = 0u;
      qf[1] = 0u;
    }
  }
  // G -> shared memory (all of it: the near-identity branch reads it all)
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    R[i * ps + j] = G[(int64_t)i * ldg + j];
  }
  __syncthreads();
  for (int i = tid; i < p; i += blockDim.x) {
    // diagonal entries are non-negative: their bit patterns order like integers
    atomicMax(reinterpret_cast<unsigned long long*>(&dmax),
              (unsigned long long)__double_as_longlong(fmax(R[i * ps + i], 0.0)));
  }
  __syncthreads();
  if (pass >= 1) {
    // A later pass of the sequence sees G = I + E with E tiny.  Then
    // M = (I + E)^(-1/2) = I - E/2 + 3/8 E^2 + O(E^3) orthonormalises the
    // block as well as R^-1 does (same span, (H M)^T (H M) = I + O(E^3)),
    // and its inverse is I + E/2 - E^2/8 + O(E^3).  E^2 only needs a few
    // digits: it is formed in FP32.
    __shared__ unsigned long long emax_bits;
    if (tid == 0) emax_bits = 0ull;
    __syncthreads();
    {
      // max |G - I| (non-negative doubles order like their bit patterns):
      // per thread, then per warp, then one shared atomic per warp
      unsigned long long mb = 0ull;
      for (int e = tid; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        const double d = fabs(R[i * ps + j] - (i == j ? 1.0 : 0.0));
        const unsigned long long b = (unsigned long long)__double_as_longlong(isfinite(d) ? d : 1e300);
        mb = b > mb ? b : mb;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = t > mb ? t : mb;
      }
      if (lane == 0) atomicMax(&emax_bits, mb);
    }
    __syncthreads();
    if (__longlong_as_double((long long)emax_bits) < 2e-3) {
      float* Ef = X32;                                   // p x ps
      for (int e = tid; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        Ef[i * ps + j] = (float)(R[i * ps + j] - (i == j ? 1.0 : 0.0));
      }
      __syncthreads();
      // E^2 in strips of 4 columns (independent accumulators)
      const int nst = (p + 3) / 4;
      for (int t = tid; t < p * nst; t += blockDim.x) {
        const int i = t / nst, j0 = 4 * (t % nst);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < p; ++k) {
          const float a = Ef[i * ps + k];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (j0 + u < p) acc[u] = fmaf(a, Ef[k * ps + j0 + u], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          if (j >= p) break;
          const double exact = R[i * ps + j] - (i == j ? 1.0 : 0.0);
          const double id = i == j ? 1.0 : 0.0;
          Rinvout[i * p + j] = id - 0.5 * exact + 0.375 * (double)acc[u];
          Rout[i * p + j] = id + 0.5 * exact - 0.125 * (double)acc[u];
        }
      }
      if (tid == 0) {
        if (pass + 1 < kCholPasses) qf[pass + 1] = ((qf[0] >> (pass - 1)) & 3u) ? 1u : 0u;
      }
      return;
    }
  }
  bool shifted = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double shift = (attempt == 0) ? 0.0 : shift_rel * dmax;
    // the shifted retry: a missing direction's pivot is the shift plus or
    // minus rounding, so only a pivot below half the shift is a failure
    const double piv_min = (attempt == 0) ? piv_rel * dmax : 0.5 * shift;
    if (attempt == 1) {
      // restart from G + shift I (upper triangle)
      for (int e = tid; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        if (j >= i) R[i * ps + j] = G[(int64_t)i * ldg + j] + (i == j ? shift : 0.0);
      }
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int kb = 0; kb < p; kb += 16) {
      const int bs = min(16, p - kb);
      if (warp == 0) {
        // ---- diagonal block [kb, kb + bs): right-looking, warp-synchronous
        for (int k = kb; k < kb + bs; ++k) {
          const double d = R[k * ps + k];
          const bool bad = !(d > piv_min) || !isfinite(d);
          if (bad) {
            if (lane == 0) fail = 1;
            break;
          }
          double y = 0.0;
          if (lane == 0) y = rsqrt_newton(d, !inv_f32);
          y = __shfl_sync(0xffffffffu, y, 0);
          const int j = kb + lane;
          if (lane == 0) dinv[k] = y;
          if (j > k && j < kb + bs) R[k * ps + j] *= y;
          if (j == k) R[k * ps + k] = d * y;
          __syncwarp();
          // rank-1 update of the block's trailing triangle, element-parallel
          const int r = kb + bs - k - 1;                 // trailing size
          for (int e = lane; e < r * r; e += 32) {
            const int ii = k + 1 + e / r, jj = k + 1 + e % r;
            if (jj >= ii) R[ii * ps + jj] -= R[k * ps + ii] * R[k * ps + jj];
          }
          __syncwarp();
        }
      }
      __syncthreads();
      if (fail) break;
      // ---- block row: R[kb+t][c] for c >= kb + bs, forward substitution
      for (int c = kb + bs + tid; c < p; c += blockDim.x) {
        for (int k = kb; k < kb + bs; ++k) {
          double v = R[k * ps + c];
          for (int t = kb; t < k; ++t) v -= R[t * ps + k] * R[t * ps + c];
          R[k * ps + c] = v * dinv[k];
        }
      }
      __syncthreads();
      // ---- trailing update: R[i][j] -= sum_t R[t][i] R[t][j], i <= j
      const int r0 = kb + bs, rn = p - r0;
      for (int e = tid; e < rn * rn; e += blockDim.x) {
        const int i = r0 + e / rn, j = r0 + e % rn;
        if (j < i) continue;
        double v = R[i * ps + j];
        for (int t = kb; t < kb + bs; ++t) v -= R[t * ps + i] * R[t * ps + j];
        R[i * ps + j] = v;
      }
      __syncthreads();
    }
    __syncthreads();
    if (!fail) break;
    if (attempt == 1 || !(dmax > 0.0) || !isfinite(dmax)) {
      if (tid == 0) atomicOr(dev_err, DEV_ERR_BREAKDOWN);
      for (int e = tid; e < p * p; e += blockDim.x) {
        double v = (e / p == e % p) ? 1.0 : 0.0;
        Rout[e] = v;
        Rinvout[e] = v;
      }
      return;
    }
    shifted = true;
    __syncthreads();
  }
  if (tid == 0) {
    if (shifted) {
      qf[0] |= 1u << pass;
      qf[1] = 1u;
      atomicOr(dev_err, DEV_ERR_SHIFTED);
      if (pass == kCholPasses - 1) atomicOr(dev_err, DEV_ERR_BREAKDOWN);
    }
    if (pass >= 1 && pass + 1 < kCholPasses) qf[pass + 1] = ((qf[0] >> (pass - 1)) & 3u) ? 1u : 0u;
  }
  // ---- Rinv.  U[i][c] = R[i][c] * dinv[i] (i < c).  X = U^-1 (unit upper):
  // at step k (from the bottom) row k of X is final; rows i < k receive
  // -U[i][k] * row k.  Then Rinv[i][c] = X[i][c] * dinv[c].
  float* U32 = X32 + p * ps;                              // FP32 copy of U (the X64 region's second half)
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int i = e / p, c = e % p;
    Rout[e] = c >= i ? R[i * ps + c] : 0.0;
    if (inv_f32) {
      X32[i * ps + c] = (i == c) ? 1.0f : 0.f;
      U32[i * ps + c] = c > i ? (float)(R[i * ps + c] * dinv[i]) : 0.f;
    } else {
      X64[i * ps + c] = (i == c) ? 1.0 : 0.0;
    }
  }
  __syncthreads();
  for (int k = p - 1; k >= 1; --k) {
    // rows i < k, columns c in [k, p)
    const int nc = p - k;
    for (int e = tid; e < k * nc; e += blockDim.x) {
      const int i = e / nc, c = k + e % nc;
      if (inv_f32) {
        X32[i * ps + c] = fmaf(-U32[i * ps + k], X32[k * ps + c], X32[i * ps + c]);
      } else {
        const double u = R[i * ps + k] * dinv[i];
        X64[i * ps + c] -= u * X64[k * ps + c];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int i = e / p, c = e % p;
    const double x = inv_f32 ? (double)X32[i * ps + c] : X64[i * ps + c];
    Rinvout[e] = c >= i ? x * dinv[c] : 0.0;
  }
}

__global__ void __launch_bounds__(256)
k_chol_global(int p, const double* __restrict__ G, int64_t ldg, double* __restrict__ Rout,
       double* __restrict__ Rinvout, int pass, double piv_rel, double shift_rel, uint32_t* qf,
       uint32_t* dev_err, const uint32_t* __restrict__ gate) {
  if (gate && *gate == 0u) return;
  const int tid = threadIdx.x;
  __shared__ int fail;
  __shared__ double dmax;
  extern __shared__ double sm_chol[];
  const bool in_smem = p <= 64;
  double* R = in_smem ? sm_chol : Rout;
  double* Rinv = in_smem ? sm_chol + p * p : Rinvout;
  const bool active = (pass < 2) || (qf[pass] != 0u);
  if (!active) {
    for (int e = tid; e < p * p; e += blockDim.x) {
      double v = (e / p == e % p) ? 1.0 : 0.0;
      Rout[e] = v;
      Rinvout[e] = v;
    }
    if (tid == 0 && pass + 1 < kCholPasses) qf[pass + 1] = 0u;
    return;
  }
  if (tid == 0) {
    dmax = 0.0;
    if (pass == 0) {
      qf[0] = 0u;
      qf[1] = 0u;
    }
  }
  __syncthreads();
  for (int i = tid; i < p; i += blockDim.x) {
    // diagonal entries are non-negative: their bit patterns order like integers
    atomicMax(reinterpret_cast<unsigned long long*>(&dmax),
              (unsigned long long)__double_as_longlong(fmax(G[(int64_t)i * ldg + i], 0.0)));
  }
  __syncthreads();
  if (pass >= 1 && in_smem) {
    // A later pass of the sequence sees G = I + E with E tiny.  Then
    // M = (I + E)^(-1/2) = I - E/2 + 3/8 E^2 + O(E^3) orthonormalises the
    // block as well as R^-1 does (same span, (H M)^T (H M) = I + O(E^3)),
    // and its inverse is I + E/2 - E^2/8 + O(E^3).  E^2 only needs a few
    // digits: it is formed in FP32.
    __shared__ unsigned long long emax_bits;
    if (tid == 0) emax_bits = 0ull;
    __syncthreads();
    {
      // max |G - I| (non-negative doubles order like their bit patterns):
      // per thread, then per warp, then one shared atomic per warp
      unsigned long long mb = 0ull;
      for (int e = tid; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        const double d = fabs(G[(int64_t)i * ldg + j] - (i == j ? 1.0 : 0.0));
        const unsigned long long b = (unsigned long long)__double_as_longlong(isfinite(d) ? d : 1e300);
        mb = b > mb ? b : mb;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = t > mb ? t : mb;
      }
      if ((tid & 31) == 0) atomicMax(&emax_bits, mb);
    }
    __syncthreads();
    if (__longlong_as_double((long long)emax_bits) < 2e-3) {
      float* Ef = reinterpret_cast<float*>(sm_chol);        // p x p
      for (int e = tid; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        Ef[e] = (float)(G[(int64_t)i * ldg + j] - (i == j ? 1.0 : 0.0));
      }
      __syncthreads();
      for (int e = tid; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        float e2 = 0.f;
        for (int k = 0; k < p; ++k) e2 = fmaf(Ef[i * p + k], Ef[k * p + j], e2);
        const double ee = G[(int64_t)i * ldg + j] - (i == j ? 1.0 : 0.0);
        const double id = i == j ? 1.0 : 0.0;
        Rinvout[e] = id - 0.5 * ee + 0.375 * (double)e2;
        Rout[e] = id + 0.5 * ee - 0.125 * (double)e2;
      }
      if (tid == 0) {
        if (pass + 1 < kCholPasses) qf[pass + 1] = ((qf[0] >> (pass - 1)) & 3u) ? 1u : 0u;
      }
      return;
    }
  }
  bool shifted = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double shift = (attempt == 0) ? 0.0 : shift_rel * dmax;
    for (int e = tid; e < p * p; e += blockDim.x) {
      int i = e / p, j = e % p;
      R[e] = (j >= i) ? G[(int64_t)i * ldg + j] + (i == j ? shift : 0.0) : 0.0;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    // the pivot's square root and reciprocal: computed once per step (FP64
    // division and square root are long instruction sequences) and shared
    __shared__ double piv_r[2];
    const double piv_min = (attempt == 0) ? piv_rel * dmax : 0.5 * shift;
    for (int k = 0; k < p; ++k) {
      double d = R[k * p + k];
      bool bad = !(d > piv_min) || !isfinite(d);
      if (bad) {
        if (tid == 0) fail = 1;
        break;
      }
      if (tid == 0) {
        const double rkk0 = sqrt(d);
        piv_r[0] = rkk0;
        piv_r[1] = 1.0 / rkk0;
      }
      __syncthreads();
      const double rkk = piv_r[0];
      const double irkk = piv_r[1];
      for (int j = k + tid; j < p; j += blockDim.x) R[k * p + j] = (j == k) ? rkk : R[k * p + j] * irkk;
      __syncthreads();
      // trailing update of the upper triangle, 16 x 16 thread tile (no
      // index division in the loop)
      {
        const int ty = tid >> 4, tx = tid & 15;
        for (int i = k + 1 + ty; i < p; i += 16) {
          const double rki = R[k * p + i];
          for (int j = i + tx; j < p; j += 16) R[i * p + j] -= rki * R[k * p + j];
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!fail) break;
    if (attempt == 1 || !(dmax > 0.0) || !isfinite(dmax)) {
      if (tid == 0) atomicOr(dev_err, DEV_ERR_BREAKDOWN);
      for (int e = tid; e < p * p; e += blockDim.x) {
        double v = (e / p == e % p) ? 1.0 : 0.0;
        Rout[e] = v;
        Rinvout[e] = v;
      }
      return;
    }
    shifted = true;
    __syncthreads();
  }
  if (tid == 0) {
    if (shifted) {
      qf[0] |= 1u << pass;
      qf[1] = 1u;
      atomicOr(dev_err, DEV_ERR_SHIFTED);
      if (pass == kCholPasses - 1) atomicOr(dev_err, DEV_ERR_BREAKDOWN);
    }
    if (pass >= 1 && pass + 1 < kCholPasses) qf[pass + 1] = ((qf[0] >> (pass - 1)) & 3u) ? 1u : 0u;
  }
  // Rinv = R^-1: rows from the bottom up, all columns in parallel
  for (int e = tid; e < p * p; e += blockDim.x) Rinv[e] = 0.0;
  __syncthreads();
  // Rinv = R^-1 by right-looking back substitution on all columns at once:
  // step k (from the bottom): row k of Rinv is final after scaling by
  // 1/R[k][k]; then rows 0..k-1 receive -R[i][k] * row k.  Every update of a
  // step is independent (no long dependent FP64 chains).
  __shared__ double rdiag[256];
  for (int i = tid; i < p && i < 256; i += blockDim.x) rdiag[i] = 1.0 / R[i * p + i];
  for (int e = tid; e < p * p; e += blockDim.x) Rinv[e] = (e / p == e % p) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = p - 1; k >= 0; --k) {
    const double rk = p <= 256 ? rdiag[k] : 1.0 / R[k * p + k];
    for (int c = k + tid; c < p; c += blockDim.x) Rinv[k * p + c] *= rk;
    __syncthreads();
    const int ty = tid >> 4, tx = tid & 15;
    for (int i = ty; i < k; i += 16) {
      const double rik = R[i * p + k];
      for (int c = k + tx; c < p; c += 16) Rinv[i * p + c] -= rik * Rinv[k * p + c];
    }
    __syncthreads();
  }
  if (in_smem) {
    for (int e = tid; e < p * p; e += blockDim.x) {
      Rout[e] = R[e];
      Rinvout[e] = Rinv[e];
    }
  }
}

// Racc (p x p) = Rk * Racc, FP64, one CTA (accumulates the triangular
// factor of a Cholesky-QR sequence: H = Q (R3 R2 R1 R0)).
__global__ void k_left_mul(int p, const double* __restrict__ Rk, double* __restrict__ Racc) {
  extern __shared__ double tmp[];
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    int i = e / p, j = e % p;
    double s = 0.0;
    for (int t = 0; t < p; ++t) s += Rk[i * p + t] * Racc[t * p + j];
    tmp[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) Racc[e] = tmp[e];
}

__global__ void k_sub_identity(int p, double* __restrict__ M) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < p) M[e * p + e] -= 1.0;
}

__global__ void k_set_identity(int p, double* __restrict__ M) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < p * p) M[e] = (e / p == e % p) ? 1.0 : 0.0;
}

// dst (rows x cols, ldd) += src (ldsrc), FP64
__global__ void k_mat_add(int rows, int cols, const double* __restrict__ src, int64_t lds,
                          double* __restrict__ dst, int64_t ldd) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int r = e / cols, c = e % cols;
  dst[(int64_t)r * ldd + c] += src[(int64_t)r * lds + c];
}

// ------------------------------------------------------------------ Jacobi
// One-sided (Hestenes) Jacobi on the columns of B (w x w), one CTA of 1024
// threads: rounds of a round-robin tournament; each warp handles up to PPW
// column pairs of a round at once (interleaved for instruction-level
// parallelism).  Columns are stored contiguously (Bc[c*w + r] = B[r][c]) and
// the rotations are accumulated in J (Jc[c*w + r] = W[r][c]); B lives in
// shared memory when it fits, J too when both fit.  On exit the columns y_j
// of Bc are B W with W = J orthogonal.
constexpr int PPW = 2;
__device__ __forceinline__ void rot_params(float al, float be, float ga, float& c, float& s) {
  const float zeta = __fdividef(be - al, 2.f * ga);
  const float t = copysignf(1.f, zeta) * __frcp_rn(fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
  c = rsqrtf(fmaf(t, t, 1.f));
  s = c * t;
}
__device__ __forceinline__ void rot_params(double al, double be, double ga, double& c, double& s) {
  const double zeta = (be - al) / (2.0 * ga);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
}
template <typename TJ>
__global__ void __launch_bounds__(1024)
k_jacobi(int w, const double* __restrict__ B, TJ* __restrict__ Bc_g, TJ* __restrict__ Jc_g, double tol_in,
         int max_sweeps, uint32_t* dev_err) {
  const TJ tol = TJ(tol_in);   // no FP64 in the inner loop of the FP32 variant
  const long long t_start = clock64();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t mat = (size_t)w * w * sizeof(TJ);
  const bool b_smem = mat <= 200 * 1024;
  const bool j_smem = 2 * mat <= 200 * 1024;
  TJ* Bw = b_smem ? reinterpret_cast<TJ*>(smem_raw) : Bc_g;
  TJ* Jw = j_smem ? reinterpret_cast<TJ*>(smem_raw) + (size_t)w * w : Jc_g;
  for (int e = tid; e < w * w; e += blockDim.x) {
    int c = e / w, r = e % w;
    Bw[e] = TJ(B[(int64_t)r * w + c]);
    Jw[e] = TJ(r == c ? 1 : 0);
  }
  __shared__ float off_max;
  __shared__ double nmax2;
  if (tid == 0) nmax2 = 0.0;
  __syncthreads();
  // largest column norm^2: couplings below the rounding noise it induces
  // (u * |b_max| * |b|) are not resolvable and do not trigger rotations
  for (int c = warp; c < w; c += nw) {
    TJ s2 = 0;
    for (int r = lane; r < w; r += 32) s2 = fma(Bw[(int64_t)c * w + r], Bw[(int64_t)c * w + r], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0)
      atomicMax(reinterpret_cast<unsigned long long*>(&nmax2), (unsigned long long)__double_as_longlong((double)s2));
  }
  __syncthreads();
  const TJ unit = sizeof(TJ) == 8 ? TJ(1.11e-16) : TJ(5.96e-8);
  const TJ noise = TJ(4) * unit * TJ(sqrt(nmax2));
  const int N = w + (w & 1);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) off_max = 0.f;
    __syncthreads();
    float local_off = 0.f;
    for (int rnd = 0; rnd < N - 1; ++rnd) {
      for (int pb = warp; pb < N / 2; pb += nw * PPW) {
        TJ* bp[PPW];
        TJ* bq[PPW];
        int pc[PPW], qc[PPW];
        bool live[PPW];
        TJ al[PPW], be[PPW], ga[PPW];
#pragma unroll
        for (int u = 0; u < PPW; ++u) {
          const int pi = pb + u * nw;
          int a = 0, b = 0;
          live[u] = pi < N / 2;
          if (live[u]) {
            if (pi == 0) { a = N - 1; b = rnd; }
            else {
              a = rnd + pi;                      // rnd, pi < N - 1
              if (a >= N - 1) a -= N - 1;
              b = rnd - pi;
              if (b < 0) b += N - 1;
            }
            live[u] = (a < w && b < w);
          }
          const int pcol = live[u] ? min(a, b) : 0, qcol = live[u] ? max(a, b) : 1;
          pc[u] = pcol;
          qc[u] = qcol;
          bp[u] = Bw + (int64_t)pcol * w;
          bq[u] = Bw + (int64_t)qcol * w;
          al[u] = be[u] = ga[u] = TJ(0);
        }
        for (int r = lane; r < w; r += 32) {
#pragma unroll
          for (int u = 0; u < PPW; ++u) {
            if (!live[u]) continue;
            TJ x = bp[u][r], y = bq[u][r];
            al[u] = fma(x, x, al[u]); be[u] = fma(y, y, be[u]); ga[u] = fma(x, y, ga[u]);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int u = 0; u < PPW; ++u) {
            al[u] += __shfl_xor_sync(0xffffffffu, al[u], o);
            be[u] += __shfl_xor_sync(0xffffffffu, be[u], o);
            ga[u] += __shfl_xor_sync(0xffffffffu, ga[u], o);
          }
        }
        TJ cs[PPW], sn[PPW];
        bool rot[PPW];
#pragma unroll
        for (int u = 0; u < PPW; ++u) {
          const TJ nrm = sqrt(al[u] * be[u]);
          rot[u] = live[u] && nrm > TJ(0) && fabs(ga[u]) > tol * nrm &&
                   fabs(ga[u]) > noise * sqrt(fmax(al[u], be[u]));
          cs[u] = TJ(1); sn[u] = TJ(0);
          if (rot[u]) {
            // any t gives an exactly orthogonal rotation through c, s below;
            // an approximate t only slows convergence negligibly
            local_off = fmaxf(local_off, (float)fabs(ga[u]) / (float)nrm);
            rot_params(al[u], be[u], ga[u], cs[u], sn[u]);
          }
        }
        for (int r = lane; r < w; r += 32) {
#pragma unroll
          for (int u = 0; u < PPW; ++u) {
            if (!rot[u]) continue;
            TJ x = bp[u][r], y = bq[u][r];
            bp[u][r] = cs[u] * x - sn[u] * y;
            bq[u][r] = sn[u] * x + cs[u] * y;
            TJ* jp = Jw + (int64_t)pc[u] * w;
            TJ* jq = Jw + (int64_t)qc[u] * w;
            TJ g = jp[r], h = jq[r];
            jp[r] = cs[u] * g - sn[u] * h;
            jq[r] = sn[u] * g + cs[u] * h;
          }
        }
      }
      __syncthreads();
    }
    if (lane == 0 && local_off > 0.f) atomicMax(reinterpret_cast<int*>(&off_max), __float_as_int(local_off));
    __syncthreads();
    if (off_max == 0.f) break;
    __syncthreads();
  }
  if (tid == 0 && sweep >= max_sweeps) atomicOr(dev_err, DEV_ERR_JACOBI);
  if (tid == 0) {
    dev_err[8] = (uint32_t)sweep;   // sweeps used (diagnostics)
    dev_err[9] = (uint32_t)((clock64() - t_start) >> 10);   // kilocycles (diagnostics)
  }
  if (j_smem)
    for (int e = tid; e < w * w; e += blockDim.x) Jc_g[e] = Jw[e];
}

// Normalise the columns of J into W (FP64, row-major w x w).
template <typename TJ>
__global__ void k_jacobi_w(int w, const TJ* __restrict__ Jc, double* __restrict__ W) {
  const int c = blockIdx.x;
  __shared__ double red[32];
  double s = 0.0;
  for (int r = threadIdx.x; r < w; r += blockDim.x) {
    double v = (double)Jc[(int64_t)c * w + r];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double inv = red[0] > 0 ? 1.0 / sqrt(red[0]) : 0.0;
  for (int r = threadIdx.x; r < w; r += blockDim.x) W[(int64_t)r * w + c] = (double)Jc[(int64_t)c * w + r] * inv;
}

// B64 = B W (W with unit columns).  Singular values = column norms of B64
// (second-order accurate in the error of W), sorted descending; Ub = B64 /
// sigma; W permuted alike.  One CTA.
__global__ void k_svd_finish(int w, const double* __restrict__ B64, const double* __restrict__ Win,
                             double* __restrict__ S, double* __restrict__ Ub, double* __restrict__ W) {
  extern __shared__ double sig[];
  double* isig = sig + w;                      // 1 / sigma (one FP64 division per column)
  int* pos = reinterpret_cast<int*>(isig + w);
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < w; ++r) { double v = B64[(int64_t)r * w + c]; s += v * v; }
    sig[c] = sqrt(s);
    isig[c] = sig[c] > 0 ? 1.0 / sig[c] : 0.0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    int rank = 0;
    for (int o = 0; o < w; ++o)
      rank += (sig[o] > sig[c]) || (sig[o] == sig[c] && o < c);
    pos[c] = rank;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    int r = e / w, c = e % w;
    int d = pos[c];
    double sc = sig[c];
    Ub[(int64_t)r * w + d] = sc > 0 ? B64[e] * isig[c] : (r == c ? 1.0 : 0.0);
    W[(int64_t)r * w + d] = Win[e];
  }
  for (int c = threadIdx.x; c < w; c += blockDim.x) S[pos[c]] = sig[c];
}



// Y = beta Y + alpha X M, FP64 storage, FP32 arithmetic.  32 x 32 output
// tiles, 256 threads (4 outputs each); X and M are converted to FP32 once per
// tile in shared memory (FP64 -> FP32 conversions are not free here).
__global__ void __launch_bounds__(256) k_small_gemm_f32(int m, int p, int q, const double* __restrict__ X,
                                                        int64_t ldx, const double* __restrict__ M, int64_t ldm,
                                                        double alpha, double beta, double* __restrict__ Y,
                                                        int64_t ldy) {
  __shared__ float xs[32][33];
  __shared__ float ms[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // ty 0..7
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < p; k0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int r = e >> 5, c = e & 31;
      xs[r][c] = (i0 + r < m && k0 + c < p) ? (float)X[(int64_t)(i0 + r) * ldx + k0 + c] : 0.f;
      ms[r][c] = (k0 + r < p && j0 + c < q) ? (float)M[(int64_t)(k0 + r) * ldm + j0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float b = ms[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(xs[ty + 8 * u][kk], b, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u, j = j0 + tx;
    if (i < m && j < q) {
      double y = alpha * (double)acc[u];
      if (beta != 0.0) y += beta * Y[(int64_t)i * ldy + j];
      Y[(int64_t)i * ldy + j] = y;
    }
  }
}

// ----------------------------------------------------------------- small ops
template <typename TA, typename TC>
__global__ void k_panel_mean(const TA* __restrict__ A, int64_t lda, int64_t rows, int64_t n,
                             const float* __restrict__ scale, TC* __restrict__ s) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int64_t r = 0; r < rows; ++r) {
    double v;
    if constexpr (std::is_same<TA, double>::value) v = A[r * lda + j];
    else v = (double)to_f32(A[r * lda + j]);
    if (scale) v *= (double)scale[j];
    acc += v;
  }
  s[j] = TC(acc / (double)rows);
}

template <typename TC>
__global__ void k_vec_mat(int64_t n, int p, const double* __restrict__ x, const TC* __restrict__ M,
                          int64_t ldm, double* __restrict__ out) {
  // one block per output column, reduction over n
  const int c = blockIdx.x;
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s += x[j] * (double)M[j * ldm + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[c] = v;
  }
}

template <typename TC>
__global__ void k_cast_from64(int64_t count, const double* __restrict__ src, TC* __restrict__ dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < count) dst[e] = TC(src[e]);
}
template <typename TC>
__global__ void k_cast_to64(int64_t count, const TC* __restrict__ src, double* __restrict__ dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < count) dst[e] = (double)src[e];
}

template <typename TC>
__global__ void k_rank1_sub(int64_t n, int p, double alpha, const double* __restrict__ x,
                            const double* __restrict__ y, TC* __restrict__ M, int64_t ldm) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  int64_t j = e / p;
  int c = (int)(e % p);
  M[j * ldm + c] = TC((double)M[j * ldm + c] - alpha * x[j] * y[c]);
}

template <typename TC>
__global__ void k_column_to_vec(int64_t n, const TC* __restrict__ F, int64_t ldf, int col,
                                double scale, double* __restrict__ d) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) d[j] = (double)F[j * ldf + col] * scale;
}

template <typename TC>
__global__ void k_col_sums(int64_t m, int p, const TC* __restrict__ Q, int64_t ldq,
                           double* __restrict__ out) {
  // grid-stride over rows, per-thread column; atomics into FP64 out (zeroed)
  const int c = threadIdx.x % 64 + blockIdx.y * 64;
  const int rl = threadIdx.x / 64;
  if (c >= p) return;
  double s = 0.0;
  for (int64_t r = blockIdx.x * 4 + rl; r < m; r += (int64_t)gridDim.x * 4) s += (double)Q[r * ldq + c];
  atomicAdd(&out[c], s);
}

template <typename TC>
__global__ void k_sub_rowvec(int64_t m, int p, const double* __restrict__ v, TC* __restrict__ H,
                             int64_t ldh) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * p) return;
  int64_t r = e / p;
  int c = (int)(e % p);
  H[r * ldh + c] -= TC(v[c]);
}

template <typename T>
__global__ void k_transpose(int64_t rows, int64_t cols, const T* __restrict__ in, int64_t ld_in,
                            T* __restrict__ out, int64_t ld_out) {
  // out[r][c] = in[c][r]; out is rows x cols
  __shared__ T tile[32][33];
  int64_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t ic = c0 + k, ir = r0 + threadIdx.x;   // in row = ic (out col), in col = ir
    if (ic < cols && ir < rows) tile[k][threadIdx.x] = in[ic * ld_in + ir];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int64_t orow = r0 + k, ocol = c0 + threadIdx.x;
    if (orow < rows && ocol < cols) out[orow * ld_out + ocol] = tile[threadIdx.x][k];
  }
}

template <typename TI, typename TO>
__global__ void k_copy_matrix(int64_t rows, int64_t cols, const TI* __restrict__ in, int64_t ld_in,
                              TO* __restrict__ out, int64_t ld_out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t r = e / cols, c = e % cols;
  out[r * ld_out + c] = TO(in[r * ld_in + c]);
}

inline unsigned grid1(int64_t count, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, cdiv(count, threads));
}

// C = X^T X (p x p, FP64, both triangles; C zeroed by the caller) for an
// FP64 X, in FP32 arithmetic: each entry is split into x = h + t (h =
// RN32(x), t = RN32(x - h)), every product h_a h_b is split exactly into
// pr + e (pr = RN(h_a h_b), e = fma(h_a, h_b, -pr)), and the pr are summed
// with Knuth's two-sum; the two-sum's rounding errors, the e and the cross
// terms h_a t_b + t_a h_b go into a compensation term (t_a t_b, below
// u32^2 |x_a x_b|, is dropped).  Each CTA sums rows_per_block rows of one
// upper tile pair (64 x 64) with 4 x 4 entries per thread, then adds s + c
// to C in FP64 (and to the mirrored entry for an off-diagonal pair).  The
// result is within a few u32^2 of sum |x_a x_b| of the exact Gram: FP64-class
// for the eigenvalues of Step 4, at FP32 arithmetic rates (the FP64 pipe
// retires about one sixtieth of the FP32 rate).  Explicit _rn intrinsics
// keep the compiler from contracting the two-sum into FMAs.
__global__ void __launch_bounds__(256)
k_gram_comp(int64_t m, int p, const double* __restrict__ X, int64_t ldx, double* __restrict__ C, int64_t ldc,
            int64_t rows_per_block, int nt) {
  constexpr int RC = 32;
  __shared__ float Xs[RC][64 + 1], Xt[RC][64 + 1];
  __shared__ float Ys[RC][64 + 1], Yt[RC][64 + 1];
  // upper tile pair (ti <= tj) of blockIdx.y
  int ti = 0, tj = 0;
  {
    int y = (int)blockIdx.y;
    while (y >= nt - ti) { y -= nt - ti; ++ti; }
    tj = ti + y;
  }
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int p0 = ti * 64, q0 = tj * 64;
  const int64_t rbeg = (int64_t)blockIdx.x * rows_per_block;
  const int64_t rend = min(m, rbeg + rows_per_block);
  float sum[4][4], cmp[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { sum[a][b] = 0.f; cmp[a][b] = 0.f; }
  for (int64_t r0 = rbeg; r0 < rend; r0 += RC) {
    for (int e = tid; e < RC * 64; e += 256) {
      const int rr = e / 64, cc = e % 64;
      const int64_t r = r0 + rr;
      const bool rok = r < rend;
      const double xa = (rok && p0 + cc < p) ? X[r * ldx + p0 + cc] : 0.0;
      const double xb = (rok && q0 + cc < p) ? X[r * ldx + q0 + cc] : 0.0;
      const float ha = (float)xa, hb = (float)xb;
      Xs[rr][cc] = ha;
      Xt[rr][cc] = (float)(xa - (double)ha);
      Ys[rr][cc] = hb;
      Yt[rr][cc] = (float)(xb - (double)hb);
    }
    __syncthreads();
#pragma unroll 2
    for (int rr = 0; rr < RC; ++rr) {
      float xv[4], yv[4], xl[4], yl[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        xv[a] = Xs[rr][ty * 4 + a];
        xl[a] = Xt[rr][ty * 4 + a];
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        yv[b] = Ys[rr][tx * 4 + b];
        yl[b] = Yt[rr][tx * 4 + b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float pr = __fmul_rn(xv[a], yv[b]);
          const float e = fmaf(xv[a], yv[b], -pr);
          const float s0 = sum[a][b];
          const float s1 = __fadd_rn(s0, pr);
          const float bp = __fsub_rn(s1, s0);
          const float err = __fadd_rn(__fsub_rn(s0, __fsub_rn(s1, bp)), __fsub_rn(pr, bp));
          const float cross = fmaf(xv[a], yl[b], __fmul_rn(xl[a], yv[b]));
          sum[a][b] = s1;
          cmp[a][b] = __fadd_rn(cmp[a][b], __fadd_rn(__fadd_rn(err, e), cross));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = p0 + ty * 4 + a, j = q0 + tx * 4 + b;
      if (i < p && j < p) {
        const double v = (double)sum[a][b] + (double)cmp[a][b];
        atomicAdd(&C[(int64_t)i * ldc + j], v);
        if (ti != tj) atomicAdd(&C[(int64_t)j * ldc + i], v);
      }
    }
}

}  // namespace

// ===================================================================== host
void gram(bool f64, int64_t m, int p, int q, const void* X, int64_t ldx, const void* Y,
          int64_t ldy, double* C, int64_t ldc, bool accumulate, cudaStream_t st,
          const uint32_t* active) {
  if (!accumulate)
    RPCA_CUDA_TRY(cudaMemset2DAsync(C, ldc * sizeof(double), 0, q * sizeof(double), p, st));
  if (m <= 0) return;
  const int tp = (int)cdiv(p, 64), tq = (int)cdiv(q, 64);
  const int sms = num_sms();
  int64_t want = std::max<int64_t>(1, (int64_t)sms * 4 / (tp * tq));
  int64_t rpb = std::max<int64_t>(256, round_up(cdiv(m, want), 32));
  unsigned gx = (unsigned)cdiv(m, rpb);
  dim3 grid(gx, tp, tq);
  if (f64)
    k_gram<double><<<grid, 256, 0, st>>>(m, p, q, (const double*)X, ldx, (const double*)Y, ldy, C, ldc, rpb, active);
  else
    k_gram<float><<<grid, 256, 0, st>>>(m, p, q, (const float*)X, ldx, (const float*)Y, ldy, C, ldc, rpb, active);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void gram_sym_comp(int64_t m, int p, const double* X, int64_t ldx, double* C, int64_t ldc, cudaStream_t st) {
  RPCA_CUDA_TRY(cudaMemset2DAsync(C, ldc * sizeof(double), 0, p * sizeof(double), p, st));
  if (m <= 0 || p <= 0) return;
  const int nt = (int)cdiv(p, 64);
  const int npair = nt * (nt + 1) / 2;
  const int64_t want = std::max<int64_t>(1, (int64_t)num_sms() / npair);
  const int64_t rpb = std::max<int64_t>(64, round_up(cdiv(m, want), 32));
  dim3 grid((unsigned)cdiv(m, rpb), (unsigned)npair);
  k_gram_comp<<<grid, 256, 0, st>>>(m, p, X, ldx, C, ldc, rpb, nt);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

template <typename TC, int BM>
static void gemm_launch(int64_t m, int p, int q, const void* X, int64_t ldx, const double* M,
                        int64_t ldm, double alpha, double beta, void* Y, int64_t ldy,
                        cudaStream_t st, const uint32_t* active) {
  size_t smem = sizeof(TC) * ((size_t)BM * p + (size_t)p * 64);
  auto kern = k_gemm_xm<TC, BM>;
  RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t nblk = cdiv(m, BM);
  unsigned g = (unsigned)std::min<int64_t>(nblk, (int64_t)num_sms() * 4);
  kern<<<std::max(1u, g), 256, smem, st>>>(m, p, q, (const TC*)X, ldx, M, ldm, alpha, beta, (TC*)Y, ldy, active);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void gemm_xm(bool f64, int64_t m, int p, int q, const void* X, int64_t ldx, const double* M,
             int64_t ldm, double alpha, double beta, void* Y, int64_t ldy, cudaStream_t st,
             const uint32_t* active) {
  if (m <= 0 || q <= 0) return;
  if (p > 256) throw Invalid("gemm_xm: p > 256");
  if (f64) {
    if (m <= 1024) gemm_launch<double, 16>(m, p, q, X, ldx, M, ldm, alpha, beta, Y, ldy, st, active);
    else gemm_launch<double, 32>(m, p, q, X, ldx, M, ldm, alpha, beta, Y, ldy, st, active);
  } else {
    if (m <= 4096) gemm_launch<float, 16>(m, p, q, X, ldx, M, ldm, alpha, beta, Y, ldy, st, active);
    else gemm_launch<float, 64>(m, p, q, X, ldx, M, ldm, alpha, beta, Y, ldy, st, active);
  }
}

void chol_small(int p, const double* G, int64_t ldg, double* R, double* Rinv, int pass,
                double piv_rel, double shift_rel, uint32_t* qf, uint32_t* dev_err, cudaStream_t st, bool inv_f32,
                const uint32_t* gate) {
  if (p <= 64) {
    const int ps = p | 1;
    const size_t sm = (size_t)2 * p * ps * sizeof(double);
    static bool attr = false;
    if (!attr) {
      RPCA_CUDA_TRY(cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 65 * 8));
      attr = true;
    }
    k_chol<<<1, 256, sm, st>>>(p, G, ldg, R, Rinv, pass, piv_rel, shift_rel, qf, dev_err, inv_f32 ? 1 : 0, gate);
  } else {
    k_chol_global<<<1, 256, 0, st>>>(p, G, ldg, R, Rinv, pass, piv_rel, shift_rel, qf, dev_err, gate);
  }
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}


void left_mul(int p, const double* Rk, double* Racc, cudaStream_t st) {
  k_left_mul<<<1, 256, (size_t)p * p * sizeof(double), st>>>(p, Rk, Racc);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void sub_identity(int p, double* M, cudaStream_t st) {
  k_sub_identity<<<grid1(p), 256, 0, st>>>(p, M);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void set_identity(int p, double* M, cudaStream_t st) {
  k_set_identity<<<grid1((int64_t)p * p), 256, 0, st>>>(p, M);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void mat_add(int rows, int cols, const double* src, int64_t lds, double* dst, int64_t ldd,
             cudaStream_t st) {
  k_mat_add<<<grid1((int64_t)rows * cols), 256, 0, st>>>(rows, cols, src, lds, dst, ldd);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

// FP64 refinement steps after the FP32 Jacobi: each squares the error
// relative to the gaps; two take an FP32-converged start to FP64 rounding.
constexpr int kRefineSteps = 2;

void jacobi_svd(bool f64, int w, int kk, const double* B, double* S, double* Ub, double* W, double* work,
                uint32_t* dev_err, cudaStream_t st) {
  (void)kk;   // all w triplets are formed
  // work layout (doubles): Bc [w*w], Jc [w*w], W0 [w*w], B64 [w*w], E [w*w]
  double* Bc = work;
  double* Jc = work + (size_t)w * w;
  double* W0 = work + 2 * (size_t)w * w;
  double* B64 = work + 3 * (size_t)w * w;
  double* Ew = work + 4 * (size_t)w * w;
  if (f64) {
    const size_t mat = (size_t)w * w * sizeof(double);
    const size_t smem = 2 * mat <= 200 * 1024 ? 2 * mat : (mat <= 200 * 1024 ? mat : 0);
    RPCA_CUDA_TRY(cudaFuncSetAttribute(k_jacobi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_jacobi<double><<<1, 1024, smem, st>>>(w, B, Bc, Jc, 4.0 * std::sqrt((double)w) * 1.11e-16, 60, dev_err);
    RPCA_CUDA_TRY(cudaGetLastError());
    k_jacobi_w<double><<<w, 128, 0, st>>>(w, Jc, W0);
  } else {
    float* Bc32 = reinterpret_cast<float*>(Bc);
    float* Jc32 = reinterpret_cast<float*>(Jc);
    const double tol = 4.0 * std::sqrt((double)w) * 5.96e-8;
    if (!jacobi_cluster_f32(w, B, Jc32, tol, 40, dev_err, st)) {
      const size_t mat = (size_t)w * w * sizeof(float);
      const size_t smem = 2 * mat <= 200 * 1024 ? 2 * mat : (mat <= 200 * 1024 ? mat : 0);
      RPCA_CUDA_TRY(cudaFuncSetAttribute(k_jacobi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      k_jacobi<float><<<1, 1024, smem, st>>>(w, B, Bc32, Jc32, tol, 40, dev_err);
      RPCA_CUDA_TRY(cudaGetLastError());
      count_launch();
    }
    k_jacobi_w<float><<<w, 128, 0, st>>>(w, Jc32, W0);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
    // FP64 refinement of the FP32 Jacobi vectors (Bc, Jc are free now)
    refine_eigvecs64(w, B, W0, Bc, Jc, B64, Ew, kRefineSteps, st);
  }
  RPCA_CUDA_TRY(cudaGetLastError());
  if (f64) count_launch(2);
  // B64 = B W0 in FP64: singular values as column norms of B times unit
  // right singular vectors (second-order accurate in their error).
  gemm64_small(w, w, w, 1.0, B, w, false, W0, w, false, 0.0, nullptr, 0, B64, w, st);
  size_t smem = (size_t)w * (2 * sizeof(double) + sizeof(int));
  k_svd_finish<<<1, 256, smem, st>>>(w, B64, W0, S, Ub, W);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (getenv("RPCA_DEBUG") && cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
    uint32_t sw[2] = {0, 0};
    cudaMemcpyAsync(sw, dev_err + 8, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    fprintf(stderr, "[rpca] jacobi w=%d sweeps=%u kcycles=%u\n", w, sw[0], sw[1]);
  }
}

// Step 4 from the Gram matrix G = T^T T (FP32-class paths).  FP32 Jacobi
// sweeps on a shifted FP32 Cholesky factor of G give approximate right
// singular vectors of T to a loose tolerance; the FP64 refinement against G
// itself then takes them to FP64 accuracy (each step squares the error), and
// sigma_j^2 are the diagonal of the refined X^T G X.  With the
// reorthogonalised Krylov blocks T is well conditioned (its singular values
// are those of A on the Krylov space), so forming G loses nothing the
// tolerances can see.
// The FP32 sweeps run to FP32 convergence (relative off-diagonal
// 4 sqrt(w) u): a looser sweep tolerance leaves vector errors of
// tolerance / relative gap near the edge of a cluster of singular values,
// outside the refinement's quadratic basin (measured at the precision
// workload: tolerance 1e-5 and three steps left U^T U - I at 3e-4).
constexpr int kGramRefineSteps = 2;

void svd_from_gram(int w, const double* G, double* S, double* Vs, double* W, double* work, uint32_t* dev_err,
                   cudaStream_t st) {
  const size_t ww = (size_t)w * w;
  double* B = work;
  float* Jc32 = reinterpret_cast<float*>(work + ww);
  double* X = work + 2 * ww;
  double* Xn = work + 3 * ww;
  double* P = work + 4 * ww;
  double* Sm = work + 5 * ww;
  double* E = B;                                   // B is free once the sweeps are done
  const double kGramJacobiTol = 4.0 * std::sqrt((double)w) * 5.96e-8;
  // FP32 eigenvectors of G: one-sided Jacobi on a shifted FP32 Cholesky
  // factor of G (relative accuracy for the small eigenvalues, which a
  // two-sided Jacobi on G in FP32 lacks), over a cluster of CTAs
  chol32_shift(w, G, B, st);
  if (!jacobi_cluster_f32(w, B, Jc32, kGramJacobiTol, 40, dev_err, st)) {
    const size_t mat = ww * sizeof(float);
    const size_t smem = 2 * mat <= 200 * 1024 ? 2 * mat : (mat <= 200 * 1024 ? mat : 0);
    RPCA_CUDA_TRY(cudaFuncSetAttribute(k_jacobi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_jacobi<float><<<1, 1024, smem, st>>>(w, B, reinterpret_cast<float*>(Xn), Jc32, kGramJacobiTol, 40, dev_err);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  k_jacobi_w<float><<<w, 128, 0, st>>>(w, Jc32, X);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
  refine_eigvecs64(w, G, X, Xn, P, Sm, E, kGramRefineSteps, st, true);
  gemm64_small(w, w, w, 1.0, G, w, false, X, w, false, 0.0, nullptr, 0, P, w, st);     // G X
  gemm64_small(w, w, w, 1.0, X, w, true, P, w, false, 0.0, nullptr, 0, Sm, w, st);    // X^T G X
  eig_finish(w, Sm, X, S, Vs, W, st);
}

void small_gemm_f32(int m, int p, int q, const double* X, int64_t ldx, const double* M, int64_t ldm,
                    double alpha, double beta, double* Y, int64_t ldy, cudaStream_t st) {
  if (m <= 0 || q <= 0) return;
  dim3 grid((unsigned)cdiv(q, 32), (unsigned)cdiv(m, 32));
  k_small_gemm_f32<<<grid, 256, 0, st>>>(m, p, q, X, ldx, M, ldm, alpha, beta, Y, ldy);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void panel_mean(rpca_dtype dt, const void* A, int64_t lda, int64_t rows, int64_t n,
                const float* scale, void* s, cudaStream_t st) {
  unsigned g = grid1(n);
  switch (dt) {
    case RPCA_F64: k_panel_mean<double, double><<<g, 256, 0, st>>>((const double*)A, lda, rows, n, scale, (double*)s); break;
    case RPCA_F32: k_panel_mean<float, float><<<g, 256, 0, st>>>((const float*)A, lda, rows, n, scale, (float*)s); break;
    case RPCA_BF16: k_panel_mean<__nv_bfloat16, float><<<g, 256, 0, st>>>((const __nv_bfloat16*)A, lda, rows, n, scale, (float*)s); break;
    case RPCA_FP8E4M3: k_panel_mean<__nv_fp8_e4m3, float><<<g, 256, 0, st>>>((const __nv_fp8_e4m3*)A, lda, rows, n, scale, (float*)s); break;
  }
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void vec_mat(bool f64, int64_t n, int p, const double* x, const void* M, int64_t ldm, double* out,
             cudaStream_t st) {
  if (f64) k_vec_mat<double><<<p, 256, 0, st>>>(n, p, x, (const double*)M, ldm, out);
  else k_vec_mat<float><<<p, 256, 0, st>>>(n, p, x, (const float*)M, ldm, out);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void cast_f64_to(bool f64, int64_t count, const double* src, void* dst, cudaStream_t st) {
  if (f64) RPCA_CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else {
    k_cast_from64<float><<<grid1(count), 256, 0, st>>>(count, src, (float*)dst);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
}

void cast_to_f64(bool f64, int64_t count, const void* src, double* dst, cudaStream_t st) {
  if (f64) RPCA_CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else {
    k_cast_to64<float><<<grid1(count), 256, 0, st>>>(count, (const float*)src, dst);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
}

void rank1_sub(bool f64, int64_t n, int p, double alpha, const double* x, const double* y, void* M,
               int64_t ldm, cudaStream_t st) {
  if (f64) k_rank1_sub<double><<<grid1(n * p), 256, 0, st>>>(n, p, alpha, x, y, (double*)M, ldm);
  else k_rank1_sub<float><<<grid1(n * p), 256, 0, st>>>(n, p, alpha, x, y, (float*)M, ldm);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void column_to_vec(bool f64, int64_t n, const void* F, int64_t ldf, int col, double scale, double* d,
                   cudaStream_t st) {
  if (f64) k_column_to_vec<double><<<grid1(n), 256, 0, st>>>(n, (const double*)F, ldf, col, scale, d);
  else k_column_to_vec<float><<<grid1(n), 256, 0, st>>>(n, (const float*)F, ldf, col, scale, d);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void col_sums(bool f64, int64_t m, int p, const void* Q, int64_t ldq, double* out, cudaStream_t st) {
  RPCA_CUDA_TRY(cudaMemsetAsync(out, 0, p * sizeof(double), st));
  dim3 grid((unsigned)std::min<int64_t>(cdiv(m, 4), 1024), (unsigned)cdiv(p, 64));
  if (f64) k_col_sums<double><<<grid, 256, 0, st>>>(m, p, (const double*)Q, ldq, out);
  else k_col_sums<float><<<grid, 256, 0, st>>>(m, p, (const float*)Q, ldq, out);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void sub_rowvec(bool f64, int64_t m, int p, const double* v, void* H, int64_t ldh, cudaStream_t st) {
  if (f64) k_sub_rowvec<double><<<grid1(m * p), 256, 0, st>>>(m, p, v, (double*)H, ldh);
  else k_sub_rowvec<float><<<grid1(m * p), 256, 0, st>>>(m, p, v, (float*)H, ldh);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void transpose(rpca_dtype dt, int64_t rows, int64_t cols, const void* in, int64_t ld_in, void* out,
               int64_t ld_out, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(cols, 32), (unsigned)cdiv(rows, 32));
  dim3 blk(32, 8);
  switch (dtype_bytes(dt)) {
    case 8: k_transpose<uint64_t><<<grid, blk, 0, st>>>(rows, cols, (const uint64_t*)in, ld_in, (uint64_t*)out, ld_out); break;
    case 4: k_transpose<uint32_t><<<grid, blk, 0, st>>>(rows, cols, (const uint32_t*)in, ld_in, (uint32_t*)out, ld_out); break;
    case 2: k_transpose<uint16_t><<<grid, blk, 0, st>>>(rows, cols, (const uint16_t*)in, ld_in, (uint16_t*)out, ld_out); break;
    default: k_transpose<uint8_t><<<grid, blk, 0, st>>>(rows, cols, (const uint8_t*)in, ld_in, (uint8_t*)out, ld_out); break;
  }
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void copy_matrix(bool in_f64, bool out_f64, int64_t rows, int64_t cols, const void* in, int64_t ld_in,
                 void* out, int64_t ld_out, cudaStream_t st) {
  unsigned g = grid1(rows * cols);
  if (in_f64 && out_f64) k_copy_matrix<double, double><<<g, 256, 0, st>>>(rows, cols, (const double*)in, ld_in, (double*)out, ld_out);
  else if (in_f64) k_copy_matrix<double, float><<<g, 256, 0, st>>>(rows, cols, (const double*)in, ld_in, (float*)out, ld_out);
  else if (out_f64) k_copy_matrix<float, double><<<g, 256, 0, st>>>(rows, cols, (const float*)in, ld_in, (double*)out, ld_out);
  else k_copy_matrix<float, float><<<g, 256, 0, st>>>(rows, cols, (const float*)in, ld_in, (float*)out, ld_out);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

}  // namespace rpca
