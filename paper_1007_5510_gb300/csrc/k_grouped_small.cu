// Grouped batch path: the CUDA-core steps between the streamed passes.
//
// One CTA per problem for the n-side steps (orthonormalising F, Step 4) and
// the small factorisations; (problem, row range) items for the m-side
// products over H.  Householder QR in shared memory (Golub and Van Loan,
// Algorithms 5.1.1 and 5.2.1, with the explicit Q formed backwards as in
// their Section 5.1.6) keeps every n-side basis orthonormal to FP32 rounding
// whatever its condition; Step 4 is a one-sided Jacobi SVD (Hestenes) of the
// triangular factor of T.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "grouped.h"

namespace rpca {
namespace grp {

constexpr int SM_THREADS = 256;
constexpr int SM_WARPS = SM_THREADS / 32;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Squared norm of rows [r0, n) of column c (one warp), FP64 total.
__device__ __forceinline__ double col_nrm2(const float* col, int r0, int n, int lane) {
  double s = 0.0;
  for (int r = r0 + lane; r < n; r += 32) {
    const float x = col[r];
    s += (double)x * x;
  }
  return warp_sum_d(s);
}

// Householder QR of the column-major n x nc matrix A (column c at A + c*ld,
// shared memory), nc <= 64, by all threads of the CTA.  On return column c
// holds the Householder vector below the diagonal (its leading entry in
// v0[c]), R's strict upper part above it, R[c][c] in rdiag[c], and the
// reflector H_c = I - tau[c] v v^T.  Each warp owns the trailing columns
// c2 = c + 1 + warp (mod SM_WARPS) of a step: dot product, update, and the
// next column's norm, so one barrier per column suffices.
__device__ void hh_qr(float* A, int n, int ld, int nc, float* tau, float* v0, float* rdiag, double* nrm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    const double s = col_nrm2(A, 0, n, lane);
    if (lane == 0) nrm[0] = s;
  }
  __syncthreads();
  for (int c = 0; c < nc; ++c) {
    const float* vc = A + (size_t)c * ld;
    const double nrm2 = nrm[c];
    const double x0 = (c < n) ? (double)vc[c] : 0.0;
    double alpha = 0.0, vv0 = 0.0, t = 0.0;
    if (nrm2 > 0.0) {
      alpha = (x0 >= 0.0) ? -sqrt(nrm2) : sqrt(nrm2);
      vv0 = x0 - alpha;
      const double vn2 = nrm2 - x0 * x0 + vv0 * vv0;
      t = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
    }
    const float fv0 = (float)vv0, ft = (float)t;
    for (int c2 = c + 1 + warp; c2 < nc; c2 += SM_WARPS) {
      float* a2 = A + (size_t)c2 * ld;
      float d = 0.f;
      for (int r = c + lane; r < n; r += 32) d += ((r == c) ? fv0 : vc[r]) * a2[r];
      d = warp_sum(d) * ft;
      for (int r = c + lane; r < n; r += 32) a2[r] -= d * ((r == c) ? fv0 : vc[r]);
      if (c2 == c + 1) {
        __syncwarp();
        const double s = col_nrm2(a2, c + 1, n, lane);
        if (lane == 0) nrm[c + 1] = s;
      }
    }
    if (threadIdx.x == 0) {
      tau[c] = ft;
      v0[c] = fv0;
      rdiag[c] = (float)alpha;
    }
    __syncthreads();
  }
}

// Overwrites the output of hh_qr with the explicit n x nc Q = H_0 ... H_{nc-1} I.
__device__ void hh_form_q(float* A, int n, int ld, int nc, const float* tau, const float* v0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = nc - 1; c >= 0; --c) {
    const float* vc = A + (size_t)c * ld;
    const float t = tau[c], fv0 = v0[c];
    for (int c2 = c + 1 + warp; c2 < nc; c2 += SM_WARPS) {
      float* a2 = A + (size_t)c2 * ld;
      float d = 0.f;
      for (int r = c + lane; r < n; r += 32) d += ((r == c) ? fv0 : vc[r]) * a2[r];
      d = warp_sum(d) * t;
      for (int r = c + lane; r < n; r += 32) a2[r] -= d * ((r == c) ? fv0 : vc[r]);
    }
    __syncthreads();
    float* ac = A + (size_t)c * ld;
    for (int r = threadIdx.x; r < n; r += SM_THREADS) {
      float q;
      if (r < c) q = 0.f;
      else if (r == c) q = 1.f - t * fv0 * fv0;
      else q = -t * ac[r] * fv0;
      ac[r] = q;
    }
    __syncthreads();
  }
}

// Offset (BF16 elements) of X[r][c] in the X^T images of the H pass: image
// r / 64 holds rows c < 32 of 128 bytes, 16-byte chunk (r % 64) / 8
// swizzled with c % 8.
__device__ __forceinline__ int64_t xt_offset(int r, int c) {
  const int kb = r >> 6, e = r & 63;
  return (int64_t)kb * 2048 + c * 64 + (((e >> 3) ^ (c & 7)) << 3) + (e & 7);
}

// ------------------------------------------------------------------ orth
// One CTA per problem.  F (n x l, ld ldf) -> column-major shared copy; for
// j >= 0 the projection F -= X_b (X_b^T F) over the earlier blocks b <= j,
// twice (block classical Gram-Schmidt with reorthogonalisation); then
// Householder QR and the explicit Q, which is X^(j+1) (X^(0) for j = -1).
// F is zeroed for the next pass's accumulation.
__global__ void __launch_bounds__(SM_THREADS)
k_grp_orth(const GrpProblem* __restrict__ probs, int j, int l, int w, int ldf, int max_n, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GrpProblem& P = probs[blockIdx.x];
  const int n = (int)P.n;
  const int ld = n | 1;   // odd: the columns of a row fall in different banks
  double* nrm = reinterpret_cast<double*>(smem_raw);       // 64
  float* tau = reinterpret_cast<float*>(nrm + 64);
  float* v0 = tau + 64;
  float* rdiag = v0 + 64;
  float* Cs = rdiag + 64;                                   // 32 x 32
  float* Xs = Cs + 32 * 32;                                 // 128 x 33 staging of X_b rows
  float* Fc = Xs + 128 * 33;                                // l x ld (column-major F)
  const int tid = threadIdx.x;

  for (int e = tid; e < n * l; e += SM_THREADS) {
    const int r = e / l, c = e % l;
    float* f = P.F + (int64_t)r * ldf + c;
    Fc[(size_t)c * ld + r] = *f;
    *f = 0.f;
  }
  __syncthreads();
  for (int round = 0; j >= 0 && round < 2; ++round) {
    for (int b = 0; b <= j; ++b) {
      // C = X_b^T F, accumulated over 128-row chunks (thread: entries e, e + 256, ...)
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int r0 = 0; r0 < n; r0 += 128) {
        const int nr = min(128, n - r0);
        for (int e = tid; e < nr * l; e += SM_THREADS) {
          const int r = e / l, c = e % l;
          Xs[r * 33 + c] = P.X[(int64_t)(r0 + r) * w + b * l + c];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + q * SM_THREADS;
          if (e < l * l) {
            const int ci = e / l, cj = e % l;
            const float* fcol = Fc + (size_t)cj * ld + r0;
            float s = 0.f;
            for (int r = 0; r < nr; ++r) s += Xs[r * 33 + ci] * fcol[r];
            acc[q] += s;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + q * SM_THREADS;
        if (e < l * l) Cs[(e / l) * 32 + e % l] = acc[q];
      }
      __syncthreads();
      // F -= X_b C
      for (int r0 = 0; r0 < n; r0 += 128) {
        const int nr = min(128, n - r0);
        for (int e = tid; e < nr * l; e += SM_THREADS) {
          const int r = e / l, c = e % l;
          Xs[r * 33 + c] = P.X[(int64_t)(r0 + r) * w + b * l + c];
        }
        __syncthreads();
        for (int e = tid; e < nr * l; e += SM_THREADS) {
          const int r = e % nr, cj = e / nr;
          float s = 0.f;
          for (int ci = 0; ci < l; ++ci) s += Xs[r * 33 + ci] * Cs[ci * 32 + cj];
          Fc[(size_t)cj * ld + r0 + r] -= s;
        }
        __syncthreads();
      }
    }
  }
  hh_qr(Fc, n, ld, l, tau, v0, rdiag, nrm);
  hh_form_q(Fc, n, ld, l, tau, v0);
  // X block (j+1), and its images for the next H pass
  const int blk = j + 1;
  for (int e = tid; e < n * l; e += SM_THREADS) {
    const int r = e / l, c = e % l;
    P.X[(int64_t)r * w + blk * l + c] = Fc[(size_t)c * ld + r];
  }
  __nv_bfloat16* xt = (j < 0) ? P.XT0 : P.XT;
  for (int e = tid; e < P.n64 * 32; e += SM_THREADS) {
    const int r = e >> 5, c = e & 31;
    const float x = (r < n && c < l) ? Fc[(size_t)c * ld + r] : 0.f;
    xt[xt_offset(r, c)] = __float2bfloat16_rn(x);
  }
  (void)err;
}

size_t orth_smem(int l, int max_n) {
  return (size_t)l * (max_n | 1) * 4 + 128 * 33 * 4 + 32 * 32 * 4 + 3 * 64 * 4 + 64 * 8 + 16;
}

void launch_orth(const GrpProblem* probs, int count, int j, int l, int w, int ldf, int max_n, uint32_t* err,
                 cudaStream_t st) {
  const size_t smem = orth_smem(l, max_n);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_orth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grp_orth<<<count, SM_THREADS, smem, st>>>(probs, j, l, w, ldf, max_n, err);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

// ------------------------------------------------------------ row kernels
// (problem, row range) items over the m side, 64 rows at a time through
// shared memory.
//   ROW_GRAM  G1 += H^T H
//   ROW_APPLY Q1 = H R1^-1 (64 x w tile), written over H (FP32) and as
//             Z = bf16(Q1); G2 += Q1^T Q1
//   ROW_U     U = Q1 MU
// The Gram products use 4 x 4 register tiles over the upper block triangle
// (FP32 within an item, FP64 reductions across items).
enum RowMode : int { ROW_GRAM = 0, ROW_APPLY = 1, ROW_U = 2 };

struct GramTile {
  int bi, bj, grp, rg, ntile;
  bool active;
};
__device__ __forceinline__ GramTile gram_tile(int w) {
  GramTile g;
  const int nb = (w + 3) / 4;
  g.ntile = nb * (nb + 1) / 2;
  g.rg = max(1, SM_THREADS / g.ntile);
  const int tid = threadIdx.x;
  g.active = tid < g.ntile * g.rg;
  const int tile = tid % g.ntile;
  g.grp = tid / g.ntile;
  int bi = 0, rem = tile;
  while (rem >= nb - bi) {
    rem -= nb - bi;
    ++bi;
  }
  g.bi = bi;
  g.bj = bi + rem;
  return g;
}

__device__ __forceinline__ void gram_rows(const GramTile& g, const float* Ts, int wp, int nr, float (&acc)[16]) {
  if (!g.active) return;
  for (int r = g.grp; r < nr; r += g.rg) {
    const float4 a = *reinterpret_cast<const float4*>(Ts + r * wp + 4 * g.bi);
    const float4 b = *reinterpret_cast<const float4*>(Ts + r * wp + 4 * g.bj);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[4 * x + y] += av[x] * bv[y];
  }
}

// Sums the threads' tiles over their row groups and adds the upper triangle
// to G (w x w FP64).  red: SM_THREADS * 16 floats of shared memory.
__device__ void gram_flush(const GramTile& g, const float (&acc)[16], float* red, double* G, int w) {
  __syncthreads();
  if (g.active)
#pragma unroll
    for (int q = 0; q < 16; ++q) red[(g.grp * g.ntile + (threadIdx.x % g.ntile)) * 16 + q] = acc[q];
  __syncthreads();
  const int nb = (w + 3) / 4;
  for (int e = threadIdx.x; e < g.ntile * 16; e += SM_THREADS) {
    const int t = e >> 4, q = e & 15;
    double s = 0.0;
    for (int gg = 0; gg < g.rg; ++gg) s += (double)red[(gg * g.ntile + t) * 16 + q];
    int bi = 0, rem = t;
    while (rem >= nb - bi) {
      rem -= nb - bi;
      ++bi;
    }
    const int i = 4 * bi + (q >> 2), jj = 4 * (bi + rem) + (q & 3);
    if (i < w && jj < w && i <= jj) atomicAdd(&G[i * w + jj], s);
  }
}

template <int MODE>
__global__ void __launch_bounds__(SM_THREADS)
k_grp_rows(const GrpProblem* __restrict__ probs, const GrpRItem* __restrict__ items, int w, int k) {
  extern __shared__ __align__(16) float rs[];
  const GrpRItem I = items[blockIdx.x];
  const GrpProblem& P = probs[I.p];
  const int wp = (w + 3) & ~3;
  const int tid = threadIdx.x;
  float* Ms = rs;                       // w x w (R1^-1) or w x k (MU)
  float* Hs = Ms + 64 * 64;             // 64 x wp
  float* Qs = Hs + 64 * wp;             // 64 x wp (ROW_APPLY)
  float* red = Qs + 64 * wp;            // SM_THREADS x 16
  if (MODE == ROW_APPLY)
    for (int e = tid; e < w * w; e += SM_THREADS) Ms[e] = P.R1inv[e];
  if (MODE == ROW_U)
    for (int e = tid; e < w * k; e += SM_THREADS) Ms[e] = P.MU[e];
  const GramTile g = gram_tile(w);
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  for (int r0 = 0; r0 < I.nrows; r0 += 64) {
    const int nr = min(64, I.nrows - r0);
    const int64_t grow0 = (int64_t)I.r0 + r0;
    __syncthreads();
    for (int e = tid; e < 64 * wp; e += SM_THREADS) {
      const int r = e / wp, c = e % wp;
      Hs[e] = (r < nr && c < w) ? P.H[(grow0 + r) * w + c] : 0.f;
    }
    __syncthreads();
    if (MODE == ROW_GRAM) {
      gram_rows(g, Hs, wp, nr, acc);
    } else if (MODE == ROW_APPLY) {
      // four threads per row, columns c = quarter, quarter + 4, ...
      const int r = tid >> 2, quarter = tid & 3;
      for (int c = quarter; c < wp; c += 4) {
        float s = 0.f;
        if (c < w)
          for (int t = 0; t <= c; ++t) s += Hs[r * wp + t] * Ms[t * w + c];
        Qs[r * wp + c] = s;
      }
      __syncthreads();
      gram_rows(g, Qs, wp, nr, acc);
      for (int e = tid; e < nr * w; e += SM_THREADS) {
        const int rr = e / w, c = e % w;
        P.H[(grow0 + rr) * w + c] = Qs[rr * wp + c];
      }
      // Z rows: 64 BF16 (columns past w zero), 8 chunks of 16 bytes per row
      for (int e = tid; e < nr * 8; e += SM_THREADS) {
        const int rr = e >> 3, ch = e & 7;
        uint32_t wd[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int c = 8 * ch + 2 * h;
          const float x0 = c < w ? Qs[rr * wp + c] : 0.f;
          const float x1 = c + 1 < w ? Qs[rr * wp + c + 1] : 0.f;
          __nv_bfloat162 b2 = __floats2bfloat162_rn(x0, x1);
          wd[h] = *reinterpret_cast<uint32_t*>(&b2);
        }
        reinterpret_cast<uint4*>(P.Z + (grow0 + rr) * 64)[ch] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      }
    } else {
      if (P.U) {
        for (int e = tid; e < nr * k; e += SM_THREADS) {
          const int r = e / k, c = e % k;
          float s = 0.f;
          for (int t = 0; t < w; ++t) s += Hs[r * wp + t] * Ms[t * k + c];
          P.U[(grow0 + r) * P.ldu + c] = s;
        }
      }
    }
  }
  if (MODE == ROW_GRAM) gram_flush(g, acc, red, P.G1, w);
  if (MODE == ROW_APPLY) gram_flush(g, acc, red, P.G2, w);
}

static size_t rows_smem(int w) {
  const int wp = (w + 3) & ~3;
  return ((size_t)64 * 64 + 2 * 64 * wp + SM_THREADS * 16) * 4;
}

template <int MODE>
static void launch_rows(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, int k,
                        cudaStream_t st) {
  if (nitems <= 0) return;
  const size_t smem = rows_smem(w);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_rows<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grp_rows<MODE><<<(unsigned)nitems, SM_THREADS, smem, st>>>(probs, items, w, k);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void launch_gram(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, cudaStream_t st) {
  launch_rows<ROW_GRAM>(probs, items, nitems, w, 0, st);
}
void launch_apply(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, cudaStream_t st) {
  launch_rows<ROW_APPLY>(probs, items, nitems, w, 0, st);
}
void launch_u(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, int k, cudaStream_t st) {
  launch_rows<ROW_U>(probs, items, nitems, w, k, st);
}

// ------------------------------------------------------------------ chol
// One CTA per problem: the w x w Gram (upper triangle, FP64) -> its
// Cholesky factor R (upper, in place); for which = 1 also R^-1 in FP32.
// A pivot below 1e-12 of the largest diagonal entry marks the problem as
// broken down (numerically rank-deficient H) and is replaced by that floor
// so the run completes.
constexpr double kGrpPivRel = 1e-12;

__global__ void __launch_bounds__(SM_THREADS)
k_grp_chol(const GrpProblem* __restrict__ probs, int w, int which, uint32_t* err) {
  extern __shared__ __align__(16) double cs[];
  const GrpProblem& P = probs[blockIdx.x];
  double* G = which == 1 ? P.G1 : P.G2;
  double* A = cs;                 // w x w
  double* Xi = cs + w * w;        // w x w: R^-1
  double* mx = Xi + w * w;
  const int tid = threadIdx.x;
  for (int e = tid; e < w * w; e += SM_THREADS) {
    const int i = e / w, j = e % w;
    A[e] = (i <= j) ? G[i * w + j] : G[j * w + i];
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < w; ++i) m = fmax(m, A[i * w + i]);
    mx[0] = m;
  }
  __syncthreads();
  const double floor_d = kGrpPivRel * mx[0];
  for (int c = 0; c < w; ++c) {
    if (tid == 0) {
      double d = A[c * w + c];
      if (!(d > floor_d)) {
        atomicOr(P.perr, DEV_ERR_BREAKDOWN);
        atomicOr(err, DEV_ERR_BREAKDOWN);
        d = floor_d > 0.0 ? floor_d : 1.0;
      }
      A[c * w + c] = sqrt(d);
    }
    __syncthreads();
    const double dinv = 1.0 / A[c * w + c];
    for (int j = c + 1 + tid; j < w; j += SM_THREADS) A[c * w + j] *= dinv;
    __syncthreads();
    const int t = w - c - 1;
    for (int e = tid; e < t * t; e += SM_THREADS) {
      const int i = c + 1 + e / t, j = c + 1 + e % t;
      if (i <= j) A[i * w + j] -= A[c * w + i] * A[c * w + j];
    }
    __syncthreads();
  }
  for (int e = tid; e < w * w; e += SM_THREADS) {
    const int i = e / w, j = e % w;
    G[e] = (i <= j) ? A[e] : 0.0;
  }
  if (which == 1) {
    // column jc of R^-1 by back substitution (thread jc)
    for (int jc = tid; jc < w; jc += SM_THREADS) {
      for (int i = w - 1; i > jc; --i) Xi[i * w + jc] = 0.0;
      Xi[jc * w + jc] = 1.0 / A[jc * w + jc];
      for (int i = jc - 1; i >= 0; --i) {
        double s = 0.0;
        for (int q = i + 1; q <= jc; ++q) s += A[i * w + q] * Xi[q * w + jc];
        Xi[i * w + jc] = -s / A[i * w + i];
      }
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += SM_THREADS) P.R1inv[e] = (float)Xi[e];
  }
}

void launch_chol(const GrpProblem* probs, int count, int w, int which, uint32_t* err, cudaStream_t st) {
  const size_t smem = (size_t)(2 * w * w + 2) * 8;
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grp_chol<<<count, SM_THREADS, smem, st>>>(probs, w, which, err);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

// ------------------------------------------------------------------- svd
// One CTA per problem: Steps 4-6 on the n side.
//   T = T1 R2^-1 (the T pass used Q1 = H R1^-1; Q = Q1 R2^-1);
//   T = Q_T R_T (Householder); R_T W = B with orthogonal columns (one-sided
//   Jacobi, round-robin pairs, FP32, to |b_a^T b_b| <= w u ||b_a|| ||b_b||);
//   sigma_c = ||b_c||, sorted descending; for the k largest:
//   S = sigma, V = T W_k Sigma^-1 = T1 (R2^-1 W_k) Sigma^-1,
//   MU = R2^-1 W_k (U = Q1 MU = Q W_k).
// Relative accuracy of sigma and the singular vectors follows from the
// backward stability of Householder QR and of one-sided Jacobi.
constexpr int kGrpMaxSweeps = 30;

// R2^-1 (FP32, w x w row-major, upper) from R2 (FP64 upper, global): thread
// jc solves column jc; entries below the diagonal are zero.
__device__ void r2_inverse(const double* __restrict__ R, int w, float* out) {
  for (int jc = threadIdx.x; jc < w; jc += SM_THREADS) {
    for (int i = w - 1; i > jc; --i) out[i * w + jc] = 0.f;
    out[jc * w + jc] = (float)(1.0 / R[jc * w + jc]);
    for (int i = jc - 1; i >= 0; --i) {
      double s = 0.0;
      for (int q = i + 1; q <= jc; ++q) s += R[i * w + q] * (double)out[q * w + jc];
      out[i * w + jc] = (float)(-s / R[i * w + i]);
    }
  }
}

__global__ void __launch_bounds__(SM_THREADS)
k_grp_svd(const GrpProblem* __restrict__ probs, int w, int ldt, int max_n, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char sv_raw[];
  const GrpProblem& P = probs[blockIdx.x];
  const int n = (int)P.n, k = P.k;
  const int ld = n | 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* nrm = reinterpret_cast<double*>(sv_raw);   // 64
  double* sig = nrm + 64;                            // 64
  int* perm = reinterpret_cast<int*>(sig + 64);      // 64
  int* flag = perm + 64;                             // 4
  float* tau = reinterpret_cast<float*>(flag + 4);   // 64
  float* v0 = tau + 64;
  float* rdiag = v0 + 64;
  float* Ms = rdiag + 64;                            // 64 x 64: R2^-1, then B (column-major)
  float* Ws = Ms + 64 * 64;                          // 64 x 64: W (column-major)
  float* Tc = Ws + 64 * 64;                          // w x ld: T (column-major), then scratch
  (void)max_n;

  // 1-2: T = T1 R2^-1
  r2_inverse(P.G2, w, Ms);
  __syncthreads();
  for (int e = tid; e < n * w; e += SM_THREADS) {
    const int c = e / n, r = e % n;
    const float* t1 = P.T + (int64_t)r * ldt;
    float s = 0.f;
    for (int q = 0; q <= c; ++q) s += t1[q] * Ms[q * w + c];
    Tc[(size_t)c * ld + r] = s;
  }
  __syncthreads();
  // 3: Householder QR of T; B = R_T, W = I
  hh_qr(Tc, n, ld, w, tau, v0, rdiag, nrm);
  for (int e = tid; e < w * w; e += SM_THREADS) {
    const int c = e / w, i = e % w;
    Ms[e] = (i < c) ? Tc[(size_t)c * ld + i] : (i == c ? rdiag[c] : 0.f);
    Ws[e] = (i == c) ? 1.f : 0.f;
  }
  __syncthreads();
  // 4: one-sided Jacobi on the columns of B
  const int wp = w + (w & 1), N = wp - 1;
  const float tol = (float)w * 5.9604645e-8f;
  int sweep = 0;
  for (; sweep < kGrpMaxSweeps; ++sweep) {
    if (tid == 0) flag[0] = 0;
    __syncthreads();
    for (int rd = 0; rd < N; ++rd) {
      for (int pi = warp; pi < wp / 2; pi += SM_WARPS) {
        const int a = (pi == 0) ? 0 : 1 + (rd + pi) % N;
        const int b = (pi == 0) ? 1 + rd % N : 1 + (rd + N - pi) % N;
        if (a >= w || b >= w) continue;
        float* Ba = Ms + a * w;
        float* Bb = Ms + b * w;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int q = lane; q < w; q += 32) {
          const float x = Ba[q], y = Bb[q];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be)) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float cs = rsqrtf(1.f + t * t), sn = cs * t;
          float* Wa = Ws + a * w;
          float* Wb = Ws + b * w;
          for (int q = lane; q < w; q += 32) {
            const float x = Ba[q], y = Bb[q];
            Ba[q] = cs * x - sn * y;
            Bb[q] = sn * x + cs * y;
            const float u = Wa[q], v = Wb[q];
            Wa[q] = cs * u - sn * v;
            Wb[q] = sn * u + cs * v;
          }
          if (lane == 0) flag[0] = 1;
        }
      }
      __syncthreads();
    }
    const int rotated = flag[0];
    __syncthreads();
    if (!rotated) break;
  }
  if (sweep == kGrpMaxSweeps && tid == 0) atomicOr(P.perr, DEV_ERR_JACOBI);
  // 5: sigma_c = ||b_c||, descending order
  for (int c = warp; c < w; c += SM_WARPS) {
    double s = 0.0;
    for (int q = lane; q < w; q += 32) s += (double)Ms[c * w + q] * Ms[c * w + q];
    s = warp_sum_d(s);
    if (lane == 0) sig[c] = sqrt(s);
  }
  __syncthreads();
  if (tid == 0) {
    for (int c = 0; c < w; ++c) perm[c] = c;
    for (int c = 0; c < w; ++c) {
      int best = c;
      for (int q = c + 1; q < w; ++q)
        if (sig[perm[q]] > sig[perm[best]]) best = q;
      const int t = perm[c];
      perm[c] = perm[best];
      perm[best] = t;
    }
  }
  __syncthreads();
  // 6: Y = R2^-1 W_k (w x k), then S, MU = Y, V = T1 Y Sigma^-1
  float* R2i = Tc;                 // w x w
  float* Y = Tc + w * w;           // w x k
  r2_inverse(P.G2, w, R2i);
  __syncthreads();
  for (int e = tid; e < w * k; e += SM_THREADS) {
    const int i = e / k, j = e % k;
    const float* wc = Ws + perm[j] * w;
    float s = 0.f;
    for (int q = i; q < w; ++q) s += R2i[i * w + q] * wc[q];
    Y[e] = s;
  }
  __syncthreads();
  if (P.S)
    for (int j = tid; j < k; j += SM_THREADS) P.S[j] = sig[perm[j]];
  for (int e = tid; e < w * k; e += SM_THREADS) P.MU[e] = Y[e];
  if (P.V) {
    for (int e = tid; e < n * k; e += SM_THREADS) {
      const int r = e / k, j = e % k;
      const float* t1 = P.T + (int64_t)r * ldt;
      float s = 0.f;
      for (int q = 0; q < w; ++q) s += t1[q] * Y[q * k + j];
      const double sj = sig[perm[j]];
      P.V[(int64_t)r * P.ldv + j] = sj > 0.0 ? (float)(s / sj) : 0.f;
    }
  }
  (void)err;
}

size_t svd_smem(int w, int max_n) {
  const size_t tc = std::max<size_t>((size_t)w * (max_n | 1), (size_t)2 * 64 * 64);
  return 64 * 8 * 2 + 68 * 4 + 3 * 64 * 4 + 2 * 64 * 64 * 4 + tc * 4 + 16;
}

void launch_svd(const GrpProblem* probs, int count, int w, int ldt, int max_n, uint32_t* err, cudaStream_t st) {
  const size_t smem = svd_smem(w, max_n);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grp_svd<<<count, SM_THREADS, smem, st>>>(probs, w, ldt, max_n, err);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

}  // namespace grp
}  // namespace rpca
