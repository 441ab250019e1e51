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
#include "tc_common.cuh"

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

// Squared norm of rows [r0, n) of column c (one warp): four independent FP32
// partial sums per lane, FP64 total.
__device__ __forceinline__ double col_nrm2(const float* col, int r0, int n, int lane) {
  float s[4] = {0.f, 0.f, 0.f, 0.f};
  int r = r0 + lane;
  for (; r + 96 < n; r += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] += col[r + 32 * u] * col[r + 32 * u];
  }
  for (; r < n; r += 32) s[0] += col[r] * col[r];
  return warp_sum_d((double)((s[0] + s[1]) + (s[2] + s[3])));
}

// v^T a over rows [c, n) with v = (v0, vc[c+1..n)) (one warp; four
// independent partial sums per lane).
__device__ __forceinline__ float hh_dot(const float* vc, const float* a2, float fv0, int c, int n, int lane) {
  float d[4] = {0.f, 0.f, 0.f, 0.f};
  int r = c + lane;
  if (r == c) {
    d[0] = fv0 * a2[c];
    r += 32;
  }
  for (; r + 96 < n; r += 128) {
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u] += vc[r + 32 * u] * a2[r + 32 * u];
  }
  for (; r < n; r += 32) d[1] += vc[r] * a2[r];
  return warp_sum((d[0] + d[1]) + (d[2] + d[3]));
}

// a -= d v over rows [c, n).
__device__ __forceinline__ void hh_axpy(const float* vc, float* a2, float fv0, float d, int c, int n, int lane) {
  int r = c + lane;
  if (r == c) {
    a2[c] -= d * fv0;
    r += 32;
  }
#pragma unroll 4
  for (; r < n; r += 32) a2[r] -= d * vc[r];
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
    if (threadIdx.x == 0) {
      // the reflector's scalars, once (FP64 division and square root are
      // slow: not in every thread)
      const double nrm2 = nrm[c];
      const double x0 = (c < n) ? (double)vc[c] : 0.0;
      double alpha = 0.0, vv0 = 0.0, t = 0.0;
      if (nrm2 > 0.0) {
        alpha = (x0 >= 0.0) ? -sqrt(nrm2) : sqrt(nrm2);
        vv0 = x0 - alpha;
        const double vn2 = nrm2 - x0 * x0 + vv0 * vv0;
        t = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
      }
      tau[c] = (float)t;
      v0[c] = (float)vv0;
      rdiag[c] = (float)alpha;
    }
    __syncthreads();
    const float fv0 = v0[c], ft = tau[c];
    for (int c2 = c + 1 + warp; c2 < nc; c2 += SM_WARPS) {
      float* a2 = A + (size_t)c2 * ld;
      const float d = hh_dot(vc, a2, fv0, c, n, lane) * ft;
      hh_axpy(vc, a2, fv0, d, c, n, lane);
      if (c2 == c + 1) {
        __syncwarp();
        const double s = col_nrm2(a2, c + 1, n, lane);
        if (lane == 0) nrm[c + 1] = s;
      }
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
      const float d = hh_dot(vc, a2, fv0, c, n, lane) * t;
      hh_axpy(vc, a2, fv0, d, c, n, lane);
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
  if (__syncthreads_or((*(volatile uint32_t*)err & DEV_ERR_TIMEOUT) != 0)) return;   // an earlier step gave up
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
        // four independent accumulation chains per thread
        int ci[4], cj[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = min(tid + q * SM_THREADS, l * l - 1);
          ci[q] = e / l;
          cj[q] = e % l;
        }
        for (int r = 0; r < nr; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += Xs[r * 33 + ci[q]] * Fc[(size_t)cj[q] * ld + r0 + r];
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
//   ROW_GRAM_T G3 += T1^T T1 (the n side: rows of T)
// The Gram products use 4 x 4 register tiles over the upper block triangle
// (FP32 within an item, FP64 reductions across items).
enum RowMode : int { ROW_GRAM = 0, ROW_APPLY = 1, ROW_U = 2, ROW_GRAM_T = 3 };

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

// Shared-memory row pitch of a staged tile: a multiple of 4 floats with an
// odd number of 16-byte chunks, so 16-byte loads of 8 consecutive rows by a
// quarter-warp hit distinct banks.
__device__ __host__ __forceinline__ int tile_ld(int wp) { return ((wp >> 2) & 1) ? wp : wp + 4; }

// 4 x 4 register tile of Y = X M for a tile X (rows rg + rs x, x < 4, of Xs
// with pitch ls) and M (rows t < tmax, pitch lm, zero past its last
// column): the columns 4 cg .. 4 cg + 3.
__device__ __forceinline__ void tile_product(const float* Xs, int ls, int rs, const float* M, int lm, int tmax,
                                             int rg, int cg, float (&y)[4][4]) {
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int q = 0; q < 4; ++q) y[x][q] = 0.f;
  for (int t = 0; t < tmax; t += 4) {
    float4 h[4], m[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) h[x] = *reinterpret_cast<const float4*>(Xs + (rg + rs * x) * ls + t);
#pragma unroll
    for (int u = 0; u < 4; ++u) m[u] = *reinterpret_cast<const float4*>(M + (t + u) * lm + 4 * cg);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const float hv[4] = {h[x].x, h[x].y, h[x].z, h[x].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        y[x][0] += hv[u] * m[u].x;
        y[x][1] += hv[u] * m[u].y;
        y[x][2] += hv[u] * m[u].z;
        y[x][3] += hv[u] * m[u].w;
      }
    }
  }
}

// Rows of an item reach shared memory through a ring of RS_STAGES bulk
// copies of 64 rows (the rows of H and T are contiguous with a pitch of wp
// floats, a multiple of 16 bytes); thread 0 refills a stage as soon as every
// thread is done with it.
constexpr int RS_STAGES = 4;

template <int MODE>
__global__ void __launch_bounds__(SM_THREADS, 2)
k_grp_rows(const GrpProblem* __restrict__ probs, const GrpRItem* __restrict__ items, int w, int k, uint32_t* err) {
  extern __shared__ __align__(16) float rs[];
  if (__syncthreads_or((*(volatile uint32_t*)err & DEV_ERR_TIMEOUT) != 0)) return;   // an earlier step or CTA gave up
  const GrpRItem I = items[blockIdx.x];
  const GrpProblem& P = probs[I.p];
  const int wp = (w + 3) & ~3;
  const int kp = (k + 3) & ~3;
  const int tid = threadIdx.x;
  const float* src = (MODE == ROW_GRAM_T) ? P.T : P.H;   // pitch wp
  float* Ms = rs;                                  // 64 x 64: R1^-1 (pitch wp) or MU (pitch kp)
  float* Qs = Ms + 64 * 64;                        // 64 x wp: Q1 rows (ROW_APPLY); flush scratch
  float* ring = Qs + 64 * 64;                      // RS_STAGES x 64 x wp
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + RS_STAGES * 64 * 64);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(full + RS_STAGES);
  const int nsub = (I.nrows + 63) / 64;
  auto issue = [&](int sidx) {
    const int nr = min(64, I.nrows - 64 * sidx);
    const uint32_t bytes = (uint32_t)(nr * wp * 4);
    uint64_t* bar = &full[sidx % RS_STAGES];
    tc::mbar_arrive_expect_tx(bar, bytes);
    tc::bulk_load_1d(ring + (sidx % RS_STAGES) * 64 * 64, src + ((int64_t)I.r0 + 64 * sidx) * wp, bytes, bar);
  };
  if (tid == 0) {
    for (int q = 0; q < RS_STAGES; ++q) tc::mbar_init(&full[q], 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    for (int q = 0; q < RS_STAGES && q < nsub; ++q) issue(q);
  }
  if (MODE == ROW_APPLY)
    for (int e = tid; e < 64 * wp; e += SM_THREADS) {
      const int t = e / wp, c = e % wp;
      Ms[e] = (t < w && c < w) ? P.R1inv[t * w + c] : 0.f;
    }
  if (MODE == ROW_U)
    for (int e = tid; e < 64 * kp; e += SM_THREADS) {
      const int t = e / kp, c = e % kp;
      Ms[e] = (t < w && c < k) ? P.MU[t * k + c] : 0.f;
    }
  __syncthreads();
  const GramTile g = gram_tile(w);
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  int sidx = 0;
  for (; sidx < nsub; ++sidx) {
    const int nr = min(64, I.nrows - 64 * sidx);
    const int64_t grow0 = (int64_t)I.r0 + 64 * sidx;
    const bool ok = tc::mbar_wait(&full[sidx % RS_STAGES], (uint32_t)((sidx / RS_STAGES) & 1), err, abort_flag);
    if (__syncthreads_or(!ok)) break;
    float* Hs = ring + (sidx % RS_STAGES) * 64 * 64;   // rows >= nr hold stale data: never used
    if (MODE == ROW_GRAM || MODE == ROW_GRAM_T) {
      gram_rows(g, Hs, wp, nr, acc);
    } else if (MODE == ROW_APPLY) {
      // Q1 = H R1^-1 (R1^-1 upper triangular: rows t <= 4 cg + 3 only)
      const int ncg = wp / 4;
      if (tid < 16 * ncg) {
        const int rg = tid & 15, cg = tid >> 4;
        float q[4][4];
        tile_product(Hs, wp, 16, Ms, wp, min(wp, 4 * cg + 4), rg, cg, q);
#pragma unroll
        for (int x = 0; x < 4; ++x)
          *reinterpret_cast<float4*>(Qs + (rg + 16 * x) * wp + 4 * cg) = make_float4(q[x][0], q[x][1], q[x][2], q[x][3]);
      }
      __syncthreads();
      gram_rows(g, Qs, wp, nr, acc);
      for (int e = tid; e < nr * wp / 4; e += SM_THREADS)
        reinterpret_cast<float4*>(P.H + grow0 * wp)[e] = reinterpret_cast<const float4*>(Qs)[e];
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
    } else if (P.U) {
      // U = Q1 MU
      const int nkg = kp / 4;
      if (tid < 16 * nkg) {
        const int rg = tid & 15, cg = tid >> 4;
        float u[4][4];
        tile_product(Hs, wp, 16, Ms, kp, wp, rg, cg, u);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int r = rg + 16 * x;
          if (r < nr) {
            float* dst = P.U + (grow0 + r) * P.ldu + 4 * cg;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (4 * cg + q < k) dst[q] = u[x][q];
          }
        }
      }
    }
    __syncthreads();   // every thread is done with this stage (and with Qs)
    if (tid == 0 && sidx + RS_STAGES < nsub) {
      tc::fence_proxy_async_smem();
      issue(sidx + RS_STAGES);
    }
  }
  if (tid == 0) {
    // after an abort, the copies still in flight land before the CTA exits
    volatile int never = 0;
    const int issued = min(nsub, sidx + RS_STAGES);
    for (int q = sidx; q < issued; ++q)
      tc::mbar_wait(&full[q % RS_STAGES], (uint32_t)((q / RS_STAGES) & 1), nullptr, &never);
  }
  if (sidx < nsub) return;   // aborted: no partial Gram is added
  if (MODE == ROW_GRAM) gram_flush(g, acc, Qs, P.G1, w);
  if (MODE == ROW_GRAM_T) gram_flush(g, acc, Qs, P.G3, w);
  if (MODE == ROW_APPLY) gram_flush(g, acc, Qs, P.G2, w);
}

static size_t rows_smem(int w) {
  (void)w;
  return ((size_t)(2 + RS_STAGES) * 64 * 64) * 4 + RS_STAGES * 8 + 16;
}

template <int MODE>
static void launch_rows(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, int k,
                        uint32_t* err, cudaStream_t st) {
  if (nitems <= 0) return;
  const size_t smem = rows_smem(w);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_rows<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grp_rows<MODE><<<(unsigned)nitems, SM_THREADS, smem, st>>>(probs, items, w, k, err);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void launch_gram(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, uint32_t* err,
                 cudaStream_t st) {
  launch_rows<ROW_GRAM>(probs, items, nitems, w, 0, err, st);
}
void launch_apply(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, uint32_t* err,
                  cudaStream_t st) {
  launch_rows<ROW_APPLY>(probs, items, nitems, w, 0, err, st);
}
void launch_u(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, int k, uint32_t* err,
              cudaStream_t st) {
  launch_rows<ROW_U>(probs, items, nitems, w, k, err, st);
}
void launch_gram_t(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, uint32_t* err,
                   cudaStream_t st) {
  launch_rows<ROW_GRAM_T>(probs, items, nitems, w, 0, err, st);
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
  if (__syncthreads_or((*(volatile uint32_t*)err & DEV_ERR_TIMEOUT) != 0)) return;
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
  {
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
    float* out = which == 1 ? P.R1inv : P.R2inv;
    for (int e = tid; e < w * w; e += SM_THREADS) out[e] = (float)Xi[e];
  }
}

void launch_chol(const GrpProblem* probs, int count, int w, int which, uint32_t* err, cudaStream_t st) {
  const size_t smem = (size_t)(2 * w * w + 2) * 8;
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grp_chol<<<count, SM_THREADS, smem, st>>>(probs, w, which, err);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

// ------------------------------------------------------------------- eig
// One CTA per problem: Steps 4-6 on the n side from the Gram of T.
//   G_T = R2^-T (T1^T T1) R2^-1 = T^T T   (T = T1 R2^-1: the T pass used
//         Q1 = H R1^-1 and Q = Q1 R2^-1)
//   G_T = R_T^T R_T (Cholesky); R_T W = B with orthogonal columns
//         (one-sided Jacobi, four lanes per column pair of a round)
//   the k largest ||b_c||: Y = R2^-1 W_k; V~ = T1 Y; sigma_j = ||V~_j||
//   (second-order accurate in the error of w_j); V = V~ Sigma^-1,
//   MU = Y (U = Q1 MU = Q W_k), S = sigma.
// Everything in FP32 (the FP64 pipe of this part is 1/64 of FP32): with
// BF16 storage the inputs carry 2^-9 relative rounding, and the FP32 Gram's
// error (~u32 sigma_1^2 in sigma_j^2) stays below the data's own error for
// the sigma_j the method resolves.
constexpr int EG_THREADS = 128;
constexpr int kGrpMaxSweeps = 30;

// C[i][j] = sum_t X[t][i] Y[t][j] (4 x 4 tile at i0, j0; pitches lx, ly).
__device__ __forceinline__ void tile_tn(const float* X, int lx, const float* Y, int ly, int K, int i0, int j0,
                                        float (&c)[4][4]) {
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) c[x][y] = 0.f;
  for (int t = 0; t < K; ++t) {
    const float4 a = *reinterpret_cast<const float4*>(X + t * lx + i0);
    const float4 b = *reinterpret_cast<const float4*>(Y + t * ly + j0);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) c[x][y] += av[x] * bv[y];
  }
}

__global__ void __launch_bounds__(EG_THREADS)
k_grp_eig(const GrpProblem* __restrict__ probs, int w, uint32_t* err) {
  extern __shared__ __align__(16) float eg[];
  if (__syncthreads_or((*(volatile uint32_t*)err & DEV_ERR_TIMEOUT) != 0)) return;
  const GrpProblem& P = probs[blockIdx.x];
  const int n = (int)P.n, k = P.k;
  const int wp = (w + 3) & ~3, kp = (k + 3) & ~3;
  const int tid = threadIdx.x;
  const int lb = w | 1;                   // odd pitch of B and W: the lanes' columns in distinct banks
  const int ls = tile_ld(wp);             // pitch of the T1 staging tile
  const int bw = (w * lb + 3) & ~3;
  float* Gs = eg;                         // wp x wp: G3, then G_T, then R_T
  float* Rs = Gs + wp * wp;               // wp x wp: R2^-1 (zero-padded)
  float* Ts = Rs + wp * wp;               // wp x wp: G3 R2^-1; then Y (wp x kp)
  float* B = Ts + wp * wp;                // w x lb column-major
  float* W = B + bw;                      // w x lb column-major
  float* S1 = W + bw;                     // 128 x ls staging of T1 rows
  float* nrm = S1 + 128 * ls;             // 64
  float* ssq = nrm + 64;                  // 64
  int* perm = reinterpret_cast<int*>(ssq + 64);   // 64

  for (int e = tid; e < wp * wp; e += EG_THREADS) {
    const int i = e / wp, j = e % wp;
    const bool in = i < w && j < w;
    Gs[e] = in ? (float)((i <= j) ? P.G3[i * w + j] : P.G3[j * w + i]) : 0.f;
    Rs[e] = in ? P.R2inv[i * w + j] : 0.f;
  }
  __syncthreads();
  // Ts = G3 R2^-1 (G3 symmetric: G3[t][i] = G3[i][t]), then G_T = R2^-T Ts
  const int nt4 = wp / 4;
  for (int tt = tid; tt < nt4 * nt4; tt += EG_THREADS) {
    const int i0 = 4 * (tt / nt4), j0 = 4 * (tt % nt4);
    float c[4][4];
    tile_tn(Gs, wp, Rs, wp, wp, i0, j0, c);
#pragma unroll
    for (int x = 0; x < 4; ++x)
      *reinterpret_cast<float4*>(Ts + (i0 + x) * wp + j0) = make_float4(c[x][0], c[x][1], c[x][2], c[x][3]);
  }
  __syncthreads();
  for (int tt = tid; tt < nt4 * nt4; tt += EG_THREADS) {
    const int i0 = 4 * (tt / nt4), j0 = 4 * (tt % nt4);
    float c[4][4];
    tile_tn(Rs, wp, Ts, wp, wp, i0, j0, c);
#pragma unroll
    for (int x = 0; x < 4; ++x)
      *reinterpret_cast<float4*>(Gs + (i0 + x) * wp + j0) = make_float4(c[x][0], c[x][1], c[x][2], c[x][3]);
  }
  __syncthreads();
  // Cholesky G_T = R_T^T R_T (upper, in place, symmetric part read from the
  // upper triangle); a pivot below 1e-10 of the largest diagonal entry is a
  // direction T does not have: its row is zero
  if (tid == 0) {
    float m = 0.f;
    for (int i = 0; i < w; ++i) m = fmaxf(m, Gs[i * wp + i]);
    nrm[0] = m;
  }
  __syncthreads();
  const float floor_d = 1e-10f * nrm[0];
  for (int c = 0; c < w; ++c) {
    const float d = Gs[c * wp + c];
    const float piv = d > floor_d ? sqrtf(d) : 0.f;
    const float inv = piv > 0.f ? 1.f / piv : 0.f;
    __syncthreads();
    if (tid == 0) Gs[c * wp + c] = piv;
    for (int j = c + 1 + tid; j < w; j += EG_THREADS) Gs[c * wp + j] *= inv;
    __syncthreads();
    const int t = w - c - 1;
    for (int e = tid; e < t * t; e += EG_THREADS) {
      const int i = c + 1 + e / t, j = c + 1 + e % t;
      if (i <= j) Gs[i * wp + j] -= Gs[c * wp + i] * Gs[c * wp + j];
    }
    __syncthreads();
  }
  // B = R_T (column c holds rows 0..c), W = I
  for (int e = tid; e < w * w; e += EG_THREADS) {
    const int c = e / w, i = e % w;
    B[c * lb + i] = (i <= c) ? Gs[i * wp + c] : 0.f;
    W[c * lb + i] = (i == c) ? 1.f : 0.f;
  }
  __syncthreads();
  // one-sided Jacobi on the columns of B: four lanes per pair (circle
  // method over wpv = w rounded up to even; index w is a dummy)
  {
    const int wpv = w + (w & 1), N = wpv - 1;
    const int pi = tid >> 2, sub = tid & 3;
    const float tol = (float)w * 5.9604645e-8f;
    int sweep = 0;
    for (; sweep < kGrpMaxSweeps; ++sweep) {
      int rot = 0;
      for (int rd = 0; rd < N; ++rd) {
        const bool act = pi < wpv / 2;
        const int a = (pi == 0) ? 0 : 1 + (rd + pi) % N;
        const int b = (pi == 0) ? 1 + rd % N : 1 + (rd + N - pi) % N;
        const bool valid = act && a < w && b < w;
        float* Ba = B + (valid ? a : 0) * lb;
        float* Bb = B + (valid ? b : 0) * lb;
        float al = 0.f, be = 0.f, ga = 0.f;
        if (valid) {
#pragma unroll 4
          for (int q = sub; q < w; q += 4) {
            const float x = Ba[q], y = Bb[q];
            al += x * x;
            be += y * y;
            ga += x * y;
          }
        }
        // the four lanes of a pair are consecutive lanes of one warp
        al += __shfl_xor_sync(0xffffffffu, al, 1);
        be += __shfl_xor_sync(0xffffffffu, be, 1);
        ga += __shfl_xor_sync(0xffffffffu, ga, 1);
        al += __shfl_xor_sync(0xffffffffu, al, 2);
        be += __shfl_xor_sync(0xffffffffu, be, 2);
        ga += __shfl_xor_sync(0xffffffffu, ga, 2);
        if (valid && ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be)) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float cs = rsqrtf(1.f + t * t), sn = cs * t;
          float* Wa = W + a * lb;
          float* Wb = W + b * lb;
#pragma unroll 4
          for (int q = sub; q < w; q += 4) {
            const float x = Ba[q], y = Bb[q];
            Ba[q] = cs * x - sn * y;
            Bb[q] = sn * x + cs * y;
            const float u = Wa[q], v = Wb[q];
            Wa[q] = cs * u - sn * v;
            Wb[q] = sn * u + cs * v;
          }
          rot = 1;
        }
        __syncthreads();
      }
      if (!__syncthreads_or(rot)) break;
    }
    if (sweep == kGrpMaxSweeps && tid == 0) atomicOr(P.perr, DEV_ERR_JACOBI);
  }
  // ||b_c||^2 (four lanes per column) and the descending order
  // (the trip count is the same for every lane: the shuffles need them all)
  for (int c0 = 0; c0 < w; c0 += EG_THREADS / 4) {
    const int c = c0 + (tid >> 2);
    float s2 = 0.f;
    if (c < w)
      for (int q = tid & 3; q < w; q += 4) s2 += B[c * lb + q] * B[c * lb + q];
    s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
    s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
    if (c < w && (tid & 3) == 0) nrm[c] = (s2 == s2) ? s2 : -1.f;   // a NaN sorts last
  }
  __syncthreads();
  // rank of each value: a permutation for any input (ties by index)
  for (int c = tid; c < w; c += EG_THREADS) {
    int r = 0;
    for (int q = 0; q < w; ++q) r += (nrm[q] > nrm[c]) || (nrm[q] == nrm[c] && q < c);
    perm[r] = c;
  }
  if (tid < 64) ssq[tid] = 0.f;
  __syncthreads();
  // Y = R2^-1 W_k (w x k, pitch kp, zero-padded), into Ts
  float* Y = Ts;
  for (int e = tid; e < wp * kp; e += EG_THREADS) {
    const int i = e / kp, j = e % kp;
    float s = 0.f;
    if (i < w && j < k) {
      const float* wc = W + perm[j] * lb;
      for (int q = i; q < w; ++q) s += Rs[i * wp + q] * wc[q];
    }
    Y[e] = s;
  }
  __syncthreads();
  // two passes over T1, 128 rows at a time: sigma_j = ||T1 Y_j||, then V.
  // Thread tile: rows rg + 32 x (x < 4) by columns 4 cg .. 4 cg + 3.
  const int nkg = kp / 4;
  const int rg = tid & 31, cg = tid >> 5;
  for (int pass = 0; pass < 2; ++pass) {
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r0 = 0; r0 < n; r0 += 128) {
      const int nr = min(128, n - r0);
      __syncthreads();
      for (int e = tid; e < 128 * wp; e += EG_THREADS) {
        const int r = e / wp, c = e % wp;
        S1[r * ls + c] = (r < nr) ? P.T[(int64_t)(r0 + r) * wp + c] : 0.f;
      }
      __syncthreads();
      for (int cgi = cg; cgi < nkg; cgi += EG_THREADS / 32) {
        float v[4][4];
        tile_product(S1, ls, 32, Y, kp, wp, rg, cgi, v);
        if (pass == 0) {
          if (cgi == cg)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int q = 0; q < 4; ++q) part[q] += v[x][q] * v[x][q];
          else
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int q = 0; q < 4; ++q) atomicAdd(&ssq[4 * cgi + q], v[x][q] * v[x][q]);
        } else if (P.V) {
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int r = rg + 32 * x;
            if (r < nr)
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int j = 4 * cgi + q;
                if (j < k) P.V[(int64_t)(r0 + r) * P.ldv + j] = nrm[j] > 0.f ? v[x][q] / nrm[j] : 0.f;
              }
          }
        }
      }
    }
    if (pass == 0) {
      if (cg < nkg)
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(&ssq[4 * cg + q], part[q]);
      __syncthreads();
      if (tid < k) nrm[tid] = sqrtf(ssq[tid]);   // nrm now holds sigma_j
      __syncthreads();
    }
  }
  for (int e = tid; e < w * k; e += EG_THREADS) P.MU[e] = Y[(e / k) * kp + e % k];
  if (P.S)
    for (int j = tid; j < k; j += EG_THREADS) P.S[j] = (double)nrm[j];
  (void)err;
}

size_t eig_smem(int w) {
  const int wp = (w + 3) & ~3, lb = w | 1, bw = (w * lb + 3) & ~3;
  return (size_t)(3 * wp * wp + 2 * bw + 128 * tile_ld(wp) + 3 * 64) * 4 + 16;
}

void launch_svd(const GrpProblem* probs, int count, int w, int ldt, int max_n, uint32_t* err, cudaStream_t st) {
  (void)max_n;
  (void)ldt;
  const size_t smem = eig_smem(w);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grp_eig<<<count, EG_THREADS, smem, st>>>(probs, w, err);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

}  // namespace grp
}  // namespace rpca
