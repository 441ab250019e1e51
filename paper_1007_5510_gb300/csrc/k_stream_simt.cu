// Streamed passes over A on CUDA cores (FP64 workloads, small or odd shapes,
// and the reference CUDA-core path for the tensor-core kernels).
//
// One pass (Section 4.2 of the paper, row-major A read by row blocks):
//   MODE_FUSED  H_b = A_b X (stored), F += A_b^T H_b         (Step 1, eqs.
//               first_prod..last_prod: the H of this pass and the F = A^T H
//               the next pass multiplies by)
//   MODE_H      H_b = A_b X only                              (last power step)
//   MODE_T      F += A_b^T Q_b with Q read from memory         (Step 3)
// A_b is centred/scaled in registers: a -> a * col_scale[j] - shift[j]; it is
// never materialised.  H rows may get a per-column correction subtracted
// (H = A~ X - 1 corr^T, the rank-one centring term), and in the first
// centred pass an all-ones column is appended to H so that F's extra column
// accumulates A~^T 1.
#include "common.cuh"
#include "kernels.h"

namespace rpca {

namespace {

constexpr int THREADS = 256;
constexpr int PW = 64;  // output column group width

template <typename TC> struct SimtCfg;
template <> struct SimtCfg<float> { static constexpr int BM = 128; };
template <> struct SimtCfg<double> { static constexpr int BM = 64; };

template <typename TA, typename TC>
__device__ __forceinline__ TC load_a(const TA* __restrict__ A, int64_t lda, int64_t r, int64_t j,
                                     int64_t m, int64_t n, const float* __restrict__ scale,
                                     const TC* __restrict__ shift) {
  if (r >= m || j >= n) return TC(0);
  TC v;
  if constexpr (std::is_same<TA, double>::value) {
    v = TC(A[r * lda + j]);
  } else {
    v = TC(to_f32(A[r * lda + j]));
  }
  if (scale) v *= TC(scale[j]);
  if (shift) v -= shift[j];
  return v;
}

// grid: (panel blocks, column groups).  Persistent over panels.
template <typename TA, typename TC, int MODE, typename TF>
__global__ void __launch_bounds__(THREADS)
k_pass_simt(const TA* __restrict__ A, int64_t lda, int64_t m, int64_t n,
            const float* __restrict__ scale, const TC* __restrict__ shift,
            const TC* __restrict__ X, int64_t ldx, int p,
            TC* __restrict__ H, int64_t ldh, const TC* __restrict__ corr, int ones_col,
            TF* __restrict__ F, int64_t ldf) {
  constexpr int BM = SimtCfg<TC>::BM;
  constexpr int KC = 32;                 // phase-1 K chunk
  constexpr int JC = 64;                 // phase-2 n chunk
  constexpr int RPT = BM / 16;           // phase-1 rows per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* Hs = reinterpret_cast<TC*>(smem_raw);              // [BM][PW+1]
  TC* As = Hs + BM * (PW + 1);                           // phase 1: [BM][KC+1]; phase 2: [BM][JC+1]
  TC* Xs = As + BM * (JC + 1);                           // [KC][PW]

  const int tid = threadIdx.x;
  const int c0 = blockIdx.y * PW;                        // output column group
  const int pc = min(PW, p - c0);                        // real columns in group
  const int64_t npan = (m + BM - 1) / BM;

  for (int64_t pan = blockIdx.x; pan < npan; pan += gridDim.x) {
    const int64_t r0 = pan * BM;
    // ------------------------------------------------ phase 1: Hs = A_b X
    if (MODE != MODE_T) {
      const int ty = tid / 16, tx = tid % 16;
      TC acc[RPT][4];
#pragma unroll
      for (int a = 0; a < RPT; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TC(0);
      for (int64_t k0 = 0; k0 < n; k0 += KC) {
        for (int e = tid; e < BM * KC; e += THREADS) {
          int rr = e / KC, kk = e % KC;
          As[rr * (KC + 1) + kk] = load_a<TA, TC>(A, lda, r0 + rr, k0 + kk, m, n, scale, shift);
        }
        for (int e = tid; e < KC * PW; e += THREADS) {
          int kk = e / PW, cc = e % PW;
          Xs[kk * PW + cc] = (k0 + kk < n && cc < pc) ? X[(k0 + kk) * ldx + c0 + cc] : TC(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
          TC xv[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) xv[b] = Xs[kk * PW + tx * 4 + b];
#pragma unroll
          for (int a = 0; a < RPT; ++a) {
            TC av = As[(ty * RPT + a) * (KC + 1) + kk];
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av, xv[b], acc[a][b]);
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int a = 0; a < RPT; ++a) {
        const int rr = ty * RPT + a;
        const int64_t r = r0 + rr;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int cc = tx * 4 + b;
          TC v = acc[a][b];
          if (corr && cc < pc) v -= corr[c0 + cc];
          if (r >= m || cc >= pc) v = TC(0);
          if (c0 + cc == ones_col && r < m) v = TC(1);
          Hs[rr * (PW + 1) + cc] = v;
          if (r < m && cc < pc && c0 + cc != ones_col) H[r * ldh + c0 + cc] = v;
        }
      }
    } else {
      for (int e = tid; e < BM * PW; e += THREADS) {
        int rr = e / PW, cc = e % PW;
        int64_t r = r0 + rr;
        Hs[rr * (PW + 1) + cc] = (r < m && cc < pc) ? H[r * ldh + c0 + cc] : TC(0);
      }
    }
    __syncthreads();
    if (MODE == MODE_H) continue;
    // ------------------------------------------- phase 2: F += A_b^T Hs
    const int fc = (ones_col >= 0 && MODE != MODE_T) ? min(PW, p + 1 - c0) : pc;
    const int ty = tid / 16, tx = tid % 16;      // ty: 4 n-rows, tx: 4 columns
    for (int64_t j0 = 0; j0 < n; j0 += JC) {
      for (int e = tid; e < BM * JC; e += THREADS) {
        int rr = e / JC, jj = e % JC;
        As[rr * (JC + 1) + jj] = load_a<TA, TC>(A, lda, r0 + rr, j0 + jj, m, n, scale, shift);
      }
      __syncthreads();
      TC acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TC(0);
#pragma unroll 4
      for (int rr = 0; rr < BM; ++rr) {
        TC hv[4], av[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) hv[b] = Hs[rr * (PW + 1) + tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[rr * (JC + 1) + ty * 4 + a];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], hv[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t j = j0 + ty * 4 + a;
        if (j >= n) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int cc = tx * 4 + b;
          if (cc < fc) atomicAdd(&F[j * ldf + c0 + cc], (TF)acc[a][b]);
        }
      }
      __syncthreads();
    }
  }
}

template <typename TA, typename TC, int MODE, typename TF>
void launch_one(const PassArgs& a, cudaStream_t st) {
  constexpr int BM = SimtCfg<TC>::BM;
  const int groups = (int)cdiv(a.p + (a.ones_col >= 0 ? 1 : 0), PW);
  size_t smem = sizeof(TC) * (size_t)(BM * (PW + 1) + BM * (64 + 1) + 32 * PW);
  auto kern = k_pass_simt<TA, TC, MODE, TF>;
  static bool attr_done = false;
  if (!attr_done) {
    RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_done = true;
  }
  int64_t npan = cdiv(a.m, BM);
  int sms = num_sms();
  int64_t gx = std::min<int64_t>(npan, (int64_t)sms * 4 / std::max(1, groups) + 1);
  dim3 grid((unsigned)std::max<int64_t>(1, gx), (unsigned)groups);
  kern<<<grid, THREADS, smem, st>>>(
      static_cast<const TA*>(a.A), a.lda, a.m, a.n, a.scale, static_cast<const TC*>(a.shift),
      static_cast<const TC*>(a.X), a.ldx, a.p, static_cast<TC*>(a.H), a.ldh,
      static_cast<const TC*>(a.corr), a.ones_col, static_cast<TF*>(a.F), a.ldf);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

template <typename TA, typename TC>
void launch_mode(const PassArgs& a, cudaStream_t st) {
  switch (a.mode) {
    case MODE_FUSED: launch_one<TA, TC, MODE_FUSED, TC>(a, st); break;
    case MODE_H: launch_one<TA, TC, MODE_H, TC>(a, st); break;
    case MODE_T:
      if (a.f_f64) launch_one<TA, TC, MODE_T, double>(a, st);
      else launch_one<TA, TC, MODE_T, TC>(a, st);
      break;
  }
}

}  // namespace

void launch_pass_simt(const PassArgs& a, cudaStream_t st) {
  if (a.F && a.mode != MODE_H && !a.accumulate_f) {
    const int fcols = a.p + (a.ones_col >= 0 ? 1 : 0);
    const size_t es = (a.dtype == RPCA_F64 || a.f_f64) ? 8 : 4;
    RPCA_CUDA_TRY(cudaMemset2DAsync(a.F, (size_t)a.ldf * es, 0, (size_t)fcols * es, (size_t)a.n, st));
  }
  switch (a.dtype) {
    case RPCA_F64: launch_mode<double, double>(a, st); break;
    case RPCA_F32: launch_mode<float, float>(a, st); break;
    case RPCA_BF16: launch_mode<__nv_bfloat16, float>(a, st); break;
    case RPCA_FP8E4M3: launch_mode<__nv_fp8_e4m3, float>(a, st); break;
  }
}

}  // namespace rpca
