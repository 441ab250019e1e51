// Tall-skinny products of Step 2 (QR of H) and Steps 5-6 on tensor cores,
// FP32-accurate.
//   gram:   C (p x q, FP64) = X^T Y over all rows, X m x p, Y m x q.  The
//           rows are the reduction (MN-major operands), done in BF16 with
//           each FP32 value split exactly into three BF16 slices (six slice
//           products); CTAs split the rows and 64-column groups of C,
//           accumulate 128-row chunks in TMEM and sum the chunks in FP32
//           registers, adding to C once.
//   apply:  Y (m x q) = beta Y + alpha X M, X m x p (K-major operand), M p x q
//           (FP64 small matrix, resident in shared memory).  Every FP32
//           operand x is carried as x (its TF32 truncation is what the MMA
//           reads) plus x_lo = x - trunc_tf32(x) in a companion array:
//               x y ~ trunc(x) trunc(y) + trunc(x) y_lo + x_lo trunc(y)
//           (three kind::tf32 MMAs, ~2^-21 relative); Y_lo is written too.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rpca {
namespace {

constexpr int G_KSUB = 32;         // rows per Gram stage

__device__ __forceinline__ float tf32_trunc(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

__global__ void k_split_lo(int64_t rows, int cols, const float* __restrict__ X, int64_t ldx,
                           float* __restrict__ Xlo, int64_t ldl) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t r = e / cols;
  int c = (int)(e % cols);
  float x = X[r * ldx + c];
  Xlo[r * ldl + c] = x - tf32_trunc(x);
}

// ------------------------------------------------------------------ Gram
// FP32 data split exactly into three BF16 slices, x = x1 + x2 + x3 (x1 =
// RNE(x), x2 = RNE(x - x1), x3 = x - x1 - x2; each fits 8 significant bits),
// so every slice product is exact in FP32 and
//     x y ~ x1 y1 + x1 y2 + x2 y1 + x1 y3 + x2 y2 + x3 y1      (error ~2^-24)
// Slices are stored as three BF16 matrices of rows x ldS (ldS = cols rounded
// up to 64) so that TMA boxes of 64 columns tile them exactly.
// Rows [rows, plane_rows) of each plane are zero so that a TMA box never
// reads into the next plane.
__global__ void k_slice3(int64_t rows, int64_t plane_rows, int cols, int ldS, const float* __restrict__ X,
                         int64_t ldx, __nv_bfloat16* __restrict__ S, const uint32_t* __restrict__ active) {
  if (active && *active == 0u) return;
  // four consecutive columns per thread, 8-byte stores per plane
  const int64_t e4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per_row = ldS / 4;
  if (e4 >= plane_rows * per_row) return;
  const int64_t r = e4 / per_row;
  const int c0 = (int)(e4 % per_row) * 4;
  __nv_bfloat16 o1[4], o2[4], o3[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = c0 + q;
    float x = (c < cols && r < rows) ? X[r * ldx + c] : 0.f;
    o1[q] = __float2bfloat16_rn(x);
    float r1 = x - __bfloat162float(o1[q]);
    o2[q] = __float2bfloat16_rn(r1);
    o3[q] = __float2bfloat16_rn(r1 - __bfloat162float(o2[q]));
  }
  const int64_t plane = plane_rows * ldS;
  const int64_t e = r * ldS + c0;
  *reinterpret_cast<uint2*>(S + e) = *reinterpret_cast<uint2*>(o1);
  *reinterpret_cast<uint2*>(S + plane + e) = *reinterpret_cast<uint2*>(o2);
  *reinterpret_cast<uint2*>(S + 2 * plane + e) = *reinterpret_cast<uint2*>(o3);
}

// A operand: X columns [t*128, t*128+128) of each slice (MN-major, 2 boxes of
// 64 columns); B operand: the 64 columns [64g, 64g+64) of Y of this CTA's
// column group g = blockIdx.y (MN-major, one box per slice).  A stage holds
// the X slices (3 x NXB boxes) and, unless X and Y coincide, the three Y
// boxes of the group; boxes are G_KSUB rows x 64 BF16 columns.
//
// Accuracy: the tensor cores add each product into the FP32 accumulator
// with rounding relative to the accumulator's magnitude, so a long run of
// same-sign products (the diagonal of X^T X) drifts by a few ulp per step.
// TMEM therefore only ever accumulates one chunk of 128 rows (a bias of
// ~1e-6 relative); two TMEM buffers alternate, and the
// epilogue warps add each finished chunk into per-thread FP32 sums on the
// CUDA cores (round-to-nearest, so the few hundred chunk partials of a CTA
// add without drift), which go to C in FP64 once at the end.

constexpr int G_EC = 32;                     // C columns per epilogue thread
constexpr int G_EPI_WARPS_PER_T = 4 * (64 / G_EC);

// KS rows per stage (box KS x 64 BF16); nxb X boxes loaded per slice.  A
// stage holds 3 x nxb X boxes, 3 Y boxes unless SAME, and one spare box: the
// M = 128 A operand of the last tile may span one box past the loaded ones
// (rows of C beyond p, discarded).
template <int NT, bool SAME, int KS>
__global__ void __launch_bounds__(64 + 32 * G_EPI_WARPS_PER_T * NT, 1)
k_gram_bf16x3(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int64_t m,
              int64_t plane_rows, int x0, int y0, int p, int q, int nxb, int ngroup, int nstages,
              uint32_t stage_bytes, double* __restrict__ C, int64_t ldc, uint32_t* __restrict__ dev_err,
              const uint32_t* __restrict__ active, int upper) {
  if (active && *active == 0u) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t BOX = KS * 128;
  constexpr int NEPI = G_EPI_WARPS_PER_T * NT;          // epilogue warps
  constexpr int DRAIN = 128 / KS;                       // stages per TMEM chunk (128 rows)
  // upper (SAME only): column group cg needs rows [0, 64 (cg + 1)) of C,
  // i.e. the first cg + 1 boxes of X; the rest of C is left to symmetry
  const int nxl = (SAME && upper) ? min(nxb, (int)blockIdx.y + 1) : nxb;
  const uint32_t tx_bytes = (uint32_t)(3 * nxl + (SAME ? 0 : 3)) * BOX;
  constexpr uint32_t TCOLS = NT == 1 ? 128 : 256;       // 2 buffers x NT x 64 columns
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nstages * stage_bytes);
  uint64_t* empty = full + nstages;
  uint64_t* tfull = empty + nstages;                    // [2]
  uint64_t* tfree = tfull + 2;                          // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfree + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int group = blockIdx.x, cg = blockIdx.y;
  const int64_t nsub = (m + KS - 1) / KS;
  const int64_t my_subs = (nsub > group) ? (nsub - group + ngroup - 1) / ngroup : 0;
  const int64_t nchunk = (my_subs + DRAIN - 1) / DRAIN;
  if (tid == 0) {
    for (int s = 0; s < nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tfree[b], NEPI);
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, TCOLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 0) {
    if (lane == 0) {
      for (int64_t it = 0; it < my_subs; ++it) {
        const int s = (int)(it % nstages);
        if (!tc::mbar_wait(&empty[s], (uint32_t)(((it / nstages) & 1) ^ 1), dev_err, abort_flag)) break;
        unsigned char* st = smem + (size_t)s * stage_bytes;
        const int64_t r0 = (group + it * ngroup) * KS;
        tc::mbar_arrive_expect_tx(&full[s], tx_bytes);
        for (int sl = 0; sl < 3; ++sl) {
          const int32_t y = (int32_t)(sl * plane_rows + r0);
          for (int j = 0; j < nxl; ++j)
            tc::tma_load_2d(st + (size_t)(sl * nxb + j) * BOX, &tmX, &full[s], x0 + 64 * j, y);
          if (!SAME) tc::tma_load_2d(st + (size_t)(3 * nxb + sl) * BOX, &tmY, &full[s], y0 + 64 * cg, y);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_make(1u, 1u, 1u, 128u, 64u);
      // slice pairs (a, b) with a + b <= 4 (1-based): (1,1) (1,2) (2,1) (1,3) (2,2) (3,1),
      // 0-based, one nibble per pair
      constexpr uint32_t PA = 0x210100u, PB = 0x012010u;
      int64_t it = 0;
      bool ok = true;
      for (int64_t c = 0; c < nchunk && ok; ++c) {
        const int b = (int)(c & 1);
        if (!tc::mbar_wait(&tfree[b], (uint32_t)(((c >> 1) & 1) ^ 1), dev_err, abort_flag)) break;
        tc::tc_fence_after();
        const int64_t it_end = (it + DRAIN < my_subs) ? it + DRAIN : my_subs;
        for (bool first = true; it < it_end; ++it, first = false) {
          const int s = (int)(it % nstages);
          if (!tc::mbar_wait(&full[s], (uint32_t)((it / nstages) & 1), dev_err, abort_flag)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t sa = tc::smem_u32(smem + (size_t)s * stage_bytes);
          const uint32_t ybase = SAME ? sa + cg * BOX : sa + 3 * nxb * BOX;
          const uint32_t ystride = SAME ? nxb * BOX : BOX;   // bytes between slices of Y
          // one descriptor per slice and operand; every MMA of the stage is
          // a compile-time offset from these (cheap issue)
          const uint64_t a0 = tc::sdesc_sw128(sa, BOX, 1024);
          const uint64_t aS[3] = {a0, tc::sdesc_add(a0, nxb * BOX), tc::sdesc_add(a0, 2 * nxb * BOX)};
          const uint64_t b0 = tc::sdesc_sw128(ybase, BOX, 1024);
          const uint64_t bS[3] = {b0, tc::sdesc_add(b0, ystride), tc::sdesc_add(b0, 2 * ystride)};
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            if (2 * t >= nxl) continue;                    // below the loaded boxes (upper)
            const uint32_t d = tmem + (uint32_t)(b * NT + t) * 64u;
#pragma unroll
            for (int kk = 0; kk < KS / 16; ++kk) {
#pragma unroll
              for (int pr = 0; pr < 6; ++pr) {
                const int a = (int)((PA >> (4 * pr)) & 0xFu), bsl = (int)((PB >> (4 * pr)) & 0xFu);
                tc::mma_f16(d, tc::sdesc_add(aS[a], t * 2 * BOX + kk * 2048), tc::sdesc_add(bS[bsl], kk * 2048),
                            idesc, (!first || kk > 0 || pr > 0) ? 1u : 0u);
              }
            }
          }
          tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(&tfull[b]);
      }
    }
  } else {
    // epilogue: warp 2 + e reads TMEM lane quadrant (warp % 4) of tile
    // t = e / G_EPI_WARPS_PER_T, columns [cs, cs + G_EC) of the 64-wide group
    const int e = warp - 2;
    const int t = e / G_EPI_WARPS_PER_T;
    const int cs = ((e % G_EPI_WARPS_PER_T) >> 2) * G_EC;
    const int quad = warp & 3;
    const int row = t * 128 + quad * 32 + lane;        // X column = row of C
    float acc[G_EC];
#pragma unroll
    for (int j = 0; j < G_EC; ++j) acc[j] = 0.f;
    bool ok = true;
    for (int64_t c = 0; c < nchunk; ++c) {
      const int b = (int)(c & 1);
      ok = tc::mbar_wait(&tfull[b], (uint32_t)((c >> 1) & 1), dev_err, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc::tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * NT + t) * 64u + cs;
#pragma unroll
      for (int piece = 0; piece < G_EC / 16; ++piece) {
        float v[16];
        tc::tmem_ld16(taddr + 16 * piece, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[16 * piece + j] += v[j];
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tfree[b]);
    }
    if (ok && row < p && row < 64 * nxl) {
      const int c0 = cg * 64 + cs;
#pragma unroll
      for (int j = 0; j < G_EC; ++j)
        if (c0 + j < q) atomicAdd(&C[(int64_t)row * ldc + c0 + j], (double)acc[j]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

// ----------------------------------------------------------------- apply
// Y[r, :] = beta Y[r, :] + alpha X[r, :] M for 128-row tiles (persistent).
// A operand: X tile, K-major (row-major X, K = p columns); each pipeline
// stage holds one 32-column K box of the tile, hi and lo (2 x 16 KB).
// B operand: M^T (N = q rows, K = p), hi and lo, K-major, resident in shared
// memory: kb = ceil(p/32) boxes of nq rows x 32 columns.  TMEM holds two
// accumulators (nq columns each) so the drain of one tile overlaps the MMAs
// of the next.
constexpr int A_THREADS = 192;     // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
__global__ void __launch_bounds__(A_THREADS, 1)
k_apply_tf32x3(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmXl, int64_t m,
               int p, int q, int nq, int kb, int nstages, const float* __restrict__ Mt,
               const float* __restrict__ Mtl, float alpha, float beta, float* Y, int64_t ldy, float* Ylo,
               int64_t ldyl, uint32_t* __restrict__ dev_err, const uint32_t* __restrict__ active) {
  if (active && *active == 0u) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t XBOX = 128 * 128;           // 128 rows x 32 FP32
  constexpr uint32_t STAGE = 2 * XBOX;           // hi + lo
  const uint32_t mbox = (uint32_t)nq * 128;      // nq rows x 32 FP32
  unsigned char* mh = smem;
  unsigned char* ml = mh + (size_t)kb * mbox;
  unsigned char* stages = ml + (size_t)kb * mbox;
  uint64_t* full = reinterpret_cast<uint64_t*>(stages + (size_t)nstages * STAGE);
  uint64_t* empty = full + nstages;
  uint64_t* afull = empty + nstages;   // [2] accumulator ready
  uint64_t* aempty = afull + 2;        // [2] accumulator drained
  uint64_t* done = aempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntile = (m + 127) / 128;
  const int64_t my_tiles = (ntile > blockIdx.x) ? (ntile - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t steps = my_tiles * kb;
  const uint32_t tcols = (2 * nq <= 64) ? 64 : (2 * nq <= 128) ? 128 : (2 * nq <= 256) ? 256 : 512;

  // resident M^T (hi, lo) in the K-major SW128 layout: element (n, k) of box
  // k/32 at row n, 16-byte chunk (k%32)/4 XOR (n%8)
  for (int e = tid; e < kb * nq * 32; e += blockDim.x) {
    const int bx = e / (nq * 32), rem = e % (nq * 32), n = rem / 32, kk = rem % 32;
    const int k = bx * 32 + kk;
    const float vh = (n < q && k < p) ? Mt[(int64_t)n * p + k] : 0.f;
    const float vl = (n < q && k < p) ? Mtl[(int64_t)n * p + k] : 0.f;
    const uint32_t off = (uint32_t)bx * mbox + n * 128 + ((((kk >> 2) ^ (n & 7))) << 4) + (kk & 3) * 4;
    *reinterpret_cast<float*>(mh + off) = vh;
    *reinterpret_cast<float*>(ml + off) = vl;
  }
  tc::fence_proxy_async_smem();
  if (tid == 0) {
    for (int s = 0; s < nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int x = 0; x < 2; ++x) {
      tc::mbar_init(&afull[x], 1);
      tc::mbar_init(&aempty[x], 4);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, tcols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;
      for (; g < steps; ++g) {
        const int s = (int)(g % nstages);
        if (!tc::mbar_wait(&empty[s], (uint32_t)(((g / nstages) & 1) ^ 1), dev_err, abort_flag)) break;
        unsigned char* st = stages + (size_t)s * STAGE;
        const int64_t tl = g / kb;
        const int bx = (int)(g % kb);
        const int32_t r0 = (int32_t)((blockIdx.x + tl * gridDim.x) * 128);
        tc::mbar_arrive_expect_tx(&full[s], STAGE);
        tc::tma_load_2d(st, &tmX, &full[s], 32 * bx, r0);
        tc::tma_load_2d(st + XBOX, &tmXl, &full[s], 32 * bx, r0);
      }
      for (int64_t h = (g > nstages ? g - nstages : 0); h < g; ++h) {
        volatile int never = 0;
        tc::mbar_wait(&full[h % nstages], (uint32_t)((h / nstages) & 1), nullptr, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_make(2u, 0u, 0u, 128u, (uint32_t)nq);
      const uint32_t mha = tc::smem_u32(mh), mla = tc::smem_u32(ml);
      for (int64_t g = 0; g < steps; ++g) {
        const int s = (int)(g % nstages);
        const int64_t tl = g / kb;
        const int bx = (int)(g % kb);
        const int x = (int)(tl & 1);
        if (!tc::mbar_wait(&full[s], (uint32_t)((g / nstages) & 1), dev_err, abort_flag)) break;
        if (bx == 0 && !tc::mbar_wait(&aempty[x], (uint32_t)(((tl >> 1) & 1) ^ 1), dev_err, abort_flag)) break;
        tc::tc_fence_after();
        const uint32_t sa = tc::smem_u32(stages + (size_t)s * STAGE);
        const uint32_t d = tmem + x * nq;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ah = tc::sdesc_sw128(sa + kk * 32, 16, 1024);
          const uint64_t al = tc::sdesc_sw128(sa + XBOX + kk * 32, 16, 1024);
          const uint64_t bh = tc::sdesc_sw128(mha + bx * mbox + kk * 32, 16, 1024);
          const uint64_t bl = tc::sdesc_sw128(mla + bx * mbox + kk * 32, 16, 1024);
          tc::mma_tf32(d, ah, bh, idesc, (bx > 0 || kk > 0) ? 1u : 0u);
          tc::mma_tf32(d, ah, bl, idesc, 1u);
          tc::mma_tf32(d, al, bh, idesc, 1u);
        }
        tc::mma_commit(&empty[s]);
        if (bx == kb - 1) tc::mma_commit(&afull[x]);
      }
      tc::mma_commit(done);
    }
  } else {
    // drain through a per-warp staging tile so that rows are written with
    // coalesced 128-byte segments (lane = column)
    float* stg = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(tmem_slot) + 16) +
                 (warp - 2) * 32 * 33;
    const int rbase = 32 * (warp & 3);
    for (int64_t tl = 0; tl < my_tiles; ++tl) {
      const int x = (int)(tl & 1);
      bool ok = tc::mbar_wait(&afull[x], (uint32_t)((tl >> 1) & 1), dev_err, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc::tc_fence_after();
      const int64_t r0 = (blockIdx.x + tl * gridDim.x) * 128 + rbase;
      for (int c32 = 0; c32 < nq; c32 += 32) {
        float v[16];
        tc::tmem_ld16(tmem + x * nq + ((uint32_t)rbase << 16) + c32, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) stg[lane * 33 + j] = v[j];
        if (c32 + 16 < nq) {
          tc::tmem_ld16(tmem + x * nq + ((uint32_t)rbase << 16) + c32 + 16, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) stg[lane * 33 + 16 + j] = v[j];
        }
        __syncwarp();
        const int c = c32 + lane;
        float yold[32];
        if (beta != 0.f) {
          // issue all loads of the old values before any store
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t r = r0 + rr;
            yold[rr] = (r < m && c < q) ? Y[r * ldy + c] : 0.f;
          }
        }
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
          const int64_t r = r0 + rr;
          if (r < m && c < q) {
            float y = alpha * stg[rr * 33 + lane];
            if (beta != 0.f) y += beta * yold[rr];
            Y[r * ldy + c] = y;
            if (Ylo) Ylo[r * ldyl + c] = y - tf32_trunc(y);
          }
        }
        __syncwarp();
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&aempty[x]);
    }
  }
  __syncwarp();
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done, 0, nullptr, &never);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, tcols);
}

// M (p x q FP64, ldm) -> M^T hi (q x p FP32) and lo.
__global__ void k_mt_split(int p, int q, const double* __restrict__ M, int64_t ldm, float* __restrict__ Mt,
                           float* __restrict__ Mtl) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * q) return;
  int n = e / p, k = e % p;
  double v = M[(int64_t)k * ldm + n];
  float h = (float)v;
  float hh = tf32_trunc(h);
  Mt[e] = h;
  Mtl[e] = (float)(v - (double)hh);
}

int g_sms_qr = 0;
constexpr size_t kStageBytes = 4 * 32 * 33 * 4;   // apply epilogue staging

}  // namespace

// ====================================================================== host
void split_lo(int64_t rows, int cols, const float* X, int64_t ldx, float* Xlo, int64_t ldl, cudaStream_t st) {
  int64_t cnt = rows * cols;
  if (cnt <= 0) return;
  k_split_lo<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(rows, cols, X, ldx, Xlo, ldl);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void slice3(int64_t rows, int64_t plane_rows, int cols, const float* X, int64_t ldx, void* S, cudaStream_t st,
            const uint32_t* active) {
  const int ldS = (int)round_up(cols, 64);
  int64_t cnt = plane_rows * ldS / 4;
  if (cnt <= 0) return;
  k_slice3<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(rows, plane_rows, cols, ldS, X, ldx,
                                                     static_cast<__nv_bfloat16*>(S), active);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

bool gram_tc(int64_t m, int p, int q, const float* X, int64_t ldx, const float* Y, int64_t ldy, double* C,
             int64_t ldc, void* slices, size_t slice_bytes, cudaStream_t st, uint32_t* dev_err,
             const uint32_t* active, bool reslice_x) {
  if (p > 256 || q > 256 || m < 256 || !slices) return false;
  const bool same = (X == Y && p == q && ldx == ldy);
  const int NT = (p > 128) ? 2 : 1;
  const int ncg = (int)cdiv(q, 64);                  // 64-column groups of C
  const int ldX = (int)round_up(p, 64), ldY = (int)round_up(q, 64);
  const int64_t prow = round_up(m, G_KSUB);
  const size_t need = (size_t)3 * prow * 2 * (ldX + (same ? 0 : ldY));
  if (need > slice_bytes) return false;
  __nv_bfloat16* SX = static_cast<__nv_bfloat16*>(slices);
  __nv_bfloat16* SY = same ? SX : SX + (size_t)3 * prow * ldX;
  CUtensorMap tX, tY;
  if (!make_tmap_2d(&tX, SX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 3 * prow, ldX, ldX, G_KSUB, 64)) return false;
  if (!make_tmap_2d(&tY, SY, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 3 * prow, ldY, ldY, G_KSUB, 64)) return false;
  const uint32_t box = G_KSUB * 128;
  const int nxb = (int)cdiv(p, 64);
  const uint32_t stage_bytes = (uint32_t)(3 * nxb + (same ? 0 : 3) + 1) * box;
  const int nstages = (int)std::min<int64_t>(6, (200 * 1024) / stage_bytes);
  if (nstages < 2) return false;
  if (reslice_x || same) slice3(m, prow, p, X, ldx, SX, st, active);
  if (!same) slice3(m, prow, q, Y, ldy, SY, st, active);
  const size_t smem = 1024 + (size_t)nstages * stage_bytes + (2 * nstages + 4) * 8 + 16;
  if (!g_sms_qr) g_sms_qr = num_sms();
  const int ngroup =
      (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(m, G_KSUB), std::max(1, g_sms_qr / ncg)));
  RPCA_CUDA_TRY(cudaMemset2DAsync(C, ldc * 8, 0, q * 8, p, st));
  auto launch = [&](auto kern) {
    RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3(ngroup, ncg), 64 + 32 * G_EPI_WARPS_PER_T * NT, smem, st>>>(
        tX, tY, m, prow, 0, 0, p, q, nxb, ngroup, nstages, stage_bytes, C, ldc, dev_err, active, 0);
    RPCA_CUDA_TRY(cudaGetLastError());
  };
  if (NT == 2) {
    if (same) launch(k_gram_bf16x3<2, true, G_KSUB>);
    else launch(k_gram_bf16x3<2, false, G_KSUB>);
  } else {
    if (same) launch(k_gram_bf16x3<1, true, G_KSUB>);
    else launch(k_gram_bf16x3<1, false, G_KSUB>);
  }
  count_launch();
  return true;
}

bool gram_slices(int64_t m, int64_t plane_rows, const void* S, int lds, int x0, int p, int y0, int q, double* C,
                 int64_t ldc, cudaStream_t st, uint32_t* dev_err, const uint32_t* active, bool upper) {
  if (p > 256 || q > 256 || (x0 & 63) || (y0 & 63) || plane_rows % 128) return false;
  const bool same = (x0 == y0 && p == q);
  if (upper && !same) return false;
  const int NT = (p > 128) ? 2 : 1;
  const int ncg = (int)cdiv(q, 64);
  const int nxb = (int)cdiv(p, 64);
  // deepest row box that leaves at least three stages (else two)
  const int nbox = 3 * nxb + (same ? 0 : 3) + 1;
  int ks = 32;
  for (int cand : {128, 64, 32}) {
    if ((size_t)3 * nbox * cand * 128 <= 200 * 1024) { ks = cand; break; }
  }
  if ((size_t)2 * nbox * ks * 128 > 200 * 1024) return false;
  const uint32_t stage_bytes = (uint32_t)nbox * ks * 128;
  const int nstages = (int)std::min<int64_t>(6, (200 * 1024) / stage_bytes);
  CUtensorMap tS;
  if (!make_tmap_2d(&tS, S, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 3 * plane_rows, lds, lds, (uint32_t)ks, 64))
    return false;
  const size_t smem = 1024 + (size_t)nstages * stage_bytes + (2 * nstages + 4) * 8 + 16;
  if (!g_sms_qr) g_sms_qr = num_sms();
  const int ngroup = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(m, ks), std::max(1, g_sms_qr / ncg)));
  RPCA_CUDA_TRY(cudaMemset2DAsync(C, ldc * 8, 0, q * 8, p, st));
  auto launch = [&](auto kern) {
    RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3(ngroup, ncg), 64 + 32 * G_EPI_WARPS_PER_T * NT, smem, st>>>(
        tS, tS, m, plane_rows, x0, y0, p, q, nxb, ngroup, nstages, stage_bytes, C, ldc, dev_err, active,
        upper ? 1 : 0);
    RPCA_CUDA_TRY(cudaGetLastError());
  };
  auto pick_ks = [&](auto nt, auto sm) {
    constexpr int NTc = decltype(nt)::value;
    constexpr bool SMc = decltype(sm)::value;
    if (ks == 128) launch(k_gram_bf16x3<NTc, SMc, 128>);
    else if (ks == 64) launch(k_gram_bf16x3<NTc, SMc, 64>);
    else launch(k_gram_bf16x3<NTc, SMc, 32>);
  };
  using T1 = std::integral_constant<int, 1>;
  using T2 = std::integral_constant<int, 2>;
  using S1 = std::integral_constant<bool, true>;
  using S0 = std::integral_constant<bool, false>;
  if (NT == 2) {
    if (same) pick_ks(T2{}, S1{});
    else pick_ks(T2{}, S0{});
  } else {
    if (same) pick_ks(T1{}, S1{});
    else pick_ks(T1{}, S0{});
  }
  count_launch();
  return true;
}

bool apply_tc(int64_t m, int p, int q, const float* X, const float* Xlo, int64_t ldx, const double* M,
              int64_t ldm, double alpha, double beta, float* Y, float* Ylo, int64_t ldy, float* scratch,
              cudaStream_t st, uint32_t* dev_err, const uint32_t* active) {
  if (p > 256 || q > 256 || m < 128) return false;
  const int nq = (int)round_up(q, 16);
  const int kb = (int)cdiv(p, 32);
  const uint32_t mbox = (uint32_t)nq * 128;
  const size_t mres = 2 * (size_t)kb * mbox;
  const size_t stage = 2 * 128 * 128;
  const size_t budget = 227 * 1024 - 1024 - 256 - kStageBytes;
  if (mres + 2 * stage > budget || 2 * nq > 512) return false;
  const int nstages = (int)std::min<size_t>(6, (budget - mres) / stage);
  CUtensorMap tX, tXl;
  if (!make_tmap_2d(&tX, X, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, m, p, ldx, 128, 32)) return false;
  if (!make_tmap_2d(&tXl, Xlo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, m, p, ldx, 128, 32)) return false;
  float* Mt = scratch;
  float* Mtl = scratch + (size_t)p * q;
  k_mt_split<<<(unsigned)cdiv((int64_t)p * q, 256), 256, 0, st>>>(p, q, M, ldm, Mt, Mtl);
  RPCA_CUDA_TRY(cudaGetLastError());
  const size_t smem = 1024 + mres + (size_t)nstages * stage + (2 * nstages + 5) * 8 + 16 + kStageBytes;
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_apply_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (!g_sms_qr) g_sms_qr = num_sms();
  const int64_t ntile = cdiv(m, 128);
  const unsigned grid = (unsigned)std::min<int64_t>(ntile, g_sms_qr);
  k_apply_tf32x3<<<grid, A_THREADS, smem, st>>>(tX, tXl, m, p, q, nq, kb, nstages, Mt, Mtl, (float)alpha,
                                                (float)beta, Y, ldy, Ylo, ldy, dev_err, active);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch(2);
  return true;
}

}  // namespace rpca
