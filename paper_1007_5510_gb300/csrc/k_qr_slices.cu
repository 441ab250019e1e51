// Step 2 (QR of H) and the products of Steps 3 and 5 on H held as three
// exact BF16 slices.
//
// Every FP32 value x of H is stored as x1 + x2 + x3 with x1 = RNE_bf16(x),
// x2 = RNE_bf16(x - x1), x3 = x - x1 - x2 (each exact in 8 significant bits),
// in three stacked planes of plane_rows x lds BF16.  Block j of H (l <= 64
// columns) occupies the 64-column box [64j, 64j + 64) with zero padding, so
// every TMA coordinate is 16-byte aligned.  Products with six slice pairs
// (a + b <= 4, 1-based) are FP32-accurate (~2^-24 relative); the tensor
// cores read the slices directly, so no FP32 copy or remainder array is
// streamed.  Slice 1 is RNE_bf16(Q) itself: the BF16 operand of the T pass.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rpca {
namespace {

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// H (m x nblk*l FP32, ld) -> three planes, block-padded; rows [m, plane_rows)
// and padding columns are zero.  Four output columns per thread.
__global__ void k_slice3_blocks(int64_t m, int64_t plane_rows, int nblk, int l, const float* __restrict__ H,
                                int64_t ld, __nv_bfloat16* __restrict__ S) {
  const int lds = nblk * 64;
  const int64_t e4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int per_row = lds / 4;
  if (e4 >= plane_rows * per_row) return;
  const int64_t r = e4 / per_row;
  const int oc = (int)(e4 % per_row) * 4;
  const int blk = oc >> 6;
  __nv_bfloat16 o1[4], o2[4], o3[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jc = (oc & 63) + q;
    const float x = (r < m && jc < l) ? H[r * ld + blk * l + jc] : 0.f;
    split3(x, o1[q], o2[q], o3[q]);
  }
  const int64_t plane = plane_rows * lds;
  const int64_t e = r * lds + oc;
  *reinterpret_cast<uint2*>(S + e) = *reinterpret_cast<uint2*>(o1);
  *reinterpret_cast<uint2*>(S + plane + e) = *reinterpret_cast<uint2*>(o2);
  *reinterpret_cast<uint2*>(S + 2 * plane + e) = *reinterpret_cast<uint2*>(o3);
}

// Slices back to FP32: H[r, blk*l + c] = x1 + x2 + x3 (exact).
__global__ void k_unslice_blocks(int64_t m, int64_t plane_rows, int nblk, int l,
                                 const __nv_bfloat16* __restrict__ S, float* __restrict__ H, int64_t ld) {
  const int w = nblk * l, lds = nblk * 64;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * w) return;
  const int64_t r = e / w;
  const int c = (int)(e % w);
  const int64_t off = r * lds + (c / l) * 64 + c % l;
  const int64_t plane = plane_rows * lds;
  H[r * ld + c] = (__bfloat162float(S[off + 2 * plane]) + __bfloat162float(S[off + plane])) + __bfloat162float(S[off]);
}

// out[c] += sum_r Q[r, c] over a row range, c in block-compact numbering.
__global__ void k_col_sums_slices(int64_t m, int64_t plane_rows, int nblk, int l, const __nv_bfloat16* __restrict__ S,
                                  double* __restrict__ out) {
  const int lds = nblk * 64;
  const int col = blockIdx.y * blockDim.x + threadIdx.x;      // padded column
  if (col >= lds || (col & 63) >= l) return;
  const int64_t plane = plane_rows * lds;
  const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * rows_per, r1 = (r0 + rows_per < m) ? r0 + rows_per : m;
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const int64_t off = r * lds + col;
    s += (double)((__bfloat162float(S[off + 2 * plane]) + __bfloat162float(S[off + plane])) + __bfloat162float(S[off]));
  }
  atomicAdd(&out[(col >> 6) * l + (col & 63)], s);
}

// M^T slices for the B operand (K-major): plane pl, row j (output column,
// j < 64), column kp (K index, kpad = nkb*64 wide) holds slice pl of
// alpha * M[src(kp), j], src(kp) = (kp/64)*rl + kp%64 when rl > 0 (block-
// padded K; kp%64 >= rl are zero), kp when rl == 0 (kp < krows).
__global__ void k_mt_slices(int krows, int q, const double* __restrict__ M, int64_t ldm, double alpha, int rl,
                            int kpad, __nv_bfloat16* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 64 * kpad) return;
  const int j = e / kpad, kp = e % kpad;
  int src = -1;
  if (rl > 0) {
    if ((kp & 63) < rl) src = (kp >> 6) * rl + (kp & 63);
  } else {
    src = kp;
  }
  double v = (j < q && src >= 0 && src < krows) ? alpha * M[(int64_t)src * ldm + j] : 0.0;
  const __nv_bfloat16 s1 = __float2bfloat16_rn((float)v);
  const double r1 = v - (double)__bfloat162float(s1);
  const __nv_bfloat16 s2 = __float2bfloat16_rn((float)r1);
  const double r2 = r1 - (double)__bfloat162float(s2);
  const __nv_bfloat16 s3 = __float2bfloat16_rn((float)r2);
  const int64_t plane = (int64_t)64 * kpad;
  out[(int64_t)j * kpad + kp] = s1;
  out[plane + (int64_t)j * kpad + kp] = s2;
  out[2 * plane + (int64_t)j * kpad + kp] = s3;
}

// C (rows x cols, block-padded indices) -> E (compact w x w).
__global__ void k_compact_sq(int nblk, int l, const double* __restrict__ C, int64_t ldc, double* __restrict__ E) {
  const int w = nblk * l;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= w * w) return;
  const int i = e / w, j = e % w;
  const int pi = (i / l) * 64 + i % l, pj = (j / l) * 64 + j % l;
  // symmetric: the lower block triangle from the upper one
  E[e] = (i / l <= j / l) ? C[(int64_t)pi * ldc + pj] : C[(int64_t)pj * ldc + pi];
}

// ------------------------------------------------------------ sliced apply
// Y (128-row tiles, 64 columns at y0) = beta * Y + X M, with X (nkb boxes of
// 64 columns at x0) and Y in slice planes and M given by its transposed
// slices (resident).  Warp 0 lane 0: TMA; warp 1 lane 0: MMA (six slice
// products per K step into a double-buffered TMEM accumulator pair: the
// hi*hi product in one, the five smaller products in the other, added with
// round-to-nearest in the epilogue -- the tensor cores' accumulation rounds
// with a bias of about one unit in the last place per MMA, so a single
// accumulator taking all six products over K = 192 drifted by ~5e-6
// relative, which showed as a 1e-5 departure from orthonormality of the
// U = Q M product at 1e6 rows); warps 2-5:
// epilogue (one tile row per thread: optional FP32 output, optional beta
// term from the old slices, re-slicing into a shared staging tile that a
// TMA store writes back).
constexpr int AS_THREADS = 192;
constexpr uint32_t AS_XBOX = 128 * 128;     // 128 rows x 64 BF16
constexpr uint32_t AS_MBOX = 64 * 128;      // 64 rows x 64 BF16

__device__ __forceinline__ bool epi4_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi4_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

struct ApplyParams {
  int64_t m, plane_rows;
  int x0, nkb, y0;
  int beta;            // 0 or 1
  int write_slices;    // store the new Y slices
  int nstages;
  float* Yf;           // optional FP32 copy of Y (columns < qf), ld ldf
  int64_t ldf;
  int qf;
  uint32_t* dev_err;
  const uint32_t* active;
};

__global__ void __launch_bounds__(AS_THREADS, 1)
k_apply_bf16x3(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmM,
               const __grid_constant__ CUtensorMap tmY, const ApplyParams p) {
  if (p.active && *p.active == 0u) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* mres = smem;                                            // 3 x nkb M boxes
  unsigned char* stages = mres + (size_t)3 * p.nkb * AS_MBOX;            // nstages x 3 X boxes
  unsigned char* ybuf = stages + (size_t)p.nstages * 3 * AS_XBOX;        // 3 Y boxes
  uint64_t* bars = reinterpret_cast<uint64_t*>(ybuf + 3 * AS_XBOX);
  uint64_t* mfull = bars;
  uint64_t* full = mfull + 1;                    // [nstages]
  uint64_t* empty = full + p.nstages;            // [nstages]
  uint64_t* tfull = empty + p.nstages;           // [2]
  uint64_t* tfree = tfull + 2;                   // [2]
  uint64_t* yfull = tfree + 2;                   // old Y tile loaded (beta)
  uint64_t* yfree = yfull + 1;                   // staging tile free again
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(yfree + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = p.plane_rows / 128;
  const int64_t my_tiles = (ntiles > blockIdx.x) ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (tid == 0) {
    tc::mbar_init(mfull, 1);
    for (int s = 0; s < p.nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tfree[b], 4);
    }
    tc::mbar_init(yfull, 1);
    tc::mbar_init(yfree, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 256);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      tc::mbar_arrive_expect_tx(mfull, 3u * p.nkb * AS_MBOX);
      for (int pl = 0; pl < 3; ++pl)
        for (int kb = 0; kb < p.nkb; ++kb)
          tc::tma_load_2d(mres + (size_t)(pl * p.nkb + kb) * AS_MBOX, &tmM, mfull, 64 * kb, 64 * pl);
      int64_t it = 0;
      bool ok = true;
      for (int64_t ti = 0; ti < my_tiles && ok; ++ti) {
        const int64_t r0 = (blockIdx.x + ti * gridDim.x) * 128;
        for (int kb = 0; kb < p.nkb; ++kb, ++it) {
          const int s = (int)(it % p.nstages);
          if (!tc::mbar_wait(&empty[s], (uint32_t)(((it / p.nstages) & 1) ^ 1), p.dev_err, abort_flag)) {
            ok = false;
            break;
          }
          unsigned char* st = stages + (size_t)s * 3 * AS_XBOX;
          tc::mbar_arrive_expect_tx(&full[s], 3 * AS_XBOX);
          for (int pl = 0; pl < 3; ++pl)
            tc::tma_load_2d(st + (size_t)pl * AS_XBOX, &tmX, &full[s], p.x0 + 64 * kb,
                            (int32_t)(pl * p.plane_rows + r0));
        }
        if (ok && p.beta) {
          // old Y tile, once the previous tile's store has read the staging tile
          if (!tc::mbar_wait(yfree, (uint32_t)((ti & 1) ^ 1), p.dev_err, abort_flag)) break;
          tc::mbar_arrive_expect_tx(yfull, 3 * AS_XBOX);
          for (int pl = 0; pl < 3; ++pl)
            tc::tma_load_2d(ybuf + (size_t)pl * AS_XBOX, &tmY, yfull, p.y0, (int32_t)(pl * p.plane_rows + r0));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // --------------------------------------------------------------- MMA
      constexpr uint32_t idesc = tc::idesc_make(1u, 0u, 0u, 128u, 64u);
      constexpr uint32_t PA = 0x210100u, PB = 0x012010u;   // slice pairs, one nibble each
      const uint32_t ma = tc::smem_u32(mres);
      bool ok = tc::mbar_wait(mfull, 0, p.dev_err, abort_flag);
      int64_t it = 0;
      for (int64_t ti = 0; ti < my_tiles && ok; ++ti) {
        const int b = (int)(ti & 1);
        if (!tc::mbar_wait(&tfree[b], (uint32_t)(((ti >> 1) & 1) ^ 1), p.dev_err, abort_flag)) break;
        tc::tc_fence_after();
        for (int kb = 0; kb < p.nkb; ++kb, ++it) {
          const int s = (int)(it % p.nstages);
          if (!tc::mbar_wait(&full[s], (uint32_t)((it / p.nstages) & 1), p.dev_err, abort_flag)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t sa = tc::smem_u32(stages + (size_t)s * 3 * AS_XBOX);
          // descriptors of the three X slices and the three M slices of this
          // K box; the K steps are compile-time offsets (cheap issue)
          const uint64_t xa = tc::sdesc_sw128(sa, 16, 1024);
          const uint64_t xS[3] = {xa, tc::sdesc_add(xa, AS_XBOX), tc::sdesc_add(xa, 2 * AS_XBOX)};
          const uint64_t mb = tc::sdesc_sw128(ma + kb * AS_MBOX, 16, 1024);
          const uint32_t mstride = (uint32_t)p.nkb * AS_MBOX;
          const uint64_t mS[3] = {mb, tc::sdesc_add(mb, mstride), tc::sdesc_add(mb, 2 * mstride)};
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
              const int a = (int)((PA >> (4 * pr)) & 0xFu), bs = (int)((PB >> (4 * pr)) & 0xFu);
              // accumulator b*128 takes hi*hi, b*128 + 64 the rest
              tc::mma_f16(tmem + b * 128 + (pr == 0 ? 0u : 64u), tc::sdesc_add(xS[a], kk * 32),
                          tc::sdesc_add(mS[bs], kk * 32), idesc, (kb > 0 || kk > 0 || pr > 1) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&tfull[b]);
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int quad = warp & 3;
    const int row = quad * 32 + lane;            // tile row = TMEM lane
    const int e = tid - 64;
    bool ok = true;
    for (int64_t ti = 0; ti < my_tiles; ++ti) {
      const int b = (int)(ti & 1);
      const int64_t r0 = (blockIdx.x + ti * gridDim.x) * 128;
      ok = tc::mbar_wait(&tfull[b], (uint32_t)((ti >> 1) & 1), p.dev_err, abort_flag);
      if (p.beta) ok = ok && tc::mbar_wait(yfull, (uint32_t)(ti & 1), p.dev_err, abort_flag);
      ok = epi4_bar_and(ok);
      if (!ok) break;
      tc::tc_fence_after();
      float acc[64];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * 128u;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float lo[16];
        tc::tmem_ld16(taddr + 16 * g, *reinterpret_cast<float(*)[16]>(&acc[16 * g]));
        tc::tmem_ld16(taddr + 64 + 16 * g, lo);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[16 * g + j] += lo[j];
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tfree[b]);
      unsigned char* yrow = ybuf + (size_t)row * 128;
      if (p.beta) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t off = (uint32_t)((c ^ (row & 7)) << 4);
          const uint4 v1 = *reinterpret_cast<const uint4*>(yrow + off);
          const uint4 v2 = *reinterpret_cast<const uint4*>(yrow + AS_XBOX + off);
          const uint4 v3 = *reinterpret_cast<const uint4*>(yrow + 2 * AS_XBOX + off);
          const __nv_bfloat16* h1 = reinterpret_cast<const __nv_bfloat16*>(&v1);
          const __nv_bfloat16* h2 = reinterpret_cast<const __nv_bfloat16*>(&v2);
          const __nv_bfloat16* h3 = reinterpret_cast<const __nv_bfloat16*>(&v3);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            acc[8 * c + i] += (__bfloat162float(h3[i]) + __bfloat162float(h2[i])) + __bfloat162float(h1[i]);
        }
      }
      const int64_t grow = r0 + row;
      if (p.Yf && grow < p.m) {
        float* yf = p.Yf + grow * p.ldf;
#pragma unroll
        for (int j = 0; j < 64; ++j)
          if (j < p.qf) yf[j] = acc[j];
      }
      if (p.write_slices) {
        epi4_bar();   // every thread is done reading the old tile (beta)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          __nv_bfloat16 s1[8], s2[8], s3[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) split3(acc[8 * c + i], s1[i], s2[i], s3[i]);
          const uint32_t off = (uint32_t)((c ^ (row & 7)) << 4);
          *reinterpret_cast<uint4*>(yrow + off) = *reinterpret_cast<const uint4*>(s1);
          *reinterpret_cast<uint4*>(yrow + AS_XBOX + off) = *reinterpret_cast<const uint4*>(s2);
          *reinterpret_cast<uint4*>(yrow + 2 * AS_XBOX + off) = *reinterpret_cast<const uint4*>(s3);
        }
        tc::fence_proxy_async_smem();
        epi4_bar();
        if (e == 0) {
          for (int pl = 0; pl < 3; ++pl)
            tc::tma_store_2d(&tmY, ybuf + (size_t)pl * AS_XBOX, p.y0, (int32_t)(pl * p.plane_rows + r0));
          tc::bulk_commit();
          tc::bulk_wait_read0();     // the staging tile may be refilled
          if (p.beta) tc::mbar_arrive(yfree);
        }
        epi4_bar();
      } else if (p.beta) {
        epi4_bar();
        if (e == 0) tc::mbar_arrive(yfree);
      }
    }
    if (e == 0) tc::bulk_wait0();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

int g_sms_sl = 0;

}  // namespace

// ------------------------------------------------------------------- host
void slice_blocks(int64_t m, int64_t plane_rows, int nblk, int l, const float* H, int64_t ld, void* S,
                  cudaStream_t st) {
  const int64_t cnt = plane_rows * (nblk * 64 / 4);
  k_slice3_blocks<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(m, plane_rows, nblk, l, H, ld,
                                                            static_cast<__nv_bfloat16*>(S));
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void unslice_blocks(int64_t m, int64_t plane_rows, int nblk, int l, const void* S, float* H, int64_t ld,
                    cudaStream_t st) {
  const int64_t cnt = m * nblk * l;
  k_unslice_blocks<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(m, plane_rows, nblk, l,
                                                             static_cast<const __nv_bfloat16*>(S), H, ld);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void col_sums_slices(int64_t m, int64_t plane_rows, int nblk, int l, const void* S, double* out, cudaStream_t st) {
  RPCA_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)nblk * l * sizeof(double), st));
  dim3 grid((unsigned)std::min<int64_t>(512, cdiv(m, 256)), (unsigned)cdiv(nblk * 64, 64));
  k_col_sums_slices<<<grid, 64, 0, st>>>(m, plane_rows, nblk, l, static_cast<const __nv_bfloat16*>(S), out);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void compact_sq(int nblk, int l, const double* C, int64_t ldc, double* E, cudaStream_t st) {
  const int w = nblk * l;
  k_compact_sq<<<(unsigned)cdiv((int64_t)w * w, 256), 256, 0, st>>>(nblk, l, C, ldc, E);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

bool apply_slices(int64_t m, int64_t plane_rows, void* S, int lds, int x0, int nkb, int y0, const double* M,
                  int krows, int q, int64_t ldm, double alpha, int rl, bool beta, bool write_slices, float* Yf,
                  int64_t ldf, int qf, void* mt, cudaStream_t st, uint32_t* dev_err, const uint32_t* active) {
  if (nkb < 1 || nkb > 3 || q > 64 || plane_rows % 128 || (x0 & 63) || (y0 & 63)) return false;
  const int kpad = nkb * 64;
  __nv_bfloat16* MT = static_cast<__nv_bfloat16*>(mt);   // 3 x 64 x kpad
  k_mt_slices<<<(unsigned)cdiv(64 * kpad, 256), 256, 0, st>>>(krows, q, M, ldm, alpha, rl, kpad, MT);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
  CUtensorMap tX, tM;
  if (!make_tmap_2d(&tX, S, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 3 * plane_rows, lds, lds, 128, 64)) return false;
  if (!make_tmap_2d(&tM, MT, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, 3 * 64, kpad, kpad, 64, 64)) return false;
  ApplyParams p;
  p.m = m;
  p.plane_rows = plane_rows;
  p.x0 = x0;
  p.nkb = nkb;
  p.y0 = y0;
  p.beta = beta ? 1 : 0;
  p.write_slices = write_slices ? 1 : 0;
  p.Yf = Yf;
  p.ldf = ldf;
  p.qf = qf;
  p.dev_err = dev_err;
  p.active = active;
  const size_t fixed = 1024 + (size_t)3 * nkb * AS_MBOX + 3 * AS_XBOX + 256;
  p.nstages = (int)std::min<size_t>(3, (227 * 1024 - fixed) / (3 * AS_XBOX));
  if (p.nstages < 2) return false;
  const size_t smem = fixed + (size_t)p.nstages * 3 * AS_XBOX;
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_apply_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (!g_sms_sl) g_sms_sl = num_sms();
  const int64_t ntiles = plane_rows / 128;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, g_sms_sl));
  k_apply_bf16x3<<<grid, AS_THREADS, smem, st>>>(tX, tM, tX, p);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
  return true;
}

}  // namespace rpca
