// Grouped kernels for batches of independent PCAs (BF16 storage).
//
// Every step of Section 3 runs once for all problems of a batch: one launch
// walks a work list of (problem, tile) items, so a batch of hundreds of
// uneven problems costs about a dozen launches instead of hundreds per
// problem.  Steps per run (block Lanczos form of Step 1, as in the
// single-problem path):
//   k_grp_hpass   H^(j) = A X^(j)       tcgen05, persistent, 128-row tiles
//   k_grp_tpass   F = A^T bf16(H^(j)),  T = A^T bf16(Q1)
//                                       tcgen05, (problem, row range) items
//                                       over all columns, FP32 reductions
//   k_grp_orth    X^(j+1) = orth(F - X X^T F) (twice), Householder in
//                 shared memory, one CTA per problem
//   k_grp_rows    H^T H, Q1 = H R1^-1, T1^T T1, U (FP32 register tiles,
//                 FP64 Gram totals)
//   k_grp_chol    Cholesky and triangular inverse (FP64), one CTA per problem
//   k_grp_apply   Q1 = H R1^-1 rows (over H) -> bf16(Q1) and Q1^T Q1
//   k_grp_eig     G_T = R2^-T (T1^T T1) R2^-1, its Cholesky factor R_T,
//                 one-sided Jacobi on R_T, S and V, and M_U = R2^-1 W_k
//   k_grp_u       U = Q1 M_U
// Step 2 is a Cholesky QR of H repeated once on Q1 = H R1^-1 (CholQR2), but
// the second factor R2 is never applied to the m-side data: T = A^T Q with
// Q = Q1 R2^-1 is T1 R2^-1 and U = Q1 R2^-1 W_k.
//
// Layouts (per problem p, all packed into a few device buffers):
//   A_p     m x n BF16 row-major, ld a multiple of 8 (TMA)
//   H_p     m x w FP32 (ld w); Z_p m x 64 BF16 (bf16(H^(j)) or bf16(Q1),
//           columns past l or w zero)
//   XT_p    32 x n64 BF16: X^(j)^T in the 128-byte-swizzled K-major layout
//           of the H pass's B operand, one 4 KB image per 64 rows of X
//   X_p     n x w FP32 (ld w): the blocks X^(0..i)
//   F_p     n x ldy FP32, T_p n x ldy FP32 (ldy = round_up(N, 4))
// Every wait is bounded (tc_common.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "grouped.h"
#include "tc_common.cuh"

namespace rpca {
namespace grp {

// ------------------------------------------------------------- helpers
// Named barrier 1 over the four epilogue warps (128 threads).
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ bool epi_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// Four FP32 reductions into 16-byte-aligned global memory.
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// ======================================================= H pass (tcgen05)
// H[:, j*l : j*l + l] = A X^(j) for every 128-row tile of every problem.
// Warp 0 lane 0: TMA (A tiles as two 64-row boxes of 64 columns; X^(j)^T as
// bulk copies of its pre-swizzled images, once per problem change); warp 1
// lane 0: MMA (M = 128, N = 32, K = 16 steps) into a double-buffered TMEM
// accumulator; warps 2-5: epilogue (thread = tile row).
constexpr int HP_THREADS = 192;
constexpr int HP_KPS = 2;                    // 64-column steps per ring stage
constexpr uint32_t HP_KCHUNK = 128 * 128;    // 128 rows x 64 BF16 (two 64-row boxes)
constexpr uint32_t HP_STAGE = HP_KPS * HP_KCHUNK;   // 256 contiguous bytes of each row
constexpr uint32_t HP_XCHUNK = 32 * 128;     // 32 rows x 64 BF16
constexpr uint32_t HP_ZSTAGE = 128 * 128;    // epilogue staging of 128 Z rows
constexpr int HP_HPITCH = 33;                // odd pitch (floats) of the H staging rows (l <= 32)

__global__ void __launch_bounds__(HP_THREADS, 1)
k_grp_hpass(const GrpProblem* __restrict__ probs, const int32_t* __restrict__ item_p,
            const int32_t* __restrict__ item_t, int64_t nitems, HPassArgs a) {
  // item_t[q]: row tile (low 24 bits) | 64-column steps of the problem (high 8)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xs = smem;                                        // X^T images (a.xbytes)
  unsigned char* ring = xs + a.xbytes;                             // nstages x HP_STAGE
  unsigned char* zst = ring + (size_t)a.nstages * HP_STAGE;        // 128 x 128 B: Z rows (swizzled)
  float* hst = reinterpret_cast<float*>(zst + HP_ZSTAGE);          // 128 x (l | 1): H rows
  uint64_t* full = reinterpret_cast<uint64_t*>(hst + 128 * HP_HPITCH);
  uint64_t* empty = full + a.nstages;
  uint64_t* tfull = empty + a.nstages;   // [2]
  uint64_t* tfree = tfull + 2;           // [2]
  uint64_t* xfull = tfree + 2;
  uint64_t* xfree = xfull + 1;
  uint64_t* done = xfree + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  if (__syncthreads_or((*(volatile uint32_t*)a.err & DEV_ERR_TIMEOUT) != 0)) return;   // an earlier step gave up
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t q0 = nitems * blockIdx.x / gridDim.x;
  const int64_t q1 = nitems * (blockIdx.x + 1) / gridDim.x;

  if (tid == 0) {
    for (int s = 0; s < a.nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tfree[b], 4);
    }
    tc::mbar_init(xfull, 1);
    tc::mbar_init(xfree, 1);
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 64);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      int prev = -1;
      int64_t it = 0, nsw = 0;   // ring stages issued, problem switches
      bool ok = true;
      // L2 prefetch cursor a.pf stages ahead of the loads
      int64_t pq = q0;
      int pkb = 0;
      auto prefetch_next = [&]() {
        if (pq >= q1) return;
        const int pp = item_p[pq];
        const uint32_t pw = (uint32_t)item_t[pq];
        const int32_t py = (int32_t)(pw & 0xffffffu) * 128;
        tc::tma_prefetch_l2_2d(&a.tmA[pp], 64 * pkb, py);
        tc::tma_prefetch_l2_2d(&a.tmA[pp], 64 * pkb, py + 64);
        if (++pkb == (int)(pw >> 24)) {
          pkb = 0;
          ++pq;
        }
      };
      for (int i = 0; i < a.pf; ++i) prefetch_next();
      // item words read one tile ahead (their latency overlaps the tile)
      int p_nx = q0 < q1 ? item_p[q0] : 0;
      uint32_t t_nx = q0 < q1 ? (uint32_t)item_t[q0] : 0u;
      for (int64_t q = q0; q < q1 && ok; ++q) {
        const int p = p_nx;
        const uint32_t tw = t_nx;
        if (q + 1 < q1) {
          p_nx = item_p[q + 1];
          t_nx = (uint32_t)item_t[q + 1];
        }
        if (p != prev) {
          const GrpProblem& P = probs[p];
          if (nsw > 0 && !tc::mbar_wait(xfree, (uint32_t)((nsw - 1) & 1), a.err, abort_flag)) break;
          const unsigned char* src = reinterpret_cast<const unsigned char*>(a.xt_first ? P.XT0 : P.XT);
          const uint32_t xb = (tw >> 24) * HP_XCHUNK;
          tc::mbar_arrive_expect_tx(xfull, xb);
          for (uint32_t off = 0; off < xb; off += HP_XCHUNK) tc::bulk_load_1d(xs + off, src + off, HP_XCHUNK, xfull);
          ++nsw;
          prev = p;
        }
        const int32_t y0 = (int32_t)(tw & 0xffffffu) * 128;
        const int nk = (int)(tw >> 24);
        for (int kb0 = 0; kb0 < nk; kb0 += HP_KPS, ++it) {
          const int nc = min(HP_KPS, nk - kb0);
          const int s = (int)(it % a.nstages);
          if (!tc::mbar_wait(&empty[s], (uint32_t)(((it / a.nstages) & 1) ^ 1), a.err, abort_flag)) {
            ok = false;
            break;
          }
          unsigned char* st = ring + (size_t)s * HP_STAGE;
          tc::mbar_arrive_expect_tx(&full[s], (uint32_t)nc * HP_KCHUNK);
          for (int c = 0; c < nc; ++c) {
            tc::tma_load_2d(st + (size_t)c * HP_KCHUNK, &a.tmA[p], &full[s], 64 * (kb0 + c), y0);
            tc::tma_load_2d(st + (size_t)c * HP_KCHUNK + HP_KCHUNK / 2, &a.tmA[p], &full[s], 64 * (kb0 + c), y0 + 64);
          }
          if (a.pf > 0)
            for (int c = 0; c < nc; ++c) prefetch_next();
        }
      }
      // after an abort, the copies still in flight land before the CTA exits
      volatile int never = 0;
      for (int64_t jt = (it > a.nstages ? it - a.nstages : 0); jt < it; ++jt)
        tc::mbar_wait(&full[jt % a.nstages], (uint32_t)((jt / a.nstages) & 1), nullptr, &never);
      if (nsw > 0) tc::mbar_wait(xfull, (uint32_t)((nsw - 1) & 1), nullptr, &never);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------------------- MMA
      constexpr uint32_t idesc = tc::idesc_make(1u, 0u, 0u, 128u, 32u);
      const uint32_t xa = tc::smem_u32(xs);
      int prev = -1;
      int64_t it = 0, nsw = 0, ti = 0;
      bool ok = true;
      int p_nx = q0 < q1 ? item_p[q0] : 0;
      uint32_t t_nx = q0 < q1 ? (uint32_t)item_t[q0] : 0u;
      for (int64_t q = q0; q < q1 && ok; ++q, ++ti) {
        const int p = p_nx;
        const int nk = (int)(t_nx >> 24);
        if (q + 1 < q1) {
          p_nx = item_p[q + 1];
          t_nx = (uint32_t)item_t[q + 1];
        }
        if (p != prev) {
          if (nsw > 0) tc::mma_commit(xfree);   // every MMA reading the old X^T has been issued
          if (!tc::mbar_wait(xfull, (uint32_t)(nsw & 1), a.err, abort_flag)) break;
          tc::tc_fence_after();
          ++nsw;
          prev = p;
        }
        const int b = (int)(ti & 1);
        if (!tc::mbar_wait(&tfree[b], (uint32_t)(((ti >> 1) & 1) ^ 1), a.err, abort_flag)) break;
        tc::tc_fence_after();
        for (int kb0 = 0; kb0 < nk; kb0 += HP_KPS, ++it) {
          const int nc = min(HP_KPS, nk - kb0);
          const int s = (int)(it % a.nstages);
          if (!tc::mbar_wait(&full[s], (uint32_t)((it / a.nstages) & 1), a.err, abort_flag)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          for (int c = 0; c < nc; ++c) {
            const int kb = kb0 + c;
            const uint64_t ad = tc::sdesc_sw128(tc::smem_u32(ring + (size_t)s * HP_STAGE + (size_t)c * HP_KCHUNK), 16, 1024);
            const uint64_t bd = tc::sdesc_sw128(xa + (uint32_t)kb * HP_XCHUNK, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc::mma_f16(tmem + (uint32_t)b * 32u, tc::sdesc_add(ad, kk * 32), tc::sdesc_add(bd, kk * 32), idesc,
                          (kb > 0 || kk > 0) ? 1u : 0u);
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&tfull[b]);
      }
      tc::mma_commit(done);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // tile rows -> shared staging (thread = row), then coalesced stores of
    // the valid rows by all four warps
    const int quad = warp & 3;
    const int row = quad * 32 + lane;   // tile row = TMEM lane
    const int et = tid - 64;            // 0..127
    int64_t ti = 0;
    for (int64_t q = q0; q < q1; ++q, ++ti) {
      const int b = (int)(ti & 1);
      bool ok = tc::mbar_wait(&tfull[b], (uint32_t)((ti >> 1) & 1), a.err, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      ok = epi_bar_and(ok);
      if (!ok) break;
      tc::tc_fence_after();
      float v[32];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * 32u;
      tc::tmem_ld16(taddr, *reinterpret_cast<float(*)[16]>(&v[0]));
      tc::tmem_ld16(taddr + 16, *reinterpret_cast<float(*)[16]>(&v[16]));
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tfree[b]);
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < a.l) hst[row * HP_HPITCH + c] = v[c];
      if (a.write_z) {
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          uint32_t wd[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 8 * g + 2 * e;   // l <= 32: columns past 31 are zero
            const float x0 = (c < a.l) ? v[c & 31] : 0.f;
            const float x1 = (c + 1 < a.l) ? v[(c + 1) & 31] : 0.f;
            __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
            wd[e] = *reinterpret_cast<uint32_t*>(&h2);
          }
          *reinterpret_cast<uint4*>(zst + row * 128 + ((g ^ (row & 7)) << 4)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
      }
      epi_bar();
      const GrpProblem& P = probs[item_p[q]];
      const int64_t row0 = (int64_t)((uint32_t)item_t[q] & 0xffffffu) * 128;
      const int nr = (int)(P.m - row0 < 128 ? P.m - row0 : 128);
      for (int e = et; e < nr * a.l; e += 128) {
        const int r = e / a.l, c = e % a.l;
        P.H[(row0 + r) * a.w + a.col0 + c] = hst[r * HP_HPITCH + c];
      }
      if (a.write_z)
        for (int e = et; e < nr * 8; e += 128) {
          const int r = e >> 3, g = e & 7;
          reinterpret_cast<uint4*>(P.Z + (row0 + r) * 64)[g] =
              *reinterpret_cast<const uint4*>(zst + r * 128 + ((g ^ (r & 7)) << 4));
        }
      epi_bar();   // the staging is free for the next tile
    }
  }
  // every MMA of this CTA has completed before TMEM is released
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done, 0, nullptr, &never);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// ================================================== T / F pass (tcgen05)
// Y_p[:, 0:N] += A_p[rows, :]^T Z_p[rows, 0:N] for every item (problem,
// range of 64-row groups), all of the problem's columns: A^T and Z are
// MN-major operands (M = 128 columns of A per tile, N = Z columns, K = rows),
// the ntile = ceil(n / 128) tile accumulators live in tensor memory for the
// whole item, and the epilogue adds them to Y with vector FP32 reductions.
//
// A stage is the Z box of a 64-row group plus the A boxes (64 rows x 64
// columns, 8 KB) of up to TPG_TPS column tiles of that group; a wide
// problem's group spans several consecutive stages, which load its Z box
// again (from L2, just read).  Each row of A is read once from memory, and
// so is each row of Z.
constexpr int TPG_THREADS = 192;
constexpr uint32_t TPG_BOX = 64 * 128;          // 64 rows x 64 BF16
constexpr int TPG_TPS = 2;
constexpr uint32_t TPG_STAGE = (1 + 2 * TPG_TPS) * TPG_BOX;

__global__ void __launch_bounds__(TPG_THREADS, 1)
k_grp_tpass(const GrpProblem* __restrict__ probs, const GrpTItem* __restrict__ items, int64_t nitems,
            TPassArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  if (__syncthreads_or((*(volatile uint32_t*)a.err & DEV_ERR_TIMEOUT) != 0)) return;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)a.nstages * TPG_STAGE);
  uint64_t* empty = full + a.nstages;
  uint64_t* tfull = empty + a.nstages;
  uint64_t* tfree = tfull + 1;
  uint64_t* done = tfree + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t my_items = nitems > blockIdx.x ? (nitems - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (tid == 0) {
    for (int s = 0; s < a.nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(tfull, 1);
    tc::mbar_init(tfree, 4);
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      int64_t it = 0;
      bool ok = true;
      // L2 prefetch cursor a.pf stages ahead of the loads
      int64_t pqi = 0;
      int pgr = 0, pt0 = 0;
      auto prefetch_next = [&]() {
        if (pqi >= my_items) return;
        const GrpTItem J = items[blockIdx.x + pqi * gridDim.x];
        const int jt = (int)((probs[J.p].n + 127) / 128);
        const int32_t r0 = (J.sub0 + pgr) * 64;
        if (pt0 == 0) tc::tma_prefetch_l2_2d(&a.tmZ[J.p], 0, r0);
        const int nt = min(TPG_TPS, jt - pt0);
        for (int bx = 0; bx < 2 * nt; ++bx) tc::tma_prefetch_l2_2d(&a.tmA[J.p], 128 * pt0 + 64 * bx, r0);
        pt0 += TPG_TPS;
        if (pt0 >= jt) {
          pt0 = 0;
          if (++pgr >= J.nsub) {
            pgr = 0;
            ++pqi;
          }
        }
      };
      for (int i = 0; i < a.pf; ++i) prefetch_next();
      for (int64_t qi = 0; qi < my_items && ok; ++qi) {
        const GrpTItem I = items[blockIdx.x + qi * gridDim.x];
        const int ntile = (int)((probs[I.p].n + 127) / 128);
        const CUtensorMap* tA = &a.tmA[I.p];
        const CUtensorMap* tZ = &a.tmZ[I.p];
        for (int gr = 0; gr < I.nsub && ok; ++gr) {
          const int32_t r0 = (I.sub0 + gr) * 64;
          for (int t0 = 0; t0 < ntile; t0 += TPG_TPS, ++it) {
            const int nt = min(TPG_TPS, ntile - t0);
            const int s = (int)(it % a.nstages);
            if (!tc::mbar_wait(&empty[s], (uint32_t)(((it / a.nstages) & 1) ^ 1), a.err, abort_flag)) {
              ok = false;
              break;
            }
            unsigned char* st = smem + (size_t)s * TPG_STAGE;
            tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(1 + 2 * nt) * TPG_BOX);
            tc::tma_load_2d(st, tZ, &full[s], 0, r0);
            for (int bx = 0; bx < 2 * nt; ++bx)
              tc::tma_load_2d(st + (size_t)(1 + bx) * TPG_BOX, tA, &full[s], 128 * t0 + 64 * bx, r0);
            if (a.pf > 0) prefetch_next();
          }
        }
      }
      volatile int never = 0;
      for (int64_t jt = (it > a.nstages ? it - a.nstages : 0); jt < it; ++jt)
        tc::mbar_wait(&full[jt % a.nstages], (uint32_t)((jt / a.nstages) & 1), nullptr, &never);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------------------- MMA
      const uint32_t idesc = tc::idesc_make(1u, 1u, 1u, 128u, (uint32_t)a.npad);
      int64_t it = 0;
      bool ok = true;
      for (int64_t qi = 0; qi < my_items && ok; ++qi) {
        const GrpTItem I = items[blockIdx.x + qi * gridDim.x];
        const int ntile = (int)((probs[I.p].n + 127) / 128);
        if (!tc::mbar_wait(tfree, (uint32_t)((qi & 1) ^ 1), a.err, abort_flag)) break;
        tc::tc_fence_after();
        for (int gr = 0; gr < I.nsub && ok; ++gr) {
          for (int t0 = 0; t0 < ntile; t0 += TPG_TPS, ++it) {
            const int nt = min(TPG_TPS, ntile - t0);
            const int s = (int)(it % a.nstages);
            if (!tc::mbar_wait(&full[s], (uint32_t)((it / a.nstages) & 1), a.err, abort_flag)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            const uint32_t sa = tc::smem_u32(smem + (size_t)s * TPG_STAGE);
            for (int tt = 0; tt < nt; ++tt) {
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = tc::sdesc_sw128(sa + (uint32_t)(1 + 2 * tt) * TPG_BOX + kk * 2048, TPG_BOX, 1024);
                const uint64_t bd = tc::sdesc_sw128(sa + kk * 2048, TPG_BOX, 1024);
                tc::mma_f16(tmem + (uint32_t)((t0 + tt) * a.npad), ad, bd, idesc, (gr > 0 || kk > 0) ? 1u : 0u);
              }
            }
            tc::mma_commit(&empty[s]);
          }
        }
        if (!ok) break;
        tc::mma_commit(tfull);
      }
      tc::mma_commit(done);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    for (int64_t qi = 0; qi < my_items; ++qi) {
      const GrpTItem I = items[blockIdx.x + qi * gridDim.x];
      const GrpProblem& P = probs[I.p];
      const int ntile = (int)((P.n + 127) / 128);
      bool ok = tc::mbar_wait(tfull, (uint32_t)(qi & 1), a.err, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc::tc_fence_after();
      float* ybase = a.mode_t ? P.T : P.F;
      for (int t = 0; t < ntile; ++t) {
        const int64_t row = (int64_t)t * 128 + quad * 32 + lane;   // n-index of Y
        float* y = ybase + row * a.ldy;
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(t * a.npad);
        for (int c16 = 0; c16 < a.npad; c16 += 16) {
          float v[16];
          tc::tmem_ld16(taddr + c16, v);
          if (row < P.n) {
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4)
              if (c16 + 4 * g4 < a.ncols)
                red_add_v4(y + c16 + 4 * g4, v[4 * g4], v[4 * g4 + 1], v[4 * g4 + 2], v[4 * g4 + 3]);
          }
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tfree);
    }
  }
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done, 0, nullptr, &never);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ------------------------------------------------------------- launchers
size_t hpass_smem(uint32_t xbytes, int nstages) {
  return 1024 + xbytes + (size_t)nstages * HP_STAGE + HP_ZSTAGE + 128 * HP_HPITCH * 4 + (2 * nstages + 7) * 8 + 16;
}
size_t tpass_smem(int nstages) { return 1024 + (size_t)nstages * TPG_STAGE + (2 * nstages + 3) * 8 + 16; }

void launch_hpass(const GrpProblem* probs, const int32_t* item_p, const int32_t* item_t, int64_t nitems,
                  const HPassArgs& a, int grid, cudaStream_t st) {
  if (nitems <= 0) return;
  const size_t smem = hpass_smem(a.xbytes, a.nstages);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_hpass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, nitems));
  k_grp_hpass<<<grid, HP_THREADS, smem, st>>>(probs, item_p, item_t, nitems, a);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

void launch_tpass(const GrpProblem* probs, const GrpTItem* items, int64_t nitems, const TPassArgs& a, int grid,
                  cudaStream_t st) {
  if (nitems <= 0) return;
  const size_t smem = tpass_smem(a.nstages);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_grp_tpass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, nitems));
  k_grp_tpass<<<grid, TPG_THREADS, smem, st>>>(probs, items, nitems, a);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

}  // namespace grp
}  // namespace rpca
