// Tensor-core streamed passes over A (tcgen05 + TMA, sm_103a).
//
// T pass (Step 3, eq. product_t3): T = A^T Q.  A is split into column slabs
// of NT*128 columns; each CTA owns one slab and a strided subset of row
// sub-panels of KSUB rows, keeps its T-slab (NT*128 x NPAD, FP32) in TMEM for
// the whole kernel, and adds it to the FP64 result once at the end.  Per
// sub-panel: TMA loads A[r0:r0+KSUB, slab] and Q[r0:r0+KSUB, :] (BF16,
// 128-byte swizzle) into a stage of the smem ring; one thread issues
// tcgen05.mma with A^T as an MN-major operand (M = slab columns, K = rows)
// and Q as an MN-major operand (N = Q columns, K = rows).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rpca {

// ----------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

bool make_tmap_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dt, size_t elem_bytes,
                  int64_t rows, int64_t cols, int64_t ld, uint32_t box_rows, uint32_t box_cols) {
  auto enc = get_encode();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  if (((size_t)ld * elem_bytes) % 16 != 0) return false;
  if (box_cols * elem_bytes != 128) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(ld * elem_bytes)};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), gdim, gstride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

// Q (FP32 m x w, ldq) -> BF16 m x wpad, zero padded columns.
__global__ void k_q_to_bf16(int64_t m, int w, int wpad, const float* __restrict__ Q, int64_t ldq,
                            __nv_bfloat16* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * wpad) return;
  int64_t r = e / wpad;
  int c = (int)(e % wpad);
  out[e] = __float2bfloat16_rn(c < w ? Q[r * ldq + c] : 0.f);
}

constexpr int TP_KSUB = 64;        // rows per pipeline stage
constexpr int TP_THREADS = 128;

struct TPassSmem {
  // offsets in bytes from the 1024-aligned dynamic smem base
  uint32_t stage_bytes, a_bytes, nstages, bar_off;
};

// T-slab accumulation in TMEM; output TF (double or float) via atomics.
template <int NT, typename TF>
__global__ void __launch_bounds__(TP_THREADS, 1)
k_tpass_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmQ, int64_t m,
             int64_t n, int w, int npad, int nqbox, int nslab, int ngroup, int nstages, uint32_t stage_bytes,
             TF* __restrict__ T, int64_t ldt, int qblk, uint32_t* __restrict__ dev_err, uint64_t wait_ns,
             int64_t withhold) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t a_bytes = NT * 2 * TP_KSUB * 128;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nstages * stage_bytes);
  uint64_t* empty = full + nstages;
  uint64_t* done = empty + nstages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slab = blockIdx.x % nslab;
  const int group = blockIdx.x / nslab;
  if (group >= ngroup) return;
  const int64_t nsub = (m + TP_KSUB - 1) / TP_KSUB;
  const int64_t my_subs = (nsub > group) ? (nsub - group + ngroup - 1) / ngroup : 0;
  const uint32_t tmem_cols = (NT * npad <= 32) ? 32 : (NT * npad <= 64) ? 64 : (NT * npad <= 128) ? 128
                             : (NT * npad <= 256) ? 256 : 512;

  if (tid == 0) {
    for (int s = 0; s < nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::tma_prefetch(&tmA);
    tc::tma_prefetch(&tmQ);
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    // wait-expiry test: sub-panel `withheld` of CTA 0 is never issued
    const int64_t withheld = blockIdx.x == 0 ? withhold : -1;
    int64_t it = 0;
    for (; it < my_subs; ++it) {
      const int s = (int)(it % nstages);
      const uint32_t ph = (uint32_t)((it / nstages) & 1);
      if (!tc::mbar_wait(&empty[s], ph ^ 1u, dev_err, abort_flag, false, wait_ns)) break;
      if (it == withheld) continue;
      unsigned char* st = smem + (size_t)s * stage_bytes;
      const int32_t r0 = (int32_t)((group + it * ngroup) * TP_KSUB);
      tc::mbar_arrive_expect_tx(&full[s], stage_bytes);
#pragma unroll
      for (int j = 0; j < 2 * NT; ++j)
        tc::tma_load_2d(st + (size_t)j * TP_KSUB * 128, &tmA, &full[s], slab * NT * 128 + 64 * j, r0);
      for (int j = 0; j < nqbox; ++j)
        tc::tma_load_2d(st + a_bytes + (size_t)j * TP_KSUB * 128, &tmQ, &full[s], 64 * j, r0);
    }
    // after an abort, let the copies still in flight land before the CTA
    // can exit
    for (int64_t jt = (it > nstages ? it - nstages : 0); jt < it; ++jt) {
      if (jt == withheld) continue;
      volatile int never = 0;
      tc::mbar_wait(&full[jt % nstages], (uint32_t)((jt / nstages) & 1), nullptr, &never);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------- MMA issue
    const uint32_t idesc = tc::idesc_make(1u, 1u, 1u, 128u, (uint32_t)npad);
    const uint32_t box = TP_KSUB * 128;
    for (int64_t it = 0; it < my_subs; ++it) {
      const int s = (int)(it % nstages);
      const uint32_t ph = (uint32_t)((it / nstages) & 1);
      if (!tc::mbar_wait(&full[s], ph, dev_err, abort_flag, false, wait_ns)) break;
      tc::tc_fence_after();
      const uint32_t sa = tc::smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t sq = sa + a_bytes;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
#pragma unroll
        for (int kk = 0; kk < TP_KSUB / 16; ++kk) {
          uint64_t ad = tc::sdesc_sw128(sa + t * 2 * box + kk * 2048, box, 1024);
          uint64_t bd = tc::sdesc_sw128(sq + kk * 2048, box, 1024);
          tc::mma_f16(tmem + t * npad, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(&empty[s]);
    }
    tc::mma_commit(done);
  }
  __syncwarp();
  // --------------------------------------------------------------- epilogue
  bool ok = (my_subs == 0) ? false : tc::mbar_wait(done, 0, dev_err, abort_flag, false, wait_ns);
  ok = __all_sync(0xffffffffu, ok);
  tc::tc_fence_after();
  if (ok) {
    const int64_t col0 = (int64_t)slab * NT * 128;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int64_t row = col0 + t * 128 + warp * 32 + lane;   // n-index of T
      for (int c16 = 0; c16 < npad; c16 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + t * npad + c16, v);
        if (row < n) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int c = c16 + q;
            if (qblk > 0) {
              // block-padded Q: column c is column (c/64)*qblk + c%64 of T
              if ((c & 63) < qblk) atomicAdd(&T[row * ldt + (c >> 6) * qblk + (c & 63)], (TF)v[q]);
            } else if (c < w) {
              atomicAdd(&T[row * ldt + c], (TF)v[q]);
            }
          }
        }
      }
    }
  }
  // every MMA issued by this CTA has completed before TMEM is released
  // (after an abort the wait above returns early; the issuer always commits
  // `done`)
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done, 0, nullptr, &never);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

int g_num_sms = 0;

}  // namespace

// ------------------------------------------------------------------- host
static bool tpass_bf16(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  if (a.dtype != RPCA_BF16 || a.mode != MODE_T) return false;
  if (a.shift || a.scale) return false;
  if (a.p > 256) return false;
  const bool pre = a.q16 != nullptr;                 // Q already BF16, block-padded
  if (!pre && !a.work) return false;
  const int wq = pre ? (int)a.q16_ld : (int)round_up(a.p, 64);   // Q16 columns (box multiple)
  if (wq > 256 || wq % 64) return false;
  const int npad = pre ? wq : (int)round_up(a.p, 16);
  if (!pre && (size_t)a.m * wq * 2 > a.work_bytes) return false;
  const int NT = (npad <= 256 && 2 * npad <= 512) ? 2 : 1;
  CUtensorMap tmA, tmQ;
  if (!make_tmap_2d(&tmA, a.A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.m, a.n, a.lda, TP_KSUB, 64)) return false;
  const __nv_bfloat16* Q16 = pre ? static_cast<const __nv_bfloat16*>(a.q16) : static_cast<__nv_bfloat16*>(a.work);
  if (!make_tmap_2d(&tmQ, Q16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.m, wq, wq, TP_KSUB, 64)) return false;
  const int qblk = pre ? a.q_blk : 0;
  // Q -> BF16 (zero-padded)
  if (!pre) {
    int64_t cnt = a.m * wq;
    k_q_to_bf16<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(a.m, a.p, wq, static_cast<const float*>(a.H), a.ldh,
                                                          static_cast<__nv_bfloat16*>(a.work));
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  const int nqbox = (int)cdiv(npad, 64);
  const uint32_t stage_bytes = (uint32_t)((NT * 2 + nqbox) * TP_KSUB * 128);
  int nstages = (int)std::min<int64_t>(8, (200 * 1024) / stage_bytes);
  if (nstages < 2) return false;
  const size_t smem = 1024 + (size_t)nstages * stage_bytes + (2 * nstages + 1) * 8 + 16;
  if (!g_num_sms) g_num_sms = num_sms();
  const int nslab = (int)cdiv(a.n, NT * 128);
  const int ngroup = std::max(1, std::min<int>((int)cdiv(a.m, TP_KSUB), g_num_sms / nslab));
  const size_t fes = a.f_f64 ? 8 : 4;
  if (!a.accumulate_f)
    RPCA_CUDA_TRY(cudaMemset2DAsync(a.F, a.ldf * fes, 0, a.p * fes, a.n, st));
  dim3 grid(nslab * ngroup);
  const WaitTest wt = take_wait_test(1);
  if (a.f_f64) {
    auto kern = NT == 2 ? k_tpass_bf16<2, double> : k_tpass_bf16<1, double>;
    RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, TP_THREADS, smem, st>>>(tmA, tmQ, a.m, a.n, a.p, npad, nqbox, nslab, ngroup, nstages,
                                          stage_bytes, static_cast<double*>(a.F), a.ldf, qblk, dev_err, wt.limit_ns,
                                          wt.withhold);
  } else {
    auto kern = NT == 2 ? k_tpass_bf16<2, float> : k_tpass_bf16<1, float>;
    RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, TP_THREADS, smem, st>>>(tmA, tmQ, a.m, a.n, a.p, npad, nqbox, nslab, ngroup, nstages,
                                          stage_bytes, static_cast<float*>(a.F), a.ldf, qblk, dev_err, wt.limit_ns,
                                          wt.withhold);
  }
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
  return true;
}

bool launch_pass_tc(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  // FP32, FP8 and shifted or scaled BF16: the converter kernels (k_stream_cvt.cu)
  if (a.dtype == RPCA_F32 || a.dtype == RPCA_FP8E4M3 || (a.dtype == RPCA_BF16 && (a.shift || a.scale)))
    return pass_cvt(a, st, dev_err);
  if (a.mode == MODE_T) return tpass_bf16(a, st, dev_err);
  return fused_pass_tc(a, st, dev_err);
}

}  // namespace rpca
