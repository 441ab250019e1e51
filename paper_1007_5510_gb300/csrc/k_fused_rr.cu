// Fused Step-1 pass on tensor cores, L2 re-read form (tcgen05 + TMA +
// cluster DSMEM), BF16 A.
//
// One pass of Section 3's Step 1 that reads A once from HBM (Section 4.2's
// row-block streaming).  For each 128-row panel A_b:
//     H_b = A_b X                  (stored, FP32)
//     F  += A_b^T H_b              (FP32 accumulators in TMEM)
// A cluster of CS CTAs shares each panel.  CTA c owns the column slab
// [c*512, (c+1)*512), keeps X[slab] (BF16) resident in shared memory and
// F[slab] (4 blocks of 128 rows) in tensor memory for the whole kernel.
//   GEMM1  P_c = A_b[:, slab] X[slab]          M=128, N=L, K=512 (K-major A)
//   reduce H_b = sum_c P_c across the cluster  (CTA c owns rows [c*128/CS, ...))
//   GEMM2  F[slab] += A_b[:, slab]^T H_b       M=128, N=L, K=128 (MN-major A)
//
// Data movement.  GEMM1's tiles come from HBM through a ring of 16 KB stages
// that is released as soon as GEMM1 has read them; GEMM2 reads the same
// bytes again, a few microseconds later, through a second ring (L2 policy:
// evict_last on the first read, evict_first on the second).  A tile is thus
// never held in shared memory across the cluster reduction, so the bytes in
// flight only have to cover HBM and L2 latency.
//
// Reduction.  Two epilogue groups of 4 warps each handle one half of H_b's
// columns, so two panels' exchanges overlap.  A thread drains its row of the
// partial from tensor memory and pushes it with st.async into the owning
// CTA's receive buffer (byte-counted on the owner's mbarrier, so the data and
// its arrival signal travel together); the owner sums the CS partials of its
// rows, stores them to H, and pushes their BF16 copy into every CTA's GEMM2
// operand buffer the same way.
//
// Roles (12 warps): warp 0 lane 0 streams GEMM1's tiles, warp 1 lane 0
// issues GEMM1, warps 2-5 and 8-11 are the two epilogue groups (which also
// flush F), warp 6 lane 0 streams GEMM2's tiles, warp 7 lane 0 issues GEMM2.
// Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rpca {
namespace {

constexpr int RR_THREADS = 384;
constexpr int RR_BM = 128;                    // panel rows
constexpr int RR_NT = 4;                      // 128-column blocks per slab
constexpr int RR_NC = RR_NT * 128;            // slab width
constexpr int RR_NBOX = RR_NC / 64;           // 64-column boxes per slab
constexpr uint32_t RR_HBOX = RR_BM * 128;     // GEMM1 stage: 128 rows x 64 cols BF16
constexpr uint32_t RR_FHALF = 64 * 128;       // 64 rows x 64 cols BF16
constexpr uint32_t RR_FST = 2 * RR_FHALF;     // GEMM2 stage: 64 rows x 128 cols
constexpr uint32_t RR_HS = RR_BM * 128;       // BF16 H_b: 128 rows x 128 B
constexpr size_t RR_SMEM_LIMIT = 232448;      // opt-in shared memory per CTA

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t nclusters_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Named barrier (id 1 + g) over the 4 warps of epilogue group g.
__device__ __forceinline__ void grp_bar(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }
// The same barrier, ANDing a predicate so an abort decision is uniform.
__device__ __forceinline__ bool grp_bar_and(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %2, 0;\n bar.red.and.pred q, %1, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(1 + g), "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(cta));
  return r;
}
// Asynchronous stores into a cluster CTA's shared memory, counted (bytes) on
// that CTA's mbarrier rbar (both shared::cluster addresses).
__device__ __forceinline__ void st_async_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                            uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   addr),
               "r"(a), "r"(b), "r"(c), "r"(d), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_async_v2(uint32_t addr, uint32_t a, uint32_t b, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "r"(a), "r"(b), "r"(rbar)
               : "memory");
}
// Arrive (no ordering of earlier memory accesses) on the barrier at the same
// offset in CTA `cta` of the cluster.
__device__ __forceinline__ void arrive_relaxed_cluster(uint64_t* bar, uint32_t cta) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(mapa(tc::smem_u32(bar), cta))
               : "memory");
}
// 32 lanes x 32-bit, N consecutive columns per thread (N = 8, 16 or 32).
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[N]) {
  if constexpr (N == 8) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  } else if constexpr (N == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    static_assert(N == 32, "column count");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// X (n x l, FP32, ldx) -> Xt (L x n8, BF16): row j holds column j of X.
__global__ void k_xt_bf16_rr(int64_t n, int l, int L, int64_t n8, const float* __restrict__ X, int64_t ldx,
                             __nv_bfloat16* __restrict__ Xt) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * n8) return;
  int j = (int)(e / n8);
  int64_t r = e % n8;
  float v = (j < l && r < n) ? X[r * ldx + j] : 0.f;
  Xt[e] = __float2bfloat16_rn(v);
}

struct RRParams {
  int64_t m, n;
  int l;            // real columns of X / H
  int ones_col;     // -1 or column index (< L) of an all-ones H column
  int nh, nf;       // stages of the GEMM1 and GEMM2 rings
  float* H;
  int64_t ldh;
  const float* corr;   // l values subtracted from every H row, or null
  float* F;            // n x (l [+1]) FP32, accumulated (zeroed by the host)
  int64_t ldf;
  uint32_t* dev_err;
  uint64_t wait_ns;    // limit of every bounded wait (2 s; shorter only under the wait-expiry test)
  int64_t withhold;    // wait-expiry test: GEMM1 stage of CTA 0 left unissued (-1: none)
};

// Shared-memory layout (bytes from a 1024-aligned base):
//   [X slab: 8 boxes of L rows x 128 B, K-major SW128]
//   [GEMM1 ring: nh x (128 rows x 128 B)]
//   [GEMM2 ring: nf x (2 boxes of 64 rows x 128 B)]      (FUSED)
//   [Rcv[2]: per epilogue group, CS senders x 128/CS rows x L/2 FP32]
//   [Hs[2]: 128 rows x 128 B BF16, SW128 MN-major operand] (FUSED; panel it uses Hs[it & 1])
//   [barriers]
template <int L, bool FUSED>
__global__ void __launch_bounds__(RR_THREADS, 1)
k_fused_rr(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
           const __grid_constant__ CUtensorMap tmX, const RRParams p) {
  constexpr uint32_t XBOX = L * 128;
  constexpr uint32_t RCV_BYTES = RR_BM * L * 2;   // one group's receive buffer
  constexpr uint32_t HS_TX = RR_BM * L * 2;       // bytes of H_b written into Hs per panel
  constexpr uint32_t TMEM_COLS = ((2 + RR_NT) * L <= 128) ? 128 : ((2 + RR_NT) * L <= 256) ? 256 : 512;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xs = smem;
  unsigned char* hring = xs + RR_NBOX * XBOX;
  unsigned char* fring = hring + (size_t)p.nh * RR_HBOX;
  unsigned char* rcvbase = fring + (size_t)p.nf * RR_FST;
  unsigned char* hs = rcvbase + 2 * RCV_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(hs + (FUSED ? 2 * RR_HS : 0));
  uint64_t* hfull = bars;                     // [nh]
  uint64_t* hempty = hfull + p.nh;            // [nh]
  uint64_t* ffull = hempty + p.nh;            // [nf]
  uint64_t* fempty = ffull + p.nf;            // [nf]
  uint64_t* pfull = fempty + p.nf;            // [2]
  uint64_t* pempty = pfull + 2;               // [2]
  uint64_t* rfull = pempty + 2;               // [2] every sender's rows have reached Rcv[g]
  uint64_t* rfree = rfull + 2;                // [2] every owner has summed this CTA's rows
  uint64_t* hready = rfree + 2;               // [2] every owner's rows of H_b have reached Hs[x]
  uint64_t* hfree = hready + 2;               // [2] every CTA's GEMM2 has read its Hs[x]
  uint64_t* xfull = hfree + 2;
  uint64_t* done1 = xfull + 1;                // GEMM1 issuer's last MMA
  uint64_t* done2 = done1 + 1;                // GEMM2 issuer's last MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done2 + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t lim = p.wait_ns;
  const int64_t withheld = blockIdx.x == 0 ? p.withhold : -1;
  const uint32_t cs = cluster_nctarank();
  const uint32_t crank = cluster_rank();
  const uint32_t cid = cluster_id_x(), ncl = nclusters_x();
  const int64_t npan = (p.m + RR_BM - 1) / RR_BM;
  const int64_t my_pan = (npan > cid) ? (npan - cid + ncl - 1) / ncl : 0;
  const uint16_t cmask = (uint16_t)((1u << cs) - 1u);
  const int rpc = RR_BM / (int)cs;            // rows of H_b reduced by this CTA
  const int row0 = (int)crank * rpc;
  const int32_t slab0 = (int32_t)(crank * RR_NC);

  if (tid == 0) {
    for (int s = 0; s < p.nh; ++s) {
      tc::mbar_init(&hfull[s], 1);
      tc::mbar_init(&hempty[s], 1);
    }
    for (int s = 0; s < p.nf; ++s) {
      tc::mbar_init(&ffull[s], 1);
      tc::mbar_init(&fempty[s], 1);
    }
    for (int x = 0; x < 2; ++x) {
      tc::mbar_init(&pfull[x], 1);
      tc::mbar_init(&pempty[x], 8);           // one arrival per epilogue warp
      tc::mbar_init(&rfull[x], 1);            // the owner's arming arrival + bytes
      tc::mbar_init(&rfree[x], cs);
    }
    for (int x = 0; x < 2; ++x) {
      tc::mbar_init(&hready[x], 1);           // GEMM2's arming arrival + bytes
      tc::mbar_init(&hfree[x], cs);
    }
    tc::mbar_init(xfull, 1);
    tc::mbar_init(done1, 1);
    tc::mbar_init(done2, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::mbar_arrive_expect_tx(&rfull[0], RCV_BYTES);
    tc::mbar_arrive_expect_tx(&rfull[1], RCV_BYTES);
    if (FUSED) {
      tc::mbar_arrive_expect_tx(&hready[0], HS_TX);
      tc::mbar_arrive_expect_tx(&hready[1], HS_TX);
    }
    tc::tma_prefetch(&tmA);
    if (FUSED) tc::tma_prefetch(&tmA2);
    tc::tma_prefetch(&tmX);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  cluster_sync_all();            // every CTA's barriers exist before remote arrivals
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tm_p = tmem;                    // P[0], P[1]: columns [0, 2L)
  const uint32_t tm_f = tmem + 2 * L;            // F slab: RR_NT blocks of L columns

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------- GEMM1 tiles (from HBM)
      // the first read keeps the lines in L2 for GEMM2's re-read (FUSED)
      const uint64_t pol = FUSED ? tc::l2_policy_evict_last() : tc::l2_policy_evict_first();
      tc::mbar_arrive_expect_tx(xfull, RR_NBOX * XBOX);
      for (int j = 0; j < RR_NBOX; ++j) tc::tma_load_2d(xs + (size_t)j * XBOX, &tmX, xfull, slab0 + 64 * j, 0);
      int64_t q = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < my_pan; ++it) {
        const int32_t r0 = (int32_t)((cid + it * ncl) * RR_BM);
        for (int j = 0; j < RR_NBOX; ++j, ++q) {
          const int s = (int)(q % p.nh);
          if (!tc::mbar_wait(&hempty[s], (uint32_t)(((q / p.nh) & 1) ^ 1), p.dev_err, abort_flag, false, lim)) {
            ok = false;
            break;
          }
          if (q == withheld) continue;        // wait-expiry test: this stage never arrives
          tc::mbar_arrive_expect_tx(&hfull[s], RR_HBOX);
          tc::tma_load_2d_hint(hring + (size_t)s * RR_HBOX, &tmA, &hfull[s], slab0 + 64 * j, r0, pol);
        }
      }
      // let in-flight copies land before the CTA can exit
      for (int64_t qq = (q > p.nh ? q - p.nh : 0); qq < q; ++qq) {
        if (qq == withheld) continue;
        volatile int never = 0;
        tc::mbar_wait(&hfull[qq % p.nh], (uint32_t)((qq / p.nh) & 1), nullptr, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------ GEMM1 issue
      constexpr uint32_t idesc1 = tc::idesc_make(1u, 0u, 0u, 128u, (uint32_t)L);
      const uint32_t xs_a = tc::smem_u32(xs);
      bool ok = tc::mbar_wait(xfull, 0, p.dev_err, abort_flag, false, lim);
      int64_t q = 0;
      for (int64_t it = 0; ok && it < my_pan; ++it) {
        const int pb = (int)(it & 1);
        if (!tc::mbar_wait(&pempty[pb], (uint32_t)(((it >> 1) & 1) ^ 1), p.dev_err, abort_flag, false, lim)) break;
        tc::tc_fence_after();
        for (int j = 0; j < RR_NBOX; ++j, ++q) {
          const int s = (int)(q % p.nh);
          if (!tc::mbar_wait(&hfull[s], (uint32_t)((q / p.nh) & 1), p.dev_err, abort_flag, false, lim)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint64_t da = tc::sdesc_sw128(tc::smem_u32(hring + (size_t)s * RR_HBOX), 16, 1024);
          const uint64_t db = tc::sdesc_sw128(xs_a + (uint32_t)j * XBOX, 16, 1024);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16(tm_p + pb * L, tc::sdesc_add(da, kk * 32), tc::sdesc_add(db, kk * 32), idesc1,
                        (j > 0 || kk > 0) ? 1u : 0u);
          tc::mma_commit(&hempty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&pfull[pb]);
      }
      tc::mma_commit(done1);
    }
  } else if (warp == 6) {
    if (FUSED && lane == 0) {
      // --------------------------------------- GEMM2 tiles (L2 re-read)
      const uint64_t pol = tc::l2_policy_evict_first();
      int64_t q = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < my_pan; ++it) {
        const int32_t r0 = (int32_t)((cid + it * ncl) * RR_BM);
        for (int u = 0; u < 2 * RR_NT; ++u, ++q) {
          const int t = u >> 1, h = u & 1;
          const int s = (int)(q % p.nf);
          if (!tc::mbar_wait(&fempty[s], (uint32_t)(((q / p.nf) & 1) ^ 1), p.dev_err, abort_flag, false, lim)) {
            ok = false;
            break;
          }
          unsigned char* st = fring + (size_t)s * RR_FST;
          tc::mbar_arrive_expect_tx(&ffull[s], RR_FST);
          tc::tma_load_2d_hint(st, &tmA2, &ffull[s], slab0 + 128 * t, r0 + 64 * h, pol);
          tc::tma_load_2d_hint(st + RR_FHALF, &tmA2, &ffull[s], slab0 + 128 * t + 64, r0 + 64 * h, pol);
        }
      }
      for (int64_t qq = (q > p.nf ? q - p.nf : 0); qq < q; ++qq) {
        volatile int never = 0;
        tc::mbar_wait(&ffull[qq % p.nf], (uint32_t)((qq / p.nf) & 1), nullptr, &never);
      }
    }
  } else if (warp == 7) {
    if (FUSED && lane == 0) {
      // ------------------------------------------------------ GEMM2 issue
      constexpr uint32_t idesc2 = tc::idesc_make(1u, 1u, 1u, 128u, (uint32_t)L);
      const uint32_t hs_a = tc::smem_u32(hs);
      int64_t q = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < my_pan; ++it) {
        const int x = (int)(it & 1);
        if (!tc::mbar_wait(&hready[x], (uint32_t)((it >> 1) & 1), p.dev_err, abort_flag, true, lim)) break;
        // Hs[x] was written by the owners' asynchronous stores; order them
        // before the tensor core's reads
        tc::fence_proxy_async_smem();
        tc::tc_fence_after();
        // arm the buffer's next use (panel it + 2: all owners' bytes of H)
        tc::mbar_arrive_expect_tx(&hready[x], HS_TX);
        for (int u = 0; u < 2 * RR_NT; ++u, ++q) {
          const int t = u >> 1, h = u & 1;
          const int s = (int)(q % p.nf);
          if (!tc::mbar_wait(&ffull[s], (uint32_t)((q / p.nf) & 1), p.dev_err, abort_flag, false, lim)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint64_t da = tc::sdesc_sw128(tc::smem_u32(fring + (size_t)s * RR_FST), RR_FHALF, 1024);
          const uint64_t db = tc::sdesc_sw128(hs_a + (uint32_t)x * RR_HS + (uint32_t)h * 8192u, RR_HS, 1024);
#pragma unroll
          for (int kr = 0; kr < 4; ++kr)
            tc::mma_f16(tm_f + t * L, tc::sdesc_add(da, kr * 2048), tc::sdesc_add(db, kr * 2048), idesc2,
                        (it > 0 || h > 0 || kr > 0) ? 1u : 0u);
          tc::mma_commit(&fempty[s]);
        }
        if (!ok) break;
        tc::mma_commit_multicast(&hfree[x], cmask);
      }
      tc::mma_commit(done2);
    }
  } else {
    // ------------------ drain, reduce, distribute: epilogue group g
    const int g = warp >= 8 ? 1 : 0;              // column half [g*HALF, (g+1)*HALF)
    const int e = g ? tid - 256 : tid - 64;       // 0..127 within the group
    const int quad = warp & 3;                    // TMEM lane quadrant of this warp
    const int trow = 32 * quad + lane;            // TMEM lane = panel row
    constexpr int HALF = L / 2;
    constexpr int CH = HALF / 4;                  // 16-byte chunks per half row
    constexpr uint32_t ROWB = HALF * 4;           // bytes of a half row (FP32)
    unsigned char* rcv = rcvbase + g * RCV_BYTES;
    const uint32_t rcv_a = tc::smem_u32(rcv);
    const uint32_t hs_a = tc::smem_u32(hs);
    uint64_t* my_rfull = &rfull[g];
    uint64_t* my_rfree = &rfree[g];
    // this thread's row goes to its owner's receive buffer, slot (crank, row)
    const uint32_t owner = (uint32_t)(trow / rpc);
    const uint32_t dst_row = mapa(rcv_a + (uint32_t)((int)crank * rpc + trow % rpc) * ROWB, owner);
    const uint32_t dst_bar = mapa(tc::smem_u32(my_rfull), owner);
    const uint32_t hready_a = tc::smem_u32(hready);     // + 8 x for Hs[x]
    bool ok = true;
    for (int64_t it = 0; it < my_pan; ++it) {
      const int pb = (int)(it & 1);
      const int64_t r0 = (cid + it * ncl) * RR_BM;
      ok = tc::mbar_wait(&pfull[pb], (uint32_t)((it >> 1) & 1), p.dev_err, abort_flag, false, lim);
      // every owner has summed this CTA's rows of the previous panel
      ok = ok && tc::mbar_wait(my_rfree, (uint32_t)((it - 1) & 1), p.dev_err, abort_flag, true, lim);
      ok = grp_bar_and(g, ok);
      if (!ok) break;
      tc::tc_fence_after();
      {
        uint32_t v[HALF];
        tmem_ld_cols<HALF>(tm_p + pb * L + ((uint32_t)(32 * quad) << 16) + g * HALF, v);
#pragma unroll
        for (int j = 0; j < CH; ++j)
          st_async_v4(dst_row + 16 * j, v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3], dst_bar);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&pempty[pb]);
      // every sender's rows of this panel have arrived
      ok = tc::mbar_wait(my_rfull, (uint32_t)(it & 1), p.dev_err, abort_flag, true, lim);
      // every CTA's GEMM2 of panel it - 2 has read its Hs[it & 1]
      if (FUSED) ok = ok && tc::mbar_wait(&hfree[pb], (uint32_t)(((it >> 1) & 1) ^ 1), p.dev_err, abort_flag, true, lim);
      ok = grp_bar_and(g, ok);
      if (!ok) break;
      if (e == 0) tc::mbar_arrive_expect_tx(my_rfull, RCV_BYTES);   // arm the next panel
      // rows [row0, row0 + rpc), columns of this half: sum the CS partials,
      // apply the centring corrections, store, and push the BF16 copies
      for (int pair = e; pair < rpc * CH; pair += 128) {
        const int rl = pair / CH, k = pair % CH;
        float4 sacc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (uint32_t c = 0; c < cs; ++c) {
          const float4 t = *reinterpret_cast<const float4*>(rcv + ((int)c * rpc + rl) * ROWB + k * 16);
          sacc.x += t.x;
          sacc.y += t.y;
          sacc.z += t.z;
          sacc.w += t.w;
        }
        const int rr = row0 + rl, col = g * HALF + 4 * k;
        const int64_t grow = r0 + rr;
        float vv[4] = {sacc.x, sacc.y, sacc.z, sacc.w};
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int cc = col + qq;
          if (p.corr && cc < p.l) vv[qq] -= p.corr[cc];
          if (grow >= p.m || cc >= p.l) vv[qq] = 0.f;
          if (cc == p.ones_col && grow < p.m) vv[qq] = 1.f;
        }
        if (FUSED) {
          // row rr of Hs[pb] (SW128, MN-major), in every CTA of the cluster
          const uint32_t hoff = (uint32_t)pb * RR_HS +
                                (uint32_t)(rr * 128 + ((((col >> 3) ^ (rr & 7))) << 4) + (col & 7) * 2);
          const uint32_t lo = pack_bf16(vv[0], vv[1]), hi = pack_bf16(vv[2], vv[3]);
          const uint32_t rb = hready_a + 8u * (uint32_t)pb;
          for (uint32_t c = 0; c < cs; ++c) st_async_v2(mapa(hs_a + hoff, c), lo, hi, mapa(rb, c));
        }
        if (grow < p.m) {
          float* hrow = p.H + grow * p.ldh;
          if (col + 3 < p.l && ((reinterpret_cast<uintptr_t>(hrow + col) & 15) == 0)) {
            *reinterpret_cast<float4*>(hrow + col) = make_float4(vv[0], vv[1], vv[2], vv[3]);
          } else {
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
              if (col + qq < p.l) hrow[col + qq] = vv[qq];
          }
        }
      }
      grp_bar(g);
      // this panel's rows have been summed: the senders may reuse their slots
      if (e < (int)cs) arrive_relaxed_cluster(my_rfree, (uint32_t)e);
    }
    // ---------------------------------------------------- flush F slab
    if (FUSED) {
      bool okd = ok && my_pan > 0 && tc::mbar_wait(done2, 0, p.dev_err, abort_flag, false, lim);
      okd = grp_bar_and(g, okd);
      tc::tc_fence_after();
      if (okd) {
        const int fcols = p.l + (p.ones_col >= 0 ? 1 : 0);
        for (int t = g; t < RR_NT; t += 2) {
          const int64_t frow = (int64_t)slab0 + t * 128 + trow;
          for (int c16 = 0; c16 < L; c16 += 16) {
            float v[16];
            tc::tmem_ld16(tm_f + t * L + ((uint32_t)(32 * quad) << 16) + c16, v);
            if (frow < p.n) {
#pragma unroll
              for (int qq = 0; qq < 16; ++qq)
                if (c16 + qq < fcols) atomicAdd(&p.F[frow * p.ldf + c16 + qq], v[qq]);
            }
          }
        }
      }
    }
  }
  __syncwarp();
  // every MMA issued by this CTA has completed before TMEM is released
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done1, 0, nullptr, &never);
    if (FUSED) tc::mbar_wait(done2, 0, nullptr, &never);
  }
  tc::tc_fence_before();
  __syncthreads();
  // after an abort, give asynchronous stores still in flight towards the
  // peers time to land before any CTA of the cluster can leave
  if (*abort_flag) __nanosleep(100000);
  cluster_sync_all();            // no CTA leaves while others may touch its smem
  if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

// Host set-up of a kernel (shared-memory opt-in, cluster residency), done
// once per (kernel, device, cluster size, shared memory) and cached, so that
// a launch recorded into a CUDA graph makes no such call while the stream is
// capturing.  A first call that does happen under capture runs in relaxed
// capture mode.  Returns the number of clusters that can be resident, 0 if
// the configuration cannot run.
int cluster_setup(const void* kern, int cs, size_t smem, const cudaLaunchConfig_t& cfg0) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, size_t>, int> cache;
  int dev = 0;
  RPCA_CUDA_TRY(cudaGetDevice(&dev));
  const auto key = std::make_tuple(kern, dev, cs, smem);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  RPCA_CUDA_TRY(cudaThreadExchangeStreamCaptureMode(&mode));
  int max_cl = 0;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cs > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = cfg0;
    cfg.stream = nullptr;
    e = cudaOccupancyMaxActiveClusters(&max_cl, kern, &cfg);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    max_cl = 0;
  }
  cudaThreadExchangeStreamCaptureMode(&mode);
  cache[key] = max_cl;
  return max_cl;
}

template <int L, bool FUSED>
bool launch_rr(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  const int64_t n8 = round_up(a.n, 8);
  const int cs0 = (int)cdiv(a.n, RR_NC);
  int cs = 1;
  while (cs < cs0) cs <<= 1;
  if (cs > 16) return false;
  __nv_bfloat16* Xt = static_cast<__nv_bfloat16*>(a.work);
  if ((size_t)L * n8 * 2 > a.work_bytes) return false;
  CUtensorMap tmA, tmA2, tmX;
  if (!make_tmap_2d(&tmA, a.A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.m, a.n, a.lda, RR_BM, 64)) return false;
  if (!make_tmap_2d(&tmA2, a.A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.m, a.n, a.lda, 64, 64)) return false;
  if (!make_tmap_2d(&tmX, Xt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, L, n8, n8, L, 64)) return false;
  RRParams p;
  p.m = a.m;
  p.n = a.n;
  p.l = a.p;
  p.ones_col = a.ones_col;
  // X slab, two receive buffers (RR_BM x L/2 FP32 each), Hs[2], barriers
  const size_t fixed = 1024 + (size_t)RR_NBOX * L * 128 + (size_t)RR_BM * L * 4 + (FUSED ? 2 * RR_HS : 0) + 512;
  if (fixed + 4 * (size_t)RR_HBOX > RR_SMEM_LIMIT) return false;
  const int total = (int)((RR_SMEM_LIMIT - fixed) / RR_HBOX);
  if (FUSED) {
    p.nf = std::max(2, std::min(4, (total + 1) / 2));
    p.nh = std::min(8, total - p.nf);
  } else {
    p.nf = 0;
    p.nh = std::min(8, total);
  }
  if (p.nh < 2) return false;
  p.H = static_cast<float*>(a.H);
  p.ldh = a.ldh;
  p.corr = static_cast<const float*>(a.corr);
  p.F = static_cast<float*>(a.F);
  p.ldf = a.ldf;
  p.dev_err = dev_err;
  {
    const WaitTest wt = take_wait_test(0);
    p.wait_ns = wt.limit_ns;
    p.withhold = wt.withhold;
  }
  const size_t smem = fixed + (size_t)p.nh * RR_HBOX + (size_t)p.nf * RR_FST;
  auto kern = k_fused_rr<L, FUSED>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(RR_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(cs);
  const int max_cl = cluster_setup(reinterpret_cast<const void*>(kern), cs, smem, cfg);
  if (max_cl <= 0) return false;
  {
    int64_t cnt = (int64_t)L * n8;
    k_xt_bf16_rr<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(a.n, a.p, L, n8, static_cast<const float*>(a.X), a.ldx,
                                                           Xt);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  if (FUSED && a.F && !a.accumulate_f) {
    const int fcols = a.p + (a.ones_col >= 0 ? 1 : 0);
    RPCA_CUDA_TRY(cudaMemset2DAsync(a.F, a.ldf * 4, 0, fcols * 4, a.n, st));
  }
  const int64_t npan = cdiv(a.m, RR_BM);
  const int ncl = (int)std::max<int64_t>(1, std::min<int64_t>(max_cl, npan));
  cfg.gridDim = dim3(cs * ncl);
  if (getenv("RPCA_DEBUG"))
    fprintf(stderr, "[rpca] fused-rr L=%d fused=%d cs=%d max_clusters=%d clusters=%d smem=%zu nh=%d nf=%d\n", L,
            (int)FUSED, cs, max_cl, ncl, smem, p.nh, p.nf);
  RPCA_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, tmA, tmA2, tmX, p));
  count_launch();
  return true;
}

template <bool FUSED>
bool dispatch_rr(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  const int need = a.p + (a.ones_col >= 0 ? 1 : 0);
  if (need <= 16) return launch_rr<16, FUSED>(a, st, dev_err);
  if (need <= 32) return launch_rr<32, FUSED>(a, st, dev_err);
  if (need <= 64) return launch_rr<64, FUSED>(a, st, dev_err);
  return false;
}

}  // namespace

bool fused_pass_tc(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  if (a.dtype != RPCA_BF16) return false;
  if (a.mode != MODE_FUSED && a.mode != MODE_H) return false;
  if (a.shift || a.scale || !a.work) return false;
  if (a.ones_col >= 0 && a.ones_col != a.p) return false;
  if (a.mode == MODE_FUSED) return dispatch_rr<true>(a, st, dev_err);
  return dispatch_rr<false>(a, st, dev_err);
}

}  // namespace rpca
