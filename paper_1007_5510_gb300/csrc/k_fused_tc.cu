// Fused Step-1 pass on tensor cores (tcgen05 + TMA + cluster DSMEM), BF16 A.
//
// One pass of Section 3's Step 1 read once from HBM (Section 4.2's row-block
// streaming): for each 128-row panel A_b
//     H_b = A_b X                  (stored, FP32)
//     F  += A_b^T H_b              (FP32 accumulators in TMEM)
// A thread-block cluster of CS CTAs shares each panel: CTA c owns the column
// slab [c*NC, (c+1)*NC), NC = NT*128, keeps X[slab] (BF16, K-major) resident
// in shared memory and F[slab] in tensor memory for the whole kernel.
//   GEMM1  P_c = A_b[:, slab] X[slab]          M=128 rows, N=L, K=NC (K-major A)
//   reduce H_b = sum_c P_c across the cluster  (distributed shared memory)
//   GEMM2  F[slab] += A_b[:, slab]^T H_b       M=128 cols, N=L, K=128 (MN-major A)
// Both GEMMs read the same TMA-staged tile of A.  Each CTA reduces 128/CS rows
// of H_b: it pulls those rows of every CTA's partial, adds them, stores them
// to H and pushes their BF16 copy into every CTA's GEMM2 operand buffer.
//
// Warp roles (6 warps): warp 0 lane 0 TMA producer, warp 1 lane 0 MMA issuer,
// warps 2-5 TMEM drain / reduction / F flush.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rpca {
namespace {

constexpr int FP_THREADS = 192;
constexpr int FP_BM = 128;

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
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
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// Named barrier over the 4 epilogue warps that also ANDs a predicate, so an
// abort decision is uniform across them.
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
__device__ __forceinline__ uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(cta));
  return r;
}
// Remote shared-memory load (no compiler barrier, so a batch of independent
// loads is issued back to back and their latencies overlap).
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}
// Bulk copy of `bytes` (multiple of 16) from this CTA's shared memory to a
// peer's (dst and its mbarrier rbar are shared::cluster addresses), counted
// on rbar; the source may be reused after cp.async.bulk.wait_group.read.
__device__ __forceinline__ void bulk_to_peer(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t rbar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "r"(src), "r"(bytes), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_cluster_b64(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared::cluster.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// X (n x l, FP32, ldx) -> Xt (L x n8, BF16): row j holds column j of X.
__global__ void k_xt_bf16(int64_t n, int l, int L, int64_t n8, const float* __restrict__ X, int64_t ldx,
                          __nv_bfloat16* __restrict__ Xt) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * n8) return;
  int j = (int)(e / n8);
  int64_t r = e % n8;
  float v = (j < l && r < n) ? X[r * ldx + j] : 0.f;
  Xt[e] = __float2bfloat16_rn(v);
}

struct FusedParams {
  int64_t m, n;
  int l;            // real columns of X / H
  int ones_col;     // -1 or column index (< L) of an all-ones H column
  int nstages;
  uint32_t stage_bytes, xs_bytes;
  float* H;
  int64_t ldh;
  const float* corr;   // l values subtracted from every H row, or null
  float* F;            // n x (l [+1]) FP32, accumulated (zeroed by the host)
  int64_t ldf;
  uint32_t* dev_err;
};

// Shared-memory layout (bytes from a 1024-aligned base):
//   [X slab: L x NC BF16, K-major SW128, NC/64 boxes of L rows]
//   [stages: nstages x (NC/64 boxes of 128 rows x 128 B)]
//   [Pst: 128 rows x L FP32, 16-byte chunks XOR-swizzled by row]
//   [Hs[2]: 128 rows x 128 B BF16, SW128 MN-major operand]
//   [Hst: this CTA's rows of H_b in BF16 (128/CS rows x 128 B), staged for
//    the bulk copies into every CTA's Hs]
//   [barriers]
template <int L, int NT, bool FUSED>
__global__ void __launch_bounds__(FP_THREADS, 1)
k_fused_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
             const FusedParams p) {
  constexpr int NC = NT * 128;
  constexpr int NBOX = NC / 64;
  constexpr uint32_t ABOX = FP_BM * 128;         // bytes of one 128 x 64 BF16 box
  constexpr uint32_t XBOX = L * 128;             // bytes of one L x 64 BF16 box
  constexpr uint32_t PST_BYTES = FP_BM * L * 4;
  constexpr uint32_t HS_BYTES = FP_BM * 128;
  constexpr uint32_t TMEM_COLS = ((2 + NT) * L <= 128) ? 128 : ((2 + NT) * L <= 256) ? 256 : 512;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xs = smem;
  unsigned char* stages = xs + p.xs_bytes;
  unsigned char* pst = stages + (size_t)p.nstages * p.stage_bytes;
  unsigned char* hs = pst + PST_BYTES;
  const uint32_t hst_bytes = (uint32_t)(FP_BM / cluster_nctarank()) * 128;   // rows of this CTA
  unsigned char* hst = hs + 2 * HS_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(hst + hst_bytes);
  uint64_t* full = bars;                      // [nstages]
  uint64_t* empty = full + p.nstages;         // [nstages]
  uint64_t* pfull = empty + p.nstages;        // [2]
  uint64_t* pempty = pfull + 2;               // [2]
  uint64_t* hready = pempty + 2;              // [2]
  uint64_t* hfree = hready + 2;               // [2]
  uint64_t* pready = hfree + 2;               // [1]
  uint64_t* pfree = pready + 1;               // [1]
  uint64_t* xfull = pfree + 1;                // [1]
  uint64_t* done = xfull + 1;                 // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t cs = cluster_nctarank();
  const uint32_t crank = cluster_rank();
  const uint32_t cid = cluster_id_x(), ncl = nclusters_x();
  const int64_t npan = (p.m + FP_BM - 1) / FP_BM;
  const int64_t my_pan = (npan > cid) ? (npan - cid + ncl - 1) / ncl : 0;
  const uint16_t cmask = (uint16_t)((1u << cs) - 1u);
  const int rpc = FP_BM / (int)cs;            // rows of H reduced by this CTA
  const int row0 = (int)crank * rpc;

  if (tid == 0) {
    for (int s = 0; s < p.nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int x = 0; x < 2; ++x) {
      tc::mbar_init(&pfull[x], 1);
      tc::mbar_init(&pempty[x], 4);
      tc::mbar_init(&hready[x], 1);   // armed with the byte count of H_b
      tc::mbar_init(&hfree[x], cs);
    }
    tc::mbar_init(pready, cs);
    tc::mbar_init(pfree, cs);
    tc::mbar_init(xfull, 1);
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    if (FUSED) {
      tc::mbar_arrive_expect_tx(&hready[0], HS_BYTES);
      tc::mbar_arrive_expect_tx(&hready[1], HS_BYTES);
    }
    tc::tma_prefetch(&tmA);
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
  const uint32_t tm_p = tmem;                    // P[0], P[1]: columns 0..2L
  const uint32_t tm_f = tmem + 2 * L;            // F slab tiles: NT x L columns

  if (warp == 0) {
    if (lane == 0) {
      // --------------------------------------------------------- producer
      tc::mbar_arrive_expect_tx(xfull, p.xs_bytes);
      for (int j = 0; j < NBOX; ++j)
        tc::tma_load_2d(xs + (size_t)j * XBOX, &tmX, xfull, (int32_t)(crank * NC + 64 * j), 0);
      int64_t it = 0;
      for (; it < my_pan; ++it) {
        const int s = (int)(it % p.nstages);
        const uint32_t ph = (uint32_t)((it / p.nstages) & 1);
        if (!tc::mbar_wait(&empty[s], ph ^ 1u, p.dev_err, abort_flag)) break;
        unsigned char* st = stages + (size_t)s * p.stage_bytes;
        const int32_t r0 = (int32_t)((cid + it * ncl) * FP_BM);
        tc::mbar_arrive_expect_tx(&full[s], p.stage_bytes);
        for (int j = 0; j < NBOX; ++j)
          tc::tma_load_2d(st + (size_t)j * ABOX, &tmA, &full[s], (int32_t)(crank * NC + 64 * j), r0);
      }
      // drain: let in-flight copies land before the CTA can exit
      for (int64_t q = (it > p.nstages ? it - p.nstages : 0); q < it; ++q) {
        volatile int never = 0;
        tc::mbar_wait(&full[q % p.nstages], (uint32_t)((q / p.nstages) & 1), nullptr, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA
      constexpr uint32_t idesc1 = tc::idesc_make(1u, 0u, 0u, 128u, (uint32_t)L);
      constexpr uint32_t idesc2 = tc::idesc_make(1u, 1u, 1u, 128u, (uint32_t)L);
      const uint32_t xs_a = tc::smem_u32(xs);
      const uint32_t hs_a = tc::smem_u32(hs);
      bool okx = tc::mbar_wait(xfull, 0, p.dev_err, abort_flag);
      int64_t it = 0;
      for (; okx && it <= my_pan; ++it) {
        if (it < my_pan) {
          // GEMM1 for panel it
          const int s = (int)(it % p.nstages);
          const int pb = (int)(it & 1);
          if (!tc::mbar_wait(&full[s], (uint32_t)((it / p.nstages) & 1), p.dev_err, abort_flag)) break;
          if (!tc::mbar_wait(&pempty[pb], (uint32_t)(((it >> 1) & 1) ^ 1), p.dev_err, abort_flag)) break;
          tc::tc_fence_after();
          const uint32_t sa = tc::smem_u32(stages + (size_t)s * p.stage_bytes);
#pragma unroll
          for (int kk = 0; kk < NC / 16; ++kk) {
            const uint32_t koff = (uint32_t)(kk >> 2) * ABOX + (uint32_t)(kk & 3) * 32;
            const uint32_t xoff = (uint32_t)(kk >> 2) * XBOX + (uint32_t)(kk & 3) * 32;
            tc::mma_f16(tm_p + pb * L, tc::sdesc_sw128(sa + koff, 16, 1024),
                        tc::sdesc_sw128(xs_a + xoff, 16, 1024), idesc1, kk > 0 ? 1u : 0u);
          }
          tc::mma_commit(&pfull[pb]);
          if (!FUSED) tc::mma_commit(&empty[s]);
        }
        if (FUSED && it >= 1) {
          // GEMM2 for panel it-1 once its H is in place
          const int64_t jt = it - 1;
          const int s = (int)(jt % p.nstages);
          const int x = (int)(jt & 1);
          if (!tc::mbar_wait(&hready[x], (uint32_t)((jt >> 1) & 1), p.dev_err, abort_flag, true)) break;
          tc::tc_fence_after();
          // next use of this buffer (panel jt + 2): all CS owners' rows
          tc::mbar_arrive_expect_tx(&hready[x], HS_BYTES);
          const uint32_t sa = tc::smem_u32(stages + (size_t)s * p.stage_bytes);
          const uint32_t hb = hs_a + x * HS_BYTES;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
#pragma unroll
            for (int kr = 0; kr < FP_BM / 16; ++kr) {
              tc::mma_f16(tm_f + t * L, tc::sdesc_sw128(sa + 2 * t * ABOX + kr * 2048, ABOX, 1024),
                          tc::sdesc_sw128(hb + kr * 2048, HS_BYTES, 1024), idesc2,
                          (jt > 0 || kr > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty[s]);
          tc::mma_commit_multicast(&hfree[x], cmask);
        }
      }
      tc::mma_commit(done);
    }
  } else {
    // ----------------------------------------- drain, reduce, distribute
    const int e = tid - 64;                       // 0..127
    const int trow = 32 * (warp & 3) + lane;      // TMEM lane = panel row
    const uint32_t pst_a = tc::smem_u32(pst);
    const uint32_t hs_a = tc::smem_u32(hs);
    constexpr int CPR = L / 4;                    // float4 chunks per row (power of 2)
    const int nch = rpc * CPR;
    bool ok = true;
    for (int64_t it = 0; it < my_pan; ++it) {
      const int pb = (int)(it & 1);
      const int x = (int)(it & 1);
      const int64_t r0 = (cid + it * ncl) * FP_BM;
      ok = tc::mbar_wait(&pfull[pb], (uint32_t)((it >> 1) & 1), p.dev_err, abort_flag);
      ok = ok && tc::mbar_wait(pfree, (uint32_t)(((it - 1) & 1)), p.dev_err, abort_flag, true);
      ok = epi_bar_and(ok);
      if (!ok) break;
      tc::tc_fence_after();
      // TMEM -> Pst (this CTA's partial of H_b), 16-byte chunks swizzled by row
#pragma unroll
      for (int c16 = 0; c16 < L; c16 += 16) {
        float v[16];
        tc::tmem_ld16(tm_p + pb * L + ((uint32_t)(32 * (warp & 3)) << 16) + c16, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int chunk = (c16 >> 2) + q;
          const int pc = chunk ^ (trow & (CPR - 1));
          float4* dst = reinterpret_cast<float4*>(pst + (size_t)trow * L * 4 + pc * 16);
          *dst = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&pempty[pb]);
      epi_bar();
      // one thread per destination CTA: the release-arrives run in parallel
      if (e < (int)cs) tc::mbar_arrive_cluster(pready, (uint32_t)e);
      ok = tc::mbar_wait(pready, (uint32_t)(it & 1), p.dev_err, abort_flag, true);
      if (FUSED)
        ok = ok && tc::mbar_wait(&hfree[x], (uint32_t)(((it >> 1) & 1) ^ 1), p.dev_err, abort_flag, true);
      // the staged rows of the previous panel have been read by their copies
      if (FUSED && e < (int)cs) tc::bulk_wait_read0();
      ok = epi_bar_and(ok);
      if (!ok) break;
      // rows [row0, row0 + rpc) of H_b: sum the cluster's partials, apply the
      // centring corrections, store, and push BF16 copies to every CTA
      for (int ch = e; ch < nch; ch += 128) {
        const int rr = row0 + ch / CPR, chunk = ch % CPR, col = chunk * 4;
        const uint32_t off = (uint32_t)(rr * L * 4 + ((chunk ^ (rr & (CPR - 1))) * 16));
        float4 sacc = make_float4(0.f, 0.f, 0.f, 0.f);
        {
          float4 v[16];   // every peer's chunk in flight at once
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < (int)cs) v[q] = ld_cluster_f4(mapa(pst_a + off, (uint32_t)q));
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < (int)cs) { sacc.x += v[q].x; sacc.y += v[q].y; sacc.z += v[q].z; sacc.w += v[q].w; }
        }
        const int64_t grow = r0 + rr;
        float vv[4] = {sacc.x, sacc.y, sacc.z, sacc.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cc = col + q;
          if (p.corr && cc < p.l) vv[q] -= p.corr[cc];
          if (grow >= p.m || cc >= p.l) vv[q] = 0.f;
          if (cc == p.ones_col && grow < p.m) vv[q] = 1.f;
        }
        if (grow < p.m) {
          float* hrow = p.H + grow * p.ldh;
          if (col + 3 < p.l && ((reinterpret_cast<uintptr_t>(hrow + col) & 15) == 0)) {
            *reinterpret_cast<float4*>(hrow + col) = make_float4(vv[0], vv[1], vv[2], vv[3]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (col + q < p.l) hrow[col + q] = vv[q];
          }
        }
        if (FUSED) {
          // row rr of Hs, swizzled as in its destination
          const uint32_t hoff = (uint32_t)((rr - row0) * 128 + ((((col >> 3) ^ (rr & 7))) << 4) + (col & 7) * 2);
          *reinterpret_cast<uint2*>(hst + hoff) = make_uint2(pack_bf16(vv[0], vv[1]),
                                                                           pack_bf16(vv[2], vv[3]));
        }
      }
      epi_bar();
      // the partials of this panel have been read: the senders may reuse Pst
      if (e < (int)cs) tc::mbar_arrive_cluster(pfree, (uint32_t)e);
      if (FUSED) {
        // (GEMM2 reads columns [0, L) of Hs only)
        tc::fence_proxy_async_smem();
        epi_bar();
        if (e < (int)cs) {
          bulk_to_peer(mapa(hs_a + x * HS_BYTES + (uint32_t)row0 * 128, (uint32_t)e),
                       tc::smem_u32(hst), (uint32_t)rpc * 128,
                       mapa(tc::smem_u32(&hready[x]), (uint32_t)e));
          tc::bulk_commit();
        }
      }
    }
    // staged rows must stay until the copies have read them
    if (FUSED && e < (int)cs) tc::bulk_wait_read0();
    // ---------------------------------------------------- flush F slab
    if (FUSED) {
      bool okd = ok && my_pan > 0 && tc::mbar_wait(done, 0, p.dev_err, abort_flag);
      okd = epi_bar_and(okd);
      tc::tc_fence_after();
      if (okd) {
        for (int t = 0; t < NT; ++t) {
          const int64_t frow = (int64_t)crank * NC + t * 128 + trow;
          for (int c16 = 0; c16 < L; c16 += 16) {
            float v[16];
            tc::tmem_ld16(tm_f + t * L + ((uint32_t)(32 * (warp & 3)) << 16) + c16, v);
            if (frow < p.n) {
              const int fcols = p.l + (p.ones_col >= 0 ? 1 : 0);
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (c16 + q < fcols) atomicAdd(&p.F[frow * p.ldf + c16 + q], v[q]);
            }
          }
        }
      }
    }
  }
  __syncwarp();
  // all MMAs issued by this CTA have completed before TMEM is released
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done, 0, nullptr, &never);
  }
  tc::tc_fence_before();
  __syncthreads();
  cluster_sync_all();            // no CTA leaves while others may touch its smem
  if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

int g_sms = 0;

template <int L, int NT, bool FUSED>
bool launch_fused(const PassArgs& a, cudaStream_t st, uint32_t* dev_err, int cs) {
  constexpr int NC = NT * 128;
  const int64_t n8 = round_up(a.n, 8);
  __nv_bfloat16* Xt = static_cast<__nv_bfloat16*>(a.work);
  if ((size_t)L * n8 * 2 > a.work_bytes) return false;
  CUtensorMap tmA, tmX;
  if (!make_tmap_2d(&tmA, a.A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.m, a.n, a.lda, FP_BM, 64)) return false;
  if (!make_tmap_2d(&tmX, Xt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, L, n8, n8, L, 64)) return false;
  {
    int64_t cnt = (int64_t)L * n8;
    k_xt_bf16<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(a.n, a.p, L, n8, static_cast<const float*>(a.X), a.ldx, Xt);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  FusedParams p;
  p.m = a.m;
  p.n = a.n;
  p.l = a.p;
  p.ones_col = a.ones_col;
  p.xs_bytes = (uint32_t)(NC / 64) * L * 128;
  p.stage_bytes = (uint32_t)(NC / 64) * FP_BM * 128;
  const size_t fixed = 1024 + p.xs_bytes + (size_t)FP_BM * L * 4 + 2 * (size_t)FP_BM * 128 +
                       (size_t)(FP_BM / cs) * 128 + 256;
  const size_t budget = 227 * 1024;
  p.nstages = (int)std::min<size_t>(4, (budget - fixed) / p.stage_bytes);
  if (p.nstages < 2) return false;
  p.H = static_cast<float*>(a.H);
  p.ldh = a.ldh;
  p.corr = static_cast<const float*>(a.corr);
  p.F = static_cast<float*>(a.F);
  p.ldf = a.ldf;
  p.dev_err = dev_err;
  const size_t smem = fixed + (size_t)p.nstages * p.stage_bytes;
  auto kern = k_fused_bf16<L, NT, FUSED>;
  RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (cs > 8) RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  if (FUSED && a.F && !a.accumulate_f) {
    const int fcols = a.p + (a.ones_col >= 0 ? 1 : 0);
    RPCA_CUDA_TRY(cudaMemset2DAsync(a.F, a.ldf * 4, 0, fcols * 4, a.n, st));
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(FP_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // number of clusters: as many as can be resident at once, at most one per panel
  cfg.gridDim = dim3(cs);
  int max_cl = 0;
  if (cudaOccupancyMaxActiveClusters(&max_cl, kern, &cfg) != cudaSuccess || max_cl <= 0) {
    cudaGetLastError();
    return false;
  }
  const int64_t npan = cdiv(a.m, FP_BM);
  const int ncl = (int)std::max<int64_t>(1, std::min<int64_t>(max_cl, npan));
  cfg.gridDim = dim3(cs * ncl);
  if (getenv("RPCA_DEBUG"))
    fprintf(stderr, "[rpca] fused L=%d NT=%d fused=%d cs=%d max_clusters=%d clusters=%d smem=%zu stages=%d\n", L,
            NT, (int)FUSED, cs, max_cl, ncl, smem, p.nstages);
  RPCA_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, tmA, tmX, p));
  count_launch();
  return true;
}

template <int L, bool FUSED>
bool dispatch_nt(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  // smallest slab width that keeps the cluster within 16 CTAs
  for (int nt : {1, 2, 4}) {
    const int cs = (int)cdiv(a.n, nt * 128);
    if (cs > 16) continue;
    if ((2 + nt) * L > 512) return false;
    if (128 % cs != 0) {
      // the reduction splits 128 rows evenly: round the cluster up
      int c2 = 1;
      while (c2 < cs) c2 <<= 1;
      if (c2 > 16) continue;
    }
    int csp = 1;
    while (csp < cs) csp <<= 1;      // 1, 2, 4, 8, 16 (extra CTAs own empty slabs)
    if (nt == 1) return launch_fused<L, 1, FUSED>(a, st, dev_err, csp);
    if (nt == 2) return launch_fused<L, 2, FUSED>(a, st, dev_err, csp);
    return launch_fused<L, 4, FUSED>(a, st, dev_err, csp);
  }
  return false;
}

template <bool FUSED>
bool dispatch_l(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  const int need = a.p + (a.ones_col >= 0 ? 1 : 0);
  if (need <= 16) return dispatch_nt<16, FUSED>(a, st, dev_err);
  if (need <= 32) return dispatch_nt<32, FUSED>(a, st, dev_err);
  if (need <= 64) return dispatch_nt<64, FUSED>(a, st, dev_err);
  return false;
}

}  // namespace

bool fused_pass_tc(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  if (a.dtype != RPCA_BF16) return false;
  // the L2 re-read form first (RPCA_FUSED_HELD=1 selects this held-tile form)
  static const bool held = getenv("RPCA_FUSED_HELD") != nullptr;
  if (!held && fused_pass_rr(a, st, dev_err)) return true;
  if (a.mode != MODE_FUSED && a.mode != MODE_H) return false;
  if (a.shift || a.scale || !a.work) return false;
  if (a.ones_col >= 0 && a.ones_col != a.p) return false;
  if (a.mode == MODE_FUSED) return dispatch_l<true>(a, st, dev_err);
  return dispatch_l<false>(a, st, dev_err);
}

}  // namespace rpca
