// Step 4 (Section 3): one-sided Jacobi SVD of the w x w factor, FP32,
// spread over a thread-block cluster.
//
// Columns are grouped into 2P blocks of b columns (w <= 2Pb, missing columns
// are zero and never rotate).  CTA p of the P-CTA cluster holds the blocks at
// tournament positions p ("top") and 2P-1-p ("bottom").  In each round a CTA
// orthogonalises the column pairs between its two blocks; the first round
// of a sweep also covers the pairs inside each block.  Between rounds the
// blocks move by the circle method (position 0 fixed, positions 1..2P-1 a
// ring), written straight into the receiving CTA's shared memory, with one
// cluster barrier per round; after 2P-1 rounds every pair of columns has met
// once and every block is back at its starting position.  Threshold and
// noise floor are those of the single-CTA kernel in k_linalg.cu; the
// rotation angle is taken with the fast reciprocal and square root.
#include <algorithm>

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace rpca {
namespace {

constexpr int JC_THREADS = 512;   // 16 warps
constexpr int JC_WARPS = JC_THREADS / 32;
constexpr int JC_MAXB = 8;        // columns per block (named barriers 1..8, one per pair)
constexpr int JC_K = 4;           // rows per lane: w <= 256 and >= 2 warps per pair

// Rotation from the pair's Gram entries.  Only c^2 + s^2 = 1 must hold to
// rounding (c and s both come from t); t itself may be approximate, which
// only changes how much of the coupling one rotation removes, so the fast
// reciprocal and square root serve.
__device__ __forceinline__ void rotation(float al, float be, float ga, float& c, float& s) {
  const float zeta = __fdividef(be - al, 2.f * ga);
  const float h = fmaf(zeta, zeta, 1.f);
  const float t = copysignf(1.f, zeta) * __fdividef(1.f, fabsf(zeta) + h * rsqrtf(h));
  c = rsqrtf(fmaf(t, t, 1.f));
  s = c * t;
}

// Shared memory: buf[2][2 slots][b columns][B | J][ws]; red[2][JC_MAXB][JC_WARPS][3];
// offs[2][16]; nrm[16].
__global__ void __launch_bounds__(JC_THREADS, 1)
k_jacobi_cluster(int w, int b, const double* __restrict__ Bin, float* __restrict__ Jc, float tol,
                 int max_sweeps, uint32_t* dev_err) {
  cg::cluster_group cluster = cg::this_cluster();
  const int P = (int)cluster.num_blocks();
  const int cr = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long t_start = clock64();
  const int ws = (w + 3) & ~3;
  const int colf = 2 * ws;                     // floats per column (B then J)
  const int blkf = b * colf;                   // floats per block
  extern __shared__ __align__(16) float sm[];
  float* buf[2] = {sm, sm + 2 * blkf};
  float* red = sm + 4 * blkf;                  // [2][JC_MAXB][JC_WARPS][3]
  float* offs = red + 2 * JC_MAXB * JC_WARPS * 3;   // [2][16]
  float* nrm = offs + 32;                      // [16]

  // ---- load this CTA's two blocks: B columns from the row-major FP64 input,
  // J = identity columns
  int cur = 0;
  for (int s = 0; s < 2; ++s) {
    const int blk = s == 0 ? cr : 2 * P - 1 - cr;
    float* dst = buf[cur] + s * blkf;
    for (int e = tid; e < b * ws; e += JC_THREADS) {
      const int j = e / ws, r = e % ws;
      const int col = blk * b + j;
      const bool in = col < w && r < w;
      dst[j * colf + r] = in ? (float)Bin[(int64_t)r * w + col] : 0.f;
      dst[j * colf + ws + r] = (in && r == col) ? 1.f : 0.f;
    }
  }
  __syncthreads();

  // ---- largest column norm^2 over the cluster (noise floor of the couplings)
  {
    float m2 = 0.f;
    for (int c = warp; c < 2 * b; c += JC_WARPS) {
      const float* col = buf[cur] + c * colf;
      float s2 = 0.f;
      for (int r = lane; r < w; r += 32) s2 = fmaf(col[r], col[r], s2);
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      m2 = fmaxf(m2, s2);
    }
    __shared__ float wmax[JC_WARPS];
    if (lane == 0) wmax[warp] = m2;
    __syncthreads();
    if (tid < P) {
      float v = 0.f;
      for (int i = 0; i < JC_WARPS; ++i) v = fmaxf(v, wmax[i]);
      float* remote = cluster.map_shared_rank(nrm, tid);
      remote[cr] = v;
    }
    cluster.sync();
  }
  float nmax2 = 0.f;
  for (int i = 0; i < P; ++i) nmax2 = fmaxf(nmax2, nrm[i]);
  const float noise = 4.f * 5.96e-8f * sqrtf(nmax2);

  // pair-group of this warp
  const int wpp = JC_WARPS / b;                // warps per pair (>= 2)
  const int pi = warp / wpp, wi = warp % wpp;
  const bool pair_live = pi < b;
  const int gthreads = 32 * wpp;
  const int nrounds = 2 * P - 1;

  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    float local_off = 0.f;
    int sub = 0;                               // running sub-round counter (red parity)
    for (int rnd = 0; rnd < nrounds; ++rnd) {
      const bool full = rnd == 0;              // intra-block pairs once per sweep
      const int nsub = full ? 2 * b - 1 : b;
      float* B0 = buf[cur];
      for (int s = 0; s < nsub; ++s, ++sub) {
        int cp = 0, cq = 0;
        if (full) {
          const int n1 = 2 * b - 1;
          if (pi == 0) { cp = n1; cq = s; }
          else {
            cp = s + pi; if (cp >= n1) cp -= n1;
            cq = s - pi; if (cq < 0) cq += n1;
          }
        } else {
          cp = pi;
          cq = pi + s; if (cq >= b) cq -= b;
          cq += b;
        }
        float* bp = B0 + cp * colf;
        float* bq = B0 + cq * colf;
        float x[JC_K], y[JC_K];
        float al = 0.f, be = 0.f, ga = 0.f;
        if (pair_live) {
#pragma unroll
          for (int k = 0; k < JC_K; ++k) {
            const int r = wi * 32 + lane + k * gthreads;
            x[k] = r < w ? bp[r] : 0.f;
            y[k] = r < w ? bq[r] : 0.f;
            al = fmaf(x[k], x[k], al);
            be = fmaf(y[k], y[k], be);
            ga = fmaf(x[k], y[k], ga);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga += __shfl_xor_sync(0xffffffffu, ga, o);
          }
          float* rd = red + (((sub & 1) * JC_MAXB + pi) * JC_WARPS) * 3;
          if (lane == 0) {
            rd[wi * 3 + 0] = al;
            rd[wi * 3 + 1] = be;
            rd[wi * 3 + 2] = ga;
          }
          asm volatile("bar.sync %0, %1;" ::"r"(1 + pi), "r"(gthreads) : "memory");
          al = be = ga = 0.f;
          for (int i = 0; i < wpp; ++i) {
            al += rd[i * 3 + 0];
            be += rd[i * 3 + 1];
            ga += rd[i * 3 + 2];
          }
          // |ga| > tol sqrt(al be) and |ga| > noise sqrt(max(al, be)), squared
          const float g2 = ga * ga, ab = al * be;
          const bool rot = ab > 0.f && g2 > tol * tol * ab && g2 > noise * noise * fmaxf(al, be);
          if (rot) {
            local_off = 1.f;
            float c, sn;
            rotation(al, be, ga, c, sn);
            float* jp = bp + ws;
            float* jq = bq + ws;
#pragma unroll
            for (int k = 0; k < JC_K; ++k) {
              const int r = wi * 32 + lane + k * gthreads;
              if (r < w) {
                bp[r] = c * x[k] - sn * y[k];
                bq[r] = sn * x[k] + c * y[k];
                const float g = jp[r], h = jq[r];
                jp[r] = c * g - sn * h;
                jq[r] = sn * g + c * h;
              }
            }
          }
        }
        __syncthreads();
      }
      // ---- end of the sweep: publish this CTA's largest rotated coupling
      const bool last = rnd == nrounds - 1;
      if (last) {
        __shared__ float woff[JC_WARPS];
        if (lane == 0) woff[warp] = 0.f;
        __syncwarp();
        if (local_off > 0.f) atomicMax(reinterpret_cast<int*>(&woff[warp]), __float_as_int(local_off));
        __syncthreads();
        if (tid < P) {
          float v = 0.f;
          for (int i = 0; i < JC_WARPS; ++i) v = fmaxf(v, woff[i]);
          float* remote = cluster.map_shared_rank(offs + (sweep & 1) * 16, tid);
          remote[cr] = v;
        }
      }
      // ---- move the blocks (circle method) into the other buffer
      if (P > 1 || last) {
        float* nxt = buf[cur ^ 1];
        // destinations of slot 0 (top) and slot 1 (bottom)
        int d0 = cr, s0 = 0, d1 = cr, s1 = 1;
        if (P > 1) {
          if (cr == 0) { d0 = 0; s0 = 0; d1 = 1; s1 = 0; }
          else {
            if (cr == P - 1) { d0 = cr; s0 = 1; }
            else { d0 = cr + 1; s0 = 0; }
            d1 = cr - 1; s1 = 1;
          }
        }
        const float4* src = reinterpret_cast<const float4*>(B0);
        float4* dst0 = reinterpret_cast<float4*>(cluster.map_shared_rank(nxt, d0) + s0 * blkf);
        float4* dst1 = reinterpret_cast<float4*>(cluster.map_shared_rank(nxt, d1) + s1 * blkf);
        const int nv = blkf / 4;
        for (int e = tid; e < 2 * nv; e += JC_THREADS) {
          if (e < nv) dst0[e] = src[e];
          else dst1[e - nv] = src[e];
        }
        cluster.sync();
        cur ^= 1;
      }
    }
    float off = 0.f;
    for (int i = 0; i < P; ++i) off = fmaxf(off, offs[(sweep & 1) * 16 + i]);
    converged = off == 0.f;
  }
  if (cr == 0 && tid == 0) {
    if (!converged) atomicOr(dev_err, DEV_ERR_JACOBI);
    dev_err[8] = (uint32_t)sweep;
    dev_err[9] = (uint32_t)((clock64() - t_start) >> 10);
  }
  // ---- J columns out (every block is back at its starting position)
  for (int s = 0; s < 2; ++s) {
    const int blk = s == 0 ? cr : 2 * P - 1 - cr;
    const float* srcb = buf[cur] + s * blkf;
    for (int e = tid; e < b * w; e += JC_THREADS) {
      const int j = e / w, r = e % w;
      const int col = blk * b + j;
      if (col < w) Jc[(int64_t)col * w + r] = srcb[j * colf + ws + r];
    }
  }
}

}  // namespace

// Cluster shape for w: P CTAs (<= 16) with blocks of b <= 8 columns.  Narrow
// blocks over many CTAs: a sub-round's shared-memory traffic (two columns
// of B and of J per pair, read and written) is spread over more SMs.  (Blocks
// of 15 columns over 6 CTAs at w = 180, with 1024 threads, cut the cluster
// barriers per sweep from 29 to 11 but were 0.8 ms slower per call.)
static void cluster_shape(int w, int& P, int& b) {
  P = std::min(16, std::max(1, (w + 11) / 12));
  b = (w + 2 * P - 1) / (2 * P);
}

bool jacobi_cluster_f32(int w, const double* B, float* Jc, double tol, int max_sweeps, uint32_t* dev_err,
                        cudaStream_t st) {
  if (w < 2 || w > 256) return false;
  int P = 1, b = 1;
  cluster_shape(w, P, b);
  if (b > JC_MAXB || JC_WARPS / b < 2 || 32 * (JC_WARPS / b) * JC_K < w) return false;
  const int ws = (w + 3) & ~3;
  const size_t smem = (size_t)4 * b * 2 * ws * sizeof(float) + (size_t)2 * JC_MAXB * JC_WARPS * 3 * sizeof(float) +
                      48 * sizeof(float);
  RPCA_CUDA_TRY(cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (P > 8) RPCA_CUDA_TRY(cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(JC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_jacobi_cluster, &cfg) != cudaSuccess || ncl < 1) {
    cudaGetLastError();
    return false;
  }
  RPCA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_jacobi_cluster, w, b, B, Jc, (float)tol, max_sweeps, dev_err));
  count_launch();
  return true;
}

}  // namespace rpca
