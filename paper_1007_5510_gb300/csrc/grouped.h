// Grouped batch path: device-side descriptors and launchers (internal).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpca {
namespace grp {

// Limits of the grouped path (the per-problem path takes everything else).
constexpr int kMaxN = 1024;     // X^T of one problem fits the H pass's shared memory
constexpr int kMaxL = 32;       // N of the H pass
constexpr int kMaxW = 64;       // N of the T pass; w x w small matrices in shared memory
constexpr int kMaxNW = 45056;   // n * w FP32 of T in the Step-4 kernel's shared memory

// One problem, as every grouped kernel sees it.
struct alignas(16) GrpProblem {
  int64_t m, n;
  int32_t n64;                  // round_up(n, 64)
  int32_t k;
  float* H;                     // m x wp FP32 (wp = w rounded up to 4): H, then Q1 = H R1^-1
  __nv_bfloat16* Z;             // m x 64 BF16
  __nv_bfloat16* XT0;           // X^(0)^T images (fixed per batch)
  __nv_bfloat16* XT;            // X^(j)^T images, j >= 1
  float* X;                     // n x w FP32, ld w
  float* F;                     // n x ldy_l FP32
  float* T;                     // n x wp FP32
  double* G1;                   // w x w: H^T H, then R1 (upper)
  double* G2;                   // w x w: Q1^T Q1, then R2 (upper)
  double* G3;                   // w x w: T1^T T1
  float* R1inv;                 // w x w FP32 (upper)
  float* R2inv;                 // w x w FP32 (upper)
  float* MU;                    // w x k FP32
  float* U;                     // user m x k FP32 (ldu) or null
  float* V;                     // user n x k FP32 (ldv) or null
  double* S;                    // user k FP64 or null
  int64_t ldu, ldv;
  uint32_t* perr;               // this problem's error word
};

// T-pass work item: problem p, 64-row groups [sub0, sub0 + nsub).
struct GrpTItem {
  int32_t p, sub0, nsub, pad;
};

// Row-range work item of the SIMT kernels over the m side.
struct GrpRItem {
  int32_t p;
  int32_t r0;
  int32_t nrows;
  int32_t pad;
};

struct HPassArgs {
  const CUtensorMap* tmA;       // one map per problem (device array)
  int nstages;
  uint32_t xbytes;              // shared-memory bytes of the X^T images
  int w, l, col0;               // H pitch (wp) and columns [col0, col0 + l)
  int write_z;                  // also write Z = bf16(H^(j))
  int xt_first;                 // read XT0 (j = 0) instead of XT
  int pf;                       // L2 prefetch distance in ring stages (0: none)
  uint32_t* err;
};

struct TPassArgs {
  const CUtensorMap* tmA;       // box 64 rows x 64 columns
  const CUtensorMap* tmZ;       // box 64 rows x 64 columns
  int nstages;
  int tmem_cols;                // power of two >= ntile_max * npad
  int npad;                     // MMA N (multiple of 16, <= 64)
  int ncols;                    // columns of Y that receive sums
  int ldy;
  int mode_t;                   // 0: Y = F, 1: Y = T
  int pf;                       // L2 prefetch distance in ring stages (0: none)
  uint32_t* err;
};

// Launchers (k_grouped.cu, k_grouped_small.cu).  All enqueue on `st`.
void launch_hpass(const GrpProblem* probs, const int32_t* item_p, const int32_t* item_t, int64_t nitems,
                  const HPassArgs& a, int grid, cudaStream_t st);
void launch_tpass(const GrpProblem* probs, const GrpTItem* items, int64_t nitems, const TPassArgs& a, int grid,
                  cudaStream_t st);
size_t hpass_smem(uint32_t xbytes, int nstages);
size_t tpass_smem(int nstages);

// X^(j+1) = orth(F - X_{<=j} X_{<=j}^T F) (j >= 0), or X^(0) = orth(G) with G
// given in F (j = -1); writes the block into X and its images into XT (XT0
// for j = -1).  One CTA per problem.
void launch_orth(const GrpProblem* probs, int count, int j, int l, int w, int ldf, int max_n, uint32_t* err,
                 cudaStream_t st);
// G1 += H^T H over the row items.
void launch_gram(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, uint32_t* err,
                 cudaStream_t st);
// which = 1: G1 -> R1 (in place) and R1inv; which = 2: G2 -> R2 and R2inv.
void launch_chol(const GrpProblem* probs, int count, int w, int which, uint32_t* err, cudaStream_t st);
// Q1 = H R1^-1 over H, Z = bf16(Q1), G2 += Q1^T Q1 over the row items.
void launch_apply(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, uint32_t* err,
                  cudaStream_t st);
// G3 += T1^T T1 over row items of the n side.
void launch_gram_t(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, uint32_t* err,
                   cudaStream_t st);
// Steps 4-6 on the n side from G3: S, V and MU.
void launch_svd(const GrpProblem* probs, int count, int w, int ldt, int max_n, uint32_t* err, cudaStream_t st);
// U = Q1 MU over the row items.
void launch_u(const GrpProblem* probs, const GrpRItem* items, int64_t nitems, int w, int k, uint32_t* err,
              cudaStream_t st);

}  // namespace grp
}  // namespace rpca

// ------------------------------------------------------------------ host
#include <string>
#include <vector>

#include "../../include/rpca.h"

namespace rpca {
namespace grp {

// Launch parameters of the grouped kernels (the batch autotuner's knobs).
struct Tuning {
  int h_stages = 4;       // H pass TMA ring stages (32 KB each)
  int t_stages = 5;       // T pass TMA ring stages (40 KB each)
  int t_rows = 2048;      // rows per T-pass item (multiple of 64)
  int r_rows = 2048;      // rows per row-kernel item
  int pf = 0;             // L2 prefetch distance of the H and T passes (stages; measured slower)
};

struct GroupedBatch;

// Whether every problem fits the grouped kernels (BF16 device matrices, no
// flags, m >= n, shared k, l, i, n <= kMaxN, l <= kMaxL, w <= kMaxW,
// n w <= kMaxNW); *why names the first reason it does not.
bool grouped_eligible(int count, const rpca_problem* problems, std::string* why);
// G[p]: problem p's n x l test matrix (FP64, row-major).  Allocates every
// buffer and forms X^(0) = orth(G) once.
GroupedBatch* grouped_create(int count, const rpca_problem* problems, const std::vector<std::vector<double>>& G,
                             cudaStream_t st);
void grouped_destroy(GroupedBatch* g);
// False (nothing enqueued) when a matrix's layout does not fit TMA (base
// 16-byte aligned, ld a multiple of 8); otherwise enqueues a whole run.
bool grouped_run(GroupedBatch* g, const rpca_matrix* A, void* const* U, const int64_t* ldu, double* const* S,
                 void* const* V, const int64_t* ldv, cudaStream_t st);
// After grouped_run: synchronises st; RPCA_OK, or the first failing
// problem's status with *bad and *msg set.
rpca_status grouped_check(GroupedBatch* g, cudaStream_t st, int* bad, std::string* msg);
void grouped_set_tuning(GroupedBatch* g, const Tuning& t);
Tuning grouped_tuning(const GroupedBatch* g);
// Kernels one run launches.
int grouped_launches(const GroupedBatch* g);

}  // namespace grp
}  // namespace rpca
