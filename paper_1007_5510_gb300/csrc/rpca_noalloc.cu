// Allocation-free variant of the tensor-core fused pass (Step 1 products,
// Section 4.2): the pass's scratch, the transposed BF16 copy of X that its
// tensor map reads, lives in a fixed file-scope device array instead of a
// per-call cudaMalloc.  The paper has no counterpart to this entry point.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rpca {

namespace {

constexpr size_t kXtBytes = (size_t)RPCA_NOALLOC_MAX_P * RPCA_NOALLOC_MAX_N * 2;  // BF16 X^T
constexpr size_t kErrWords = 64;
static_assert(kXtBytes + kErrWords * sizeof(uint32_t) == RPCA_NOALLOC_SCRATCH_BYTES,
              "scratch layout and its declared size disagree");
static_assert(kXtBytes % 256 == 0, "error words must stay 256-byte aligned");

}  // namespace

// X^T in BF16 (up to 64 x 4096), then the device error words of the pass.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RPCA_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Address of the scratch on the current device, looked up once per device.
unsigned char* scratch_address() {
  int dev = 0;
  RPCA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Invalid("device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    RPCA_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) throw CudaFailure(cudaErrorInvalidSymbol, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  return g_addr[dev];
}

}  // namespace
}  // namespace rpca

using namespace rpca;

extern "C" rpca_status rpca_op_fused_pass_noalloc(int64_t m, int64_t n, int32_t p, const void* A, int64_t lda,
                                                  const float* X, int64_t ldx, float* H, int64_t ldh, float* F,
                                                  int64_t ldf, void* stream) {
  try {
    if (m < 1 || n < 1 || p < 1 || lda < n || ldx < p || ldh < p || (F && ldf < p)) return RPCA_EINVAL;
    if (n > RPCA_NOALLOC_MAX_N || p > RPCA_NOALLOC_MAX_P) return RPCA_EINVAL;  // beyond the fixed scratch
    if (!A || !X || !H) return RPCA_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      return RPCA_ENODEV;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = scratch_address();
    uint32_t* err = reinterpret_cast<uint32_t*>(base + kXtBytes);
    // The error words must start at zero; X^T is rewritten in full by the pass.
    RPCA_CUDA_TRY(cudaMemsetAsync(err, 0, kErrWords * sizeof(uint32_t), st));
    PassArgs a;
    a.dtype = RPCA_BF16;
    a.mode = F ? MODE_FUSED : MODE_H;
    a.A = A;
    a.lda = lda;
    a.m = m;
    a.n = n;
    a.X = X;
    a.ldx = ldx;
    a.p = p;
    a.H = H;
    a.ldh = ldh;
    a.F = F;
    a.ldf = ldf;
    a.work = base;
    a.work_bytes = kXtBytes;
    if (!fused_pass_tc(a, st, err)) return RPCA_EINVAL;  // alignment or cluster shape unsupported
    uint32_t flags = 0;
    RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, err, sizeof(flags), cudaMemcpyDeviceToHost, st));
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags & DEV_ERR_TIMEOUT) return RPCA_ETIMEOUT;
    return RPCA_OK;
  } catch (const CudaFailure& e) {
    if (e.code == cudaErrorNoDevice || e.code == cudaErrorInsufficientDriver) return RPCA_ENODEV;
    return RPCA_ECUDA;
  } catch (const Invalid&) {
    return RPCA_EINVAL;
  }
}
