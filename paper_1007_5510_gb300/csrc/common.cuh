// Shared device/host helpers for the PCA library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <atomic>
#include <string>

#include "../../include/rpca.h"

namespace rpca {

// Launch counter (reported through rpca_kernel_launches).
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Device-side error word bits (ctx->dev_err).
enum : uint32_t {
  DEV_ERR_BREAKDOWN = 1u,   // Cholesky failed even after the shift
  DEV_ERR_TIMEOUT = 2u,     // a bounded wait gave up
  DEV_ERR_SHIFTED = 4u,     // informational: a shifted Cholesky was used
  DEV_ERR_JACOBI = 8u,      // Jacobi SVD hit its sweep limit
};

struct Err {
  rpca_status st = RPCA_OK;
  std::string msg;
};

#define RPCA_CUDA_TRY(expr)                                                  \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) {                                                 \
      throw ::rpca::CudaFailure(_e, #expr, __FILE__, __LINE__);              \
    }                                                                        \
  } while (0)

struct CudaFailure {
  cudaError_t code;
  std::string what;
  CudaFailure(cudaError_t c, const char* expr, const char* file, int line)
      : code(c) {
    what = std::string(cudaGetErrorString(c)) + " in " + expr + " at " + file + ":" +
           std::to_string(line);
  }
};

struct Invalid {
  std::string what;
  explicit Invalid(std::string w) : what(std::move(w)) {}
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// -------------------------------------------------------------- conversions
template <typename T> __device__ __forceinline__ float to_f32(T x);
template <> __device__ __forceinline__ float to_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <> __device__ __forceinline__ float to_f32<__nv_fp8_e4m3>(__nv_fp8_e4m3 x) {
  return float(x);
}

// Storage element for each dtype.
template <int DT> struct Storage;
template <> struct Storage<RPCA_F64> { using T = double; };
template <> struct Storage<RPCA_F32> { using T = float; };
template <> struct Storage<RPCA_BF16> { using T = __nv_bfloat16; };
template <> struct Storage<RPCA_FP8E4M3> { using T = __nv_fp8_e4m3; };

inline size_t dtype_bytes(rpca_dtype d) {
  switch (d) {
    case RPCA_F64: return 8;
    case RPCA_F32: return 4;
    case RPCA_BF16: return 2;
    case RPCA_FP8E4M3: return 1;
  }
  return 0;
}

inline int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace rpca
