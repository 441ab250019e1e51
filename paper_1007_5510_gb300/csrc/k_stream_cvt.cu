// Tensor-core streamed passes for A stored in FP32 or FP8-e4m3, and for
// any storage with a centring shift (tcgen05 + TMA, sm_103a).
//
// The passes of Section 3 -- Step 1's H^(j) = A_c X and F = A_c^T H^(j),
// Step 3's T = A_c^T Q -- with A_c = A diag(scale) - 1 shift^T (Section 1's
// column centring as a shift, never materialised).  The tensor cores take
// BF16 operands (kind::f16, FP32 accumulation in tensor memory), so every
// A tile passes through converter warps between its TMA load and the MMA:
//   FP32 (or any storage with a shift or a per-column scale):
//       v = a * scale_c - shift_c  (one FMA in FP32; exact for a - shift
//       when the shift is close to a, Sterbenz), then v = hi + lo with
//       hi = bf16(v), lo = bf16(v - hi): 16 significant bits;
//   FP8-e4m3 without shift: v = a, widened exactly to BF16 (the scale is
//       folded into the small operand and into the result rows instead).
// The small operand (X, H or Q) is split the same way into BF16 slices, and
// the products hi*hi + lo*hi + hi*lo (FP32 data) or a*hi + a*lo (exact
// BF16 A) are accumulated, which leaves ~2^-16 relative error per product:
// FP32-class results from BF16 tensor cores.
//
// For FP32 tiles the conversion is in place: a TMA box pair of R rows x 2x32
// FP32 (two 128-byte-swizzled boxes) becomes R rows x 64 BF16 hi then R rows
// x 64 BF16 lo, each in the layout a BF16 TMA box of 64 columns would have.
// Every converter thread owns one tile row, so it reads a row of the raw
// boxes and writes the same row of the two outputs: no other thread touches
// those bytes.  FP8 and shifted BF16 tiles convert into a separate buffer.
//
// Kernels
//   k_hpass_cvt   H = A_c X (128-row panels, persistent CTAs, K = n in
//                 64-column steps; X^T slices streamed from L2; accumulator
//                 double-buffered in tensor memory so a panel's epilogue
//                 overlaps the next panel's MMAs).  Also writes the BF16
//                 slices of H that the F pass reads.
//   k_tpass_cvt   T = A_c^T Y (column slabs of NT*128, row sub-panels of 64,
//                 the slab's accumulator resident in tensor memory, added to
//                 the output once at the end), Y given as BF16 slices.
// Every wait is bounded (tc_common.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rpca {
namespace {

// Source formats of A as the converter sees them.
enum CvtSrc : int {
  SRC_F32 = 0,      // FP32 storage: v = a*scale - shift, split hi/lo
  SRC_FP8 = 1,      // FP8-e4m3, no shift: widened exactly (scale folded outside)
  SRC_FP8_SH = 2,   // FP8-e4m3 with a shift: v = a*scale - shift, split hi/lo
  SRC_BF16_SH = 3,  // BF16 with a shift: v = a*scale - shift, split hi/lo
};
template <int S> struct SrcInfo;
template <> struct SrcInfo<SRC_F32> { static constexpr int EB = 4, NA = 2; };
template <> struct SrcInfo<SRC_FP8> { static constexpr int EB = 1, NA = 1; };
template <> struct SrcInfo<SRC_FP8_SH> { static constexpr int EB = 1, NA = 2; };
template <> struct SrcInfo<SRC_BF16_SH> { static constexpr int EB = 2, NA = 2; };

// Offset of 16-byte chunk j of row r in a 128-byte-swizzled tile (TMA
// SWIZZLE_128B; the tile starts on a 1024-byte boundary).
__device__ __forceinline__ uint32_t sw128(int r, int j) { return (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4)); }

__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float bf16_lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// 8 values -> the hi and lo 16-byte chunks (BF16 x 8 each).
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = bf16x2_bits(v[2 * q], v[2 * q + 1]);
    l[q] = bf16x2_bits(v[2 * q] - bf16_lo_f(h[q]), v[2 * q + 1] - bf16_hi_f(h[q]));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// FP8-e4m3 (4 bytes of w) -> 4 floats (exact)
__device__ __forceinline__ void e4m3x4(uint32_t w, float* out) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __nv_fp8_e4m3 b;
    b.__x = (__nv_fp8_storage_t)((w >> (8 * q)) & 0xffu);
    out[q] = float(b);
  }
}

// Convert row r (of R rows) of one 64-column group of a stage.
//   raw: start of the group's raw bytes (FP32: two boxes of R x 32 at raw and
//        raw + R*128; FP8: the 128-column box at raw, of which the group is
//        columns [64 half, 64 half + 64); BF16: one box of R x 64)
//   hi, lo: output tiles (R x 64 BF16 each); lo unused when NA == 1
//   scg, shg: global scale and shift at the group's first column (null: 1
//        and 0); nvalid: columns of the group inside A (the rest are zero)
// The whole raw row is read before anything is written (the FP32 output
// overwrites it in place).
template <int SRC>
__device__ __forceinline__ void convert_row(const unsigned char* raw, int R, int half, unsigned char* hi,
                                            unsigned char* lo, int r, const float* __restrict__ scg,
                                            const float* __restrict__ shg, int nvalid) {
  float v[64];
  if constexpr (SRC == SRC_F32) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const unsigned char* box = raw + (size_t)b * R * 128;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 t = *reinterpret_cast<const float4*>(box + sw128(r, j));
        v[32 * b + 4 * j] = t.x;
        v[32 * b + 4 * j + 1] = t.y;
        v[32 * b + 4 * j + 2] = t.z;
        v[32 * b + 4 * j + 3] = t.w;
      }
    }
  } else if constexpr (SRC == SRC_BF16_SH) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 t = *reinterpret_cast<const uint4*>(raw + sw128(r, j));
      const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[8 * j + 2 * q] = bf16_lo_f(w[q]);
        v[8 * j + 2 * q + 1] = bf16_hi_f(w[q]);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 t = *reinterpret_cast<const uint4*>(raw + sw128(r, 4 * half + j));
      e4m3x4(t.x, &v[16 * j]);
      e4m3x4(t.y, &v[16 * j + 4]);
      e4m3x4(t.z, &v[16 * j + 8]);
      e4m3x4(t.w, &v[16 * j + 12]);
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float t[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = 8 * j + q;
      float x = v[c];
      if constexpr (SRC != SRC_FP8) {
        if (scg) x *= __ldg(scg + c);
        if (shg) x -= __ldg(shg + c);
      }
      t[q] = c < nvalid ? x : 0.f;
    }
    uint4 h, l;
    split8(t, h, l);
    *reinterpret_cast<uint4*>(hi + sw128(r, j)) = h;
    if constexpr (SrcInfo<SRC>::NA == 2) *reinterpret_cast<uint4*>(lo + sw128(r, j)) = l;
  }
}

// Named barrier over the 4 warps of a 128-thread group (ids 1..).
__device__ __forceinline__ void bar128(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

template <int N>
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[N]) {
  static_assert(N == 16, "16 columns per load");
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace
}  // namespace rpca
