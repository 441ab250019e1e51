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
  SRC_BF16 = 4,     // BF16 as stored (T pass only): no conversion
};
template <int S> struct SrcInfo;
// NA: BF16 slices per converted element (2: hi and lo; 1: exact in BF16)
template <> struct SrcInfo<SRC_F32> { static constexpr int NA = 2; };
template <> struct SrcInfo<SRC_FP8> { static constexpr int NA = 1; };
template <> struct SrcInfo<SRC_FP8_SH> { static constexpr int NA = 2; };
template <> struct SrcInfo<SRC_BF16_SH> { static constexpr int NA = 2; };
template <> struct SrcInfo<SRC_BF16> { static constexpr int NA = 1; };

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

// Two e4m3 values (16 bits) -> two BF16 (32 bits), exactly: the hardware
// conversion to f16 (every e4m3 value is a normal f16 or zero), then the f16
// bits re-biased to BF16 (exponent + 112; the low 3 mantissa bits of an
// e4m3-derived f16 are zero, so shifting them out loses nothing).
__device__ __forceinline__ uint32_t e4m3x2_to_bf16x2(uint32_t v16) {
  uint32_t h;
  asm("{\n .reg .b16 a;\n cvt.u16.u32 a, %1;\n cvt.rn.f16x2.e4m3x2 %0, a;\n}" : "=r"(h) : "r"(v16));
  const uint32_t em = h & 0x7fff7fffu;
  const uint32_t t = (em >> 3) & 0x0fff0fffu;
  return (h & 0x80008000u) | (t + (__vcmpne2(em, 0u) & 0x38003800u));
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
  if constexpr (SRC == SRC_FP8) {
    // exact widening, no scale or shift: BF16 words straight from the bytes
    // (columns past A are zero bytes from TMA's fill, hence zero here)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 t = *reinterpret_cast<const uint4*>(raw + sw128(r, 4 * half + j));
      const uint32_t w[4] = {t.x, t.y, t.z, t.w};
      uint32_t o[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        o[2 * q] = e4m3x2_to_bf16x2(w[q] & 0xffffu);
        o[2 * q + 1] = e4m3x2_to_bf16x2(w[q] >> 16);
      }
      *reinterpret_cast<uint4*>(hi + sw128(r, 2 * j)) = make_uint4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<uint4*>(hi + sw128(r, 2 * j + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
    }
    (void)lo;
    (void)scg;
    (void)shg;
    (void)nvalid;
    (void)R;
    return;
  }
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


// ------------------------------------------------------------------ H pass
struct HcParams {
  int64_t m, n;
  int l;                 // real columns of X / H
  int ones_col;          // -1, or the H16 column (< 64) set to 1 (centring: F gets A~^T 1)
  int nkb;               // stages per panel (K steps of 64 G columns)
  int nstages;
  uint32_t stage_bytes;
  const float* scale;    // per-column scale applied by the converter (or null)
  const float* shift;    // per-column shift (or null)
  const float* corr;     // l values subtracted from every H row (or null)
  float* H;              // m x l FP32 (ldh), or null
  int64_t ldh;
  __nv_bfloat16* H16;    // hi plane then lo plane (plane16 elements apart), m x 64, or null
  int64_t plane16;
  uint32_t* dev_err;
  uint64_t wait_ns;
  int64_t withhold;      // wait-expiry test hook (-1: none)
};

constexpr int HC_THREADS = 384;
// K stages per accumulation chunk of the H pass: each chunk is summed in
// tensor memory from zero and the chunks are added in FP32 registers
// (rounding to nearest), which bounds the accumulator's biased rounding
// (see TC_FL below) to one chunk.
constexpr int HC_FLK = 8;

// Stage geometry of the H pass (bytes): raw A tile(s), converted tiles
// (FP32: in place), then the X^T boxes (G groups x NSX slices, L rows x
// 128 B each).
template <int SRC> struct HcGeom {
  static constexpr int G = (SRC == SRC_FP8 || SRC == SRC_FP8_SH) ? 2 : 1;   // 64-column groups per stage
  static constexpr uint32_t RAW = SRC == SRC_F32 ? 32768u : 16384u;
  static constexpr bool INPLACE = SRC == SRC_F32;
  static constexpr uint32_t OUT = INPLACE ? 0u : (uint32_t)G * SrcInfo<SRC>::NA * 16384u;
  __device__ __forceinline__ static uint32_t hi(int g) {
    return INPLACE ? 0u : RAW + (uint32_t)g * SrcInfo<SRC>::NA * 16384u;
  }
  __device__ __forceinline__ static uint32_t lo(int g) { return hi(g) + 16384u; }
};

template <int SRC, int L, int NSX>
__global__ void __launch_bounds__(HC_THREADS, 1)
k_hpass_cvt(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX0,
            const __grid_constant__ CUtensorMap tmX1, const HcParams p) {
  using Geo = HcGeom<SRC>;
  constexpr int G = Geo::G;
  constexpr int NA = SrcInfo<SRC>::NA;
  constexpr uint32_t XB = L * 128;                         // one X^T box: L rows x 64 BF16
  constexpr uint32_t XOFF = Geo::RAW + Geo::OUT;           // X boxes after the A tiles
  constexpr uint32_t TX = Geo::RAW + (uint32_t)G * NSX * XB;
  constexpr uint32_t TMEM_COLS = (2 * L <= 32) ? 32 : (2 * L <= 64) ? 64 : 128;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = p.nstages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * p.stage_bytes);
  uint64_t* conv = full + S;
  uint64_t* empty = conv + S;
  uint64_t* tfull = empty + S;      // [2]
  uint64_t* tempty = tfull + 2;     // [2]
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t lim = p.wait_ns;
  const int64_t npan = (p.m + 127) / 128;
  const int64_t my_pan = (npan > blockIdx.x) ? (npan - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&conv[s], 4);
      tc::mbar_init(&empty[s], 1);
    }
    for (int x = 0; x < 2; ++x) {
      tc::mbar_init(&tfull[x], 1);
      tc::mbar_init(&tempty[x], 4);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::tma_prefetch(&tmA);
    tc::tma_prefetch(&tmX0);
    if (NSX == 2) tc::tma_prefetch(&tmX1);
  }
  if (warp == 2) {
    tc::tmem_alloc(tmem_slot, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ TMA
      const int64_t withheld = blockIdx.x == 0 ? p.withhold : -1;
      const uint64_t pol = tc::l2_policy_evict_first();      // A is read once
      int64_t q = 0;
      bool ok = true;
      for (int64_t it = 0; ok && it < my_pan; ++it) {
        const int32_t r0 = (int32_t)((blockIdx.x + it * gridDim.x) * 128);
        for (int kb = 0; kb < p.nkb; ++kb, ++q) {
          const int s = (int)(q % S);
          if (!tc::mbar_wait(&empty[s], (uint32_t)(((q / S) & 1) ^ 1), p.dev_err, abort_flag, false, lim)) {
            ok = false;
            break;
          }
          if (q == withheld) continue;             // wait-expiry test: never arrives
          unsigned char* st = smem + (size_t)s * p.stage_bytes;
          const int32_t c0 = kb * 64 * G;
          tc::mbar_arrive_expect_tx(&full[s], TX);
          if constexpr (SRC == SRC_F32) {
            tc::tma_load_2d_hint(st, &tmA, &full[s], c0, r0, pol);
            tc::tma_load_2d_hint(st + 16384, &tmA, &full[s], c0 + 32, r0, pol);
          } else {
            tc::tma_load_2d_hint(st, &tmA, &full[s], c0, r0, pol);
          }
#pragma unroll
          for (int g = 0; g < G; ++g) {
            tc::tma_load_2d(st + XOFF + (uint32_t)(g * NSX) * XB, &tmX0, &full[s], c0 + 64 * g, 0);
            if (NSX == 2) tc::tma_load_2d(st + XOFF + (uint32_t)(g * NSX + 1) * XB, &tmX1, &full[s], c0 + 64 * g, 0);
          }
        }
      }
      for (int64_t qq = (q > S ? q - S : 0); qq < q; ++qq) {
        if (qq == withheld) continue;
        volatile int never = 0;
        tc::mbar_wait(&full[qq % S], (uint32_t)((qq / S) & 1), nullptr, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA
      constexpr uint32_t idesc = tc::idesc_make(1u, 0u, 0u, 128u, (uint32_t)L);
      int64_t q = 0;
      bool ok = true;
      int64_t gch = 0;                           // accumulation chunks so far
      for (int64_t it = 0; ok && it < my_pan; ++it) {
        int ab = 0;
        uint32_t d = tmem;
        for (int kb = 0; kb < p.nkb; ++kb, ++q) {
          if (kb % HC_FLK == 0) {
            ab = (int)(gch & 1);
            if (!tc::mbar_wait(&tempty[ab], (uint32_t)(((gch >> 1) & 1) ^ 1), p.dev_err, abort_flag, false, lim)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            d = tmem + (uint32_t)(ab * L);
          }
          const int s = (int)(q % S);
          if (!tc::mbar_wait(&conv[s], (uint32_t)((q / S) & 1), p.dev_err, abort_flag, false, lim)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t sb = tc::smem_u32(smem + (size_t)s * p.stage_bytes);
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const uint64_t ah = tc::sdesc_sw128(sb + Geo::hi(g), 16, 1024);
            const uint64_t al = tc::sdesc_sw128(sb + Geo::lo(g), 16, 1024);
            const uint64_t x0 = tc::sdesc_sw128(sb + XOFF + (uint32_t)(g * NSX) * XB, 16, 1024);
            const uint64_t x1 = tc::sdesc_sw128(sb + XOFF + (uint32_t)(g * NSX + 1) * XB, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t acc = ((kb % HC_FLK) > 0 || g > 0 || kk > 0) ? 1u : 0u;
              tc::mma_f16(d, tc::sdesc_add(ah, kk * 32), tc::sdesc_add(x0, kk * 32), idesc, acc);
              if (NA == 2) tc::mma_f16(d, tc::sdesc_add(al, kk * 32), tc::sdesc_add(x0, kk * 32), idesc, 1u);
              if (NSX == 2) tc::mma_f16(d, tc::sdesc_add(ah, kk * 32), tc::sdesc_add(x1, kk * 32), idesc, 1u);
            }
          }
          tc::mma_commit(&empty[s]);
          if (kb % HC_FLK == HC_FLK - 1 || kb == p.nkb - 1) {
            tc::mma_commit(&tfull[ab]);
            ++gch;
          }
        }
      }
      tc::mma_commit(done);
    }
  } else if (warp >= 4 && warp < 8) {
    // --------------------------------------------------------- converters
    const int r = tid - 128;                       // tile row
    int64_t q = 0;
    bool ok = true;
    for (int64_t it = 0; ok && it < my_pan; ++it) {
      for (int kb = 0; kb < p.nkb; ++kb, ++q) {
        const int s = (int)(q % S);
        if (!tc::mbar_wait(&full[s], (uint32_t)((q / S) & 1), p.dev_err, abort_flag, false, lim)) {
          ok = false;
          break;
        }
        unsigned char* st = smem + (size_t)s * p.stage_bytes;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int64_t cg = (int64_t)kb * 64 * G + 64 * g;
          convert_row<SRC>(st, 128, g, st + Geo::hi(g), st + Geo::lo(g), r, p.scale ? p.scale + cg : nullptr,
                           p.shift ? p.shift + cg : nullptr, (int)(p.n - cg > 64 ? 64 : p.n - cg));
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&conv[s]);
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int row = 32 * quad + lane;
    const int nch = (p.nkb + HC_FLK - 1) / HC_FLK;     // chunks per panel
    int64_t gch = 0;
    bool ok = true;
    for (int64_t it = 0; ok && it < my_pan; ++it) {
      const int64_t grow = (blockIdx.x + it * gridDim.x) * 128 + row;
      float v[L];
#pragma unroll
      for (int c = 0; c < L; ++c) v[c] = 0.f;
      for (int ch = 0; ch < nch; ++ch, ++gch) {
        const int ab = (int)(gch & 1);
        if (!tc::mbar_wait(&tfull[ab], (uint32_t)((gch >> 1) & 1), p.dev_err, abort_flag, false, lim)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
#pragma unroll
        for (int c16 = 0; c16 < L; c16 += 16) {
          uint32_t u[16];
          tmem_ld32<16>(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(ab * L + c16), u);
#pragma unroll
          for (int q = 0; q < 16; ++q) v[c16 + q] += __uint_as_float(u[q]);
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[ab]);   // the accumulator may be reused
      }
      if (!ok) break;
#pragma unroll
      for (int c = 0; c < L; ++c) {
        if (p.corr && c < p.l) v[c] -= __ldg(p.corr + c);
        if (c >= p.l) v[c] = 0.f;
      }
      if (grow < p.m) {
        if (p.H) {
          float* hrow = p.H + grow * p.ldh;
          const bool vec = ((reinterpret_cast<uintptr_t>(hrow) | (uintptr_t)(p.ldh * 4)) & 15) == 0;
#pragma unroll
          for (int c = 0; c < L; c += 4) {
            if (vec && c + 3 < p.l) {
              *reinterpret_cast<float4*>(hrow + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (c + q < p.l) hrow[c + q] = v[c + q];
            }
          }
        }
        if (p.H16) {
          uint4* hi = reinterpret_cast<uint4*>(p.H16 + grow * 64);
          uint4* lo = reinterpret_cast<uint4*>(p.H16 + p.plane16 + grow * 64);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float t[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int c = 8 * j + q;
              t[q] = c < L ? v[c < L ? c : 0] : 0.f;
              if (c == p.ones_col) t[q] = 1.f;
            }
            uint4 h, l;
            split8(t, h, l);
            hi[j] = h;
            lo[j] = l;
          }
        }
      }
    }
  }
  __syncwarp();
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done, 0, nullptr, &never);       // every MMA has completed
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, TMEM_COLS);
}

// X (n x l FP32, ldx) -> X^T slices (L x n64 BF16 each): hi = bf16(v),
// lo = bf16(v - hi), v = X[r][j] * fold[r] (fold: the FP8 column scale, or
// null).
__global__ void k_xt_split(int64_t n, int l, int L, int64_t n64, const float* __restrict__ X, int64_t ldx,
                           const float* __restrict__ fold, __nv_bfloat16* __restrict__ Xh,
                           __nv_bfloat16* __restrict__ Xl) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * n64) return;
  const int j = (int)(e / n64);
  const int64_t r = e % n64;
  float v = (j < l && r < n) ? X[r * ldx + j] : 0.f;
  if (fold && r < n) v *= fold[r];
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  Xh[e] = h;
  if (Xl) Xl[e] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// ---------------------------------------------------------------- T pass
constexpr int TC_KSUB = 32;          // rows per stage
constexpr int TC_THREADS = 384;
constexpr uint32_t TC_BOX = TC_KSUB * 128;   // one 32-row, 128-byte box
// Sub-panels per accumulation chunk: the tensor cores' FP32 accumulation
// loses about one unit in the last place of the running sum per MMA, with a
// bias (it does not round to nearest), so a sum over ~1e5 rows drifts by a
// few 1e-4.  Each chunk of TC_FL sub-panels (512 rows) is therefore
// accumulated in tensor memory from zero and then added, rounding to
// nearest, into FP32 sums in shared memory; the drift of one chunk is a few
// 1e-6 and the chunk sums random-walk.
constexpr int TC_FL = 16;

struct TcParams {
  int64_t m, n;
  int p;                 // columns of the result (compact)
  int npad;              // MMA N: columns of Y as stored (multiple of 16, <= 256)
  int nyb;               // 64-column boxes of Y per slice
  int qblk;              // > 0: Y is block-padded (block b of qblk columns at 64 b)
  int nslab, ngroup, nstages;
  uint32_t stage_bytes;
  const float* scale;    // converter scale (or null)
  const float* shift;    // converter shift (or null)
  const float* rowscale; // result row r multiplied by rowscale[r] (FP8 folding), or null
  void* T;               // n x p (ldt), TF, accumulated with atomics
  int64_t ldt;
  uint32_t* dev_err;
  uint64_t wait_ns;
  int64_t withhold;
};

// Stage geometry of the T pass (bytes from the stage base).  Group g is the
// 64 columns [64 g, 64 g + 64) of the slab; its hi (and lo) tile is 32 rows
// x 128 B in the layout of a BF16 TMA box.
template <int SRC, int NT> struct TcGeom {
  static constexpr int NG = 2 * NT;
  static constexpr uint32_t RAW = SRC == SRC_F32 ? NG * 2 * TC_BOX                // 2 FP32 boxes per group
                                  : (SRC == SRC_BF16_SH || SRC == SRC_BF16) ? NG * TC_BOX   // 1 BF16 box
                                                                           : NT * TC_BOX;   // FP8: 1 box / 2 groups
  static constexpr bool INPLACE = SRC == SRC_F32 || SRC == SRC_BF16;
  static constexpr int NA = SrcInfo<SRC>::NA;
  static constexpr uint32_t OUT = INPLACE ? 0u : (uint32_t)NG * NA * TC_BOX;
  // FP32 in place: group g at 2 g boxes, hi then lo; BF16: the raw boxes
  // themselves; otherwise after RAW
  __device__ __forceinline__ static uint32_t hi(int g) {
    return SRC == SRC_BF16 ? (uint32_t)g * TC_BOX
           : INPLACE       ? (uint32_t)(2 * g) * TC_BOX
                           : RAW + (uint32_t)(g * NA) * TC_BOX;
  }
  __device__ __forceinline__ static uint32_t lo(int g) { return hi(g) + TC_BOX; }
  // distance between the hi tiles of groups 2t and 2t + 1 (the MMA's LBO)
  static constexpr uint32_t LBO = (SRC == SRC_BF16 ? 1 : INPLACE ? 2 : NA) * TC_BOX;
  // raw location of group g's data (FP8: half g & 1 of box g >> 1)
  __device__ __forceinline__ static uint32_t raw(int g) {
    return SRC == SRC_F32 ? (uint32_t)(2 * g) * TC_BOX
           : (SRC == SRC_BF16_SH || SRC == SRC_BF16) ? (uint32_t)g * TC_BOX
                                                     : (uint32_t)(g >> 1) * TC_BOX;
  }
};

// Roles (12 warps): warp 0 lane 0 TMA, warp 1 lane 0 MMA, warp 2 owns the
// tensor memory, warps 4-7 convert (not for plain BF16), warps 8-11 drain
// the accumulator chunks into the shared-memory sums and finally add those
// to T.  NB accumulator buffers in tensor memory (2 when they fit).
template <int SRC, int NT, typename TF, int NSY>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tpass_cvt(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmY0,
            const __grid_constant__ CUtensorMap tmY1, const TcParams p) {
  using Geo = TcGeom<SRC, NT>;
  constexpr int NA = SrcInfo<SRC>::NA;
  constexpr bool CONVERT = SRC != SRC_BF16;
  const uint32_t YOFF = Geo::RAW + Geo::OUT;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = p.nstages;
  float* accs = reinterpret_cast<float*>(smem + (size_t)S * p.stage_bytes);   // [NT][npad][128]
  uint64_t* full = reinterpret_cast<uint64_t*>(accs + (size_t)NT * p.npad * 128);
  uint64_t* conv = full + S;
  uint64_t* empty = conv + S;
  uint64_t* cfull = empty + S;      // [2] chunk accumulated in buffer b
  uint64_t* cempty = cfull + 2;     // [2] buffer b drained
  uint64_t* done = cempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t lim = p.wait_ns;
  const int slab = blockIdx.x % p.nslab;
  const int group = blockIdx.x / p.nslab;
  if (group >= p.ngroup) return;
  const int64_t nsub = (p.m + TC_KSUB - 1) / TC_KSUB;
  const int64_t my_subs = (nsub > group) ? (nsub - group + p.ngroup - 1) / p.ngroup : 0;
  const int64_t nchunks = (my_subs + TC_FL - 1) / TC_FL;
  const int acc_cols = NT * p.npad;
  const int NB = 2 * acc_cols <= 512 ? 2 : 1;
  const int ncols = NB * acc_cols;
  const uint32_t tmem_cols = ncols <= 32 ? 32 : ncols <= 64 ? 64 : ncols <= 128 ? 128 : ncols <= 256 ? 256 : 512;
  const uint32_t TX = Geo::RAW + (uint32_t)(NSY * p.nyb) * TC_BOX;
  const int32_t col0 = slab * NT * 128;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&conv[s], 4);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&cfull[b], 1);
      tc::mbar_init(&cempty[b], 4);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::tma_prefetch(&tmA);
    tc::tma_prefetch(&tmY0);
    if (NSY == 2) tc::tma_prefetch(&tmY1);
  }
  if (warp >= 8)
    for (int e = tid - 256; e < acc_cols * 128; e += 128) accs[e] = 0.f;
  if (warp == 2) {
    tc::tmem_alloc(tmem_slot, tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // -------------------------------------------------------------- TMA
    const int64_t withheld = blockIdx.x == 0 ? p.withhold : -1;
    const uint64_t pol = tc::l2_policy_evict_first();
    int64_t it = 0;
    for (; it < my_subs; ++it) {
      const int s = (int)(it % S);
      if (!tc::mbar_wait(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), p.dev_err, abort_flag, false, lim)) break;
      if (it == withheld) continue;
      unsigned char* st = smem + (size_t)s * p.stage_bytes;
      const int32_t r0 = (int32_t)((group + it * p.ngroup) * TC_KSUB);
      tc::mbar_arrive_expect_tx(&full[s], TX);
      if constexpr (SRC == SRC_F32) {
        for (int b = 0; b < 4 * NT; ++b)
          tc::tma_load_2d_hint(st + (uint32_t)b * TC_BOX, &tmA, &full[s], col0 + 32 * b, r0, pol);
      } else if constexpr (SRC == SRC_BF16_SH || SRC == SRC_BF16) {
        for (int b = 0; b < 2 * NT; ++b)
          tc::tma_load_2d_hint(st + (uint32_t)b * TC_BOX, &tmA, &full[s], col0 + 64 * b, r0, pol);
      } else {
        for (int b = 0; b < NT; ++b)
          tc::tma_load_2d_hint(st + (uint32_t)b * TC_BOX, &tmA, &full[s], col0 + 128 * b, r0, pol);
      }
      for (int b = 0; b < p.nyb; ++b) {
        tc::tma_load_2d(st + YOFF + (uint32_t)b * TC_BOX, &tmY0, &full[s], 64 * b, r0);
        if (NSY == 2) tc::tma_load_2d(st + YOFF + (uint32_t)(p.nyb + b) * TC_BOX, &tmY1, &full[s], 64 * b, r0);
      }
    }
    for (int64_t jt = (it > S ? it - S : 0); jt < it; ++jt) {
      if (jt == withheld) continue;
      volatile int never = 0;
      tc::mbar_wait(&full[jt % S], (uint32_t)((jt / S) & 1), nullptr, &never);
    }
  } else if (warp == 1 && lane == 0) {
    // -------------------------------------------------------------- MMA
    const uint32_t idesc = tc::idesc_make(1u, 1u, 1u, 128u, (uint32_t)p.npad);
    for (int64_t it = 0; it < my_subs; ++it) {
      const int64_t ch = it / TC_FL;
      const int b = (int)(ch % NB);
      const bool first = (it % TC_FL) == 0;
      if (first && !tc::mbar_wait(&cempty[b], (uint32_t)(((ch / NB) & 1) ^ 1), p.dev_err, abort_flag, false, lim))
        break;
      const int s = (int)(it % S);
      uint64_t* ready = CONVERT ? &conv[s] : &full[s];
      if (!tc::mbar_wait(ready, (uint32_t)((it / S) & 1), p.dev_err, abort_flag, false, lim)) break;
      tc::tc_fence_after();
      const uint32_t sb = tc::smem_u32(smem + (size_t)s * p.stage_bytes);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const uint64_t ah = tc::sdesc_sw128(sb + Geo::hi(2 * t), Geo::LBO, 1024);
        const uint64_t al = tc::sdesc_sw128(sb + Geo::lo(2 * t), Geo::LBO, 1024);
        const uint64_t y0 = tc::sdesc_sw128(sb + YOFF, TC_BOX, 1024);
        const uint64_t y1 = tc::sdesc_sw128(sb + YOFF + (uint32_t)p.nyb * TC_BOX, TC_BOX, 1024);
        const uint32_t d = tmem + (uint32_t)(b * acc_cols + t * p.npad);
#pragma unroll
        for (int kk = 0; kk < TC_KSUB / 16; ++kk) {
          const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
          tc::mma_f16(d, tc::sdesc_add(ah, kk * 2048), tc::sdesc_add(y0, kk * 2048), idesc, acc);
          if (NA == 2) tc::mma_f16(d, tc::sdesc_add(al, kk * 2048), tc::sdesc_add(y0, kk * 2048), idesc, 1u);
          if (NSY == 2) tc::mma_f16(d, tc::sdesc_add(ah, kk * 2048), tc::sdesc_add(y1, kk * 2048), idesc, 1u);
        }
      }
      tc::mma_commit(&empty[s]);
      if ((it % TC_FL) == TC_FL - 1 || it == my_subs - 1) tc::mma_commit(&cfull[b]);
    }
    tc::mma_commit(done);
  } else if (warp >= 4 && warp < 8) {
    // --------------------------------------------------------- converters
    if (CONVERT) {
      const int e = tid - 128;
      const int r = e & (TC_KSUB - 1), g = e / TC_KSUB;     // row and 64-column group
      const bool mine = g < Geo::NG;
      for (int64_t it = 0; it < my_subs; ++it) {
        const int s = (int)(it % S);
        if (!tc::mbar_wait(&full[s], (uint32_t)((it / S) & 1), p.dev_err, abort_flag, false, lim)) break;
        unsigned char* st = smem + (size_t)s * p.stage_bytes;
        if (mine) {
          const int64_t cg = (int64_t)col0 + 64 * g;
          if constexpr (SRC != SRC_BF16)
            convert_row<SRC>(st + Geo::raw(g), TC_KSUB, g & 1, st + Geo::hi(g), st + Geo::lo(g), r,
                             p.scale ? p.scale + cg : nullptr, p.shift ? p.shift + cg : nullptr,
                             (int)(p.n - cg < 0 ? 0 : (p.n - cg > 64 ? 64 : p.n - cg)));
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&conv[s]);
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------ chunk drains, then the output
    const int quad = warp & 3;
    const int row = 32 * quad + lane;             // accumulator lane = slab column
    bool ok = true;
    for (int64_t ch = 0; ch < nchunks; ++ch) {
      const int b = (int)(ch % NB);
      if (!tc::mbar_wait(&cfull[b], (uint32_t)((ch / NB) & 1), p.dev_err, abort_flag, false, lim)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      for (int t = 0; t < NT; ++t)
        for (int c16 = 0; c16 < p.npad; c16 += 16) {
          uint32_t u[16];
          tmem_ld32<16>(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(b * acc_cols + t * p.npad + c16), u);
          float* a = accs + ((size_t)(t * p.npad + c16) * 128 + row);
#pragma unroll
          for (int q = 0; q < 16; ++q) a[(size_t)q * 128] += __uint_as_float(u[q]);
        }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&cempty[b]);
    }
    if (ok && my_subs > 0) {
      TF* T = static_cast<TF*>(p.T);
      for (int t = 0; t < NT; ++t) {
        const int64_t trow = (int64_t)col0 + t * 128 + row;     // row of T = column of A
        if (trow >= p.n) continue;
        const float rs = p.rowscale ? p.rowscale[trow] : 1.f;
        for (int c = 0; c < p.npad; ++c) {
          const float v = accs[(size_t)(t * p.npad + c) * 128 + row] * rs;
          if (p.qblk > 0) {
            if ((c & 63) < p.qblk && (c >> 6) * p.qblk + (c & 63) < p.p)
              atomicAdd(&T[trow * p.ldt + (c >> 6) * p.qblk + (c & 63)], (TF)v);
          } else if (c < p.p) {
            atomicAdd(&T[trow * p.ldt + c], (TF)v);
          }
        }
      }
    }
  }
  __syncwarp();
  if (warp == 1 && lane == 0) {
    volatile int never = 0;
    tc::mbar_wait(done, 0, nullptr, &never);       // every MMA has completed
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, tmem_cols);
}

// ------------------------------------------------------------------- host
// Q (FP32 m x w, ldq) -> two BF16 planes (hi, lo) of m x wq, zero-padded.
__global__ void k_split_planes(int64_t m, int w, int wq, const float* __restrict__ Q, int64_t ldq,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * wq) return;
  const int64_t r = e / wq;
  const int c = (int)(e % wq);
  const float v = c < w ? Q[r * ldq + c] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[e] = h;
  if (lo) lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
}

template <typename K>
void set_smem(K kern, size_t smem) {
  RPCA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
}

constexpr size_t CVT_SMEM_LIMIT = 227 * 1024;

CUtensorMapDataType a_tmap_type(int src) {
  return src == SRC_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
         : (src == SRC_BF16_SH || src == SRC_BF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT8;
}
size_t a_elem(int src) { return src == SRC_F32 ? 4 : (src == SRC_BF16_SH || src == SRC_BF16) ? 2 : 1; }

template <int SRC, int L, int NSX>
bool launch_hpass(const PassArgs& a, const __nv_bfloat16* Xh, const __nv_bfloat16* Xl, int64_t n64,
                  __nv_bfloat16* H16, int64_t plane16, cudaStream_t st, uint32_t* dev_err, const WaitTest& wt) {
  using Geo = HcGeom<SRC>;
  CUtensorMap tmA, tmX0, tmX1;
  const uint32_t abox_cols = SRC == SRC_F32 ? 32 : SRC == SRC_BF16_SH ? 64 : 128;
  if (!make_tmap_2d(&tmA, a.A, a_tmap_type(SRC), a_elem(SRC), a.m, a.n, a.lda, 128, abox_cols)) return false;
  if (!make_tmap_2d(&tmX0, Xh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, L, n64, n64, L, 64)) return false;
  if (!make_tmap_2d(&tmX1, NSX == 2 ? Xl : Xh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, L, n64, n64, L, 64))
    return false;
  HcParams p;
  p.m = a.m;
  p.n = a.n;
  p.l = a.p;
  p.ones_col = a.ones_col;
  p.nkb = (int)cdiv(a.n, 64 * Geo::G);
  p.stage_bytes = (uint32_t)round_up(Geo::RAW + Geo::OUT + (uint32_t)Geo::G * NSX * L * 128, 1024);
  p.nstages = (int)std::min<size_t>(8, (CVT_SMEM_LIMIT - 2048) / p.stage_bytes);
  if (p.nstages < 2) return false;
  p.scale = SRC == SRC_FP8 ? nullptr : a.scale;
  p.shift = static_cast<const float*>(a.shift);
  p.corr = static_cast<const float*>(a.corr);
  p.H = static_cast<float*>(a.H);
  p.ldh = a.ldh;
  p.H16 = H16;
  p.plane16 = plane16;
  p.dev_err = dev_err;
  p.wait_ns = wt.limit_ns;
  p.withhold = wt.withhold;
  const size_t smem = 1024 + (size_t)p.nstages * p.stage_bytes + 256;
  auto kern = k_hpass_cvt<SRC, L, NSX>;
  set_smem(kern, smem);
  const int64_t npan = cdiv(a.m, 128);
  const int grid = (int)std::min<int64_t>(npan, num_sms());
  kern<<<grid, HC_THREADS, smem, st>>>(tmA, tmX0, tmX1, p);
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
  if (getenv("RPCA_DEBUG"))
    fprintf(stderr, "[rpca] hpass-cvt src=%d L=%d nsx=%d grid=%d stages=%d stage=%u\n", SRC, L, NSX, grid, p.nstages,
            p.stage_bytes);
  return true;
}

// T (n x p) (+)= A_c^T Y, Y = NSY BF16 planes (m x ldy, plane stride `plane`)
// with nyb 64-column boxes; qblk > 0: block-padded Y.
template <int SRC, int NSY>
bool launch_tpass(const PassArgs& a, const __nv_bfloat16* Y, int64_t ldy, int64_t plane, int nyb, int npad, int qblk,
                  bool f_f64, cudaStream_t st, uint32_t* dev_err, const WaitTest& wt) {
  // two slabs per CTA when two tensor-memory buffers of both still fit and
  // the shared-memory sums stay small; else one slab
  const int NT = (npad <= 64) ? 2 : 1;
  CUtensorMap tmA, tmY0, tmY1;
  const uint32_t abox_cols = SRC == SRC_F32 ? 32 : (SRC == SRC_BF16_SH || SRC == SRC_BF16) ? 64 : 128;
  if (!make_tmap_2d(&tmA, a.A, a_tmap_type(SRC), a_elem(SRC), a.m, a.n, a.lda, TC_KSUB, abox_cols)) return false;
  if (!make_tmap_2d(&tmY0, Y, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.m, ldy, ldy, TC_KSUB, 64)) return false;
  if (!make_tmap_2d(&tmY1, NSY == 2 ? Y + plane : Y, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.m, ldy, ldy, TC_KSUB, 64))
    return false;
  TcParams p;
  p.m = a.m;
  p.n = a.n;
  p.p = a.mode == MODE_T ? a.p : a.p + (a.ones_col >= 0 ? 1 : 0);
  p.npad = npad;
  p.nyb = nyb;
  p.qblk = qblk;
  const uint32_t raw_out = NT == 2 ? TcGeom<SRC, 2>::RAW + TcGeom<SRC, 2>::OUT : TcGeom<SRC, 1>::RAW + TcGeom<SRC, 1>::OUT;
  p.stage_bytes = (uint32_t)round_up(raw_out + (uint32_t)(NSY * nyb) * TC_BOX, 1024);
  const size_t acc_bytes = (size_t)NT * npad * 128 * sizeof(float);
  if (acc_bytes + 2048 + 2 * (size_t)p.stage_bytes > CVT_SMEM_LIMIT) return false;
  p.nstages = (int)std::min<size_t>(8, (CVT_SMEM_LIMIT - 2048 - acc_bytes) / p.stage_bytes);
  p.nslab = (int)cdiv(a.n, NT * 128);
  const int sms = num_sms();
  p.ngroup = std::max(1, std::min<int>((int)cdiv(a.m, TC_KSUB), sms / p.nslab));
  p.scale = SRC == SRC_FP8 ? nullptr : a.scale;
  p.shift = static_cast<const float*>(a.shift);
  p.rowscale = SRC == SRC_FP8 ? a.scale : nullptr;
  p.T = a.F;
  p.ldt = a.ldf;
  p.dev_err = dev_err;
  p.wait_ns = wt.limit_ns;
  p.withhold = wt.withhold;
  const size_t smem = 1024 + (size_t)p.nstages * p.stage_bytes + acc_bytes + 256;
  dim3 grid(p.nslab * p.ngroup);
  if (f_f64) {
    auto kern = NT == 2 ? k_tpass_cvt<SRC, 2, double, NSY> : k_tpass_cvt<SRC, 1, double, NSY>;
    set_smem(kern, smem);
    kern<<<grid, TC_THREADS, smem, st>>>(tmA, tmY0, tmY1, p);
  } else {
    auto kern = NT == 2 ? k_tpass_cvt<SRC, 2, float, NSY> : k_tpass_cvt<SRC, 1, float, NSY>;
    set_smem(kern, smem);
    kern<<<grid, TC_THREADS, smem, st>>>(tmA, tmY0, tmY1, p);
  }
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
  if (getenv("RPCA_DEBUG"))
    fprintf(stderr, "[rpca] tpass-cvt src=%d NT=%d nsy=%d npad=%d nyb=%d grid=%d stages=%d stage=%u\n", SRC, NT, NSY,
            npad, nyb, p.nslab * p.ngroup, p.nstages, p.stage_bytes);
  return true;
}

template <int SRC>
bool pass_cvt_src(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  const int64_t n64 = round_up(a.n, 128);
  unsigned char* work = static_cast<unsigned char*>(a.work);
  if (a.mode == MODE_T) {
    // Y = Q: the sliced QR's first two BF16 slices when given, else Q in
    // FP32 split into two planes here
    const __nv_bfloat16* Y;
    int64_t ldy, plane;
    int qblk;
    if (a.q16) {
      if (!a.q16_plane) return false;
      Y = static_cast<const __nv_bfloat16*>(a.q16);
      ldy = a.q16_ld;
      plane = a.q16_plane;
      qblk = a.q_blk;
    } else {
      const int wq = (int)round_up(a.p, 64);
      if (wq > 256) return false;
      if ((size_t)2 * a.m * wq * 2 > a.work_bytes) return false;
      __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(work);
      __nv_bfloat16* lo = hi + (size_t)a.m * wq;
      const int64_t cnt = a.m * wq;
      k_split_planes<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(a.m, a.p, wq, static_cast<const float*>(a.H), a.ldh,
                                                              hi, lo);
      RPCA_CUDA_TRY(cudaGetLastError());
      count_launch();
      Y = hi;
      ldy = wq;
      plane = (int64_t)a.m * wq;
      qblk = 0;
    }
    const int nyb = (int)(ldy / 64);
    const int npad = qblk > 0 ? (int)ldy : (int)round_up(a.p, 16);
    if (npad > 256) return false;
    const size_t fes = a.f_f64 ? 8 : 4;
    if (!a.accumulate_f) RPCA_CUDA_TRY(cudaMemset2DAsync(a.F, a.ldf * fes, 0, a.p * fes, a.n, st));
    return launch_tpass<SRC, 2>(a, Y, ldy, plane, nyb, npad, qblk, a.f_f64, st, dev_err, take_wait_test(1));
  }
  // Step 1 pass: X^T slices, H pass, then (fused) F = A_c^T H from the BF16
  // slices of H
  const int need = a.p + (a.ones_col >= 0 ? 1 : 0);
  const int L = need <= 16 ? 16 : need <= 32 ? 32 : need <= 64 ? 64 : 0;
  if (!L) return false;
  const size_t xt_bytes = (size_t)2 * L * n64 * 2;
  const bool fused = a.mode == MODE_FUSED && a.F;
  const size_t h16_bytes = fused ? (size_t)2 * a.m * 64 * 2 : 0;
  if (xt_bytes + h16_bytes + 256 > a.work_bytes) return false;
  __nv_bfloat16* Xh = reinterpret_cast<__nv_bfloat16*>(work);
  __nv_bfloat16* Xl = Xh + (size_t)L * n64;
  __nv_bfloat16* H16 = fused ? reinterpret_cast<__nv_bfloat16*>(work + round_up(xt_bytes, 256)) : nullptr;
  {
    const int64_t cnt = (int64_t)L * n64;
    k_xt_split<<<(unsigned)cdiv(cnt, 256), 256, 0, st>>>(a.n, a.p, L, n64, static_cast<const float*>(a.X), a.ldx,
                                                         SRC == SRC_FP8 ? a.scale : nullptr, Xh, Xl);
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  const WaitTest wt = take_wait_test(0);
  bool ok;
  if (L == 16) ok = launch_hpass<SRC, 16, 2>(a, Xh, Xl, n64, H16, (int64_t)a.m * 64, st, dev_err, wt);
  else if (L == 32) ok = launch_hpass<SRC, 32, 2>(a, Xh, Xl, n64, H16, (int64_t)a.m * 64, st, dev_err, wt);
  else ok = launch_hpass<SRC, 64, 2>(a, Xh, Xl, n64, H16, (int64_t)a.m * 64, st, dev_err, wt);
  if (!ok || !fused) return ok;
  if (!a.accumulate_f) RPCA_CUDA_TRY(cudaMemset2DAsync(a.F, a.ldf * 4, 0, need * 4, a.n, st));
  const WaitTest none = {2000000000ull, -1};
  return launch_tpass<SRC, 2>(a, H16, 64, (int64_t)a.m * 64, 1, L, 0, false, st, dev_err, none);
}


}  // namespace

// Whether the converting tensor-core kernels take this pass (see the top of
// the file), and the pass itself.
bool pass_cvt(const PassArgs& a, cudaStream_t st, uint32_t* dev_err) {
  if (a.mode != MODE_T && a.mode != MODE_H && a.mode != MODE_FUSED) return false;
  if (!a.work) return false;
  if (a.ones_col >= 0 && a.ones_col != a.p) return false;
  if (a.dtype == RPCA_F32) return pass_cvt_src<SRC_F32>(a, st, dev_err);
  if (a.dtype == RPCA_FP8E4M3) {
    if (!a.scale) return false;
    return a.shift ? pass_cvt_src<SRC_FP8_SH>(a, st, dev_err) : pass_cvt_src<SRC_FP8>(a, st, dev_err);
  }
  if (a.dtype == RPCA_BF16 && (a.shift || a.scale)) return pass_cvt_src<SRC_BF16_SH>(a, st, dev_err);
  return false;
}

}  // namespace rpca
