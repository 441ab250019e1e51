// C-ABI and host orchestration of the randomized block-Lanczos PCA
// (Halko, Martinsson, Shkolnisky, Tygert, Section 3, Steps 1-6; streamed
// passes as in Section 4.2).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "grouped.h"

namespace rpca {

std::atomic<uint64_t> g_launches{0};

// -------------------------------------------------- wait-expiry test hook
static std::mutex g_wait_test_mu;
static WaitTest g_wait_test[2] = {{2000000000ull, -1}, {2000000000ull, -1}};

WaitTest take_wait_test(int kind) {
  std::lock_guard<std::mutex> lock(g_wait_test_mu);
  const WaitTest w = g_wait_test[kind];
  g_wait_test[kind] = {2000000000ull, -1};
  return w;
}

// Error text of the last failed rpca_batch_init (no batch object remains).
static std::string& last_batch_error() {
  static thread_local std::string s;
  return s;
}

// ------------------------------------------------------------- Philox (host)
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with key bumps by the Weyl constants.
static void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Standard normals: counter (p, 0, domain, 0); two 53-bit uniforms per
// counter; Box-Muller gives elements 2p and 2p+1.
static void gaussian_stream(uint64_t seed, uint32_t domain, int64_t count, double* out) {
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  const double two_pi = 6.283185307179586476925286766559;
  const double scale = 1.0 / 9007199254740992.0;  // 2^-53
  for (int64_t p = 0; 2 * p < count; ++p) {
    uint32_t c[4] = {(uint32_t)((uint64_t)p & 0xffffffffu), (uint32_t)((uint64_t)p >> 32), domain, 0u};
    philox4x32_10(c, k0, k1);
    double u1 = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6) + 0.5) * scale;
    double u2 = ((double)(c[2] >> 5) * 67108864.0 + (double)(c[3] >> 6) + 0.5) * scale;
    double r = std::sqrt(-2.0 * std::log(u1));
    double t = two_pi * u2;
    out[2 * p] = r * std::cos(t);
    if (2 * p + 1 < count) out[2 * p + 1] = r * std::sin(t);
  }
}

// --------------------------------------------------------------- utilities
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  void alloc(size_t b) {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = b;
    if (b == 0) return;
    cudaError_t e = cudaMalloc(&ptr, b);
    if (e != cudaSuccess) {
      ptr = nullptr;
      throw CudaFailure(e, "cudaMalloc", __FILE__, __LINE__);
    }
  }
  ~DevBuf() {
    if (ptr) cudaFree(ptr);
  }
  template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

static bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    throw CudaFailure(cudaErrorNoDevice, "cudaGetDeviceCount", __FILE__, __LINE__);
  }
}

// Block Gram-Schmidt twice + Cholesky QR (up to 4 passes) on H (m x nblk*l):
// Step 2 with Gram matrices and Cholesky factors in FP64.  Optional R_out
// (w x w FP64, ld w, zeroed here) receives the triangular factor.
struct QrScratch {
  double* C = nullptr;     // w x l
  double* Gm = nullptr;    // l x l
  double* Rk = nullptr;    // l x l
  double* Rinv = nullptr;  // l x l
  double* Racc = nullptr;  // l x l
  uint32_t* qf = nullptr;  // kQfWords words per block
  float* mt = nullptr;     // 2 * 256 * 256 floats (tensor-core products)
  void* slices = nullptr;  // BF16 slice scratch for tensor-core Grams
  size_t slice_bytes = 0;
  double* G64 = nullptr;   // 64 x 64   (sliced QR: Gram of one padded block)
  double* C64 = nullptr;   // 192 x 64  (sliced QR: projection coefficients)
  double* Cfull = nullptr; // 192 x 192 (sliced QR: Q^T Q with padded indices)
};

// Step 2 on H held in three BF16 slices (k_qr_slices.cu) applies to FP32 H
// with at least kTcMinRows rows, 40 <= l <= 64 (blocks padded to 64
// columns), at most three blocks and k <= 64.
static bool sliced_ok(bool f64, int64_t m, int nblk, int l, int k) {
  return !f64 && m >= 8192 && l >= 40 && l <= 64 && nblk >= 1 && nblk <= 3 && k <= 64;
}
constexpr size_t kSliceScratchDoubles = 64 * 64 + 192 * 64 + 192 * 192;

// Tensor-core (TF32 x3) tall products apply to FP32 data with at least this
// many rows; Hlo is the remainder array of H (same layout).
constexpr int64_t kTcMinRows = 8192;

static void qr_gram(bool f64, int64_t m, int p, int q, const void* X, int64_t ldx, const void* Y, int64_t ldy,
                    double* C, int64_t ldc, const QrScratch& s, cudaStream_t st, uint32_t* dev_err,
                    const uint32_t* active = nullptr, bool reslice_x = true) {
  if (!f64 && s.slices && m >= kTcMinRows &&
      gram_tc(m, p, q, (const float*)X, ldx, (const float*)Y, ldy, C, ldc, s.slices, s.slice_bytes, st, dev_err,
              active, reslice_x))
    return;
  gram(f64, m, p, q, X, ldx, Y, ldy, C, ldc, false, st, active);
}

static void qr_apply(bool f64, int64_t m, int p, int q, const void* X, const float* Xlo, int64_t ldx,
                     const double* M, int64_t ldm, double alpha, double beta, void* Y, float* Ylo, int64_t ldy,
                     const QrScratch& s, cudaStream_t st, uint32_t* dev_err, const uint32_t* active = nullptr) {
  if (!f64 && Xlo && m >= kTcMinRows &&
      apply_tc(m, p, q, (const float*)X, Xlo, ldx, M, ldm, alpha, beta, (float*)Y, Ylo, ldy, s.mt, st, dev_err,
               active))
    return;
  gemm_xm(f64, m, p, q, X, ldx, M, ldm, alpha, beta, Y, ldy, st, active);
  if (Ylo) split_lo(m, q, (const float*)Y, ldy, Ylo, ldy, st);
}

// A block whose Cholesky needed a shift is numerically rank deficient: the
// passes have multiplied the projection's rounding residue against the
// earlier blocks by the block's condition number.  When qf[1] says so (set
// by the Cholesky kernel; every launch here is a no-op otherwise), project once more against the
// earlier blocks and re-orthonormalise with one more pass.  (The triangular
// factor is not tracked here: callers that want it skip this step.)
static void reorth_after_shift(bool f64, int64_t m, int jl, int l, void* H, float* Hlo, int64_t ld, void* Hj,
                               float* Hjlo, uint32_t* qf, double piv_rel, double shift_rel, const QrScratch& s,
                               uint32_t* dev_err, cudaStream_t st) {
  const uint32_t* g = qf + 1;
  qr_gram(f64, m, jl, l, H, ld, Hj, ld, s.C, l, s, st, dev_err, g, true);
  qr_apply(f64, m, jl, l, H, Hlo, ld, s.C, l, -1.0, 1.0, Hj, Hjlo, ld, s, st, dev_err, g);
  qr_gram(f64, m, l, l, Hj, ld, Hj, ld, s.Gm, l, s, st, dev_err, g);
  chol_small(l, s.Gm, l, s.Rk, s.Rinv, 1, piv_rel, shift_rel, qf, dev_err, st, false, g);
  qr_apply(f64, m, l, l, Hj, Hjlo, ld, s.Rinv, l, 1.0, 0.0, Hj, Hjlo, ld, s, st, dev_err, g);
}

// E_out (w x w FP64, optional): Q^T Q - I of the stored Q, measured with an
// FP64-accumulated Gram, so that consumers can apply the first-order
// orthonormalisation Q (I - E/2) in FP64 without rewriting Q.
// Hlo (optional, FP32 data only): remainder array of H, kept up to date.
static void block_qr(bool f64, int64_t m, int nblk, int l, void* H, int64_t ld, double* R_out,
                     double* E_out, const QrScratch& s, uint32_t* dev_err, cudaStream_t st,
                     float* Hlo = nullptr) {
  const size_t es = f64 ? 8 : 4;
  const int w = nblk * l;
  const double piv_rel = f64 ? 1e-12 : 1e-5;
  const double shift_rel = f64 ? 1e-12 : 1e-5;
  if (f64 || m < kTcMinRows) Hlo = nullptr;
  if (Hlo) split_lo(m, w, (const float*)H, ld, Hlo, ld, st);
  if (R_out) RPCA_CUDA_TRY(cudaMemsetAsync(R_out, 0, (size_t)w * w * sizeof(double), st));
  for (int j = 0; j < nblk; ++j) {
    char* Hj = static_cast<char*>(H) + (size_t)j * l * es;
    float* Hjlo = Hlo ? Hlo + (size_t)j * l : nullptr;
    const int jl = j * l;
    if (j > 0) {
      for (int rep = 0; rep < 2; ++rep) {
        qr_gram(f64, m, jl, l, H, ld, Hj, ld, s.C, l, s, st, dev_err, nullptr, rep == 0);
        qr_apply(f64, m, jl, l, H, Hlo, ld, s.C, l, -1.0, 1.0, Hj, Hjlo, ld, s, st, dev_err);
        if (R_out) mat_add(jl, l, s.C, l, R_out + jl, w, st);
      }
    }
    uint32_t* qf = s.qf + kQfWords * j;
    if (R_out) set_identity(l, s.Racc, st);
    for (int pass = 0; pass < kCholPasses; ++pass) {
      const uint32_t* active = pass >= 2 ? qf + pass : nullptr;
      qr_gram(f64, m, l, l, Hj, ld, Hj, ld, s.Gm, l, s, st, dev_err, active);
      chol_small(l, s.Gm, l, s.Rk, s.Rinv, pass, piv_rel, shift_rel, qf, dev_err, st, false);
      qr_apply(f64, m, l, l, Hj, Hjlo, ld, s.Rinv, l, 1.0, 0.0, Hj, Hjlo, ld, s, st, dev_err, active);
      if (R_out) left_mul(l, s.Rk, s.Racc, st);
    }
    if (j > 0 && !R_out) reorth_after_shift(f64, m, jl, l, H, Hlo, ld, Hj, Hjlo, qf, piv_rel, shift_rel, s, dev_err,
                                            st);
    if (R_out) mat_add(l, l, s.Racc, l, R_out + (size_t)jl * w + jl, w, st);
  }
  if (E_out) {
    qr_gram(f64, m, w, w, H, ld, H, ld, E_out, w, s, st, dev_err);
    sub_identity(w, E_out, st);
  }
}

// Step 2 with H held in three exact BF16 slices (S: 3 planes of prow x nblk*64,
// block j at columns [64j, 64j + l)): block Gram-Schmidt twice and Cholesky
// QR (up to four passes) per block as in block_qr, Gram matrices and
// Cholesky factors in FP64, every tall product on tensor cores reading and
// writing the slices.  E_out (compact w x w) = Q^T Q - I.  fp32_out: Q is
// also written back to H in FP32.
static void block_qr_sliced(int64_t m, int nblk, int l, float* H, int64_t ld, void* S, int64_t prow, double* E_out,
                            bool fp32_out, const QrScratch& s, uint32_t* dev_err, cudaStream_t st) {
  const int lds = nblk * 64;
  const double piv_rel = 1e-5, shift_rel = 1e-5;
  auto need = [](bool ok) {
    if (!ok) throw Invalid("sliced tensor-core QR: unsupported shape");
  };
  slice_blocks(m, prow, nblk, l, H, ld, S, st);
  for (int j = 0; j < nblk; ++j) {
    if (j > 0) {
      for (int rep = 0; rep < 2; ++rep) {
        need(gram_slices(m, prow, S, lds, 0, 64 * j, 64 * j, 64, s.C64, 64, st, dev_err, nullptr));
        need(apply_slices(m, prow, S, lds, 0, j, 64 * j, s.C64, 64 * j, 64, 64, -1.0, 0, true, true, nullptr, 0, 0,
                          s.mt, st, dev_err, nullptr));
      }
    }
    uint32_t* qf = s.qf + kQfWords * j;
    for (int pass = 0; pass < kCholPasses; ++pass) {
      const uint32_t* active = pass >= 2 ? qf + pass : nullptr;
      need(gram_slices(m, prow, S, lds, 64 * j, 64, 64 * j, 64, s.G64, 64, st, dev_err, active));
      chol_small(l, s.G64, 64, s.Rk, s.Rinv, pass, piv_rel, shift_rel, qf, dev_err, st, false);
      need(apply_slices(m, prow, S, lds, 64 * j, 1, 64 * j, s.Rinv, l, l, l, 1.0, l, false, true, nullptr, 0, 0,
                        s.mt, st, dev_err, active));
    }
    if (j > 0) {
      // numerically rank-deficient block: one more projection and pass
      // (launches are no-ops unless a pass above needed a shift)
      const uint32_t* g = qf + 1;
      need(gram_slices(m, prow, S, lds, 0, 64 * j, 64 * j, 64, s.C64, 64, st, dev_err, g));
      need(apply_slices(m, prow, S, lds, 0, j, 64 * j, s.C64, 64 * j, 64, 64, -1.0, 0, true, true, nullptr, 0, 0,
                        s.mt, st, dev_err, g));
      need(gram_slices(m, prow, S, lds, 64 * j, 64, 64 * j, 64, s.G64, 64, st, dev_err, g));
      chol_small(l, s.G64, 64, s.Rk, s.Rinv, 1, piv_rel, shift_rel, qf, dev_err, st, false, g);
      need(apply_slices(m, prow, S, lds, 64 * j, 1, 64 * j, s.Rinv, l, l, l, 1.0, l, false, true, nullptr, 0, 0,
                        s.mt, st, dev_err, g));
    }
  }
  if (E_out) {
    // Q^T Q is symmetric: form the upper block triangle only (one read of
    // block j per block column >= j instead of every block per column)
    need(gram_slices(m, prow, S, lds, 0, lds, 0, lds, s.Cfull, lds, st, dev_err, nullptr, true));
    compact_sq(nblk, l, s.Cfull, lds, E_out, st);
    sub_identity(nblk * l, E_out, st);
  }
  if (fp32_out) unslice_blocks(m, prow, nblk, l, S, H, ld, st);
}

// Step 2 on H held in three exact BF16 slices as ONE Cholesky QR of all
// w = nblk l columns: the FP64 Gram G = H^T H (upper block triangle from
// the slices), the FP64 Cholesky G = R^T R by l x l blocks (k_chol on the
// diagonal blocks, FP64 products for the rest), then Q = H R^-1 block column
// by block column, the last first, in place.  With the block Lanczos form of
// Step 1 the columns of H are far from dependent (kappa(H) is that of A on
// the Krylov space), so one pass leaves Q^T Q - I at the rounding of the
// apply, which the first-order correction with the measured E_out absorbs.
// When the factor's conditioning estimate kappa (max / min |diag R|) is at
// most skip_e_kappa, that rounding is a few units of FP32 (u32 kappa) and
// the second Gram is not formed: E_out = 0 and *e_zero is set.
// The factorisation is checked before H is touched: when a diagonal block
// needed a shifted Cholesky (numerical rank loss) this returns false with H
// unchanged, and the block path with its shifted passes runs instead.  The
// check reads one word on the host, so this path is not used while the
// stream is being captured.
static bool block_qr_sliced_whole(int64_t m, int nblk, int l, float* H, int64_t ld, void* S, int64_t prow,
                                  double* E_out, bool fp32_out, const QrScratch& s, double* G, double* R,
                                  double* Rinv, double* tmp, uint32_t* dev_err, cudaStream_t st,
                                  double* kappa = nullptr, double skip_e_kappa = 0.0, bool* e_zero = nullptr) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RPCA_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) return false;
  const int lds = nblk * 64, w = nblk * l;
  const double piv_rel = 1e-5, shift_rel = 1e-5;
  auto need = [](bool ok) {
    if (!ok) throw Invalid("sliced tensor-core QR: unsupported shape");
  };
  slice_blocks(m, prow, nblk, l, H, ld, S, st);
  need(gram_slices(m, prow, S, lds, 0, lds, 0, lds, s.Cfull, lds, st, dev_err, nullptr, true));
  compact_sq(nblk, l, s.Cfull, lds, G, st);
  RPCA_CUDA_TRY(cudaMemsetAsync(R, 0, (size_t)w * w * sizeof(double), st));
  RPCA_CUDA_TRY(cudaMemsetAsync(Rinv, 0, (size_t)w * w * sizeof(double), st));
  auto blk = [&](double* M, int b, int c) { return M + (size_t)b * l * w + (size_t)c * l; };
  for (int b = 0; b < nblk; ++b) {
    // G_bb - sum_{a<b} R_ab^T R_ab, factored; R_bc = R_bb^-T (G_bc - sum_{a<b} R_ab^T R_ac)
    copy_matrix(true, true, l, l, blk(G, b, b), w, s.Gm, l, st);
    for (int a = 0; a < b; ++a)
      gemm64_small(l, l, l, -1.0, blk(R, a, b), w, true, blk(R, a, b), w, false, 1.0, s.Gm, l, s.Gm, l, st);
    chol_small(l, s.Gm, l, s.Rk, s.Rinv, 0, piv_rel, shift_rel, s.qf + kQfWords * b, dev_err, st, false);
    copy_matrix(true, true, l, l, s.Rk, l, blk(R, b, b), w, st);
    copy_matrix(true, true, l, l, s.Rinv, l, blk(Rinv, b, b), w, st);
    for (int c = b + 1; c < nblk; ++c) {
      copy_matrix(true, true, l, l, blk(G, b, c), w, tmp, l, st);
      for (int a = 0; a < b; ++a)
        gemm64_small(l, l, l, -1.0, blk(R, a, b), w, true, blk(R, a, c), w, false, 1.0, tmp, l, tmp, l, st);
      gemm64_small(l, l, l, 1.0, s.Rinv, l, true, tmp, l, false, 0.0, nullptr, 0, blk(R, b, c), w, st);
    }
  }
  // any shifted diagonal block: leave H to the block path
  std::vector<uint32_t> qf((size_t)kQfWords * nblk);
  std::vector<double> rd(w);
  RPCA_CUDA_TRY(cudaMemcpyAsync(qf.data(), s.qf, qf.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RPCA_CUDA_TRY(cudaMemcpy2DAsync(rd.data(), sizeof(double), R, (size_t)(w + 1) * sizeof(double), sizeof(double), w,
                                  cudaMemcpyDeviceToHost, st));
  RPCA_CUDA_TRY(cudaStreamSynchronize(st));
  for (int b = 0; b < nblk; ++b)
    if (qf[(size_t)kQfWords * b + 1]) return false;
  double kap;
  {
    double lo = INFINITY, hi = 0.0;
    for (double v : rd) {
      lo = std::min(lo, std::fabs(v));
      hi = std::max(hi, std::fabs(v));
    }
    kap = lo > 0.0 ? hi / lo : INFINITY;
  }
  if (kappa) *kappa = kap;
  const bool skip_e = E_out && kap <= skip_e_kappa;
  if (e_zero) *e_zero = skip_e;
  // R^-1 (upper): Rinv_bc = -R_bb^-1 sum_{b<a<=c} R_ba Rinv_ac, from the diagonal outwards
  for (int c = 1; c < nblk; ++c)
    for (int b = c - 1; b >= 0; --b) {
      RPCA_CUDA_TRY(cudaMemsetAsync(tmp, 0, (size_t)l * l * sizeof(double), st));
      for (int a = b + 1; a <= c; ++a)
        gemm64_small(l, l, l, 1.0, blk(R, b, a), w, false, blk(Rinv, a, c), w, false, 1.0, tmp, l, tmp, l, st);
      gemm64_small(l, l, l, -1.0, blk(Rinv, b, b), w, false, tmp, l, false, 0.0, nullptr, 0, blk(Rinv, b, c), w, st);
    }
  // Q_j = sum_{b<=j} H_b Rinv_bj, last block first (each reads the blocks at or before it)
  for (int j = nblk - 1; j >= 0; --j)
    need(apply_slices(m, prow, S, lds, 0, j + 1, 64 * j, Rinv + (size_t)j * l, (j + 1) * l, l, w, 1.0, l, false,
                      true, nullptr, 0, 0, s.mt, st, dev_err, nullptr));
  if (skip_e) {
    RPCA_CUDA_TRY(cudaMemsetAsync(E_out, 0, (size_t)w * w * sizeof(double), st));
  } else if (E_out) {
    need(gram_slices(m, prow, S, lds, 0, lds, 0, lds, s.Cfull, lds, st, dev_err, nullptr, true));
    compact_sq(nblk, l, s.Cfull, lds, E_out, st);
    sub_identity(nblk * l, E_out, st);
  }
  if (fp32_out) unslice_blocks(m, prow, nblk, l, S, H, ld, st);
  return true;
}

// Step 4 on T (n x w, ld w, compute type): T = Q_T R_T with Q_T from the
// block QR (in place of T) and R_T = Q_T^T T_orig (FP64-accumulated Gram);
// with E_T = Q_T^T Q_T - I the orthonormal basis is Q_T (I - E_T/2) to first
// order and its triangular factor (I - E_T/2) R_T.  Then R_T' = Ub S W^T by
// one-sided Jacobi.  Tc: n x w scratch (copy of T).
static void svd_of_T(bool f64, int64_t n, int nblk, int l, int kk, void* T, void* Tc, float* Tlo, double* ET,
                     double* RT, double* RT2, double* S, double* Ub, double* W, double* svdwork,
                     const QrScratch& qs, uint32_t* dev_err, cudaStream_t st) {
  const int w = nblk * l;
  const size_t es = f64 ? 8 : 4;
  RPCA_CUDA_TRY(cudaMemcpyAsync(Tc, T, (size_t)n * w * es, cudaMemcpyDeviceToDevice, st));
  block_qr(f64, n, nblk, l, T, w, nullptr, ET, qs, dev_err, st, Tlo);
  qr_gram(f64, n, w, w, T, w, Tc, w, RT, w, qs, st, dev_err);
  // R_T' = (I - E_T/2) R_T in FP64
  gemm64_small(w, w, w, -0.5, ET, w, false, RT, w, false, 1.0, RT, w, RT2, w, st);
  jacobi_svd(f64, w, kk, RT2, S, Ub, W, svdwork, dev_err, st);
}

// Mk (w x k) = (I - E/2) M[:, :k]  (first-order orthonormalisation applied
// to the small factor)
static void fold_fixup(bool f64, int w, int k, const double* E, const double* M, double* Mk, cudaStream_t st) {
  (void)f64;
  gemm64_small(w, k, w, -0.5, E, w, false, M, w, false, 1.0, M, w, Mk, k, st);
}

}  // namespace rpca

using namespace rpca;

// ============================================================ the context
struct rpca_ctx {
  rpca_problem prob{};
  bool f64 = false, transposed = false, host_a = false, simt = false;
  // block Lanczos form (every context but RPCA_ADJOINT ones): the n-side
  // blocks X^(0..i) are kept orthonormal to each other in Xall (n x w)
  bool reorth = false;
  DevBuf Xall;
  // T without its own pass over A: T = A^T Q = [F^(0) .. F^(i)] R^-1 from
  // the F blocks the fused passes accumulate anyway (Fall, n x w FP32), when
  // the whole-H Cholesky QR ran and kappa(R) is small (the F blocks' error
  // is amplified by it).  Converter-kernel storage only (FP32, FP8), whose F
  // carries FP32-class error.
  bool mirror = false;
  bool mirrored_last = false;    // the last run formed T this way
  double last_kappa = 0.0;       // max/min diagonal of R in the last whole-H QR
  bool e_zero = false;           // the last run's E = Q^T Q - I was taken as 0 (kappa small)
  DevBuf Fall;
  // RPCA_HOST_RESIDENT: device copy of host A, valid once this run's first
  // pass has copied every tile
  bool resident = false, resident_valid = false;
  DevBuf Ares;
  int64_t m = 0, n = 0;   // working orientation (m >= n)
  int k = 0, l = 0, i = 0, w = 0;
  int64_t ldx = 0;        // ld of X and F (compute type)
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  int next_pass = 0;
  bool centered = false;
  std::string last_error;

  DevBuf X, F, H, T, Tc, shift, corr, d, vtmp, q1, G64, small, err, At, tiles[2], work, Hlo, Tlo, mt, slices;
  // adjoint: saved X^(j) blocks and backward workspace
  bool adjoint = false, fwd_done = false;
  DevBuf Xsave, Bcat, XM, Hb, Tm, Xb64, Xb, Dn, Fb, Mw, Pf, Zf, bsmall;
  // H in three BF16 slices for the tensor-core QR (sliced_ok)
  bool sliced = false;
  int64_t hs_rows = 0;
  DevBuf Hs, sq;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  int64_t tile_rows = 0;
  QrScratch qs;
  double *RT = nullptr, *S = nullptr, *Ub = nullptr, *W = nullptr, *svdwork = nullptr;
  double *E = nullptr, *ET = nullptr, *RT2 = nullptr, *MU = nullptr, *MV = nullptr;
  DevBuf T64;
  DevBuf outU, outV;
  // per-phase CUDA-event timing (RPCA_TIMING): phases 0..i are the fused
  // passes' streaming kernels, i+1 the QR of H, i+2 the T pass, i+3 Step 4
  // (QR of T and the small SVD), i+4 the products forming U and V
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  std::vector<double> phase_ms;
  int timed_runs = 0;

  void tic(int ph) {
    if (timing) RPCA_CUDA_TRY(cudaEventRecord(ev[2 * ph], stream));
  }
  void toc(int ph) {
    if (timing) RPCA_CUDA_TRY(cudaEventRecord(ev[2 * ph + 1], stream));
  }

  ~rpca_ctx() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (int t = 0; t < 2; ++t) {
      if (ev_copied[t]) cudaEventDestroy(ev_copied[t]);
      if (ev_used[t]) cudaEventDestroy(ev_used[t]);
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
  }
  size_t cbytes() const { return f64 ? 8 : 4; }
  uint32_t* dev_err() const { return err.as<uint32_t>(); }
};

namespace {

rpca_status fail(rpca_ctx* c, rpca_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

template <typename Fn>
rpca_status guarded(rpca_ctx* c, Fn&& fn) {
  try {
    return fn();
  } catch (const CudaFailure& e) {
    rpca_status s = RPCA_ECUDA;
    if (e.code == cudaErrorMemoryAllocation) s = RPCA_ENOMEM;
    if (e.code == cudaErrorNoDevice || e.code == cudaErrorInsufficientDriver) s = RPCA_ENODEV;
    return fail(c, s, e.what);
  } catch (const Invalid& e) {
    return fail(c, RPCA_EINVAL, e.what);
  } catch (const std::bad_alloc&) {
    return fail(c, RPCA_ENOMEM, "host allocation failed");
  }
}

void validate(const rpca_problem* p) {
  if (!p) throw Invalid("null problem");
  if (p->m < 1 || p->n < 1) throw Invalid("m and n must be positive");
  const int64_t mn = std::min(p->m, p->n);
  if (p->k < 1 || p->k >= mn) throw Invalid("need 1 <= k < min(m, n)");
  if (p->l < p->k) throw Invalid("need l >= k");
  if (p->i < 0) throw Invalid("need i >= 0");
  if ((int64_t)(p->i + 1) * p->l > mn) throw Invalid("need (i+1) l <= min(m, n)");
  if (p->l > 255) throw Invalid("l > 255 is not supported");
  if ((int64_t)(p->i + 1) * p->l > 256) throw Invalid("(i+1) l > 256 is not supported");
  if (p->dtype < RPCA_F64 || p->dtype > RPCA_FP8E4M3) throw Invalid("unknown dtype");
  if (p->flags & ~(RPCA_CENTER | RPCA_HOST_A | RPCA_SIMT | RPCA_TIMING | RPCA_ADJOINT | RPCA_HOST_RESIDENT |
                   RPCA_KEEP_T_PASS | RPCA_NO_GROUPED))
    throw Invalid("unknown flag");
  if ((p->flags & RPCA_HOST_RESIDENT) && !(p->flags & RPCA_HOST_A)) throw Invalid("RPCA_HOST_RESIDENT needs RPCA_HOST_A");
  if ((p->flags & RPCA_ADJOINT) && ((p->flags & (RPCA_CENTER | RPCA_HOST_A)) || p->n > p->m))
    throw Invalid("RPCA_ADJOINT needs m >= n, no centring and device A");
  if ((p->flags & RPCA_HOST_A) && p->n > p->m) throw Invalid("RPCA_HOST_A needs n <= m");
}

// Device scratch of the tensor-core passes: the BF16 copy of Q (T pass),
// or, for FP32 A (converter kernels), two BF16 planes of Q, or the X^T
// slices plus the two BF16 planes of H that the F pass reads.
size_t tc_work_bytes(rpca_dtype dt, int64_t m, int64_t n, int w) {
  (void)dt;   // every storage type may take the converter kernels (FP32, FP8, shifted BF16)
  const size_t b = std::max<size_t>((size_t)2 * m * round_up(w, 64) * 2,
                                    (size_t)2 * 64 * round_up(n, 128) * 2 + 256 + (size_t)2 * m * 64 * 2);
  return b + 4096;
}

// kappa(R) up to which T is formed from the F blocks: their relative error
// (~1e-5 from the BF16 hi/lo products) times kappa stays below the FP32
// tolerance on sigma (1e-4).
constexpr double kMirrorKappa = 8.0;
// Largest kappa estimate of the whole-H factor for which E = Q^T Q - I is
// taken as 0 (no second Gram): u32 kappa stays below 1e-6.
constexpr double kSkipEKappa = 16.0;

// Smallest sigma_k / sigma_1 for which Step 4 stays on the Gram route (its
// FP32 preconditioner shifts G by 1e-6 of the largest eigenvalue).
constexpr double kGramMinRatio = 1.7e-3;

// Step 4 from the Gram of T (FP32-class storage; the single-CTA Cholesky
// preconditioner takes w <= 192), else from a QR of T.
bool gram_step4(const rpca_ctx* c) { return !c->f64 && c->w <= 192 && !c->adjoint && c->reorth; }

// Will the T pass of an FP32 context read the first two BF16 slices of the
// sliced Q directly (converter kernel; TMA-aligned A)?
bool tpass_f32_slices_ok(const rpca_ctx* c, const rpca_matrix* Am) {
  const rpca_dtype dt = c->prob.dtype;
  if ((dt != RPCA_F32 && dt != RPCA_FP8E4M3) || !c->sliced || c->simt || c->adjoint) return false;
  const int64_t eb = (int64_t)dtype_bytes(dt);
  if (c->host_a) return (c->n * eb) % 16 == 0;
  const void* A = c->transposed ? c->At.ptr : Am->data;
  const int64_t lda = c->transposed ? c->n : Am->ld;
  return (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda * eb) % 16 == 0;
}

// One streamed pass over the working matrix (device-resident or tiles).
// Will the T pass run on the BF16 tensor-core kernel (TMA-aligned A, no
// centring shift or column scale)?
bool tpass_bf16_ok(const rpca_ctx* c, const rpca_matrix* Am) {
  if (c->prob.dtype != RPCA_BF16 || c->centered || c->simt || Am->col_scale) return false;
  if (c->host_a) return (c->n * 2) % 16 == 0 && (!c->resident || c->w <= 192);
  const void* A = c->transposed ? c->At.ptr : Am->data;
  const int64_t lda = c->transposed ? c->n : Am->ld;
  return (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda * 2) % 16 == 0 && c->w <= 192;
}

void run_pass(rpca_ctx* c, const rpca_matrix* Am, PassArgs a) {
  const size_t ab = dtype_bytes(c->prob.dtype);
  a.work = c->work.ptr;
  a.work_bytes = c->work.bytes;
  if (!c->host_a || (c->resident && c->resident_valid)) {
    const bool res = c->host_a;                     // the context's device copy of A
    a.A = res ? c->Ares.ptr : (c->transposed ? c->At.ptr : Am->data);
    a.lda = res ? c->n : (c->transposed ? c->n : Am->ld);
    a.m = c->m;
    if (!(c->simt) && launch_pass_tc(a, c->stream, c->dev_err())) return;
    if (a.q16) throw Invalid("T pass: tensor-core kernel refused its BF16 operand");
    launch_pass_simt(a, c->stream);
    return;
  }
  // Out-of-core form (Section 4.2): stream tiles of rows from host memory,
  // two device buffers, copies on their own stream overlapping the kernels.
  const int64_t tr = c->tile_rows;
  const int64_t ntiles = cdiv(c->m, tr);
  const size_t es = c->cbytes();
  const size_t fcols = a.p + (a.ones_col >= 0 ? 1 : 0);
  const size_t fes = a.f_f64 ? 8 : es;
  if (a.F && a.mode != MODE_H)
    RPCA_CUDA_TRY(cudaMemset2DAsync(a.F, a.ldf * fes, 0, fcols * fes, a.n, c->stream));
  // resident copy: tile t lands in its final place (no buffer reuse, so no
  // wait for the kernel of tile t - 2)
  const bool to_res = c->resident;
  for (int64_t t = 0; t < ntiles; ++t) {
    const int b = (int)(t & 1);
    const int64_t r0 = t * tr, rows = std::min(tr, c->m - r0);
    char* dst = to_res ? static_cast<char*>(c->Ares.ptr) + (size_t)r0 * c->n * ab : static_cast<char*>(c->tiles[b].ptr);
    if (!to_res) RPCA_CUDA_TRY(cudaStreamWaitEvent(c->copy_stream, c->ev_used[b], 0));
    const char* src = static_cast<const char*>(Am->data) + (size_t)r0 * Am->ld * ab;
    RPCA_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)c->n * ab, src, (size_t)Am->ld * ab,
                                    (size_t)c->n * ab, (size_t)rows, cudaMemcpyHostToDevice,
                                    c->copy_stream));
    RPCA_CUDA_TRY(cudaEventRecord(c->ev_copied[b], c->copy_stream));
    RPCA_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_copied[b], 0));
    PassArgs ta = a;
    ta.A = dst;
    ta.lda = c->n;
    ta.m = rows;
    ta.H = static_cast<char*>(a.H) + (size_t)r0 * a.ldh * es;
    if (a.q16) ta.q16 = static_cast<const __nv_bfloat16*>(a.q16) + (size_t)r0 * a.q16_ld;
    ta.accumulate_f = true;
    if (!(c->simt) && launch_pass_tc(ta, c->stream, c->dev_err())) {
    } else {
      if (ta.q16) throw Invalid("T pass: tensor-core kernel refused its BF16 operand");
      launch_pass_simt(ta, c->stream);
    }
    RPCA_CUDA_TRY(cudaEventRecord(c->ev_used[b], c->stream));
  }
  if (to_res) c->resident_valid = true;
}

void compute_shift(rpca_ctx* c, const rpca_matrix* Am) {
  // s = column means of the first rows (at most 128) of A, in the compute type
  const int64_t rows = std::min<int64_t>(c->m, 128);
  if (c->host_a) {
    const size_t ab = dtype_bytes(c->prob.dtype);
    RPCA_CUDA_TRY(cudaMemcpy2DAsync(c->tiles[0].ptr, (size_t)c->n * ab, Am->data, (size_t)Am->ld * ab,
                                    (size_t)c->n * ab, (size_t)rows, cudaMemcpyHostToDevice, c->stream));
    panel_mean(c->prob.dtype, c->tiles[0].ptr, c->n, rows, c->n, Am->col_scale, c->shift.ptr, c->stream);
    RPCA_CUDA_TRY(cudaEventRecord(c->ev_used[0], c->stream));
  } else {
    const void* A = c->transposed ? c->At.ptr : Am->data;
    const int64_t lda = c->transposed ? c->n : Am->ld;
    panel_mean(c->prob.dtype, A, lda, rows, c->n, Am->col_scale, c->shift.ptr, c->stream);
  }
}

void reset_x(rpca_ctx* c) {
  // X = G in the compute type, ld = ldx (the normalised iteration without
  // reorthogonalisation; the block Lanczos form keeps X^(0) = orth(G) in Xall)
  if (!c->reorth) copy_matrix(true, c->f64, c->n, c->l, c->G64.ptr, c->l, c->X.ptr, c->ldx, c->stream);
}

// n-side block j of the block Lanczos basis (Xall, ld w)
static void* xall_block(rpca_ctx* c, int j) { return static_cast<char*>(c->Xall.ptr) + (size_t)j * c->l * c->cbytes(); }

rpca_status do_pass(rpca_ctx* c, const rpca_matrix* Am) {
  if (!Am || !Am->data) throw Invalid("null matrix");
  if (c->next_pass > c->i + 1) throw Invalid("all passes already done");
  const bool f64 = c->f64;
  const size_t es = c->cbytes();
  const int64_t ld_orig = Am->ld;
  const int64_t ncols_orig = c->transposed ? c->m : c->n;
  if (ld_orig < ncols_orig) throw Invalid("ld < n");
  if (c->prob.dtype == RPCA_FP8E4M3 && !Am->col_scale) throw Invalid("FP8 needs col_scale");
  if (c->transposed && Am->col_scale) throw Invalid("col_scale with n > m is not supported");
  cudaStream_t st = c->stream;
  const int j = c->next_pass;
  if (j == 0) {
    RPCA_CUDA_TRY(cudaMemsetAsync(c->err.ptr, 0, 64 * sizeof(uint32_t), st));
    c->fwd_done = false;
    c->resident_valid = false;         // this run's A is copied by its first pass
    if (c->transposed)
      transpose(c->prob.dtype, c->m, c->n, Am->data, Am->ld, c->At.ptr, c->n, st);
    if (c->centered) compute_shift(c, Am);
    reset_x(c);
    if (c->adjoint) copy_matrix(f64, f64, c->n, c->l, c->X.ptr, c->ldx, c->Xsave.ptr, c->l, st);
  }
  PassArgs a;
  a.dtype = c->prob.dtype;
  a.n = c->n;
  a.scale = Am->col_scale;
  a.shift = c->centered ? c->shift.ptr : nullptr;
  if (j <= c->i) {
    // Step 1: pass j forms H^(j) = A_c X and (j < i) F = A_c^T H^(j)
    a.mode = (j < c->i || c->mirror) ? MODE_FUSED : MODE_H;
    void* Xj = c->reorth ? xall_block(c, j) : c->X.ptr;
    const int64_t ldxj = c->reorth ? c->w : c->ldx;
    a.X = Xj;
    a.ldx = ldxj;
    a.p = c->l;
    a.H = static_cast<char*>(c->H.ptr) + (size_t)j * c->l * es;
    a.ldh = c->w;
    a.F = c->F.ptr;
    a.ldf = c->ldx;
    if (c->centered && j == 0 && c->i > 0) a.ones_col = c->l;
    if (c->centered && j == 0 && c->i == 0) a.ones_col = c->l, a.mode = MODE_FUSED;
    if (c->centered && j > 0) {
      // corr = d^T X: H = A~ X - 1 (d^T X)   (A_c = A~ - 1 d^T)
      vec_mat(f64, c->n, c->l, c->d.as<double>(), Xj, ldxj, c->vtmp.as<double>(), st);
      cast_f64_to(f64, c->l, c->vtmp.as<double>(), c->corr.ptr, st);
      a.corr = c->corr.ptr;
    }
    c->tic(j);
    run_pass(c, Am, a);
    c->toc(j);
    if (c->centered && j == 0) {
      // d = A~^T 1 / m = c - s;  H^(0) -= 1 (d^T G);  F -= m d (d^T G)
      column_to_vec(f64, c->n, c->F.ptr, c->ldx, c->l, 1.0 / (double)c->m, c->d.as<double>(), st);
      vec_mat(f64, c->n, c->l, c->d.as<double>(), Xj, ldxj, c->vtmp.as<double>(), st);
      sub_rowvec(f64, c->m, c->l, c->vtmp.as<double>(), c->H.ptr, c->w, st);
      if (j < c->i || c->mirror)
        rank1_sub(f64, c->n, c->l, (double)c->m, c->d.as<double>(), c->vtmp.as<double>(), c->F.ptr,
                  c->ldx, st);
    }
    // F^(j) = A_c^T H^(j), kept for forming T without a pass
    if (c->mirror)
      copy_matrix(f64, f64, c->n, c->l, c->F.ptr, c->ldx, static_cast<char*>(c->Fall.ptr) + (size_t)j * c->l * es,
                  c->w, st);
    if (j < c->i && c->reorth) {
      // block Lanczos: X^(j+1) = orth(F - X_{<=j} X_{<=j}^T F), the
      // projection applied twice (same Krylov space as orth(F), far better
      // conditioned H)
      const int jl = (j + 1) * c->l;
      for (int rep = 0; rep < 2; ++rep) {
        qr_gram(f64, c->n, jl, c->l, c->Xall.ptr, c->w, c->F.ptr, c->ldx, c->qs.C, c->l, c->qs, st, c->dev_err());
        qr_apply(f64, c->n, jl, c->l, c->Xall.ptr, nullptr, c->w, c->qs.C, c->l, -1.0, 1.0, c->F.ptr, nullptr,
                 c->ldx, c->qs, st, c->dev_err());
      }
      block_qr(f64, c->n, 1, c->l, c->F.ptr, c->ldx, nullptr, nullptr, c->qs, c->dev_err(), st);
      copy_matrix(f64, f64, c->n, c->l, c->F.ptr, c->ldx, xall_block(c, j + 1), c->w, st);
    } else if (j < c->i) {
      // normalised iteration: X = orth(F)
      block_qr(f64, c->n, 1, c->l, c->F.ptr, c->ldx, nullptr, nullptr, c->qs, c->dev_err(), st);
      std::swap(c->X.ptr, c->F.ptr);
      std::swap(c->X.bytes, c->F.bytes);
      if (c->adjoint)
        copy_matrix(f64, f64, c->n, c->l, c->X.ptr, c->ldx,
                    static_cast<char*>(c->Xsave.ptr) + (size_t)(j + 1) * c->n * c->l * es, c->l, st);
    }
    c->next_pass = j + 1;
    return RPCA_MORE;
  }
  // Step 2: H = Q R (Q in place of H); Step 3: T = A_c^T Q
  // The BF16 tensor-core T pass reads slice 1 of the sliced Q (= RNE_bf16(Q));
  // every other T pass reads Q in FP32.
  const bool t16 = c->sliced && tpass_bf16_ok(c, Am);
  const bool t32s = tpass_f32_slices_ok(c, Am);
  c->tic(c->i + 1);
  const bool q32 = !(t16 || t32s) || c->adjoint;
  bool whole = false;
  c->e_zero = false;
  if (c->sliced) {
    // the whole-H Cholesky QR's scratch (G, R, R^-1, one block): Step 4's
    // work area, free until then
    const size_t ww = (size_t)c->w * c->w;
    double* sw = c->svdwork;
    whole = c->reorth && block_qr_sliced_whole(c->m, c->i + 1, c->l, c->H.as<float>(), c->w, c->Hs.ptr, c->hs_rows,
                                               c->E, q32, c->qs, sw, sw + 2 * ww, sw + ww, sw + 3 * ww, c->dev_err(),
                                               st, &c->last_kappa, kSkipEKappa, &c->e_zero);
    if (!whole)
      block_qr_sliced(c->m, c->i + 1, c->l, c->H.as<float>(), c->w, c->Hs.ptr, c->hs_rows, c->E, q32, c->qs,
                      c->dev_err(), st);
  } else {
    block_qr(f64, c->m, c->i + 1, c->l, c->H.ptr, c->w, nullptr, c->E, c->qs, c->dev_err(), st,
             c->Hlo.as<float>());
  }
  c->toc(c->i + 1);
  // T = [F^(0) .. F^(i)] R^-1 (FP32 products; R^-1 from the whole-H
  // factorisation, still in Step 4's work area) when kappa(R) keeps the F
  // blocks' FP32-class error below the FP32 tolerances
  c->mirrored_last = c->mirror && whole && c->last_kappa <= kMirrorKappa;
  if (c->mirrored_last) {
    c->tic(c->i + 2);
    gemm_xm(false, c->n, c->w, c->w, c->Fall.ptr, c->w, c->svdwork + (size_t)c->w * c->w, c->w, 1.0, 0.0, c->T.ptr,
            c->w, st);
    copy_matrix(false, true, c->n, c->w, c->T.ptr, c->w, c->T64.ptr, c->w, st);
    c->toc(c->i + 2);
    if (!gram_step4(c) && !c->e_zero)
      gemm_xm(f64, c->n, c->w, c->w, c->T.ptr, c->w, c->E, c->w, -0.5, 1.0, c->T.ptr, c->w, st);
    c->next_pass = c->i + 2;
    return RPCA_OK;
  }
  a.mode = MODE_T;
  a.p = c->w;
  a.H = c->H.ptr;
  a.ldh = c->w;
  if (t16 || t32s) {
    a.q16 = c->Hs.ptr;
    a.q16_ld = (c->i + 1) * 64;
    a.q_blk = c->l;
    // FP32: Q = slice 1 + slice 2 (the third slice is below 2^-17 of Q)
    if (t32s) a.q16_plane = c->hs_rows * (c->i + 1) * 64;
  }
  a.F = c->T64.ptr;   // FP64 accumulation across row blocks
  a.ldf = c->w;
  a.f_f64 = true;
  c->tic(c->i + 2);
  run_pass(c, Am, a);
  c->toc(c->i + 2);
  const bool q_in_h = !(c->sliced && (t16 || t32s) && !c->adjoint);   // Q also in H (FP32)
  if (gram_step4(c)) {
    // T = A~^T Q - d (1^T Q), kept in FP64 for the Gram of Step 4; the
    // first-order orthonormalisation (I - E/2) is applied to that Gram and
    // to the small factor instead of to T
    if (c->centered) {
      if (q_in_h) col_sums(f64, c->m, c->w, c->H.ptr, c->w, c->q1.as<double>(), st);
      else col_sums_slices(c->m, c->hs_rows, c->i + 1, c->l, c->Hs.ptr, c->q1.as<double>(), st);
      rank1_sub(true, c->n, c->w, 1.0, c->d.as<double>(), c->q1.as<double>(), c->T64.ptr, c->w, st);
    }
    copy_matrix(true, f64, c->n, c->w, c->T64.ptr, c->w, c->T.ptr, c->w, st);
    c->next_pass = c->i + 2;
    return RPCA_OK;
  }
  copy_matrix(true, f64, c->n, c->w, c->T64.ptr, c->w, c->T.ptr, c->w, st);
  if (c->centered) {
    // T = A~^T Q - d (1^T Q)
    if (q_in_h) col_sums(f64, c->m, c->w, c->H.ptr, c->w, c->q1.as<double>(), st);
    else col_sums_slices(c->m, c->hs_rows, c->i + 1, c->l, c->Hs.ptr, c->q1.as<double>(), st);
    rank1_sub(f64, c->n, c->w, 1.0, c->d.as<double>(), c->q1.as<double>(), c->T.ptr, c->w, st);
  }
  // T <- T (I - E/2): the Rayleigh-Ritz matrix of the orthonormalised basis
  if (!c->e_zero) gemm_xm(f64, c->n, c->w, c->w, c->T.ptr, c->w, c->E, c->w, -0.5, 1.0, c->T.ptr, c->w, st);
  c->next_pass = c->i + 2;
  return RPCA_OK;
}

// Steps 4-6 and the copies into the caller's buffers, queued on the context
// stream only (no host synchronisation: usable inside a stream capture).
void do_finish_enqueue(rpca_ctx* c, void* U, int64_t ldu, double* S, void* V, int64_t ldv) {
  if (c->next_pass != c->i + 2) throw Invalid("finish before all passes");
  const bool f64 = c->f64;
  cudaStream_t st = c->stream;
  const size_t es = c->cbytes();
  // Step 4: T = Q_T R_T; with E_T = Q_T^T Q_T - I, T = (Q_T (I - E_T/2))
  // ((I + E_T/2) R_T) to first order; R_T' = Ub S W^T  =>  V~ = Q_T (I - E_T/2) Ub
  const int w = c->w, k = c->k;
  bool g4 = gram_step4(c);
  c->tic(c->i + 3);
  if (g4) {
    // Step 4 from G = T^T T (FP64-class, in FP32 arithmetic with compensated
    // sums): G' = (I - E/2) G (I - E/2) is the Gram
    // of the Rayleigh-Ritz matrix of the orthonormalised basis; its
    // eigenvectors W are T's right singular vectors and V = T (I - E/2) W / sigma
    gram_sym_comp(c->n, w, c->T64.as<double>(), w, c->RT, w, st);
    if (!c->e_zero) {
      gemm64_small(w, w, w, -0.5, c->E, w, false, c->RT, w, false, 1.0, c->RT, w, c->RT2, w, st);
      gemm64_small(w, w, w, -0.5, c->RT2, w, false, c->E, w, false, 1.0, c->RT2, w, c->RT, w, st);
    }
    svd_from_gram(w, c->RT, c->S, c->Ub, c->W, c->svdwork, c->dev_err(), st);
    // The FP32 preconditioner of that route shifts G by 1e-6 of its largest
    // eigenvalue: eigenvalues below a few shifts (sigma_k / sigma_1 < 1.7e-3)
    // are not resolved, and the QR route of Step 4 (relative accuracy for
    // the small singular values) runs instead.  The check reads two words
    // on the host, so it is left out while the stream is captured.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    RPCA_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap == cudaStreamCaptureStatusNone) {
      double s0 = 0.0, sk = 0.0;
      RPCA_CUDA_TRY(cudaMemcpyAsync(&s0, c->S, sizeof(double), cudaMemcpyDeviceToHost, st));
      RPCA_CUDA_TRY(cudaMemcpyAsync(&sk, c->S + (k - 1), sizeof(double), cudaMemcpyDeviceToHost, st));
      RPCA_CUDA_TRY(cudaStreamSynchronize(st));
      if (sk < kGramMinRatio * s0) {
        if (!c->e_zero) gemm_xm(f64, c->n, w, w, c->T.ptr, w, c->E, w, -0.5, 1.0, c->T.ptr, w, st);   // T (I - E/2)
        g4 = false;
      }
    }
  }
  if (!g4) {
    svd_of_T(f64, c->n, c->i + 1, c->l, c->k, c->T.ptr, c->Tc.ptr, c->Tlo.as<float>(), c->ET, c->RT, c->RT2, c->S,
             c->Ub, c->W, c->svdwork, c->qs, c->dev_err(), st);
  }
  c->toc(c->i + 3);
  c->tic(c->i + 4);
  // Steps 5-6: U = Q (I - E/2) W[:, :k], V = Q_T (I - E_T/2) Ub[:, :k] (QR
  // form) or V = T (I - E/2) Ub[:, :k] with Ub = W / sigma (Gram form)
  // (working orientation; swapped back when the problem was transposed)
  if (g4 && c->e_zero) copy_matrix(true, true, w, k, c->Ub, w, c->MV, k, st);
  else fold_fixup(f64, w, k, g4 ? c->E : c->ET, c->Ub, c->MV, st);
  if (c->e_zero) copy_matrix(true, true, w, k, c->W, w, c->MU, k, st);
  else fold_fixup(f64, w, k, c->E, c->W, c->MU, st);
  const bool tlo = !g4 && c->Tlo.ptr && c->n >= kTcMinRows;
  const bool hlo = c->Hlo.ptr && c->m >= kTcMinRows;
  qr_apply(f64, c->n, w, k, c->T.ptr, tlo ? c->Tlo.as<float>() : nullptr, w, c->MV, k, 1.0, 0.0, c->outV.ptr,
           nullptr, k, c->qs, st, c->dev_err());
  if (c->sliced) {
    // U = Q M_U with Q in slices (block-padded rows of M_U)
    if (!apply_slices(c->m, c->hs_rows, c->Hs.ptr, (c->i + 1) * 64, 0, c->i + 1, 0, c->MU, w, k, k, 1.0, c->l,
                      false, false, c->outU.as<float>(), k, k, c->qs.mt, st, c->dev_err(), nullptr))
      throw Invalid("sliced tensor-core product U = Q M: unsupported shape");
  } else {
    qr_apply(f64, c->m, w, k, c->H.ptr, hlo ? c->Hlo.as<float>() : nullptr, w, c->MU, k, 1.0, 0.0, c->outU.ptr,
             nullptr, k, c->qs, st, c->dev_err());
  }
  c->toc(c->i + 4);
  void* Uw = c->transposed ? V : U;
  int64_t ldUw = c->transposed ? ldv : ldu;
  void* Vw = c->transposed ? U : V;
  int64_t ldVw = c->transposed ? ldu : ldv;
  if (Uw) {
    if (ldUw < c->k) throw Invalid("ldu/ldv < k");
    RPCA_CUDA_TRY(cudaMemcpy2DAsync(Uw, ldUw * es, c->outU.ptr, c->k * es, c->k * es, c->m,
                                    cudaMemcpyDefault, st));
  }
  if (Vw) {
    if (ldVw < c->k) throw Invalid("ldu/ldv < k");
    RPCA_CUDA_TRY(cudaMemcpy2DAsync(Vw, ldVw * es, c->outV.ptr, c->k * es, c->k * es, c->n,
                                    cudaMemcpyDefault, st));
  }
  if (S) RPCA_CUDA_TRY(cudaMemcpyAsync(S, c->S, c->k * sizeof(double), cudaMemcpyDefault, st));
  c->fwd_done = true;
}

// Waits for the context stream and reports device-side errors of the run.
rpca_status do_finish_check(rpca_ctx* c) {
  cudaStream_t st = c->stream;
  uint32_t flags = 0;
  RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, c->err.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RPCA_CUDA_TRY(cudaStreamSynchronize(st));
  if (c->timing) {
    for (size_t ph = 0; ph < c->phase_ms.size(); ++ph) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev[2 * ph], c->ev[2 * ph + 1]) == cudaSuccess) c->phase_ms[ph] += ms;
      else cudaGetLastError();
    }
    c->timed_runs += 1;
  }
  if (flags & DEV_ERR_TIMEOUT) return fail(c, RPCA_ETIMEOUT, "a device-side wait timed out");
  if (flags & DEV_ERR_BREAKDOWN) return fail(c, RPCA_EBREAKDOWN, "Cholesky QR broke down");
  return RPCA_OK;
}

rpca_status do_finish(rpca_ctx* c, void* U, int64_t ldu, double* S, void* V, int64_t ldv) {
  do_finish_enqueue(c, U, ldu, S, V, ldv);
  return do_finish_check(c);
}

rpca_status do_init(rpca_ctx* c, const rpca_problem* p) {
  validate(p);
  check_device();
  c->prob = *p;
  c->f64 = p->dtype == RPCA_F64;
  c->transposed = p->n > p->m;
  c->host_a = (p->flags & RPCA_HOST_A) != 0;
  c->simt = (p->flags & RPCA_SIMT) != 0 || c->f64;
  c->centered = (p->flags & RPCA_CENTER) != 0;
  c->m = c->transposed ? p->n : p->m;
  c->n = c->transposed ? p->m : p->n;
  c->k = p->k;
  c->l = p->l;
  c->i = p->i;
  c->w = (p->i + 1) * p->l;
  c->ldx = c->l + 1;
  const size_t es = c->cbytes();
  c->stream = static_cast<cudaStream_t>(p->stream);  // NULL: the legacy default stream
  c->X.alloc((size_t)c->n * c->ldx * es);
  c->F.alloc((size_t)c->n * c->ldx * es);
  c->H.alloc((size_t)c->m * c->w * es);
  c->T.alloc((size_t)c->n * c->w * es);
  c->T64.alloc((size_t)c->n * c->w * sizeof(double));
  c->Tc.alloc((size_t)c->n * c->w * es);
  c->shift.alloc((size_t)c->n * es);
  c->corr.alloc((size_t)256 * es);
  c->d.alloc((size_t)c->n * sizeof(double));
  c->vtmp.alloc(256 * sizeof(double));
  c->q1.alloc(256 * sizeof(double));
  c->err.alloc(64 * sizeof(uint32_t));
  c->outU.alloc((size_t)c->m * c->k * es);
  c->outV.alloc((size_t)c->n * c->k * es);
  const size_t w = c->w, l = c->l;
  const size_t small_doubles = w * l + 4 * l * l + w * w * 4 + w + 5 * w * w + 3 * w * w + 2 * w * c->k;
  const size_t qf_words = (size_t)kQfWords * (c->i + 1);   // the most blocks any QR here has
  c->small.alloc(small_doubles * sizeof(double) + qf_words * sizeof(uint32_t));
  double* s = c->small.as<double>();
  c->qs.C = s; s += w * l;
  c->qs.Gm = s; s += l * l;
  c->qs.Rk = s; s += l * l;
  c->qs.Rinv = s; s += l * l;
  c->qs.Racc = s; s += l * l;
  c->RT = s; s += w * w;
  c->Ub = s; s += w * w;
  c->W = s; s += w * w;
  c->S = s; s += w;
  c->svdwork = s; s += 6 * w * w;
  c->E = s; s += w * w;
  c->ET = s; s += w * w;
  c->RT2 = s; s += w * w;
  c->MU = s; s += w * c->k;
  c->MV = s; s += w * c->k;
  c->qs.qf = reinterpret_cast<uint32_t*>(s);
  RPCA_CUDA_TRY(cudaMemsetAsync(c->qs.qf, 0, qf_words * sizeof(uint32_t), c->stream));
  if (c->transposed) c->At.alloc((size_t)c->m * c->n * dtype_bytes(p->dtype));
  if (!c->simt) c->work.alloc(tc_work_bytes(p->dtype, c->m, c->n, c->w));
  if (!c->f64) {
    c->mt.alloc(2 * 256 * 256 * sizeof(float));
    c->qs.mt = c->mt.as<float>();
    if (!c->simt) {
      c->sliced = sliced_ok(false, c->m, c->i + 1, c->l, c->k);
      if (c->sliced) {
        c->hs_rows = round_up(c->m, 128);
        c->Hs.alloc((size_t)3 * c->hs_rows * (c->i + 1) * 64 * 2);
        c->sq.alloc(kSliceScratchDoubles * sizeof(double));
        c->qs.G64 = c->sq.as<double>();
        c->qs.C64 = c->qs.G64 + 64 * 64;
        c->qs.Cfull = c->qs.C64 + 192 * 64;
      } else {
        c->Hlo.alloc((size_t)c->m * c->w * sizeof(float));
      }
      if (c->n >= kTcMinRows) c->Tlo.alloc((size_t)c->n * c->w * sizeof(float));
      const int64_t srows = c->sliced ? (c->n >= kTcMinRows ? c->n : 0) : std::max(c->m, c->n);
      if (srows > 0) {
        const size_t sb = (size_t)6 * round_up(srows, 32) * (2 * round_up(c->w, 64));
        c->slices.alloc(sb);
        c->qs.slices = c->slices.ptr;
        c->qs.slice_bytes = sb;
      }
    }
  }
  if (c->host_a) {
    const size_t ab = dtype_bytes(p->dtype);
    c->resident = (p->flags & RPCA_HOST_RESIDENT) != 0;
    if (c->resident) c->Ares.alloc((size_t)c->m * c->n * ab);
    int64_t tr = p->tile_rows > 0 ? p->tile_rows : std::max<int64_t>(128, (int64_t)((1ull << 30) / (c->n * ab)));
    tr = std::min<int64_t>(tr, c->m);
    c->tile_rows = tr;
    for (int t = 0; t < 2; ++t) {
      c->tiles[t].alloc((size_t)tr * c->n * ab);
      RPCA_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_copied[t], cudaEventDisableTiming));
      RPCA_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_used[t], cudaEventDisableTiming));
    }
    RPCA_CUDA_TRY(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  }
  // G (n x l, working orientation): caller's, or the Philox stream of `seed`
  std::vector<double> G((size_t)c->n * c->l);
  if (p->G) std::memcpy(G.data(), p->G, G.size() * sizeof(double));
  else gaussian_stream(p->seed, 0u, (int64_t)G.size(), G.data());
  c->adjoint = (p->flags & RPCA_ADJOINT) != 0;
  if (c->adjoint) {
    const int64_t m = c->m, n = c->n;
    const int k = c->k, l = c->l, i = c->i, w = c->w;
    const int r = k + w + i * l;
    c->Xsave.alloc((size_t)(i + 1) * n * l * es);
    c->Bcat.alloc((size_t)m * 2 * w * es);
    c->XM.alloc((size_t)n * 2 * w * es);
    c->Hb.alloc((size_t)m * w * es);
    c->Tm.alloc((size_t)m * l * es);
    c->Xb64.alloc((size_t)n * l * sizeof(double));
    c->Xb.alloc((size_t)n * l * es);
    c->Dn.alloc((size_t)n * l * es);
    c->Fb.alloc((size_t)std::max(1, i) * n * l * es);
    c->Mw.alloc((size_t)n * w * es);
    c->Pf.alloc((size_t)m * r * es);
    c->Zf.alloc((size_t)n * r * es);
    c->bsmall.alloc(((size_t)k * w + 3 * (size_t)w * w + 2 * (size_t)w * w + 3 * (size_t)l * l + 2 * (size_t)l * l) *
                    sizeof(double));
  }
  c->G64.alloc(G.size() * sizeof(double));
  RPCA_CUDA_TRY(cudaMemcpy(c->G64.ptr, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice));
  c->reorth = !c->adjoint;
  c->mirror = c->reorth && c->sliced && !c->simt && (p->dtype == RPCA_F32 || p->dtype == RPCA_FP8E4M3) &&
              !(p->flags & RPCA_KEEP_T_PASS);
  if (c->mirror) c->Fall.alloc((size_t)c->n * c->w * es);
  if (c->reorth) {
    // X^(0) = orth(G), once per context (G is fixed)
    c->Xall.alloc((size_t)c->n * c->w * es);
    copy_matrix(true, c->f64, c->n, c->l, c->G64.ptr, c->l, c->Xall.ptr, c->w, c->stream);
    RPCA_CUDA_TRY(cudaMemsetAsync(c->err.ptr, 0, 64 * sizeof(uint32_t), c->stream));
    block_qr(c->f64, c->n, 1, c->l, c->Xall.ptr, c->w, nullptr, nullptr, c->qs, c->dev_err(), c->stream);
  }
  c->timing = (p->flags & RPCA_TIMING) != 0;
  if (c->timing) {
    const int nph = c->i + 5;
    c->ev.assign(2 * nph, nullptr);
    for (auto& e : c->ev) RPCA_CUDA_TRY(cudaEventCreate(&e));
    c->phase_ms.assign(nph, 0.0);
  }
  c->next_pass = 0;
  return RPCA_OK;
}

// --------------------------------------------------------------- adjoint
// Gradient of L(sigma_1..k) with respect to A, G fixed.  With T = A^T Q =
// V~ S~ W^T and c_j = dL/dsigma_j, dL = <M, dT> for M = V~_k C W_k^T, so
//   A-bar = Q M^T + (terms through Q),  Q-bar = A M.
// L depends on each orthonormalised block only through its span, so for
// any orthonormal X with span(X) = span(F) and R = X^T F the map F -> X
// back-propagates as F-bar = (X-bar - X (X^T X-bar)) R^-T.  Through
// H^(j) = A X^(j) and F^(j) = A^T H^(j):
//   X-bar^(j) = A^T H-bar^(j),  A-bar += H-bar^(j) X^(j)T + H^(j-1) F-bar^(j-1)T,
//   H-bar^(j-1) += A F-bar^(j-1),  R^(j-1) = X^(j)T F^(j-1) = H^(j)T H^(j-1).
// A-bar is the thin product P Z^T with
//   P = [U, H-bar^(0..i), H^(0..i-1)],  Z = [V C, X^(0..i), F-bar^(0..i-1)].
void do_backward_enqueue(rpca_ctx* c, const rpca_matrix* Am, const double* dS, void* dA, int64_t ldda) {
  if (!c->adjoint) throw Invalid("context created without RPCA_ADJOINT");
  if (!c->fwd_done) throw Invalid("backward before a completed run");
  if (!Am || !Am->data || !dS || !dA) throw Invalid("null pointer");
  const bool f64 = c->f64;
  const size_t es = c->cbytes();
  cudaStream_t st = c->stream;
  const int64_t m = c->m, n = c->n;
  const int k = c->k, l = c->l, i = c->i, w = c->w;
  const int r = k + w + i * l;
  if (ldda < n || Am->ld < n) throw Invalid("ld < n");
  auto at = [&](const DevBuf& b, size_t elems) { return static_cast<char*>(b.ptr) + elems * es; };
  PassArgs base;
  base.dtype = c->prob.dtype;
  base.A = Am->data;
  base.lda = Am->ld;
  base.m = m;
  base.n = n;
  base.scale = Am->col_scale;
  // the re-streams of A run on the tensor-core kernels where the storage
  // type and layout allow (BF16, FP32, FP8 converters), else on CUDA cores
  base.work = c->work.ptr;
  base.work_bytes = c->work.bytes;
  auto pass_h = [&](const void* X, int64_t ldx, int p, void* Hout, int64_t ldh) {   // Hout = A X
    PassArgs a = base;
    a.mode = MODE_H;
    a.X = X;
    a.ldx = ldx;
    a.p = p;
    a.H = Hout;
    a.ldh = ldh;
    if (c->simt || p > 64 || !launch_pass_tc(a, st, c->dev_err())) launch_pass_simt(a, st);
  };
  auto pass_t = [&](const void* Y, int64_t ldy, int p, double* Out, int64_t ldo) {   // Out = A^T Y (FP64)
    PassArgs a = base;
    a.mode = MODE_T;
    a.p = p;
    a.H = const_cast<void*>(Y);
    a.ldh = ldy;
    a.F = Out;
    a.ldf = ldo;
    a.f_f64 = true;
    if (c->simt || !launch_pass_tc(a, st, c->dev_err())) launch_pass_simt(a, st);
  };
  double* s = c->bsmall.as<double>();
  double* Mk = s; s += (size_t)k * w;
  double* RH = s; s += (size_t)w * w;
  double* Bw = s; s += (size_t)w * w;
  double* RHit = s; s += (size_t)w * w;
  double* aug = s; s += 2 * (size_t)w * w;
  double* Om = s; s += (size_t)l * l;
  double* Rl = s; s += (size_t)l * l;
  double* Rlit = s; s += (size_t)l * l;
  double* augl = s;
  uint32_t* err = c->dev_err();
  RPCA_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), st));
  // M = V C W_k^T (n x w)
  make_mk(k, w, dS, c->W, Mk, st);
  gemm_xm(f64, n, k, w, c->outV.ptr, k, Mk, w, 1.0, 0.0, c->Mw.ptr, w, st);
  // [H | Q-bar] = A [X^(0..i) | M]  (H recomputed from the saved blocks)
  for (int j = 0; j <= i; ++j)
    copy_matrix(f64, f64, n, l, at(c->Xsave, (size_t)j * n * l), l, at(c->XM, (size_t)j * l), 2 * w, st);
  copy_matrix(f64, f64, n, w, c->Mw.ptr, w, at(c->XM, (size_t)w), 2 * w, st);
  if (2 * w <= 256) {
    pass_h(c->XM.ptr, 2 * w, 2 * w, c->Bcat.ptr, 2 * w);
  } else {
    pass_h(c->XM.ptr, 2 * w, w, c->Bcat.ptr, 2 * w);
    pass_h(at(c->XM, (size_t)w), 2 * w, w, at(c->Bcat, (size_t)w), 2 * w);
  }
  void* Hc = c->Bcat.ptr;
  void* Qb = at(c->Bcat, (size_t)w);
  // H-bar = (Q-bar - Q (Q^T Q-bar)) R_H^-T with R_H = Q^T H
  gram(f64, m, w, w, c->H.ptr, w, Hc, 2 * w, RH, w, false, st);
  gram(f64, m, w, w, c->H.ptr, w, Qb, 2 * w, Bw, w, false, st);
  gemm_xm(f64, m, w, w, c->H.ptr, w, Bw, w, -1.0, 1.0, Qb, 2 * w, st);
  small_inv_t(w, RH, w, aug, RHit, err, st);
  gemm_xm(f64, m, w, w, Qb, 2 * w, RHit, w, 1.0, 0.0, c->Hb.ptr, w, st);
  for (int j = i; j >= 1; --j) {
    // X-bar^(j) = A^T H-bar^(j)
    pass_t(at(c->Hb, (size_t)j * l), w, l, c->Xb64.as<double>(), l);
    copy_matrix(true, f64, n, l, c->Xb64.ptr, l, c->Xb.ptr, l, st);
    const void* Xj = at(c->Xsave, (size_t)j * n * l);
    // F-bar^(j-1) = (X-bar - X (X^T X-bar)) R^-T,  R = H^(j)T H^(j-1)
    gram(f64, n, l, l, Xj, l, c->Xb.ptr, l, Om, l, false, st);
    copy_matrix(f64, f64, n, l, c->Xb.ptr, l, c->Dn.ptr, l, st);
    gemm_xm(f64, n, l, l, Xj, l, Om, l, -1.0, 1.0, c->Dn.ptr, l, st);
    gram(f64, m, l, l, at(c->Bcat, (size_t)j * l), 2 * w, at(c->Bcat, (size_t)(j - 1) * l), 2 * w, Rl, l, false, st);
    small_inv_t(l, Rl, l, augl, Rlit, err, st);
    void* Fbj = at(c->Fb, (size_t)(j - 1) * n * l);
    gemm_xm(f64, n, l, l, c->Dn.ptr, l, Rlit, l, 1.0, 0.0, Fbj, l, st);
    // H-bar^(j-1) += A F-bar^(j-1)
    pass_h(Fbj, l, l, c->Tm.ptr, l);
    add_matrix(f64, m, l, c->Tm.ptr, l, at(c->Hb, (size_t)(j - 1) * l), w, st);
  }
  // P = [U, H-bar, H^(0..i-1)],  Z = [V C, X^(0..i), F-bar^(0..i-1)]
  copy_matrix(f64, f64, m, k, c->outU.ptr, k, c->Pf.ptr, r, st);
  scale_cols(f64, n, k, c->outV.ptr, k, dS, c->Zf.ptr, r, st);
  copy_matrix(f64, f64, m, w, c->Hb.ptr, w, at(c->Pf, (size_t)k), r, st);
  for (int j = 0; j <= i; ++j)
    copy_matrix(f64, f64, n, l, at(c->Xsave, (size_t)j * n * l), l, at(c->Zf, (size_t)(k + j * l)), r, st);
  for (int j = 1; j <= i; ++j) {
    copy_matrix(f64, f64, m, l, at(c->Bcat, (size_t)(j - 1) * l), 2 * w, at(c->Pf, (size_t)(k + w + (j - 1) * l)), r,
                st);
    copy_matrix(f64, f64, n, l, at(c->Fb, (size_t)(j - 1) * n * l), l, at(c->Zf, (size_t)(k + w + (j - 1) * l)), r, st);
  }
  lowrank_out(f64, m, n, r, c->Pf.ptr, r, c->Zf.ptr, r, dA, ldda, st);
}

rpca_status do_backward(rpca_ctx* c, const rpca_matrix* Am, const double* dS, void* dA, int64_t ldda) {
  do_backward_enqueue(c, Am, dS, dA, ldda);
  uint32_t flags = 0;
  RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, c->dev_err(), sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  RPCA_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (flags & DEV_ERR_BREAKDOWN) return fail(c, RPCA_EBREAKDOWN, "a small factor of the adjoint is singular");
  if (flags & DEV_ERR_TIMEOUT) return fail(c, RPCA_ETIMEOUT, "a device-side wait timed out");
  return RPCA_OK;
}

// --------------------------------------------------------------- batches
// Many independent problems: one context each, spread over a pool of
// streams forked from and joined to the caller's stream.  The first run is
// executed directly (every lazy set-up happens outside a capture) and then
// recorded once as a CUDA graph; later runs with the same buffers replay
// that graph with one launch.
__global__ void k_gather_flags(const uint32_t* const* __restrict__ src, int count, uint32_t* __restrict__ dst) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) dst[p] = *src[p];
}

}  // namespace

struct rpca_batch {
  std::vector<rpca_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr, ev_in = nullptr, ev_out = nullptr;
  cudaStream_t caller = nullptr;         // problems[0].stream (may be the legacy stream)
  cudaStream_t origin = nullptr;         // the batch's own stream: captured, ordered after caller
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;          // buffers the graph was recorded with
  uint64_t graph_kernels = 0;            // kernels in the recorded graph
  rpca::DevBuf err_ptrs, flags;          // device array of the contexts' error words, gathered words
  std::vector<uint32_t> host_flags;
  int bad = -1;                          // index of the last failing problem
  std::string last_error;
  // grouped kernels over all problems (BF16 batches that fit them); the
  // per-problem contexts are then made only if a run's layout needs them
  rpca::grp::GroupedBatch* grp = nullptr;
  bool last_grouped = false;
  std::vector<rpca_problem> problems;
  int nstreams = 1;
  ~rpca_batch() {
    if (grp) rpca::grp::grouped_destroy(grp);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto* c : ctx) rpca_destroy(c);
    for (auto e : ev_join) if (e) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    for (auto s : streams) if (s) cudaStreamDestroy(s);
    if (origin) cudaStreamDestroy(origin);
  }
};

namespace {

void batch_enqueue(rpca_batch* b, const rpca_matrix* A, void* const* U, const int64_t* ldu, double* const* S,
                   void* const* V, const int64_t* ldv) {
  RPCA_CUDA_TRY(cudaEventRecord(b->ev_fork, b->origin));
  for (auto st : b->streams) RPCA_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_fork, 0));
  for (size_t p = 0; p < b->ctx.size(); ++p) {
    rpca_ctx* c = b->ctx[p];
    c->next_pass = 0;
    while (do_pass(c, &A[p]) == RPCA_MORE) {
    }
    do_finish_enqueue(c, U ? U[p] : nullptr, ldu ? ldu[p] : 0, S ? S[p] : nullptr, V ? V[p] : nullptr,
                      ldv ? ldv[p] : 0);
  }
  for (size_t s = 0; s < b->streams.size(); ++s) {
    RPCA_CUDA_TRY(cudaEventRecord(b->ev_join[s], b->streams[s]));
    RPCA_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_join[s], 0));
  }
  const int count = (int)b->ctx.size();
  k_gather_flags<<<(unsigned)cdiv(count, 256), 256, 0, b->origin>>>(b->err_ptrs.as<const uint32_t*>(), count,
                                                                    b->flags.as<uint32_t>());
  RPCA_CUDA_TRY(cudaGetLastError());
  count_launch();
}

// One context per problem over the batch's stream pool (the per-problem
// form; also made lazily for a grouped batch whose run needs it).
rpca_status batch_make_contexts(rpca_batch* b) {
  const int32_t count = (int32_t)b->problems.size();
  const int ns = std::min<int32_t>(b->nstreams, count);
  b->streams.assign(ns, nullptr);
  b->ev_join.assign(ns, nullptr);
  for (int i = 0; i < ns; ++i) {
    RPCA_CUDA_TRY(cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking));
    RPCA_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming));
  }
  RPCA_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  std::vector<const uint32_t*> ptrs(count);
  for (int32_t p = 0; p < count; ++p) {
    rpca_problem q = b->problems[p];
    q.stream = b->streams[p % ns];
    rpca_ctx* c = new rpca_ctx();
    b->ctx.push_back(c);
    rpca_status si = guarded(c, [&] { return do_init(c, &q); });
    if (si != RPCA_OK) {
      b->last_error = "problem " + std::to_string(p) + ": " + c->last_error;
      return si;
    }
    ptrs[p] = c->err.as<uint32_t>();
  }
  b->err_ptrs.alloc(count * sizeof(uint32_t*));
  b->flags.alloc(count * sizeof(uint32_t));
  b->host_flags.assign(count, 0u);
  RPCA_CUDA_TRY(cudaMemcpy(b->err_ptrs.ptr, ptrs.data(), count * sizeof(uint32_t*), cudaMemcpyHostToDevice));
  return RPCA_OK;
}

// A grouped run: after the caller's queued work; the caller's stream waits
// for it.  False when the layout of A needs the per-problem form.
bool batch_grouped_run(rpca_batch* b, const rpca_matrix* A, void* const* U, const int64_t* ldu, double* const* S,
                       void* const* V, const int64_t* ldv, rpca_status* st) {
  RPCA_CUDA_TRY(cudaEventRecord(b->ev_in, b->caller));
  RPCA_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
  if (!rpca::grp::grouped_run(b->grp, A, U, ldu, S, V, ldv, b->origin)) return false;
  RPCA_CUDA_TRY(cudaEventRecord(b->ev_out, b->origin));
  RPCA_CUDA_TRY(cudaStreamWaitEvent(b->caller, b->ev_out, 0));
  *st = rpca::grp::grouped_check(b->grp, b->origin, &b->bad, &b->last_error);
  return true;
}

// ----------------------------------------------------------- autotuner
// Cache file: {"rpca_batch_tuning": {"<key>": [h, t, trows, rrows, pf], ...}}
std::string tune_key(const rpca_batch* b) {
  int64_t maxn = 0;
  double meanm = 0.0;
  for (const auto& q : b->problems) {
    maxn = std::max<int64_t>(maxn, q.n);
    meanm += (double)q.m;
  }
  meanm /= (double)b->problems.size();
  auto bucket = [](double v) {
    int64_t e = 1;
    while ((double)e < v) e <<= 1;
    return e;
  };
  const rpca_problem& q = b->problems[0];
  return "bf16/n" + std::to_string(bucket((double)maxn)) + "/m" + std::to_string(bucket(meanm)) + "/k" +
         std::to_string(q.k) + "/l" + std::to_string(q.l) + "/i" + std::to_string(q.i);
}

std::vector<std::pair<std::string, std::vector<int>>> read_tune_cache(const char* path) {
  std::vector<std::pair<std::string, std::vector<int>>> out;
  if (!path) return out;
  FILE* f = std::fopen(path, "rb");
  if (!f) return out;
  std::string t;
  char buf[4096];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof buf, f)) > 0) t.append(buf, r);
  std::fclose(f);
  const size_t top = t.find("\"rpca_batch_tuning\"");
  if (top == std::string::npos) return out;
  size_t pos = t.find('{', top);
  while (pos != std::string::npos) {
    const size_t k0 = t.find('"', pos + 1);
    if (k0 == std::string::npos) break;
    const size_t k1 = t.find('"', k0 + 1);
    const size_t a0 = t.find('[', k1);
    const size_t a1 = t.find(']', a0);
    if (k1 == std::string::npos || a0 == std::string::npos || a1 == std::string::npos) break;
    std::vector<int> v;
    const char* c = t.c_str() + a0 + 1;
    while (c < t.c_str() + a1) {
      char* e = nullptr;
      const long x = std::strtol(c, &e, 10);
      if (e == c) {
        ++c;
        continue;
      }
      v.push_back((int)x);
      c = e;
    }
    if (v.size() == 5) out.emplace_back(t.substr(k0 + 1, k1 - k0 - 1), v);
    pos = t.find(',', a1);
    if (pos == std::string::npos || t.find('"', pos) == std::string::npos) break;
  }
  return out;
}

void write_tune_cache(const char* path, const std::vector<std::pair<std::string, std::vector<int>>>& e) {
  if (!path) return;
  FILE* f = std::fopen(path, "wb");
  if (!f) throw Invalid(std::string("cannot write the tuning cache ") + path);
  std::fprintf(f, "{\"rpca_batch_tuning\": {");
  for (size_t i = 0; i < e.size(); ++i)
    std::fprintf(f, "%s\n  \"%s\": [%d, %d, %d, %d, %d]", i ? "," : "", e[i].first.c_str(), e[i].second[0],
                 e[i].second[1], e[i].second[2], e[i].second[3], e[i].second[4]);
  std::fprintf(f, "\n}}\n");
  std::fclose(f);
}

rpca_status batch_tune(rpca_batch* b, const rpca_matrix* A, void* const* U, const int64_t* ldu, double* const* S,
                       void* const* V, const int64_t* ldv, const char* path) {
  const std::string key = tune_key(b);
  auto cache = read_tune_cache(path);
  for (const auto& e : cache)
    if (e.first == key) {
      rpca::grp::Tuning v{e.second[0], e.second[1], e.second[2], e.second[3], e.second[4]};
      rpca::grp::grouped_set_tuning(b->grp, v);
      rpca_status st = RPCA_OK;
      if (!batch_grouped_run(b, A, U, ldu, S, V, ldv, &st)) throw Invalid("the matrices' layout needs the per-problem form");
      return st;
    }
  cudaEvent_t e0, e1;
  RPCA_CUDA_TRY(cudaEventCreate(&e0));
  RPCA_CUDA_TRY(cudaEventCreate(&e1));
  auto time_one = [&](const rpca::grp::Tuning& v, float* ms) -> rpca_status {
    rpca::grp::grouped_set_tuning(b->grp, v);
    rpca_status st = RPCA_OK;
    if (!batch_grouped_run(b, A, U, ldu, S, V, ldv, &st)) throw Invalid("the matrices' layout needs the per-problem form");
    if (st != RPCA_OK) return st;
    RPCA_CUDA_TRY(cudaEventRecord(e0, b->origin));
    if (!rpca::grp::grouped_run(b->grp, A, U, ldu, S, V, ldv, b->origin)) throw Invalid("layout");
    RPCA_CUDA_TRY(cudaEventRecord(e1, b->origin));
    st = rpca::grp::grouped_check(b->grp, b->origin, &b->bad, &b->last_error);
    RPCA_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return st;
  };
  rpca::grp::Tuning best = rpca::grp::grouped_tuning(b->grp);
  float best_ms = 0.f;
  rpca_status st = time_one(best, &best_ms);
  const int cand[5][3] = {{2, 3, 4}, {3, 4, 5}, {2048, 4096, 8192}, {1024, 2048, 4096}, {0, 8, 16}};
  for (int d = 0; d < 5 && st == RPCA_OK; ++d)
    for (int c = 0; c < 3 && st == RPCA_OK; ++c) {
      rpca::grp::Tuning v = best;
      int* f[5] = {&v.h_stages, &v.t_stages, &v.t_rows, &v.r_rows, &v.pf};
      if (*f[d] == cand[d][c]) continue;
      *f[d] = cand[d][c];
      float ms = 0.f;
      st = time_one(v, &ms);
      if (st == RPCA_OK && ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RPCA_OK) return st;
  rpca::grp::grouped_set_tuning(b->grp, best);
  st = RPCA_OK;
  batch_grouped_run(b, A, U, ldu, S, V, ldv, &st);
  if (st == RPCA_OK && path) {
    cache.emplace_back(key, std::vector<int>{best.h_stages, best.t_stages, best.t_rows, best.r_rows, best.pf});
    write_tune_cache(path, cache);
  }
  return st;
}

rpca_status batch_check(rpca_batch* b) {
  const int count = (int)b->ctx.size();
  RPCA_CUDA_TRY(cudaMemcpyAsync(b->host_flags.data(), b->flags.ptr, count * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, b->origin));
  RPCA_CUDA_TRY(cudaEventRecord(b->ev_out, b->origin));
  RPCA_CUDA_TRY(cudaStreamWaitEvent(b->caller, b->ev_out, 0));
  RPCA_CUDA_TRY(cudaStreamSynchronize(b->origin));
  for (int p = 0; p < count; ++p) {
    const uint32_t f = b->host_flags[p];
    if (f & (DEV_ERR_TIMEOUT | DEV_ERR_BREAKDOWN)) {
      b->bad = p;
      b->last_error = "problem " + std::to_string(p) +
                      ((f & DEV_ERR_TIMEOUT) ? ": a device-side wait timed out" : ": Cholesky QR broke down");
      return (f & DEV_ERR_TIMEOUT) ? RPCA_ETIMEOUT : RPCA_EBREAKDOWN;
    }
  }
  return RPCA_OK;
}

template <typename Fn>
rpca_status bguarded(rpca_batch* b, Fn&& fn) {
  try {
    return fn();
  } catch (const CudaFailure& e) {
    if (b) b->last_error = e.what;
    if (e.code == cudaErrorMemoryAllocation) return RPCA_ENOMEM;
    if (e.code == cudaErrorNoDevice || e.code == cudaErrorInsufficientDriver) return RPCA_ENODEV;
    return RPCA_ECUDA;
  } catch (const Invalid& e) {
    if (b) b->last_error = e.what;
    return RPCA_EINVAL;
  } catch (const std::bad_alloc&) {
    if (b) b->last_error = "host allocation failed";
    return RPCA_ENOMEM;
  }
}

// Single-op entries: wait for the stream and turn the kernel's error word
// into a status.
rpca_status read_op_error(const DevBuf& err, cudaStream_t st) {
  uint32_t flags = 0;
  RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, err.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RPCA_CUDA_TRY(cudaStreamSynchronize(st));
  if (flags & DEV_ERR_TIMEOUT) return RPCA_ETIMEOUT;
  return RPCA_OK;
}

// ------------------------------------------------- error estimate (Appendix)
// p_{j,q}(D) for D = A - U diag(S) V^T: j steps of the power method on D^T D
// from q start vectors, each step D then D^T applied to the block (an H
// pass and a T pass over A, with the rank-kd corrections), the columns
// renormalised after every step; p = max_c sqrt(||D^T D w_c||) with w_c the
// unit column after j - 1 steps.
rpca_status do_estimate(const rpca_problem* p, const rpca_matrix* Am, const void* U, int64_t ldu, const double* S,
                        const void* V, int64_t ldv, int kd, int j, int q, const double* omega, double* est,
                        double* col_est) {
  check_device();
  if (!p || !Am || !Am->data || !U || !S || !V || !est) throw Invalid("null pointer");
  if (p->m < 1 || p->n < 1 || kd < 1 || kd > 255 || kd > std::min(p->m, p->n) || j < 1 || j > 64 || q < 1 ||
      q > 255 || q > p->n)
    throw Invalid("bad sizes");
  if (p->flags & (RPCA_CENTER | RPCA_HOST_A)) throw Invalid("the estimate takes an uncentred device matrix");
  if (Am->ld < p->n || ldu < kd || ldv < kd) throw Invalid("bad leading dimension");
  if (p->dtype < RPCA_F64 || p->dtype > RPCA_FP8E4M3) throw Invalid("unknown dtype");
  const bool f64 = p->dtype == RPCA_F64;
  const size_t es = f64 ? 8 : 4;
  const int64_t m = p->m, n = p->n;
  cudaStream_t st = static_cast<cudaStream_t>(p->stream);
  DevBuf W, H, F, VS, small, err, work;
  W.alloc((size_t)n * q * es);
  H.alloc((size_t)m * q * es);
  F.alloc((size_t)n * q * es);
  VS.alloc((size_t)n * kd * es);
  const size_t kq = (size_t)kd * q, kk = (size_t)kd * kd;
  small.alloc((3 * kq + 3 * kk + (size_t)q * q + (size_t)q * q) * sizeof(double));
  double* B = small.as<double>();
  double* C = B + kq;
  double* DS = C + kq + 2 * kk;
  double* Gq = DS + kk;
  double* Dn = Gq + (size_t)q * q;
  DevBuf sb;
  sb.alloc(kq * sizeof(double));
  auto DSB = [&](const double* Bm) {   // diag(S) Bm (kd x q), FP64
    gemm64_small(kd, q, kd, 1.0, DS, kd, false, Bm, q, false, 0.0, nullptr, 0, sb.as<double>(), q, st);
    return sb.as<double>();
  };
  err.alloc(64 * sizeof(uint32_t));
  RPCA_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, 64 * sizeof(uint32_t), st));
  if (!f64) {
    work.alloc(tc_work_bytes(p->dtype, m, n, std::max(q, kd)));
  }
  auto pass = [&](int mode, const void* X, int64_t ldx, int cols, void* Hout, int64_t ldh, void* Fout, int64_t ldf) {
    PassArgs a;
    a.dtype = p->dtype;
    a.mode = mode;
    a.A = Am->data; a.lda = Am->ld; a.m = m; a.n = n; a.scale = Am->col_scale;
    a.X = X; a.ldx = ldx; a.p = cols; a.H = Hout; a.ldh = ldh; a.F = Fout; a.ldf = ldf;
    a.work = work.ptr; a.work_bytes = work.bytes;
    if (f64 || !launch_pass_tc(a, st, err.as<uint32_t>())) launch_pass_simt(a, st);
  };
  // start vectors (n x q, row-major): given, or the Philox stream of the
  // problem's seed, domain 1 (G uses domain 0)
  std::vector<double> om((size_t)n * q);
  if (omega) std::memcpy(om.data(), omega, om.size() * sizeof(double));
  else gaussian_stream(p->seed, 1u, (int64_t)om.size(), om.data());
  {
    DevBuf om64;
    om64.alloc(om.size() * sizeof(double));
    RPCA_CUDA_TRY(cudaMemcpyAsync(om64.ptr, om.data(), om.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    cast_f64_to(f64, (int64_t)om.size(), om64.as<double>(), W.ptr, st);
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
  }
  // the iteration's constant terms: diag(S), VS = V S
  std::vector<double> ds(kk, 0.0), sv(kd);
  RPCA_CUDA_TRY(cudaMemcpyAsync(sv.data(), S, kd * sizeof(double), cudaMemcpyDefault, st));
  RPCA_CUDA_TRY(cudaStreamSynchronize(st));
  for (int c = 0; c < kd; ++c) ds[(size_t)c * kd + c] = sv[c];
  RPCA_CUDA_TRY(cudaMemcpyAsync(DS, ds.data(), kk * sizeof(double), cudaMemcpyHostToDevice, st));
  gemm_xm(f64, n, kd, kd, V, ldv, DS, kd, 1.0, 0.0, VS.ptr, kd, st);
  std::vector<double> gq((size_t)q * q), dn((size_t)q * q, 0.0);
  std::vector<double> ratio(q, 0.0);
  for (int step = 0; step < j; ++step) {
    // Y = D W = A W - U S (V^T W), then D^T Y = A^T Y - V S (U^T Y): D and
    // D^T applied in turn (forming A^T A W first would subtract quantities
    // of size ||A||^2 to get ||D||^2, and lose it in FP32 when ||D|| is
    // below sqrt(u32) ||A||)
    pass(MODE_H, W.ptr, q, q, H.ptr, q, nullptr, 0);                   // H = A W
    gram(f64, n, kd, q, V, ldv, W.ptr, q, B, q, false, st);            // B = V^T W
    gemm_xm(f64, m, kd, q, U, ldu, DSB(B), q, -1.0, 1.0, H.ptr, q, st); // H -= U S B
    pass(MODE_T, nullptr, 0, q, H.ptr, q, F.ptr, q);                   // F = A^T H
    gram(f64, m, kd, q, U, ldu, H.ptr, q, C, q, false, st);            // C = U^T H
    gemm_xm(f64, n, kd, q, VS.ptr, kd, C, q, -1.0, 1.0, F.ptr, q, st);  // F -= V S C
    gram(f64, n, q, q, F.ptr, q, F.ptr, q, Gq, q, false, st);
    RPCA_CUDA_TRY(cudaMemcpyAsync(gq.data(), Gq, gq.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
    for (int c = 0; c < q; ++c) ratio[c] = std::sqrt(std::max(gq[(size_t)c * q + c], 0.0));   // ||D^T D w_c||
    if (step + 1 < j) {
      for (int c = 0; c < q; ++c) dn[(size_t)c * q + c] = ratio[c] > 0.0 ? 1.0 / ratio[c] : 0.0;
      RPCA_CUDA_TRY(cudaMemcpyAsync(Dn, dn.data(), dn.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      gemm_xm(f64, n, q, q, F.ptr, q, Dn, q, 1.0, 0.0, W.ptr, q, st);                 // W = F / ||F||
    }
  }
  double best = 0.0;
  for (int c = 0; c < q; ++c) {
    const double pc = std::sqrt(ratio[c]);
    if (col_est) col_est[c] = pc;
    best = std::max(best, pc);
  }
  *est = best;
  return read_op_error(err, st);
}

}  // namespace

// ================================================================== C-ABI
extern "C" {

rpca_status rpca_test_arm_wait_expiry(int32_t kernel, uint64_t limit_ns, int64_t withhold_stage) {
  if (kernel < 0 || kernel > 1 || limit_ns < 100000ull || limit_ns > 2000000000ull || withhold_stage < -1)
    return RPCA_EINVAL;
  std::lock_guard<std::mutex> lock(g_wait_test_mu);
  g_wait_test[kernel] = {limit_ns, withhold_stage};
  return RPCA_OK;
}

rpca_status rpca_init(rpca_ctx** out, const rpca_problem* p) {
  if (!out) return RPCA_EINVAL;
  *out = nullptr;
  rpca_ctx* c = new (std::nothrow) rpca_ctx();
  if (!c) return RPCA_ENOMEM;
  rpca_status s = guarded(c, [&] { return do_init(c, p); });
  if (s != RPCA_OK) {
    delete c;
    return s;
  }
  *out = c;
  return RPCA_OK;
}

rpca_status rpca_pass(rpca_ctx* c, const rpca_matrix* A) {
  if (!c) return RPCA_EINVAL;
  return guarded(c, [&] { return do_pass(c, A); });
}

rpca_status rpca_finish(rpca_ctx* c, void* U, int64_t ldu, double* S, void* V, int64_t ldv) {
  if (!c) return RPCA_EINVAL;
  return guarded(c, [&] {
    if (c->next_pass != c->i + 2) return fail(c, RPCA_ESTATE, "finish before all passes");
    return do_finish(c, U, ldu, S, V, ldv);
  });
}

void rpca_destroy(rpca_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  delete c;
}

rpca_status rpca_rerun(rpca_ctx* c, const rpca_matrix* A, void* U, int64_t ldu, double* S, void* V,
                       int64_t ldv) {
  if (!c) return RPCA_EINVAL;
  c->next_pass = 0;
  for (;;) {
    rpca_status s = rpca_pass(c, A);
    if (s == RPCA_OK) break;
    if (s != RPCA_MORE) return s;
  }
  return rpca_finish(c, U, ldu, S, V, ldv);
}

rpca_status rpca_run(const rpca_problem* p, const rpca_matrix* A, void* U, int64_t ldu, double* S,
                     void* V, int64_t ldv) {
  rpca_ctx* c = nullptr;
  rpca_status s = rpca_init(&c, p);
  if (s != RPCA_OK) return s;
  s = rpca_rerun(c, A, U, ldu, S, V, ldv);
  rpca_destroy(c);
  return s;
}

rpca_status rpca_backward(rpca_ctx* c, const rpca_matrix* A, const double* dS, void* dA, int64_t ldda) {
  if (!c) return RPCA_EINVAL;
  return guarded(c, [&] { return do_backward(c, A, dS, dA, ldda); });
}

rpca_status rpca_batch_init(rpca_batch** out, int32_t count, const rpca_problem* problems, int32_t nstreams) {
  if (!out) return RPCA_EINVAL;
  *out = nullptr;
  if (count < 1 || !problems || nstreams < 1) return RPCA_EINVAL;
  rpca_batch* b = new (std::nothrow) rpca_batch();
  if (!b) return RPCA_ENOMEM;
  rpca_status s = bguarded(b, [&] {
    check_device();
    for (int32_t p = 0; p < count; ++p) {
      if (problems[p].flags & RPCA_HOST_A) throw Invalid("batched problems take device matrices");
      if (problems[p].flags & RPCA_TIMING) throw Invalid("batched problems are not timed per phase");
      try {
        validate(&problems[p]);
      } catch (const Invalid& e) {
        throw Invalid("problem " + std::to_string(p) + ": " + e.what);
      }
    }
    b->caller = static_cast<cudaStream_t>(problems[0].stream);
    b->problems.assign(problems, problems + count);
    b->nstreams = nstreams;
    RPCA_CUDA_TRY(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    RPCA_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    RPCA_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    if (rpca::grp::grouped_eligible(count, problems, nullptr)) {
      std::vector<std::vector<double>> G(count);
      for (int32_t p = 0; p < count; ++p) {
        G[p].resize((size_t)problems[p].n * problems[p].l);
        if (problems[p].G) std::memcpy(G[p].data(), problems[p].G, G[p].size() * sizeof(double));
        else gaussian_stream(problems[p].seed, 0u, (int64_t)G[p].size(), G[p].data());
      }
      b->grp = rpca::grp::grouped_create(count, problems, G, b->origin);
      b->last_grouped = true;
      return RPCA_OK;
    }
    return batch_make_contexts(b);
  });
  if (s != RPCA_OK) {
    last_batch_error() = b->last_error;
    delete b;
    return s;
  }
  *out = b;
  return RPCA_OK;
}

rpca_status rpca_batch_run(rpca_batch* b, const rpca_matrix* A, void* const* U, const int64_t* ldu,
                           double* const* S, void* const* V, const int64_t* ldv) {
  if (!b || !A) return RPCA_EINVAL;
  return bguarded(b, [&] {
    if (b->grp) {
      rpca_status gs = RPCA_OK;
      if (batch_grouped_run(b, A, U, ldu, S, V, ldv, &gs)) {
        b->last_grouped = true;
        return gs;
      }
      if (b->ctx.empty()) {
        rpca_status cs = batch_make_contexts(b);
        if (cs != RPCA_OK) return cs;
      }
    }
    b->last_grouped = false;
    const size_t count = b->ctx.size();
    std::vector<const void*> key;
    key.reserve(6 * count);
    for (size_t p = 0; p < count; ++p) {
      key.push_back(A[p].data);
      key.push_back(reinterpret_cast<const void*>(A[p].ld));
      key.push_back(A[p].col_scale);
      key.push_back(U ? U[p] : nullptr);
      key.push_back(S ? S[p] : nullptr);
      key.push_back(V ? V[p] : nullptr);
    }
    // the batch runs after the caller's queued work
    RPCA_CUDA_TRY(cudaEventRecord(b->ev_in, b->caller));
    RPCA_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
    if (b->exec && key == b->key) {
      RPCA_CUDA_TRY(cudaGraphLaunch(b->exec, b->origin));
      count_launch(b->graph_kernels);
      return batch_check(b);
    }
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
    }
    // direct run (lazy set-up happens here), then record the graph
    batch_enqueue(b, A, U, ldu, S, V, ldv);
    rpca_status s = batch_check(b);
    if (s != RPCA_OK) return s;
    const uint64_t launches_before = g_launches.load();
    RPCA_CUDA_TRY(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    try {
      batch_enqueue(b, A, U, ldu, S, V, ldv);
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(b->origin, &g);
      if (g) cudaGraphDestroy(g);
      g_launches.store(launches_before);
      throw;
    }
    b->graph_kernels = g_launches.load() - launches_before;
    g_launches.store(launches_before);     // recorded, not launched
    RPCA_CUDA_TRY(cudaStreamEndCapture(b->origin, &b->graph));
    RPCA_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->key = key;
    return RPCA_OK;
  });
}

rpca_status rpca_batch_backward(rpca_batch* b, const rpca_matrix* A, const double* const* dS, void* const* dA,
                                const int64_t* ldda) {
  if (!b || !A || !dS || !dA || !ldda) return RPCA_EINVAL;
  return bguarded(b, [&] {
    if (b->ctx.empty()) throw Invalid("the batch's problems were created without RPCA_ADJOINT");
    const size_t count = b->ctx.size();
    for (size_t p = 0; p < count; ++p)
      if (!b->ctx[p]->adjoint) throw Invalid("problem " + std::to_string(p) + " was created without RPCA_ADJOINT");
    // the problems' backward passes run on the batch's streams, after the
    // caller's queued work, and the caller's stream waits for all of them
    RPCA_CUDA_TRY(cudaEventRecord(b->ev_in, b->caller));
    RPCA_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
    RPCA_CUDA_TRY(cudaEventRecord(b->ev_fork, b->origin));
    for (auto st : b->streams) RPCA_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_fork, 0));
    for (size_t p = 0; p < count; ++p) do_backward_enqueue(b->ctx[p], &A[p], dS[p], dA[p], ldda[p]);
    for (size_t s = 0; s < b->streams.size(); ++s) {
      RPCA_CUDA_TRY(cudaEventRecord(b->ev_join[s], b->streams[s]));
      RPCA_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_join[s], 0));
    }
    const int cnt = (int)count;
    k_gather_flags<<<(unsigned)cdiv(cnt, 256), 256, 0, b->origin>>>(b->err_ptrs.as<const uint32_t*>(), cnt,
                                                                  b->flags.as<uint32_t>());
    RPCA_CUDA_TRY(cudaGetLastError());
    count_launch();
    return batch_check(b);
  });
}

void rpca_batch_destroy(rpca_batch* b) {
  if (!b) return;
  if (b->origin) cudaStreamSynchronize(b->origin);
  for (auto st : b->streams) cudaStreamSynchronize(st);
  delete b;
}

const char* rpca_batch_last_error(const rpca_batch* b) {
  return b ? b->last_error.c_str() : last_batch_error().c_str();
}

int32_t rpca_batch_grouped(const rpca_batch* b) { return (b && b->grp && b->last_grouped) ? 1 : 0; }

rpca_status rpca_estimate_error(const rpca_problem* p, const rpca_matrix* A, const void* U, int64_t ldu,
                                const double* S, const void* V, int64_t ldv, int32_t kd, int32_t j, int32_t q,
                                const double* omega, double* est, double* col_est) {
  return guarded(nullptr, [&] { return do_estimate(p, A, U, ldu, S, V, ldv, kd, j, q, omega, est, col_est); });
}

rpca_status rpca_run_adaptive(const rpca_problem* p, const rpca_matrix* A, double tol, int32_t kmax, int32_t j,
                              void* U, int64_t ldu, double* S, void* V, int64_t ldv, int32_t* k_out,
                              double* eps_out) {
  if (!p || !A || !U || !S || !V || !k_out || !eps_out || !(tol > 0.0) || j < 1) return RPCA_EINVAL;
  if (kmax < p->k || ldu < kmax || ldv < kmax) return RPCA_EINVAL;
  // the estimate takes an uncentred device matrix: refuse before any run
  if (p->flags & (RPCA_CENTER | RPCA_HOST_A)) return RPCA_EINVAL;
  const int over = p->l - p->k;
  if (over < 0) return RPCA_EINVAL;
  const int64_t mn = std::min(p->m, p->n);
  int k = p->k;
  for (;;) {
    rpca_problem q = *p;
    q.k = k;
    q.l = k + over;
    if ((int64_t)(q.i + 1) * q.l > mn || q.l > 255 || (int64_t)(q.i + 1) * q.l > 256) return RPCA_EINVAL;
    rpca_status s = rpca_run(&q, A, U, ldu, S, V, ldv);
    if (s != RPCA_OK) return s;
    double eps = 0.0;
    s = rpca_estimate_error(&q, A, U, ldu, S, V, ldv, k, j, k, nullptr, &eps, nullptr);
    if (s != RPCA_OK) return s;
    *k_out = k;
    *eps_out = eps;
    if (eps <= tol || k >= kmax) return RPCA_OK;
    // the next rank: doubled, within kmax and the method's limits
    int next = std::min<int>(2 * k, kmax);
    while (next > k && ((int64_t)(q.i + 1) * (next + over) > std::min<int64_t>(mn, 256) || next >= mn)) --next;
    if (next <= k) return RPCA_OK;
    k = next;
  }
}

rpca_status rpca_batch_get_tuning(const rpca_batch* b, int32_t* t) {
  if (!b || !b->grp || !t) return RPCA_EINVAL;
  const rpca::grp::Tuning v = rpca::grp::grouped_tuning(b->grp);
  t[0] = v.h_stages;
  t[1] = v.t_stages;
  t[2] = v.t_rows;
  t[3] = v.r_rows;
  t[4] = v.pf;
  return RPCA_OK;
}

rpca_status rpca_batch_set_tuning(rpca_batch* b, const int32_t* t) {
  if (!b || !b->grp || !t) return RPCA_EINVAL;
  return bguarded(b, [&] {
    rpca::grp::Tuning v;
    v.h_stages = t[0];
    v.t_stages = t[1];
    v.t_rows = t[2];
    v.r_rows = t[3];
    v.pf = t[4];
    rpca::grp::grouped_set_tuning(b->grp, v);
    return RPCA_OK;
  });
}

rpca_status rpca_batch_tune(rpca_batch* b, const rpca_matrix* A, void* const* U, const int64_t* ldu,
                            double* const* S, void* const* V, const int64_t* ldv, const char* cache_path,
                            int32_t* chosen) {
  if (!b || !b->grp || !A) return RPCA_EINVAL;
  return bguarded(b, [&] {
    rpca_status st = batch_tune(b, A, U, ldu, S, V, ldv, cache_path);
    if (st == RPCA_OK && chosen) rpca_batch_get_tuning(b, chosen);
    return st;
  });
}

const char* rpca_strerror(rpca_status s) {
  switch (s) {
    case RPCA_OK: return "ok";
    case RPCA_MORE: return "more passes remain";
    case RPCA_EINVAL: return "invalid argument";
    case RPCA_ENOMEM: return "out of memory";
    case RPCA_ECUDA: return "CUDA error";
    case RPCA_ENODEV: return "no CUDA device";
    case RPCA_EBREAKDOWN: return "QR breakdown";
    case RPCA_ETIMEOUT: return "device wait timed out";
    case RPCA_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* rpca_last_error(const rpca_ctx* c) { return c ? c->last_error.c_str() : ""; }

rpca_status rpca_gaussian(uint64_t seed, uint32_t domain, int64_t count, double* out) {
  if (count < 0 || (count > 0 && !out)) return RPCA_EINVAL;
  gaussian_stream(seed, domain, count, out);
  return RPCA_OK;
}

uint64_t rpca_kernel_launches(void) { return g_launches.load(); }

int32_t rpca_last_run_passes(const rpca_ctx* c) {
  if (!c || c->next_pass != c->i + 2) return 0;
  return c->i + 1 + (c->mirrored_last ? 0 : 1);
}

int32_t rpca_phase_times(rpca_ctx* c, double* ms, int32_t cap, int32_t* runs) {
  if (!c || !c->timing) return 0;
  const int n = (int)c->phase_ms.size();
  for (int t = 0; t < n && t < cap; ++t) ms[t] = c->phase_ms[t];
  if (runs) *runs = c->timed_runs;
  for (auto& v : c->phase_ms) v = 0.0;
  c->timed_runs = 0;
  return n;
}

// ------------------------------------------------------------ single ops
rpca_status rpca_op_fused_pass(rpca_dtype dtype, int64_t m, int64_t n, int32_t p, const void* A,
                               int64_t lda, const float* col_scale, const void* shift, const void* X,
                               int64_t ldx, void* H, int64_t ldh, void* F, int64_t ldf,
                               int32_t kernel, void* stream) {
  return guarded(nullptr, [&] {
    check_device();
    if (m < 1 || n < 1 || p < 1 || p > 255 || lda < n || ldx < p || ldh < p) throw Invalid("bad sizes");
    if (F && ldf < p) throw Invalid("bad ldf");
    if (!A || !X || !H) throw Invalid("null pointer");
    PassArgs a;
    a.dtype = dtype;
    a.mode = F ? MODE_FUSED : MODE_H;
    a.A = A; a.lda = lda; a.m = m; a.n = n; a.scale = col_scale; a.shift = shift;
    a.X = X; a.ldx = ldx; a.p = p; a.H = H; a.ldh = ldh; a.F = F; a.ldf = ldf;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf work, err;
    err.alloc(64 * sizeof(uint32_t));
    RPCA_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, 64 * sizeof(uint32_t), st));
    if (kernel != 1 && dtype != RPCA_F64) {
      work.alloc(tc_work_bytes(dtype, m, n, 64));
      a.work = work.ptr;
      a.work_bytes = work.bytes;
    }
    if (kernel == 2) {
      if (!launch_pass_tc(a, st, err.as<uint32_t>())) throw Invalid("tensor-core pass unsupported for this shape");
    } else if (kernel == 1 || !launch_pass_tc(a, st, err.as<uint32_t>())) {
      launch_pass_simt(a, st);
    }
    return read_op_error(err, st);
  });
}

rpca_status rpca_op_t_pass(rpca_dtype dtype, int64_t m, int64_t n, int32_t w, const void* A, int64_t lda,
                           const float* col_scale, const void* shift, const void* Q, int64_t ldq,
                           void* T, int64_t ldt, int32_t kernel, void* stream) {
  return guarded(nullptr, [&] {
    check_device();
    if (m < 1 || n < 1 || w < 1 || w > 256 || lda < n || ldq < w || ldt < w) throw Invalid("bad sizes");
    if (!A || !Q || !T) throw Invalid("null pointer");
    PassArgs a;
    a.dtype = dtype;
    a.mode = MODE_T;
    a.A = A; a.lda = lda; a.m = m; a.n = n; a.scale = col_scale; a.shift = shift;
    a.p = w; a.H = const_cast<void*>(Q); a.ldh = ldq; a.F = T; a.ldf = ldt;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf work, err;
    err.alloc(64 * sizeof(uint32_t));
    RPCA_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, 64 * sizeof(uint32_t), st));
    if (kernel != 1 && dtype != RPCA_F64) {
      work.alloc(tc_work_bytes(dtype, m, n, w));
      a.work = work.ptr;
      a.work_bytes = work.bytes;
    }
    if (kernel == 2) {
      if (!launch_pass_tc(a, st, err.as<uint32_t>())) throw Invalid("tensor-core pass unsupported for this shape");
    } else if (kernel == 1 || !launch_pass_tc(a, st, err.as<uint32_t>())) {
      launch_pass_simt(a, st);
    }
    return read_op_error(err, st);
  });
}

rpca_status rpca_op_qr(int32_t f64, int64_t m, int32_t nblk, int32_t l, void* H, int64_t ld, void* stream) {
  return guarded(nullptr, [&] {
    check_device();
    if (m < 1 || nblk < 1 || l < 1 || l > 255 || (int64_t)nblk * l > 256 || ld < (int64_t)nblk * l ||
        (int64_t)nblk * l > m)
      throw Invalid("bad sizes");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf scratch;
    const size_t w = (size_t)nblk * l;
    scratch.alloc((w * l + 4 * (size_t)l * l) * sizeof(double) + (size_t)kQfWords * nblk * sizeof(uint32_t) +
                  64 * sizeof(uint32_t));
    QrScratch qs;
    double* s = scratch.as<double>();
    qs.C = s; s += w * l;
    qs.Gm = s; s += (size_t)l * l;
    qs.Rk = s; s += (size_t)l * l;
    qs.Rinv = s; s += (size_t)l * l;
    qs.Racc = s; s += (size_t)l * l;
    qs.qf = reinterpret_cast<uint32_t*>(s);
    uint32_t* err = qs.qf + kQfWords * nblk;
    RPCA_CUDA_TRY(cudaMemsetAsync(qs.qf, 0, ((size_t)kQfWords * nblk + 64) * sizeof(uint32_t), st));
    if (sliced_ok(f64 != 0, m, nblk, l, 0)) {
      // H held in three BF16 slices through the whole QR (tensor cores)
      const int64_t prow = round_up(m, 128);
      DevBuf hs, sq, mt16;
      hs.alloc((size_t)3 * prow * nblk * 64 * 2);
      sq.alloc(kSliceScratchDoubles * sizeof(double));
      mt16.alloc((size_t)3 * 64 * 192 * 2);
      qs.G64 = sq.as<double>();
      qs.C64 = qs.G64 + 64 * 64;
      qs.Cfull = qs.C64 + 192 * 64;
      qs.mt = mt16.as<float>();
      block_qr_sliced(m, nblk, l, static_cast<float*>(H), ld, hs.ptr, prow, nullptr, true, qs, err, st);
      uint32_t flags = 0;
      RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      RPCA_CUDA_TRY(cudaStreamSynchronize(st));
      if (flags & DEV_ERR_BREAKDOWN) return RPCA_EBREAKDOWN;
      if (flags & DEV_ERR_TIMEOUT) return RPCA_ETIMEOUT;
      return RPCA_OK;
    }
    DevBuf hlo, mt, sl;
    if (!f64 && m >= kTcMinRows) {
      hlo.alloc((size_t)m * ld * sizeof(float));
      mt.alloc(2 * 256 * 256 * sizeof(float));
      qs.mt = mt.as<float>();
      sl.alloc((size_t)6 * round_up(m, 32) * 2 * round_up((int64_t)nblk * l, 64));
      qs.slices = sl.ptr;
      qs.slice_bytes = sl.bytes;
    }
    block_qr(f64 != 0, m, nblk, l, H, ld, nullptr, nullptr, qs, err, st, hlo.as<float>());
    uint32_t flags = 0;
    RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags & DEV_ERR_BREAKDOWN) return RPCA_EBREAKDOWN;
    return RPCA_OK;
  });
}

rpca_status rpca_op_gram(int64_t m, int32_t p, int32_t q, const float* X, int64_t ldx, const float* Y,
                          int64_t ldy, double* C, int64_t ldc, int32_t kernel, void* stream) {
  return guarded(nullptr, [&] {
    check_device();
    if (m < 1 || p < 1 || q < 1 || p > 256 || q > 256 || ldx < p || ldy < q || ldc < q) throw Invalid("bad sizes");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf xl, yl, err;
    err.alloc(64 * sizeof(uint32_t));
    RPCA_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, 64 * sizeof(uint32_t), st));
    bool done = false;
    if (kernel != 1) {
      xl.alloc((size_t)6 * round_up(m, 32) * (round_up(p, 64) + round_up(q, 64)));
      done = gram_tc(m, p, q, X, ldx, Y, ldy, C, ldc, xl.ptr, xl.bytes, st, err.as<uint32_t>());
      if (!done && kernel == 2) throw Invalid("tensor-core Gram unsupported for this shape");
    }
    if (!done) gram(false, m, p, q, X, ldx, Y, ldy, C, ldc, false, st);
    uint32_t flags = 0;
    RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, err.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags & DEV_ERR_TIMEOUT) return RPCA_ETIMEOUT;
    return RPCA_OK;
  });
}

rpca_status rpca_op_apply(int64_t m, int32_t p, int32_t q, const float* X, int64_t ldx, const double* M,
                          int64_t ldm, double alpha, double beta, float* Y, int64_t ldy, int32_t kernel,
                          void* stream) {
  return guarded(nullptr, [&] {
    check_device();
    if (m < 1 || p < 1 || q < 1 || p > 256 || q > 256 || ldx < p || ldy < q || ldm < q) throw Invalid("bad sizes");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf xl, err, mt;
    err.alloc(64 * sizeof(uint32_t));
    mt.alloc(2 * 256 * 256 * sizeof(float));
    RPCA_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, 64 * sizeof(uint32_t), st));
    bool done = false;
    if (kernel != 1) {
      xl.alloc((size_t)m * ldx * sizeof(float));
      split_lo(m, p, X, ldx, xl.as<float>(), ldx, st);
      done = apply_tc(m, p, q, X, xl.as<float>(), ldx, M, ldm, alpha, beta, Y, nullptr, ldy, mt.as<float>(), st,
                      err.as<uint32_t>());
      if (!done && kernel == 2) throw Invalid("tensor-core apply unsupported for this shape");
    }
    if (!done) gemm_xm(false, m, p, q, X, ldx, M, ldm, alpha, beta, Y, ldy, st);
    uint32_t flags = 0;
    RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, err.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags & DEV_ERR_TIMEOUT) return RPCA_ETIMEOUT;
    return RPCA_OK;
  });
}

rpca_status rpca_op_small_svd(int32_t f64, int64_t n, int32_t w, const void* T, int64_t ldt, double* S,
                              void* Vt, int64_t ldv, double* W, void* stream) {
  return guarded(nullptr, [&] {
    check_device();
    if (n < w || w < 1 || w > 256 || ldt < w || ldv < w) throw Invalid("bad sizes");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = f64 ? 8 : 4;
    // blocks: the largest divisor of w that is at most 64
    int l = std::min(64, (int)w);
    while (w % l) --l;
    const int nblk = w / l;
    DevBuf Tq, scratch;
    Tq.alloc((size_t)n * w * es);
    RPCA_CUDA_TRY(cudaMemcpy2DAsync(Tq.ptr, w * es, T, ldt * es, w * es, n, cudaMemcpyDeviceToDevice, st));
    const size_t ww = (size_t)w * w;
    scratch.alloc((w * l + 4 * (size_t)l * l + ww * 10) * sizeof(double) +
                  ((size_t)kQfWords * nblk + 64) * sizeof(uint32_t));
    QrScratch qs;
    double* s = scratch.as<double>();
    qs.C = s; s += (size_t)w * l;
    qs.Gm = s; s += (size_t)l * l;
    qs.Rk = s; s += (size_t)l * l;
    qs.Rinv = s; s += (size_t)l * l;
    qs.Racc = s; s += (size_t)l * l;
    double* RT = s; s += ww;
    double* RT2 = s; s += ww;
    double* ET = s; s += ww;
    double* Ub = s; s += ww;
    double* MV = s; s += ww;
    double* work = s; s += 5 * ww;
    qs.qf = reinterpret_cast<uint32_t*>(s);
    uint32_t* err = qs.qf + kQfWords * nblk;
    RPCA_CUDA_TRY(cudaMemsetAsync(qs.qf, 0, ((size_t)kQfWords * nblk + 64) * sizeof(uint32_t), st));
    DevBuf Tc, tlo, mt, sl;
    Tc.alloc((size_t)n * w * es);
    if (!f64 && n >= kTcMinRows) {
      tlo.alloc((size_t)n * w * sizeof(float));
      mt.alloc(2 * 256 * 256 * sizeof(float));
      qs.mt = mt.as<float>();
      sl.alloc((size_t)6 * round_up(n, 32) * 2 * round_up(w, 64));
      qs.slices = sl.ptr;
      qs.slice_bytes = sl.bytes;
    }
    svd_of_T(f64 != 0, n, nblk, l, w, Tq.ptr, Tc.ptr, tlo.as<float>(), ET, RT, RT2, S, Ub, W, work, qs, err, st);
    fold_fixup(f64 != 0, w, w, ET, Ub, MV, st);
    qr_apply(f64 != 0, n, w, w, Tq.ptr, (!f64 && n >= kTcMinRows) ? tlo.as<float>() : nullptr, w, MV, w, 1.0, 0.0,
             Vt, nullptr, ldv, qs, st, err);
    uint32_t flags = 0;
    RPCA_CUDA_TRY(cudaMemcpyAsync(&flags, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags & DEV_ERR_BREAKDOWN) return RPCA_EBREAKDOWN;
    return RPCA_OK;
  });
}

}  // extern "C"
