// Grouped batch path: buffers, work lists and the launch sequence of one run
// over all problems of a batch (kernels in k_grouped.cu and
// k_grouped_small.cu).
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "grouped.h"
#include "tc_common.cuh"

namespace rpca {
namespace grp {
namespace {

struct Mem {
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
  ~Mem() {
    if (ptr) cudaFree(ptr);
  }
  template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

// Offsets of one problem's slices in the packed buffers.
struct Slot {
  size_t h, z, xt, x, f, t, g, r, mu;
};

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct GroupedBatch {
  int count = 0, k = 0, l = 0, i = 0, w = 0;
  int max_n = 0, ldf = 0, ldt = 0, sms = 1;
  std::vector<GrpProblem> hp;
  std::vector<Slot> slot;
  std::vector<int64_t> m, n;
  Mem dH, dZ, dXT0, dXT, dX, dAcc, dSmall, dProbs, dMaps, dHitems, dTF, dTT, dR, dRT, dErr;
  size_t acc_bytes = 0;
  std::vector<CUtensorMap> maps;   // [0, count): A; [count, 2 count): Z (64 x 64 boxes)
  int64_t n_h = 0, n_tf = 0, n_tt = 0, n_r = 0, n_rt = 0;
  std::vector<const void*> key;
  Tuning tune;
  std::vector<uint32_t> hflags;
};

bool grouped_eligible(int count, const rpca_problem* P, std::string* why) {
  auto no = [&](const std::string& s) {
    if (why) *why = s;
    return false;
  };
  if (count < 1) return no("empty batch");
  for (int p = 0; p < count; ++p) {
    const rpca_problem& q = P[p];
    if (q.dtype != RPCA_BF16) return no("storage is not BF16");
    if (q.flags & ~RPCA_KEEP_T_PASS) return no("flags");
    if (q.n > q.m) return no("n > m");
    if (q.k != P[0].k || q.l != P[0].l || q.i != P[0].i) return no("k, l, i differ between problems");
    if (q.n > kMaxN || q.l > kMaxL || (q.i + 1) * q.l > kMaxW) return no("n, l or w above the grouped limits");
    if (q.n * (int64_t)(q.i + 1) * q.l > kMaxNW) return no("n w above the grouped limit");
    if (q.m >= ((int64_t)1 << 30)) return no("m too large for the grouped work lists");
    if (q.k < 1 || q.k >= q.n || q.l < q.k || (int64_t)(q.i + 1) * q.l > q.n) return no("invalid k, l, i");
  }
  return true;
}

static void build_items(GroupedBatch* g) {
  std::vector<int32_t> hp_, ht_;
  std::vector<GrpTItem> tf, tt;
  std::vector<GrpRItem> ri, rt;
  const int sub_per_item = std::max(1, g->tune.t_rows / 64);
  for (int p = 0; p < g->count; ++p) {
    const int64_t m = g->m[p], n = g->n[p];
    // tile index | 64-column steps << 24 (n <= 1024: at most 16 steps)
    const uint32_t nk = (uint32_t)cdiv(n, 64);
    for (int64_t t = 0; t < cdiv(m, 128); ++t) {
      hp_.push_back(p);
      ht_.push_back((int32_t)((uint32_t)t | (nk << 24)));
    }
    // (problem, range of 64-row groups), all columns of A at once
    const int nsub = (int)cdiv(m, 64);
    for (int s0 = 0; s0 < nsub; s0 += sub_per_item) {
      GrpTItem it{p, s0, std::min(sub_per_item, nsub - s0), 0};
      tf.push_back(it);
      tt.push_back(it);
    }
    for (int64_t r0 = 0; r0 < m; r0 += g->tune.r_rows)
      ri.push_back(GrpRItem{p, (int32_t)r0, (int32_t)std::min<int64_t>(g->tune.r_rows, m - r0), 0});
    for (int64_t r0 = 0; r0 < n; r0 += 256)
      rt.push_back(GrpRItem{p, (int32_t)r0, (int32_t)std::min<int64_t>(256, n - r0), 0});
  }
  g->n_h = (int64_t)hp_.size();
  g->n_tf = (int64_t)tf.size();
  g->n_tt = (int64_t)tt.size();
  g->n_r = (int64_t)ri.size();
  g->dHitems.alloc(2 * g->n_h * sizeof(int32_t));
  RPCA_CUDA_TRY(cudaMemcpy(g->dHitems.as<int32_t>(), hp_.data(), g->n_h * sizeof(int32_t), cudaMemcpyHostToDevice));
  RPCA_CUDA_TRY(cudaMemcpy(g->dHitems.as<int32_t>() + g->n_h, ht_.data(), g->n_h * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
  g->dTF.alloc(g->n_tf * sizeof(GrpTItem));
  RPCA_CUDA_TRY(cudaMemcpy(g->dTF.ptr, tf.data(), g->n_tf * sizeof(GrpTItem), cudaMemcpyHostToDevice));
  g->dTT.alloc(g->n_tt * sizeof(GrpTItem));
  RPCA_CUDA_TRY(cudaMemcpy(g->dTT.ptr, tt.data(), g->n_tt * sizeof(GrpTItem), cudaMemcpyHostToDevice));
  g->dR.alloc(g->n_r * sizeof(GrpRItem));
  RPCA_CUDA_TRY(cudaMemcpy(g->dR.ptr, ri.data(), g->n_r * sizeof(GrpRItem), cudaMemcpyHostToDevice));
  g->n_rt = (int64_t)rt.size();
  g->dRT.alloc(g->n_rt * sizeof(GrpRItem));
  RPCA_CUDA_TRY(cudaMemcpy(g->dRT.ptr, rt.data(), g->n_rt * sizeof(GrpRItem), cudaMemcpyHostToDevice));
}

GroupedBatch* grouped_create(int count, const rpca_problem* P, const std::vector<std::vector<double>>& G,
                             cudaStream_t st) {
  GroupedBatch* g = new GroupedBatch();
  try {
    g->count = count;
    g->k = P[0].k;
    g->l = P[0].l;
    g->i = P[0].i;
    g->w = (g->i + 1) * g->l;
    g->ldf = (int)round_up(g->l, 4);
    g->ldt = (int)round_up(g->w, 4);
    g->sms = num_sms();
    g->hp.resize(count);
    g->slot.resize(count);
    g->m.resize(count);
    g->n.resize(count);
    size_t oh = 0, oz = 0, oxt = 0, ox = 0, of = 0, ot = 0, og = 0, orr = 0, omu = 0;
    const size_t w = g->w;
    for (int p = 0; p < count; ++p) {
      const int64_t m = P[p].m, n = P[p].n;
      g->m[p] = m;
      g->n[p] = n;
      g->max_n = std::max<int>(g->max_n, (int)n);
      Slot s;
      s.h = oh;   oh = up(oh + (size_t)m * g->ldt * 4, 256);
      s.z = oz;   oz = up(oz + (size_t)m * 64 * 2, 1024);
      s.xt = oxt; oxt = up(oxt + (size_t)round_up(n, 64) * 32 * 2, 1024);
      s.x = ox;   ox = up(ox + (size_t)n * w * 4, 256);
      s.f = of;   of = up(of + (size_t)n * g->ldf * 4, 256);
      s.t = ot;   ot = up(ot + (size_t)n * g->ldt * 4, 256);
      s.g = og;   og = up(og + 3 * w * w * 8, 256);
      s.r = orr;  orr = up(orr + 2 * w * w * 4, 256);
      s.mu = omu; omu = up(omu + w * g->k * 4, 256);
      g->slot[p] = s;
    }
    g->dH.alloc(oh);
    RPCA_CUDA_TRY(cudaMemset(g->dH.ptr, 0, oh));   // the pitch's pad columns stay zero
    g->dZ.alloc(oz);
    g->dXT0.alloc(oxt);
    g->dXT.alloc(oxt);
    g->dX.alloc(ox);
    // accumulators zeroed at the start of each run: F, T, G1/G2, error words
    const size_t acc_f = 0, acc_t = up(of, 256), acc_g = acc_t + up(ot, 256), acc_e = acc_g + up(og, 256);
    g->acc_bytes = acc_e + up((size_t)(count + 1) * 4, 256);
    g->dAcc.alloc(g->acc_bytes);
    g->dSmall.alloc(orr + omu);
    unsigned char* acc = g->dAcc.as<unsigned char>();
    uint32_t* perr = reinterpret_cast<uint32_t*>(acc + acc_e);
    for (int p = 0; p < count; ++p) {
      const Slot& s = g->slot[p];
      GrpProblem& q = g->hp[p];
      std::memset(&q, 0, sizeof(q));
      q.m = g->m[p];
      q.n = g->n[p];
      q.n64 = (int32_t)round_up(q.n, 64);
      q.k = g->k;
      q.H = reinterpret_cast<float*>(g->dH.as<unsigned char>() + s.h);
      q.Z = reinterpret_cast<__nv_bfloat16*>(g->dZ.as<unsigned char>() + s.z);
      q.XT0 = reinterpret_cast<__nv_bfloat16*>(g->dXT0.as<unsigned char>() + s.xt);
      q.XT = reinterpret_cast<__nv_bfloat16*>(g->dXT.as<unsigned char>() + s.xt);
      q.X = reinterpret_cast<float*>(g->dX.as<unsigned char>() + s.x);
      q.F = reinterpret_cast<float*>(acc + acc_f + s.f);
      q.T = reinterpret_cast<float*>(acc + acc_t + s.t);
      q.G1 = reinterpret_cast<double*>(acc + acc_g + s.g);
      q.G2 = q.G1 + w * w;
      q.G3 = q.G2 + w * w;
      q.R1inv = reinterpret_cast<float*>(g->dSmall.as<unsigned char>() + s.r);
      q.R2inv = q.R1inv + w * w;
      q.MU = reinterpret_cast<float*>(g->dSmall.as<unsigned char>() + orr + s.mu);
      q.perr = perr + p;
    }
    // Z (m x 64 BF16) tensor maps, fixed for the batch; A's maps per run
    g->maps.resize(2 * (size_t)count);
    for (int p = 0; p < count; ++p)
      if (!make_tmap_2d(&g->maps[count + p], g->hp[p].Z, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g->m[p], 64, 64, 64,
                        64))
        throw Invalid("grouped batch: tensor map of Z");
    g->dMaps.alloc(g->maps.size() * sizeof(CUtensorMap));
    g->dProbs.alloc(count * sizeof(GrpProblem));
    g->dErr.alloc(4 * sizeof(uint32_t));
    build_items(g);
    // X^(0) = orth(G): G (FP32) through F, then the orth kernel with j = -1
    RPCA_CUDA_TRY(cudaMemset(g->dAcc.ptr, 0, g->acc_bytes));
    RPCA_CUDA_TRY(cudaMemset(g->dErr.ptr, 0, 4 * sizeof(uint32_t)));
    for (int p = 0; p < count; ++p) {
      const int64_t n = g->n[p];
      std::vector<float> f((size_t)n * g->ldf, 0.f);
      for (int64_t r = 0; r < n; ++r)
        for (int c = 0; c < g->l; ++c) f[(size_t)r * g->ldf + c] = (float)G[p][(size_t)r * g->l + c];
      RPCA_CUDA_TRY(cudaMemcpy(g->hp[p].F, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    RPCA_CUDA_TRY(cudaMemcpy(g->dProbs.ptr, g->hp.data(), count * sizeof(GrpProblem), cudaMemcpyHostToDevice));
    launch_orth(g->dProbs.as<GrpProblem>(), count, -1, g->l, g->w, g->ldf, g->max_n, g->dErr.as<uint32_t>(), st);
    RPCA_CUDA_TRY(cudaStreamSynchronize(st));
    g->hflags.assign(count + 1, 0u);
    return g;
  } catch (...) {
    delete g;
    throw;
  }
}

void grouped_destroy(GroupedBatch* g) { delete g; }

void grouped_set_tuning(GroupedBatch* g, const Tuning& t) {
  Tuning v = t;
  v.h_stages = std::max(2, std::min(4, v.h_stages));
  v.t_stages = std::max(2, std::min(5, v.t_stages));
  v.t_rows = std::max(64, (int)round_up(std::min(v.t_rows, 1 << 20), 64));
  v.r_rows = std::max(64, (int)round_up(std::min(v.r_rows, 1 << 20), 64));
  v.pf = std::max(0, std::min(64, v.pf));
  const bool rebuild = v.t_rows != g->tune.t_rows || v.r_rows != g->tune.r_rows;
  g->tune = v;
  if (rebuild) build_items(g);
}
Tuning grouped_tuning(const GroupedBatch* g) { return g->tune; }

int grouped_launches(const GroupedBatch* g) {
  // per pass j < i: H, F, orth; then H, Gram, chol, apply, chol, T,
  // Gram of T, eig, U
  return 3 * g->i + 9;
}

bool grouped_run(GroupedBatch* g, const rpca_matrix* A, void* const* U, const int64_t* ldu, double* const* S,
                 void* const* V, const int64_t* ldv, cudaStream_t st) {
  const int count = g->count;
  std::vector<const void*> key;
  key.reserve(7 * count);
  for (int p = 0; p < count; ++p) {
    key.push_back(A[p].data);
    key.push_back(reinterpret_cast<const void*>(A[p].ld));
    key.push_back(U ? U[p] : nullptr);
    key.push_back(reinterpret_cast<const void*>(ldu ? ldu[p] : 0));
    key.push_back(S ? S[p] : nullptr);
    key.push_back(V ? V[p] : nullptr);
    key.push_back(reinterpret_cast<const void*>(ldv ? ldv[p] : 0));
  }
  if (key != g->key) {
    for (int p = 0; p < count; ++p) {
      if (A[p].col_scale) return false;
      if (A[p].ld < g->n[p]) throw Invalid("problem " + std::to_string(p) + ": ld < n");
      if (!make_tmap_2d(&g->maps[p], A[p].data, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g->m[p], g->n[p], A[p].ld, 64,
                        64))
        return false;
      GrpProblem& q = g->hp[p];
      q.U = U ? static_cast<float*>(U[p]) : nullptr;
      q.V = V ? static_cast<float*>(V[p]) : nullptr;
      q.S = S ? S[p] : nullptr;
      q.ldu = ldu ? ldu[p] : g->k;
      q.ldv = ldv ? ldv[p] : g->k;
      if ((q.U && q.ldu < g->k) || (q.V && q.ldv < g->k)) throw Invalid("problem " + std::to_string(p) + ": ldu/ldv < k");
    }
    // nothing of an earlier run is in flight (grouped_check synchronised it)
    RPCA_CUDA_TRY(cudaMemcpy(g->dMaps.ptr, g->maps.data(), g->maps.size() * sizeof(CUtensorMap),
                             cudaMemcpyHostToDevice));
    RPCA_CUDA_TRY(cudaMemcpy(g->dProbs.ptr, g->hp.data(), count * sizeof(GrpProblem), cudaMemcpyHostToDevice));
    g->key = key;
  }
  const GrpProblem* probs = g->dProbs.as<GrpProblem>();
  const CUtensorMap* mA = g->dMaps.as<CUtensorMap>();
  const CUtensorMap* mZ = mA + count;
  auto pow2 = [](int v) {
    int c = 32;
    while (c < v) c <<= 1;
    return c;
  };
  const int ntile_max = (int)cdiv(g->max_n, 128);
  uint32_t* err = g->dErr.as<uint32_t>();
  const int32_t* ip = g->dHitems.as<int32_t>();
  const int32_t* it = ip + g->n_h;
  RPCA_CUDA_TRY(cudaMemsetAsync(g->dAcc.ptr, 0, g->acc_bytes, st));
  RPCA_CUDA_TRY(cudaMemsetAsync(err, 0, 4 * sizeof(uint32_t), st));
  // RPCA_GROUPED_TRACE=1: wait for each launch and report it on stderr; a
  // launch still running after 30 s ends the process (its kernels with it)
  static const bool trace = std::getenv("RPCA_GROUPED_TRACE") != nullptr;
  auto step = [&](const char* name) {
    if (!trace) return;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      const cudaError_t q = cudaStreamQuery(st);
      const double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (q == cudaSuccess) {
        std::fprintf(stderr, "grouped trace: %s %.3f ms\n", name, 1e3 * s);
        return;
      }
      if (q != cudaErrorNotReady) {
        std::fprintf(stderr, "grouped trace: %s failed: %s\n", name, cudaGetErrorString(q));
        std::abort();
      }
      if (s > 30.0) {
        std::fprintf(stderr, "grouped trace: %s still running after 30 s\n", name);
        std::fflush(stderr);
        std::abort();
      }
    }
  };
  const uint32_t xbytes = (uint32_t)(round_up(g->max_n, 64) / 64) * 32 * 128;
  for (int j = 0; j <= g->i; ++j) {
    HPassArgs h{mA, g->tune.h_stages, xbytes, g->ldt, g->l, j * g->l, j < g->i ? 1 : 0, j == 0 ? 1 : 0, g->tune.pf, err};
    launch_hpass(probs, ip, it, g->n_h, h, g->sms, st);
    step("h pass");
    if (j < g->i) {
      const int npf = (int)round_up(g->l, 16);
      TPassArgs t{mA, mZ, g->tune.t_stages, pow2(ntile_max * npf), npf, g->l, g->ldf, 0, g->tune.pf, err};
      launch_tpass(probs, g->dTF.as<GrpTItem>(), g->n_tf, t, g->sms, st);
      step("f pass");
      launch_orth(probs, count, j, g->l, g->w, g->ldf, g->max_n, err, st);
      step("orth");
    }
  }
  launch_gram(probs, g->dR.as<GrpRItem>(), g->n_r, g->w, err, st);
  step("gram of H");
  launch_chol(probs, count, g->w, 1, err, st);
  step("chol 1");
  launch_apply(probs, g->dR.as<GrpRItem>(), g->n_r, g->w, err, st);
  step("apply");
  launch_chol(probs, count, g->w, 2, err, st);
  step("chol 2");
  const int npt = (int)round_up(g->w, 16);
  TPassArgs t{mA, mZ, g->tune.t_stages, pow2(ntile_max * npt), npt, g->w, g->ldt, 1, g->tune.pf, err};
  launch_tpass(probs, g->dTT.as<GrpTItem>(), g->n_tt, t, g->sms, st);
  step("t pass");
  launch_gram_t(probs, g->dRT.as<GrpRItem>(), g->n_rt, g->w, err, st);
  step("gram of T");
  launch_svd(probs, count, g->w, g->ldt, g->max_n, err, st);
  step("eig");
  launch_u(probs, g->dR.as<GrpRItem>(), g->n_r, g->w, g->k, err, st);
  step("u");
  return true;
}

rpca_status grouped_check(GroupedBatch* g, cudaStream_t st, int* bad, std::string* msg) {
  const int count = g->count;
  const size_t perr_off = g->acc_bytes - up((size_t)(count + 1) * 4, 256);
  RPCA_CUDA_TRY(cudaMemcpyAsync(g->hflags.data(), g->dAcc.as<unsigned char>() + perr_off, count * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, st));
  uint32_t gerr = 0;
  RPCA_CUDA_TRY(cudaMemcpyAsync(&gerr, g->dErr.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  RPCA_CUDA_TRY(cudaStreamSynchronize(st));
  if (gerr & DEV_ERR_TIMEOUT) {
    *bad = -1;
    *msg = "grouped batch: a device-side wait timed out";
    return RPCA_ETIMEOUT;
  }
  for (int p = 0; p < count; ++p)
    if (g->hflags[p] & DEV_ERR_BREAKDOWN) {
      *bad = p;
      *msg = "problem " + std::to_string(p) + ": Cholesky QR of H broke down (numerically rank-deficient)";
      return RPCA_EBREAKDOWN;
    }
  return RPCA_OK;
}

}  // namespace grp
}  // namespace rpca
