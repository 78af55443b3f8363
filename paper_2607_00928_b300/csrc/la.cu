// Batched complex dense linear algebra kernels (GEMM, Householder QR with compact-WY panel
// factors, reflector application, triangular inverse, one-sided Jacobi SVD) and the small
// data-movement kernels the HSS construction needs.  See la.cuh for the contracts.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include <cooperative_groups.h>

#include "la.cuh"
#include "qp.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace nh {

// =============================================================================== helpers
template <typename R> __device__ __forceinline__ cplx<R> ld_op(const cplx<R>* p, int op) {
  cplx<R> v = *p;
  if (op == OP_C) v.y = -v.y;
  return v;
}

// find problem by exclusive tile prefix (last i with pre[i] <= t)
__device__ __forceinline__ int find_prob(const int* pre, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename R> void* Ops<R>::stage(const void* src, size_t bytes) {
  void* d = ar_->alloc(bytes);
  staged_ += (bytes + 15) & ~(size_t)15;
  const void* from = src;
  if (pool_) {                      // graph capture: copy from memory that outlives the graph
    void* h = pool_->alloc(bytes);
    std::memcpy(h, src, bytes);
    from = h;
  }
  NH_CK(cudaMemcpyAsync(d, from, bytes, cudaMemcpyHostToDevice, st_));
  return d;
}

template <typename R> template <typename D> D* Ops<R>::upload(const std::vector<D>& v) {
  return (D*)stage(v.data(), v.size() * sizeof(D));
}

template <typename R> int* Ops<R>::upload_ints(const std::vector<int>& v) {
  return (int*)stage(v.data(), v.size() * sizeof(int));
}

// =============================================================================== profiling
const char* kclass_name(int c) {
  static const char* n[] = {"gemm", "qr_panel", "jacobi", "other", "qrcp", "sweep", "gemm_tc", "jacobi_tc"};
  return (c >= 0 && c < K_NCLASS) ? n[c] : "?";
}
Prof::~Prof() {
  for (auto e : pool_) cudaEventDestroy(e);
  for (auto& p : pend_) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
}
cudaEvent_t Prof::get() {
  if (!pool_.empty()) { cudaEvent_t e = pool_.back(); pool_.pop_back(); return e; }
  cudaEvent_t e;
  NH_CK(cudaEventCreate(&e));
  return e;
}
void Prof::begin(cudaStream_t st) {
  if (!on) return;
  cur_ = get();
  NH_CK(cudaEventRecord(cur_, st));
}
void Prof::end(cudaStream_t st, int cls, double flops, double bytes, int nlaunch) {
  if (!on || !cur_) return;
  cudaEvent_t b = get();
  NH_CK(cudaEventRecord(b, st));
  pend_.push_back({cls, cur_, b, flops, bytes, nlaunch});
  cur_ = nullptr;
  if (pend_.size() > 4096) collect();
}
void Prof::collect() {
  for (auto& p : pend_) {
    NH_CK(cudaEventSynchronize(p.b));
    float ms = 0;
    NH_CK(cudaEventElapsedTime(&ms, p.a, p.b));
    stats[p.cls].ms += ms;
    stats[p.cls].flops += p.flops;
    stats[p.cls].bytes += p.bytes;
    stats[p.cls].launches += p.n;
    pool_.push_back(p.a);
    pool_.push_back(p.b);
  }
  pend_.clear();
}

// =============================================================================== GEMM
// C = alpha op(A) op(B) + beta C.  One CTA per BM x BN output tile of one problem; tiles of
// all problems are numbered consecutively (exclusive prefix `pre`).
// Split-k: problem pi has ks[pi] k-chunks; chunk s writes its unscaled partial tile to
// ws[pi] + s*m*n and k_gemm_reduce sums the chunks in order (deterministic).
// TA / TB: op(A) / op(B) reads the stored matrix transposed (op T or C); every problem of one
// launch has the same layout class, so the staging index arithmetic is resolved at compile time.
template <typename R, int TM, int TN, int BK, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(const GemmD<R>* __restrict__ ds, const int* __restrict__ pre,
                                              int np, const int* __restrict__ ks, cplx<R>* const* __restrict__ ws) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;   // elements each thread stages per k tile
  __shared__ cplx<R> As[BK][BM + 1];
  __shared__ cplx<R> Bs[BK][BN + 1];
  const int pi = find_prob(pre, np, blockIdx.x);
  GemmD<R> g = ds[pi];
  int lt = blockIdx.x - pre[pi];
  const int tiles_m = (g.m + BM - 1) / BM;
  const int tiles_mn = tiles_m * ((g.n + BN - 1) / BN);
  const int nsplit = ks ? ks[pi] : 1;
  const int split = lt / tiles_mn;
  lt -= split * tiles_mn;
  int kbeg = 0;
  if (nsplit > 1) {
    const int kc = (((g.k + nsplit - 1) / nsplit) + BK - 1) / BK * BK;
    kbeg = split * kc;
    const int kend = min(g.k, kbeg + kc);
    g.A = !TA ? g.A + (size_t)kbeg * g.lda : g.A + kbeg;
    g.B = !TB ? g.B + kbeg : g.B + (size_t)kbeg * g.ldb;
    g.k = max(0, kend - kbeg);
  }
  const int row0 = (lt % tiles_m) * BM, col0 = (lt / tiles_m) * BN;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  cplx<R> acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = czero<R>();
  cplx<R> ra[LA], rb[LB];
  // Stage the k tile starting at k0 into registers, zero padded.  The values are not touched
  // here (no conjugation, no select), so the loads stay in flight across the FMA loop that
  // follows; the op is applied when they are stored to shared memory.
  const R sa = g.opA == OP_C ? R(-1) : R(1), sb = g.opB == OP_C ? R(-1) : R(1);
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + q * 256;
      int ii, kk;
      if (!TA) { ii = e % BM; kk = e / BM; } else { kk = e % BK; ii = e / BK; }
      const int gi = row0 + ii, gk = k0 + kk;
      const size_t off = !TA ? (size_t)gi + (size_t)gk * g.lda : (size_t)gk + (size_t)gi * g.lda;
      ra[q] = czero<R>();
      if (gi < g.m && gk < g.k) ra[q] = g.A[off];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + q * 256;
      int jj, kk;
      if (!TB) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
      const int gj = col0 + jj, gk = k0 + kk;
      const size_t off = !TB ? (size_t)gk + (size_t)gj * g.ldb : (size_t)gj + (size_t)gk * g.ldb;
      rb[q] = czero<R>();
      if (gj < g.n && gk < g.k) rb[q] = g.B[off];
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + q * 256;
      int ii, kk;
      if (!TA) { ii = e % BM; kk = e / BM; } else { kk = e % BK; ii = e / BK; }
      As[kk][ii] = mkc(ra[q].x, sa * ra[q].y);
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + q * 256;
      int jj, kk;
      if (!TB) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
      Bs[kk][jj] = mkc(rb[q].x, sb * rb[q].y);
    }
  };
  if (g.k > 0) load(0);
  for (int k0 = 0; k0 < g.k; k0 += BK) {
    store();
    __syncthreads();
    if (k0 + BK < g.k) load(k0 + BK);      // global loads of the next tile overlap the FMAs below
#pragma unroll(TM * TN >= 64 ? 2 : BK)
    for (int kk = 0; kk < BK; ++kk) {
      cplx<R> av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
  }
  if (nsplit > 1) {
    cplx<R>* w = ws[pi] + (size_t)split * g.m * g.n;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int i = row0 + ty + 16 * a;
      if (i >= g.m) continue;
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        const int j = col0 + tx + 16 * b;
        if (j < g.n) w[(size_t)i + (size_t)j * g.m] = acc[a][b];
      }
    }
    return;
  }
  // per output row: all loads of a beta != 0 update are issued before the stores, so they overlap
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int i = row0 + ty + 16 * a;
    if (i >= g.m) continue;
    cplx<R> old[TN];
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int j = col0 + tx + 16 * b;
      old[b] = (g.beta != R(0) && j < g.n) ? g.C[(size_t)i + (size_t)j * g.ldc] : czero<R>();
    }
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int j = col0 + tx + 16 * b;
      if (j < g.n) g.C[(size_t)i + (size_t)j * g.ldc] = g.alpha * acc[a][b] + g.beta * old[b];
    }
  }
}

// C = alpha * sum_s ws[s] + beta * C for the split problems (elements numbered per problem).
template <typename R>
__global__ void k_gemm_reduce(const GemmD<R>* __restrict__ ds, const int* __restrict__ ks,
                              cplx<R>* const* __restrict__ ws, const int* __restrict__ epre, int np) {
  const int e0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int pi = find_prob(epre, np, blockIdx.x * blockDim.x);
  // a block may straddle problems: resolve per element
  int p = pi;
  while (p + 1 < np && epre[p + 1] <= e0) ++p;
  const GemmD<R> g = ds[p];
  const int e = e0 - epre[p];
  if (ks[p] <= 1 || e >= g.m * g.n) return;
  const int i = e % g.m, j = e / g.m;
  cplx<R> s = czero<R>();
  for (int q = 0; q < ks[p]; ++q) s = s + ws[p][(size_t)q * g.m * g.n + e];
  cplx<R>* c = g.C + (size_t)i + (size_t)j * g.ldc;
  cplx<R> v = g.alpha * s;
  if (g.beta != R(0)) v = v + g.beta * (*c);
  *c = v;
}

template <typename R> struct GemmCfg;
template <> struct GemmCfg<double> { static constexpr int TM = 2, TN = 2, BK = 16; };
template <> struct GemmCfg<float> { static constexpr int TM = 4, TN = 4, BK = 16; };

template <typename R, int TM, int TN, int BK>
static void launch_gemm(int cls, int grid, cudaStream_t st, const GemmD<R>* dd, const int* dp, int np, const int* ks,
                        cplx<R>* const* ws) {
  switch (cls) {
    case 0: k_gemm<R, TM, TN, BK, false, false><<<grid, 256, 0, st>>>(dd, dp, np, ks, ws); break;
    case 1: k_gemm<R, TM, TN, BK, false, true><<<grid, 256, 0, st>>>(dd, dp, np, ks, ws); break;
    case 2: k_gemm<R, TM, TN, BK, true, false><<<grid, 256, 0, st>>>(dd, dp, np, ks, ws); break;
    default: k_gemm<R, TM, TN, BK, true, true><<<grid, 256, 0, st>>>(dd, dp, np, ks, ws); break;
  }
  NH_LAUNCH_CK();
}

template <typename R> void Ops<R>::gemm(const std::vector<GemmD<R>>& d0) {
  std::vector<GemmD<R>> part[4];
  for (const auto& g : d0) {
    if (g.m <= 0 || g.n <= 0) continue;
    if (g.k <= 0 && g.beta == R(1)) continue;
    part[(g.opA != OP_N ? 2 : 0) + (g.opB != OP_N ? 1 : 0)].push_back(g);
  }
  for (int c = 0; c < 4; ++c)
    if (!part[c].empty()) gemm_class(part[c], c);
}

// ------------------------------------------------------------------------------- kernel choice
// Three kernels serve a batch of one operand-layout class: CUDA-core 64 x 64 tiles (32 x 32 in
// FP64) with split-K when the tiles cannot fill the GPU, CUDA-core 128 x 128 tiles (FP32), and
// the tensor-core kernel (FP32).  gemm_heuristic is the static rule; the autotuner replaces it per
// shape class by measurement.
enum GemmKind { GK_TILE64 = 0, GK_TILE128 = 1, GK_TC = 2 };

template <typename R> static int gemm_heuristic(const std::vector<GemmD<R>>& d) {
  if constexpr (sizeof(R) == 8) {
    return GK_TILE64;
  } else {
    int tiles_big = 0;
    double work = 0, work_big_ok = 0, work_tc = 0;
    for (const auto& g : d) {
      tiles_big += ((g.m + 127) / 128) * ((g.n + 127) / 128);
      const double w = (double)g.m * g.n * std::max(g.k, 1);
      work += w;
      if (g.m >= 128 && g.n >= 128) work_big_ok += w;
      // the tensor-core kernel pays for operand packing and a pipeline fill per tile: it wins on
      // products with long reductions or large faces (measured: 128^3 products run faster on CUDA cores)
      if (g.m >= 128 && g.n >= 128 && (g.k >= 256 || std::min(g.m, g.n) >= 256)) work_tc += w;
    }
    if (work_big_ok >= 0.8 * work && tiles_big >= 2 * 148)
      return (gemm_tc_enabled() && work_tc >= 0.8 * work) ? GK_TC : GK_TILE128;
    return GK_TILE64;
  }
}

// Autotuner.  Key: precision, layout class, and log2 buckets of the largest m, n, k and of the
// problem count of the batch.  The first batch of at least 4 GFLOP with a new key runs every
// candidate kernel twice on scratch outputs (beta = 0) and keeps the fastest second run; later
// batches with the key use that kernel.  The cache lives for the process (NH_AUTOTUNE=0 turns
// tuning off and leaves the static rule).  No tuning happens while the stream is being captured.
namespace {
struct TuneKey {
  int prec, cls, lm, ln, lk, lb;
  bool operator<(const TuneKey& o) const {
    return std::tie(prec, cls, lm, ln, lk, lb) < std::tie(o.prec, o.cls, o.lm, o.ln, o.lk, o.lb);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
int ilog2c(int v) { int l = 0; while ((1 << l) < std::max(v, 1)) ++l; return l; }
bool autotune_enabled() {
  const char* e = std::getenv("NH_AUTOTUNE");
  return !(e && std::strcmp(e, "0") == 0);
}
}  // namespace

int gemm_tune_entries() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune.size();
}

template <typename R> int Ops<R>::gemm_pick(const std::vector<GemmD<R>>& d, int cls) {
  const int h = gemm_heuristic<R>(d);
  if constexpr (sizeof(R) == 8) return h;   // one FP64 kernel
  if (pool_ || !autotune_enabled()) return h;
  int mx = 0, nx = 0, kx = 0;
  double fl = 0, out_bytes = 0;
  for (const auto& g : d) {
    mx = std::max(mx, g.m); nx = std::max(nx, g.n); kx = std::max(kx, g.k);
    fl += 8.0 * g.m * g.n * std::max(g.k, 0);
    out_bytes += (double)g.m * g.n * sizeof(cplx<R>);
  }
  // only batches where the choice matters are measured (at least 4 GFLOP), and only when the
  // scratch outputs stay modest; the rest follow the static rule
  if (fl < 4e9 || out_bytes > 4e9) return h;
  const TuneKey key{(int)sizeof(R), cls, ilog2c(mx), ilog2c(nx), ilog2c(kx), ilog2c((int)d.size())};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  std::vector<int> cand = {GK_TILE64, GK_TILE128};
  if (gemm_tc_enabled()) cand.push_back(GK_TC);
  auto mk = ar_->mark();
  std::vector<GemmD<R>> dt(d);
  for (auto& g : dt) {
    g.C = (cplx<R>*)ar_->alloc((size_t)g.m * g.n * sizeof(cplx<R>));
    g.ldc = g.m;
    g.beta = R(0);
  }
  const bool pon = prof.on;
  const int nl = launches_;
  prof.on = false;
  cudaEvent_t e0, e1;
  NH_CK(cudaEventCreate(&e0));
  NH_CK(cudaEventCreate(&e1));
  int best = h;
  float best_ms = 1e30f;
  for (int kind : cand) {
    gemm_run(dt, cls, kind);                 // first run: one-time launch set-up
    NH_CK(cudaEventRecord(e0, st_));
    gemm_run(dt, cls, kind);
    NH_CK(cudaEventRecord(e1, st_));
    NH_CK(cudaEventSynchronize(e1));
    float ms = 0;
    NH_CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) { best_ms = ms; best = kind; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  prof.on = pon;
  launches_ = nl;
  ar_->release(mk);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

template <typename R> void Ops<R>::gemm_class(const std::vector<GemmD<R>>& d, int cls) {
  if (d.empty()) return;
  gemm_run(d, cls, gemm_pick(d, cls));
}

template <typename R> void Ops<R>::gemm_run(const std::vector<GemmD<R>>& d, int cls, int kind) {
  constexpr int BM = 16 * GemmCfg<R>::TM, BN = 16 * GemmCfg<R>::TN;
  double fl = 0, by = 0;
  if (prof.on)
    for (const auto& g : d) {
      fl += 8.0 * g.m * g.n * std::max(g.k, 0);
      by += (double)sizeof(cplx<R>) * ((double)g.m * g.k + (double)g.k * g.n + (g.beta != R(0) ? 2.0 : 1.0) * g.m * g.n);
    }
  if constexpr (sizeof(R) == 4) {
    if (kind == GK_TC) {
      // the packed operands live until the GEMM has run; later scratch users on this stream are
      // ordered after it, so the space is handed back at once
      auto mk = ar_->mark();
      prof.begin(st_);
      const int nl = gemm_tc_run(d, cls, *ar_, st_, &Ops<R>::stage_cb, this);
      count(nl);
      prof.end(st_, K_GEMM_TC, fl, by, nl);
      ar_->release(mk);
      return;
    }
    if (kind == GK_TILE128) {
      std::vector<int> preb;
      int t = 0;
      for (const auto& g : d) {
        preb.push_back(t);
        t += ((g.m + 127) / 128) * ((g.n + 127) / 128);
      }
      GemmD<R>* dd = upload(d);
      int* dp = upload_ints(preb);
      prof.begin(st_);
      launch_gemm<R, 8, 8, 8>(cls, t, st_, dd, dp, (int)d.size(), nullptr, nullptr);
      prof.end(st_, K_GEMM, fl, by);
      count();
      return;
    }
  }
  int tiles = 0;
  for (const auto& g : d) tiles += ((g.m + BM - 1) / BM) * ((g.n + BN - 1) / BN);
  // split long reductions when the output tiles alone cannot fill the GPU
  std::vector<int> ks(d.size(), 1);
  bool any_split = false;
  if (tiles < 2 * 148) {
    constexpr int BK = GemmCfg<R>::BK;
    for (size_t i = 0; i < d.size(); ++i) {
      const GemmD<R>& g = d[i];
      const int t = ((g.m + BM - 1) / BM) * ((g.n + BN - 1) / BN);
      const int want = std::max(1, (2 * 148) / std::max(tiles, 1));
      const int kmax_split = std::max(1, g.k / (8 * BK));     // keep >= 8 k tiles per chunk
      const int sp = std::min(want, kmax_split);
      if (sp > 1 && (long long)sp * t <= 4096) { ks[i] = sp; any_split = true; }
    }
  }
  std::vector<int> pre2;
  std::vector<cplx<R>*> wsp(d.size(), nullptr);
  int tiles2 = 0;
  for (size_t i = 0; i < d.size(); ++i) {
    const GemmD<R>& g = d[i];
    pre2.push_back(tiles2);
    tiles2 += ((g.m + BM - 1) / BM) * ((g.n + BN - 1) / BN) * ks[i];
    if (ks[i] > 1) wsp[i] = (cplx<R>*)ar_->alloc((size_t)ks[i] * g.m * g.n * sizeof(cplx<R>));
  }
  GemmD<R>* dd = upload(d);
  int* dp = upload_ints(pre2);
  int* dks = any_split ? upload_ints(ks) : nullptr;
  cplx<R>* const* dws = any_split ? upload(wsp) : nullptr;
  prof.begin(st_);
  launch_gemm<R, GemmCfg<R>::TM, GemmCfg<R>::TN, GemmCfg<R>::BK>(cls, tiles2, st_, dd, dp, (int)d.size(), dks, dws);
  if (any_split) {
    // elements of unsplit problems are skipped inside the kernel; number only the split ones
    std::vector<GemmD<R>> ds2;
    std::vector<int> ks2, ep2;
    std::vector<cplx<R>*> ws2;
    int n2 = 0;
    for (size_t i = 0; i < d.size(); ++i)
      if (ks[i] > 1) { ds2.push_back(d[i]); ks2.push_back(ks[i]); ws2.push_back(wsp[i]); ep2.push_back(n2); n2 += d[i].m * d[i].n; }
    auto dd2 = upload(ds2);
    int* dk2 = upload_ints(ks2);
    cplx<R>* const* dw2 = upload(ws2);
    int* de2 = upload_ints(ep2);
    k_gemm_reduce<R><<<(n2 + 255) / 256, 256, 0, st_>>>(dd2, dk2, dw2, de2, (int)ds2.size());
    NH_LAUNCH_CK();
    count();
  }
  prof.end(st_, K_GEMM, fl, by);
  count();
}

// =============================================================================== copies
template <typename R>
__global__ void k_copy(const CopyD<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob(pre, np, blockIdx.x);
  const CopyD<R> c = ds[pi];
  const int lt = blockIdx.x - pre[pi];
  const int tm = (c.m + 31) / 32;
  const int i0 = (lt % tm) * 32, j0 = (lt / tm) * 32;
  __shared__ cplx<R> t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads: 32 x 8
  if (c.op == OP_N) {
    for (int jj = ty; jj < 32; jj += 8) {
      const int i = i0 + tx, j = j0 + jj;
      if (i < c.m && j < c.n) {
        cplx<R> v = (c.rs ? c.alpha * c.rs[i] : c.alpha) * c.src[(size_t)i + (size_t)j * c.lds];
        cplx<R>* o = c.dst + (size_t)i + (size_t)j * c.ldd;
        if (c.beta != R(0)) v = v + c.beta * (*o);
        *o = v;
      }
    }
  } else {
    // dst(i, j) = src(j, i) (conj): read src rows coalesced through shared memory
    for (int ii = ty; ii < 32; ii += 8) {
      const int j = j0 + tx, i = i0 + ii;     // src(j, i) at src[j + i*lds]
      if (i < c.m && j < c.n) t[ii][tx] = ld_op<R>(c.src + (size_t)j + (size_t)i * c.lds, c.op);
    }
    __syncthreads();
    for (int jj = ty; jj < 32; jj += 8) {
      const int i = i0 + tx, j = j0 + jj;
      if (i < c.m && j < c.n) {
        cplx<R> v = (c.rs ? c.alpha * c.rs[i] : c.alpha) * t[tx][jj];
        cplx<R>* o = c.dst + (size_t)i + (size_t)j * c.ldd;
        if (c.beta != R(0)) v = v + c.beta * (*o);
        *o = v;
      }
    }
  }
}

template <typename R> void Ops<R>::copy(const std::vector<CopyD<R>>& d0) {
  std::vector<CopyD<R>> d;
  std::vector<int> pre;
  int tiles = 0;
  for (const auto& c : d0) {
    if (c.m <= 0 || c.n <= 0) continue;
    d.push_back(c);
    pre.push_back(tiles);
    tiles += ((c.m + 31) / 32) * ((c.n + 31) / 32);
  }
  if (d.empty()) return;
  auto dd = upload(d);
  int* dp = upload_ints(pre);
  k_copy<R><<<tiles, 256, 0, st_>>>(dd, dp, (int)d.size());
  NH_LAUNCH_CK();
  count();
}

// kron: grid over 32x32 tiles of the destination
template <typename R>
__global__ void k_kron(const KronD<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob(pre, np, blockIdx.x);
  const KronD<R> k = ds[pi];
  const int lt = blockIdx.x - pre[pi];
  const int M = k.ma * k.mb, N = k.na * k.nb;
  const int tm = (M + 31) / 32;
  const int i0 = (lt % tm) * 32, j0 = (lt / tm) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int jj = ty; jj < 32; jj += 8) {
    const int r = i0 + tx, c = j0 + jj;
    if (r >= M || c >= N) continue;
    const int i = r / k.mb, kk = r % k.mb, j = c / k.nb, l = c % k.nb;
    cplx<R> a = k.A ? k.A[(size_t)i + (size_t)j * k.lda] : mkc(R(i == j), R(0));
    cplx<R> b = k.B ? k.B[(size_t)kk + (size_t)l * k.ldb] : mkc(R(kk == l), R(0));
    k.dst[(size_t)r + (size_t)c * k.ldd] = k.alpha * (a * b);
  }
}

template <typename R> void Ops<R>::kron(const std::vector<KronD<R>>& d0) {
  std::vector<KronD<R>> d;
  std::vector<int> pre;
  int tiles = 0;
  for (const auto& k : d0) {
    const int M = k.ma * k.mb, N = k.na * k.nb;
    if (M <= 0 || N <= 0) continue;
    d.push_back(k);
    pre.push_back(tiles);
    tiles += ((M + 31) / 32) * ((N + 31) / 32);
  }
  if (d.empty()) return;
  auto dd = upload(d);
  int* dp = upload_ints(pre);
  k_kron<R><<<tiles, 256, 0, st_>>>(dd, dp, (int)d.size());
  NH_LAUNCH_CK();
  count();
}

template <typename R>
__global__ void k_face(const FaceD<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob(pre, np, blockIdx.x);
  const FaceD<R> f = ds[pi];
  const int lt = blockIdx.x - pre[pi];
  const int N = f.na * f.nb;
  const int tm = (f.m + 31) / 32;
  const int i0 = (lt % tm) * 32, j0 = (lt / tm) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int jj = ty; jj < 32; jj += 8) {
    const int r = i0 + tx, c = j0 + jj;
    if (r >= f.m || c >= N) continue;
    const int a = c / f.nb, s = c % f.nb;
    f.dst[(size_t)r + (size_t)c * f.ldd] = f.A[(size_t)r + (size_t)a * f.lda] * f.B[(size_t)r + (size_t)s * f.ldb];
  }
}

template <typename R> void Ops<R>::face(const std::vector<FaceD<R>>& d0) {
  std::vector<FaceD<R>> d;
  std::vector<int> pre;
  int tiles = 0;
  for (const auto& f : d0) {
    const int N = f.na * f.nb;
    if (f.m <= 0 || N <= 0) continue;
    d.push_back(f);
    pre.push_back(tiles);
    tiles += ((f.m + 31) / 32) * ((N + 31) / 32);
  }
  if (d.empty()) return;
  auto dd = upload(d);
  int* dp = upload_ints(pre);
  k_face<R><<<tiles, 256, 0, st_>>>(dd, dp, (int)d.size());
  NH_LAUNCH_CK();
  count();
}

template <typename R>
__global__ void k_gather(const GatherD<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob(pre, np, blockIdx.x);
  const GatherD<R> g = ds[pi];
  const int lt = blockIdx.x - pre[pi];
  const int tm = (g.m + 31) / 32;
  const int i0 = (lt % tm) * 32, j0 = (lt / tm) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = i0 + tx;
  if (i >= g.m) return;
  const int si = g.idx[i] + g.base;
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj;
    if (j < g.n) g.dst[(size_t)i + (size_t)j * g.ldd] = g.src[(size_t)si + (size_t)j * g.lds];
  }
}

template <typename R> void Ops<R>::gather(const std::vector<GatherD<R>>& d0) {
  std::vector<GatherD<R>> d;
  std::vector<int> pre;
  int tiles = 0;
  for (const auto& g : d0) {
    if (g.m <= 0 || g.n <= 0) continue;
    d.push_back(g);
    pre.push_back(tiles);
    tiles += ((g.m + 31) / 32) * ((g.n + 31) / 32);
  }
  if (d.empty()) return;
  auto dd = upload(d);
  int* dp = upload_ints(pre);
  k_gather<R><<<tiles, 256, 0, st_>>>(dd, dp, (int)d.size());
  NH_LAUNCH_CK();
  count();
}

template <typename R> __global__ void k_set_identity(const Mat<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob(pre, np, blockIdx.x);
  const Mat<R> a = ds[pi];
  const int lt = blockIdx.x - pre[pi];
  const int tm = (a.m + 31) / 32;
  const int i0 = (lt % tm) * 32, j0 = (lt / tm) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = i0 + tx, j = j0 + jj;
    if (i < a.m && j < a.n) a.p[(size_t)i + (size_t)j * a.ld] = mkc(R(i == j), R(0));
  }
}

template <typename R> void Ops<R>::set_identity(const std::vector<Mat<R>>& d0) {
  std::vector<Mat<R>> d;
  std::vector<int> pre;
  int tiles = 0;
  for (const auto& a : d0) {
    if (a.m <= 0 || a.n <= 0) continue;
    d.push_back(a);
    pre.push_back(tiles);
    tiles += ((a.m + 31) / 32) * ((a.n + 31) / 32);
  }
  if (d.empty()) return;
  auto dd = upload(d);
  int* dp = upload_ints(pre);
  k_set_identity<R><<<tiles, 256, 0, st_>>>(dd, dp, (int)d.size());
  NH_LAUNCH_CK();
  count();
}

// =============================================================================== Householder QR
// Block reduction of a real value over 256 threads.
template <typename R> __device__ R block_sum(R v, R* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  R t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : R(0);
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  R r = sh[0];
  __syncthreads();
  return r;
}

// Householder panel of 32 columns.  Reflector H = I - tau v v^*, v[0] = 1, tau = 2 / ||v||^2 real
// (Hermitian, unitary); v = x + phase(x0) ||x|| e1 so H x = -phase(x0) ||x|| e1.  A zero column
// gets v = e1, tau = 2.  The panel's compact-WY T (Q_p = I - V_p T V_p^*) is written to Tp.
// Panel factorization, rows [j0, m) split into qcs slabs (one per CTA of a cluster; qcs = 1: one
// CTA, no cluster).  Per column: partial norms -> barrier -> every CTA forms the same reflector
// from the gathered partials (fixed order, so identical) -> one pass over its own rows writes the
// reflector entries and accumulates the partial dots of ALL remaining panel columns at once (each
// thread owns rows, so the loads of a pass are independent and coalesced along the rows) ->
// barrier -> a second pass updates the remaining columns and accumulates the next column's norm.
// The compact-WY T of the panel comes from the reduced Gram V_p^* V_p (staged 32 rows at a time).
template <typename R, bool CL>
__global__ void __launch_bounds__(256) k_qr_panel2(const QRD<R>* __restrict__ ds, int j0, int nb, int qcs) {
  int crank = 0;
  if constexpr (CL) crank = (int)cg::this_cluster().block_rank();
  const QRD<R> q = ds[blockIdx.x / qcs];
  const int k = min(q.m, q.n);
  if (j0 >= k) return;                       // uniform over the cluster
  const int b = min(nb, k - j0);
  const int rows = q.m - j0, per = (rows + qcs - 1) / qcs;
  const int lo = j0 + crank * per, hi = min(q.m, lo + per);
  __shared__ R pn[2][8];                     // partial norm^2 per warp
  __shared__ cplx<R> pd[2][8][32];           // partial dots per warp and remaining column
  __shared__ cplx<R> wt[32];
  __shared__ cplx<R> Ts[32][33];
  __shared__ cplx<R> Ys[32][33];
  cplx<R>(*Vs)[33] = Ts;                     // the Gram's row chunks, before Ts is needed
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto csync = [&]() {
    if constexpr (CL) cg::this_cluster().sync();
    else __syncthreads();
  };
  auto rmt = [&](auto* ptr, int r) {
    if constexpr (CL) return cg::this_cluster().map_shared_rank(ptr, r);
    else { (void)r; return ptr; }
  };
  {
    const cplx<R>* x = q.A + (size_t)j0 * q.lda;
    R sn = 0;
    for (int i = lo + tid; i < hi; i += 256) sn += abs2(x[i]);
    sn = warp_sum(sn);
    if (lane == 0) pn[0][warp] = sn;
  }
  for (int jj = 0; jj < b; ++jj) {
    const int col = j0 + jj, buf = jj & 1, nc = b - jj - 1;
    csync();
    R nrm2 = 0;
    {
      R v = 0;
      for (int e = lane; e < qcs * 8; e += 32) v += rmt(&pn[buf][0], e >> 3)[e & 7];
      nrm2 = warp_sum(v);                    // the same value in every warp and CTA
    }
    cplx<R>* x = q.A + (size_t)col * q.lda;
    const cplx<R> a0 = x[col];               // the owner overwrites it only after the next barrier
    const R nrm = sqrt(nrm2);
    const R aa = sqrt(abs2(a0));
    const cplx<R> ph = aa > R(0) ? mkc(a0.x / aa, a0.y / aa) : mkc(R(1), R(0));
    cplx<R> v0 = czero<R>();
    R tau = R(2);
    if (nrm > R(0)) {
      v0 = a0 + nrm * ph;
      tau = R(2) / (R(1) + (nrm2 - aa * aa) / abs2(v0));
    }
    const R v0a2 = abs2(v0);
    cplx<R>* vcol = q.V + (size_t)col * q.ldv;
    const int r0 = max(lo, col);
    // pass 1: reflector entries of own rows, partial dots v^* y_c of the nc remaining columns
    cplx<R> acc[31];
#pragma unroll
    for (int c = 0; c < 31; ++c) acc[c] = czero<R>();
    for (int i = r0 + tid; i < hi; i += 256) {
      cplx<R> v;
      if (i == col) {
        v = mkc(R(1), R(0));
        vcol[i] = v;
      } else {
        const cplx<R> xv = x[i];
        v = (v0a2 > R(0)) ? mkc((xv.x * v0.x + xv.y * v0.y) / v0a2, (xv.y * v0.x - xv.x * v0.y) / v0a2) : czero<R>();
        vcol[i] = v;
        x[i] = czero<R>();
      }
      const cplx<R>* y = x + q.lda + i;
#pragma unroll
      for (int c = 0; c < 31; ++c)
        if (c < nc) cfmac(acc[c], v, y[(size_t)c * q.lda]);
    }
#pragma unroll
    for (int c = 0; c < 31; ++c)
      if (c < nc) {
        const R wx = warp_sum(acc[c].x), wy = warp_sum(acc[c].y);
        if (lane == 0) pd[buf][warp][c] = mkc(wx, wy);
      }
    csync();
    if (tid < nc) {
      cplx<R> sw = czero<R>();
      for (int r = 0; r < qcs; ++r) {
        const cplx<R>* pr = rmt(&pd[buf][0][0], r);
        for (int w = 0; w < 8; ++w) sw = sw + pr[w * 32 + tid];
      }
      wt[tid] = tau * sw;
    }
    if (tid == 0 && col >= lo && col < hi) {
      x[col] = (nrm > R(0)) ? mkc(-nrm * ph.x, -nrm * ph.y) : czero<R>();
      q.tau[col] = tau;
    }
    __syncthreads();
    // pass 2: y_c -= v w_c on own rows; the next column's partial norm (rows > col)
    R sn = 0;
    for (int i = r0 + tid; i < hi; i += 256) {
      const cplx<R> v = (i == col) ? mkc(R(1), R(0)) : vcol[i];
      cplx<R>* y = x + q.lda + i;
#pragma unroll
      for (int c = 0; c < 31; ++c)
        if (c < nc) {
          const cplx<R> yn = y[(size_t)c * q.lda] - v * wt[c];
          y[(size_t)c * q.lda] = yn;
          if (c == 0 && i > col) sn += abs2(yn);
        }
    }
    sn = warp_sum(sn);
    if (lane == 0) pn[buf ^ 1][warp] = sn;
  }
  // Gram Y = V_p^* V_p (strict upper part) over own rows: 32-row chunks staged in shared memory,
  // each thread accumulating up to two (i, j) pairs
  const int npair = b * (b - 1) / 2;
  int pi[2], pj[2];
  cplx<R> ya[2] = {czero<R>(), czero<R>()};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int p = tid + 256 * h;
    int j = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
    while (j * (j - 1) / 2 > p) --j;
    while ((j + 1) * j / 2 <= p) ++j;
    pj[h] = j;
    pi[h] = p - j * (j - 1) / 2;
  }
  for (int rb = lo; rb < hi; rb += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * b; e += 256) {
      const int r = e & 31, c = e >> 5;
      Vs[r][c] = (rb + r < hi) ? q.V[(size_t)(rb + r) + (size_t)(j0 + c) * q.ldv] : czero<R>();
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (tid + 256 * h < npair)
        for (int r = 0; r < 32; ++r) cfmac(ya[h], Vs[r][pi[h]], Vs[r][pj[h]]);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (tid + 256 * h < npair) Ys[pi[h]][pj[h]] = ya[h];
  csync();
  if (crank == 0) {
    for (int e = tid; e < b * b; e += 256) {
      const int i = e / b, j = e % b;
      if (i >= j) continue;
      cplx<R> s2 = czero<R>();
      for (int rk = 0; rk < qcs; ++rk) s2 = s2 + *rmt(&Ys[i][j], rk);
      Ts[i][j] = s2;       // staged: Gram in the strict upper part of Ts
    }
  }
  csync();                 // peers may exit only after rank 0 has read their Gram partials
  if (crank != 0) return;
  for (int e = tid; e < 32 * 32; e += 256) {
    const int i = e / 32, j = e % 32;
    if (i < j && i < b && j < b) Ys[i][j] = Ts[i][j];
  }
  __syncthreads();
  for (int e = tid; e < 32 * 33; e += 256) Ts[e / 33][e % 33] = czero<R>();
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    const R tj = q.tau[j0 + j];
    if (tid < j) {
      cplx<R> a2 = czero<R>();
      for (int l = tid; l < j; ++l) cfma(a2, Ts[tid][l], Ys[l][j]);
      Ts[tid][j] = (-tj) * a2;
    }
    if (tid == 0) Ts[j][j] = mkc(tj, R(0));
    __syncthreads();
  }
  cplx<R>* Tp = q.Tp + (size_t)(j0 / nb) * nb * nb;
  for (int e = tid; e < nb * nb; e += 256) {
    const int i = e % nb, j = e / nb;
    Tp[e] = (i < b && j < b) ? Ts[i][j] : czero<R>();
  }
}

// S = strictly-upper(Y) + diag(1/tau), tau read from the diagonal of the panel T blocks.
template <typename R> struct GrpD { cplx<R>* Y; const cplx<R>* Tp; int w, g0, ldy; };
template <typename R> __global__ void k_group_s(const GrpD<R>* __restrict__ ds, int nb) {
  const GrpD<R> d = ds[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.w * d.w) return;
  const int i = e % d.w, j = e / d.w;
  cplx<R>& y = d.Y[(size_t)i + (size_t)j * d.ldy];
  if (i > j) y = czero<R>();
  else if (i == j) {
    const int c = d.g0 + i, p = c / nb, o = c % nb;
    const R tau = d.Tp[(size_t)p * nb * nb + o + (size_t)o * nb].x;
    y = mkc(R(1) / tau, R(0));
  }
}

template <typename R>
std::vector<QFac<R>> Ops<R>::qr(const std::vector<Mat<R>>& A, Arena& keep) {
  std::vector<QFac<R>> out(A.size());
  std::vector<QRD<R>> d(A.size());
  int kmax = 0;
  auto mk = ar_->mark();
  for (size_t i = 0; i < A.size(); ++i) {
    const Mat<R>& a = A[i];
    const int k = std::min(a.m, a.n);
    QFac<R>& f = out[i];
    f.m = a.m; f.k = k;
    f.ldv = std::max(a.m, 1);
    if (k > 0) {
      f.V = (cplx<R>*)keep.alloc((size_t)f.ldv * k * sizeof(cplx<R>));
      NH_CK(cudaMemsetAsync(f.V, 0, (size_t)f.ldv * k * sizeof(cplx<R>), st_));
      const int np = (k + NB - 1) / NB;
      f.Tp = (cplx<R>*)keep.alloc((size_t)np * NB * NB * sizeof(cplx<R>));
    }
    QRD<R>& q = d[i];
    q.A = a.p; q.lda = a.ld; q.m = a.m; q.n = a.n;
    q.V = f.V; q.ldv = f.ldv;
    q.tau = (R*)ar_->alloc(std::max(k, 1) * sizeof(R));
    q.Tp = f.Tp;
    q.W = (cplx<R>*)ar_->alloc((size_t)2 * (k > GW ? GW : NB) * std::max(a.n, 1) * sizeof(cplx<R>));
    if (k > GW) f.Tg = (cplx<R>*)keep.alloc((size_t)((k + GW - 1) / GW) * GW * GW * sizeof(cplx<R>));
    kmax = std::max(kmax, k);
  }
  if (kmax == 0) { ar_->release(mk); return out; }
  QRD<R>* dd = upload(d);
  // rows per CTA ~ 512: tall panels are shared by a cluster of up to 8 CTAs
  int mmax = 0;
  for (auto& q : d) mmax = std::max(mmax, q.m);
  int qcs = 1;
  while (qcs < 8 && (long long)qcs * 512 < mmax) qcs *= 2;
  // Two-level blocking for k > GW: the 32-column panels of one group of GW columns update only
  // the group's own columns; then the group's merged compact-WY factor (T_g from the UT identity,
  // as in group_wy) updates the rest of the matrix with GEMMs of depth GW.  Matrices with k <= GW
  // update their whole trailing matrix panel by panel.
  for (int J0 = 0; J0 < kmax; J0 += GW) {
  const int J1 = J0 + GW;
  for (int j0 = J0; j0 < std::min(J1, kmax); j0 += NB) {
    double fl = 0;
    if (prof.on)
      for (const auto& q : d) {
        const int k = std::min(q.m, q.n);
        if (j0 >= k) continue;
        const double b = std::min(NB, k - j0), mm = q.m - j0;
        fl += 8.0 * mm * b * b + 8.0 * mm * b * b / 2;   // panel reflections + V_p^* V_p
      }
    prof.begin(st_);
    if (qcs > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(d.size() * qcs));
      cfg.blockDim = dim3(256);
      cfg.stream = st_;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = qcs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      NH_CK(cudaLaunchKernelEx(&cfg, k_qr_panel2<R, true>, (const QRD<R>*)dd, j0, (int)NB, qcs));
    } else {
      k_qr_panel2<R, false><<<(int)d.size(), 256, 0, st_>>>(dd, j0, NB, 1);
      NH_LAUNCH_CK();
    }
    prof.end(st_, K_QR_PANEL, fl, 0);
    count();
    // trailing update A2 <- Q_p^* A2 = A2 - V_p T_p^* (V_p^* A2)
    std::vector<GemmD<R>> g1, g2, g3;
    for (size_t i = 0; i < d.size(); ++i) {
      const QRD<R>& q = d[i];
      const int k = std::min(q.m, q.n);
      if (j0 >= k) continue;
      const int b = std::min(NB, k - j0);
      const int cend = k > GW ? std::min(J1, q.n) : q.n;   // columns this panel updates
      const int n2 = cend - j0 - b;
      if (n2 <= 0) continue;
      const int mm = q.m - j0;
      cplx<R>* Vp = q.V + (size_t)j0 + (size_t)j0 * q.ldv;
      cplx<R>* A2 = q.A + (size_t)j0 + (size_t)(j0 + b) * q.lda;
      cplx<R>* W1 = q.W;
      cplx<R>* W2 = q.W + (size_t)NB * std::max(q.n, 1);
      cplx<R>* Tp = q.Tp + (size_t)(j0 / NB) * NB * NB;
      g1.push_back({Vp, A2, W1, b, n2, mm, q.ldv, q.lda, NB, OP_C, OP_N, R(1), R(0)});
      g2.push_back({Tp, W1, W2, b, n2, b, NB, NB, NB, OP_C, OP_N, R(1), R(0)});
      g3.push_back({Vp, W2, A2, mm, n2, b, q.ldv, NB, q.lda, OP_N, OP_N, R(-1), R(1)});
    }
    gemm(g1);
    gemm(g2);
    gemm(g3);
  }
  // the group's T_g = (striu(V_g^* V_g) + diag(1 / tau))^{-1}, then the rest of the matrix
  {
    auto mg = ar_->mark();
    std::vector<GemmD<R>> gs, g1, g2, g3;
    std::vector<GrpD<R>> gd;
    std::vector<Mat<R>> S, T;
    int wmax = 0;
    for (size_t i = 0; i < d.size(); ++i) {
      const QRD<R>& q = d[i];
      const int k = std::min(q.m, q.n);
      if (k <= GW || J0 >= k) continue;
      const int w = std::min(GW, k - J0), mm = q.m - J0;
      const cplx<R>* Vg = q.V + (size_t)J0 + (size_t)J0 * q.ldv;
      Mat<R> Sm = ar_->template mat<R>(w, w);
      gs.push_back({Vg, Vg, Sm.p, w, w, mm, q.ldv, q.ldv, Sm.ld, OP_C, OP_N, R(1), R(0)});
      gd.push_back({Sm.p, q.Tp, w, J0, Sm.ld});
      S.push_back(Sm);
      Mat<R> Tm;
      Tm.p = out[i].Tg + (size_t)(J0 / GW) * GW * GW; Tm.m = w; Tm.n = w; Tm.ld = GW;
      T.push_back(Tm);
      wmax = std::max(wmax, w);
      const int n2 = q.n - J1;
      if (n2 <= 0) continue;
      cplx<R>* A2 = q.A + (size_t)J0 + (size_t)J1 * q.lda;
      cplx<R>* W1 = q.W;
      cplx<R>* W2 = q.W + (size_t)GW * std::max(q.n, 1);
      g1.push_back({Vg, A2, W1, w, n2, mm, q.ldv, q.lda, GW, OP_C, OP_N, R(1), R(0)});
      g2.push_back({Tm.p, W1, W2, w, n2, w, GW, GW, GW, OP_C, OP_N, R(1), R(0)});
      g3.push_back({Vg, W2, A2, mm, n2, w, q.ldv, GW, q.lda, OP_N, OP_N, R(-1), R(1)});
    }
    if (!gs.empty()) {
      gemm(gs);
      auto dg = upload(gd);
      dim3 grid((wmax * wmax + 255) / 256, (unsigned)gd.size());
      k_group_s<R><<<grid, 256, 0, st_>>>(dg, NB);
      NH_LAUNCH_CK();
      count();
      trinv(S, T);
      gemm(g1);
      gemm(g2);
      gemm(g3);
    }
    ar_->release(mg);
  }
  }
  ar_->release(mk);
  return out;
}

template <typename R> void Ops<R>::group_wy(std::vector<QFac<R>>& Q, Arena& keep) {
  auto mk = ar_->mark();
  std::vector<GemmD<R>> g;
  std::vector<GrpD<R>> gd;
  std::vector<Mat<R>> S, T;
  int wmax = 0;
  for (auto& q : Q) {
    if (q.k <= NB || q.Tg) continue;              // a single panel is one block; qr() merged k > GW
    const int ng = (q.k + GW - 1) / GW;
    q.Tg = (cplx<R>*)keep.alloc((size_t)ng * GW * GW * sizeof(cplx<R>));
    for (int gi = 0; gi < ng; ++gi) {
      const int g0 = gi * GW, w = std::min(GW, q.k - g0);
      Mat<R> Sm = ar_->template mat<R>(w, w);
      const cplx<R>* Vg = q.V + (size_t)g0 + (size_t)g0 * q.ldv;
      g.push_back({Vg, Vg, Sm.p, w, w, q.m - g0, q.ldv, q.ldv, Sm.ld, OP_C, OP_N, R(1), R(0)});
      gd.push_back({Sm.p, q.Tp, w, g0, Sm.ld});
      S.push_back(Sm);
      Mat<R> Tm;
      Tm.p = q.Tg + (size_t)gi * GW * GW; Tm.m = w; Tm.n = w; Tm.ld = GW;
      T.push_back(Tm);
      wmax = std::max(wmax, w);
    }
  }
  if (g.empty()) { ar_->release(mk); return; }
  gemm(g);
  auto dg = upload(gd);
  dim3 grid((wmax * wmax + 255) / 256, (unsigned)gd.size());
  k_group_s<R><<<grid, 256, 0, st_>>>(dg, NB);
  NH_LAUNCH_CK();
  count();
  trinv(S, T);
  ar_->release(mk);
}

template <typename R>
void Ops<R>::apply_q_left(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj) {
  // Q = Q_0 Q_1 ... (blocks of BW columns: panels, or merged groups when Tg is present);
  // Q^* C applies blocks in increasing order, Q C in decreasing order.
  auto bw = [](const QFac<R>& q) { return q.Tg ? GW : NB; };
  int pmax = 0;
  for (auto& q : Q) pmax = std::max(pmax, (q.k + bw(q) - 1) / bw(q));
  if (pmax == 0) return;
  auto mk = ar_->mark();
  std::vector<cplx<R>*> W1(Q.size()), W2(Q.size());
  for (size_t i = 0; i < Q.size(); ++i) {
    W1[i] = (cplx<R>*)ar_->alloc((size_t)bw(Q[i]) * std::max(C[i].n, 1) * sizeof(cplx<R>));
    W2[i] = (cplx<R>*)ar_->alloc((size_t)bw(Q[i]) * std::max(C[i].n, 1) * sizeof(cplx<R>));
  }
  for (int s = 0; s < pmax; ++s) {
    std::vector<GemmD<R>> g1, g2, g3;
    for (size_t i = 0; i < Q.size(); ++i) {
      const QFac<R>& q = Q[i];
      const int B = bw(q);
      const int np = (q.k + B - 1) / B;
      if (s >= np || C[i].n <= 0) continue;
      const int p = conj ? s : (np - 1 - s);
      const int j0 = p * B, b = std::min(B, q.k - j0), mm = q.m - j0;
      const cplx<R>* Vp = q.V + (size_t)j0 + (size_t)j0 * q.ldv;
      const cplx<R>* Tp = (q.Tg ? q.Tg : q.Tp) + (size_t)p * B * B;
      cplx<R>* Cp = C[i].p + j0;
      g1.push_back({Vp, Cp, W1[i], b, C[i].n, mm, q.ldv, C[i].ld, B, OP_C, OP_N, R(1), R(0)});
      g2.push_back({Tp, W1[i], W2[i], b, C[i].n, b, B, B, B, conj ? OP_C : OP_N, OP_N, R(1), R(0)});
      g3.push_back({Vp, W2[i], Cp, mm, C[i].n, b, q.ldv, B, C[i].ld, OP_N, OP_N, R(-1), R(1)});
    }
    gemm(g1);
    gemm(g2);
    gemm(g3);
  }
  ar_->release(mk);
}

template <typename R>
void Ops<R>::apply_q_right(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj) {
  // C Q = C - (C V) T V^* per block, blocks in increasing order; C Q^* in decreasing order.
  auto bw = [](const QFac<R>& q) { return q.Tg ? GW : NB; };
  int pmax = 0;
  for (auto& q : Q) pmax = std::max(pmax, (q.k + bw(q) - 1) / bw(q));
  if (pmax == 0) return;
  auto mk = ar_->mark();
  std::vector<cplx<R>*> W1(Q.size()), W2(Q.size());
  for (size_t i = 0; i < Q.size(); ++i) {
    const int ld = std::max(C[i].m, 1);
    W1[i] = (cplx<R>*)ar_->alloc((size_t)ld * bw(Q[i]) * sizeof(cplx<R>));
    W2[i] = (cplx<R>*)ar_->alloc((size_t)ld * bw(Q[i]) * sizeof(cplx<R>));
  }
  for (int s = 0; s < pmax; ++s) {
    std::vector<GemmD<R>> g1, g2, g3;
    for (size_t i = 0; i < Q.size(); ++i) {
      const QFac<R>& q = Q[i];
      const int B = bw(q);
      const int np = (q.k + B - 1) / B;
      if (s >= np || C[i].m <= 0) continue;
      const int p = conj ? (np - 1 - s) : s;
      const int j0 = p * B, b = std::min(B, q.k - j0), nn = q.m - j0;
      const int ld = std::max(C[i].m, 1);
      const cplx<R>* Vp = q.V + (size_t)j0 + (size_t)j0 * q.ldv;
      const cplx<R>* Tp = (q.Tg ? q.Tg : q.Tp) + (size_t)p * B * B;
      cplx<R>* Cp = C[i].p + (size_t)j0 * C[i].ld;   // columns j0.. of C
      g1.push_back({Cp, Vp, W1[i], C[i].m, b, nn, C[i].ld, q.ldv, ld, OP_N, OP_N, R(1), R(0)});
      g2.push_back({W1[i], Tp, W2[i], C[i].m, b, b, ld, B, ld, OP_N, conj ? OP_C : OP_N, R(1), R(0)});
      g3.push_back({W2[i], Vp, Cp, C[i].m, nn, b, ld, q.ldv, C[i].ld, OP_N, OP_C, R(-1), R(1)});
    }
    gemm(g1);
    gemm(g2);
    gemm(g3);
  }
  ar_->release(mk);
}

// =============================================================================== triangular inverse
// Invert 32x32 diagonal blocks of upper-triangular matrices: one CTA (32 threads x 32) per block.
template <typename R> struct TriD { const cplx<R>* A; cplx<R>* X; int n, lda, ldx; };

template <typename R>
__global__ void k_trinv_diag(const TriD<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob(pre, np, blockIdx.x);
  const TriD<R> t = ds[pi];
  const int blk = blockIdx.x - pre[pi];
  const int o = blk * 32, b = min(32, t.n - o);
  __shared__ cplx<R> U[32][33];
  __shared__ cplx<R> X[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    U[tx][j] = (tx < b && j < b && tx <= j) ? t.A[(size_t)(o + tx) + (size_t)(o + j) * t.lda] : czero<R>();
    X[tx][j] = czero<R>();
  }
  __syncthreads();
  // column j of X solves U x = e_j by back substitution; thread tx owns column tx
  if (ty == 0 && tx < b) {
    const int j = tx;
    for (int i = j; i >= 0; --i) {
      cplx<R> s = (i == j) ? mkc(R(1), R(0)) : czero<R>();
      for (int l = i + 1; l <= j; ++l) s = s - U[i][l] * X[l][j];
      const cplx<R> d = U[i][i];
      const R dd = abs2(d);
      X[i][j] = mkc((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd);
    }
  }
  __syncthreads();
  for (int j = ty; j < b; j += 8)
    if (tx < b) t.X[(size_t)(o + tx) + (size_t)(o + j) * t.ldx] = X[tx][j];
}

template <typename R>
void Ops<R>::trinv(const std::vector<Mat<R>>& A, const std::vector<Mat<R>>& X) {
  std::vector<TriD<R>> d;
  std::vector<int> pre;
  int blocks = 0, nmax = 0;
  std::vector<Mat<R>> Xz;
  for (size_t i = 0; i < A.size(); ++i) {
    if (A[i].n <= 0) continue;
    d.push_back({A[i].p, X[i].p, A[i].n, A[i].ld, X[i].ld});
    pre.push_back(blocks);
    blocks += (A[i].n + 31) / 32;
    nmax = std::max(nmax, A[i].n);
    NH_CK(cudaMemset2DAsync(X[i].p, (size_t)X[i].ld * sizeof(cplx<R>), 0, (size_t)A[i].n * sizeof(cplx<R>),
                            A[i].n, st_));
  }
  if (d.empty()) return;
  auto mk = ar_->mark();
  auto dd = upload(d);
  int* dp = upload_ints(pre);
  k_trinv_diag<R><<<blocks, 256, 0, st_>>>(dd, dp, (int)d.size());
  NH_LAUNCH_CK();
  count();
  // doubling: blocks of size s are inverted; combine pairs into 2s:
  //   X12 = -X11 A12 X22
  for (int s = 32; s < nmax; s *= 2) {
    std::vector<GemmD<R>> g1, g2;
    std::vector<cplx<R>*> tmp;
    for (auto& t : d) {
      for (int o = 0; o + s < t.n; o += 2 * s) {
        const int n1 = s, n2 = std::min(s, t.n - o - s);
        cplx<R>* W = (cplx<R>*)ar_->alloc((size_t)n1 * n2 * sizeof(cplx<R>));
        const cplx<R>* A12 = t.A + (size_t)o + (size_t)(o + s) * t.lda;
        const cplx<R>* X22 = t.X + (size_t)(o + s) + (size_t)(o + s) * t.ldx;
        const cplx<R>* X11 = t.X + (size_t)o + (size_t)o * t.ldx;
        cplx<R>* X12 = t.X + (size_t)o + (size_t)(o + s) * t.ldx;
        g1.push_back({A12, X22, W, n1, n2, n2, t.lda, t.ldx, n1, OP_N, OP_N, R(1), R(0)});
        g2.push_back({X11, W, X12, n1, n2, n1, t.ldx, n1, t.ldx, OP_N, OP_N, R(-1), R(0)});
      }
    }
    gemm(g1);
    gemm(g2);
  }
  ar_->release(mk);
}

// =============================================================================== Jacobi SVD
// One-sided (Hestenes) Jacobi on the columns of X (r x k), block-pair cyclic ordering:
// columns are split into blocks of 16; each launch is one round of a round-robin
// tournament over blocks; a CTA takes one block pair and sweeps all 32-choose-2 column
// pairs of it (16 warps, one column pair per warp per inner round).
// A pair found orthogonal is recorded with the versions of its two blocks and the noise floor of
// that visit; while neither block has been rotated since and the floor has not come down, the pair
// is still orthogonal and later visits skip it without forming its Gram.
struct JacSeen { unsigned va, vb; double floor2; };

template <typename R> struct JacD {
  cplx<R>* X; int ld, r, k, nblk;   // nblk even
  unsigned* off;                    // max |gamma|/sqrt(alpha beta) of this sweep (float bits)
  const int* done;                  // converged flag from the previous sweep
  R* amax;                          // max squared column norm at the start of the sweep
  unsigned* ver;                    // per 32-column block: how many blocked steps rotated it (blocked kernels)
  JacSeen* seen;                    // per block pair (I < J): the record of its last orthogonal visit
};

// the pair's record, or nullptr when the kernel keeps none
template <typename R> __device__ __forceinline__ JacSeen* jac_seen(const JacD<R>& d, int I, int J) {
  if (!d.seen) return nullptr;
  const int a = min(I, J), b = max(I, J);
  return d.seen + (size_t)a * d.nblk + b;
}
// true when the pair is known to be orthogonal (uniform: thread 0 decides, one barrier)
template <typename R>
__device__ __forceinline__ bool jac_known_orthogonal(const JacD<R>& d, int I, int J, double floor2, int* flag) {
  if (threadIdx.x == 0) {
    int k = 0;
    if (const JacSeen* sp = jac_seen(d, I, J)) {
      const JacSeen sn = *sp;
      const int a = min(I, J), b = max(I, J);
      k = sn.va == d.ver[a] && sn.vb == d.ver[b] && floor2 >= sn.floor2;
    }
    *flag = k;
  }
  __syncthreads();
  return *flag != 0;
}
template <typename R> __device__ __forceinline__ void jac_mark_orthogonal(const JacD<R>& d, int I, int J, double floor2) {
  if (JacSeen* sp = jac_seen(d, I, J)) {
    const int a = min(I, J), b = max(I, J);
    *sp = JacSeen{d.ver[a], d.ver[b], floor2};
  }
}
template <typename R> __device__ __forceinline__ void jac_mark_rotated(const JacD<R>& d, int I, int J) {
  if (d.ver) {   // each block is in one pair per round: no other CTA of this launch touches these
    d.ver[I] += 1u;
    d.ver[J] += 1u;
  }
}

// Largest squared column norm of each matrix (one CTA per matrix): the scale below which a
// column counts as numerically zero in the Jacobi sweeps.
template <typename R> __global__ void __launch_bounds__(256) k_colmax(const JacD<R>* __restrict__ ds) {
  const JacD<R> d = ds[blockIdx.x];
  __shared__ R red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R m = 0;
  for (int j = warp; j < d.k; j += 8) {
    R acc = 0;
    for (int i = lane; i < d.r; i += 32) acc += abs2(d.X[(size_t)i + (size_t)j * d.ld]);
    acc = warp_sum(acc);
    m = fmax(m, acc);
  }
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    R t = 0;
    for (int w = 0; w < 8; ++w) t = fmax(t, red[w]);
    *d.amax = t;
  }
}

__device__ __forceinline__ void rr_pair(int p, int r, int n, int& a, int& b) {
  // circle method for n (even) players: player 0 fixed
  if (p == 0) { a = 0; b = 1 + (r % (n - 1)); }
  else { a = 1 + (r + p) % (n - 1); b = 1 + (r - p + n - 1) % (n - 1); }
}

// Cyclic two-sided Jacobi on the Hermitian W x W Gram G in shared memory (leading dimension ldg),
// accumulating V <- V J for every rotation J, until a sweep rotates nothing or max_inner sweeps.
// A round rotates W / 2 disjoint column pairs (round-robin order) with the one-sided rotation
// formula evaluated on Gram entries; pairs whose cosine is at most tol, or with a column below the
// noise floor, are left alone.  G <- J^* G J is applied block by block: output 2 x 2 block (P, Q)
// depends only on input block (P, Q), so one thread updates it in place -- two barriers per round.
// Shared scratch: rc, rse, ract, pa, pb (W / 2 entries each) and *any_s.  Called by all 256
// threads of the CTA.
template <typename R, int W>
__device__ void jac_inner(cplx<R>* G, cplx<R>* V, int ldg, R floor2, R tol, int max_inner, R* rc, cplx<R>* rse,
                          int* ract, int* pa, int* pb, int* any_s) {
  constexpr int NP = W / 2;
  const int tid = threadIdx.x;
  for (int e = tid; e < W * W; e += 256) {
    const int i = e / W, j = e - i * W;
    V[i * ldg + j] = mkc(R(i == j ? 1 : 0), R(0));
  }
  // exact Hermitian symmetry (the rounds below update one half and mirror it)
  for (int e = tid; e < W * W; e += 256) {
    const int i = e / W, j = e - i * W;
    if (i < j) G[j * ldg + i] = conj(G[i * ldg + j]);
    else if (i == j) G[i * ldg + i].y = R(0);
  }
  if (tid == 0) *any_s = 0;
  __syncthreads();
  for (int sw = 0; sw < max_inner; ++sw) {
    for (int ir = 0; ir < W - 1; ++ir) {
      if (tid < NP) {
        int a, b;
        rr_pair(tid, ir, W, a, b);
        pa[tid] = a;
        pb[tid] = b;
        const R al = G[a * ldg + a].x, be = G[b * ldg + b].x;
        const cplx<R> ga = G[a * ldg + b];
        const R g = sqrt(abs2(ga));
        int act = 0;
        R c = R(1);
        cplx<R> se = czero<R>();
        if (al > floor2 && be > floor2 && g > R(0) && g / (sqrt(al) * sqrt(be)) > tol) {
          const R zeta = (be - al) / (R(2) * g);
          const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
          c = R(1) / sqrt(R(1) + t * t);
          const R sn = c * t;
          se = mkc(sn * ga.x / g, sn * ga.y / g);
          act = 1;
          *any_s = 1;
        }
        rc[tid] = c;
        rse[tid] = se;
        ract[tid] = act;
      }
      __syncthreads();
      // J of pair P: columns (a, b) -> (c x_a - conj(se) x_b, se x_a + c x_b); identity when inactive.
      // Blocks (P, Q) with P <= Q only; block (Q, P) is the conjugate transpose.
      for (int e = tid; e < NP * (NP + 1) / 2; e += 256) {
        int Q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (Q * (Q + 1) / 2 > e) --Q;
        while ((Q + 1) * (Q + 2) / 2 <= e) ++Q;
        const int P = e - Q * (Q + 1) / 2;
        const int aP = ract[P], aQ = ract[Q];
        if (!aP && !aQ) continue;
        const int ra = pa[P], rb = pb[P], ca = pa[Q], cb = pb[Q];
        const R cp = rc[P], cq = rc[Q];
        const cplx<R> sp = rse[P], sq = rse[Q];
        const cplx<R> g00 = G[ra * ldg + ca], g01 = G[ra * ldg + cb], g10 = G[rb * ldg + ca], g11 = G[rb * ldg + cb];
        // T = g J_Q
        const cplx<R> t00 = cq * g00 - conj(sq) * g01, t01 = sq * g00 + cq * g01;
        const cplx<R> t10 = cq * g10 - conj(sq) * g11, t11 = sq * g10 + cq * g11;
        // J_P^* T
        cplx<R> n00 = cp * t00 - sp * t10, n01 = cp * t01 - sp * t11;
        cplx<R> n10 = conj(sp) * t00 + cp * t10, n11 = conj(sp) * t01 + cp * t11;
        if (P == Q) {   // the rotated pair: off-diagonal zero, real diagonal
          n01 = czero<R>();
          n10 = czero<R>();
          n00.y = R(0);
          n11.y = R(0);
        }
        G[ra * ldg + ca] = n00;
        G[ra * ldg + cb] = n01;
        G[rb * ldg + ca] = n10;
        G[rb * ldg + cb] = n11;
        if (P != Q) {
          G[ca * ldg + ra] = conj(n00);
          G[cb * ldg + ra] = conj(n01);
          G[ca * ldg + rb] = conj(n10);
          G[cb * ldg + rb] = conj(n11);
        }
      }
      for (int e = tid; e < W * NP; e += 256) {
        const int i = e / NP, Q = e - i * NP;
        if (!ract[Q]) continue;
        const int ca = pa[Q], cb = pb[Q];
        const R c = rc[Q];
        const cplx<R> se = rse[Q];
        const cplx<R> x = V[i * ldg + ca], y = V[i * ldg + cb];
        V[i * ldg + ca] = c * x - conj(se) * y;
        V[i * ldg + cb] = se * x + c * y;
      }
      __syncthreads();
    }
    const int more = *any_s;
    __syncthreads();
    if (!more) break;
    if (tid == 0) *any_s = 0;
    __syncthreads();
  }
}

template <typename R>
__device__ void jac_rotate(cplx<R>* xa, cplx<R>* xb, int r, R tol, unsigned* off, R floor2) {
  const int lane = threadIdx.x & 31;
  R al = 0, be = 0;
  cplx<R> ga = czero<R>();
  for (int i = lane; i < r; i += 32) {
    const cplx<R> a = xa[i], b = xb[i];
    al += abs2(a);
    be += abs2(b);
    cfmac(ga, a, b);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga.x = warp_sum(ga.x);
  ga.y = warp_sum(ga.y);
  const R g = sqrt(abs2(ga));
  if (!(al > R(0)) || !(be > R(0)) || g == R(0)) return;
  // a column below the noise floor is numerically zero: leave it out of rotations and of the
  // convergence test (its direction is rounding noise and would only pollute the other column)
  if (fmin(al, be) <= floor2) return;
  const R rel = g / sqrt(al * be);
  if (lane == 0) atomicMax(off, __float_as_uint((float)rel));
  if (rel <= tol) return;
  const R zeta = (be - al) / (R(2) * g);
  const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
  const R c = R(1) / sqrt(R(1) + t * t);
  const R s = c * t;
  const cplx<R> e = mkc(ga.x / g, ga.y / g);       // phase of gamma
  const cplx<R> se = mkc(s * e.x, s * e.y);
  const cplx<R> sec = mkc(s * e.x, -s * e.y);
  for (int i = lane; i < r; i += 32) {
    const cplx<R> a = xa[i], b = xb[i];
    xa[i] = c * a - sec * b;
    xb[i] = se * a + c * b;
  }
}

template <typename R>
__global__ void __launch_bounds__(512) k_jacobi_round(const JacD<R>* __restrict__ ds, int round, R tol, R negl2) {
  const JacD<R> d = ds[blockIdx.y];
  if (*d.done) return;
  if (round >= d.nblk - 1 || (int)blockIdx.x >= d.nblk / 2) return;
  int I, J;
  rr_pair(blockIdx.x, round, d.nblk, I, J);
  __shared__ int cidx[32];
  __shared__ int nc;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int q = 0; q < 2; ++q) {
      const int B = q ? J : I;
      for (int j = B * 16; j < min(B * 16 + 16, d.k); ++j) cidx[c++] = j;
    }
    nc = c;
  }
  __syncthreads();
  const int n = nc;
  if (n < 2) return;
  const int warp = threadIdx.x >> 5;
  // inner round-robin over 32 slots (empty slots skipped)
  for (int ir = 0; ir < 31; ++ir) {
    int a, b;
    rr_pair(warp, ir, 32, a, b);
    if (a < n && b < n) {
      const int ca = min(cidx[a], cidx[b]), cb = max(cidx[a], cidx[b]);
      jac_rotate<R>(d.X + (size_t)ca * d.ld, d.X + (size_t)cb * d.ld, d.r, tol, d.off, negl2 * (*d.amax));
    }
    __syncthreads();
  }
}

// Cluster-resident variant: the 32 columns of a block pair live in shared memory, split by
// rows over a cluster of JCS CTAs.  Each inner round needs the three dot products of every
// column pair over all rows: every CTA writes its partials, one cluster barrier, then each
// warp gathers the JCS partials over DSMEM in a fixed order, so all CTAs compute the same
// rotation and apply it to their own rows.  Data leaves shared memory once per round.
template <typename R>
__global__ void __launch_bounds__(512) k_jacobi_cluster(const JacD<R>* __restrict__ ds, int round, R tol, int rpc,
                                                         R negl2) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int JCS = (int)cluster.num_blocks();     // 8 or 16 CTAs share the rows of a block pair
  const JacD<R> d = ds[blockIdx.y];
  const int pair = blockIdx.x / JCS;
  // every CTA of a cluster shares (blockIdx.y, pair), so these exits are cluster-uniform
  if (*d.done) return;
  if (round >= d.nblk - 1 || pair >= d.nblk / 2) return;
  extern __shared__ unsigned char smraw_j[];
  cplx<R>* S = (cplx<R>*)smraw_j;
  __shared__ R part[2][16][4];
  __shared__ int cidx[32];
  __shared__ int nc_s;
  int I, J;
  rr_pair(pair, round, d.nblk, I, J);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int q = 0; q < 2; ++q) {
      const int B = q ? J : I;
      for (int j = B * 16; j < min(B * 16 + 16, d.k); ++j) cidx[c++] = j;
    }
    nc_s = c;
  }
  __syncthreads();
  const int n = nc_s;
  const int r0 = crank * rpc, r1 = min(d.r, r0 + rpc), rl = max(0, r1 - r0);
  for (int e = threadIdx.x; e < n * rl; e += blockDim.x) {
    const int c = e / rl, i = e - c * rl;
    S[(size_t)c * rpc + i] = d.X[(size_t)(r0 + i) + (size_t)cidx[c] * d.ld];
  }
  cluster.sync();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int ir = 0; ir < 31; ++ir) {
    const int buf = ir & 1;
    int a, b;
    rr_pair(warp, ir, 32, a, b);
    const bool act = (a < n && b < n);
    int sa = a, sb = b;
    if (act && cidx[a] > cidx[b]) { sa = b; sb = a; }
    R al = 0, be = 0;
    cplx<R> ga = czero<R>();
    if (act) {
      const cplx<R>* xa = S + (size_t)sa * rpc;
      const cplx<R>* xb = S + (size_t)sb * rpc;
      for (int i = lane; i < rl; i += 32) {
        const cplx<R> u = xa[i], v = xb[i];
        al += abs2(u);
        be += abs2(v);
        cfmac(ga, u, v);
      }
    }
    al = warp_sum(al);
    be = warp_sum(be);
    ga.x = warp_sum(ga.x);
    ga.y = warp_sum(ga.y);
    if (lane == 0) {
      part[buf][warp][0] = al; part[buf][warp][1] = be; part[buf][warp][2] = ga.x; part[buf][warp][3] = ga.y;
    }
    cluster.sync();
    R v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    if (lane < JCS) {
      const R* p = cluster.map_shared_rank(&part[buf][warp][0], lane);
      v0 = p[0]; v1 = p[1]; v2 = p[2]; v3 = p[3];
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    v3 = warp_sum(v3);
    if (act) {
      const R g = sqrt(v2 * v2 + v3 * v3);
      if (v0 > R(0) && v1 > R(0) && g > R(0) && fmin(v0, v1) > negl2 * (*d.amax)) {
        const R rel = g / sqrt(v0 * v1);
        if (crank == 0 && lane == 0) atomicMax(d.off, __float_as_uint((float)rel));
        if (rel > tol) {
          const R zeta = (v1 - v0) / (R(2) * g);
          const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
          const R c = R(1) / sqrt(R(1) + t * t);
          const R s = c * t;
          const cplx<R> se = mkc(s * v2 / g, s * v3 / g);
          const cplx<R> sec = mkc(s * v2 / g, -s * v3 / g);
          cplx<R>* xa = S + (size_t)sa * rpc;
          cplx<R>* xb = S + (size_t)sb * rpc;
          for (int i = lane; i < rl; i += 32) {
            const cplx<R> u = xa[i], v = xb[i];
            xa[i] = c * u - sec * v;
            xb[i] = se * u + c * v;
          }
        }
      }
    }
    __syncthreads();
  }
  cluster.sync();
  for (int e = threadIdx.x; e < n * rl; e += blockDim.x) {
    const int c = e / rl, i = e - c * rl;
    d.X[(size_t)(r0 + i) + (size_t)cidx[c] * d.ld] = S[(size_t)c * rpc + i];
  }
}

// Blocked one-sided Jacobi step (hierarchical blocking): the up to 64 columns of a block pair
// (two blocks of 32) are orthogonalized together.  Their Gram matrix G = X_P^* X_P is formed
// in one pass over the rows; a cyclic two-sided Jacobi on G in shared memory accumulates the
// unitary V with V^* G V diagonal; a second pass applies X_P <- X_P V.  The rotations on G are
// exactly the one-sided rotations of the column pairs (same angle formula as jac_rotate), only
// evaluated on the Gram entries instead of re-reading the columns, so the data are read twice
// per block pair instead of once per column pair.  The convergence measure of a pair is taken
// from the freshly formed G; a pair within tol_out is left untouched, the inner rotations go
// down to tol < tol_out.  The gap keeps pairs whose cosines sit at the rounding level of the
// Gram (a few u sqrt(r)) from being reprocessed sweep after sweep.
template <typename R> struct JbCfg {
  static constexpr int W = 64;                           // columns per block pair
  static constexpr int T = sizeof(R) == 4 ? 64 : 32;     // rows per staged chunk
  static constexpr int LDX = T + 1, LDG = W + 1;         // padded strides (bank spread)
  static constexpr int KP = T / 16;                      // chunk rows per thread in the update
  static constexpr int PF = W * T / 256;                 // chunk elements each thread stages
  static constexpr size_t smem = (size_t)(2 * W * LDG + W * LDX) * sizeof(cplx<R>);
};

template <typename R>
__device__ __forceinline__ void jb_load(const JacD<R>& d, const int* cidx, int r0, cplx<R> (&pf)[JbCfg<R>::PF]) {
  constexpr int T = JbCfg<R>::T;
#pragma unroll
  for (int q = 0; q < JbCfg<R>::PF; ++q) {
    const int e = threadIdx.x + 256 * q, c = e / T, k = e - c * T, row = r0 + k, col = cidx[c];
    pf[q] = (col >= 0 && row < d.r) ? d.X[(size_t)row + (size_t)col * d.ld] : czero<R>();
  }
}

template <typename R>
__device__ __forceinline__ void jb_stage(cplx<R>* Xs, const cplx<R> (&pf)[JbCfg<R>::PF]) {
  constexpr int T = JbCfg<R>::T, LDX = JbCfg<R>::LDX;
#pragma unroll
  for (int q = 0; q < JbCfg<R>::PF; ++q) {
    const int e = threadIdx.x + 256 * q, c = e / T, k = e - c * T;
    Xs[c * LDX + k] = pf[q];
  }
}

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1)
    k_jacobi_blk(const JacD<R>* __restrict__ ds, int round, R tol, R tol_out, R negl2, int max_inner,
                 unsigned long long* __restrict__ rows_updated) {
  using C = JbCfg<R>;
  constexpr int W = C::W, T = C::T, LDX = C::LDX, LDG = C::LDG, KP = C::KP;
  const JacD<R> d = ds[blockIdx.y];
  if (*d.done) return;
  if (round >= d.nblk - 1 || (int)blockIdx.x >= d.nblk / 2) return;
  extern __shared__ unsigned char smraw_b[];
  cplx<R>* G = (cplx<R>*)smraw_b;      // G[i * LDG + j] = x_i^* x_j
  cplx<R>* V = G + W * LDG;            // V[i * LDG + j]
  cplx<R>* Xs = V + W * LDG;           // chunk, column-major: Xs[c * LDX + k]
  __shared__ int cidx[W];
  __shared__ R rc[W / 2];
  __shared__ cplx<R> rse[W / 2];
  __shared__ int ract[W / 2], rpa[W / 2], rpb[W / 2];
  __shared__ int any_s, known;
  __shared__ float offw[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int I, J;
  rr_pair(blockIdx.x, round, d.nblk, I, J);
  if (tid < W) {
    const int c = (tid < 32 ? I : J) * 32 + (tid & 31);
    cidx[tid] = c < d.k ? c : -1;
  }
  __syncthreads();
  const R floor2 = negl2 * (*d.amax);
  if (jac_known_orthogonal(d, I, J, (double)floor2, &known)) return;
  // ---- 1. Gram: thread (ti, tj) owns G[ti + 16p][tj + 16q], p, q < 4
  const int ti = tid >> 4, tj = tid & 15;
  {
    cplx<R> acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = czero<R>();
    cplx<R> pf[C::PF];
    jb_load<R>(d, cidx, 0, pf);
    for (int r0 = 0; r0 < d.r; r0 += T) {
      jb_stage<R>(Xs, pf);
      __syncthreads();
      if (r0 + T < d.r) jb_load<R>(d, cidx, r0 + T, pf);
#pragma unroll 4
      for (int k = 0; k < T; ++k) {
        cplx<R> a[4], b[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) a[p] = Xs[(ti + 16 * p) * LDX + k];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Xs[(tj + 16 * q) * LDX + k];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) cfmac(acc[p][q], a[p], b[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) G[(ti + 16 * p) * LDG + tj + 16 * q] = acc[p][q];
  }
  __syncthreads();
  // ---- 2. largest cosine of the fresh Gram (columns above the noise floor only)
  {
    float m = 0.f;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ti + 16 * p, j = tj + 16 * q;
        const R di = G[i * LDG + i].x, dj = G[j * LDG + j].x;
        if (i != j && di > floor2 && dj > floor2) {
          const R g = sqrt(abs2(G[i * LDG + j]));
          m = fmaxf(m, (float)(g / (sqrt(di) * sqrt(dj))));
        }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) offw[warp] = m;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < 8; ++w) t = fmaxf(t, offw[w]);
      offw[0] = t;
      if (t > 0.f) atomicMax(d.off, __float_as_uint(t));
    }
    __syncthreads();
    if ((R)offw[0] <= tol_out) {         // uniform: the pair is already orthogonal
      if (tid == 0) jac_mark_orthogonal(d, I, J, (double)floor2);
      return;
    }
  }
  // ---- 3. two-sided Jacobi on G, V <- V J for every rotation J
  jac_inner<R, W>(G, V, LDG, floor2, tol, max_inner, rc, rse, ract, rpa, rpb, &any_s);
  // ---- 4. X_P <- X_P V, chunk by chunk (in place; each chunk's rows are read before written)
  const int tk = ti;
  cplx<R> pf[C::PF];
  jb_load<R>(d, cidx, 0, pf);
  for (int r0 = 0; r0 < d.r; r0 += T) {
    jb_stage<R>(Xs, pf);
    __syncthreads();
    if (r0 + T < d.r) jb_load<R>(d, cidx, r0 + T, pf);
    cplx<R> acc[KP][4];
#pragma unroll
    for (int p = 0; p < KP; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = czero<R>();
#pragma unroll 4
    for (int c = 0; c < W; ++c) {
      cplx<R> a[KP], b[4];
#pragma unroll
      for (int p = 0; p < KP; ++p) a[p] = Xs[c * LDX + tk + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = V[c * LDG + tj + 16 * q];
#pragma unroll
      for (int p = 0; p < KP; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc[p][q], a[p], b[q]);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < KP; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) Xs[(tj + 16 * q) * LDX + tk + 16 * p] = acc[p][q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < C::PF; ++q) {
      const int e = tid + 256 * q, c = e / T, k = e - c * T, row = r0 + k, col = cidx[c];
      if (col >= 0 && row < d.r) d.X[(size_t)row + (size_t)col * d.ld] = Xs[c * LDX + k];
    }
    __syncthreads();
  }
  if (tid == 0) {
    atomicAdd(rows_updated, (unsigned long long)d.r);
    jac_mark_rotated(d, I, J);
  }
}

// =============================================================================== blocked Jacobi on tensor cores
// The FP32 blocked Jacobi step of k_jacobi_blk with both of its products on the tensor cores
// (tcgen05 kind::tf32, 3xTF32 split), one CTA per block pair:
//  1. Gram G = X_P^* X_P, X_P = the pair's 64 columns, as the real Gram of the stacked operand
//     S = [Re X_P, Im X_P]^T (128 x rows): D = S S^T holds Re^T Re, Re^T Im, Im^T Re, Im^T Im, and
//     G = (Re^T Re + Im^T Im) + i (Re^T Im - Im^T Re).  One M = N = 128 MMA per k = 8 step and split
//     term: 3 MMAs, against 12 of M = N = 64 for the complex form.  Chunks of 64 rows are split into
//     TF32 hi/lo planes in shared memory (two buffers; loads run two chunks ahead in registers).
//     Groups of four chunks (256 rows) accumulate in one of two tensor-memory accumulators; a
//     finished group is added (FP32, round to nearest) into four real quarter Grams in shared memory,
//     one per warp pair, while the next group's MMAs run, so no tensor-core accumulation runs longer
//     than 256 rows (its truncation stays near 1e-6 relative).
//  2. The largest cosine and the two-sided Jacobi on G -> V, exactly as in k_jacobi_blk.
//  3. X_P <- X_P V over chunks of 128 rows: A = the chunk (complex planes), B = the planes of V^T,
//     12 MMAs of M = 128, N = 64 per k = 8 step into one of two accumulators; the previous chunk's
//     product is written back while the current chunk's MMAs run.
// Every wait is bounded: one that runs out sets g_jac_error, and the CTA leaves X untouched.
namespace {
constexpr int JT_W = 64;                          // pair width
constexpr int JT_CH = 64;                         // Gram: rows per chunk
constexpr int JT_GRP = 4;                         // Gram: chunks per tensor-memory accumulation
constexpr int JT_CU = 128;                        // update: rows per chunk
constexpr uint32_t JT_SBO = 16 * 128;             // 8-row group stride of a 64-deep K-major plane
constexpr int JT_P64 = 64 * 64 * 4;               // one real plane, 64 rows x 64 deep (16 KB)
constexpr int JT_P128 = 128 * 64 * 4;             // one real plane, 128 rows x 64 deep (32 KB)
constexpr int JT_REGION = 4 * JT_P64;             // 64 KB
constexpr int JT_LDG = JT_W + 1;
constexpr int JT_LDQ = JT_W + 1;                  // quarter Grams: 64 x 65 floats
constexpr size_t JT_QUART = 4 * (size_t)JT_W * JT_LDQ * sizeof(float);
constexpr size_t JT_SMEM = 2 * (size_t)JT_REGION + JT_QUART + 1024;
static_assert(JT_QUART >= (size_t)4 * JT_P64, "the B planes of the update live in the quarter region");
static_assert((size_t)2 * JT_W * JT_LDG * sizeof(float2) <= (size_t)2 * JT_REGION, "G and V fit in regions 0-1");
}  // namespace

__device__ int g_jac_error;

// the 12 MMAs of one k = 8 step of a complex product D = A B^T given as TF32 planes (A: m rows,
// planes pa bytes apart; B: 64 rows, planes JT_P64 apart)
__device__ __forceinline__ void jt_mma12(uint32_t dr, uint32_t di, uint32_t a, uint32_t pa, uint32_t b, uint32_t ko,
                                         uint32_t f, uint32_t idp, uint32_t idn) {
  const uint64_t arh = tc_desc(a + ko, JT_SBO), arl = tc_desc(a + pa + ko, JT_SBO),
                 aih = tc_desc(a + 2 * pa + ko, JT_SBO), ail = tc_desc(a + 3 * pa + ko, JT_SBO);
  const uint64_t brh = tc_desc(b + ko, JT_SBO), brl = tc_desc(b + JT_P64 + ko, JT_SBO),
                 bih = tc_desc(b + 2 * JT_P64 + ko, JT_SBO), bil = tc_desc(b + 3 * JT_P64 + ko, JT_SBO);
  // D = A B: Dr = Ar Br - Ai Bi, Di = Ar Bi + Ai Br
  tc_mma(dr, arh, brh, idp, f); tc_mma(dr, arh, brl, idp, 1u); tc_mma(dr, arl, brh, idp, 1u);
  tc_mma(dr, aih, bih, idn, 1u); tc_mma(dr, aih, bil, idn, 1u); tc_mma(dr, ail, bih, idn, 1u);
  tc_mma(di, arh, bih, idp, f); tc_mma(di, arh, bil, idp, 1u); tc_mma(di, arl, bih, idp, 1u);
  tc_mma(di, aih, brh, idp, 1u); tc_mma(di, aih, brl, idp, 1u); tc_mma(di, ail, brh, idp, 1u);
}

// four consecutive values along k of one complex operand row, split into the four planes (pl
// bytes apart) at byte offset off
__device__ __forceinline__ void jt_store4(unsigned char* buf, uint32_t pl, uint32_t off, const float2 (&v)[4]) {
  uint32_t p[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    tc_split(v[e].x, p[0][e], p[1][e]);
    tc_split(v[e].y, p[2][e], p[3][e]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<uint4*>(buf + q * pl + off) = make_uint4(p[q][0], p[q][1], p[q][2], p[q][3]);
}

__global__ void __launch_bounds__(256, 1)
    k_jacobi_tc(const JacD<float>* __restrict__ ds, int round, float tol, float tol_out, float negl2, int max_inner,
                unsigned long long* __restrict__ rows_updated) {
  constexpr int W = JT_W, LDG = JT_LDG;
  const JacD<float> d = ds[blockIdx.y];
  if (*d.done) return;
  if (round >= d.nblk - 1 || (int)blockIdx.x >= d.nblk / 2) return;
  extern __shared__ unsigned char jt_raw[];
  const uint32_t raw_s = tc_smem_u32(jt_raw);
  unsigned char* sm = jt_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  // shared memory: regions 0 and 1 (64 KB each), then the quarter region.  Gram: chunk plane
  // buffers in regions 0/1, quarter Grams after them.  Jacobi: G and V in regions 0-1.  Update: B =
  // V^T planes in the quarter region, the 128-row A chunk over regions 0-1.
  unsigned char* reg0 = sm;
  unsigned char* reg1 = sm + JT_REGION;
  float* Qg = reinterpret_cast<float*>(sm + 2 * JT_REGION);   // quarters q: Qg[q * 64 * LDQ + i * LDQ + j]
  float2* G = reinterpret_cast<float2*>(sm);                   // G[i * LDG + j] = x_i^* x_j
  float2* V = G + W * LDG;
  __shared__ int cidx[W];
  __shared__ float rc[W / 2];
  __shared__ float2 rse[W / 2];
  __shared__ int ract[W / 2], rpa[W / 2], rpb[W / 2];
  __shared__ int any_s, fail, skip, known;
  __shared__ float offw[8];
  __shared__ uint64_t mbar[5];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, quad = warp & 3;
  int I, J;
  rr_pair(blockIdx.x, round, d.nblk, I, J);
  const float floor2 = negl2 * (*d.amax);
  if (jac_known_orthogonal(d, I, J, (double)floor2, &known)) return;
  if (tid < W) {
    const int c = (tid < 32 ? I : J) * 32 + (tid & 31);
    cidx[tid] = c < d.k ? c : -1;
  }
  if (warp == 0) tc_alloc(&tslot, 256);
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) tc_bar_init(&mbar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
    skip = 0;
  }
  for (int e = tid; e < 4 * W * JT_LDQ; e += 256) Qg[e] = 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const int nch = (d.r + JT_CH - 1) / JT_CH;
  const int ngr = (nch + JT_GRP - 1) / JT_GRP;

  // ---- 1. Gram.  Unit e = tid + 256 q: column c = 8 (e >> 7) + (e & 7), chunk rows 4 kq .. 4 kq + 3
  //      with kq = (e >> 3) & 15 -- eight lanes fill one 8-row x 16-byte core matrix, so a warp's
  //      16-byte stores cover 512 contiguous bytes.  Re parts go to stacked rows c, Im to 64 + c.
  {
    float2 pa[4][4], pb[4][4];
    auto load_g = [&](int t, float2 (&pf)[4][4]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + 256 * q, c = 8 * (e >> 7) + (e & 7), r0 = t * JT_CH + 4 * ((e >> 3) & 15);
        const int col = cidx[c];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          pf[q][i] = (col >= 0 && r0 + i < d.r) ? d.X[(size_t)(r0 + i) + (size_t)col * d.ld] : make_float2(0.f, 0.f);
      }
    };
    auto store_g = [&](unsigned char* b, const float2 (&pf)[4][4]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = tid + 256 * q, c = 8 * (e >> 7) + (e & 7), kq = (e >> 3) & 15;
        uint32_t h[2][4], l[2][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          tc_split(pf[q][i].x, h[0][i], l[0][i]);
          tc_split(pf[q][i].y, h[1][i], l[1][i]);
        }
        const uint32_t ore = tc_kmajor(c, 4 * kq, JT_SBO), oim = tc_kmajor(64 + c, 4 * kq, JT_SBO);
        *reinterpret_cast<uint4*>(b + ore) = make_uint4(h[0][0], h[0][1], h[0][2], h[0][3]);
        *reinterpret_cast<uint4*>(b + JT_P128 + ore) = make_uint4(l[0][0], l[0][1], l[0][2], l[0][3]);
        *reinterpret_cast<uint4*>(b + oim) = make_uint4(h[1][0], h[1][1], h[1][2], h[1][3]);
        *reinterpret_cast<uint4*>(b + JT_P128 + oim) = make_uint4(l[1][0], l[1][1], l[1][2], l[1][3]);
      }
    };
    // chunk t accumulates into group (t / JT_GRP)'s accumulator; the group's last chunk commits
    auto mma_g = [&](unsigned char* b, int t) {
      if (tid == 0 && !fail) {
        tc_fence_after();
        const int g = t / JT_GRP;
        const bool first = t % JT_GRP == 0;
        const uint32_t hi = tc_smem_u32(b), lo = hi + JT_P128, dd = tmem + (uint32_t)(g & 1) * 128;
        const uint32_t id = tc_idesc(128, 128, false);
#pragma unroll
        for (int ks = 0; ks < JT_CH / 8; ++ks) {
          const uint64_t h = tc_desc(hi + (uint32_t)ks * 256, JT_SBO), l = tc_desc(lo + (uint32_t)ks * 256, JT_SBO);
          tc_mma(dd, h, h, id, (first && ks == 0) ? 0u : 1u);
          tc_mma(dd, h, l, id, 1u);
          tc_mma(dd, l, h, id, 1u);
        }
        // the buffer is free again once these MMAs are done; the group is done after its last chunk
        tc_commit(&mbar[t & 1]);
      }
    };
    // warp (quad, h = warp >> 2) adds rows 32 quad .. + 31, columns 64 h .. + 63 of group g's D
    // into quarter 2 (quad >= 2) + h: Re^T Re, Re^T Im, Im^T Re, Im^T Im (rows i = s mod 64)
    auto drain_g = [&](int g) {
      tc_fence_after();
      const int h = warp >> 2, i = (32 * quad + lane) & 63;
      float* dst = Qg + ((quad >= 2 ? 2 : 0) + h) * W * JT_LDQ + i * JT_LDQ;
      const uint32_t base = tmem + (uint32_t)(g & 1) * 128 + (uint32_t)(64 * h) + ((uint32_t)(32 * quad) << 16);
      for (int c0 = 0; c0 < W; c0 += 16) {
        uint32_t v[16];
        tc_ld16(base + (uint32_t)c0, v);
        tc_wait_ld();
        if (!fail) {
#pragma unroll
          for (int j = 0; j < 16; ++j) dst[c0 + j] += __uint_as_float(v[j]);
        }
      }
      tc_fence_before();
    };
    // Before storing chunk t into buffer t & 1, the MMAs of chunk t - 2 (its last reader) must be
    // done: wait for the (t - 2)-th completion of that buffer's barrier.  When chunk t - 1 closed
    // a group, that group is drained here, while chunk t's MMAs run.
    auto step_g = [&](int t, float2 (&pf)[4][4]) {
      if (t >= 2 && !fail && !tc_wait(&mbar[t & 1], (uint32_t)(((t - 2) >> 1) & 1))) atomicExch(&fail, 1);
      if (t < nch) {
        unsigned char* b = (t & 1) ? reg1 : reg0;
        store_g(b, pf);
        if (t + 2 < nch) load_g(t + 2, pf);
        tc_fence_async_smem();
      }
      __syncthreads();
      if (t < nch) mma_g((t & 1) ? reg1 : reg0, t);
      if (t >= 1 && ((t - 1) % JT_GRP == JT_GRP - 1 || t - 1 == nch - 1)) {
        // group (t - 1) / JT_GRP is complete once chunk t - 1's MMAs are
        const int u = t - 1;
        if (!fail && !tc_wait(&mbar[u & 1], (uint32_t)((u >> 1) & 1))) atomicExch(&fail, 1);
        drain_g(u / JT_GRP);
      }
      __syncthreads();
    };
    load_g(0, pa);
    if (nch > 1) load_g(1, pb);
    // chunk t's barrier parity: completion number t >> 1 of barrier t & 1.  A wait at step t for
    // chunk t - 2 and at step t + 1 for chunk t are both satisfied by the same completion count,
    // so barrier phases only ever advance.
    for (int t = 0; t <= nch; t += 2) {
      step_g(t, pa);
      if (t + 1 <= nch) step_g(t + 1, pb);
    }
    (void)ngr;
  }
  if (fail) goto cleanup;
  // G = (Re^T Re + Im^T Im) + i (Re^T Im - Im^T Re), in regions 0-1 (the plane buffers are done)
  for (int e = tid; e < W * W; e += 256) {
    const int i = e / W, j = e - i * W, o = i * JT_LDQ + j;
    G[i * LDG + j] = make_float2(Qg[o] + Qg[3 * W * JT_LDQ + o], Qg[W * JT_LDQ + o] - Qg[2 * W * JT_LDQ + o]);
  }
  __syncthreads();
  // ---- 2. largest cosine of the fresh Gram (columns above the noise floor only)
  {
    const int ti = tid >> 4, tj = tid & 15;
    float m = 0.f;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ti + 16 * p, j = tj + 16 * q;
        const float di = G[i * LDG + i].x, dj = G[j * LDG + j].x;
        if (i != j && di > floor2 && dj > floor2) {
          const float gg = sqrtf(abs2(G[i * LDG + j]));
          m = fmaxf(m, gg / (sqrtf(di) * sqrtf(dj)));
        }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) offw[warp] = m;
    __syncthreads();
    if (tid == 0) {
      float tt = 0.f;
      for (int w = 0; w < 8; ++w) tt = fmaxf(tt, offw[w]);
      if (tt > 0.f) atomicMax(d.off, __float_as_uint(tt));
      skip = tt <= tol_out;            // the pair is already orthogonal
      if (skip) jac_mark_orthogonal(d, I, J, (double)floor2);
    }
    __syncthreads();
    if (skip) goto cleanup;
  }
  // ---- 3. two-sided Jacobi on G, V <- V J for every rotation J
  jac_inner<float, W>(G, V, LDG, floor2, tol, max_inner, rc, rse, ract, rpa, rpb, &any_s);
  // ---- 4. X_P <- X_P V.  B = V^T planes in the quarter region: B(n, k) = V(k, n)
  {
    unsigned char* bpl = sm + 2 * JT_REGION;
    for (int e = tid; e < W * (W / 4); e += 256) {
      const int n = e >> 4, kq = e & 15;
      float2 v4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v4[i] = V[(4 * kq + i) * LDG + n];
      jt_store4(bpl, JT_P64, tc_kmajor(n, 4 * kq, JT_SBO), v4);
    }
    __syncthreads();   // V is read: regions 0-1 now take the A chunk
    const int ncu = (d.r + JT_CU - 1) / JT_CU;
    float2 pf[8][4];
    // A: unit e = tid + 256 q stages row m = e % 128 of the chunk, columns 4 (e / 128) .. + 3
    auto load_u = [&](int t) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = tid + 256 * q, m = e & 127, cq = e >> 7, row = t * JT_CU + m;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int col = cidx[4 * cq + i];
          pf[q][i] = (col >= 0 && row < d.r) ? d.X[(size_t)row + (size_t)col * d.ld] : make_float2(0.f, 0.f);
        }
      }
    };
    auto mma_u = [&](int t) {
      if (tid == 0 && !fail) {
        tc_fence_after();
        const uint32_t a = tc_smem_u32(sm), bb = tc_smem_u32(bpl), dd = tmem + (uint32_t)(t & 1) * 128;
        const uint32_t idp = tc_idesc(128, 64, false), idn = tc_idesc(128, 64, true);
#pragma unroll
        for (int ks = 0; ks < W / 8; ++ks)
          jt_mma12(dd, dd + 64, a, JT_P128, bb, (uint32_t)ks * 256, ks == 0 ? 0u : 1u, idp, idn);
        tc_commit(&mbar[2 + (t & 1)]);
      }
    };
    // warp (quad, h = warp >> 2): rows 32 quad + lane of chunk u, output columns 32 h .. + 31
    auto drain_u = [&](int u) {
      if (!fail && !tc_wait(&mbar[2 + (u & 1)], (uint32_t)((u >> 1) & 1))) atomicExch(&fail, 1);
      tc_fence_after();
      const int n0 = 32 * (warp >> 2), row = u * JT_CU + 32 * quad + lane;
      for (int c0 = 0; c0 < 32; c0 += 16) {
        uint32_t vr[16], vi[16];
        const uint32_t la = tmem + (uint32_t)(u & 1) * 128 + ((uint32_t)(32 * quad) << 16) + (uint32_t)(n0 + c0);
        tc_ld16(la, vr);
        tc_ld16(la + 64, vi);
        tc_wait_ld();
        if (row < d.r && !fail) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = cidx[n0 + c0 + j];
            if (col >= 0) d.X[(size_t)row + (size_t)col * d.ld] = make_float2(__uint_as_float(vr[j]), __uint_as_float(vi[j]));
          }
        }
      }
      tc_fence_before();
    };
    load_u(0);
    for (int t = 0; t <= ncu; ++t) {
      if (t < ncu) {
        // the single A buffer: chunk t - 1's MMAs must be done before it is overwritten
        if (t >= 1 && !fail && !tc_wait(&mbar[2 + ((t - 1) & 1)], (uint32_t)(((t - 1) >> 1) & 1))) atomicExch(&fail, 1);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = tid + 256 * q;
          jt_store4(sm, JT_P128, tc_kmajor(e & 127, 4 * (e >> 7), JT_SBO), pf[q]);
        }
        if (t + 1 < ncu) load_u(t + 1);   // rows of the next chunk: disjoint from the ones written below
        tc_fence_async_smem();
      }
      __syncthreads();
      if (t < ncu) mma_u(t);
      if (t >= 1) drain_u(t - 1);   // overlaps chunk t's MMAs (the other accumulator)
      __syncthreads();
    }
  }
  if (tid == 0 && !fail) {
    atomicAdd(rows_updated, (unsigned long long)d.r);
    jac_mark_rotated(d, I, J);
  }
cleanup:
  if (tid == 0) {
    if (fail) atomicExch(&g_jac_error, 1);
    tc_commit(&mbar[4]);                // MMAs still in flight after a failed wait finish first
    tc_wait(&mbar[4], 0u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 256);
}

int jacobi_tc_error(bool reset) {
  int v = 0;
  NH_CK(cudaMemcpyFromSymbol(&v, g_jac_error, sizeof(int)));
  if (reset && v) {
    const int z = 0;
    NH_CK(cudaMemcpyToSymbol(g_jac_error, &z, sizeof(int)));
  }
  return v;
}

// sigma_j = ||x_j||; rank positions by counting (descending, ties by index); count retained.
template <typename R> struct SortD {
  const cplx<R>* X; int ld, r, k;
  R* sig;       // k: sorted descending
  int* order;   // k: column index of the i-th largest
  int* rank;    // out: number with sigma > eps * sigma_max
};

template <typename R>
__global__ void __launch_bounds__(256) k_svd_sort(const SortD<R>* __restrict__ ds, R eps) {
  const SortD<R> d = ds[blockIdx.x];
  extern __shared__ unsigned char smraw[];
  R* s = (R*)smraw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < d.k; j += 8) {
    R acc = 0;
    for (int i = lane; i < d.r; i += 32) acc += abs2(d.X[(size_t)i + (size_t)j * d.ld]);
    acc = warp_sum(acc);
    if (lane == 0) s[j] = sqrt(acc);
  }
  __syncthreads();
  R smax = 0;
  for (int j = 0; j < d.k; ++j) smax = fmax(smax, s[j]);
  int cnt = 0;
  for (int j = threadIdx.x; j < d.k; j += 256) {
    const R v = s[j];
    int pos = 0;
    for (int l = 0; l < d.k; ++l) {
      const R w = s[l];
      pos += (w > v) || (w == v && l < j);
    }
    d.sig[pos] = v;
    d.order[pos] = j;
    cnt += (v > eps * smax && v > R(0));
  }
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  atomicAdd(&tot, cnt);
  __syncthreads();
  if (threadIdx.x == 0) *d.rank = tot;
}

// P(:, i) = X(:, order[i]) / sig[i], i < rank
template <typename R> struct SelD {
  const cplx<R>* X; int ld, r; const R* sig; const int* order; cplx<R>* P; int ldp, rank;
  const int* rowperm;   // P(rowperm[t], i) = X(t, order[i]) / sig[i]
};

template <typename R> __global__ void k_svd_select(const SelD<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob(pre, np, blockIdx.x);
  const SelD<R> d = ds[pi];
  const int i = blockIdx.x - pre[pi];   // one CTA per selected column
  const int c = d.order[i];
  const R inv = R(1) / d.sig[i];
  for (int t = threadIdx.x; t < d.r; t += blockDim.x) {
    const int row = d.rowperm ? d.rowperm[t] : t;
    d.P[(size_t)row + (size_t)i * d.ldp] = inv * d.X[(size_t)t + (size_t)c * d.ld];
  }
}

// |R_kk| of the pivoted QR (one thread per diagonal entry).
template <typename R> __global__ void k_rdiag(const QpD<R>* __restrict__ ds, R* const* __restrict__ out) {
  const QpD<R> d = ds[blockIdx.y];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < min(d.m, d.n)) out[blockIdx.y][k] = sqrt(abs2(d.A[(size_t)k + (size_t)k * d.lda]));
}

template <typename R>
void Ops<R>::tsvd_ct(const std::vector<Mat<R>>& Ct, double eps, Arena& keep, std::vector<Mat<R>>& P,
                     std::vector<std::vector<double>>& S) {
  const size_t nm = Ct.size();
  P.assign(nm, Mat<R>());
  S.assign(nm, {});
  auto mk = ar_->mark();
  // 0. tall inputs (w well above r): unpivoted blocked Householder QR first.  Ct = Q0 R0 with
  //    R0 (r x r) in the top block of Ct; the pivoted QR below then runs on R0, which has the
  //    same column norms, pivots and R as Ct (Q0 has orthonormal columns), at r/w of the cost.
  std::vector<Mat<R>> Cw(Ct.begin(), Ct.end());
  {
    std::vector<Mat<R>> tall;
    std::vector<size_t> ti;
    for (size_t i = 0; i < nm; ++i)
      if (Ct[i].n >= 64 && (long long)Ct[i].m * 4 > (long long)Ct[i].n * 5) {
        tall.push_back(Ct[i]);
        ti.push_back(i);
      }
    if (!tall.empty()) {
      qr(tall, *ar_);   // factors are not kept: only R0 (zero below the diagonal) is needed
      for (size_t q = 0; q < ti.size(); ++q) Cw[ti[q]].m = Cw[ti[q]].n;
    }
  }
  // 1. pivoted QR of Ct (w x r): Ct Pi = Q R, R (p x r), p = min(w, r).  Then
  //    C = Pi R^* Q^*, so the left singular vectors of C are Pi times those of R^*.
  //    Default: pivots chosen blockwise on random sketches (qrcp_sketch), which also stops at the
  //    pre-truncation rank; NH_QRCP=exact runs the classical one-pivot-per-step form below.
  std::vector<int*> perms(nm, nullptr);
  std::vector<int> peff(nm, 0);
  const char* qe = std::getenv("NH_QRCP");
  if (!(qe && !std::strcmp(qe, "exact"))) {
    for (size_t i = 0; i < nm; ++i) perms[i] = ar_->template arr<int>(std::max(Cw[i].n, 1));
    qrcp_sketch(Cw, perms, eps, peff);
    for (size_t i = 0; i < nm; ++i) {
      const int p = std::min(Cw[i].m, Cw[i].n);
      peff[i] = std::max(peff[i], std::min(2, p));
    }
  } else {
    std::vector<QpD<R>> qp;
    int pmax = 0, nmax = 0;
    for (size_t i = 0; i < nm; ++i) {
      const int w = Cw[i].m, r = Cw[i].n;
      perms[i] = ar_->template arr<int>(std::max(r, 1));
      if (w <= 0 || r <= 0) continue;
      QpD<R> q;
      q.A = Cw[i].p; q.lda = Cw[i].ld; q.m = w; q.n = r;
      q.perm = perms[i];
      q.vn1 = ar_->template arr<R>(r);
      q.vn2 = ar_->template arr<R>(r);
      q.v = ar_->template arr<cplx<R>>(w);
      q.tau = ar_->template arr<R>(1);
      qp.push_back(q);
      pmax = std::max(pmax, std::min(w, r));
      nmax = std::max(nmax, r);
    }
    if (!qp.empty()) {
      auto dq = upload(qp);
      const R tol3z = (R)std::sqrt(sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08);
      dim3 gi((nmax + 7) / 8, (unsigned)qp.size());
      k_qp_init<R><<<gi, 256, 0, st_>>>(dq);
      NH_LAUNCH_CK();
      count();
      double fl = 0;
      if (prof.on)
        for (auto& q : qp) fl += 8.0 * (double)q.m * q.n * std::min(q.m, q.n);
      prof.begin(st_);
      int mmax = 0;
      for (auto& q : qp) mmax = std::max(mmax, q.m);
      for (int k = 0; k < pmax; ++k) {
        k_qp_pivot<R><<<(int)qp.size(), 256, 0, st_>>>(dq, k);
        NH_LAUNCH_CK();
        const int cols = nmax - k - 1, rows = mmax - k;
        if (cols > 0) {
          dim3 gc((unsigned)cols, (unsigned)qp.size());
          if (rows <= 256 * 4) k_qp_update_cta<R, 4><<<gc, 256, 0, st_>>>(dq, k, tol3z);
          else if (rows <= 256 * 8) k_qp_update_cta<R, 8><<<gc, 256, 0, st_>>>(dq, k, tol3z);
          else if (rows <= 256 * 16) k_qp_update_cta<R, 16><<<gc, 256, 0, st_>>>(dq, k, tol3z);
          else if (rows <= 256 * 32) k_qp_update_cta<R, 32><<<gc, 256, 0, st_>>>(dq, k, tol3z);
          else k_qp_update<R><<<dim3((cols + 7) / 8, (unsigned)qp.size()), 256, 0, st_>>>(dq, k, tol3z);
          NH_LAUNCH_CK();
        }
        count(2);
      }
      prof.end(st_, K_QRCP, fl, 0, 2 * pmax);
    }
    // 1b. pre-truncation: the pivoted QR reveals the rank, so rows of R with |R_kk| two decades
    //     below the truncation threshold (and the trailing block under them) are dropped before
    //     the Jacobi sweeps; they cannot reach the retained singular values.
    {
      std::vector<R*> dgp;
      std::vector<int> pq;
      int pm = 0;
      for (size_t i = 0, q = 0; i < nm; ++i) {
        const int w = Cw[i].m, r = Cw[i].n;
        peff[i] = std::min(w, r);
        if (w <= 0 || r <= 0) continue;
        dgp.push_back(ar_->template arr<R>(peff[i]));
        pq.push_back((int)i);
        pm = std::max(pm, peff[i]);
        (void)q;
      }
      if (!dgp.empty()) {
        auto dq = upload(qp);
        auto dd = upload(dgp);
        dim3 g((pm + 255) / 256, (unsigned)qp.size());
        k_rdiag<R><<<g, 256, 0, st_>>>(dq, dd);
        NH_LAUNCH_CK();
        count();
        std::vector<std::vector<R>> hd(dgp.size());
        for (size_t q = 0; q < dgp.size(); ++q) {
          hd[q].resize(peff[pq[q]]);
          NH_CK(cudaMemcpyAsync(hd[q].data(), dgp[q], hd[q].size() * sizeof(R), cudaMemcpyDeviceToHost, st_));
        }
        NH_CK(cudaStreamSynchronize(st_));
        for (size_t q = 0; q < dgp.size(); ++q) {
          R mx = 0;
          for (R v : hd[q]) mx = std::max(mx, v);
          const double cut = 0.01 * eps * (double)mx;
          int k = 0;   // keep through the last row above the cut (|R_kk| is only roughly monotone)
          for (int j = 0; j < (int)hd[q].size(); ++j)
            if ((double)hd[q][j] > cut) k = j + 1;
          peff[pq[q]] = std::max(k, std::min(2, (int)hd[q].size()));
        }
      }
    }
  }
  // 2. X = R^* (r x p) (the pivoted QR zeroes the part below the diagonal)
  std::vector<Mat<R>> X(nm);
  std::vector<CopyD<R>> cp;
  for (size_t i = 0; i < nm; ++i) {
    const int w = Cw[i].m, r = Cw[i].n, p = std::min(peff[i], std::min(w, r));
    X[i] = ar_->template mat<R>(r, p);
    if (r > 0 && p > 0) cp.push_back({Cw[i].p, X[i].p, r, p, Cw[i].ld, X[i].ld, OP_C, R(1), R(0)});
  }
  copy(cp);
  // 3. Jacobi sweeps
  std::vector<JacD<R>> jd;
  std::vector<int> jmap;
  unsigned* offs = ar_->template arr<unsigned>(nm + 1);
  int* done = ar_->template arr<int>(nm + 1, true);
  R* amaxv = ar_->template arr<R>(nm + 1, true);
  // Ordering: block pairs in round-robin order.  Matrices with many rows use the blocked
  // (Gram) step on pairs of 32-column blocks; small ones the scalar rotations on pairs of
  // 16-column blocks, where the Gram step's fixed cost would dominate.
  int rmax_all = 0;
  for (size_t i = 0; i < nm; ++i)
    if (X[i].n >= 2) rmax_all = std::max(rmax_all, X[i].m);
  enum { J_SCALAR, J_CLUSTER, J_BLOCK } jmode = rmax_all >= 512 ? J_BLOCK : J_SCALAR;
  if (const char* e = std::getenv("NH_JACOBI_MODE")) {
    if (!std::strcmp(e, "scalar")) jmode = J_SCALAR;
    else if (!std::strcmp(e, "cluster")) jmode = J_CLUSTER;
    else if (!std::strcmp(e, "block")) jmode = J_BLOCK;
  }
  const int bw = jmode == J_BLOCK ? 32 : 16;
  int maxblk = 0;
  for (size_t i = 0; i < nm; ++i) {
    const int p = X[i].n;
    if (p < 2 || X[i].m == 0) continue;
    int nb = (p + bw - 1) / bw;
    if (nb < 2) nb = 2;
    if (nb & 1) nb++;
    jd.push_back({X[i].p, X[i].ld, X[i].m, p, nb, offs + i, done + i, amaxv + i, nullptr, nullptr});
    if (jmode == J_BLOCK) {
      jd.back().ver = ar_->template arr<unsigned>(nb, true);
      jd.back().seen = ar_->template arr<JacSeen>((size_t)nb * nb);
      NH_CK(cudaMemsetAsync(jd.back().seen, 0xFF, (size_t)nb * nb * sizeof(JacSeen), st_));
    }
    jmap.push_back((int)i);
    maxblk = std::max(maxblk, nb);
  }
  unsigned long long* rows_upd = ar_->template arr<unsigned long long>(1, true);
  bool jtc = false;   // FP32 blocked steps run their Gram and update products on the tensor cores
  const double u = sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
  if (!jd.empty()) {
    auto djd = upload(jd);
    std::vector<unsigned> hoff(nm);
    std::vector<int> hdone(nm, 0);
    int rmax = 0;
    for (auto& j : jd) rmax = std::max(rmax, j.r);
    const R tol = (R)(4.0 * u * std::sqrt((double)std::max(rmax, 1)));
    // Large matrices: cluster-resident rounds (the 32 columns of a block pair stay in shared
    // memory, split by rows over 8 or 16 CTAs).  Small ones: global-memory rounds.
    int JCS = 8;
    if ((size_t)32 * ((rmax + 7) / 8) * sizeof(cplx<R>) > (size_t)200 * 1024) JCS = 16;
    const int rpc = (rmax + JCS - 1) / JCS;
    const size_t jsmem = (size_t)32 * rpc * sizeof(cplx<R>);
    if (jmode == J_CLUSTER && jsmem > (size_t)200 * 1024) jmode = J_SCALAR;
    const bool use_cluster = jmode == J_CLUSTER;
    if constexpr (sizeof(R) == 4) jtc = jmode == J_BLOCK && gemm_tc_enabled();
    if (jtc)
      NH_CK(cudaFuncSetAttribute(k_jacobi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JT_SMEM));
    else if (jmode == J_BLOCK)
      NH_CK(cudaFuncSetAttribute(k_jacobi_blk<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JbCfg<R>::smem));
    if (use_cluster) {
      NH_CK(cudaFuncSetAttribute(k_jacobi_cluster<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(jsmem, 1)));
      if (JCS > 8) NH_CK(cudaFuncSetAttribute(k_jacobi_cluster<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    // columns with norm <= delta * (largest column norm) are numerically zero; delta sits well
    // below the truncation threshold eps so no retained direction is affected
    const double delta = 0.1 * eps;
    const R negl2 = (R)(delta * delta);
    // sweeps end when no pair's cosine exceeds tol_out (blocked steps: twice the rotation threshold)
    const R tol_out = jmode == J_BLOCK ? R(2) * tol : tol;
    for (int sweep = 0; sweep < 40; ++sweep) {
      NH_CK(cudaMemsetAsync(offs, 0, nm * sizeof(unsigned), st_));
      k_colmax<R><<<(int)jd.size(), 256, 0, st_>>>(djd);
      NH_LAUNCH_CK();
      count();
      double fl = 0;
      if (prof.on)
        for (size_t q = 0; q < jd.size(); ++q) {
          if (hdone[jmap[q]]) continue;
          if (jmode == J_BLOCK)   // Gram of every block pair: 8 W^2 flops per row
            fl += 8.0 * JbCfg<R>::W * JbCfg<R>::W * jd[q].r * (double)(jd[q].nblk / 2) * (jd[q].nblk - 1);
          else
            fl += 40.0 * jd[q].r * ((double)jd[q].k * (jd[q].k - 1) / 2.0);
        }
      prof.begin(st_);
      for (int rd = 0; rd < maxblk - 1; ++rd) {
        if (jmode == J_BLOCK) {
          dim3 grid(maxblk / 2, (unsigned)jd.size());
          if constexpr (sizeof(R) == 4) {
            if (jtc) k_jacobi_tc<<<grid, 256, JT_SMEM, st_>>>(djd, rd, tol, tol_out, negl2, 16, rows_upd);
            else k_jacobi_blk<R><<<grid, 256, JbCfg<R>::smem, st_>>>(djd, rd, tol, tol_out, negl2, 16, rows_upd);
          } else {
            k_jacobi_blk<R><<<grid, 256, JbCfg<R>::smem, st_>>>(djd, rd, tol, tol_out, negl2, 16, rows_upd);
          }
          NH_LAUNCH_CK();
        } else if (use_cluster) {
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3((unsigned)(maxblk / 2 * JCS), (unsigned)jd.size());
          cfg.blockDim = dim3(512);
          cfg.dynamicSmemBytes = jsmem;
          cfg.stream = st_;
          cudaLaunchAttribute at[1];
          at[0].id = cudaLaunchAttributeClusterDimension;
          at[0].val.clusterDim.x = JCS;
          at[0].val.clusterDim.y = 1;
          at[0].val.clusterDim.z = 1;
          cfg.attrs = at;
          cfg.numAttrs = 1;
          NH_CK(cudaLaunchKernelEx(&cfg, k_jacobi_cluster<R>, (const JacD<R>*)djd, rd, tol, rpc, negl2));
        } else {
          dim3 grid(maxblk / 2, (unsigned)jd.size());
          k_jacobi_round<R><<<grid, 512, 0, st_>>>(djd, rd, tol, negl2);
          NH_LAUNCH_CK();
        }
        count();
      }
      prof.end(st_, jtc ? K_JACOBI_TC : K_JACOBI, fl, 0, maxblk - 1);
      NH_CK(cudaMemcpyAsync(hoff.data(), offs, nm * sizeof(unsigned), cudaMemcpyDeviceToHost, st_));
      NH_CK(cudaStreamSynchronize(st_));
      bool all = true;
      for (size_t q = 0; q < jd.size(); ++q) {
        const int i = jmap[q];
        if (hdone[i]) continue;
        float f;
        std::memcpy(&f, &hoff[i], 4);
        if ((double)f <= (double)tol_out) hdone[i] = 1; else all = false;
      }
      NH_CK(cudaMemcpyAsync(done, hdone.data(), nm * sizeof(int), cudaMemcpyHostToDevice, st_));
      if (all || sweep == 39) {
        break;
      }
    }
  }
  if constexpr (sizeof(R) == 4) {
    if (jmode == J_BLOCK && !jd.empty() && gemm_tc_enabled() && jacobi_tc_error(true))
      throw Error(ST_ETIMEOUT, "tsvd: a bounded wait of the tensor-core Jacobi step ran out");
  }
  if (prof.on && jmode == J_BLOCK && !jd.empty()) {   // X_P V of the block pairs that rotated
    unsigned long long ru = 0;
    NH_CK(cudaMemcpyAsync(&ru, rows_upd, sizeof(ru), cudaMemcpyDeviceToHost, st_));
    NH_CK(cudaStreamSynchronize(st_));
    prof.add_flops(jtc ? K_JACOBI_TC : K_JACOBI, 8.0 * JbCfg<R>::W * JbCfg<R>::W * (double)ru);
  }
  // 4. sort + count
  std::vector<SortD<R>> sd;
  int* ranks = ar_->template arr<int>(nm + 1, true);
  std::vector<R*> sig(nm, nullptr);
  std::vector<int*> order(nm, nullptr);
  int kmax = 1;
  for (size_t i = 0; i < nm; ++i) {
    const int p = X[i].n;
    sig[i] = ar_->template arr<R>(std::max(p, 1));
    order[i] = ar_->template arr<int>(std::max(p, 1));
    if (p > 0 && X[i].m > 0) {
      sd.push_back({X[i].p, X[i].ld, X[i].m, p, sig[i], order[i], ranks + i});
      kmax = std::max(kmax, p);
    }
  }
  if (!sd.empty()) {
    auto dsd = upload(sd);
    const size_t smem = (size_t)kmax * sizeof(R);
    if (smem > 48 * 1024)
      NH_CK(cudaFuncSetAttribute(k_svd_sort<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_svd_sort<R><<<(int)sd.size(), 256, smem, st_>>>(dsd, (R)eps);
    NH_LAUNCH_CK();
    count();
  }
  std::vector<int> hr(nm, 0);
  NH_CK(cudaMemcpyAsync(hr.data(), ranks, nm * sizeof(int), cudaMemcpyDeviceToHost, st_));
  NH_CK(cudaStreamSynchronize(st_));
  // 5. select
  std::vector<SelD<R>> sel;
  std::vector<int> pre;
  int tot = 0;
  std::vector<std::vector<R>> hs(nm);
  for (size_t i = 0; i < nm; ++i) {
    const int r = X[i].m;
    const int rk = (X[i].n > 0 && r > 0) ? hr[i] : 0;
    P[i] = keep.template mat<R>(r, rk);
    if (rk > 0) {
      sel.push_back({X[i].p, X[i].ld, r, sig[i], order[i], P[i].p, P[i].ld, rk, perms[i]});
      pre.push_back(tot);
      tot += rk;
      hs[i].resize(rk);
      NH_CK(cudaMemcpyAsync(hs[i].data(), sig[i], rk * sizeof(R), cudaMemcpyDeviceToHost, st_));
    }
  }
  if (!sel.empty()) {
    auto dsel = upload(sel);
    int* dp = upload_ints(pre);
    k_svd_select<R><<<tot, 256, 0, st_>>>(dsel, dp, (int)sel.size());
    NH_LAUNCH_CK();
    count();
  }
  NH_CK(cudaStreamSynchronize(st_));
  for (size_t i = 0; i < nm; ++i) S[i].assign(hs[i].begin(), hs[i].end());
  ar_->release(mk);
}

void gemm_launch_raw(const GemmD<double>* desc, const int* pre, int np, int tiles, cudaStream_t st) {
  if (tiles <= 0) return;
  launch_gemm<double, GemmCfg<double>::TM, GemmCfg<double>::TN, GemmCfg<double>::BK>(0, tiles, st, desc, pre, np,
                                                                                     nullptr, nullptr);
}

int gemm_tiles(const GemmD<double>& g) {
  constexpr int BM = 16 * GemmCfg<double>::TM, BN = 16 * GemmCfg<double>::TN;
  return ((g.m + BM - 1) / BM) * ((g.n + BN - 1) / BN);
}

template class Ops<double>;
template class Ops<float>;

}  // namespace nh
