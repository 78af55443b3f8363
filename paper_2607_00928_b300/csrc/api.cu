// C-ABI of the solver (include/nudft2_hss.h): argument checking, the exact FP64 apply,
// the 2D inverse DFT, mixed-precision iterative refinement, and dispatch to Hss<R>.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/nudft2_hss.h"
#include "hss.cuh"
#include "retry.h"

using namespace nh;

// factor store file: "NUDF" "T2HS" (ASCII, little-endian words), then the version
constexpr uint32_t STORE_MAGIC0 = 0x4644554Eu, STORE_MAGIC1 = 0x53483254u, STORE_VERSION = 1u;
thread_local std::string nudft2_err_tls;
#define g_err nudft2_err_tls

// One captured URV solve (Sec. 2.3 sweeps) for a fixed number of right-hand sides: fixed
// input/output buffers, the instantiated graph and the pinned descriptor copies it reads.
template <typename R> struct SolveGraph {
  cplx<R>* f2 = nullptr;
  cplx<R>* yt = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t kernels = 0;              // kernel nodes in the graph (for launch accounting)
  bool failed = false;
  PinnedPool pool;
  ~SolveGraph() { if (exec) cudaGraphExecDestroy(exec); }
};

struct nudft2_hss_s {
  nudft2_opts opt{};
  int M = 0, nx = 0, ny = 0, L = 0, N = 0;
  cudaStream_t st = 0;             // handle-owned stream (capturable); callers' streams are joined by events
  cudaEvent_t join = nullptr;
  std::map<int, std::unique_ptr<SolveGraph<double>>> g64;
  std::map<int, std::unique_ptr<SolveGraph<float>>> g32;
  Arena keep{(size_t)64 << 20, true};
  Arena scr{(size_t)256 << 20};
  Plan pl;
  std::unique_ptr<Hss<double>> h64;
  std::unique_ptr<Hss<float>> h32;
  std::unique_ptr<Ops<double>> ops;
  double2 *Ax = nullptr, *Ay = nullptr;              // exp(-2 pi i k x_j), caller order
  float2 *Ax32 = nullptr, *Ay32 = nullptr;           // the same in FP32 (MIXED: correction applies)
  double2 *Fxi = nullptr, *Fyi = nullptr;            // inverse DFT matrices (1/n included)
  double2 *Fxf = nullptr, *Fyf = nullptr;            // forward DFT matrices
  bool factored = false;
  int graphs_ok = 0, graphs_failed = 0, replays = 0;
  double t_build = 0, t_factor = 0, t_solve = 0, relres = 0;
  int iters = 0;
};

template <typename F> static nudft2_status guard(F&& f) {
  try {
    f();
    g_err.clear();
    return NUDFT2_OK;
  } catch (Error& e) {
    g_err = e.what();
    return (nudft2_status)e.code;
  } catch (std::exception& e) {
    g_err = e.what();
    return NUDFT2_ECUDA;
  }
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static GemmD<double> g64(const double2* A, int lda, int opA, const double2* B, int ldb, int opB, double2* C, int ldc,
                         int m, int n, int k, double alpha = 1.0, double beta = 0.0) {
  return GemmD<double>{A, B, C, m, n, k, lda, ldb, ldc, opA, opB, alpha, beta};
}

// ----------------------------------------------------------------------------- exact apply (Eq. 1)
// Twiddle tables Ax(j,k) = exp(-2 pi i k x_j) (M x nx), Ay (M x ny), caller point order.
struct Exact {
  int M, nx, ny;
  const double2 *Ax, *Ay;
};

// f_j = sum_kx Ax(j,kx) sum_ky Ay(j,ky) c(kx,ky): inner sum as a GEMM Ay * C (C viewed ny x nx).
static void exact_fwd_impl(Ops<double>& ops, Arena& scr, cudaStream_t st, const Exact& e, const double2* c,
                           int64_t ldc, int s, double2* f, int64_t ldf) {
  const int M = e.M, nx = e.nx, ny = e.ny, N = nx * ny;
  const int sc = std::max(1, std::min(s, (int)std::max<int64_t>(1, ((int64_t)1 << 31) / ((int64_t)M * nx * 16))));
  auto mk = scr.mark();
  double2* T = scr.arr<double2>((size_t)M * nx * sc);
  double2* Cc = (ldc == N) ? nullptr : scr.arr<double2>((size_t)N * sc);
  for (int q0 = 0; q0 < s; q0 += sc) {
    const int qs = std::min(sc, s - q0);
    const double2* C = c + (size_t)q0 * ldc;
    if (Cc) {
      NH_CK(cudaMemcpy2DAsync(Cc, N * sizeof(double2), C, ldc * sizeof(double2), N * sizeof(double2), qs,
                              cudaMemcpyDeviceToDevice, st));
      C = Cc;
    }
    ops.gemm({GemmD<double>{e.Ay, C, T, M, nx * qs, ny, M, ny, M, OP_N, OP_N, 1.0, 0.0}});
    rowdot(st, e.Ax, M, T, M, M, nx, qs, f + (size_t)q0 * ldf, (int)ldf);
    ops.count();
  }
  scr.release(mk);
}

// (A^* f)(kx, ky) = sum_j conj(Ay(j,ky)) * (f_j conj(Ax(j,kx))): GEMM Ay^* Z, Z = f o conj(Ax).
static void exact_adj_impl(Ops<double>& ops, Arena& scr, cudaStream_t st, const Exact& e, const double2* f,
                           int64_t ldf, int s, double2* out, int64_t ldo) {
  const int M = e.M, nx = e.nx, ny = e.ny, N = nx * ny;
  const int sc = std::max(1, std::min(s, (int)std::max<int64_t>(1, ((int64_t)1 << 31) / ((int64_t)M * nx * 16))));
  auto mk = scr.mark();
  double2* Z = scr.arr<double2>((size_t)M * nx * sc);
  double2* Oc = (ldo == N) ? nullptr : scr.arr<double2>((size_t)N * sc);
  for (int q0 = 0; q0 < s; q0 += sc) {
    const int qs = std::min(sc, s - q0);
    scale_rows_conj_multi(st, e.Ax, M, f + (size_t)q0 * ldf, (int)ldf, M, nx, qs, Z, M);
    ops.count();
    double2* O = Oc ? Oc : out + (size_t)q0 * ldo;
    ops.gemm({GemmD<double>{e.Ay, Z, O, ny, nx * qs, M, M, M, ny, OP_C, OP_N, 1.0, 0.0}});
    if (Oc)
      NH_CK(cudaMemcpy2DAsync(out + (size_t)q0 * ldo, ldo * sizeof(double2), Oc, N * sizeof(double2),
                              N * sizeof(double2), qs, cudaMemcpyDeviceToDevice, st));
  }
  scr.release(mk);
}

// r -= A d in FP32 arithmetic (tables, products and sums in FP32 on the tensor-core GEMM path;
// the subtraction in FP64).  Used for the refinement residual after its first step, where d is
// a correction of size O(eps) ||c||, so its FP32 rounding is O(eps u_32) ||f|| (see do_solve).
static void exact_fwd_sub32(nudft2_hss_s* h, const double2* d, int64_t ldd, int s, double2* r, int64_t ldr) {
  const int M = h->M, nx = h->nx, ny = h->ny, N = h->N;
  Ops<float>& ops = h->h32->ops();
  const int sc = std::max(1, std::min(s, (int)std::max<int64_t>(1, ((int64_t)1 << 31) / ((int64_t)M * nx * 8))));
  auto mk = h->scr.mark();
  float2* T = h->scr.arr<float2>((size_t)M * nx * sc);
  float2* C = h->scr.arr<float2>((size_t)N * sc);
  for (int q0 = 0; q0 < s; q0 += sc) {
    const int qs = std::min(sc, s - q0);
    convert_gather<double, float>(h->st, d + (size_t)q0 * ldd, (int)ldd, nullptr, N, qs, C, N, 1.0);
    ops.gemm({GemmD<float>{h->Ay32, C, T, M, nx * qs, ny, M, ny, M, OP_N, OP_N, 1.f, 0.f}});
    rowdot_sub32(h->st, h->Ax32, M, T, M, M, nx, qs, r + (size_t)q0 * ldr, (int)ldr);
    ops.count(2);
  }
  h->scr.release(mk);
}

// out -= A^* e in FP32 arithmetic, the adjoint counterpart of exact_fwd_sub32.
static void exact_adj_sub32(nudft2_hss_s* h, const double2* e, int64_t lde, int s, double2* out, int64_t ldo) {
  const int M = h->M, nx = h->nx, ny = h->ny, N = h->N;
  Ops<float>& ops = h->h32->ops();
  const int sc = std::max(1, std::min(s, (int)std::max<int64_t>(1, ((int64_t)1 << 31) / ((int64_t)M * nx * 8))));
  auto mk = h->scr.mark();
  float2* Z = h->scr.arr<float2>((size_t)M * nx * sc);
  float2* O = h->scr.arr<float2>((size_t)N * sc);
  double2* O64 = h->scr.arr<double2>((size_t)N * sc);
  for (int q0 = 0; q0 < s; q0 += sc) {
    const int qs = std::min(sc, s - q0);
    scale_rows_conj32(h->st, h->Ax32, M, e + (size_t)q0 * lde, (int)lde, M, nx, qs, Z, M);
    ops.gemm({GemmD<float>{h->Ay32, Z, O, ny, nx * qs, M, M, M, ny, OP_C, OP_N, 1.f, 0.f}});
    convert_gather<float, double>(h->st, O, N, nullptr, N, qs, O64, N, 1.0);
    axpy2(h->st, N, qs, -1.0, O64, N, out + (size_t)q0 * ldo, (int)ldo);
    ops.count(3);
  }
  h->scr.release(mk);
}

static void exact_fwd(nudft2_hss_s* h, const double2* c, int64_t ldc, int s, double2* f, int64_t ldf) {
  exact_fwd_impl(*h->ops, h->scr, h->st, Exact{h->M, h->nx, h->ny, h->Ax, h->Ay}, c, ldc, s, f, ldf);
}
static void exact_adj(nudft2_hss_s* h, const double2* f, int64_t ldf, int s, double2* out, int64_t ldo) {
  exact_adj_impl(*h->ops, h->scr, h->st, Exact{h->M, h->nx, h->ny, h->Ax, h->Ay}, f, ldf, s, out, ldo);
}

// c = F^{-1} y per column: C = Fy^{-1} Y Fx^{-1} with Y viewed ny x nx (lexicographic order)
static void dft2(nudft2_hss_s* h, const double2* y, int64_t ldy, int s, double2* c, int64_t ldc, bool inverse,
                 double scale = 1.0) {
  const int nx = h->nx, ny = h->ny;
  auto mk = h->scr.mark();
  double2* T = h->scr.arr<double2>((size_t)h->N * s);
  std::vector<GemmD<double>> g1, g2;
  const double2* Fy = inverse ? h->Fyi : h->Fyf;
  const double2* Fx = inverse ? h->Fxi : h->Fxf;
  for (int q = 0; q < s; ++q) {
    g1.push_back(g64(Fy, ny, OP_N, y + (size_t)q * ldy, ny, OP_N, T + (size_t)q * h->N, ny, ny, nx, ny));
    g2.push_back(g64(T + (size_t)q * h->N, ny, OP_N, Fx, nx, OP_N, c + (size_t)q * ldc, ny, ny, nx, nx, scale));
  }
  h->ops->gemm(g1);
  h->ops->gemm(g2);
  h->scr.release(mk);
}

template <typename R> static std::map<int, std::unique_ptr<SolveGraph<R>>>& graphs(nudft2_hss_s* h);
template <> std::map<int, std::unique_ptr<SolveGraph<double>>>& graphs<double>(nudft2_hss_s* h) { return h->g64; }
template <> std::map<int, std::unique_ptr<SolveGraph<float>>>& graphs<float>(nudft2_hss_s* h) { return h->g32; }

// G~_hss^+ f through the URV sweeps, f in caller point order, result in lexicographic column
// order.  The sweeps of each right-hand-side count are captured once into a CUDA graph (after
// one ordinary run that sizes the scratch arena) and replayed afterwards.
template <typename R> static void hss_solve_lex(nudft2_hss_s* h, Hss<R>& H, const double2* f, int64_t ldf, int s,
                                                double2* ylex) {
  const int M = h->M, N = h->N;
  auto& gm = graphs<R>(h);
  auto it = gm.find(s);
  SolveGraph<R>* G = nullptr;
  if (it == gm.end()) {
    auto g = std::make_unique<SolveGraph<R>>();
    g->f2 = h->keep.arr<cplx<R>>((size_t)M * s);
    g->yt = h->keep.arr<cplx<R>>((size_t)N * s);
    G = g.get();
    gm[s] = std::move(g);
    convert_gather<double, R>(h->st, f, (int)ldf, h->pl.perm2, M, s, G->f2, M, 1.0);
    H.ops().reset_staged();
    H.solve(G->f2, M, s, G->yt, N);            // ordinary run: result used, arenas sized
    convert_scatter<R, double>(h->st, G->yt, N, h->pl.colmap, N, s, ylex, N, 1.0);
    // capture the sweeps for the next calls; their descriptor copies come from pinned memory that
    // lives with the graph, reserved here (no allocation is allowed during the capture)
    G->pool.reserve(H.ops().staged() * 2 + 65536);
    const bool prof = H.ops().prof.on;
    H.ops().prof.on = false;
    H.ops().set_capture(&G->pool);
    H.freeze_scratch(true);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      try {
        H.solve(G->f2, M, s, G->yt, N);
      } catch (Error&) {
        G->failed = true;
      }
      e = cudaStreamEndCapture(h->st, &graph);
      if (e == cudaSuccess && !G->failed) {
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
          std::vector<cudaGraphNode_t> nodes(nn);
          cudaGraphGetNodes(graph, nodes.data(), &nn);
          for (auto nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) G->kernels++;
          }
        }
        e = cudaGraphInstantiate(&G->exec, graph, 0);
      }
      if (graph) cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) { G->failed = true; cudaGetLastError(); }
    if (G->failed) h->graphs_failed++; else h->graphs_ok++;
    H.freeze_scratch(false);
    H.ops().set_capture(nullptr);
    H.ops().prof.on = prof;
    return;
  }
  G = it->second.get();
  convert_gather<double, R>(h->st, f, (int)ldf, h->pl.perm2, M, s, G->f2, M, 1.0);
  if (G->exec && !G->failed) {
    Prof& pf = H.ops().prof;
    pf.begin(h->st);
    NH_CK(cudaGraphLaunch(G->exec, h->st));
    if (pf.on) {
      const double e = H.solve_entries();
      pf.end(h->st, K_SWEEP, 8.0 * e * s, e * sizeof(cplx<R>) + 2.0 * ((double)M + N) * s * sizeof(cplx<R>));
    }
    H.ops().count((int)G->kernels);
    h->replays++;
  } else {
    H.solve(G->f2, M, s, G->yt, N);
  }
  convert_scatter<R, double>(h->st, G->yt, N, h->pl.colmap, N, s, ylex, N, 1.0);
}

// Make the handle's stream wait for the work the caller queued on its own stream.
static void enter(nudft2_hss_s* h, void* user_stream) {
  NH_CK(cudaEventRecord(h->join, (cudaStream_t)user_stream));
  NH_CK(cudaStreamWaitEvent(h->st, h->join, 0));
}

// Recompute factors handed back by nudft2_hss_checkpoint before a call that needs them; captured
// solve graphs refer to the old factor addresses and are dropped when that happens.
static void ensure_factors(nudft2_hss_s* h) {
  const bool changed = h->h64 ? h->h64->ensure_factored() : h->h32->ensure_factored();
  if (changed) {
    h->g64.clear();
    h->g32.clear();
  }
}

// ----------------------------------------------------------------------------- LA test hooks
template <typename R>
static void la_tsvd(void* d_ct, int w, int r, int ldct, double eps, void* d_p, int ldp, int* rank, double* sig,
                    cudaStream_t st) {
  Arena scr, keep;
  scr.set_stream(st);
  keep.set_stream(st);
  Ops<R> ops(st, &scr);
  Mat<R> Ct;
  Ct.p = (cplx<R>*)d_ct; Ct.m = w; Ct.n = r; Ct.ld = ldct;
  std::vector<Mat<R>> P;
  std::vector<std::vector<double>> S;
  // all singular values: truncate at the smallest positive threshold, then apply eps on the host
  ops.tsvd_ct({Ct}, 1e-300, keep, P, S);
  const int p = std::min(w, r);
  int rk = 0;
  for (size_t i = 0; i < S[0].size(); ++i)
    if (S[0][i] > eps * S[0][0]) rk++;
  for (int i = 0; i < p; ++i) sig[i] = i < (int)S[0].size() ? S[0][i] : 0.0;
  if (rk > 0)
    NH_CK(cudaMemcpy2DAsync(d_p, (size_t)ldp * sizeof(cplx<R>), P[0].p, (size_t)P[0].ld * sizeof(cplx<R>),
                            (size_t)r * sizeof(cplx<R>), rk, cudaMemcpyDeviceToDevice, st));
  *rank = rk;
  NH_CK(cudaStreamSynchronize(st));
}

template <typename R>
static void la_qr(void* d_a, int m, int n, int lda, void* d_q, int ldq, int grouped, cudaStream_t st) {
  Arena scr, keep;
  scr.set_stream(st);
  keep.set_stream(st);
  Ops<R> ops(st, &scr);
  Mat<R> A;
  A.p = (cplx<R>*)d_a; A.m = m; A.n = n; A.ld = lda;
  auto Q = ops.qr({A}, keep);
  if (grouped) ops.group_wy(Q, keep);
  else Q[0].Tg = nullptr;   // apply panel by panel
  Mat<R> Qm;
  Qm.p = (cplx<R>*)d_q; Qm.m = m; Qm.n = m; Qm.ld = ldq;
  ops.set_identity({Qm});
  ops.apply_q_left(Q, {Qm}, false);
  NH_CK(cudaStreamSynchronize(st));
}

template <typename R>
static void la_qr_apply(void* d_a, int m, int n, int lda, void* d_c, int s, int ldc, bool conj, int grouped,
                        cudaStream_t st) {
  Arena scr, keep;
  scr.set_stream(st);
  keep.set_stream(st);
  Ops<R> ops(st, &scr);
  Mat<R> A;
  A.p = (cplx<R>*)d_a; A.m = m; A.n = n; A.ld = lda;
  auto Q = ops.qr({A}, keep);
  if (grouped) ops.group_wy(Q, keep);
  else Q[0].Tg = nullptr;   // apply panel by panel
  Mat<R> C;
  C.p = (cplx<R>*)d_c; C.m = m; C.n = s; C.ld = ldc;
  ops.apply_q_stream(Q, {C}, conj);
  NH_CK(cudaStreamSynchronize(st));
}

template <typename R>
static void la_gemm(int opa, int opb, int m, int n, int k, double alpha, const void* A, int lda, int64_t sa,
                    const void* B, int ldb, int64_t sb, double beta, void* C, int ldc, int64_t sc, int batch,
                    cudaStream_t st) {
  Arena scr;
  scr.set_stream(st);
  Ops<R> ops(st, &scr);
  std::vector<GemmD<R>> d((size_t)batch);
  for (int b = 0; b < batch; ++b)
    d[b] = {(const cplx<R>*)A + (size_t)b * sa, (const cplx<R>*)B + (size_t)b * sb, (cplx<R>*)C + (size_t)b * sc,
            m, n, k, lda, ldb, ldc, opa, opb, (R)alpha, (R)beta};
  ops.gemm(d);
  NH_CK(cudaStreamSynchronize(st));   // the descriptor staging above lives on this host frame
  if (sizeof(R) == 4 && gemm_tc_enabled() && gemm_tc_error(true))
    throw Error(ST_ETIMEOUT, "la_gemm: a bounded wait of the tensor-core GEMM ran out");
}

// lam (M x s, caller point order) = (G~_hss^+)^* ylex, ylex in lexicographic column order.
template <typename R> static void hss_solve_adj_lex(nudft2_hss_s* h, Hss<R>& H, const double2* ylex, int s,
                                                    double2* lam, int64_t ldl) {
  const int M = h->M, N = h->N;
  auto mk = h->scr.mark();
  cplx<R>* yt = h->scr.arr<cplx<R>>((size_t)N * s);
  cplx<R>* f2 = h->scr.arr<cplx<R>>((size_t)M * s);
  convert_gather<double, R>(h->st, ylex, N, h->pl.colmap, N, s, yt, N, 1.0);
  H.solve_adj(yt, N, s, f2, M);
  convert_scatter<R, double>(h->st, f2, M, h->pl.perm2, M, s, lam, (int)ldl, 1.0);
  h->scr.release(mk);
}

// lam = (A^+)^* g with A^+ = F^{-1} G~^+ (the solve); (F^{-1})^* = F / N.  In mixed precision the
// FP32 adjoint is refined on A^* lam = g with the FP64 exact adjoint apply, like the solve.
static void do_solve_adj(nudft2_hss_s* h, const double2* g, int64_t ldg, int s, double2* lam, int64_t ldl) {
  const int M = h->M, N = h->N;
  auto mk = h->scr.mark();
  double2* ylex = h->scr.arr<double2>((size_t)N * s);
  if (h->h64) {
    dft2(h, g, ldg, s, ylex, N, false, 1.0 / N);
    hss_solve_adj_lex<double>(h, *h->h64, ylex, s, lam, ldl);
    h->iters = 0;
    h->relres = -1;
  } else {
    double2* r = h->scr.arr<double2>((size_t)N * s);
    double2* d = h->scr.arr<double2>((size_t)M * s);
    double* gn = h->scr.arr<double>(s);
    double* rn = h->scr.arr<double>(s);
    NH_CK(cudaMemcpy2DAsync(r, N * sizeof(double2), g, ldg * sizeof(double2), N * sizeof(double2), s,
                            cudaMemcpyDeviceToDevice, h->st));
    NH_CK(cudaMemset2DAsync(lam, ldl * sizeof(double2), 0, M * sizeof(double2), s, h->st));
    colnorm2(h->st, N, s, r, N, gn);
    std::vector<double> hg(s), hr(s);
    NH_CK(cudaMemcpyAsync(hg.data(), gn, s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    int it = 0;
    double worst = 1.0;
    const bool full = (h->opt.flags & NUDFT2_FLAG_FP64_RESIDUALS) != 0;
    for (it = 1; it <= std::max(1, h->opt.refine_max); ++it) {
      dft2(h, r, N, s, ylex, N, false, 1.0 / N);
      hss_solve_adj_lex<float>(h, *h->h32, ylex, s, d, M);
      axpy2(h->st, M, s, 1.0, d, M, lam, (int)ldl);
      if (it == 1 || full) {
        exact_adj(h, lam, ldl, s, r, N);              // r = A^* lam (FP64)
        axpy2(h->st, N, s, -1.0, g, (int)ldg, r, N);  // r = A^* lam - g
        axpy2(h->st, N, s, -2.0, r, N, r, N);         // r = g - A^* lam
      } else {
        exact_adj_sub32(h, d, M, s, r, N);            // r -= A^* d: the correction is O(eps) small
      }
      colnorm2(h->st, N, s, r, N, rn);
      NH_CK(cudaMemcpyAsync(hr.data(), rn, s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      NH_CK(cudaStreamSynchronize(h->st));
      worst = 0;
      for (int q = 0; q < s; ++q) worst = std::max(worst, std::sqrt(hr[q] / std::max(hg[q], 1e-300)));
      if (worst <= h->opt.refine_tol) break;
    }
    h->iters = std::min(it, std::max(1, h->opt.refine_max));
    h->relres = worst;
  }
  h->scr.release(mk);
}

// The direct solver as a preconditioner (Sec. 4.1): P = F^{-1} G~_hss^+ applied once (no
// refinement), and its adjoint P^* = G~_hss^{+*} F / N.
static void precond_apply(nudft2_hss_s* h, const double2* f, int64_t ldf, int s, double2* c, int64_t ldc) {
  auto mk = h->scr.mark();
  double2* ylex = h->scr.arr<double2>((size_t)h->N * s);
  if (h->h64) hss_solve_lex<double>(h, *h->h64, f, ldf, s, ylex);
  else hss_solve_lex<float>(h, *h->h32, f, ldf, s, ylex);
  dft2(h, ylex, h->N, s, c, ldc, true);
  h->scr.release(mk);
}
static void precond_adjoint(nudft2_hss_s* h, const double2* g, int64_t ldg, int s, double2* lam, int64_t ldl) {
  auto mk = h->scr.mark();
  double2* ylex = h->scr.arr<double2>((size_t)h->N * s);
  dft2(h, g, ldg, s, ylex, h->N, false, 1.0 / h->N);
  if (h->h64) hss_solve_adj_lex<double>(h, *h->h64, ylex, s, lam, ldl);
  else hss_solve_adj_lex<float>(h, *h->h32, ylex, s, lam, ldl);
  h->scr.release(mk);
}

// LSQR (Paige & Saunders) on the preconditioned system B x = P r with B = P A, N x N and close
// to the identity; B v = P (A v) and B^* u = A^* (P^* u), A and A^* by the exact FP64 apply.
// Columns iterate together, each with its own scalars.  A column stops when its estimated
// ||P r - B x|| drops to tol * ||P r|| (or its Lanczos vectors vanish); a column whose ||P r||
// is at most skip[q] does not iterate at all (x = 0).  beta1 returns ||P r|| per column; the
// return value is the iteration count of the slowest column.
static int lsqr_core(nudft2_hss_s* h, const double2* r, int64_t ldr, int s, double2* x, int64_t ldx, double tol,
                     int maxit, const std::vector<double>& skip, std::vector<double>& beta1) {
  const int M = h->M, N = h->N;
  auto mk = h->scr.mark();
  double2* u = h->scr.arr<double2>((size_t)N * s);
  double2* v = h->scr.arr<double2>((size_t)N * s);
  double2* w = h->scr.arr<double2>((size_t)N * s);
  double2* tn = h->scr.arr<double2>((size_t)N * s);
  double2* tm = h->scr.arr<double2>((size_t)M * s);
  double* dn = h->scr.arr<double>(s);
  double* ca = h->scr.arr<double>(s);
  double* cb = h->scr.arr<double>(s);
  std::vector<double> hn(s), ha(s), hb(s);
  auto norms = [&](const double2* z, int m) {
    colnorm2(h->st, m, s, z, m, dn);
    NH_CK(cudaMemcpyAsync(hn.data(), dn, s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    NH_CK(cudaStreamSynchronize(h->st));
    for (int q = 0; q < s; ++q) hn[q] = std::sqrt(hn[q]);
    return hn;
  };
  auto axpby = [&](const double2* xs, int ldxs, double2* y, int ldy, int m) {   // y = ha x + hb y
    NH_CK(cudaMemcpyAsync(ca, ha.data(), s * sizeof(double), cudaMemcpyHostToDevice, h->st));
    NH_CK(cudaMemcpyAsync(cb, hb.data(), s * sizeof(double), cudaMemcpyHostToDevice, h->st));
    axpby_cols(h->st, m, s, ca, xs, ldxs, cb, y, ldy);
    NH_CK(cudaStreamSynchronize(h->st));   // the host coefficient vectors are reused next
  };
  auto applyB = [&](const double2* in, double2* out) {     // out = P (A in)
    exact_fwd(h, in, N, s, tm, M);
    precond_apply(h, tm, M, s, out, N);
  };
  auto applyBh = [&](const double2* in, double2* out) {    // out = A^* (P^* in)
    precond_adjoint(h, in, N, s, tm, M);
    exact_adj(h, tm, M, s, out, N);
  };
  std::vector<double> alpha(s), beta(s), rhobar(s), phibar(s);
  std::vector<char> active(s, 1);
  // beta1 u = P r ; alpha v = B^* u ; w = v ; x = 0
  precond_apply(h, r, ldr, s, u, N);
  beta1 = norms(u, N);
  for (int q = 0; q < s; ++q) {
    if (!(beta1[q] > skip[q])) active[q] = 0;
    ha[q] = 0;
    hb[q] = active[q] ? 1.0 / beta1[q] : 0.0;
  }
  axpby(nullptr, N, u, N, N);
  applyBh(u, v);
  alpha = norms(v, N);
  for (int q = 0; q < s; ++q) { ha[q] = 0; hb[q] = alpha[q] > 0 ? 1.0 / alpha[q] : 0.0; if (!(alpha[q] > 0)) active[q] = 0; }
  axpby(nullptr, N, v, N, N);
  NH_CK(cudaMemcpy2DAsync(w, N * sizeof(double2), v, N * sizeof(double2), N * sizeof(double2), s,
                          cudaMemcpyDeviceToDevice, h->st));
  NH_CK(cudaMemset2DAsync(x, ldx * sizeof(double2), 0, N * sizeof(double2), s, h->st));
  for (int q = 0; q < s; ++q) { phibar[q] = beta1[q]; rhobar[q] = alpha[q]; }
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    bool any = false;
    for (int q = 0; q < s; ++q) any = any || active[q];
    if (!any) { --it; break; }
    // beta u = B v - alpha u
    applyB(v, tn);
    for (int q = 0; q < s; ++q) { ha[q] = active[q] ? 1.0 : 0.0; hb[q] = active[q] ? -alpha[q] : 1.0; }
    axpby(tn, N, u, N, N);
    beta = norms(u, N);
    for (int q = 0; q < s; ++q) { ha[q] = 0; hb[q] = (active[q] && beta[q] > 0) ? 1.0 / beta[q] : 1.0; }
    axpby(nullptr, N, u, N, N);
    // alpha v = B^* u - beta v
    applyBh(u, tn);
    std::vector<double> anew(s);
    for (int q = 0; q < s; ++q) { ha[q] = active[q] ? 1.0 : 0.0; hb[q] = active[q] ? -beta[q] : 1.0; }
    axpby(tn, N, v, N, N);
    anew = norms(v, N);
    for (int q = 0; q < s; ++q) { ha[q] = 0; hb[q] = (active[q] && anew[q] > 0) ? 1.0 / anew[q] : 1.0; }
    axpby(nullptr, N, v, N, N);
    // plane rotation, then x += (phi / rho) w ; w = v - (theta / rho) w
    std::vector<double> cx(s, 0.0), cw(s, 1.0), ccw(s, 0.0);
    for (int q = 0; q < s; ++q) {
      if (!active[q]) continue;
      const double rho = std::hypot(rhobar[q], beta[q]);
      const double c = rhobar[q] / rho, sn = beta[q] / rho;
      const double theta = sn * anew[q];
      rhobar[q] = -c * anew[q];
      const double phi = c * phibar[q];
      phibar[q] = sn * phibar[q];
      cx[q] = phi / rho;
      cw[q] = -theta / rho;
      ccw[q] = 1.0;
      alpha[q] = anew[q];
      if (!(phibar[q] > tol * beta1[q]) || !(beta[q] > 0) || !(anew[q] > 0)) active[q] = 0;
    }
    for (int q = 0; q < s; ++q) { ha[q] = cx[q]; hb[q] = 1.0; }
    axpby(w, N, x, (int)ldx, N);
    for (int q = 0; q < s; ++q) { ha[q] = ccw[q]; hb[q] = ccw[q] > 0 ? cw[q] : 1.0; }
    axpby(v, N, w, N, N);
  }
  h->scr.release(mk);
  return std::min(it, maxit);
}

// plsqr: the direct solver as a preconditioner (Sec. 4.1).  With an FP64 factorization it is one
// LSQR run on B c = P f.  With a MIXED (FP32) factorization the applications of P and P^* carry FP32
// rounding, so B = P A is linear and self-consistent only to FP32 level and a single Krylov
// recursion stalls near u_32 times the conditioning.  There the LSQR runs inside an outer
// defect correction whose residual is exact FP64: r = f - A c; x = LSQR(B, P r) to a modest
// tolerance; c += x; repeated until ||P r|| <= tol ||P f|| per column.  Each pass reduces the
// preconditioned residual by the inner tolerance (or the FP32 floor), so a few passes reach tol.
// Returns the total LSQR iterations over all passes (slowest column per pass) and the largest
// ||f - A c|| / ||f|| (exact apply) over the columns.
static void do_plsqr(nudft2_hss_s* h, const double2* f, int64_t ldf, int s, double2* x, int64_t ldx, double tol,
                     int maxit, int* iters_out, double* relres_out) {
  const int M = h->M, N = h->N;
  auto mk = h->scr.mark();
  double2* tm = h->scr.arr<double2>((size_t)M * s);
  double* dn = h->scr.arr<double>(s);
  std::vector<double> hn(s);
  auto norms = [&](const double2* z, int m) {
    colnorm2(h->st, m, s, z, m, dn);
    NH_CK(cudaMemcpyAsync(hn.data(), dn, s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    NH_CK(cudaStreamSynchronize(h->st));
    for (int q = 0; q < s; ++q) hn[q] = std::sqrt(hn[q]);
    return hn;
  };
  std::vector<double> beta1, pf, skip(s, 0.0);
  int total = 0;
  if (h->h64) {
    total = lsqr_core(h, f, ldf, s, x, ldx, tol, maxit, skip, beta1);
  } else {
    // outer defect correction with the exact FP64 residual
    const double tol_in = std::max(tol, 1e-5);
    double2* r = h->scr.arr<double2>((size_t)M * s);
    double2* dx = h->scr.arr<double2>((size_t)N * s);
    NH_CK(cudaMemcpy2DAsync(r, M * sizeof(double2), f, ldf * sizeof(double2), M * sizeof(double2), s,
                            cudaMemcpyDeviceToDevice, h->st));
    NH_CK(cudaMemset2DAsync(x, ldx * sizeof(double2), 0, N * sizeof(double2), s, h->st));
    for (int pass = 0; pass < 20 && total < maxit; ++pass) {
      total += lsqr_core(h, r, M, s, dx, N, tol_in, maxit - total, skip, beta1);
      if (pass == 0) {
        pf = beta1;
        for (int q = 0; q < s; ++q) skip[q] = tol * pf[q];
      } else {
        bool done = true;
        for (int q = 0; q < s; ++q) done = done && !(beta1[q] > skip[q]);
        if (done) break;
      }
      axpy2(h->st, N, s, 1.0, dx, N, x, (int)ldx);      // c += x (zero for converged columns)
      exact_fwd(h, x, ldx, s, r, M);                    // r = A c (FP64, Eq. 1)
      axpy2(h->st, M, s, -1.0, f, (int)ldf, r, M);      // r = A c - f
      axpy2(h->st, M, s, -2.0, r, M, r, M);             // r = f - A c
    }
  }
  *iters_out = total;
  // true residual of the original problem
  exact_fwd(h, x, ldx, s, tm, M);
  axpy2(h->st, M, s, -1.0, f, (int)ldf, tm, M);         // tm = A x - f
  std::vector<double> rn = norms(tm, M);
  NH_CK(cudaMemcpy2DAsync(tm, M * sizeof(double2), f, ldf * sizeof(double2), M * sizeof(double2), s,
                          cudaMemcpyDeviceToDevice, h->st));
  std::vector<double> fn = norms(tm, M);
  double worst = 0;
  for (int q = 0; q < s; ++q) worst = std::max(worst, rn[q] / std::max(fn[q], 1e-300));
  *relres_out = worst;
  h->scr.release(mk);
}

// Runs fn(i) for every i < count on up to `threads` host threads (the caller's thread included),
// each with the caller's device current.  Every problem owns its handle and its stream, so the
// problems' kernels overlap on the GPU while each thread drives its own problem's host-side steps
// (rank readbacks, descriptor uploads).  fn must not throw.
template <typename F> static void run_pool(int count, int threads, F&& fn) {
  int dev = 0;
  NH_CK(cudaGetDevice(&dev));
  const int T = std::max(1, std::min(threads > 0 ? threads : 8, count));
  std::atomic<int> next{0};
  auto work = [&] {
    cudaSetDevice(dev);
    for (int i = next++; i < count; i = next++) fn(i);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
}

// First failing problem of a batch (status and message), or OK.
static nudft2_status batch_result(const std::vector<nudft2_status>& st, const std::vector<std::string>& msg) {
  for (size_t i = 0; i < st.size(); ++i)
    if (st[i] != NUDFT2_OK) {
      g_err = "problem " + std::to_string(i) + ": " + msg[i];
      return st[i];
    }
  g_err.clear();
  return NUDFT2_OK;
}

// Handle state shared by build and load: stream, arenas, the plan (binning and sorting of the
// points) and the exact-apply and DFT tables.
static void init_handle(nudft2_hss_s* h, const double* d_x, const double* d_y, int64_t M, int nx, int ny,
                        const nudft2_opts& opt, int Lx, int Ly, void* stream) {
  h->opt = opt;
  h->M = (int)M; h->nx = nx; h->ny = ny; h->L = std::max(Lx, Ly); h->N = nx * ny;
  NH_CK(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
  NH_CK(cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming));
  enter(h, stream);
  h->keep.set_stream(h->st);
  h->scr.set_stream(h->st);
  h->ops.reset(new Ops<double>(h->st, &h->scr));
  make_plan(h->st, h->keep, h->scr, d_x, d_y, (int)M, nx, ny, Lx, Ly, h->pl);
  h->Ax = h->keep.arr<double2>((size_t)M * nx);
  h->Ay = h->keep.arr<double2>((size_t)M * ny);
  twiddle_table(h->st, h->pl.x, (int)M, nx, h->Ax);
  twiddle_table(h->st, h->pl.y, (int)M, ny, h->Ay);
  h->Fxi = h->keep.arr<double2>((size_t)nx * nx);
  h->Fyi = h->keep.arr<double2>((size_t)ny * ny);
  h->Fxf = h->keep.arr<double2>((size_t)nx * nx);
  h->Fyf = h->keep.arr<double2>((size_t)ny * ny);
  dft_matrix<double>(h->st, nx, +1, 1.0 / nx, h->Fxi);
  dft_matrix<double>(h->st, ny, +1, 1.0 / ny, h->Fyi);
  dft_matrix<double>(h->st, nx, -1, 1.0, h->Fxf);
  dft_matrix<double>(h->st, ny, -1, 1.0, h->Fyf);
  h->ops->count(8);
}

// ----------------------------------------------------------------------------- C-ABI
extern "C" {

const char* nudft2_last_error(void) { return g_err.c_str(); }

nudft2_status nudft2_psi_eval(const double* d_x, int64_t M, int n, void* d_out, void* stream) {
  return guard([&] {
    NH_REQUIRE(d_x && d_out && M > 0 && n > 0 && M < (1LL << 31), ST_EINVAL, "nudft2_psi_eval: bad arguments");
    Arena scr;
    scr.set_stream((cudaStream_t)stream);
    Ops<double> ops((cudaStream_t)stream, &scr);
    psi_eval<double>(ops, {PsiD<double>{d_x, (int)M, 0, n, n, (double2*)d_out, (int)M}});
    NH_CK(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

void nudft2_hss_free(nudft2_hss_t h);

nudft2_status nudft2_exact_apply(const double* d_x, const double* d_y, int64_t M, int nx, int ny, int op,
                                 const void* d_in, int64_t ldi, int nrhs, void* d_out, int64_t ldo, void* stream) {
  return guard([&] {
    NH_REQUIRE(d_x && d_y && d_in && d_out && M >= 1 && nx >= 1 && ny >= 1 && nrhs >= 0 && M < (1LL << 31),
               ST_EINVAL, "exact_apply: bad arguments");
    NH_REQUIRE(op == NUDFT2_EXACT_FWD || op == NUDFT2_EXACT_ADJ, ST_EINVAL, "exact_apply: op must be EXACT_FWD/ADJ");
    const int64_t N = (int64_t)nx * ny;
    NH_REQUIRE(op == NUDFT2_EXACT_FWD ? (ldi >= N && ldo >= M) : (ldi >= M && ldo >= N), ST_EINVAL,
               "exact_apply: leading dimension too small");
    if (nrhs == 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    Arena scr;
    scr.set_stream(st);
    Ops<double> ops(st, &scr);
    double2* Ax = scr.arr<double2>((size_t)M * nx);
    double2* Ay = scr.arr<double2>((size_t)M * ny);
    twiddle_table(st, d_x, (int)M, nx, Ax);
    twiddle_table(st, d_y, (int)M, ny, Ay);
    const Exact e{(int)M, nx, ny, Ax, Ay};
    if (op == NUDFT2_EXACT_FWD)
      exact_fwd_impl(ops, scr, st, e, (const double2*)d_in, ldi, nrhs, (double2*)d_out, ldo);
    else
      exact_adj_impl(ops, scr, st, e, (const double2*)d_in, ldi, nrhs, (double2*)d_out, ldo);
    NH_CK(cudaStreamSynchronize(st));
  });
}

nudft2_status nudft2_hss_build(const double* d_x, const double* d_y, int64_t M, int nx, int ny,
                               const nudft2_opts* o, void* stream, nudft2_hss_t* out) {
  nudft2_hss_s* h = nullptr;
  auto st = guard([&] {
    NH_REQUIRE(out != nullptr, ST_EINVAL, "out is NULL");
    *out = nullptr;
    NH_REQUIRE(d_x && d_y, ST_EINVAL, "points are NULL");
    NH_REQUIRE(nx >= 1 && ny >= 1 && (int64_t)nx * ny <= (1LL << 26), ST_EINVAL, "bad frequency grid");
    NH_REQUIRE(M >= (int64_t)nx * ny, ST_EINVAL, "least squares needs M >= N = nx*ny");
    NH_REQUIRE(M < (1LL << 31), ST_EINVAL, "M too large");
    nudft2_opts opt{1e-10, 0, 64, NUDFT2_FP64, 1e-8, 8, 0, 0};
    if (o) opt = *o;
    NH_REQUIRE(opt.eps > 0 && opt.eps < 1, ST_EINVAL, "eps must lie in (0,1)");
    NH_REQUIRE(opt.prec == NUDFT2_FP64 || opt.prec == NUDFT2_MIXED, ST_EINVAL, "unknown precision");
    int L = opt.levels;
    if (L <= 0) {
      // smallest depth whose product leaves have at most `leaf` columns
      const int leaf = std::max(opt.leaf, 1);
      L = 1;
      while (L < 12 && (int64_t)(nx >> L) * (ny >> L) > leaf && (nx >> (L + 1)) >= 1 && (ny >> (L + 1)) >= 1) ++L;
    }
    const int Lx = L, Ly = opt.levels_y > 0 ? opt.levels_y : L;
    NH_REQUIRE(Lx >= 1 && Lx <= 12 && Ly >= 1 && Ly <= 12 && (nx >> Lx) >= 1 && (ny >> Ly) >= 1, ST_EINVAL,
               "levels must satisfy 1 <= L and 2^Lx <= nx, 2^Ly <= ny");
    // validate points on the host: finite and in [0, 1)
    {
      std::vector<double> hx(M), hy(M);
      NH_CK(cudaMemcpy(hx.data(), d_x, M * sizeof(double), cudaMemcpyDeviceToHost));
      NH_CK(cudaMemcpy(hy.data(), d_y, M * sizeof(double), cudaMemcpyDeviceToHost));
      for (int64_t j = 0; j < M; ++j)
        NH_REQUIRE(std::isfinite(hx[j]) && std::isfinite(hy[j]) && hx[j] >= 0 && hx[j] < 1 && hy[j] >= 0 && hy[j] < 1,
                   ST_EINVAL, "points must be finite and lie in [0,1)^2");
    }
    h = new nudft2_hss_s();
    const double t0 = now_ms();
    init_handle(h, d_x, d_y, M, nx, ny, opt, Lx, Ly, stream);
    const bool prof = (opt.flags & NUDFT2_FLAG_PROFILE) != 0;
    h->ops->prof.on = prof;
    if (opt.prec == NUDFT2_FP64) {
      h->h64.reset(new Hss<double>(h->st, &h->pl));
      h->h64->ops().prof.on = prof;
      h->h64->build(opt.eps, (opt.flags & NUDFT2_FLAG_FADI) != 0);
    } else {
      h->h32.reset(new Hss<float>(h->st, &h->pl));
      h->h32->ops().prof.on = prof;
      h->Ax32 = h->keep.arr<float2>((size_t)M * nx);
      h->Ay32 = h->keep.arr<float2>((size_t)M * ny);
      convert_gather<double, float>(h->st, h->Ax, (int)M, nullptr, (int)M, nx, h->Ax32, (int)M, 1.0);
      convert_gather<double, float>(h->st, h->Ay, (int)M, nullptr, (int)M, ny, h->Ay32, (int)M, 1.0);
      h->h32->build(opt.eps, (opt.flags & NUDFT2_FLAG_FADI) != 0);
    }
    NH_CK(cudaStreamSynchronize(h->st));
    if (h->h32 && gemm_tc_error(true))
      throw Error(ST_ETIMEOUT, "build: a bounded wait of the tensor-core GEMM ran out");
    h->t_build = now_ms() - t0;
    *out = h;
  });
  if (st != NUDFT2_OK && h) {
    const std::string msg = g_err;
    nudft2_hss_free(h);
    g_err = msg;
  }
  return st;
}

nudft2_status nudft2_hss_factor(nudft2_hss_t h, void* stream) {
  return guard([&] {
    NH_REQUIRE(h != nullptr, ST_ESTATE, "factor: no handle (build first)");
    enter(h, stream);
    const double t0 = now_ms();
    if (h->h64) h->h64->factor();
    else h->h32->factor();
    NH_CK(cudaStreamSynchronize(h->st));
    if (h->h32 && gemm_tc_error(true))
      throw Error(ST_ETIMEOUT, "factor: a bounded wait of the tensor-core GEMM ran out");
    h->t_factor = now_ms() - t0;
    h->factored = true;
  });
}

static void do_solve(nudft2_hss_t h, const double2* f, int64_t ldf, int s, double2* c, int64_t ldc) {
  const int M = h->M, N = h->N;
  auto mk = h->scr.mark();
  double2* ylex = h->scr.arr<double2>((size_t)N * s);
  if (h->h64) {
    hss_solve_lex<double>(h, *h->h64, f, ldf, s, ylex);
    dft2(h, ylex, N, s, c, ldc, true);
    h->iters = 0;
    h->relres = -1;
  } else {
    // mixed precision: c <- c + F^{-1} G~32^+ (f - A c), residual in FP64 (exact apply)
    double2* r = h->scr.arr<double2>((size_t)M * s);
    double2* d = h->scr.arr<double2>((size_t)N * s);
    double* fn = h->scr.arr<double>(s);
    double* rn = h->scr.arr<double>(s);
    double* dn = h->scr.arr<double>(2 * s);
    NH_CK(cudaMemcpy2DAsync(r, M * sizeof(double2), f, ldf * sizeof(double2), M * sizeof(double2), s,
                            cudaMemcpyDeviceToDevice, h->st));
    NH_CK(cudaMemset2DAsync(c, ldc * sizeof(double2), 0, N * sizeof(double2), s, h->st));
    colnorm2(h->st, M, s, r, M, fn);
    std::vector<double> hf(s), hr(s), hd(2 * s);
    NH_CK(cudaMemcpyAsync(hf.data(), fn, s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    int it = 0;
    double worst = 1.0;
    // Stops when the relative residual ||f - A c|| / ||f|| reaches refine_tol (consistent data), or
    // when the last correction is below refine_tol relative to c (data with a nonzero
    // least-squares residual, whose residual norm levels off at ||r_LS||).
    const bool full = (h->opt.flags & NUDFT2_FLAG_FP64_RESIDUALS) != 0;
    for (it = 1; it <= std::max(1, h->opt.refine_max); ++it) {
      hss_solve_lex<float>(h, *h->h32, r, M, s, ylex);
      dft2(h, ylex, N, s, d, N, true);
      axpy2(h->st, N, s, 1.0, d, N, c, (int)ldc);
      colnorm2(h->st, N, s, d, N, dn);
      colnorm2(h->st, N, s, c, (int)ldc, dn + s);
      if (it == 1 || full) {
        exact_fwd(h, c, ldc, s, r, M);                // r = A c (FP64, Eq. 1)
        axpy2(h->st, M, s, -1.0, f, (int)ldf, r, M);  // r = A c - f
        axpy2(h->st, M, s, -2.0, r, M, r, M);         // r = f - A c
      } else {
        exact_fwd_sub32(h, d, N, s, r, M);            // r -= A d: the correction is O(eps) small
      }
      colnorm2(h->st, M, s, r, M, rn);
      NH_CK(cudaMemcpyAsync(hr.data(), rn, s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      NH_CK(cudaMemcpyAsync(hd.data(), dn, 2 * s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      NH_CK(cudaStreamSynchronize(h->st));
      worst = 0;
      double dworst = 0;
      for (int q = 0; q < s; ++q) {
        worst = std::max(worst, std::sqrt(hr[q] / std::max(hf[q], 1e-300)));
        if (hd[s + q] > 0) dworst = std::max(dworst, std::sqrt(hd[q] / hd[s + q]));
      }
      if (worst <= h->opt.refine_tol || (it > 1 && dworst <= h->opt.refine_tol)) break;
    }
    h->iters = std::min(it, std::max(1, h->opt.refine_max));
    // Data with a nonzero least-squares residual: the loop above stops at the fixed point
    // P (f - A c) = 0 of the FP32 pseudo-inverse P, which differs from the least-squares solution
    // by O(eps) ||r_LS||.  Polish on the normal equations: c += P P^* A^* r with A^* r from the exact
    // FP64 adjoint; P P^* approximates (A^* A)^{-1}, and the fixed point is A^* (f - A c) = 0.
    if (worst > h->opt.refine_tol) {
      double2* t = h->scr.arr<double2>((size_t)N * s);
      double2* u = h->scr.arr<double2>((size_t)M * s);
      for (int k = 1; k <= std::max(1, h->opt.refine_max); ++k) {
        exact_adj(h, r, M, s, t, N);                     // t = A^* r (FP64)
        dft2(h, t, N, s, ylex, N, false, 1.0 / N);       // P^* t = G~^{+*} F t / N
        hss_solve_adj_lex<float>(h, *h->h32, ylex, s, u, M);
        hss_solve_lex<float>(h, *h->h32, u, M, s, ylex); // d = P u
        dft2(h, ylex, N, s, d, N, true);
        axpy2(h->st, N, s, 1.0, d, N, c, (int)ldc);
        colnorm2(h->st, N, s, d, N, dn);
        colnorm2(h->st, N, s, c, (int)ldc, dn + s);
        if (full) {
          exact_fwd(h, c, ldc, s, r, M);
          axpy2(h->st, M, s, -1.0, f, (int)ldf, r, M);
          axpy2(h->st, M, s, -2.0, r, M, r, M);
        } else {
          exact_fwd_sub32(h, d, N, s, r, M);
        }
        colnorm2(h->st, M, s, r, M, rn);
        NH_CK(cudaMemcpyAsync(hr.data(), rn, s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        NH_CK(cudaMemcpyAsync(hd.data(), dn, 2 * s * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        NH_CK(cudaStreamSynchronize(h->st));
        worst = 0;
        double dworst = 0;
        for (int q = 0; q < s; ++q) {
          worst = std::max(worst, std::sqrt(hr[q] / std::max(hf[q], 1e-300)));
          if (hd[s + q] > 0) dworst = std::max(dworst, std::sqrt(hd[q] / hd[s + q]));
        }
        h->iters++;
        if (dworst <= h->opt.refine_tol) break;
      }
    }
    h->relres = worst;
  }
  h->scr.release(mk);
}

nudft2_status nudft2_hss_solve(nudft2_hss_t h, const void* d_f, int64_t ldf, int nrhs, void* d_c, int64_t ldc,
                               void* stream) {
  return guard([&] {
    NH_REQUIRE(h != nullptr, ST_ESTATE, "solve: no handle");
    NH_REQUIRE(h->factored, ST_ESTATE, "solve before factor");
    NH_REQUIRE(nrhs >= 0 && d_f && d_c && ldf >= h->M && ldc >= h->N, ST_EINVAL, "solve: bad arguments");
    enter(h, stream);
    if (nrhs == 0) return;
    ensure_factors(h);
    const double t0 = now_ms();
    do_solve(h, (const double2*)d_f, ldf, nrhs, (double2*)d_c, ldc);
    NH_CK(cudaStreamSynchronize(h->st));
    h->t_solve = now_ms() - t0;
  });
}

nudft2_status nudft2_hss_apply(nudft2_hss_t h, int op, const void* d_in, int64_t ldi, int nrhs, void* d_out,
                               int64_t ldo, void* stream) {
  return guard([&] {
    NH_REQUIRE(h != nullptr, ST_ESTATE, "apply: no handle");
    NH_REQUIRE(nrhs >= 0 && d_in && d_out, ST_EINVAL, "apply: bad arguments");
    enter(h, stream);
    if (nrhs == 0) return;
    const int M = h->M, N = h->N;
    switch (op) {
      case NUDFT2_EXACT_FWD:
        NH_REQUIRE(ldi >= N && ldo >= M, ST_EINVAL, "apply: leading dimension too small");
        exact_fwd(h, (const double2*)d_in, ldi, nrhs, (double2*)d_out, ldo);
        break;
      case NUDFT2_EXACT_ADJ:
        NH_REQUIRE(ldi >= M && ldo >= N, ST_EINVAL, "apply: leading dimension too small");
        exact_adj(h, (const double2*)d_in, ldi, nrhs, (double2*)d_out, ldo);
        break;
      case NUDFT2_PINV:
        NH_REQUIRE(h->factored, ST_ESTATE, "apply PINV before factor");
        NH_REQUIRE(ldi >= M && ldo >= N, ST_EINVAL, "apply: leading dimension too small");
        ensure_factors(h);
        do_solve(h, (const double2*)d_in, ldi, nrhs, (double2*)d_out, ldo);
        break;
      case NUDFT2_FAST_FWD: {
        NH_REQUIRE(ldi >= N && ldo >= M, ST_EINVAL, "apply: leading dimension too small");
        auto mk = h->scr.mark();
        double2* y = h->scr.arr<double2>((size_t)N * nrhs);
        dft2(h, (const double2*)d_in, ldi, nrhs, y, N, false);
        if (h->h64) {
          double2* yt = h->scr.arr<double2>((size_t)N * nrhs);
          double2* o2 = h->scr.arr<double2>((size_t)M * nrhs);
          convert_gather<double, double>(h->st, y, N, h->pl.colmap, N, nrhs, yt, N, 1.0);
          h->h64->matvec(yt, N, nrhs, o2, M);
          convert_scatter<double, double>(h->st, o2, M, h->pl.perm2, M, nrhs, (double2*)d_out, (int)ldo, 1.0);
        } else {
          float2* yt = h->scr.arr<float2>((size_t)N * nrhs);
          float2* o2 = h->scr.arr<float2>((size_t)M * nrhs);
          convert_gather<double, float>(h->st, y, N, h->pl.colmap, N, nrhs, yt, N, 1.0);
          h->h32->matvec(yt, N, nrhs, o2, M);
          convert_scatter<float, double>(h->st, o2, M, h->pl.perm2, M, nrhs, (double2*)d_out, (int)ldo, 1.0);
        }
        h->scr.release(mk);
        break;
      }
      case NUDFT2_PINV_ADJ:
        NH_REQUIRE(h->factored, ST_ESTATE, "apply PINV_ADJ before factor");
        NH_REQUIRE(ldi >= N && ldo >= M, ST_EINVAL, "apply: leading dimension too small");
        ensure_factors(h);
        do_solve_adj(h, (const double2*)d_in, ldi, nrhs, (double2*)d_out, ldo);
        break;
      case NUDFT2_FAST_ADJ: {
        // A_fast^* = (G~_hss F)^* = F^* G~_hss^* with F^* = N F^{-1} (F symmetric, F^{-1} = conj(F) / N)
        NH_REQUIRE(ldi >= M && ldo >= N, ST_EINVAL, "apply: leading dimension too small");
        auto mk = h->scr.mark();
        double2* y = h->scr.arr<double2>((size_t)N * nrhs);
        if (h->h64) {
          double2* z2 = h->scr.arr<double2>((size_t)M * nrhs);
          double2* yt = h->scr.arr<double2>((size_t)N * nrhs);
          convert_gather<double, double>(h->st, (const double2*)d_in, (int)ldi, h->pl.perm2, M, nrhs, z2, M, 1.0);
          h->h64->matvec_adj(z2, M, nrhs, yt, N);
          convert_scatter<double, double>(h->st, yt, N, h->pl.colmap, N, nrhs, y, N, 1.0);
        } else {
          float2* z2 = h->scr.arr<float2>((size_t)M * nrhs);
          float2* yt = h->scr.arr<float2>((size_t)N * nrhs);
          convert_gather<double, float>(h->st, (const double2*)d_in, (int)ldi, h->pl.perm2, M, nrhs, z2, M, 1.0);
          h->h32->matvec_adj(z2, M, nrhs, yt, N);
          convert_scatter<float, double>(h->st, yt, N, h->pl.colmap, N, nrhs, y, N, 1.0);
        }
        dft2(h, y, N, nrhs, (double2*)d_out, ldo, true, (double)N);
        h->scr.release(mk);
        break;
      }
      default:
        throw Error(ST_EINVAL, "apply: unknown operator");
    }
    NH_CK(cudaStreamSynchronize(h->st));
  });
}

nudft2_status nudft2_hss_grad(nudft2_hss_t h, const void* d_f, int64_t ldf, const void* d_c, int64_t ldc,
                              const void* d_g, int64_t ldg, int nrhs, void* d_gf, int64_t ldgf, double* d_gx,
                              double* d_gy, void* stream) {
  return guard([&] {
    NH_REQUIRE(h != nullptr, ST_ESTATE, "grad: no handle");
    NH_REQUIRE(h->factored, ST_ESTATE, "grad before factor");
    const int M = h->M, N = h->N, s = nrhs;
    NH_REQUIRE(s >= 1 && d_f && d_c && d_g && ldf >= M && ldc >= N && ldg >= N && (!d_gf || ldgf >= M) &&
                   ((d_gx == nullptr) == (d_gy == nullptr)),
               ST_EINVAL, "grad: bad arguments");
    enter(h, stream);
    ensure_factors(h);
    auto mk = h->scr.mark();
    // lam = (A^+)^* g  (also the gradient with respect to f)
    double2* lam = d_gf ? (double2*)d_gf : h->scr.arr<double2>((size_t)M * s);
    const int64_t ldl = d_gf ? ldgf : M;
    do_solve_adj(h, (const double2*)d_g, ldg, s, lam, ldl);
    double2* mu = nullptr;
    if (d_gx || !h->h64) {
      // mu = A^+ lam
      mu = h->scr.arr<double2>((size_t)N * s);
      do_solve(h, lam, ldl, s, mu, N);
    }
    if (!h->h64) {
      // MIXED: the refined adjoint solves A^* lam = g, but its fixed point lies in the range of the
      // FP32 HSS adjoint, which differs from range(A) by O(eps).  mu = A^+ lam is refined to the
      // exact least-squares solution, and A^+ annihilates the part of lam outside range(A), so
      // lam = A mu (exact FP64 apply) is the minimum-norm solution (A^+)^* g itself.
      exact_fwd(h, mu, N, s, lam, ldl);
    }
    if (d_gx) {
      // W = [c, Dx c, Dy c, Dx mu, Dy mu] ; E = A W (exact, FP64)
      double2* W = h->scr.arr<double2>((size_t)N * 5 * s);
      double2* E = h->scr.arr<double2>((size_t)M * 5 * s);
      NH_CK(cudaMemcpy2DAsync(W, N * sizeof(double2), d_c, ldc * sizeof(double2), N * sizeof(double2), s,
                              cudaMemcpyDeviceToDevice, h->st));
      deriv_weights(h->st, h->nx, h->ny, s, (const double2*)d_c, (int)ldc, W + (size_t)N * s, W + (size_t)2 * N * s, N);
      deriv_weights(h->st, h->nx, h->ny, s, mu, N, W + (size_t)3 * N * s, W + (size_t)4 * N * s, N);
      exact_fwd(h, W, N, 5 * s, E, M);
      // r = f - A c (in place over the first block)
      axpy2(h->st, M, s, -2.0, E, M, E, M);
      axpy2(h->st, M, s, 1.0, (const double2*)d_f, (int)ldf, E, M);
      grad_combine(h->st, M, s, lam, (int)ldl, E + (size_t)M * s, E + (size_t)2 * M * s, E + (size_t)3 * M * s,
                   E + (size_t)4 * M * s, E, M, d_gx, d_gy);
    }
    NH_CK(cudaStreamSynchronize(h->st));
    h->scr.release(mk);
  });
}

nudft2_status nudft2_hss_plsqr(nudft2_hss_t h, const void* d_f, int64_t ldf, int nrhs, void* d_c, int64_t ldc,
                               double tol, int maxit, int* iters, double* relres, void* stream) {
  return guard([&] {
    NH_REQUIRE(h != nullptr, ST_ESTATE, "plsqr: no handle");
    NH_REQUIRE(h->factored, ST_ESTATE, "plsqr before factor");
    NH_REQUIRE(nrhs >= 1 && d_f && d_c && ldf >= h->M && ldc >= h->N && tol > 0 && maxit >= 1, ST_EINVAL,
               "plsqr: bad arguments");
    enter(h, stream);
    ensure_factors(h);
    int it = 0;
    double rr = -1;
    do_plsqr(h, (const double2*)d_f, ldf, nrhs, (double2*)d_c, ldc, tol, maxit, &it, &rr);
    NH_CK(cudaStreamSynchronize(h->st));
    if (iters) *iters = it;
    if (relres) *relres = rr;
  });
}

nudft2_status nudft2_hss_checkpoint(nudft2_hss_t h, int levels, void* stream) {
  return guard([&] {
    NH_REQUIRE(h != nullptr, ST_ESTATE, "checkpoint: no handle");
    NH_REQUIRE(h->factored, ST_ESTATE, "checkpoint before factor");
    NH_REQUIRE(levels >= 0, ST_EINVAL, "checkpoint: levels must be >= 0");
    enter(h, stream);
    h->g64.clear();            // captured solves refer to the factors handed back here
    h->g32.clear();
    if (h->h64) h->h64->checkpoint(levels);
    else h->h32->checkpoint(levels);
  });
}

nudft2_status nudft2_hss_info(nudft2_hss_t h, nudft2_info* info) {
  return guard([&] {
    NH_REQUIRE(h && info, ST_EINVAL, "info: NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->M = h->M; info->nx = h->nx; info->ny = h->ny; info->levels = h->L; info->prec = h->opt.prec;
    std::vector<int> lr = h->h64 ? h->h64->level_ranks() : h->h32->level_ranks();
    info->max_rank = h->h64 ? h->h64->max_rank() : h->h32->max_rank();
    for (size_t i = 0; i < lr.size() && i < 16; ++i) info->level_rank[i] = lr[i];
    info->t_build_ms = h->t_build;
    info->t_factor_ms = h->t_factor;
    info->t_solve_ms = h->t_solve;
    info->refine_iters = h->iters;
    info->refine_relres = h->relres;
    info->device_bytes = h->keep.reserved() + h->scr.reserved() + (h->h64 ? h->h64->bytes() : h->h32->bytes());
    info->launches = h->ops->launches() + (h->h64 ? h->h64->ops().launches() : h->h32->ops().launches());
    info->gemm_tuned = gemm_tune_entries();
    info->solve_graphs = h->graphs_ok;
    info->solve_graph_failures = h->graphs_failed;
    info->solve_replays = h->replays;
    info->checkpointed_levels = h->h64 ? h->h64->dropped_levels() : h->h32->dropped_levels();
  });
}

nudft2_status nudft2_hss_kstats(nudft2_hss_t h, nudft2_kstat* out, int max, int* n) {
  return guard([&] {
    NH_REQUIRE(h && out && n && max >= 0, ST_EINVAL, "kstats: NULL argument");
    // The handle's own FP64 operations (exact applies, DFTs) and the HSS operations.  In MIXED
    // mode the HSS runs in FP32, so the FP64 classes are reported apart, with a "_fp64" suffix:
    // they run on a different pipe.
    Prof* ps[2] = {h->h64 ? &h->h64->ops().prof : &h->h32->ops().prof, &h->ops->prof};
    const bool split = !h->h64;
    KStat acc[2][K_NCLASS];
    for (int q = 0; q < 2; ++q) {
      ps[q]->collect();
      KStat* a = acc[split ? q : 0];
      for (int c = 0; c < K_NCLASS; ++c) {
        a[c].ms += ps[q]->stats[c].ms;
        a[c].flops += ps[q]->stats[c].flops;
        a[c].bytes += ps[q]->stats[c].bytes;
        a[c].launches += ps[q]->stats[c].launches;
      }
    }
    int k = 0;
    for (int q = 0; q < (split ? 2 : 1); ++q)
      for (int c = 0; c < K_NCLASS && k < max; ++c) {
        if (acc[q][c].launches == 0) continue;
        std::memset(&out[k], 0, sizeof(out[k]));
        std::string name = kclass_name(c);
        if (q == 1) name += "_fp64";
        std::strncpy(out[k].name, name.c_str(), sizeof(out[k].name) - 1);
        out[k].ms = acc[q][c].ms;
        out[k].flops = acc[q][c].flops;
        out[k].bytes = acc[q][c].bytes;
        out[k].launches = acc[q][c].launches;
        ++k;
      }
    *n = k;
  });
}

nudft2_status nudft2_la_tsvd(int prec, void* d_ct, int64_t w, int64_t r, int64_t ldct, double eps, void* d_p,
                             int64_t ldp, int* rank, double* h_sigma, void* stream) {
  return guard([&] {
    NH_REQUIRE(d_ct && d_p && rank && h_sigma && w >= 0 && r >= 0 && ldct >= std::max<int64_t>(w, 1) &&
                   ldp >= std::max<int64_t>(r, 1) && eps > 0,
               ST_EINVAL, "la_tsvd: bad arguments");
    if (prec == NUDFT2_FP64)
      la_tsvd<double>(d_ct, (int)w, (int)r, (int)ldct, eps, d_p, (int)ldp, rank, h_sigma, (cudaStream_t)stream);
    else
      la_tsvd<float>(d_ct, (int)w, (int)r, (int)ldct, eps, d_p, (int)ldp, rank, h_sigma, (cudaStream_t)stream);
  });
}

nudft2_status nudft2_la_qr(int prec, void* d_a, int64_t m, int64_t n, int64_t lda, void* d_q, int64_t ldq,
                           int grouped, void* stream) {
  return guard([&] {
    NH_REQUIRE(d_a && d_q && m >= 1 && n >= 1 && lda >= m && ldq >= m, ST_EINVAL, "la_qr: bad arguments");
    if (prec == NUDFT2_FP64)
      la_qr<double>(d_a, (int)m, (int)n, (int)lda, d_q, (int)ldq, grouped, (cudaStream_t)stream);
    else
      la_qr<float>(d_a, (int)m, (int)n, (int)lda, d_q, (int)ldq, grouped, (cudaStream_t)stream);
  });
}

void nudft2_test_fail_alloc(long long k) { fault_alloc_countdown().store(k > 0 ? k : 0); }

nudft2_status nudft2_la_qr_apply(int prec, void* d_a, int64_t m, int64_t n, int64_t lda, void* d_c, int64_t s,
                                 int64_t ldc, int conj, int grouped, void* stream) {
  return guard([&] {
    NH_REQUIRE(d_a && m >= 1 && n >= 1 && lda >= m && s >= 0 && (s == 0 || (d_c && ldc >= m)) && m < (1LL << 31) &&
                   n < (1LL << 31) && s < (1LL << 31),
               ST_EINVAL, "la_qr_apply: bad arguments");
    if (prec == NUDFT2_FP64)
      la_qr_apply<double>(d_a, (int)m, (int)n, (int)lda, d_c, (int)s, (int)ldc, conj != 0, grouped,
                          (cudaStream_t)stream);
    else
      la_qr_apply<float>(d_a, (int)m, (int)n, (int)lda, d_c, (int)s, (int)ldc, conj != 0, grouped,
                         (cudaStream_t)stream);
  });
}

nudft2_status nudft2_la_gemm(int prec, int opa, int opb, int64_t m, int64_t n, int64_t k, double alpha,
                             const void* d_a, int64_t lda, int64_t stride_a, const void* d_b, int64_t ldb,
                             int64_t stride_b, double beta, void* d_c, int64_t ldc, int64_t stride_c, int batch,
                             void* stream) {
  return guard([&] {
    const bool ok_op = opa >= 0 && opa <= 2 && opb >= 0 && opb <= 2;
    const int64_t ra = opa == 0 ? m : k, rb = opb == 0 ? k : n;
    NH_REQUIRE(ok_op && (k == 0 || (d_a && d_b)) && d_c && m >= 1 && n >= 1 && k >= 0 && batch >= 1 && lda >= std::max<int64_t>(ra, 1) &&
                   ldb >= std::max<int64_t>(rb, 1) && ldc >= m && stride_a >= 0 && stride_b >= 0 && stride_c >= 0 &&
                   m < (1LL << 31) && n < (1LL << 31) && k < (1LL << 31) && (int64_t)m * n < (1LL << 31),
               ST_EINVAL, "la_gemm: bad arguments");
    if (prec == NUDFT2_FP64)
      la_gemm<double>(opa, opb, (int)m, (int)n, (int)k, alpha, d_a, (int)lda, stride_a, d_b, (int)ldb, stride_b,
                      beta, d_c, (int)ldc, stride_c, batch, (cudaStream_t)stream);
    else
      la_gemm<float>(opa, opb, (int)m, (int)n, (int)k, alpha, d_a, (int)lda, stride_a, d_b, (int)ldb, stride_b,
                     beta, d_c, (int)ldc, stride_c, batch, (cudaStream_t)stream);
  });
}

nudft2_status nudft2_hss_build_batched(int count, const double* const* d_x, const double* const* d_y,
                                       const int64_t* M, const int* nx, const int* ny, const nudft2_opts* opts,
                                       int factor, int threads, void* stream, nudft2_hss_t* out,
                                       nudft2_status* status) {
  if (count < 1 || !d_x || !d_y || !M || !nx || !ny || !out) {
    g_err = "build_batched: bad arguments";
    return NUDFT2_EINVAL;
  }
  std::vector<nudft2_status> st((size_t)count, NUDFT2_OK);
  std::vector<std::string> msg((size_t)count);
  auto r = guard([&] {
    run_pool(count, threads, [&](int i) {
      nudft2_hss_t h = nullptr;
      nudft2_status s = nudft2_hss_build(d_x[i], d_y[i], M[i], nx[i], ny[i], opts ? &opts[i] : nullptr, stream, &h);
      if (s == NUDFT2_OK && factor) s = nudft2_hss_factor(h, stream);
      if (s != NUDFT2_OK) {
        msg[i] = nudft2_last_error();
        if (h) nudft2_hss_free(h);
        h = nullptr;
      }
      st[i] = s;
      out[i] = h;
    });
  });
  if (r != NUDFT2_OK) return r;
  if (status)
    for (int i = 0; i < count; ++i) status[i] = st[i];
  return batch_result(st, msg);
}

nudft2_status nudft2_hss_solve_batched(int count, const nudft2_hss_t* h, const void* const* d_f, const int64_t* ldf,
                                       const int* nrhs, void* const* d_c, const int64_t* ldc, int threads,
                                       void* stream, nudft2_status* status) {
  if (count < 1 || !h || !d_f || !ldf || !nrhs || !d_c || !ldc) {
    g_err = "solve_batched: bad arguments";
    return NUDFT2_EINVAL;
  }
  std::vector<nudft2_status> st((size_t)count, NUDFT2_OK);
  std::vector<std::string> msg((size_t)count);
  auto r = guard([&] {
    run_pool(count, threads, [&](int i) {
      st[i] = nudft2_hss_solve(h[i], d_f[i], ldf[i], nrhs[i], d_c[i], ldc[i], stream);
      if (st[i] != NUDFT2_OK) msg[i] = nudft2_last_error();
    });
  });
  if (r != NUDFT2_OK) return r;
  if (status)
    for (int i = 0; i < count; ++i) status[i] = st[i];
  return batch_result(st, msg);
}

nudft2_status nudft2_hss_run_batched(int count, const double* const* d_x, const double* const* d_y,
                                     const int64_t* M, const int* nx, const int* ny, const nudft2_opts* opts,
                                     const void* const* d_f, const int64_t* ldf, const int* nrhs, void* const* d_c,
                                     const int64_t* ldc, int threads, void* stream, nudft2_status* status) {
  if (count < 1 || !d_x || !d_y || !M || !nx || !ny || !d_f || !ldf || !nrhs || !d_c || !ldc) {
    g_err = "run_batched: bad arguments";
    return NUDFT2_EINVAL;
  }
  // largest problems first, so that the last ones to start are the short ones
  std::vector<int> order((size_t)count);
  for (int i = 0; i < count; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)M[a] * std::sqrt((double)nx[a] * ny[a]) > (double)M[b] * std::sqrt((double)nx[b] * ny[b]);
  });
  std::vector<nudft2_status> st((size_t)count, NUDFT2_OK);
  std::vector<std::string> msg((size_t)count);
  MemoryRetry retry;
  auto r = guard([&] {
    run_pool(count, threads, [&](int k) {
      const int i = order[(size_t)k];
      retry.begin();
      // out of device memory while other problems hold theirs: wait for one of them to finish, then
      // start this one again (MemoryRetry); every handle of a failed attempt is freed first
      const int s = retry.run(
          [&]() -> int {
            nudft2_hss_t h = nullptr;
            nudft2_status a = nudft2_hss_build(d_x[i], d_y[i], M[i], nx[i], ny[i], opts ? &opts[i] : nullptr, stream, &h);
            if (a == NUDFT2_OK) a = nudft2_hss_factor(h, stream);
            if (a == NUDFT2_OK) a = nudft2_hss_solve(h, d_f[i], ldf[i], nrhs[i], d_c[i], ldc[i], stream);
            if (a != NUDFT2_OK) msg[(size_t)i] = nudft2_last_error();
            if (h) nudft2_hss_free(h);
            return (int)a;
          },
          (int)NUDFT2_ENOMEM);
      st[(size_t)i] = (nudft2_status)s;
      retry.end();
    });
  });
  if (r != NUDFT2_OK) return r;
  if (status)
    for (int i = 0; i < count; ++i) status[i] = st[(size_t)i];
  return batch_result(st, msg);
}

nudft2_status nudft2_hss_save(nudft2_hss_t h, const char* path) {
  return guard([&] {
    NH_REQUIRE(h != nullptr && path != nullptr, ST_EINVAL, "save: bad arguments");
    NH_REQUIRE(h->factored, ST_ESTATE, "save before factor");
    ensure_factors(h);
    NH_CK(cudaStreamSynchronize(h->st));
    std::unique_ptr<FILE, int (*)(FILE*)> f(std::fopen(path, "wb"), &std::fclose);
    NH_REQUIRE(f != nullptr, ST_EINVAL, "save: cannot open the file");
    auto wr = [&](const void* p, size_t n) {
      NH_REQUIRE(n == 0 || std::fwrite(p, 1, n, f.get()) == n, ST_EINVAL, "save: write failed");
    };
    const uint32_t head[4] = {STORE_MAGIC0, STORE_MAGIC1, STORE_VERSION, (uint32_t)sizeof(nudft2_opts)};
    wr(head, sizeof(head));
    wr(&h->opt, sizeof(nudft2_opts));
    const int64_t M = h->M;
    const int32_t dims[4] = {h->nx, h->ny, h->pl.Lx, h->pl.Ly};
    wr(&M, sizeof(M));
    wr(dims, sizeof(dims));
    std::vector<double> hx((size_t)M), hy((size_t)M);
    NH_CK(cudaMemcpy(hx.data(), h->pl.x, M * sizeof(double), cudaMemcpyDeviceToHost));
    NH_CK(cudaMemcpy(hy.data(), h->pl.y, M * sizeof(double), cudaMemcpyDeviceToHost));
    wr(hx.data(), hx.size() * sizeof(double));
    wr(hy.data(), hy.size() * sizeof(double));
    if (h->h64) h->h64->save(f.get());
    else h->h32->save(f.get());
  });
}

nudft2_status nudft2_hss_load(const char* path, void* stream, nudft2_hss_t* out) {
  nudft2_hss_s* h = nullptr;
  double* dxy = nullptr;
  auto st = guard([&] {
    NH_REQUIRE(path != nullptr && out != nullptr, ST_EINVAL, "load: bad arguments");
    *out = nullptr;
    std::unique_ptr<FILE, int (*)(FILE*)> f(std::fopen(path, "rb"), &std::fclose);
    NH_REQUIRE(f != nullptr, ST_EINVAL, "load: cannot open the file");
    auto rd = [&](void* p, size_t n) {
      NH_REQUIRE(n == 0 || std::fread(p, 1, n, f.get()) == n, ST_EINVAL, "load: file truncated or corrupt");
    };
    // header and points: checked on the host before any device work
    uint32_t head[4];
    rd(head, sizeof(head));
    NH_REQUIRE(head[0] == STORE_MAGIC0 && head[1] == STORE_MAGIC1, ST_EINVAL, "load: not a factor store");
    NH_REQUIRE(head[2] == STORE_VERSION && head[3] == (uint32_t)sizeof(nudft2_opts), ST_EINVAL,
               "load: factor store of another version");
    nudft2_opts opt;
    rd(&opt, sizeof(opt));
    int64_t M = 0;
    int32_t dims[4];
    rd(&M, sizeof(M));
    rd(dims, sizeof(dims));
    const int nx = dims[0], ny = dims[1], Lx = dims[2], Ly = dims[3];
    NH_REQUIRE(nx >= 1 && ny >= 1 && (int64_t)nx * ny <= (1LL << 26) && M >= (int64_t)nx * ny && M < (1LL << 31),
               ST_EINVAL, "load: bad problem sizes");
    NH_REQUIRE(Lx >= 1 && Lx <= 12 && Ly >= 1 && Ly <= 12 && (nx >> Lx) >= 1 && (ny >> Ly) >= 1, ST_EINVAL,
               "load: bad tree depths");
    NH_REQUIRE(opt.prec == NUDFT2_FP64 || opt.prec == NUDFT2_MIXED, ST_EINVAL, "load: unknown precision");
    std::vector<double> hxy((size_t)2 * M);
    rd(hxy.data(), hxy.size() * sizeof(double));
    for (double v : hxy)
      NH_REQUIRE(std::isfinite(v) && v >= 0 && v < 1, ST_EINVAL, "load: points must be finite and lie in [0,1)^2");
    NH_CK(cudaMalloc(&dxy, hxy.size() * sizeof(double)));
    NH_CK(cudaMemcpy(dxy, hxy.data(), hxy.size() * sizeof(double), cudaMemcpyHostToDevice));
    h = new nudft2_hss_s();
    init_handle(h, dxy, dxy + M, M, nx, ny, opt, Lx, Ly, stream);
    NH_CK(cudaStreamSynchronize(h->st));
    if (opt.prec == NUDFT2_FP64) {
      h->h64.reset(new Hss<double>(h->st, &h->pl));
      h->h64->load(f.get());
    } else {
      h->h32.reset(new Hss<float>(h->st, &h->pl));
      h->Ax32 = h->keep.arr<float2>((size_t)M * nx);
      h->Ay32 = h->keep.arr<float2>((size_t)M * ny);
      convert_gather<double, float>(h->st, h->Ax, (int)M, nullptr, (int)M, nx, h->Ax32, (int)M, 1.0);
      convert_gather<double, float>(h->st, h->Ay, (int)M, nullptr, (int)M, ny, h->Ay32, (int)M, 1.0);
      h->h32->load(f.get());
    }
    const bool prof = (opt.flags & NUDFT2_FLAG_PROFILE) != 0;
    h->ops->prof.on = prof;
    if (h->h64) h->h64->ops().prof.on = prof;
    else h->h32->ops().prof.on = prof;
    NH_CK(cudaStreamSynchronize(h->st));
    h->factored = true;
    *out = h;
  });
  if (dxy) cudaFree(dxy);
  if (st != NUDFT2_OK && h) {
    const std::string msg = g_err;
    nudft2_hss_free(h);
    g_err = msg;
  }
  return st;
}

void nudft2_hss_free(nudft2_hss_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  cudaStream_t st = h->st;
  cudaEvent_t ev = h->join;
  delete h;                       // arenas release their chunks on st
  cudaStreamSynchronize(st);
  if (ev) cudaEventDestroy(ev);
  if (st) cudaStreamDestroy(st);
}

}  // extern "C"
