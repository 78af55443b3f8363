// Batched complex dense linear algebra on variable-size problems.
//
// Every routine takes a host vector of descriptors (one per independent problem), uploads
// it, and covers the whole batch with ONE launch per algorithmic step, so each tree level
// of the HSS algorithms costs a fixed number of launches regardless of how many nodes it
// has.  Matrices are column major complex (double2 / float2).
#pragma once
#include <vector>

#include "common.cuh"

namespace nh {

enum Op { OP_N = 0, OP_T = 1, OP_C = 2 };

template <typename R> struct GemmD {
  const cplx<R>* A; const cplx<R>* B; cplx<R>* C;
  int m, n, k, lda, ldb, ldc;
  int opA, opB;
  R alpha, beta;
};

// dst(i,j) = alpha * rs[i] * op(src)(i,j) (+ beta * dst when beta != 0); op in {N, T, C};
// rs == nullptr means no row scaling.
template <typename R> struct CopyD {
  const cplx<R>* src; cplx<R>* dst;
  int m, n, lds, ldd, op;
  R alpha, beta;
  const R* rs = nullptr;
};

// dst block (ma*mb x na*nb) = alpha * kron(A, B); A == nullptr means the identity of size
// ma (= na), likewise for B.  Entry ((i*mb + k), (j*nb + l)) = A(i,j) * B(k,l).
template <typename R> struct KronD {
  const cplx<R>* A; const cplx<R>* B; cplx<R>* dst;
  int ma, na, lda, mb, nb, ldb, ldd;
  R alpha;
};

// Row-wise Kronecker (face-splitting) product: dst(j, a*nb + s) = A(j, a) * B(j, s).
template <typename R> struct FaceD {
  const cplx<R>* A; const cplx<R>* B; cplx<R>* dst;
  int m, na, nb, lda, ldb, ldd;
};

// dst(i, :) = src(idx[i] + base, :) for i < m, n columns.
template <typename R> struct GatherD {
  const cplx<R>* src; cplx<R>* dst; const int* idx;
  int m, n, lds, ldd, base;
};

// In-place Householder QR of A (m x n).  Output: R in the upper trapezoid of A, explicit
// unit-lower-trapezoidal reflectors in V (m x min(m,n), caller zero-fills), real tau and
// the per-panel compact-WY factors Tp (nb x nb for every panel, stacked by panel).
template <typename R> struct QRD {
  cplx<R>* A; int lda; int m, n;
  cplx<R>* V; int ldv;
  R* tau;
  cplx<R>* Tp;   // ceil(k/nb) blocks of nb*nb
  cplx<R>* W;    // scratch 2*nb x n
};

// A QR factor kept for later applications: Q = H_0 ... H_{k-1}, applied panel by panel, or
// -- after group_wy() -- by groups of GW columns with one merged compact-WY T per group.
template <typename R> struct QFac {
  cplx<R>* V = nullptr; int ldv = 1; int m = 0, k = 0;
  cplx<R>* Tp = nullptr;
  cplx<R>* Tg = nullptr;   // ceil(k/GW) blocks of GW*GW when grouped
};

// Per-kernel-class accounting (CUDA events around each launch on the launching stream),
// enabled per handle for measurement runs.  flops are the algorithmic counts of the launch.
// K_SWEEP: one whole URV solve (Sec. 2.3 sweeps) replayed from its CUDA graph, with the bytes of
// the factors it streams.
// K_GEMM_TC: the tensor-core complex GEMM (operand packing included); K_GEMM: the CUDA-core one.
// K_JACOBI_TC: the blocked Jacobi step with its Gram and update products on the tensor cores.
enum KClass { K_GEMM = 0, K_QR_PANEL = 1, K_JACOBI = 2, K_OTHER = 3, K_QRCP = 4, K_SWEEP = 5, K_GEMM_TC = 6,
              K_JACOBI_TC = 7, K_NCLASS = 8 };
struct KStat { double ms = 0, flops = 0, bytes = 0; int launches = 0; };
const char* kclass_name(int c);

class Prof {
 public:
  ~Prof();
  bool on = false;
  void begin(cudaStream_t st);
  // nlaunch: kernel launches inside the region (per-launch averages use it)
  void end(cudaStream_t st, int cls, double flops, double bytes, int nlaunch = 1);
  void collect();   // synchronises the recorded events and accumulates
  void add_flops(int cls, double f) { if (on) stats[cls].flops += f; }
  KStat stats[K_NCLASS];

 private:
  struct Pend { int cls; cudaEvent_t a, b; double flops, bytes; int n; };
  cudaEvent_t get();
  std::vector<cudaEvent_t> pool_;
  std::vector<Pend> pend_;
  cudaEvent_t cur_ = nullptr;
};

// Launch the batched GEMM kernel on caller-provided device descriptors (no allocation, no
// copies): desc[np] and the exclusive tile prefix pre[np] already live in device memory.
// Every descriptor must have opA == opB == OP_N.
void gemm_launch_raw(const GemmD<double>* desc, const int* pre, int np, int tiles, cudaStream_t st);
int gemm_tiles(const GemmD<double>& g);

// Tensor-core (tcgen05, 3xTF32) complex FP32 GEMM: used in place of the CUDA-core kernel for
// batches of large FP32 products (on by default; NH_GEMM_TC=0 turns it off).  cls is the
// operand-layout class (2 * (opA != N) + (opB != N)).  The operands are packed into split TF32
// planes in scratch memory from `ar`; descriptor arrays are uploaded through `stage(ctx, src,
// bytes)`.  Returns the number of kernel launches.  gemm_tc_error reads (and optionally clears)
// the flag set when one of the kernel's bounded waits ran out.
bool gemm_tc_enabled();
int gemm_tc_run(const std::vector<GemmD<float>>& d, int cls, Arena& ar, cudaStream_t st,
                void* (*stage)(void*, const void*, size_t), void* ctx);
int gemm_tc_error(bool reset);
// Flag of the tensor-core Jacobi step's bounded waits (read, optionally cleared).
int jacobi_tc_error(bool reset);
// Number of shape classes the GEMM autotuner has measured in this process.
int gemm_tune_entries();

template <typename R> class Ops {
 public:
  explicit Ops(cudaStream_t s, Arena* scratch) : st_(s), ar_(scratch) {}
  Prof prof;
  cudaStream_t stream() const { return st_; }
  Arena* scratch() { return ar_; }
  static constexpr int NB = 32;   // Householder panel width
  static constexpr int GW = 256;  // columns per merged compact-WY group used for applications

  void gemm(const std::vector<GemmD<R>>& d);
  void copy(const std::vector<CopyD<R>>& d);
  void kron(const std::vector<KronD<R>>& d);
  void face(const std::vector<FaceD<R>>& d);
  void gather(const std::vector<GatherD<R>>& d);
  void set_identity(const std::vector<Mat<R>>& d);   // zero then unit diagonal
  // Householder QR of every A in place; returns the stored factors (V, Tp from the arena `keep`).
  std::vector<QFac<R>> qr(const std::vector<Mat<R>>& A, Arena& keep);
  // Merge the panel T's of every factor into one T per group of GW columns:
  // T_g = (striu(V_g^* V_g) + diag(1/tau))^{-1} (the compact-WY identity), from `keep`.
  void group_wy(std::vector<QFac<R>>& Q, Arena& keep);
  // C <- Q C (conj=false) or Q^* C (conj=true), from the left.  C has Q.m rows.
  void apply_q_left(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj);
  // The same product by streaming kernels (one pass over each block of reflectors per chunk of
  // up to 16 columns of C, no GEMM tiles): the form the solve sweeps use for few right-hand sides.
  void apply_q_stream(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj);
  // apply_q_stream, or apply_q_left when NH_SWEEP_STREAM=0 (for comparison runs)
  void apply_q_sweep(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj);
  // C <- C Q (conj=false) or C Q^*, from the right.  C has Q.m columns.
  void apply_q_right(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj);
  // X <- inverse of the upper triangle of A (square); X must not alias A.
  void trinv(const std::vector<Mat<R>>& A, const std::vector<Mat<R>>& X);
  // Truncated SVD through the conjugate transpose Ct = C^* (w x r) of each C (r x w).
  // Ct is overwritten.  Returns left singular vectors P (r x rank) allocated from `keep`
  // and the retained singular values (rank, host copy) with sigma_i > eps * sigma_1.
  void tsvd_ct(const std::vector<Mat<R>>& Ct, double eps, Arena& keep,
               std::vector<Mat<R>>& P, std::vector<std::vector<double>>& S);

  // Row interpolative decomposition of every basis B_i (mc_i x q_i, q_i <= 1024), passed as
  // W_i = B_i^* (q_i x mc_i, overwritten by its column-pivoted QR): rank r_i = the leading pivots
  // with |R_kk| > tol |R_00| (at least 1 when mc_i >= 1), skeleton sk_i = the first r_i pivots
  // (host), interpolation matrix T_i (mc_i x r_i, from `keep`) with T_i(sk_i, :) = I and
  // B_i ~= T_i B_i(sk_i, :).  fadi.cu.
  void row_id(const std::vector<Mat<R>>& W, double tol, Arena& keep, std::vector<Mat<R>>& T,
              std::vector<std::vector<int>>& sk);

  int launches() const { return launches_; }
  void count(int n = 1) { launches_ += n; }
  // Capture mode: host->device descriptor copies are staged in `pool` (kept alive with the graph).
  void set_capture(PinnedPool* pool) { pool_ = pool; }
  // host bytes staged to the device since the last reset (sizes the pinned pool of a capture)
  void reset_staged() { staged_ = 0; }
  size_t staged() const { return staged_; }
  int* upload_ints(const std::vector<int>& v);
  // host -> device copy of bytes into the scratch arena (capture-safe), for launchers outside
  // this class; ctx is the Ops object
  static void* stage_cb(void* ctx, const void* src, size_t bytes) { return ((Ops*)ctx)->stage(src, bytes); }

 private:
  void gemm_class(const std::vector<GemmD<R>>& d, int cls);   // one operand-layout class
  int gemm_pick(const std::vector<GemmD<R>>& d, int cls);     // kernel kind: static rule or autotuner
  void gemm_run(const std::vector<GemmD<R>>& d, int cls, int kind);
  // rank-revealing column-pivoted QR of every A (in place: R in the upper trapezoid of the first
  // peff rows, zero below its diagonal) with pivots chosen blockwise on random sketches; perm[i]
  // (A[i].n entries, device) receives the column order; stops at the rank the truncated SVD at
  // eps can use (every remaining column norm <= 0.01 eps max column norm).
  void qrcp_sketch(const std::vector<Mat<R>>& A, const std::vector<int*>& perm, double eps, std::vector<int>& peff);
  template <int S> void apply_q_stream_s(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj);
  template <typename D> D* upload(const std::vector<D>& v);
  void* stage(const void* src, size_t bytes);
  cudaStream_t st_;
  Arena* ar_;
  PinnedPool* pool_ = nullptr;
  size_t staged_ = 0;
  int launches_ = 0;
};

}  // namespace nh
