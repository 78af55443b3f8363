// HSS construction (1D compression, face-splitting assembly, recompression), URV
// factorization and URV solve for the transformed 2D NUDFT matrix G~ = A F^{-1}.
#pragma once
#include <complex>
#include <cstdio>
#include <map>
#include <memory>
#include <tuple>
#include <vector>

#include "la.cuh"
#include "nudft.cuh"

namespace nh {

// ---------------------------------------------------------------- trees and point order
// 1D binary trees T^x (depth Lx) and T^y (depth Ly) over the column index sets (bisection of the
// periodic interval, Sec. 2.4) and their face-splitting product T = T^x . T^y (Def. 3.3), of
// depth L = max(Lx, Ly).  A level-l node splits in x when l < Lx and in y when l < Ly: four
// children when both split (Def. 3.3 (4)), two when only one does (Def. 3.3 (2), (3): the other
// 1D node is already a leaf).  The fan-out is the same for every node of a level.  Child c of node
// p of level l is node fan[l] * p + c of level l + 1; with both splits c = 2 i + j for the x child
// i and the y child j (children order (1,1),(1,2),(2,1),(2,2) of the proof of Thm. 3.5).
struct Tree1D {
  int n = 0, L = 0;
  std::vector<std::vector<int>> c0, c1;   // column range of node (l, i)
  std::vector<std::vector<int>> r0, m;    // row range in this dimension's sorted point order
  std::vector<int> leaf_of_col;           // column -> leaf index
};

struct Plan {
  int M = 0, nx = 0, ny = 0, L = 0, N = 0;
  int Lx = 0, Ly = 0;                     // depths of T^x and T^y; L = max(Lx, Ly)
  Tree1D tx, ty;
  std::vector<int> fan;                   // fan[l]: children of every level-l node (l < L)
  std::vector<int> nn;                    // nodes per level
  std::vector<std::vector<int>> ix, iy;   // (l, p) -> node of T^x at level lvx(l), of T^y at lvy(l)
  int lvx(int l) const { return l < Lx ? l : Lx; }
  int lvy(int l) const { return l < Ly ? l : Ly; }
  bool splitx(int l) const { return l < Lx; }
  bool splity(int l) const { return l < Ly; }
  // x child and y child (0 or 1; 0 when that dimension does not split) of child c of a level-l node
  int cxi(int l, int c) const { return splitx(l) ? (splity(l) ? c >> 1 : c) : 0; }
  int cyj(int l, int c) const { return splity(l) ? (splitx(l) ? c & 1 : c) : 0; }
  // 2D: per level l, per node p: rows [r0, r0+m) in 2D order, columns [c0, c0+nc) in tree order
  std::vector<std::vector<int>> r0, m, c0, nc;
  std::vector<int> leaf_lx, leaf_ly;      // per leaf p: 1D leaf indices
  // device arrays (owned by the handle's persistent arena)
  double *x = nullptr, *y = nullptr;      // caller order
  double *x2 = nullptr, *y2 = nullptr;    // 2D leaf order
  double *xo = nullptr, *yo = nullptr;    // x-bin order / y-bin order
  int *perm2 = nullptr;                   // 2D position -> caller index
  int *posx = nullptr, *posy = nullptr;   // 2D position -> position in x-order / y-order
  int *colmap = nullptr;                  // tree column -> lexicographic (kx*ny + ky)
};

// Build the plan: bins points on the device, sorts them (stable counting sort) into the
// three orders and reads the per-bin counts back to size the trees.
void make_plan(cudaStream_t st, Arena& keep, Arena& scr, const double* d_x, const double* d_y, int M, int nx, int ny,
               int Lx, int Ly, Plan& pl);

// ---------------------------------------------------------------- HSS generators and URV factors
template <typename R> struct Gen1D {    // one node of a 1D HSS (Sec. 2.2, Def. 2.2)
  int ru = 0, rv = 0;
  Mat<R> U, V, P, R_, W, Bs, Rst, Wst;  // U leaf; V explicit; P = U^* G(J,:); R_,W transfer; Bs = B_{this,sibling}
};

template <typename R> struct Node2 {
  int ku = 0, kv = 0;                   // basis sizes (ranks after recompression)
  Mat<R> D, U, V;                       // leaf generators
  Mat<R> R_, W;                         // transfer to the parent
  Mat<R> B[4];                          // B_{this, sibling c'}; B[self] unused
  // recompression temporaries
  Mat<R> F, G;
  int pu = 0, pv = 0;
  std::vector<double> SU, SV;
  // URV factor (Sec. 2.3)
  bool omega = false;
  QFac<R> Om, Qv, P;
  int m = 0, n = 0, mc = 0, n1 = 0, rows2 = 0;
  Mat<R> Wk;                            // [U D] working matrix after factorization
  Mat<R> D11inv, V2;
};

// Plan of one node of the fADI + ID construction of a 1D HSS (fadi.cu), for a node of d columns
// out of n in its own frame (first column 0).  side 0: the row block G~(J, K^c); side 1: the
// column block G~(J^c, K).  The candidate basis row of a point (side 0) or a column (side 1) is
// a^T C with a = [exact part (ex.size() entries), z_1 .. z_J] (the fADI factor with the shifts
// alpha_i = exp(-2 pi i xa_i), beta_i = exp(-2 pi i xb_i)).
struct FadiPlan {
  int J = 0;
  std::vector<int> ex;                    // side 0: exact columns; side 1: exact unit columns
  std::vector<double> xa, xb;             // shift positions in units of the circle
  std::vector<std::complex<double>> C;    // (ex.size() + J)^2, column major
  double ratio = 0;                       // bound on max_E |r| / min_F |r| of the shifts
  int q() const { return (int)ex.size() + J; }
};
constexpr int FADI_JMAX = 64;             // at most 64 shifts, so a basis has at most 65 columns
FadiPlan fadi_plan(int side, int d, int n, double eps1, int jmax);

template <typename R> class Hss {
 public:
  Hss(cudaStream_t st, const Plan* pl);
  // fadi: the 1D HSS approximations by fADI + interpolative decomposition (the construction the
  // paper cites for Alg. 1 step 1) instead of truncated SVDs of the kernel-entry blocks
  void build(double eps, bool fadi = false);
  void factor();
  // Per-level checkpointing: hand back the URV factors of the top `levels` levels (and the root);
  // ensure_factored() recomputes them from the generators and the kept factors of the levels below
  // (returns true when it did, i.e. device addresses of factors changed).
  void checkpoint(int levels);
  // Factor store: write every generator and URV factor (device -> file), or read them back into a
  // fresh object built on the same plan (file -> device) and mark it factored.  The file position
  // advances past this object's section.
  void save(FILE* f);
  void load(FILE* f);
  bool ensure_factored();
  int dropped_levels() const { return dropped_; }
  // y (N x s, tree column order) = G~_hss^+ f (f: M x s in 2D row order); both device
  void solve(const cplx<R>* f2, int ldf, int s, cplx<R>* ytree, int ldy);
  // f2 (M x s, 2D order) = (G~_hss^+)^* y (N x s, tree column order): the adjoint of solve()
  void solve_adj(const cplx<R>* ytree, int ldy, int s, cplx<R>* f2, int ldf);
  // y = G~_hss x (x: N x s tree order, y: M x s 2D order): the HSS matrix-vector product
  void matvec(const cplx<R>* x, int ldx, int s, cplx<R>* y, int ldy);
  // x = G~_hss^* y (y: M x s 2D order, x: N x s tree order): the adjoint of matvec()
  void matvec_adj(const cplx<R>* y, int ldy, int s, cplx<R>* x, int ldx);
  // Complex entries of the factors one URV solve streams (Householder vectors of Omega, P, Q_v
  // and the root, D11^{-1}, D12, U1, V2, B, R, the root R^{-1}); every one is read at least once
  // per right-hand-side batch.
  double solve_entries() const;
  int max_rank() const;
  std::vector<int> level_ranks() const;
  size_t bytes() const {
    size_t b = keep_.reserved() + (gen_ ? gen_->reserved() : 0);
    for (auto& a : fac_) b += a->reserved();
    return b;
  }
  Ops<R>& ops() { return ops_; }
  // While a solve is captured into a CUDA graph the scratch arena must not grow.
  void freeze_scratch(bool f) { scr_.freeze(f); }
  bool factored = false;

 private:
  void build_1d(const Tree1D& t, const double* xo, double eps, std::vector<std::vector<Gen1D<R>>>& g,
                Mat<R>& G);
  void build_1d_fadi(const Tree1D& t, const double* xo, double eps, std::vector<std::vector<Gen1D<R>>>& g);
  const FadiPlan& fadi_plan_of(int side, int d, int n, double eps1);
  void assemble_2d();
  void recompress(double eps);
  void factor_level(int l);
  void factor_root();
  void compact_generators();
  cudaStream_t st_;
  const Plan* pl_;
  Arena keep_, scr_, tmp_;
  Ops<R> ops_;
  std::vector<std::vector<Gen1D<R>>> gx_, gy_;
  Mat<R> Gx_, Gy_;
  std::vector<std::vector<Node2<R>>> t_;
  std::unique_ptr<Arena> gen_;                 // the final generators (after build)
  std::vector<std::unique_ptr<Arena>> fac_;   // factor storage per level (0 = root)
  int dropped_ = 0;                            // top levels whose factors were handed back
  std::map<std::tuple<int, int, int>, FadiPlan> fplans_;   // fADI plans by (side, d, n)
  // root factor
  QFac<R> Proot_;
  Mat<R> Droot_, Rinv_;
  int root_rows_ = 0, root_cols_ = 0;
};

}  // namespace nh
