// HSS construction, URV factorization and URV solve (see hss.cuh).
//
// Stage map (Li & Liu):
//   build_1d     -- HSS approximations of the transformed 1D matrices at eps/10 (Alg. 1, step 1),
//                   by kernel-entry evaluation and per-node truncated SVD compression
//                   (fadi.cu: build_1d_fadi, the fADI + interpolative decomposition route).
//   assemble_2d  -- generators of the face-splitting product on T^x . T^y from the constructive
//                   proof of Thm. 3.5 (leaf D, U, V; B, R, W from Kronecker products).
//   recompress   -- Sec. 2.2: bottom-up orthogonalization then top-down truncated-SVD compression.
//   factor       -- Sec. 2.3: size reduction, basis elimination, partial decomposition, merge,
//                   root QR.
//   solve        -- Sec. 2.3: bottom-up application of Omega^*, P^*; root least squares;
//                   top-down back substitution.
#include <algorithm>
#include <cstdio>
#include <cmath>

#include "hss.cuh"

namespace nh {

// =============================================================================== plan
static void make_tree(Tree1D& t, int n, int L) {
  t.n = n;
  t.L = L;
  t.c0.assign(L + 1, {});
  t.c1.assign(L + 1, {});
  t.c0[0] = {0};
  t.c1[0] = {n};
  for (int l = 1; l <= L; ++l) {
    for (size_t i = 0; i < t.c0[l - 1].size(); ++i) {
      const int a = t.c0[l - 1][i], b = t.c1[l - 1][i], h = a + (b - a) / 2;
      t.c0[l].push_back(a); t.c1[l].push_back(h);
      t.c0[l].push_back(h); t.c1[l].push_back(b);
    }
  }
  t.leaf_of_col.assign(n, 0);
  for (size_t i = 0; i < t.c0[L].size(); ++i) {
    NH_REQUIRE(t.c1[L][i] > t.c0[L][i], ST_EINVAL, "every 1D leaf needs at least one column (n >= 2^L)");
    for (int k = t.c0[L][i]; k < t.c1[L][i]; ++k) t.leaf_of_col[k] = (int)i;
  }
}

void make_plan(cudaStream_t st, Arena& keep, Arena& scr, const double* d_x, const double* d_y, int M, int nx, int ny,
               int Lx, int Ly, Plan& pl) {
  const int L = std::max(Lx, Ly);
  pl.M = M; pl.nx = nx; pl.ny = ny; pl.L = L; pl.N = nx * ny;
  pl.Lx = Lx; pl.Ly = Ly;
  make_tree(pl.tx, nx, Lx);
  make_tree(pl.ty, ny, Ly);
  // product tree (Def. 3.3): fan-out per level, node -> (T^x node, T^y node)
  pl.fan.assign(L + 1, 0);
  pl.nn.assign(L + 1, 1);
  pl.ix.assign(L + 1, {});
  pl.iy.assign(L + 1, {});
  pl.ix[0] = {0};
  pl.iy[0] = {0};
  for (int l = 0; l < L; ++l) {
    const int F = (pl.splitx(l) ? 2 : 1) * (pl.splity(l) ? 2 : 1);
    pl.fan[l] = F;
    pl.nn[l + 1] = pl.nn[l] * F;
    for (int p = 0; p < pl.nn[l]; ++p)
      for (int c = 0; c < F; ++c) {
        pl.ix[l + 1].push_back(pl.splitx(l) ? 2 * pl.ix[l][p] + pl.cxi(l, c) : pl.ix[l][p]);
        pl.iy[l + 1].push_back(pl.splity(l) ? 2 * pl.iy[l][p] + pl.cyj(l, c) : pl.iy[l][p]);
      }
  }
  const int nleaf = pl.nn[L];
  const int nlx = 1 << Lx, nly = 1 << Ly;
  std::vector<int> leafid((size_t)nlx * nly, 0);
  for (int p = 0; p < nleaf; ++p) leafid[(size_t)pl.ix[L][p] * nly + pl.iy[L][p]] = p;
  pl.x = keep.arr<double>(M);
  pl.y = keep.arr<double>(M);
  NH_CK(cudaMemcpyAsync(pl.x, d_x, M * sizeof(double), cudaMemcpyDeviceToDevice, st));
  NH_CK(cudaMemcpyAsync(pl.y, d_y, M * sizeof(double), cudaMemcpyDeviceToDevice, st));
  auto mk = scr.mark();
  int* lfx = scr.arr<int>(nx);
  int* lfy = scr.arr<int>(ny);
  int* lid = scr.arr<int>(leafid.size());
  NH_CK(cudaMemcpyAsync(lfx, pl.tx.leaf_of_col.data(), nx * sizeof(int), cudaMemcpyHostToDevice, st));
  NH_CK(cudaMemcpyAsync(lfy, pl.ty.leaf_of_col.data(), ny * sizeof(int), cudaMemcpyHostToDevice, st));
  NH_CK(cudaMemcpyAsync(lid, leafid.data(), leafid.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  int* k2 = scr.arr<int>(M);
  int* kx = scr.arr<int>(M);
  int* ky = scr.arr<int>(M);
  bin_points(st, pl.x, pl.y, M, nx, ny, lfx, lfy, lid, nly, k2, kx, ky);
  pl.perm2 = keep.arr<int>(M);
  int* permx = scr.arr<int>(M);
  int* permy = scr.arr<int>(M);
  int* c2 = scr.arr<int>(nleaf);
  int* cx = scr.arr<int>(nx);
  int* cy = scr.arr<int>(ny);
  counting_sort(st, scr, k2, M, nleaf, pl.perm2, c2);
  counting_sort(st, scr, kx, M, nx, permx, cx);
  counting_sort(st, scr, ky, M, ny, permy, cy);
  std::vector<int> h2(nleaf), hx(nx), hy(ny);
  NH_CK(cudaMemcpyAsync(h2.data(), c2, nleaf * sizeof(int), cudaMemcpyDeviceToHost, st));
  NH_CK(cudaMemcpyAsync(hx.data(), cx, nx * sizeof(int), cudaMemcpyDeviceToHost, st));
  NH_CK(cudaMemcpyAsync(hy.data(), cy, ny * sizeof(int), cudaMemcpyDeviceToHost, st));
  pl.x2 = keep.arr<double>(M); pl.y2 = keep.arr<double>(M);
  pl.xo = keep.arr<double>(M); pl.yo = keep.arr<double>(M);
  permute_double(st, pl.x, pl.perm2, M, pl.x2);
  permute_double(st, pl.y, pl.perm2, M, pl.y2);
  permute_double(st, pl.x, permx, M, pl.xo);
  permute_double(st, pl.y, permy, M, pl.yo);
  int* invx = scr.arr<int>(M);
  int* invy = scr.arr<int>(M);
  inverse_perm(st, permx, M, invx);
  inverse_perm(st, permy, M, invy);
  pl.posx = keep.arr<int>(M);
  pl.posy = keep.arr<int>(M);
  compose(st, invx, pl.perm2, M, pl.posx);
  compose(st, invy, pl.perm2, M, pl.posy);
  NH_CK(cudaStreamSynchronize(st));
  scr.release(mk);
  // 1D row ranges: rows of node (l,i) = points whose bin lies in [c0, c1)
  auto rows1d = [&](Tree1D& t, const std::vector<int>& cnt) {
    std::vector<int> pre(t.n + 1, 0);
    for (int k = 0; k < t.n; ++k) pre[k + 1] = pre[k] + cnt[k];
    t.r0.assign(t.L + 1, {});
    t.m.assign(t.L + 1, {});
    for (int l = 0; l <= t.L; ++l)
      for (size_t i = 0; i < t.c0[l].size(); ++i) {
        t.r0[l].push_back(pre[t.c0[l][i]]);
        t.m[l].push_back(pre[t.c1[l][i]] - pre[t.c0[l][i]]);
      }
  };
  rows1d(pl.tx, hx);
  rows1d(pl.ty, hy);
  // 2D rows and columns
  pl.r0.assign(L + 1, {}); pl.m.assign(L + 1, {}); pl.c0.assign(L + 1, {}); pl.nc.assign(L + 1, {});
  std::vector<int> rpre(nleaf + 1, 0), cpre(nleaf + 1, 0);
  pl.leaf_lx.assign(nleaf, 0);
  pl.leaf_ly.assign(nleaf, 0);
  for (int p = 0; p < nleaf; ++p) {
    const int lx = pl.ix[L][p], ly = pl.iy[L][p];
    pl.leaf_lx[p] = lx; pl.leaf_ly[p] = ly;
    rpre[p + 1] = rpre[p] + h2[p];
    cpre[p + 1] = cpre[p] + (pl.tx.c1[Lx][lx] - pl.tx.c0[Lx][lx]) * (pl.ty.c1[Ly][ly] - pl.ty.c0[Ly][ly]);
  }
  for (int l = 0; l <= L; ++l) {
    const int span = nleaf / pl.nn[l];
    for (int p = 0; p < pl.nn[l]; ++p) {
      pl.r0[l].push_back(rpre[p * span]);
      pl.m[l].push_back(rpre[(p + 1) * span] - rpre[p * span]);
      pl.c0[l].push_back(cpre[p * span]);
      pl.nc[l].push_back(cpre[(p + 1) * span] - cpre[p * span]);
    }
  }
  std::vector<int> cm(pl.N);
  for (int p = 0; p < nleaf; ++p) {
    const int lx = pl.leaf_lx[p], ly = pl.leaf_ly[p];
    const int x0 = pl.tx.c0[Lx][lx], x1 = pl.tx.c1[Lx][lx], y0 = pl.ty.c0[Ly][ly], y1 = pl.ty.c1[Ly][ly];
    const int dy = y1 - y0;
    for (int a = 0; a < x1 - x0; ++a)
      for (int b = 0; b < dy; ++b) cm[cpre[p] + a * dy + b] = (x0 + a) * ny + (y0 + b);
  }
  pl.colmap = keep.arr<int>(pl.N);
  NH_CK(cudaMemcpyAsync(pl.colmap, cm.data(), pl.N * sizeof(int), cudaMemcpyHostToDevice, st));
  NH_CK(cudaStreamSynchronize(st));
}

// =============================================================================== Hss
template <typename R>
Hss<R>::Hss(cudaStream_t st, const Plan* pl) : st_(st), pl_(pl), keep_((size_t)256 << 20, true), scr_((size_t)64 << 20),
                                                tmp_((size_t)512 << 20), ops_(st, &scr_) {
  keep_.set_stream(st);
  scr_.set_stream(st);
  tmp_.set_stream(st);
}

template <typename R> static GemmD<R> gd(const Mat<R>& A, int opA, const Mat<R>& B, int opB, const Mat<R>& C,
                                         R alpha = R(1), R beta = R(0)) {
  const int m = C.m, n = C.n;
  const int k = (opA == OP_N) ? A.n : A.m;
  return GemmD<R>{A.p, B.p, C.p, m, n, k, A.ld, B.ld, C.ld, opA, opB, alpha, beta};
}

// ------------------------------------------------------------------------------- 1D HSS
template <typename R>
void Hss<R>::build_1d(const Tree1D& t, const double* xo, double eps1, std::vector<std::vector<Gen1D<R>>>& g,
                      Mat<R>& G) {
  const int L = t.L, n = t.n, M = pl_->M;
  g.assign(L + 1, {});
  for (int l = 0; l <= L; ++l) g[l].resize(t.c0[l].size());
  // kernel entries of the transformed 1D matrix, rows in bin order (Sec. 2.4)
  G = keep_.mat<R>(M, n);
  psi_eval<R>(ops_, {PsiD<R>{xo, M, 0, n, n, G.p, G.ld}});
  // leaves: U = left singular vectors of G(J, K^c); V = those of G(J^c, K)^*
  {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    std::vector<Mat<R>> Ct;
    std::vector<CopyD<R>> cp;
    const int nl = (int)t.c0[L].size();
    for (int i = 0; i < nl; ++i) {
      const int r0 = t.r0[L][i], m = t.m[L][i], c0 = t.c0[L][i], c1 = t.c1[L][i], d = c1 - c0;
      Mat<R> cu = tmp_.mat<R>(n - d, m);
      cp.push_back({G.at(r0, 0), cu.p, c0, m, G.ld, cu.ld, OP_C, R(1), R(0)});
      cp.push_back({G.at(r0, c1), cu.at(c0, 0), n - c1, m, G.ld, cu.ld, OP_C, R(1), R(0)});
      Ct.push_back(cu);
    }
    for (int i = 0; i < nl; ++i) {
      const int r0 = t.r0[L][i], m = t.m[L][i], c0 = t.c0[L][i], c1 = t.c1[L][i], d = c1 - c0;
      Mat<R> cv = tmp_.mat<R>(M - m, d);
      cp.push_back({G.at(0, c0), cv.p, r0, d, G.ld, cv.ld, OP_N, R(1), R(0)});
      cp.push_back({G.at(r0 + m, c0), cv.at(r0, 0), M - r0 - m, d, G.ld, cv.ld, OP_N, R(1), R(0)});
      Ct.push_back(cv);
    }
    ops_.copy(cp);
    std::vector<Mat<R>> P;
    std::vector<std::vector<double>> S;
    ops_.tsvd_ct(Ct, eps1, keep_, P, S);
    std::vector<GemmD<R>> gm;
    for (int i = 0; i < nl; ++i) {
      Gen1D<R>& q = g[L][i];
      q.U = P[i];
      q.V = P[nl + i];
      q.ru = q.U.n;
      q.rv = q.V.n;
      q.P = keep_.mat<R>(q.ru, n);
      gm.push_back(gd<R>(q.U, OP_C, G.block(t.r0[L][i], 0, t.m[L][i], n), OP_N, q.P));
    }
    ops_.gemm(gm);
    tmp_.release(tk);
    scr_.release(mk);
  }
  for (int l = L - 1; l >= 0; --l) {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    const int nn = (int)t.c0[l].size();
    std::vector<GemmD<R>> gm;
    for (int i = 0; i < nn; ++i) {
      Gen1D<R>& a = g[l + 1][2 * i];
      Gen1D<R>& b = g[l + 1][2 * i + 1];
      const int ca0 = t.c0[l + 1][2 * i], ca1 = t.c1[l + 1][2 * i];
      const int cb0 = t.c0[l + 1][2 * i + 1], cb1 = t.c1[l + 1][2 * i + 1];
      a.Bs = keep_.mat<R>(a.ru, b.rv);
      b.Bs = keep_.mat<R>(b.ru, a.rv);
      gm.push_back(gd<R>(a.P.block(0, cb0, a.ru, cb1 - cb0), OP_N, b.V, OP_N, a.Bs));
      gm.push_back(gd<R>(b.P.block(0, ca0, b.ru, ca1 - ca0), OP_N, a.V, OP_N, b.Bs));
    }
    ops_.gemm(gm);
    if (l == 0) { tmp_.release(tk); scr_.release(mk); break; }
    std::vector<Mat<R>> Ct;
    std::vector<CopyD<R>> cp;
    gm.clear();
    for (int i = 0; i < nn; ++i) {
      Gen1D<R>& a = g[l + 1][2 * i];
      Gen1D<R>& b = g[l + 1][2 * i + 1];
      const int c0 = t.c0[l][i], c1 = t.c1[l][i], d = c1 - c0;
      Mat<R> cu = tmp_.mat<R>(n - d, a.ru + b.ru);
      int co = 0;
      for (Gen1D<R>* ch : {&a, &b}) {
        cp.push_back({ch->P.p, cu.at(0, co), c0, ch->ru, ch->P.ld, cu.ld, OP_C, R(1), R(0)});
        cp.push_back({ch->P.at(0, c1), cu.at(c0, co), n - c1, ch->ru, ch->P.ld, cu.ld, OP_C, R(1), R(0)});
        co += ch->ru;
      }
      Ct.push_back(cu);
    }
    for (int i = 0; i < nn; ++i) {
      Gen1D<R>& a = g[l + 1][2 * i];
      Gen1D<R>& b = g[l + 1][2 * i + 1];
      const int r0 = t.r0[l][i], m = t.m[l][i];
      Mat<R> z = tmp_.mat<R>(M - m, a.rv + b.rv);
      int co = 0;
      int kk = 0;
      for (Gen1D<R>* ch : {&a, &b}) {
        const int cc0 = t.c0[l + 1][2 * i + kk], cc1 = t.c1[l + 1][2 * i + kk];
        gm.push_back(gd<R>(G.block(0, cc0, r0, cc1 - cc0), OP_N, ch->V, OP_N, z.block(0, co, r0, ch->rv)));
        gm.push_back(gd<R>(G.block(r0 + m, cc0, M - r0 - m, cc1 - cc0), OP_N, ch->V, OP_N,
                           z.block(r0, co, M - r0 - m, ch->rv)));
        co += ch->rv;
        kk++;
      }
      Ct.push_back(z);
    }
    ops_.copy(cp);
    ops_.gemm(gm);
    std::vector<Mat<R>> P;
    std::vector<std::vector<double>> S;
    ops_.tsvd_ct(Ct, eps1, keep_, P, S);
    std::vector<GemmD<R>> g1, g2;
    for (int i = 0; i < nn; ++i) {
      Gen1D<R>& a = g[l + 1][2 * i];
      Gen1D<R>& b = g[l + 1][2 * i + 1];
      Gen1D<R>& q = g[l][i];
      q.Rst = P[i];
      q.Wst = P[nn + i];
      q.ru = q.Rst.n;
      q.rv = q.Wst.n;
      a.R_ = q.Rst.block(0, 0, a.ru, q.ru);
      b.R_ = q.Rst.block(a.ru, 0, b.ru, q.ru);
      a.W = q.Wst.block(0, 0, a.rv, q.rv);
      b.W = q.Wst.block(a.rv, 0, b.rv, q.rv);
      q.P = keep_.mat<R>(q.ru, n);
      g1.push_back(gd<R>(a.R_, OP_C, a.P, OP_N, q.P));
      g2.push_back(gd<R>(b.R_, OP_C, b.P, OP_N, q.P, R(1), R(1)));
      const int d = t.c1[l][i] - t.c0[l][i];
      const int da = t.c1[l + 1][2 * i] - t.c0[l + 1][2 * i];
      q.V = keep_.mat<R>(d, q.rv);
      g1.push_back(gd<R>(a.V, OP_N, a.W, OP_N, q.V.block(0, 0, da, q.rv)));
      g1.push_back(gd<R>(b.V, OP_N, b.W, OP_N, q.V.block(da, 0, d - da, q.rv)));
    }
    ops_.gemm(g1);
    ops_.gemm(g2);
    tmp_.release(tk);
    scr_.release(mk);
  }
}

// ------------------------------------------------------------------------------- face-splitting assembly
// Generators of G~_hss = H^x . H^y on T = T^x . T^y (proof of Thm. 3.5).  For a node
// xi = (alpha, beta) with 1D column counts dx, dy and 1D ranks rux, ruy (rows), rvx, rvy
// (columns):
//   U_xi = [D^x . U^y, U^x . D^y, U^x . U^y]  (leaf; rows of xi)
//   V_xi = [I (x) V^y, V^x (x) I, V^x (x) V^y]
//   B between siblings: diag(I (x) B^y, 0, 0) | diag(0, B^x (x) I, 0) | diag(0, 0, B^x (x) B^y)
//   R = [[E_x (x) R^y, 0, 0], [0, R^x (x) E_y, 0], [(B^x V'^x*)_sel (x) R^y, R^x (x) (B^y V'^y*)_sel, R^x (x) R^y]]
//   W = diag(E_x (x) W^y, W^x (x) E_y, W^x (x) W^y)
// A dimension that does not split at a level (its 1D node is already a leaf: Def. 3.3 (2), (3))
// keeps the parent's 1D node for every child: its selector E and transfer R (or W) are the
// identity and it has no sibling terms (the same derivation with a single child in that
// dimension), and siblings differ only in the other dimension.
template <typename R> void Hss<R>::assemble_2d() {
  const Plan& pl = *pl_;
  const int L = pl.L;
  const Tree1D &tx = pl.tx, &ty = pl.ty;
  auto gx = [&](int l, int p) -> const Gen1D<R>& { return gx_[pl.lvx(l)][pl.ix[l][p]]; };
  auto gy = [&](int l, int p) -> const Gen1D<R>& { return gy_[pl.lvy(l)][pl.iy[l][p]]; };
  auto dxo = [&](int l, int p) { const int i = pl.ix[l][p], lv = pl.lvx(l); return tx.c1[lv][i] - tx.c0[lv][i]; };
  auto dyo = [&](int l, int p) { const int i = pl.iy[l][p], lv = pl.lvy(l); return ty.c1[lv][i] - ty.c0[lv][i]; };
  t_.assign(L + 1, {});
  for (int l = 0; l <= L; ++l) t_[l].resize((size_t)pl.nn[l]);
  for (int l = 1; l <= L; ++l)
    for (int p = 0; p < pl.nn[l]; ++p) {
      const Gen1D<R>&ax = gx(l, p), &ay = gy(l, p);
      const int dx = dxo(l, p), dy = dyo(l, p);
      Node2<R>& nd = t_[l][p];
      nd.ku = dx * ay.ru + ax.ru * dy + ax.ru * ay.ru;
      nd.kv = dx * ay.rv + ax.rv * dy + ax.rv * ay.rv;
    }
  // ---------------- leaves: D, U, V
  {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    std::vector<PsiD<R>> ps;
    std::vector<GatherD<R>> ga;
    std::vector<FaceD<R>> fc;
    std::vector<KronD<R>> kr;
    const int Lx = pl.Lx, Ly = pl.Ly;
    for (int p = 0; p < pl.nn[L]; ++p) {
      const int ix = pl.leaf_lx[p], iy = pl.leaf_ly[p];
      const Gen1D<R>&ax = gx_[Lx][ix], &ay = gy_[Ly][iy];
      const int r0 = pl.r0[L][p], m = pl.m[L][p];
      const int dx = tx.c1[Lx][ix] - tx.c0[Lx][ix], dy = ty.c1[Ly][iy] - ty.c0[Ly][iy];
      Node2<R>& nd = t_[L][p];
      Mat<R> Dx = tmp_.mat<R>(m, dx), Dy = tmp_.mat<R>(m, dy);
      Mat<R> Ux = tmp_.mat<R>(m, ax.ru), Uy = tmp_.mat<R>(m, ay.ru);
      ps.push_back({pl.x2 + r0, m, tx.c0[Lx][ix], dx, pl.nx, Dx.p, Dx.ld});
      ps.push_back({pl.y2 + r0, m, ty.c0[Ly][iy], dy, pl.ny, Dy.p, Dy.ld});
      ga.push_back({ax.U.p, Ux.p, pl.posx + r0, m, ax.ru, ax.U.ld, Ux.ld, -tx.r0[Lx][ix]});
      ga.push_back({ay.U.p, Uy.p, pl.posy + r0, m, ay.ru, ay.U.ld, Uy.ld, -ty.r0[Ly][iy]});
      nd.D = keep_.mat<R>(m, dx * dy);
      nd.U = keep_.mat<R>(m, nd.ku);
      nd.V = keep_.mat<R>(dx * dy, nd.kv);
      fc.push_back({Dx.p, Dy.p, nd.D.p, m, dx, dy, Dx.ld, Dy.ld, nd.D.ld});
      int o = 0;
      fc.push_back({Dx.p, Uy.p, nd.U.at(0, o), m, dx, ay.ru, Dx.ld, Uy.ld, nd.U.ld}); o += dx * ay.ru;
      fc.push_back({Ux.p, Dy.p, nd.U.at(0, o), m, ax.ru, dy, Ux.ld, Dy.ld, nd.U.ld}); o += ax.ru * dy;
      fc.push_back({Ux.p, Uy.p, nd.U.at(0, o), m, ax.ru, ay.ru, Ux.ld, Uy.ld, nd.U.ld});
      o = 0;
      kr.push_back({nullptr, ay.V.p, nd.V.at(0, o), dx, dx, 1, dy, ay.rv, ay.V.ld, nd.V.ld, R(1)}); o += dx * ay.rv;
      kr.push_back({ax.V.p, nullptr, nd.V.at(0, o), dx, ax.rv, ax.V.ld, dy, dy, 1, nd.V.ld, R(1)}); o += ax.rv * dy;
      kr.push_back({ax.V.p, ay.V.p, nd.V.at(0, o), dx, ax.rv, ax.V.ld, dy, ay.rv, ay.V.ld, nd.V.ld, R(1)});
    }
    psi_eval<R>(ops_, ps);
    ops_.gather(ga);
    ops_.face(fc);
    ops_.kron(kr);
    tmp_.release(tk);
    scr_.release(mk);
  }
  // ---------------- nonleaf: B for every sibling pair, R and W for nonroot parents
  for (int l = 0; l < L; ++l) {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    std::vector<KronD<R>> kr;
    std::vector<Mat<R>> ids;
    std::vector<GemmD<R>> gm;
    const int cl = l + 1, F = pl.fan[l];
    const bool sx = pl.splitx(l), sy = pl.splity(l);
    for (int p = 0; p < pl.nn[l]; ++p) {
      const Gen1D<R>&tX = gx(l, p), &tY = gy(l, p);
      const int dxt = dxo(l, p), dyt = dyo(l, p);
      Node2<R>& tau = t_[l][p];
      for (int c = 0; c < F; ++c) {
        const int q = F * p + c, i = pl.cxi(l, c), j = pl.cyj(l, c);
        const Gen1D<R>&gxc = gx(cl, q), &gyc = gy(cl, q);
        const int dxc = dxo(cl, q), dyc = dyo(cl, q);
        Node2<R>& ch = t_[cl][q];
        const int r1 = dxc * gyc.ru, r2 = gxc.ru * dyc;
        // B_{c, c'}
        for (int c2 = 0; c2 < F; ++c2) {
          if (c2 == c) continue;
          const int q2 = F * p + c2, i2 = pl.cxi(l, c2), j2 = pl.cyj(l, c2);
          const Gen1D<R>&gx2 = gx(cl, q2), &gy2 = gy(cl, q2);
          const int dx2 = dxo(cl, q2), dy2 = dyo(cl, q2);
          Node2<R>& sib = t_[cl][q2];
          Mat<R> B = keep_.mat<R>(ch.ku, sib.kv, true);
          ch.B[c2] = B;
          const int v1 = dx2 * gy2.rv, v2 = gx2.rv * dy2;
          if (i == i2) {          // same x child: I (x) B^y
            kr.push_back({nullptr, gyc.Bs.p, B.p, dxc, dxc, 1, gyc.ru, gy2.rv, gyc.Bs.ld, B.ld, R(1)});
          } else if (j == j2) {   // same y child: B^x (x) I
            kr.push_back({gxc.Bs.p, nullptr, B.at(r1, v1), gxc.ru, gx2.rv, gxc.Bs.ld, dyc, dyc, 1, B.ld, R(1)});
          } else {                // B^x (x) B^y
            kr.push_back({gxc.Bs.p, gyc.Bs.p, B.at(r1 + r2, v1 + v2), gxc.ru, gx2.rv, gxc.Bs.ld, gyc.ru, gy2.rv,
                          gyc.Bs.ld, B.ld, R(1)});
          }
        }
        if (l == 0) continue;
        // selectors and (B V'^*) blocks of the 1D siblings (only in a dimension that splits)
        const int offi = sx ? (i ? (dxt - dxc) : 0) : 0, offi2 = i ? 0 : dxc;
        const int offj = sy ? (j ? (dyt - dyc) : 0) : 0, offj2 = j ? 0 : dyc;
        const int dxs = dxt - dxc, dys = dyt - dyc;
        Mat<R> Ex = tmp_.mat<R>(dxc, dxt, true);
        Mat<R> Ey = tmp_.mat<R>(dyc, dyt, true);
        ids.push_back(Ex.block(0, offi, dxc, dxc));
        ids.push_back(Ey.block(0, offj, dyc, dyc));
        Mat<R> BVx = tmp_.mat<R>(gxc.ru, dxt, true);
        Mat<R> BVy = tmp_.mat<R>(gyc.ru, dyt, true);
        if (sx) {
          const int sxi = 2 * pl.ix[l][p] + (1 - i);
          gm.push_back(gd<R>(gxc.Bs, OP_N, gx_[pl.lvx(cl)][sxi].V, OP_C, BVx.block(0, offi2, gxc.ru, dxs)));
        }
        if (sy) {
          const int syj = 2 * pl.iy[l][p] + (1 - j);
          gm.push_back(gd<R>(gyc.Bs, OP_N, gy_[pl.lvy(cl)][syj].V, OP_C, BVy.block(0, offj2, gyc.ru, dys)));
        }
        // 1D transfers of the children (identity, A == nullptr, in a dimension that does not split)
        const cplx<R>* Rx = sx ? gxc.R_.p : nullptr;
        const cplx<R>* Ry = sy ? gyc.R_.p : nullptr;
        const cplx<R>* Wx = sx ? gxc.W.p : nullptr;
        const cplx<R>* Wy = sy ? gyc.W.p : nullptr;
        const int ldRx = sx ? gxc.R_.ld : 1, ldRy = sy ? gyc.R_.ld : 1, ldWx = sx ? gxc.W.ld : 1, ldWy = sy ? gyc.W.ld : 1;
        // R_c (ku_c x ku_tau)
        Mat<R> Rm = keep_.mat<R>(ch.ku, tau.ku, true);
        ch.R_ = Rm;
        const int c1 = dxt * tY.ru, c2 = tX.ru * dyt;
        kr.push_back({Ex.p, Ry, Rm.p, dxc, dxt, Ex.ld, gyc.ru, tY.ru, ldRy, Rm.ld, R(1)});
        if (sx)
          kr.push_back({BVx.p, Ry, Rm.at(r1 + r2, 0), gxc.ru, dxt, BVx.ld, gyc.ru, tY.ru, ldRy, Rm.ld, R(1)});
        kr.push_back({Rx, Ey.p, Rm.at(r1, c1), gxc.ru, tX.ru, ldRx, dyc, dyt, Ey.ld, Rm.ld, R(1)});
        if (sy)
          kr.push_back({Rx, BVy.p, Rm.at(r1 + r2, c1), gxc.ru, tX.ru, ldRx, gyc.ru, dyt, BVy.ld, Rm.ld, R(1)});
        kr.push_back({Rx, Ry, Rm.at(r1 + r2, c1 + c2), gxc.ru, tX.ru, ldRx, gyc.ru, tY.ru, ldRy, Rm.ld, R(1)});
        // W_c (kv_c x kv_tau)
        Mat<R> Wm = keep_.mat<R>(ch.kv, tau.kv, true);
        ch.W = Wm;
        const int q1 = dxc * gyc.rv, q2 = gxc.rv * dyc;
        const int e1 = dxt * tY.rv, e2 = tX.rv * dyt;
        kr.push_back({Ex.p, Wy, Wm.p, dxc, dxt, Ex.ld, gyc.rv, tY.rv, ldWy, Wm.ld, R(1)});
        kr.push_back({Wx, Ey.p, Wm.at(q1, e1), gxc.rv, tX.rv, ldWx, dyc, dyt, Ey.ld, Wm.ld, R(1)});
        kr.push_back({Wx, Wy, Wm.at(q1 + q2, e1 + e2), gxc.rv, tX.rv, ldWx, gyc.rv, tY.rv, ldWy, Wm.ld, R(1)});
      }
    }
    ops_.set_identity(ids);
    ops_.gemm(gm);
    ops_.kron(kr);
    tmp_.release(tk);
    scr_.release(mk);
  }
}

// ------------------------------------------------------------------------------- recompression (Sec. 2.2)
template <typename R> void Hss<R>::recompress(double eps) {
  const int L = pl_->L;
  // ---- stage 1: orthogonalization, bottom-up.  Leaves: U = U~ F, V = V~ G (thin QR).
  {
    auto mk = scr_.mark();
    std::vector<Mat<R>> A;
    const int nl = (int)t_[L].size();
    for (auto& nd : t_[L]) A.push_back(nd.U);
    for (auto& nd : t_[L]) A.push_back(nd.V);
    auto Q = ops_.qr(A, tmp_);
    std::vector<CopyD<R>> cp;
    std::vector<Mat<R>> Id;
    std::vector<QFac<R>> qf;
    for (int i = 0; i < nl; ++i) {
      Node2<R>& nd = t_[L][i];
      const int pu = std::min(nd.U.m, nd.U.n), pv = std::min(nd.V.m, nd.V.n);
      nd.pu = pu; nd.pv = pv;
      nd.F = keep_.mat<R>(pu, nd.U.n, true);
      nd.G = keep_.mat<R>(pv, nd.V.n, true);
      cp.push_back({nd.U.p, nd.F.p, pu, nd.U.n, nd.U.ld, nd.F.ld, OP_N, R(1), R(0)});
      cp.push_back({nd.V.p, nd.G.p, pv, nd.V.n, nd.V.ld, nd.G.ld, OP_N, R(1), R(0)});
    }
    ops_.copy(cp);   // R factors (lower parts were zeroed by the QR)
    for (int i = 0; i < nl; ++i) {
      Node2<R>& nd = t_[L][i];
      nd.U = keep_.mat<R>(nd.U.m, nd.pu);
      nd.V = keep_.mat<R>(nd.V.m, nd.pv);
      Id.push_back(nd.U);
      Id.push_back(nd.V);
      qf.push_back(Q[i]);
      qf.push_back(Q[nl + i]);
    }
    ops_.set_identity(Id);
    ops_.apply_q_left(qf, Id, false);   // U~ = Q [I; 0]
    scr_.release(mk);
  }
  // nonleaf, nonroot: [F_c R_c] stacked = [R~_c] F_tau
  for (int l = L - 1; l >= 1; --l) {
    auto mk = scr_.mark();
    std::vector<Mat<R>> SU, SV;
    std::vector<GemmD<R>> gm;
    for (auto& tau : t_[l]) (void)tau;
    const int nn = (int)t_[l].size();
    const int F = pl_->fan[l];
    for (int p = 0; p < nn; ++p) {
      Node2<R>& tau = t_[l][p];
      int su = 0, sv = 0;
      for (int c = 0; c < F; ++c) { su += t_[l + 1][F * p + c].pu; sv += t_[l + 1][F * p + c].pv; }
      Mat<R> S1 = tmp_.mat<R>(su, tau.ku), S2 = tmp_.mat<R>(sv, tau.kv);
      int ou = 0, ov = 0;
      for (int c = 0; c < F; ++c) {
        Node2<R>& ch = t_[l + 1][F * p + c];
        gm.push_back(gd<R>(ch.F, OP_N, ch.R_, OP_N, S1.block(ou, 0, ch.pu, tau.ku)));
        gm.push_back(gd<R>(ch.G, OP_N, ch.W, OP_N, S2.block(ov, 0, ch.pv, tau.kv)));
        ou += ch.pu; ov += ch.pv;
      }
      SU.push_back(S1);
      SV.push_back(S2);
    }
    ops_.gemm(gm);
    std::vector<Mat<R>> A(SU);
    A.insert(A.end(), SV.begin(), SV.end());
    auto Q = ops_.qr(A, tmp_);
    std::vector<CopyD<R>> cp;
    std::vector<Mat<R>> Id;
    std::vector<QFac<R>> qf;
    for (int p = 0; p < nn; ++p) {
      Node2<R>& tau = t_[l][p];
      tau.pu = std::min(SU[p].m, SU[p].n);
      tau.pv = std::min(SV[p].m, SV[p].n);
      tau.F = keep_.mat<R>(tau.pu, tau.ku, true);
      tau.G = keep_.mat<R>(tau.pv, tau.kv, true);
      cp.push_back({SU[p].p, tau.F.p, tau.pu, tau.ku, SU[p].ld, tau.F.ld, OP_N, R(1), R(0)});
      cp.push_back({SV[p].p, tau.G.p, tau.pv, tau.kv, SV[p].ld, tau.G.ld, OP_N, R(1), R(0)});
    }
    ops_.copy(cp);
    for (int p = 0; p < nn; ++p) {
      Node2<R>& tau = t_[l][p];
      Mat<R> Rs = keep_.mat<R>(SU[p].m, tau.pu), Ws = keep_.mat<R>(SV[p].m, tau.pv);
      Id.push_back(Rs);
      Id.push_back(Ws);
      qf.push_back(Q[p]);
      qf.push_back(Q[nn + p]);
      int ou = 0, ov = 0;
      for (int c = 0; c < F; ++c) {
        Node2<R>& ch = t_[l + 1][F * p + c];
        ch.R_ = Rs.block(ou, 0, ch.pu, tau.pu);
        ch.W = Ws.block(ov, 0, ch.pv, tau.pv);
        ou += ch.pu; ov += ch.pv;
      }
    }
    ops_.set_identity(Id);
    ops_.apply_q_left(qf, Id, false);
    scr_.release(mk);
  }
  // B~_{c,c'} = F_c B_{c,c'} G_{c'}^*, every nonleaf parent (root included)
  for (int l = 0; l < L; ++l) {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    std::vector<GemmD<R>> g1, g2;
    std::vector<Mat<R>> outs;
    const int F = pl_->fan[l];
    for (int p = 0; p < pl_->nn[l]; ++p)
      for (int c = 0; c < F; ++c) {
        Node2<R>& ch = t_[l + 1][F * p + c];
        for (int c2 = 0; c2 < F; ++c2) {
          if (c2 == c) continue;
          Node2<R>& sb = t_[l + 1][F * p + c2];
          Mat<R> T1 = tmp_.mat<R>(ch.ku, sb.pv);
          Mat<R> Bn = keep_.mat<R>(ch.pu, sb.pv);
          g1.push_back(gd<R>(ch.B[c2], OP_N, sb.G, OP_C, T1));
          g2.push_back(gd<R>(ch.F, OP_N, T1, OP_N, Bn));
          ch.B[c2] = Bn;
        }
      }
    ops_.gemm(g1);
    ops_.gemm(g2);
    tmp_.release(tk);
    scr_.release(mk);
  }
  // ---- stage 2: top-down truncation.
  for (int l = 1; l <= L; ++l) {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    const int nn = (int)t_[l].size();
    const int F = pl_->fan[l - 1];
    std::vector<Mat<R>> Ct;
    std::vector<CopyD<R>> cp;
    std::vector<R*> sdev;
    for (int q = 0; q < nn; ++q) {
      const int p = q / F, c = q % F;
      Node2<R>& ch = t_[l][q];
      const Node2<R>& tau = t_[l - 1][p];
      int w = 0;
      for (int c2 = 0; c2 < F; ++c2) if (c2 != c) w += t_[l][F * p + c2].pv;
      const int rt = (l >= 2) ? (int)tau.SU.size() : 0;
      Mat<R> cu = tmp_.mat<R>(w + rt, ch.pu);
      int o = 0;
      for (int c2 = 0; c2 < F; ++c2) {
        if (c2 == c) continue;
        const Mat<R>& B = ch.B[c2];
        cp.push_back({B.p, cu.at(o, 0), B.n, B.m, B.ld, cu.ld, OP_C, R(1), R(0)});
        o += B.n;
      }
      if (rt > 0) {
        std::vector<R> hs(tau.SU.begin(), tau.SU.end());
        R* ds = tmp_.arr<R>(rt);
        NH_CK(cudaMemcpyAsync(ds, hs.data(), rt * sizeof(R), cudaMemcpyHostToDevice, st_));
        cp.push_back({ch.R_.p, cu.at(o, 0), rt, ch.pu, ch.R_.ld, cu.ld, OP_C, R(1), R(0), ds});
      }
      Ct.push_back(cu);
    }
    for (int q = 0; q < nn; ++q) {
      const int p = q / F, c = q % F;
      Node2<R>& ch = t_[l][q];
      const Node2<R>& tau = t_[l - 1][p];
      int w = 0;
      for (int c2 = 0; c2 < F; ++c2) if (c2 != c) w += t_[l][F * p + c2].pu;
      const int rt = (l >= 2) ? (int)tau.SV.size() : 0;
      Mat<R> cv = tmp_.mat<R>(w + rt, ch.pv);
      int o = 0;
      for (int c2 = 0; c2 < F; ++c2) {
        if (c2 == c) continue;
        const Mat<R>& B = t_[l][F * p + c2].B[c];    // B_{c', c}: pu_{c'} x pv_c
        cp.push_back({B.p, cv.at(o, 0), B.m, B.n, B.ld, cv.ld, OP_N, R(1), R(0)});
        o += B.m;
      }
      if (rt > 0) {
        std::vector<R> hs(tau.SV.begin(), tau.SV.end());
        R* ds = tmp_.arr<R>(rt);
        NH_CK(cudaMemcpyAsync(ds, hs.data(), rt * sizeof(R), cudaMemcpyHostToDevice, st_));
        cp.push_back({ch.W.p, cv.at(o, 0), rt, ch.pv, ch.W.ld, cv.ld, OP_C, R(1), R(0), ds});
      }
      Ct.push_back(cv);
    }
    NH_CK(cudaStreamSynchronize(st_));   // host staging vectors above go out of scope
    ops_.copy(cp);
    std::vector<Mat<R>> P;
    std::vector<std::vector<double>> S;
    ops_.tsvd_ct(Ct, eps, keep_, P, S);
    // updates
    std::vector<GemmD<R>> g1, g2;
    for (int q = 0; q < nn; ++q) {
      Node2<R>& ch = t_[l][q];
      ch.SU = S[q];
      ch.SV = S[nn + q];
    }
    for (int q = 0; q < nn; ++q) {
      const int p = q / F, c = q % F;
      Node2<R>& ch = t_[l][q];
      const Mat<R>& Pc = P[q];
      for (int c2 = 0; c2 < F; ++c2) {
        if (c2 == c) continue;
        const Mat<R>& Qc2 = P[nn + F * p + c2];
        Mat<R> T1 = tmp_.mat<R>(ch.B[c2].m, Qc2.n);
        Mat<R> Bn = keep_.mat<R>(Pc.n, Qc2.n);
        g1.push_back(gd<R>(ch.B[c2], OP_N, Qc2, OP_N, T1));
        g2.push_back(gd<R>(Pc, OP_C, T1, OP_N, Bn));
        ch.B[c2] = Bn;
      }
      const Mat<R>& Qc = P[nn + q];
      if (l >= 2) {
        Mat<R> Rn = keep_.mat<R>(Pc.n, ch.R_.n), Wn = keep_.mat<R>(Qc.n, ch.W.n);
        g1.push_back(gd<R>(Pc, OP_C, ch.R_, OP_N, Rn));
        g1.push_back(gd<R>(Qc, OP_C, ch.W, OP_N, Wn));
        ch.R_ = Rn;
        ch.W = Wn;
      }
      if (l == L) {
        Mat<R> Un = keep_.mat<R>(ch.U.m, Pc.n), Vn = keep_.mat<R>(ch.V.m, Qc.n);
        g1.push_back(gd<R>(ch.U, OP_N, Pc, OP_N, Un));
        g1.push_back(gd<R>(ch.V, OP_N, Qc, OP_N, Vn));
        ch.U = Un;
        ch.V = Vn;
      } else {
        const int F1 = pl_->fan[l];
        for (int c3 = 0; c3 < F1; ++c3) {
          Node2<R>& gc = t_[l + 1][F1 * q + c3];
          Mat<R> Rn = keep_.mat<R>(gc.R_.m, Pc.n), Wn = keep_.mat<R>(gc.W.m, Qc.n);
          g1.push_back(gd<R>(gc.R_, OP_N, Pc, OP_N, Rn));
          g1.push_back(gd<R>(gc.W, OP_N, Qc, OP_N, Wn));
          gc.R_ = Rn;
          gc.W = Wn;
        }
      }
      ch.ku = Pc.n;
      ch.kv = Qc.n;
    }
    ops_.gemm(g1);
    ops_.gemm(g2);
    tmp_.release(tk);
    scr_.release(mk);
  }
}

template <typename R> void Hss<R>::build(double eps, bool fadi) {
  if (fadi) {
    build_1d_fadi(pl_->tx, pl_->xo, eps / 10.0, gx_);
    build_1d_fadi(pl_->ty, pl_->yo, eps / 10.0, gy_);
  } else {
    build_1d(pl_->tx, pl_->xo, eps / 10.0, gx_, Gx_);
    build_1d(pl_->ty, pl_->yo, eps / 10.0, gy_, Gy_);
  }
  assemble_2d();
  recompress(eps);
  compact_generators();
  tmp_.free_all();
}

// The construction leaves every intermediate version of the generators in keep_ (the 1D HSS
// and dense 1D kernel matrices, the face-split generators before recompression, the thin-QR
// factors F, G, the truncated-SVD bases).  Only the final D, U, V (leaves), B, R and W are read
// afterwards (factorization, matvecs, recomputation of checkpointed levels): they are copied into
// a fresh arena and keep_ is handed back.
template <typename R> void Hss<R>::compact_generators() {
  auto gen = std::make_unique<Arena>((size_t)256 << 20, true);
  gen->set_stream(st_);
  std::vector<CopyD<R>> cp;
  auto move = [&](Mat<R>& a) {
    if (!a.p || a.m <= 0 || a.n <= 0) return;   // empty blocks are never dereferenced
    Mat<R> b = gen->template mat<R>(a.m, a.n);
    cp.push_back({a.p, b.p, a.m, a.n, a.ld, b.ld, OP_N, R(1), R(0)});
    a = b;
  };
  const int L = pl_->L;
  for (int l = 1; l <= L; ++l)
    for (Node2<R>& nd : t_[l]) {
      if (l == L) { move(nd.D); move(nd.U); move(nd.V); }
      for (int c = 0; c < 4; ++c) move(nd.B[c]);
      move(nd.R_);
      move(nd.W);
      nd.F = Mat<R>();
      nd.G = Mat<R>();
    }
  ops_.copy(cp);
  NH_CK(cudaStreamSynchronize(st_));
  keep_.free_all();
  gen_ = std::move(gen);
  gx_.clear();
  gy_.clear();
  Gx_ = Mat<R>();
  Gy_ = Mat<R>();
}

// ------------------------------------------------------------------------------- URV factorization (Sec. 2.3)
// The factors of level l (and those of the root) are allocated from their own arena fac_[l]
// (fac_[0] for the root), so that checkpoint() can hand back the top levels' factors and
// ensure_factored() can recompute them from the generators and the kept lower-level factors.
template <typename R> void Hss<R>::factor_level(int l) {
  const int L = pl_->L;
  Arena& fa = *fac_[l];
  const int F = l < L ? pl_->fan[l] : 0;
  auto mk = scr_.mark();
  auto tk = tmp_.mark();
  const int nn = (int)t_[l].size();
  // working matrix Wk = [U D] and V for every node of the level
  std::vector<Mat<R>> Vs(nn);
  std::vector<CopyD<R>> cp;
  std::vector<GemmD<R>> gm;
  for (int p = 0; p < nn; ++p) {
    Node2<R>& nd = t_[l][p];
    if (l == L) {
      nd.m = nd.D.m; nd.n = nd.D.n;
      nd.Wk = fa.template mat<R>(nd.m, nd.ku + nd.n);
      cp.push_back({nd.U.p, nd.Wk.p, nd.m, nd.ku, nd.U.ld, nd.Wk.ld, OP_N, R(1), R(0)});
      cp.push_back({nd.D.p, nd.Wk.at(0, nd.ku), nd.m, nd.n, nd.D.ld, nd.Wk.ld, OP_N, R(1), R(0)});
      Vs[p] = tmp_.mat<R>(nd.V.m, nd.kv);
      cp.push_back({nd.V.p, Vs[p].p, nd.V.m, nd.kv, nd.V.ld, Vs[p].ld, OP_N, R(1), R(0)});
    } else {
      // merge the children (Sec. 2.3): D+ blocks, U+ = stack U2_c R_c, V+ = stack V2_c W_c
      int rows = 0, cols = 0;
      for (int c = 0; c < F; ++c) { rows += t_[l + 1][F * p + c].rows2; cols += t_[l + 1][F * p + c].kv; }
      nd.m = rows; nd.n = cols;
      nd.Wk = fa.template mat<R>(rows, nd.ku + cols);
      Vs[p] = tmp_.mat<R>(cols, nd.kv);
      int ro = 0;
      for (int c = 0; c < F; ++c) {
        Node2<R>& a = t_[l + 1][F * p + c];
        Mat<R> U2 = a.Wk.block(a.n1, 0, a.rows2, a.ku);
        gm.push_back(gd<R>(U2, OP_N, a.R_, OP_N, nd.Wk.block(ro, 0, a.rows2, nd.ku)));
        int co = nd.ku;
        for (int c2 = 0; c2 < F; ++c2) {
          Node2<R>& b = t_[l + 1][F * p + c2];
          Mat<R> dst = nd.Wk.block(ro, co, a.rows2, b.kv);
          if (c2 == c) {
            Mat<R> D22 = a.Wk.block(a.n1, a.ku, a.rows2, a.kv);
            cp.push_back({D22.p, dst.p, a.rows2, a.kv, D22.ld, dst.ld, OP_N, R(1), R(0)});
          } else {
            Mat<R> T1 = tmp_.mat<R>(a.ku, b.kv);
            gm.push_back(gd<R>(a.B[c2], OP_N, b.V2, OP_C, T1));
            // second product issued after the first batch completes (ordering below)
            (void)dst;
          }
          co += b.kv;
        }
        ro += a.rows2;
      }
      int vo = 0;
      for (int c = 0; c < F; ++c) {
        Node2<R>& a = t_[l + 1][F * p + c];
        gm.push_back(gd<R>(a.V2, OP_N, a.W, OP_N, Vs[p].block(vo, 0, a.kv, nd.kv)));
        vo += a.kv;
      }
    }
  }
  ops_.copy(cp);
  if (l < L) {
    // gm holds: U+ products, T1 = B V2^*, V+ products.  Run them, then Wk blocks = U2 T1.
    ops_.gemm(gm);
    std::vector<GemmD<R>> g2;
    // recompute the T1 pointers in the same order as allocated above
    for (int p = 0, gi = 0; p < nn; ++p) {
      Node2<R>& nd = t_[l][p];
      int ro = 0;
      for (int c = 0; c < F; ++c) {
        Node2<R>& a = t_[l + 1][F * p + c];
        gi++;   // U+ product
        int co = nd.ku;
        for (int c2 = 0; c2 < F; ++c2) {
          Node2<R>& b = t_[l + 1][F * p + c2];
          if (c2 != c) {
            const GemmD<R>& t1 = gm[gi++];
            Mat<R> T1;
            T1.p = t1.C; T1.m = a.ku; T1.n = b.kv; T1.ld = t1.ldc;
            Mat<R> U2 = a.Wk.block(a.n1, 0, a.rows2, a.ku);
            g2.push_back(gd<R>(U2, OP_N, T1, OP_N, nd.Wk.block(ro, co, a.rows2, b.kv)));
          }
          co += b.kv;
        }
        ro += a.rows2;
      }
      gi += F;   // V+ products
    }
    ops_.gemm(g2);
  }
  // 1. size reduction: QR of [U D] when m >= n + ku
  std::vector<Mat<R>> Aq;
  std::vector<int> qi;
  for (int p = 0; p < nn; ++p) {
    Node2<R>& nd = t_[l][p];
    nd.omega = nd.m >= nd.n + nd.ku;
    nd.mc = nd.omega ? nd.n + nd.ku : nd.m;
    if (nd.omega) { Aq.push_back(nd.Wk); qi.push_back(p); }
  }
  if (!Aq.empty()) {
    auto Q = ops_.qr(Aq, fa);
    ops_.group_wy(Q, fa);
    for (size_t i = 0; i < qi.size(); ++i) t_[l][qi[i]].Om = Q[i];
  }
  // 2. basis elimination: V = Q_v [V2; 0] (standard QR; columns of D Q_v reordered so the
  //    eliminated block comes first, Sec. 2.3 Eq. for basis elimination)
  {
    auto Q = ops_.qr(Vs, fa);
    ops_.group_wy(Q, fa);
    std::vector<CopyD<R>> c2;
    std::vector<Mat<R>> Dc;
    for (int p = 0; p < nn; ++p) {
      Node2<R>& nd = t_[l][p];
      NH_REQUIRE(nd.kv <= nd.n, ST_ERANK, "column basis wider than the node");
      nd.Qv = Q[p];
      nd.V2 = fa.template mat<R>(nd.kv, nd.kv);
      c2.push_back({Vs[p].p, nd.V2.p, nd.kv, nd.kv, Vs[p].ld, nd.V2.ld, OP_N, R(1), R(0)});
      Dc.push_back(nd.Wk.block(0, nd.ku, nd.mc, nd.n));
    }
    ops_.copy(c2);
    // 3. D~ = D Q_v
    ops_.apply_q_right(Q, Dc, false);
  }
  // 4. partial decomposition: QR of the eliminated columns D~[:, kv:n]
  {
    std::vector<Mat<R>> A1, A2;
    for (int p = 0; p < nn; ++p) {
      Node2<R>& nd = t_[l][p];
      nd.n1 = nd.n - nd.kv;
      NH_REQUIRE(nd.mc >= nd.n1, ST_ERANK, "node has fewer rows than eliminated columns");
      nd.rows2 = nd.mc - nd.n1;
      A1.push_back(nd.Wk.block(0, nd.ku + nd.kv, nd.mc, nd.n1));
      A2.push_back(nd.Wk.block(0, 0, nd.mc, nd.ku + nd.kv));
    }
    auto Q = ops_.qr(A1, fa);
    ops_.group_wy(Q, fa);
    for (int p = 0; p < nn; ++p) t_[l][p].P = Q[p];
    // [U1; U2], [D12; D22] = P^* [U D~2]
    ops_.apply_q_left(Q, A2, true);
    // D11^{-1}
    std::vector<Mat<R>> T, X;
    for (int p = 0; p < nn; ++p) {
      Node2<R>& nd = t_[l][p];
      nd.D11inv = fa.template mat<R>(nd.n1, nd.n1);
      T.push_back(nd.Wk.block(0, nd.ku + nd.kv, nd.n1, nd.n1));
      X.push_back(nd.D11inv);
    }
    ops_.trinv(T, X);
  }
  tmp_.release(tk);
  scr_.release(mk);
}

template <typename R> void Hss<R>::factor_root() {
  Arena& fa = *fac_[0];
  const int F = pl_->fan[0];
  // root: D+ = P_root R_root
  {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    int rows = 0, cols = 0;
    for (int c = 0; c < F; ++c) { rows += t_[1][c].rows2; cols += t_[1][c].kv; }
    NH_REQUIRE(rows >= cols, ST_ERANK, "root block has fewer rows than columns");
    root_rows_ = rows; root_cols_ = cols;
    Droot_ = fa.template mat<R>(rows, cols);
    std::vector<CopyD<R>> cp;
    std::vector<GemmD<R>> g1, g2;
    int ro = 0;
    for (int c = 0; c < F; ++c) {
      Node2<R>& a = t_[1][c];
      int co = 0;
      for (int c2 = 0; c2 < F; ++c2) {
        Node2<R>& b = t_[1][c2];
        if (c2 == c) {
          Mat<R> D22 = a.Wk.block(a.n1, a.ku, a.rows2, a.kv);
          cp.push_back({D22.p, Droot_.at(ro, co), a.rows2, a.kv, D22.ld, Droot_.ld, OP_N, R(1), R(0)});
        } else {
          Mat<R> T1 = tmp_.mat<R>(a.ku, b.kv);
          g1.push_back(gd<R>(a.B[c2], OP_N, b.V2, OP_C, T1));
          g2.push_back(gd<R>(a.Wk.block(a.n1, 0, a.rows2, a.ku), OP_N, T1, OP_N, Droot_.block(ro, co, a.rows2, b.kv)));
        }
        co += b.kv;
      }
      ro += a.rows2;
    }
    ops_.copy(cp);
    ops_.gemm(g1);
    ops_.gemm(g2);
    auto Q = ops_.qr({Droot_}, fa);
    ops_.group_wy(Q, fa);
    Proot_ = Q[0];
    Rinv_ = fa.template mat<R>(cols, cols);
    ops_.trinv({Droot_.block(0, 0, cols, cols)}, {Rinv_});
    tmp_.release(tk);
    scr_.release(mk);
  }
}

template <typename R> void Hss<R>::factor() {
  const int L = pl_->L;
  fac_.clear();
  for (int l = 0; l <= L; ++l) {
    fac_.emplace_back(new Arena((size_t)64 << 20, true));
    fac_.back()->set_stream(st_);
  }
  for (int l = L; l >= 1; --l) factor_level(l);
  factor_root();
  NH_CK(cudaStreamSynchronize(st_));
  tmp_.free_all();
  factored = true;
  dropped_ = 0;
}

template <typename R> void Hss<R>::checkpoint(int levels) {
  NH_REQUIRE(factored, ST_ESTATE, "checkpoint before factor");
  const int L = pl_->L;
  const int k = std::max(0, std::min(levels, L));
  if (k <= dropped_) return;
  NH_CK(cudaStreamSynchronize(st_));
  for (int l = 1; l <= k; ++l) {
    fac_[l]->free_all();
    for (Node2<R>& nd : t_[l]) {
      nd.Wk = Mat<R>(); nd.V2 = Mat<R>(); nd.D11inv = Mat<R>();
      nd.Om = QFac<R>(); nd.Qv = QFac<R>(); nd.P = QFac<R>();
    }
  }
  fac_[0]->free_all();
  Droot_ = Mat<R>(); Rinv_ = Mat<R>(); Proot_ = QFac<R>();
  dropped_ = k;
}

template <typename R> bool Hss<R>::ensure_factored() {
  NH_REQUIRE(factored, ST_ESTATE, "solve before factor");
  if (dropped_ == 0) return false;
  for (int l = dropped_; l >= 1; --l) factor_level(l);
  factor_root();
  NH_CK(cudaStreamSynchronize(st_));
  tmp_.free_all();
  dropped_ = 0;
  return true;
}

// ------------------------------------------------------------------------------- URV solve (Sec. 2.3)
template <typename R> void Hss<R>::solve(const cplx<R>* f2, int ldf, int s, cplx<R>* ytree, int ldy) {
  NH_REQUIRE(factored, ST_ESTATE, "solve before factor");
  const int L = pl_->L;
  auto mk = scr_.mark();
  // per-level right-hand-side buffers; node rows at offsets
  std::vector<std::vector<Mat<R>>> Fl(L + 1);
  for (int l = L; l >= 1; --l) {
    const int nn = (int)t_[l].size();
    Fl[l].resize(nn);
    for (int p = 0; p < nn; ++p) Fl[l][p] = scr_.mat<R>(std::max(t_[l][p].m, 1), s);
  }
  {
    std::vector<CopyD<R>> cp;
    for (int p = 0; p < (int)t_[L].size(); ++p) {
      const int r0 = pl_->r0[L][p], m = pl_->m[L][p];
      cp.push_back({f2 + r0, Fl[L][p].p, m, s, ldf, Fl[L][p].ld, OP_N, R(1), R(0)});
    }
    ops_.copy(cp);
  }
  // ---- bottom-up: f <- Omega^* f (first mc rows kept), f^ = P^* f; parent stacks f^_2
  for (int l = L; l >= 1; --l) {
    const int nn = (int)t_[l].size();
    std::vector<QFac<R>> qo, qp;
    std::vector<Mat<R>> co, cpm;
    for (int p = 0; p < nn; ++p) {
      Node2<R>& nd = t_[l][p];
      if (nd.omega) { qo.push_back(nd.Om); co.push_back(Fl[l][p].block(0, 0, nd.m, s)); }
      qp.push_back(nd.P);
      cpm.push_back(Fl[l][p].block(0, 0, nd.mc, s));
    }
    ops_.apply_q_sweep(qo, co, true);
    ops_.apply_q_sweep(qp, cpm, true);
    if (l > 1) {
      std::vector<CopyD<R>> cp;
      const int F = pl_->fan[l - 1];
      for (int p = 0; p < (int)t_[l - 1].size(); ++p) {
        int ro = 0;
        for (int c = 0; c < F; ++c) {
          Node2<R>& a = t_[l][F * p + c];
          cp.push_back({Fl[l][F * p + c].at(a.n1, 0), Fl[l - 1][p].at(ro, 0), a.rows2, s, Fl[l][F * p + c].ld,
                        Fl[l - 1][p].ld, OP_N, R(1), R(0)});
          ro += a.rows2;
        }
      }
      ops_.copy(cp);
    }
  }
  // ---- root: min || R c+ - P^* f+ ||
  Mat<R> froot = scr_.mat<R>(root_rows_, s);
  {
    std::vector<CopyD<R>> cp;
    int ro = 0;
    for (int c = 0; c < pl_->fan[0]; ++c) {
      Node2<R>& a = t_[1][c];
      cp.push_back({Fl[1][c].at(a.n1, 0), froot.at(ro, 0), a.rows2, s, Fl[1][c].ld, froot.ld, OP_N, R(1), R(0)});
      ro += a.rows2;
    }
    ops_.copy(cp);
    ops_.apply_q_sweep({Proot_}, {froot}, true);
  }
  Mat<R> croot = scr_.mat<R>(root_cols_, s);
  ops_.gemm({gd<R>(Rinv_, OP_N, froot.block(0, 0, root_cols_, s), OP_N, croot)});
  // ---- top-down
  std::vector<std::vector<Mat<R>>> Cl(L + 1), Bl(L + 1);
  std::vector<Mat<R>> parentC = {croot};
  for (int l = 1; l <= L; ++l) {
    const int nn = (int)t_[l].size();
    const int F = pl_->fan[l - 1];
    Cl[l].resize(nn);
    Bl[l].resize(nn);
    std::vector<Mat<R>> Z(nn), C2(nn);
    std::vector<GemmD<R>> gz;
    for (int q = 0; q < nn; ++q) {
      const int p = q / F, c = q % F;
      int off = 0;
      for (int c2 = 0; c2 < c; ++c2) off += t_[l][F * p + c2].kv;
      const Mat<R>& pc = (l == 1) ? parentC[0] : Cl[l - 1][p];
      C2[q] = pc.block(off, 0, t_[l][q].kv, s);
      Z[q] = scr_.mat<R>(t_[l][q].kv, s);
      gz.push_back(gd<R>(t_[l][q].V2, OP_C, C2[q], OP_N, Z[q]));
    }
    ops_.gemm(gz);
    // b_c = R_c b_tau + sum_{c' != c} B_{c,c'} z_{c'}  (one accumulation per launch)
    for (int q = 0; q < nn; ++q) Bl[l][q] = scr_.mat<R>(t_[l][q].ku, s);
    {
      std::vector<GemmD<R>> g0;
      for (int q = 0; q < nn; ++q) {
        const int p = q / F;
        if (l >= 2) g0.push_back(gd<R>(t_[l][q].R_, OP_N, Bl[l - 1][p], OP_N, Bl[l][q]));
        else g0.push_back(gd<R>(t_[l][q].R_, OP_N, Bl[l][q], OP_N, Bl[l][q], R(0), R(0)));
      }
      if (l == 1) {
        // zero-initialise b: k = 0 product writes alpha*0 + 0
        for (auto& g : g0) { g.k = 0; g.A = nullptr; g.B = nullptr; }
      }
      ops_.gemm(g0);
      for (int j = 1; j < F; ++j) {
        std::vector<GemmD<R>> gj;
        for (int q = 0; q < nn; ++q) {
          const int p = q / F, c = q % F, c2 = (c + j) % F;
          gj.push_back(gd<R>(t_[l][q].B[c2], OP_N, Z[F * p + c2], OP_N, Bl[l][q], R(1), R(1)));
        }
        ops_.gemm(gj);
      }
    }
    // rhs = f1 - D12 c2 - U1 b ; c1 = D11^{-1} rhs ; c+ = Q_v [c2; c1]
    std::vector<GemmD<R>> ga, gb, gc;
    std::vector<Mat<R>> Y(nn);
    for (int q = 0; q < nn; ++q) {
      Node2<R>& nd = t_[l][q];
      Mat<R> f1 = Fl[l][q].block(0, 0, nd.n1, s);
      Mat<R> D12 = nd.Wk.block(0, nd.ku, nd.n1, nd.kv);
      Mat<R> U1 = nd.Wk.block(0, 0, nd.n1, nd.ku);
      ga.push_back(gd<R>(D12, OP_N, C2[q], OP_N, f1, R(-1), R(1)));
      gb.push_back(gd<R>(U1, OP_N, Bl[l][q], OP_N, f1, R(-1), R(1)));
      Y[q] = scr_.mat<R>(nd.n, s);
      gc.push_back(gd<R>(nd.D11inv, OP_N, f1, OP_N, Y[q].block(nd.kv, 0, nd.n1, s)));
    }
    ops_.gemm(ga);
    ops_.gemm(gb);
    ops_.gemm(gc);
    {
      std::vector<CopyD<R>> cp;
      std::vector<QFac<R>> qv;
      for (int q = 0; q < nn; ++q) {
        cp.push_back({C2[q].p, Y[q].p, C2[q].m, s, C2[q].ld, Y[q].ld, OP_N, R(1), R(0)});
        qv.push_back(t_[l][q].Qv);
      }
      ops_.copy(cp);
      ops_.apply_q_sweep(qv, Y, false);
    }
    Cl[l] = Y;
  }
  {
    std::vector<CopyD<R>> cp;
    for (int p = 0; p < (int)t_[L].size(); ++p)
      cp.push_back({Cl[L][p].p, ytree + pl_->c0[L][p], pl_->nc[L][p], s, Cl[L][p].ld, ldy, OP_N, R(1), R(0)});
    ops_.copy(cp);
  }
  scr_.release(mk);   // no synchronisation here: the solve is captured into a CUDA graph
}

// ------------------------------------------------------------------------------- adjoint solve
// f2 = (G~_hss^+)^* y: the solve above is a fixed chain of linear steps (unitary transforms,
// copies into sub-blocks, products with the factor blocks, triangular inverses), so its adjoint
// runs the adjoint of each step in the reverse order: first the top-down sweep backwards
// (Q_v^* on each node, then D11^{-*}, U1^*, D12^*, V2 and the B / R couplings), then the root
// (R^{-*}, then P_root), then the bottom-up sweep backwards (P, then Omega, each applied
// without conjugation, level 1 down to the leaves).  Rows that the solve discards (the
// least-squares residual rows) get zero.
template <typename R> void Hss<R>::solve_adj(const cplx<R>* ytree, int ldy, int s, cplx<R>* f2, int ldf) {
  NH_REQUIRE(factored, ST_ESTATE, "adjoint solve before factor");
  const int L = pl_->L;
  auto mk = scr_.mark();
  std::vector<std::vector<Mat<R>>> Yb(L + 1), Fb(L + 1), Bb(L + 2);
  for (int l = 1; l <= L; ++l) {
    const int nn = (int)t_[l].size();
    Fb[l].resize(nn);
    Yb[l].resize(nn);
    for (int p = 0; p < nn; ++p) Fb[l][p] = scr_.mat<R>(std::max(t_[l][p].m, 1), s, true);
  }
  {
    std::vector<CopyD<R>> cp;
    for (int p = 0; p < (int)t_[L].size(); ++p) {
      Yb[L][p] = scr_.mat<R>(std::max(t_[L][p].n, 1), s);
      cp.push_back({ytree + pl_->c0[L][p], Yb[L][p].p, pl_->nc[L][p], s, ldy, Yb[L][p].ld, OP_N, R(1), R(0)});
    }
    ops_.copy(cp);
  }
  Mat<R> crootb = scr_.mat<R>(std::max(root_cols_, 1), s);
  // ---- top-down sweep, backwards
  for (int l = L; l >= 1; --l) {
    const int nn = (int)t_[l].size();
    {
      std::vector<QFac<R>> qv;
      for (int q = 0; q < nn; ++q) qv.push_back(t_[l][q].Qv);
      ops_.apply_q_sweep(qv, Yb[l], true);                        // Y <- Q_v^* Y
    }
    // destination of the C2 adjoints: the parent's Y adjoint (or the root's c adjoint)
    if (l >= 2) {
      Yb[l - 1].resize(t_[l - 1].size());
      for (int p = 0; p < (int)t_[l - 1].size(); ++p) Yb[l - 1][p] = scr_.mat<R>(std::max(t_[l - 1][p].n, 1), s);
    }
    std::vector<Mat<R>> F1b(nn), C2b(nn);
    std::vector<GemmD<R>> gf, gb, gc;
    std::vector<CopyD<R>> cp;
    Bb[l].resize(nn);
    const int F = pl_->fan[l - 1];
    for (int q = 0; q < nn; ++q) {
      const int p = q / F, c = q % F;
      Node2<R>& nd = t_[l][q];
      int off = 0;
      for (int c2 = 0; c2 < c; ++c2) off += t_[l][F * p + c2].kv;
      const Mat<R>& dst = (l == 1) ? crootb : Yb[l - 1][p];
      C2b[q] = dst.block(off, 0, nd.kv, s);
      F1b[q] = Fb[l][q].block(0, 0, nd.n1, s);
      // c1 = D11^{-1} f1  =>  f1b = D11^{-*} Yb[kv:kv+n1]
      gf.push_back(gd<R>(nd.D11inv, OP_C, Yb[l][q].block(nd.kv, 0, nd.n1, s), OP_N, F1b[q]));
      // Y[0:kv] = C2  =>  C2b = Yb[0:kv]
      cp.push_back({Yb[l][q].p, C2b[q].p, nd.kv, s, Yb[l][q].ld, C2b[q].ld, OP_N, R(1), R(0)});
      Bb[l][q] = scr_.mat<R>(std::max(nd.ku, 1), s);
    }
    ops_.gemm(gf);
    ops_.copy(cp);
    // f1 = F1 - D12 C2 - U1 b  =>  C2b -= D12^* f1b ; bb = -U1^* f1b + sum_children R_child^* bb_child
    for (int q = 0; q < nn; ++q) {
      Node2<R>& nd = t_[l][q];
      gb.push_back(gd<R>(nd.Wk.block(0, nd.ku, nd.n1, nd.kv), OP_C, F1b[q], OP_N, C2b[q], R(-1), R(1)));
      gc.push_back(gd<R>(nd.Wk.block(0, 0, nd.n1, nd.ku), OP_C, F1b[q], OP_N, Bb[l][q], R(-1), R(0)));
    }
    ops_.gemm(gb);
    ops_.gemm(gc);
    if (l < L) {
      const int F1 = pl_->fan[l];
      for (int c = 0; c < F1; ++c) {
        std::vector<GemmD<R>> g;
        for (int q = 0; q < nn; ++q)
          g.push_back(gd<R>(t_[l + 1][F1 * q + c].R_, OP_C, Bb[l + 1][F1 * q + c], OP_N, Bb[l][q], R(1), R(1)));
        ops_.gemm(g);
      }
    }
    // b_q = ... + sum_{c2 != c} B_{q,c2} z_{c2}  =>  zb_{q2} = sum_{q != q2} B_{q,c2}^* bb_q ; z = V2^* C2  =>  C2b += V2 zb
    std::vector<Mat<R>> Zb(nn);
    for (int q = 0; q < nn; ++q) Zb[q] = scr_.mat<R>(std::max(t_[l][q].kv, 1), s);
    for (int j = 1; j < F; ++j) {
      std::vector<GemmD<R>> g;
      for (int q2 = 0; q2 < nn; ++q2) {
        const int p = q2 / F, c2 = q2 % F, c = (c2 + j) % F, q = F * p + c;
        g.push_back(gd<R>(t_[l][q].B[c2], OP_C, Bb[l][q], OP_N, Zb[q2], R(1), j == 1 ? R(0) : R(1)));
      }
      ops_.gemm(g);
    }
    std::vector<GemmD<R>> gv;
    for (int q = 0; q < nn; ++q) gv.push_back(gd<R>(t_[l][q].V2, OP_N, Zb[q], OP_N, C2b[q], R(1), R(1)));
    ops_.gemm(gv);
  }
  // ---- root: croot = R^{-1} (P_root^* froot)[0:cols]  =>  frootb = P_root [R^{-*} crootb; 0]
  Mat<R> frootb = scr_.mat<R>(std::max(root_rows_, 1), s, true);
  ops_.gemm({gd<R>(Rinv_, OP_C, crootb.block(0, 0, root_cols_, s), OP_N, frootb.block(0, 0, root_cols_, s))});
  ops_.apply_q_sweep({Proot_}, {frootb}, false);
  {
    std::vector<CopyD<R>> cp;
    int ro = 0;
    for (int c = 0; c < pl_->fan[0]; ++c) {
      Node2<R>& a = t_[1][c];
      cp.push_back({frootb.at(ro, 0), Fb[1][c].at(a.n1, 0), a.rows2, s, frootb.ld, Fb[1][c].ld, OP_N, R(1), R(0)});
      ro += a.rows2;
    }
    ops_.copy(cp);
  }
  // ---- bottom-up sweep, backwards: Fb <- P Fb[0:mc], then Fb <- Omega Fb, then hand rows to the children
  for (int l = 1; l <= L; ++l) {
    const int nn = (int)t_[l].size();
    std::vector<QFac<R>> qo, qp;
    std::vector<Mat<R>> co, cpm;
    for (int p = 0; p < nn; ++p) {
      Node2<R>& nd = t_[l][p];
      qp.push_back(nd.P);
      cpm.push_back(Fb[l][p].block(0, 0, nd.mc, s));
      if (nd.omega) { qo.push_back(nd.Om); co.push_back(Fb[l][p].block(0, 0, nd.m, s)); }
    }
    ops_.apply_q_sweep(qp, cpm, false);
    ops_.apply_q_sweep(qo, co, false);
    if (l < L) {
      std::vector<CopyD<R>> cp;
      const int F1 = pl_->fan[l];
      for (int p = 0; p < nn; ++p) {
        int ro = 0;
        for (int c = 0; c < F1; ++c) {
          Node2<R>& a = t_[l + 1][F1 * p + c];
          cp.push_back({Fb[l][p].at(ro, 0), Fb[l + 1][F1 * p + c].at(a.n1, 0), a.rows2, s, Fb[l][p].ld,
                        Fb[l + 1][F1 * p + c].ld, OP_N, R(1), R(0)});
          ro += a.rows2;
        }
      }
      ops_.copy(cp);
    }
  }
  {
    std::vector<CopyD<R>> cp;
    for (int p = 0; p < (int)t_[L].size(); ++p) {
      const int r0 = pl_->r0[L][p], m = pl_->m[L][p];
      cp.push_back({Fb[L][p].p, f2 + r0, m, s, Fb[L][p].ld, ldf, OP_N, R(1), R(0)});
    }
    ops_.copy(cp);
  }
  scr_.release(mk);
}

// ------------------------------------------------------------------------------- HSS matvec
template <typename R> void Hss<R>::matvec(const cplx<R>* x, int ldx, int s, cplx<R>* y, int ldy) {
  const int L = pl_->L;
  auto mk = scr_.mark();
  std::vector<std::vector<Mat<R>>> xh(L + 1), yh(L + 1);
  // up: x^_leaf = V^* x_leaf ; x^_tau = sum W_c^* x^_c
  {
    std::vector<GemmD<R>> g;
    xh[L].resize(t_[L].size());
    for (int p = 0; p < (int)t_[L].size(); ++p) {
      Node2<R>& nd = t_[L][p];
      xh[L][p] = scr_.mat<R>(nd.kv, s);
      Mat<R> xl;
      xl.p = const_cast<cplx<R>*>(x) + pl_->c0[L][p]; xl.m = pl_->nc[L][p]; xl.n = s; xl.ld = ldx;
      g.push_back(gd<R>(nd.V, OP_C, xl, OP_N, xh[L][p]));
    }
    ops_.gemm(g);
  }
  for (int l = L - 1; l >= 1; --l) {
    xh[l].resize(t_[l].size());
    for (int p = 0; p < (int)t_[l].size(); ++p) xh[l][p] = scr_.mat<R>(t_[l][p].kv, s);
    const int F = pl_->fan[l];
    for (int c = 0; c < F; ++c) {
      std::vector<GemmD<R>> g;
      for (int p = 0; p < (int)t_[l].size(); ++p)
        g.push_back(gd<R>(t_[l + 1][F * p + c].W, OP_C, xh[l + 1][F * p + c], OP_N, xh[l][p], R(1), c ? R(1) : R(0)));
      ops_.gemm(g);
    }
  }
  // down: y^_c = R_c y^_tau + sum B_{c,c'} x^_{c'}
  for (int l = 1; l <= L; ++l) {
    const int nn = (int)t_[l].size();
    yh[l].resize(nn);
    for (int q = 0; q < nn; ++q) yh[l][q] = scr_.mat<R>(t_[l][q].ku, s);
    const int F = pl_->fan[l - 1];
    for (int j = 0; j < F; ++j) {
      std::vector<GemmD<R>> g;
      for (int q = 0; q < nn; ++q) {
        const int p = q / F, c = q % F;
        if (j == 0) {
          if (l >= 2) g.push_back(gd<R>(t_[l][q].R_, OP_N, yh[l - 1][p], OP_N, yh[l][q]));
          else {
            GemmD<R> z = gd<R>(t_[l][q].R_, OP_N, yh[l][q], OP_N, yh[l][q], R(0), R(0));
            z.k = 0;
            g.push_back(z);
          }
        } else {
          const int c2 = (c + j) % F;
          g.push_back(gd<R>(t_[l][q].B[c2], OP_N, xh[l][F * p + c2], OP_N, yh[l][q], R(1), R(1)));
        }
      }
      ops_.gemm(g);
    }
  }
  {
    std::vector<GemmD<R>> g1, g2;
    for (int p = 0; p < (int)t_[L].size(); ++p) {
      Node2<R>& nd = t_[L][p];
      Mat<R> xl, yl;
      xl.p = const_cast<cplx<R>*>(x) + pl_->c0[L][p]; xl.m = pl_->nc[L][p]; xl.n = s; xl.ld = ldx;
      yl.p = y + pl_->r0[L][p]; yl.m = pl_->m[L][p]; yl.n = s; yl.ld = ldy;
      g1.push_back(gd<R>(nd.D, OP_N, xl, OP_N, yl));
      g2.push_back(gd<R>(nd.U, OP_N, yh[L][p], OP_N, yl, R(1), R(1)));
    }
    ops_.gemm(g1);
    ops_.gemm(g2);
  }
  NH_CK(cudaStreamSynchronize(st_));
  scr_.release(mk);
}

// ------------------------------------------------------------------------------- HSS adjoint matvec
// The adjoint of the nested product above (Def. 2.2): the row bases U (leaf) and R (transfer)
// now project the input, the column bases V and W expand the output, and each coupling
// B_{c,c'} acts as B_{c,c'}^* from the row side of c to the column side of c':
//   up:   z^_leaf = U^* z_leaf ;  z^_tau = sum_c R_c^* z^_c
//   down: x^_c = W_c x^_tau + sum_{c' != c} B_{c',c}^* z^_{c'}
//   leaf: x_leaf = D^* z_leaf + V x^_leaf
template <typename R> void Hss<R>::matvec_adj(const cplx<R>* y, int ldy, int s, cplx<R>* x, int ldx) {
  const int L = pl_->L;
  auto mk = scr_.mark();
  std::vector<std::vector<Mat<R>>> zh(L + 1), xh(L + 1);
  {
    std::vector<GemmD<R>> g;
    zh[L].resize(t_[L].size());
    for (int p = 0; p < (int)t_[L].size(); ++p) {
      Node2<R>& nd = t_[L][p];
      zh[L][p] = scr_.mat<R>(nd.ku, s);
      Mat<R> yl;
      yl.p = const_cast<cplx<R>*>(y) + pl_->r0[L][p]; yl.m = pl_->m[L][p]; yl.n = s; yl.ld = ldy;
      g.push_back(gd<R>(nd.U, OP_C, yl, OP_N, zh[L][p]));
    }
    ops_.gemm(g);
  }
  for (int l = L - 1; l >= 1; --l) {
    zh[l].resize(t_[l].size());
    for (int p = 0; p < (int)t_[l].size(); ++p) zh[l][p] = scr_.mat<R>(t_[l][p].ku, s);
    const int F = pl_->fan[l];
    for (int c = 0; c < F; ++c) {
      std::vector<GemmD<R>> g;
      for (int p = 0; p < (int)t_[l].size(); ++p)
        g.push_back(gd<R>(t_[l + 1][F * p + c].R_, OP_C, zh[l + 1][F * p + c], OP_N, zh[l][p], R(1), c ? R(1) : R(0)));
      ops_.gemm(g);
    }
  }
  for (int l = 1; l <= L; ++l) {
    const int nn = (int)t_[l].size();
    xh[l].resize(nn);
    for (int q = 0; q < nn; ++q) xh[l][q] = scr_.mat<R>(t_[l][q].kv, s);
    const int F = pl_->fan[l - 1];
    for (int j = 0; j < F; ++j) {
      std::vector<GemmD<R>> g;
      for (int q = 0; q < nn; ++q) {
        const int p = q / F, c = q % F;
        if (j == 0) {
          if (l >= 2) g.push_back(gd<R>(t_[l][q].W, OP_N, xh[l - 1][p], OP_N, xh[l][q]));
          else {
            GemmD<R> z = gd<R>(t_[l][q].W, OP_N, xh[l][q], OP_N, xh[l][q], R(0), R(0));
            z.k = 0;
            g.push_back(z);
          }
        } else {
          const int c2 = (c + j) % F;
          g.push_back(gd<R>(t_[l][F * p + c2].B[c], OP_C, zh[l][F * p + c2], OP_N, xh[l][q], R(1), R(1)));
        }
      }
      ops_.gemm(g);
    }
  }
  {
    std::vector<GemmD<R>> g1, g2;
    for (int p = 0; p < (int)t_[L].size(); ++p) {
      Node2<R>& nd = t_[L][p];
      Mat<R> xl, yl;
      yl.p = const_cast<cplx<R>*>(y) + pl_->r0[L][p]; yl.m = pl_->m[L][p]; yl.n = s; yl.ld = ldy;
      xl.p = x + pl_->c0[L][p]; xl.m = pl_->nc[L][p]; xl.n = s; xl.ld = ldx;
      g1.push_back(gd<R>(nd.D, OP_C, yl, OP_N, xl));
      g2.push_back(gd<R>(nd.V, OP_N, xh[L][p], OP_N, xl, R(1), R(1)));
    }
    ops_.gemm(g1);
    ops_.gemm(g2);
  }
  NH_CK(cudaStreamSynchronize(st_));
  scr_.release(mk);
}

// ------------------------------------------------------------------------------- factor store
// Section layout (all little-endian, as written by this host): per tree level l = 1..L and node p
// the ten integers (ku, kv, pu, pv, m, n, mc, n1, rows2, omega), the matrices D, U, V, R, W, B[0..3],
// Wk, D11inv, V2 and the Householder factors Om, Qv, P; then the root's two sizes, its Householder
// factor and R^{-1}.  A matrix is (int32 rows, int32 cols, rows x cols complex entries column by
// column); a Householder factor is (int32 m, int32 k, int32 merged) then V (m x k), the k / 32
// panel T blocks and, when merged, the k / 256 group T blocks.
namespace {
void fwr(FILE* f, const void* p, size_t n) {
  NH_REQUIRE(n == 0 || std::fwrite(p, 1, n, f) == n, ST_EINVAL, "save: write failed");
}
void frd(FILE* f, void* p, size_t n) {
  NH_REQUIRE(n == 0 || std::fread(p, 1, n, f) == n, ST_EINVAL, "load: file truncated or corrupt");
}
template <typename R> void save_mat(FILE* f, const Mat<R>& a) {
  const int32_t mn[2] = {a.p ? a.m : 0, a.p ? a.n : 0};
  fwr(f, mn, sizeof(mn));
  if ((size_t)mn[0] * mn[1] == 0) return;
  std::vector<cplx<R>> h((size_t)mn[0] * mn[1]);
  NH_CK(cudaMemcpy2D(h.data(), (size_t)mn[0] * sizeof(cplx<R>), a.p, (size_t)a.ld * sizeof(cplx<R>),
                     (size_t)mn[0] * sizeof(cplx<R>), mn[1], cudaMemcpyDeviceToHost));
  fwr(f, h.data(), h.size() * sizeof(cplx<R>));
}
// (copies into arena memory run on the arena's stream: its allocations are stream-ordered)
template <typename R> Mat<R> load_mat(FILE* f, Arena& ar, cudaStream_t st) {
  int32_t mn[2];
  frd(f, mn, sizeof(mn));
  NH_REQUIRE(mn[0] >= 0 && mn[1] >= 0 && (int64_t)mn[0] * mn[1] < (1LL << 40), ST_EINVAL, "load: bad matrix size");
  if ((size_t)mn[0] * mn[1] == 0) {
    Mat<R> e;
    e.m = mn[0]; e.n = mn[1]; e.ld = std::max(mn[0], 1);
    return e;
  }
  Mat<R> a = ar.template mat<R>(mn[0], mn[1]);
  std::vector<cplx<R>> h((size_t)mn[0] * mn[1]);
  frd(f, h.data(), h.size() * sizeof(cplx<R>));
  NH_CK(cudaMemcpyAsync(a.p, h.data(), h.size() * sizeof(cplx<R>), cudaMemcpyHostToDevice, st));
  NH_CK(cudaStreamSynchronize(st));
  return a;
}
template <typename R> void save_raw(FILE* f, const cplx<R>* d, size_t n) {
  std::vector<cplx<R>> h(n);
  if (n) NH_CK(cudaMemcpy(h.data(), d, n * sizeof(cplx<R>), cudaMemcpyDeviceToHost));
  fwr(f, h.data(), n * sizeof(cplx<R>));
}
template <typename R> cplx<R>* load_raw(FILE* f, Arena& ar, size_t n, cudaStream_t st) {
  std::vector<cplx<R>> h(n);
  frd(f, h.data(), n * sizeof(cplx<R>));
  cplx<R>* d = (cplx<R>*)ar.alloc(std::max<size_t>(n, 1) * sizeof(cplx<R>));
  if (n) {
    NH_CK(cudaMemcpyAsync(d, h.data(), n * sizeof(cplx<R>), cudaMemcpyHostToDevice, st));
    NH_CK(cudaStreamSynchronize(st));
  }
  return d;
}
template <typename R> void save_qf(FILE* f, const QFac<R>& q) {
  const int32_t h[3] = {q.V ? q.m : 0, q.V ? q.k : 0, q.Tg ? 1 : 0};
  fwr(f, h, sizeof(h));
  if (h[1] == 0) return;
  Mat<R> v;
  v.p = q.V; v.m = q.m; v.n = q.k; v.ld = q.ldv;
  save_mat(f, v);
  constexpr int NB = Ops<R>::NB, GW = Ops<R>::GW;
  save_raw<R>(f, q.Tp, (size_t)((q.k + NB - 1) / NB) * NB * NB);
  if (h[2]) save_raw<R>(f, q.Tg, (size_t)((q.k + GW - 1) / GW) * GW * GW);
}
template <typename R> QFac<R> load_qf(FILE* f, Arena& ar, cudaStream_t st) {
  int32_t h[3];
  frd(f, h, sizeof(h));
  NH_REQUIRE(h[0] >= 0 && h[1] >= 0 && h[1] <= h[0] && (h[2] == 0 || h[2] == 1), ST_EINVAL, "load: bad factor header");
  QFac<R> q;
  q.m = h[0]; q.k = h[1];
  if (h[1] == 0) return q;
  Mat<R> v = load_mat<R>(f, ar, st);
  NH_REQUIRE(v.m == h[0] && v.n == h[1], ST_EINVAL, "load: factor size mismatch");
  q.V = v.p; q.ldv = v.ld;
  constexpr int NB = Ops<R>::NB, GW = Ops<R>::GW;
  q.Tp = load_raw<R>(f, ar, (size_t)((q.k + NB - 1) / NB) * NB * NB, st);
  if (h[2]) q.Tg = load_raw<R>(f, ar, (size_t)((q.k + GW - 1) / GW) * GW * GW, st);
  return q;
}
}  // namespace

template <typename R> void Hss<R>::save(FILE* f) {
  NH_REQUIRE(factored && dropped_ == 0, ST_ESTATE, "save: factor (and recompute checkpointed levels) first");
  NH_CK(cudaStreamSynchronize(st_));
  const int L = pl_->L;
  for (int l = 1; l <= L; ++l)
    for (Node2<R>& nd : t_[l]) {
      const int32_t iv[10] = {nd.ku, nd.kv, nd.pu, nd.pv, nd.m, nd.n, nd.mc, nd.n1, nd.rows2, nd.omega ? 1 : 0};
      fwr(f, iv, sizeof(iv));
      save_mat(f, nd.D);
      save_mat(f, nd.U);
      save_mat(f, nd.V);
      save_mat(f, nd.R_);
      save_mat(f, nd.W);
      for (int c = 0; c < 4; ++c) save_mat(f, nd.B[c]);
      save_mat(f, nd.Wk);
      save_mat(f, nd.D11inv);
      save_mat(f, nd.V2);
      save_qf(f, nd.omega ? nd.Om : QFac<R>());
      save_qf(f, nd.Qv);
      save_qf(f, nd.P);
    }
  const int32_t rs[2] = {root_rows_, root_cols_};
  fwr(f, rs, sizeof(rs));
  save_qf(f, Proot_);
  save_mat(f, Rinv_);
}

template <typename R> void Hss<R>::load(FILE* f) {
  const int L = pl_->L;
  t_.assign(L + 1, {});
  for (int l = 0; l <= L; ++l) t_[l].resize((size_t)pl_->nn[l]);
  gen_.reset(new Arena((size_t)256 << 20, true));
  gen_->set_stream(st_);
  fac_.clear();
  for (int l = 0; l <= L; ++l) {
    fac_.emplace_back(new Arena((size_t)64 << 20, true));
    fac_.back()->set_stream(st_);
  }
  for (int l = 1; l <= L; ++l)
    for (Node2<R>& nd : t_[l]) {
      int32_t iv[10];
      frd(f, iv, sizeof(iv));
      for (int q = 0; q < 9; ++q) NH_REQUIRE(iv[q] >= 0, ST_EINVAL, "load: bad node header");
      nd.ku = iv[0]; nd.kv = iv[1]; nd.pu = iv[2]; nd.pv = iv[3];
      nd.m = iv[4]; nd.n = iv[5]; nd.mc = iv[6]; nd.n1 = iv[7]; nd.rows2 = iv[8]; nd.omega = iv[9] != 0;
      nd.D = load_mat<R>(f, *gen_, st_);
      nd.U = load_mat<R>(f, *gen_, st_);
      nd.V = load_mat<R>(f, *gen_, st_);
      nd.R_ = load_mat<R>(f, *gen_, st_);
      nd.W = load_mat<R>(f, *gen_, st_);
      for (int c = 0; c < 4; ++c) nd.B[c] = load_mat<R>(f, *gen_, st_);
      Arena& fa = *fac_[l];
      nd.Wk = load_mat<R>(f, fa, st_);
      nd.D11inv = load_mat<R>(f, fa, st_);
      nd.V2 = load_mat<R>(f, fa, st_);
      nd.Om = load_qf<R>(f, fa, st_);
      nd.Qv = load_qf<R>(f, fa, st_);
      nd.P = load_qf<R>(f, fa, st_);
    }
  int32_t rs[2];
  frd(f, rs, sizeof(rs));
  NH_REQUIRE(rs[0] >= rs[1] && rs[1] >= 0, ST_EINVAL, "load: bad root sizes");
  root_rows_ = rs[0];
  root_cols_ = rs[1];
  Proot_ = load_qf<R>(f, *fac_[0], st_);
  Rinv_ = load_mat<R>(f, *fac_[0], st_);
  NH_REQUIRE(Rinv_.m == root_cols_ && Rinv_.n == root_cols_, ST_EINVAL, "load: root size mismatch");
  factored = true;
  dropped_ = 0;
}

template <typename R> double Hss<R>::solve_entries() const {
  // Householder vectors: the lower trapezoid (unit diagonal included) of each m x k factor
  auto trap = [](const QFac<R>& q) { return (double)q.m * q.k - 0.5 * (double)q.k * (q.k - 1); };
  double e = 0;
  const int L = pl_->L;
  for (int l = 1; l <= L; ++l)
    for (const Node2<R>& nd : t_[l]) {
      if (nd.omega) e += trap(nd.Om);
      e += trap(nd.P) + trap(nd.Qv);
      e += (double)nd.n1 * nd.n1 + (double)nd.n1 * (nd.kv + nd.ku) + (double)nd.kv * nd.kv;
      for (int c = 0; c < 4; ++c) e += (double)nd.B[c].m * nd.B[c].n;
      if (l >= 2) e += (double)nd.R_.m * nd.R_.n;
    }
  e += trap(Proot_) + (double)root_cols_ * root_cols_;
  return e;
}

template <typename R> int Hss<R>::max_rank() const {
  int r = 0;
  for (auto& lv : t_)
    for (auto& nd : lv) r = std::max(r, std::max(nd.ku, nd.kv));
  return r;
}
template <typename R> std::vector<int> Hss<R>::level_ranks() const {
  std::vector<int> out;
  for (auto& lv : t_) {
    int r = 0;
    for (auto& nd : lv) r = std::max(r, std::max(nd.ku, nd.kv));
    out.push_back(r);
  }
  return out;
}

template class Hss<double>;
template class Hss<float>;

}  // namespace nh
