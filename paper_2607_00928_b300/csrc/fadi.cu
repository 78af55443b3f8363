// fADI + interpolative decomposition construction of the 1D HSS approximations (Alg. 1 step 1
// by the route the paper cites in Sec. 3.1: factored ADI on the Sylvester equation
// S G~ - G~ D = u v^T of the transformed 1D matrix, whose entries are u_j v_k / (s_j - d_k),
// s_j = exp(-2 pi i x_j), d_k = exp(-2 pi i k / n), u_j = s_j^n - 1, v_k = d_k / n, and the
// interpolative decomposition).  Selected by NUDFT2_FLAG_FADI; the default route is the truncated
// SVD of hss.cu's build_1d.
//
// Per node a (columns [c0, c1), d = c1 - c0; every quantity in the node's frame, c0 = 0):
//   row block G~(J_a, K_a^c): the column c1 (mod n) touches the node's points and is kept exactly;
//     the far columns d+1 .. n-1 lie at least 1/n from the points' arc [0, d/n] and go through
//     fADI with J shift pairs: z_1 = u / (s - beta_1), z_{i+1} = z_i (s - alpha_i) / (s - beta_{i+1}).
//   column block G~(J_a^c, K_a): column 0 touches the outside points and is kept as a unit
//     direction; columns 1 .. d-1 go through fADI against the outside points' arc [d/n, 1].
//   Shifts: Zolotarev-optimal for the two arcs (Moebius map onto [-gamma, -1] u [1, gamma] and
//   Wachspress's p_j = gamma dn((2j-1) K(k') / (2J), k')), J the least count whose error bound
//   max|r| / min|r| is below eps1 / 100.  When the fADI set has no more columns than J, all of
//   the block's columns are kept exactly.
//   Energy weighting: the basis row is a^T C with a = [exact entries, z_1 .. z_J] and C folding
//   in g_i = beta_i - alpha_i and the R factor of the other fADI factor Y (far columns, or a
//   uniform proxy of 4 samples per 1/n on the outside arc), so the basis carries the block's
//   singular values and the ID's pivot cut (eps1 / 10 of the leading pivot) measures them.
//   ID: column-pivoted QR of W = B^* (rows) or W = B^T (columns, so that the interpolation matrix
//   is V itself); nested: a parent's candidates are its children's skeletons.
//   Generators: U, V (leaves) and R, W (transfers) are interpolation matrices; B_ab is the kernel
//   at a's skeleton points and b's skeleton columns.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "hss.cuh"
#include "qp.cuh"

namespace nh {

using cd = std::complex<double>;
static constexpr double FADI_PI = 3.14159265358979323846;
static constexpr int FADI_PROXY_PER_COL = 4;     // outside-arc proxy samples per 1/n
static constexpr double FADI_TARGET = 0.01;      // fADI error bound target, relative to eps1
static constexpr double FADI_ID_TOL = 0.1;       // pivot cut of the ID, relative to eps1
static constexpr int FADI_SAMPLES = 4001;        // geometric samples of [1, gamma] for the bound
static constexpr int FB_MAXQ = FADI_JMAX + 1;

// ============================================================================ host: shifts
// K(m) = pi / (2 AGM(1, sqrt(1 - m))) (Abramowitz & Stegun 17.6); m1 = 1 - m is passed so that
// K stays accurate for m close to 1.
static double ellip_k(double m1) {
  double a = 1.0, b = std::sqrt(m1);
  for (int i = 0; i < 64 && std::fabs(a - b) > 1e-16 * a; ++i) {
    const double t = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = t;
  }
  return FADI_PI / (2.0 * a);
}

// Jacobi dn(u | m), m = 1 - m1, by the descending AGM scale (Abramowitz & Stegun 16.4):
// a_0 = 1, b_0 = sqrt(m1), c_0 = sqrt(m); a_{i+1} = (a_i + b_i)/2, b_{i+1} = sqrt(a_i b_i),
// c_{i+1} = (a_i - b_i)/2 until c_N vanishes; phi_N = 2^N a_N u, phi_{i-1} = (phi_i +
// asin(c_i sin(phi_i) / a_i)) / 2; dn = cos(phi_0) / cos(phi_1 - phi_0).
static double jacobi_dn(double u, double m1) {
  if (m1 >= 1.0) return 1.0;
  double a[66], c[66];
  double b = std::sqrt(m1);
  a[0] = 1.0;
  c[0] = std::sqrt(1.0 - m1);
  int N = 0;
  while (N < 64 && std::fabs(c[N]) > 1e-17 * a[N]) {
    a[N + 1] = 0.5 * (a[N] + b);
    c[N + 1] = 0.5 * (a[N] - b);
    b = std::sqrt(a[N] * b);
    ++N;
  }
  if (N == 0) return 1.0;
  double phi = std::ldexp(a[N] * u, N);
  double phi1 = phi;
  for (int i = N; i >= 1; --i) {
    phi1 = phi;
    double s = c[i] * std::sin(phi) / a[i];
    s = std::max(-1.0, std::min(1.0, s));
    phi = 0.5 * (phi + std::asin(s));
  }
  return std::cos(phi) / std::cos(phi1 - phi);
}

struct Arcs {
  double g, t[4], gamma;
};

// Arcs E = [e1, e2], F = [f1, f2] in units of the circle (e1 <= e2 < f1 <= f2 < e1 + 1): the
// centre g of the gap from f2 to e1 + 1, the endpoints under t = tan(theta / 2) with
// theta = 2 pi (x - g) + pi, and gamma > 1 with the cross-ratio of (-gamma, -1, 1, gamma).
static Arcs arcs(double e1, double e2, double f1, double f2) {
  Arcs A;
  A.g = 0.5 * (f2 + e1 + 1.0);
  const double xs[4] = {e1, e2, f1, f2};
  for (int i = 0; i < 4; ++i) A.t[i] = std::tan(0.5 * (2.0 * FADI_PI * (xs[i] - A.g) + FADI_PI));
  const double* t = A.t;
  const double c = (t[2] - t[0]) * (t[3] - t[1]) / ((t[2] - t[1]) * (t[3] - t[0]));
  A.gamma = 2.0 * c - 1.0 + 2.0 * std::sqrt(std::max(c * (c - 1.0), 0.0));
  return A;
}

// The point of the circle (units of the circle) whose image under the Moebius map that sends
// t2, t3, t4 to -1, 1, gamma is w: CR(t; t2, t3, t4) = CR(w; -1, 1, gamma).
static double arc_point(const Arcs& A, double w) {
  const double t2 = A.t[1], t3 = A.t[2], t4 = A.t[3];
  const double a = -2.0 * (w - A.gamma), b = (w - 1.0) * (-1.0 - A.gamma);
  const double t = (t3 * (t2 - t4) * a - b * t4 * (t2 - t3)) / ((t2 - t4) * a - b * (t2 - t3));
  return (2.0 * std::atan(t) - FADI_PI) / (2.0 * FADI_PI) + A.g;
}

static std::vector<double> wachspress(double gamma, int J) {
  const double m1 = 1.0 / (gamma * gamma);
  const double K = ellip_k(m1);
  std::vector<double> p(J);
  for (int j = 0; j < J; ++j) p[j] = gamma * jacobi_dn((2.0 * (j + 1) - 1.0) / (2.0 * J) * K, m1);
  return p;
}

static double zratio(double gamma, const std::vector<double>& p) {
  double mx = 0;
  for (int i = 0; i < FADI_SAMPLES; ++i) {
    const double y = std::pow(gamma, (double)i / (FADI_SAMPLES - 1));
    double v = 1.0;
    for (double pj : p) v *= std::fabs(y - pj) / (y + pj);
    mx = std::max(mx, v);
  }
  return mx * mx;
}

static cd em(double t) {   // exp(-2 pi i t), t reduced to [-1/2, 1/2)
  t -= std::floor(t + 0.5);
  return cd(std::cos(2.0 * FADI_PI * t), -std::sin(2.0 * FADI_PI * t));
}

static cd psi_host(double x, int k, int n) {   // the kernel entry (transformed 1D matrix)
  double t = x - (double)k / n;
  t -= std::floor(t + 0.5);
  if (t == 0.0) return cd(1.0, 0.0);
  const double r = std::sin(FADI_PI * n * t) / (n * std::sin(FADI_PI * t));
  return r * cd(std::cos(FADI_PI * (n - 1) * t), -std::sin(FADI_PI * (n - 1) * t));
}

// R factor (cols x cols, column major) of the Householder QR of A (rows x cols, rows >= cols)
static std::vector<cd> qr_r(std::vector<cd> A, int rows, int cols) {
  std::vector<cd> v(rows);
  for (int j = 0; j < cols; ++j) {
    double nrm = 0;
    for (int i = j; i < rows; ++i) nrm += std::norm(A[i + (size_t)j * rows]);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const cd a0 = A[j + (size_t)j * rows];
    const cd ph = std::abs(a0) > 0 ? a0 / std::abs(a0) : cd(1.0, 0.0);
    double vv = 0;
    for (int i = j; i < rows; ++i) {
      v[i] = A[i + (size_t)j * rows];
      if (i == j) v[i] += ph * nrm;
      vv += std::norm(v[i]);
    }
    for (int c = j; c < cols; ++c) {
      cd s = 0;
      for (int i = j; i < rows; ++i) s += std::conj(v[i]) * A[i + (size_t)c * rows];
      s *= 2.0 / vv;
      for (int i = j; i < rows; ++i) A[i + (size_t)c * rows] -= s * v[i];
    }
  }
  std::vector<cd> R((size_t)cols * cols, cd(0.0, 0.0));
  for (int j = 0; j < cols; ++j)
    for (int i = 0; i <= j; ++i) R[i + (size_t)j * cols] = A[i + (size_t)j * rows];
  return R;
}

// y_1 = cv / (cn - alpha_1), y_{i+1} = y_i (cn - beta_i) / (cn - alpha_{i+1}) (column factor of fADI)
static void fadi_y(const std::vector<cd>& cn, const std::vector<cd>& cv, const std::vector<cd>& al,
                   const std::vector<cd>& be, std::vector<cd>& Y, int col0, int ldy) {
  const int J = (int)al.size();
  for (size_t r = 0; r < cn.size(); ++r) {
    cd y = cv[r] / (cn[r] - al[0]);
    for (int i = 0; i < J; ++i) {
      Y[r + (size_t)(col0 + i) * ldy] = y;
      if (i + 1 < J) y = y * (cn[r] - be[i]) / (cn[r] - al[i + 1]);
    }
  }
}

FadiPlan fadi_plan(int side, int d, int n, double eps1, int jmax) {
  NH_REQUIRE((side == 0 || side == 1) && d >= 1 && d < n && jmax >= 1 && jmax <= FADI_JMAX, ST_EINVAL,
             "fadi_plan: bad node");
  FadiPlan P;
  const int nset = side == 0 ? n - d - 1 : d - 1;
  double e1, e2, f1, f2;
  if (side == 0) { e1 = 0.0; e2 = (double)d / n; f1 = (double)(d + 1) / n; f2 = (double)(n - 1) / n; }
  else { e1 = 1.0 / n; e2 = (double)(d - 1) / n; f1 = (double)d / n; f2 = 1.0; }
  int J = 0;
  std::vector<double> p;
  Arcs A{};
  if (nset >= 2) {
    A = arcs(e1, e2, f1, f2);
    for (J = 1; J <= jmax; ++J) {
      p = wachspress(A.gamma, J);
      P.ratio = zratio(A.gamma, p);
      if (1.1 * P.ratio <= FADI_TARGET * eps1) break;
    }
    if (J > jmax) {
      NH_REQUIRE(nset <= jmax, ST_EINVAL,
                 "NUDFT2_FLAG_FADI: eps too small for this n (more than 64 ADI shifts would be needed)");
      J = jmax;
    }
  }
  if (nset < 2 || J >= nset) {   // keep every column of the block
    const int q = side == 0 ? n - d : d;
    P.J = 0;
    P.ratio = 0;
    for (int i = 0; i < q; ++i) P.ex.push_back(side == 0 ? d + i : i);
    P.C.assign((size_t)q * q, cd(0.0, 0.0));
    for (int i = 0; i < q; ++i) P.C[i + (size_t)i * q] = 1.0;
    return P;
  }
  P.J = J;
  P.ex = {side == 0 ? d : 0};
  std::vector<cd> al(J), be(J);
  for (int j = 0; j < J; ++j) {
    P.xa.push_back(arc_point(A, -p[j]));
    P.xb.push_back(arc_point(A, p[j]));
    al[j] = em(P.xa[j]);
    be[j] = em(P.xb[j]);
  }
  const int q = 1 + J;
  P.C.assign((size_t)q * q, cd(0.0, 0.0));
  if (side == 0) {
    // Y on the far columns: cn = d_k, cv = d_k / n; C = blkdiag(1, diag(g) R_Y^T)
    std::vector<cd> cn, cv;
    for (int k = d + 1; k < n; ++k) {
      cn.push_back(em((double)k / n));
      cv.push_back(cn.back() / (double)n);
    }
    std::vector<cd> Y(cn.size() * J);
    fadi_y(cn, cv, al, be, Y, 0, (int)cn.size());
    const std::vector<cd> R = qr_r(Y, (int)cn.size(), J);
    P.C[0] = 1.0;
    for (int l = 0; l < J; ++l)
      for (int i = 0; i < J; ++i) P.C[(1 + l) + (size_t)(1 + i) * q] = (be[l] - al[l]) * R[i + (size_t)l * J];
  } else {
    // Y on the proxy of the outside arc: cn = s(x_P), cv = u(x_P) = s^n - 1, with the kernel
    // column of the unit direction first; C = diag(1, g) R^T
    const int np = FADI_PROXY_PER_COL * (n - d);
    std::vector<cd> cn(np), cv(np);
    std::vector<cd> Y((size_t)np * q);
    for (int i = 0; i < np; ++i) {
      const double x = (double)d / n + (i + 0.5) / ((double)FADI_PROXY_PER_COL * n);
      cn[i] = em(x);
      cv[i] = em((double)n * x) - 1.0;
      Y[i] = psi_host(x, 0, n);
    }
    fadi_y(cn, cv, al, be, Y, 1, np);
    const std::vector<cd> R = qr_r(Y, np, q);
    for (int l = 0; l < q; ++l) {
      const cd gl = l == 0 ? cd(1.0, 0.0) : be[l - 1] - al[l - 1];
      for (int i = 0; i < q; ++i) P.C[l + (size_t)i * q] = gl * R[i + (size_t)l * q];
    }
  }
  return P;
}

// ============================================================================ device kernels
template <typename R> struct FbD {
  const double* x;      // side 0: points (the dimension's sorted order)
  const int* cand;      // side 0: point positions; side 1: column indices
  int mc, side, n, c0, ne, J;
  const int* ex;        // ne exact columns (offsets from c0)
  const double2* al;    // J zeros, node frame
  const double2* be;    // J poles, node frame
  const double2* C;     // (ne + J)^2 column major
  cplx<R>* W; int ldw;  // (ne + J) x mc
};

__device__ __forceinline__ double2 cdivd(double2 a, double2 b) {
  const double s = 1.0 / (b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}

// One thread per candidate: the basis row a^T C, stored conjugated (side 0) or plain (side 1)
// as column c of W.
template <typename R> __global__ void __launch_bounds__(128) k_fadi_basis(const FbD<R>* __restrict__ ds) {
  const FbD<R> d = ds[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.mc) return;
  const int q = d.ne + d.J;
  double2 a[FB_MAXQ];
  if (d.side == 0) {
    const double x = d.x[d.cand[c]];
    for (int i = 0; i < d.ne; ++i) a[i] = psi_entry(x, (d.c0 + d.ex[i]) % d.n, d.n);
    if (d.J > 0) {
      const double xr = x - (double)d.c0 / (double)d.n;
      double sn, cs;
      sincospi(-2.0 * xr, &sn, &cs);
      const double2 s = make_double2(cs, sn);
      double t = (double)d.n * xr;
      t -= floor(t + 0.5);
      sincospi(-2.0 * t, &sn, &cs);
      double2 z = cdivd(make_double2(cs - 1.0, sn), s - d.be[0]);
      for (int i = 0; i < d.J; ++i) {
        a[d.ne + i] = z;
        if (i + 1 < d.J) z = z * cdivd(s - d.al[i], s - d.be[i + 1]);
      }
    }
  } else {
    const int kr = ((d.cand[c] - d.c0) % d.n + d.n) % d.n;
    bool isex = false;
    for (int i = 0; i < d.ne; ++i) {
      const bool e = kr == d.ex[i];
      a[i] = make_double2(e ? 1.0 : 0.0, 0.0);
      isex = isex || e;
    }
    if (d.J > 0) {
      if (isex) {
        for (int i = 0; i < d.J; ++i) a[d.ne + i] = make_double2(0.0, 0.0);
      } else {
        double sn, cs;
        sincospi(-2.0 * (double)kr / (double)d.n, &sn, &cs);
        const double2 dk = make_double2(cs, sn);
        double2 z = cdivd(make_double2(-cs / d.n, -sn / d.n), dk - d.be[0]);
        for (int i = 0; i < d.J; ++i) {
          a[d.ne + i] = z;
          if (i + 1 < d.J) z = z * cdivd(dk - d.al[i], dk - d.be[i + 1]);
        }
      }
    }
  }
  for (int i = 0; i < q; ++i) {
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < q; ++l) cfma(acc, a[l], d.C[l + (size_t)i * q]);
    if (d.side == 0) acc.y = -acc.y;
    d.W[i + (size_t)c * d.ldw] = mkc((R)acc.x, (R)acc.y);
  }
}

// out(i, j) = Psi(x[rows[i]], cols[j]; n): the kernel at skeleton points and skeleton columns
template <typename R> struct PsiIxD {
  const double* x; const int* rows; const int* cols; int m, nk, n; cplx<R>* out; int ld;
};
template <typename R> __global__ void __launch_bounds__(256) k_psi_idx(const PsiIxD<R>* __restrict__ ds) {
  const PsiIxD<R> d = ds[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.m * d.nk) return;
  const int i = t % d.m, j = t / d.m;
  const double2 v = psi_entry(d.x[d.rows[i]], d.cols[j], d.n);
  d.out[(size_t)i + (size_t)j * d.ld] = mkc((R)v.x, (R)v.y);
}

// |R_kk| of a pivoted QR into one array (one CTA per matrix)
template <typename R> struct DgD { const cplx<R>* A; int lda, k; R* out; };
template <typename R> __global__ void k_id_diag(const DgD<R>* __restrict__ ds) {
  const DgD<R> d = ds[blockIdx.x];
  for (int i = threadIdx.x; i < d.k; i += blockDim.x) d.out[i] = sqrt(abs2(d.A[(size_t)i + (size_t)i * d.lda]));
}

// ============================================================================ interpolative decomposition
template <typename R>
void Ops<R>::row_id(const std::vector<Mat<R>>& W, double tol, Arena& keep, std::vector<Mat<R>>& T,
                    std::vector<std::vector<int>>& sk) {
  const size_t nm = W.size();
  T.assign(nm, Mat<R>());
  sk.assign(nm, {});
  auto mk = ar_->mark();
  std::vector<size_t> poff(nm, 0), doff(nm, 0);
  size_t ptot = 0, dtot = 0;
  std::vector<int> act;
  int nmax = 0, pmax = 0;
  for (size_t i = 0; i < nm; ++i) {
    if (W[i].m <= 0 || W[i].n <= 0) continue;
    NH_REQUIRE(W[i].m <= 1024, ST_EINVAL, "row_id: a basis has more than 1024 columns");
    act.push_back((int)i);
    poff[i] = ptot;
    ptot += W[i].n;
    doff[i] = dtot;
    dtot += std::min(W[i].m, W[i].n);
    nmax = std::max(nmax, W[i].n);
    pmax = std::max(pmax, std::min(W[i].m, W[i].n));
  }
  if (act.empty()) { ar_->release(mk); return; }
  int* perm = ar_->template arr<int>(ptot);
  R* dg = ar_->template arr<R>(dtot);
  std::vector<QpD<R>> qp;
  std::vector<DgD<R>> dd;
  for (int i : act) {
    QpD<R> q;
    q.A = W[i].p; q.lda = W[i].ld; q.m = W[i].m; q.n = W[i].n;
    q.perm = perm + poff[i];
    q.vn1 = ar_->template arr<R>(W[i].n);
    q.vn2 = ar_->template arr<R>(W[i].n);
    q.v = ar_->template arr<cplx<R>>(W[i].m);
    q.tau = ar_->template arr<R>(1);
    qp.push_back(q);
    dd.push_back({W[i].p, W[i].ld, std::min(W[i].m, W[i].n), dg + doff[i]});
  }
  const R tol3z = (R)std::sqrt(sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08);
  auto dq = (const QpD<R>*)stage(qp.data(), qp.size() * sizeof(QpD<R>));
  prof.begin(st_);
  k_qp_init<R><<<dim3((nmax + 7) / 8, (unsigned)qp.size()), 256, 0, st_>>>(dq);
  NH_LAUNCH_CK();
  count();
  for (int kk = 0; kk < pmax; ++kk) {
    k_qp_pivot<R><<<(int)qp.size(), 256, 0, st_>>>(dq, kk);
    NH_LAUNCH_CK();
    const int cols = nmax - kk - 1;
    if (cols > 0) {
      k_qp_update_cta<R, 4><<<dim3((unsigned)cols, (unsigned)qp.size()), 256, 0, st_>>>(dq, kk, tol3z);
      NH_LAUNCH_CK();
    }
    count(2);
  }
  auto ddd = (const DgD<R>*)stage(dd.data(), dd.size() * sizeof(DgD<R>));
  k_id_diag<R><<<(int)dd.size(), 128, 0, st_>>>(ddd);
  NH_LAUNCH_CK();
  count();
  prof.end(st_, K_QRCP, 0, 0, 2 + 2 * pmax);
  std::vector<int> hperm(ptot);
  std::vector<R> hdg(dtot);
  NH_CK(cudaMemcpyAsync(hperm.data(), perm, ptot * sizeof(int), cudaMemcpyDeviceToHost, st_));
  NH_CK(cudaMemcpyAsync(hdg.data(), dg, dtot * sizeof(R), cudaMemcpyDeviceToHost, st_));
  NH_CK(cudaStreamSynchronize(st_));
  // ranks, skeletons and the inverse permutations (host)
  std::vector<int> rk(nm, 0), inv(ptot);
  std::vector<Mat<R>> tri, triX, Tp;
  std::vector<GemmD<R>> gm;
  std::vector<CopyD<R>> cp;
  std::vector<Mat<R>> Xs(nm);
  // a basis whose largest pivot is (numerically) zero is the zero block: on points exactly on the
  // grid k/n the kernel entries are exact zeros.  It keeps rank 1 with T = the unit vector of its
  // first pivot (an exact ID of the zero block) instead of inverting a zero R_11.
  const double zero_pivot = sizeof(R) == 8 ? 1e-300 : 1e-30;
  for (int i : act) {
    const int mc = W[i].n, p = std::min(W[i].m, W[i].n);
    const R* g = hdg.data() + doff[i];
    const double cut = tol * (double)g[0];
    const bool zero = !((double)g[0] > zero_pivot);
    int r = 0;
    if (!zero)
      while (r < p && (double)g[r] > cut) ++r;
    r = std::max(r, 1);
    rk[i] = r;
    const int* pm = hperm.data() + poff[i];
    sk[i].assign(pm, pm + r);
    for (int j = 0; j < mc; ++j) inv[poff[i] + pm[j]] = j;
    Mat<R> tp = ar_->template mat<R>(mc, r);   // [I; X^*] in pivot order (set_identity below)
    Tp.push_back(tp);
    if (zero) continue;
    // X = R11^{-1} R12 (r x (mc - r))
    Mat<R> S = ar_->template mat<R>(r, r);
    tri.push_back(W[i].block(0, 0, r, r));
    triX.push_back(S);
    if (mc > r) {
      Xs[i] = ar_->template mat<R>(r, mc - r);
      gm.push_back({S.p, W[i].at(0, r), Xs[i].p, r, mc - r, r, S.ld, W[i].ld, Xs[i].ld, OP_N, OP_N, R(1), R(0)});
      cp.push_back({Xs[i].p, tp.at(r, 0), mc - r, r, Xs[i].ld, tp.ld, OP_C, R(1), R(0)});
    }
  }
  trinv(tri, triX);
  gemm(gm);
  set_identity(Tp);
  copy(cp);
  // T(i, :) = Tp(inv[i], :)
  int* dinv = upload_ints(inv);
  std::vector<GatherD<R>> ga;
  size_t t = 0;
  for (int i : act) {
    const int mc = W[i].n, r = rk[i];
    T[i] = keep.template mat<R>(mc, r);
    ga.push_back({Tp[t].p, T[i].p, dinv + poff[i], mc, r, Tp[t].ld, T[i].ld, 0});
    ++t;
  }
  gather(ga);
  ar_->release(mk);
}

template void Ops<double>::row_id(const std::vector<Mat<double>>&, double, Arena&, std::vector<Mat<double>>&,
                                  std::vector<std::vector<int>>&);
template void Ops<float>::row_id(const std::vector<Mat<float>>&, double, Arena&, std::vector<Mat<float>>&,
                                 std::vector<std::vector<int>>&);

// ============================================================================ nested 1D HSS
// C = op(A) op(B) descriptor for blocks of column-major matrices
template <typename R> static GemmD<R> gemm_d(const Mat<R>& A, const Mat<R>& B, const Mat<R>& C) {
  return GemmD<R>{A.p, B.p, C.p, C.m, C.n, A.n, A.ld, B.ld, C.ld, OP_N, OP_N, R(1), R(0)};
}

template <typename R> const FadiPlan& Hss<R>::fadi_plan_of(int side, int d, int n, double eps1) {
  const auto key = std::make_tuple(side, d, n);
  auto it = fplans_.find(key);
  if (it == fplans_.end()) it = fplans_.emplace(key, fadi_plan(side, d, n, eps1, FADI_JMAX)).first;
  return it->second;
}

template <typename R>
void Hss<R>::build_1d_fadi(const Tree1D& t, const double* xo, double eps1, std::vector<std::vector<Gen1D<R>>>& g) {
  const int L = t.L, n = t.n;
  g.assign(L + 1, {});
  for (int l = 0; l <= L; ++l) g[l].resize(t.c0[l].size());
  // the pivot cut stays above the rounding level of the working precision (FP32 in MIXED mode)
  const double idtol = std::max(FADI_ID_TOL * eps1, sizeof(R) == 4 ? 1.2e-7 : 0.0);
  // host skeletons per node of the level below the current one: point positions, columns
  std::vector<std::vector<int>> srow, scol;
  std::vector<std::vector<std::vector<int>>> Srow(L + 1), Scol(L + 1);
  for (int l = L; l >= 1; --l) {
    auto mk = scr_.mark();
    auto tk = tmp_.mark();
    const int nn = (int)t.c0[l].size();
    std::vector<std::vector<int>> crow(nn), ccol(nn);
    for (int i = 0; i < nn; ++i) {
      const int c0 = t.c0[l][i], c1 = t.c1[l][i];
      if (l == L) {
        for (int j = 0; j < t.m[L][i]; ++j) crow[i].push_back(t.r0[L][i] + j);
        for (int k = c0; k < c1; ++k) ccol[i].push_back(k);
      } else {
        for (int c = 0; c < 2; ++c) {
          crow[i].insert(crow[i].end(), Srow[l + 1][2 * i + c].begin(), Srow[l + 1][2 * i + c].end());
          ccol[i].insert(ccol[i].end(), Scol[l + 1][2 * i + c].begin(), Scol[l + 1][2 * i + c].end());
        }
      }
    }
    // bases: W[i] (rows of node i), W[nn + i] (columns of node i)
    std::vector<Mat<R>> W(2 * nn);
    std::vector<FbD<R>> fb;
    std::vector<int> cand_all;
    std::vector<size_t> coff(2 * nn);
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < nn; ++i) {
        coff[s * nn + i] = cand_all.size();
        const auto& cl = s == 0 ? crow[i] : ccol[i];
        cand_all.insert(cand_all.end(), cl.begin(), cl.end());
      }
    int* dcand = ops_.upload_ints(cand_all.empty() ? std::vector<int>{0} : cand_all);
    int mcmax = 0;
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < nn; ++i) {
        const int c0 = t.c0[l][i], d = t.c1[l][i] - t.c0[l][i];
        const int mc = (int)(s == 0 ? crow[i] : ccol[i]).size();
        const FadiPlan& P = fadi_plan_of(s, d, n, eps1);
        const int q = P.q();
        NH_REQUIRE(q <= FB_MAXQ, ST_EINVAL, "fADI basis wider than 65 columns");
        W[s * nn + i] = tmp_.mat<R>(q, mc);
        if (mc == 0) continue;
        // plan data: ex, alpha, beta, C
        std::vector<double2> hab(2 * (size_t)std::max(P.J, 1)), hc((size_t)q * q);
        for (int j = 0; j < P.J; ++j) {
          const cd a = std::exp(cd(0.0, -2.0 * FADI_PI * P.xa[j]));
          const cd b = std::exp(cd(0.0, -2.0 * FADI_PI * P.xb[j]));
          hab[j] = make_double2(a.real(), a.imag());
          hab[P.J + j] = make_double2(b.real(), b.imag());
        }
        for (size_t e = 0; e < hc.size(); ++e) hc[e] = make_double2(P.C[e].real(), P.C[e].imag());
        auto dab = (double2*)Ops<R>::stage_cb(&ops_, hab.data(), hab.size() * sizeof(double2));
        auto dc = (double2*)Ops<R>::stage_cb(&ops_, hc.data(), hc.size() * sizeof(double2));
        int* dex = ops_.upload_ints(P.ex);
        FbD<R> f;
        f.x = xo; f.cand = dcand + coff[s * nn + i]; f.mc = mc; f.side = s; f.n = n; f.c0 = c0;
        f.ne = (int)P.ex.size(); f.J = P.J; f.ex = dex; f.al = dab; f.be = dab + P.J; f.C = dc;
        f.W = W[s * nn + i].p; f.ldw = W[s * nn + i].ld;
        fb.push_back(f);
        mcmax = std::max(mcmax, mc);
      }
    if (!fb.empty()) {
      auto dfb = (const FbD<R>*)Ops<R>::stage_cb(&ops_, fb.data(), fb.size() * sizeof(FbD<R>));
      k_fadi_basis<R><<<dim3((mcmax + 127) / 128, (unsigned)fb.size()), 128, 0, st_>>>(dfb);
      NH_LAUNCH_CK();
      ops_.count();
    }
    std::vector<Mat<R>> T;
    std::vector<std::vector<int>> sk;
    ops_.row_id(W, idtol, keep_, T, sk);
    Srow[l].assign(nn, {});
    Scol[l].assign(nn, {});
    std::vector<GemmD<R>> gv;
    for (int i = 0; i < nn; ++i) {
      for (int j : sk[i]) Srow[l][i].push_back(crow[i][j]);
      for (int j : sk[nn + i]) Scol[l][i].push_back(ccol[i][j]);
      Gen1D<R>& q = g[l][i];
      q.ru = (int)sk[i].size();
      q.rv = (int)sk[nn + i].size();
      if (l == L) {
        q.U = T[i];
        q.V = T[nn + i];
        continue;
      }
      Gen1D<R>& a = g[l + 1][2 * i];
      Gen1D<R>& b = g[l + 1][2 * i + 1];
      q.Rst = T[i];
      q.Wst = T[nn + i];
      a.R_ = q.Rst.block(0, 0, a.ru, q.ru);
      b.R_ = q.Rst.block(a.ru, 0, b.ru, q.ru);
      a.W = q.Wst.block(0, 0, a.rv, q.rv);
      b.W = q.Wst.block(a.rv, 0, b.rv, q.rv);
      // explicit column basis of the node: [V_a W_a; V_b W_b]
      const int d = t.c1[l][i] - t.c0[l][i];
      const int da = t.c1[l + 1][2 * i] - t.c0[l + 1][2 * i];
      q.V = keep_.mat<R>(d, q.rv);
      gv.push_back(gemm_d<R>(a.V, a.W, q.V.block(0, 0, da, q.rv)));
      gv.push_back(gemm_d<R>(b.V, b.W, q.V.block(da, 0, d - da, q.rv)));
    }
    ops_.gemm(gv);
    tmp_.release(tk);
    scr_.release(mk);
  }
  // B of every sibling pair: the kernel at a's skeleton points and b's skeleton columns
  {
    auto mk = scr_.mark();
    std::vector<PsiIxD<R>> pd;
    std::vector<int> idx;
    std::vector<std::pair<size_t, size_t>> off;
    int tmax = 0;
    for (int l = 1; l <= L; ++l)
      for (int i = 0; i < (int)t.c0[l].size(); ++i) {
        Gen1D<R>& a = g[l][i];
        const int sib = i ^ 1;
        a.Bs = keep_.mat<R>(a.ru, g[l][sib].rv);
        const size_t o1 = idx.size();
        idx.insert(idx.end(), Srow[l][i].begin(), Srow[l][i].end());
        const size_t o2 = idx.size();
        idx.insert(idx.end(), Scol[l][sib].begin(), Scol[l][sib].end());
        off.push_back({o1, o2});
        tmax = std::max(tmax, a.ru * g[l][sib].rv);
      }
    int* didx = ops_.upload_ints(idx.empty() ? std::vector<int>{0} : idx);
    size_t e = 0;
    for (int l = 1; l <= L; ++l)
      for (int i = 0; i < (int)t.c0[l].size(); ++i, ++e) {
        Gen1D<R>& a = g[l][i];
        const int nk = g[l][i ^ 1].rv;
        if (a.ru > 0 && nk > 0)
          pd.push_back({xo, didx + off[e].first, didx + off[e].second, a.ru, nk, n, a.Bs.p, a.Bs.ld});
      }
    if (!pd.empty()) {
      auto dpd = (const PsiIxD<R>*)Ops<R>::stage_cb(&ops_, pd.data(), pd.size() * sizeof(PsiIxD<R>));
      k_psi_idx<R><<<dim3((tmax + 255) / 256, (unsigned)pd.size()), 256, 0, st_>>>(dpd);
      NH_LAUNCH_CK();
      ops_.count();
    }
    NH_CK(cudaStreamSynchronize(st_));
    scr_.release(mk);
  }
}

template const FadiPlan& Hss<double>::fadi_plan_of(int, int, int, double);
template const FadiPlan& Hss<float>::fadi_plan_of(int, int, int, double);
template void Hss<double>::build_1d_fadi(const Tree1D&, const double*, double, std::vector<std::vector<Gen1D<double>>>&);
template void Hss<float>::build_1d_fadi(const Tree1D&, const double*, double, std::vector<std::vector<Gen1D<float>>>&);

}  // namespace nh

// Host-only view of a node's fADI plan (no device work), for tests of the shift computation.
extern "C" int nudft2_fadi_plan(int side, int d, int n, double eps1, int* ne, int* J, int* ex, double* xa,
                                double* xb, double* C, double* ratio) {
  try {
    const nh::FadiPlan P = nh::fadi_plan(side, d, n, eps1, nh::FADI_JMAX);
    *ne = (int)P.ex.size();
    *J = P.J;
    for (size_t i = 0; i < P.ex.size(); ++i) ex[i] = P.ex[i];
    for (int j = 0; j < P.J; ++j) { xa[j] = P.xa[j]; xb[j] = P.xb[j]; }
    for (size_t e = 0; e < P.C.size(); ++e) { C[2 * e] = P.C[e].real(); C[2 * e + 1] = P.C[e].imag(); }
    *ratio = P.ratio;
    return 0;
  } catch (const nh::Error& e) {
    return e.code;
  } catch (...) {
    return 3;
  }
}
