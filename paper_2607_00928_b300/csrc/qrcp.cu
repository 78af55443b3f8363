// Column-pivoted Householder QR by blocks of pivots chosen on a random sketch: the rank-revealing
// first step of the truncated SVD (pivoted QR, then one-sided Jacobi on R^*), without the
// per-pivot pass over the whole trailing matrix of the classical pivoted QR.
//
// The scheme follows Martinsson, Quintana-Orti, Heavner and van de Geijn, "Householder QR
// factorization with randomization for column pivoting (HQRRP)", SIAM J. Sci. Comput. 39 (2017):
// the pivots of a block of b columns are the first b pivots of a column-pivoted QR of the sketch
// Y = G A22 (G a Gaussian d x rows matrix, d = b + 8: column norms and mutual angles of A22 are
// kept to within small factors), then the block is factored by an unpivoted Householder panel and
// the trailing matrix updated by GEMMs of depth b.  Here every block draws a fresh G (instead of
// down-dating one sketch: the down-dating formula divides by the block's R11, which is
// ill-conditioned exactly where the truncation stops).
//
// Stopping rule (the pre-truncation of the SVD): with cut = 0.01 eps max_c ||A e_c||, the
// factorization stops before block j when every column of the trailing matrix A22 has norm
// <= cut; the rows factored so far are returned as p_eff and the dropped block has 2-norm at
// most sqrt(cols) cut.  The sketch norms estimate the trailing column norms (E ||G x||^2 = d
// ||x||^2), so the exact norms are only computed once the estimate is within a factor 4 of the
// cut.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "la.cuh"
#include "qp.cuh"

namespace nh {

namespace {
constexpr int QS_B = 32;            // pivots per block (the Householder panel width)
constexpr int QS_D = QS_B + 8;      // sketch rows
constexpr int QS_LIST = 2 * QS_B;   // positions a block's pivot swaps can move
}  // namespace

// complex standard normal entries (E|g|^2 = 1): a splitmix64 hash of (seed, index) gives two
// uniforms, Box-Muller turns them into the real and imaginary parts
__host__ __device__ __forceinline__ unsigned long long qs_mix(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
template <typename R>
__global__ void k_gauss(cplx<R>* __restrict__ g, long long n, unsigned long long seed) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long h = qs_mix(seed ^ qs_mix((unsigned long long)i));
  const double u1 = ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);            // (0, 1)
  const double u2 = (double)(qs_mix(h) >> 11) * (1.0 / 9007199254740992.0);             // [0, 1)
  const double r = sqrt(-log(u1));                                                      // sqrt(-2 ln u1) / sqrt(2)
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  g[i] = mkc(R(r * c), R(r * s));
}

template <typename R> struct QsD {
  cplx<R>* A; int lda, m, n;    // the whole matrix
  int j;                        // first column of this block
  int* gperm;                   // gperm[c] = original column now at position c
  const int* psub;              // the sketch's pivoted order of columns j.. (from its QRCP)
  int* list; int* cnt;          // positions (relative to j) the swaps moved, and their count
  cplx<R>* tmp; int* tmpi;      // rows x QS_LIST columns, QS_LIST ints
  R* out;                       // one value per matrix (max norms)
};

// largest column norm of A[j:, j:] (one warp per column), as the bits of a nonnegative float
template <typename R>
__global__ void __launch_bounds__(256) k_qs_maxnorm(const QsD<R>* __restrict__ ds, unsigned long long* __restrict__ out) {
  const QsD<R> d = ds[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = d.j + blockIdx.x * 8 + warp;
  if (c >= d.n) return;
  const cplx<R>* col = d.A + (size_t)c * d.lda;
  double s = 0;
  for (int i = d.j + lane; i < d.m; i += 32) s += (double)abs2(col[i]);
  s = warp_sum(s);
  if (lane == 0) atomicMax(&out[blockIdx.y], (unsigned long long)__double_as_longlong(sqrt(s)));
}

// largest sketch column norm (the QRCP's initial norms vn1[0 .. n)), one CTA per matrix
template <typename R>
__global__ void __launch_bounds__(256) k_qs_vmax(const QpD<R>* __restrict__ qd, double* __restrict__ out) {
  const QpD<R> d = qd[blockIdx.x];
  __shared__ double red[8];
  double m = 0;
  for (int c = threadIdx.x; c < d.n; c += 256) m = fmax(m, (double)d.vn1[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t = fmax(t, red[w]);
    out[blockIdx.x] = t;
  }
}

// positions q (relative to j) whose column the sketch's pivoting moved
template <typename R> __global__ void k_qs_list(const QsD<R>* __restrict__ ds) {
  const QsD<R> d = ds[blockIdx.y];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.n - d.j) return;
  if (d.psub[q] != q) {
    const int t = atomicAdd(d.cnt, 1);
    if (t < QS_LIST) d.list[t] = q;
  }
}

// tmp[:, t] = A[:, j + psub[list[t]]] (all rows), tmpi[t] = gperm[j + psub[list[t]]]
template <typename R> __global__ void __launch_bounds__(256) k_qs_gather(const QsD<R>* __restrict__ ds) {
  const QsD<R> d = ds[blockIdx.y];
  const int t = blockIdx.x;
  if (t >= min(*d.cnt, QS_LIST)) return;
  const int src = d.j + d.psub[d.list[t]];
  const cplx<R>* a = d.A + (size_t)src * d.lda;
  cplx<R>* o = d.tmp + (size_t)t * d.m;
  for (int i = threadIdx.x; i < d.m; i += 256) o[i] = a[i];
  if (threadIdx.x == 0) d.tmpi[t] = d.gperm[src];
}

// A[:, j + list[t]] = tmp[:, t], gperm[j + list[t]] = tmpi[t]
template <typename R> __global__ void __launch_bounds__(256) k_qs_scatter(const QsD<R>* __restrict__ ds) {
  const QsD<R> d = ds[blockIdx.y];
  const int t = blockIdx.x;
  if (t >= min(*d.cnt, QS_LIST)) return;
  const int dst = d.j + d.list[t];
  cplx<R>* a = d.A + (size_t)dst * d.lda;
  const cplx<R>* o = d.tmp + (size_t)t * d.m;
  for (int i = threadIdx.x; i < d.m; i += 256) a[i] = o[i];
  if (threadIdx.x == 0) d.gperm[dst] = d.tmpi[t];
}

template <typename R> __global__ void k_qs_iota(int* __restrict__ p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

template <typename R>
void Ops<R>::qrcp_sketch(const std::vector<Mat<R>>& A, const std::vector<int*>& perm, double eps,
                         std::vector<int>& peff) {
  const size_t nm = A.size();
  peff.assign(nm, 0);
  auto mk = ar_->mark();
  const R tol3z = (R)std::sqrt(sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08);
  std::vector<int> act;
  int mmax = 0;
  for (size_t i = 0; i < nm; ++i) {
    const int k = std::min(A[i].m, A[i].n);
    if (k <= 0) continue;
    act.push_back((int)i);
    mmax = std::max(mmax, A[i].m);
    k_qs_iota<R><<<(A[i].n + 255) / 256, 256, 0, st_>>>(perm[i], A[i].n);
    NH_LAUNCH_CK();
    count();
  }
  if (act.empty()) { ar_->release(mk); return; }
  // per-matrix scratch: sketch (d x n), its QRCP state, swap list and staging columns
  struct Sc { cplx<R>* Y; int* psub; R* vn1; R* vn2; cplx<R>* v; R* tau; int* list; int* cnt; cplx<R>* tmp; int* tmpi; };
  std::vector<Sc> sc(nm);
  for (int i : act) {
    Sc& s = sc[i];
    const int n = A[i].n;
    s.Y = ar_->template arr<cplx<R>>((size_t)QS_D * n);
    s.psub = ar_->template arr<int>(n);
    s.vn1 = ar_->template arr<R>(n);
    s.vn2 = ar_->template arr<R>(n);
    s.v = ar_->template arr<cplx<R>>(QS_D);
    s.tau = ar_->template arr<R>(1);
    s.list = ar_->template arr<int>(QS_LIST);
    s.cnt = ar_->template arr<int>(1);
    s.tmp = ar_->template arr<cplx<R>>((size_t)A[i].m * QS_LIST);
    s.tmpi = ar_->template arr<int>(QS_LIST);
  }
  cplx<R>* G = ar_->template arr<cplx<R>>((size_t)QS_D * mmax);
  unsigned long long* nrm_bits = ar_->template arr<unsigned long long>(nm);
  double* vmax = ar_->template arr<double>(nm);
  std::vector<unsigned long long> hbits(nm);
  std::vector<double> hv(nm);
  // max column norm of each matrix -> cut
  auto maxnorms = [&](const std::vector<int>& ids, int j) {
    std::vector<QsD<R>> qd;
    int cmax = 0;
    for (int i : ids) {
      QsD<R> q{};
      q.A = A[i].p; q.lda = A[i].ld; q.m = A[i].m; q.n = A[i].n; q.j = j;
      qd.push_back(q);
      cmax = std::max(cmax, A[i].n - j);
    }
    NH_CK(cudaMemsetAsync(nrm_bits, 0, nm * sizeof(unsigned long long), st_));
    auto dq = (const QsD<R>*)stage(qd.data(), qd.size() * sizeof(QsD<R>));
    k_qs_maxnorm<R><<<dim3((cmax + 7) / 8, (unsigned)ids.size()), 256, 0, st_>>>(dq, nrm_bits);
    NH_LAUNCH_CK();
    count();
    NH_CK(cudaMemcpyAsync(hbits.data(), nrm_bits, ids.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          st_));
    NH_CK(cudaStreamSynchronize(st_));
    std::vector<double> out(ids.size());
    for (size_t q = 0; q < ids.size(); ++q) std::memcpy(&out[q], &hbits[q], sizeof(double));
    return out;
  };
  Arena pk((size_t)64 << 20);   // the panels' reflectors (qr() releases its scratch arena)
  pk.set_stream(st_);
  std::vector<double> cut(nm, 0.0);
  {
    auto n0 = maxnorms(act, 0);
    for (size_t q = 0; q < act.size(); ++q) cut[act[q]] = 0.01 * eps * n0[q];
  }
  // the seed depends only on the shapes: the same input gives the same pivots (and factors) on
  // every run and from every thread
  unsigned long long seed = qs_mix((unsigned long long)nm);
  for (size_t i = 0; i < nm; ++i) seed = qs_mix(seed ^ ((unsigned long long)A[i].m << 32 | (unsigned)A[i].n));
  for (int j = 0; !act.empty(); j += QS_B) {
    // ---- fresh sketch Y = G A[j:, j:] of every active matrix
    int mr = 0;
    for (int i : act) mr = std::max(mr, A[i].m - j);
    {
      const long long ng = (long long)QS_D * mr;
      k_gauss<R><<<(unsigned)((ng + 255) / 256), 256, 0, st_>>>(G, ng, seed + 0x1000003ull * (unsigned long long)j);
      NH_LAUNCH_CK();
      count();
      std::vector<GemmD<R>> gy;
      for (int i : act)
        gy.push_back({G, A[i].p + (size_t)j + (size_t)j * A[i].ld, sc[i].Y, QS_D, A[i].n - j, A[i].m - j, QS_D,
                      A[i].ld, QS_D, OP_N, OP_N, R(1), R(0)});
      gemm(gy);
    }
    prof.begin(st_);
    std::vector<QpD<R>> qp;
    int nmax = 0;
    for (int i : act) {
      QpD<R> q;
      q.A = sc[i].Y; q.lda = QS_D; q.m = QS_D; q.n = A[i].n - j;
      q.perm = sc[i].psub; q.vn1 = sc[i].vn1; q.vn2 = sc[i].vn2; q.v = sc[i].v; q.tau = sc[i].tau;
      qp.push_back(q);
      nmax = std::max(nmax, q.n);
    }
    auto dq = (const QpD<R>*)stage(qp.data(), qp.size() * sizeof(QpD<R>));
    k_qp_init<R><<<dim3((nmax + 7) / 8, (unsigned)qp.size()), 256, 0, st_>>>(dq);
    NH_LAUNCH_CK();
    k_qs_vmax<R><<<(int)qp.size(), 256, 0, st_>>>(dq, vmax);
    NH_LAUNCH_CK();
    count(2);
    prof.end(st_, K_QRCP, 0, 0, 2);
    // ---- stopping rule: estimate from the sketch, exact norms when the estimate is close
    NH_CK(cudaMemcpyAsync(hv.data(), vmax, act.size() * sizeof(double), cudaMemcpyDeviceToHost, st_));
    NH_CK(cudaStreamSynchronize(st_));
    std::vector<int> chk;
    for (size_t q = 0; q < act.size(); ++q)
      if (hv[q] / std::sqrt((double)QS_D) <= 4.0 * cut[act[q]]) chk.push_back(act[q]);
    if (!chk.empty()) {
      auto nj = maxnorms(chk, j);
      std::vector<int> stop;
      for (size_t q = 0; q < chk.size(); ++q)
        if (nj[q] <= cut[chk[q]]) stop.push_back(chk[q]);
      if (!stop.empty()) {
        for (int i : stop) peff[i] = j;
        std::vector<int> keep_act;
        for (int i : act)
          if (std::find(stop.begin(), stop.end(), i) == stop.end()) keep_act.push_back(i);
        act.swap(keep_act);
        if (act.empty()) break;
        qp.clear();
        nmax = 0;
        for (int i : act) {
          QpD<R> q;
          q.A = sc[i].Y; q.lda = QS_D; q.m = QS_D; q.n = A[i].n - j;
          q.perm = sc[i].psub; q.vn1 = sc[i].vn1; q.vn2 = sc[i].vn2; q.v = sc[i].v; q.tau = sc[i].tau;
          qp.push_back(q);
          nmax = std::max(nmax, q.n);
        }
        dq = (const QpD<R>*)stage(qp.data(), qp.size() * sizeof(QpD<R>));
      }
    }
    // ---- the block's pivots: QS_B steps of the pivoted QR of the sketch
    prof.begin(st_);
    for (int kk = 0; kk < QS_B; ++kk) {
      k_qp_pivot<R><<<(int)qp.size(), 256, 0, st_>>>(dq, kk);
      NH_LAUNCH_CK();
      const int cols = nmax - kk - 1;
      if (cols > 0) {
        k_qp_update_cta<R, 4><<<dim3((unsigned)cols, (unsigned)qp.size()), 256, 0, st_>>>(dq, kk, tol3z);
        NH_LAUNCH_CK();
      }
      count(2);
    }
    // ---- move the chosen columns (and the ones they displaced) in A and in the permutation
    std::vector<QsD<R>> sd;
    for (int i : act) {
      QsD<R> q{};
      q.A = A[i].p; q.lda = A[i].ld; q.m = A[i].m; q.n = A[i].n; q.j = j;
      q.gperm = perm[i]; q.psub = sc[i].psub; q.list = sc[i].list; q.cnt = sc[i].cnt;
      q.tmp = sc[i].tmp; q.tmpi = sc[i].tmpi;
      NH_CK(cudaMemsetAsync(sc[i].cnt, 0, sizeof(int), st_));
      sd.push_back(q);
    }
    auto ds = (const QsD<R>*)stage(sd.data(), sd.size() * sizeof(QsD<R>));
    k_qs_list<R><<<dim3((nmax + 255) / 256, (unsigned)sd.size()), 256, 0, st_>>>(ds);
    NH_LAUNCH_CK();
    k_qs_gather<R><<<dim3(QS_LIST, (unsigned)sd.size()), 256, 0, st_>>>(ds);
    NH_LAUNCH_CK();
    k_qs_scatter<R><<<dim3(QS_LIST, (unsigned)sd.size()), 256, 0, st_>>>(ds);
    NH_LAUNCH_CK();
    count(3);
    prof.end(st_, K_QRCP, 0, 0, 2 * QS_B + 3);
    // ---- unpivoted panel of the block, then the trailing matrix
    std::vector<Mat<R>> pan, trail;
    std::vector<int> tr_of;
    for (int i : act) {
      const int bj = std::min(QS_B, std::min(A[i].m, A[i].n) - j);
      pan.push_back(A[i].block(j, j, A[i].m - j, bj));
    }
    auto pm = pk.mark();
    auto Q = qr(pan, pk);
    std::vector<QFac<R>> qf;
    for (size_t q = 0; q < act.size(); ++q) {
      const int i = act[q];
      const int bj = pan[q].n, n2 = A[i].n - j - bj;
      if (n2 <= 0) continue;
      trail.push_back(A[i].block(j, j + bj, A[i].m - j, n2));
      qf.push_back(Q[q]);
    }
    if (!trail.empty()) apply_q_left(qf, trail, true);
    pk.release(pm);
    // matrices whose last block this was
    std::vector<int> keep_act;
    for (int i : act) {
      if (j + QS_B >= std::min(A[i].m, A[i].n)) peff[i] = std::min(A[i].m, A[i].n);
      else keep_act.push_back(i);
    }
    act.swap(keep_act);
  }
  ar_->release(mk);
}

template void Ops<double>::qrcp_sketch(const std::vector<Mat<double>>&, const std::vector<int*>&, double,
                                       std::vector<int>&);
template void Ops<float>::qrcp_sketch(const std::vector<Mat<float>>&, const std::vector<int*>&, double,
                                      std::vector<int>&);

}  // namespace nh
