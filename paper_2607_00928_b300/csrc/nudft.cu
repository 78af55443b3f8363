// NUDFT-specific kernels (see nudft.cuh).
#include <algorithm>

#include "nudft.cuh"

namespace nh {

static int* up_ints(Arena& ar, cudaStream_t st, const std::vector<int>& v) {
  int* d = (int*)ar.alloc(v.size() * sizeof(int));
  NH_CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  return d;
}

__device__ __forceinline__ int find_prob2(const int* pre, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- kernel entries (Sec. 2.4)
template <typename R>
__global__ void k_psi(const PsiD<R>* __restrict__ ds, const int* __restrict__ pre, int np) {
  const int pi = find_prob2(pre, np, blockIdx.x);
  const PsiD<R> d = ds[pi];
  const int lt = blockIdx.x - pre[pi];
  const int tm = (d.m + 31) / 32;
  const int i = (lt % tm) * 32 + (threadIdx.x & 31);
  const int j0 = (lt / tm) * 32;
  if (i >= d.m) return;
  const double x = d.x[i];
  for (int jj = threadIdx.x >> 5; jj < 32; jj += 8) {
    const int k = j0 + jj;
    if (k >= d.nk) break;
    const double2 v = psi_entry(x, d.k0 + k, d.n);
    d.out[(size_t)i + (size_t)k * d.ld] = mkc((R)v.x, (R)v.y);
  }
}

template <typename R> void psi_eval(Ops<R>& ops, const std::vector<PsiD<R>>& d0) {
  std::vector<PsiD<R>> d;
  std::vector<int> pre;
  int tiles = 0;
  for (auto& p : d0) {
    if (p.m <= 0 || p.nk <= 0) continue;
    d.push_back(p);
    pre.push_back(tiles);
    tiles += ((p.m + 31) / 32) * ((p.nk + 31) / 32);
  }
  if (d.empty()) return;
  Arena& ar = *ops.scratch();
  PsiD<R>* dd = (PsiD<R>*)ar.alloc(d.size() * sizeof(PsiD<R>));
  NH_CK(cudaMemcpyAsync(dd, d.data(), d.size() * sizeof(PsiD<R>), cudaMemcpyHostToDevice, ops.stream()));
  int* dp = up_ints(ar, ops.stream(), pre);
  k_psi<R><<<tiles, 256, 0, ops.stream()>>>(dd, dp, (int)d.size());
  NH_LAUNCH_CK();
  ops.count();
}
template void psi_eval<double>(Ops<double>&, const std::vector<PsiD<double>>&);
template void psi_eval<float>(Ops<float>&, const std::vector<PsiD<float>>&);

// ---------------------------------------------------------------- exact apply helpers (Eq. 1)
__global__ void k_twiddle(const double* __restrict__ x, int M, int n, double2* __restrict__ tab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double xj = x[j];
  for (int k = blockIdx.y; k < n; k += gridDim.y) {
    const double p = (double)k * xj;
    const double e = fma((double)k, xj, -p);    // exact rounding error of the product
    double t = (p - floor(p)) + e;
    t -= floor(t + 0.5);
    double s, c;
    sincospi(2.0 * t, &s, &c);
    tab[(size_t)j + (size_t)k * M] = make_double2(c, -s);
  }
}

void twiddle_table(cudaStream_t st, const double* x, int M, int n, double2* tab) {
  if (M <= 0 || n <= 0) return;
  dim3 grid((M + 255) / 256, std::min(n, 64));
  k_twiddle<<<grid, 256, 0, st>>>(x, M, n, tab);
  NH_LAUNCH_CK();
}

__global__ void k_rowdot(const double2* __restrict__ A, int lda, const double2* __restrict__ T, int ldt, int M,
                         int nk, int nrhs, double2* __restrict__ out, int ldo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (j >= M || q >= nrhs) return;
  double2 acc = make_double2(0, 0);
  const double2* Tq = T + (size_t)q * nk * ldt;
  for (int k = 0; k < nk; ++k) cfma(acc, A[(size_t)j + (size_t)k * lda], Tq[(size_t)j + (size_t)k * ldt]);
  out[(size_t)j + (size_t)q * ldo] = acc;
}

// out(j, q) -= sum_k A(j, k) T(j, k + q nk) with FP32 operands and sum, subtracted in FP64
__global__ void k_rowdot_sub32(const float2* __restrict__ A, int lda, const float2* __restrict__ T, int ldt, int M,
                               int nk, int nrhs, double2* __restrict__ out, int ldo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (j >= M || q >= nrhs) return;
  float2 acc = make_float2(0.f, 0.f);
  const float2* Tq = T + (size_t)q * nk * ldt;
  for (int k = 0; k < nk; ++k) cfma(acc, A[(size_t)j + (size_t)k * lda], Tq[(size_t)j + (size_t)k * ldt]);
  double2& o = out[(size_t)j + (size_t)q * ldo];
  o = make_double2(o.x - (double)acc.x, o.y - (double)acc.y);
}

void rowdot_sub32(cudaStream_t st, const float2* A, int lda, const float2* T, int ldt, int M, int nk, int nrhs,
                  double2* out, int ldo) {
  if (M <= 0 || nrhs <= 0) return;
  dim3 grid((M + 255) / 256, nrhs);
  k_rowdot_sub32<<<grid, 256, 0, st>>>(A, lda, T, ldt, M, nk, nrhs, out, ldo);
  NH_LAUNCH_CK();
}

// Z(j, k + q n) = (FP32) f(j, q) * conj(A(j, k))
__global__ void k_scale_rows_conj32(const float2* __restrict__ A, int lda, const double2* __restrict__ f, int ldf,
                                    int M, int n, float2* __restrict__ Z, int ldz) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (j >= M) return;
  const double2 fd = f[(size_t)j + (size_t)q * ldf];
  const float2 fj = make_float2((float)fd.x, (float)fd.y);
  float2* Zq = Z + (size_t)q * n * ldz;
  for (int k = 0; k < n; ++k) Zq[(size_t)j + (size_t)k * ldz] = fj * conj(A[(size_t)j + (size_t)k * lda]);
}

void scale_rows_conj32(cudaStream_t st, const float2* A, int lda, const double2* f, int ldf, int M, int n, int nrhs,
                       float2* Z, int ldz) {
  if (M <= 0 || nrhs <= 0) return;
  dim3 grid((M + 255) / 256, nrhs);
  k_scale_rows_conj32<<<grid, 256, 0, st>>>(A, lda, f, ldf, M, n, Z, ldz);
  NH_LAUNCH_CK();
}

void rowdot(cudaStream_t st, const double2* A, int lda, const double2* T, int ldt, int M, int nk, int nrhs,
            double2* out, int ldo) {
  if (M <= 0 || nrhs <= 0) return;
  dim3 grid((M + 255) / 256, nrhs);
  k_rowdot<<<grid, 256, 0, st>>>(A, lda, T, ldt, M, nk, nrhs, out, ldo);
  NH_LAUNCH_CK();
}

__global__ void k_scale_rows_conj(const double2* __restrict__ A, int lda, const double2* __restrict__ f, int ldf,
                                  int M, int n, double2* __restrict__ Z, int ldz) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (j >= M) return;
  const double2 fj = f[(size_t)j + (size_t)q * ldf];
  double2* Zq = Z + (size_t)q * n * ldz;
  for (int k = 0; k < n; ++k) Zq[(size_t)j + (size_t)k * ldz] = fj * conj(A[(size_t)j + (size_t)k * lda]);
}

void scale_rows_conj_multi(cudaStream_t st, const double2* A, int lda, const double2* f, int ldf, int M, int n,
                           int nrhs, double2* Z, int ldz) {
  if (M <= 0 || nrhs <= 0) return;
  dim3 grid((M + 255) / 256, nrhs);
  k_scale_rows_conj<<<grid, 256, 0, st>>>(A, lda, f, ldf, M, n, Z, ldz);
  NH_LAUNCH_CK();
}

void scale_rows_conj(cudaStream_t st, const double2* A, int lda, const double2* f, int M, int n, double2* Z,
                     int ldz) {
  scale_rows_conj_multi(st, A, lda, f, M, M, n, 1, Z, ldz);
}

template <typename R> __global__ void k_dft(int n, int sign, double scale, cplx<R>* F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  if (k >= n) return;
  const long long kl = ((long long)k * l) % n;
  double s, c;
  sincospi(2.0 * (double)kl / (double)n, &s, &c);
  F[(size_t)k + (size_t)l * n] = mkc((R)(scale * c), (R)(scale * sign * s));
}

template <typename R> void dft_matrix(cudaStream_t st, int n, int sign, double scale, cplx<R>* F) {
  dim3 grid((n + 127) / 128, n);
  k_dft<R><<<grid, 128, 0, st>>>(n, sign, scale, F);
  NH_LAUNCH_CK();
}
template void dft_matrix<double>(cudaStream_t, int, int, double, double2*);
template void dft_matrix<float>(cudaStream_t, int, int, double, float2*);

// ---------------------------------------------------------------- binning (Sec. 3.2 product tree)
__global__ void k_bin(const double* __restrict__ x, const double* __restrict__ y, int M, int nx, int ny,
                      const int* __restrict__ leafx, const int* __restrict__ leafy, const int* __restrict__ leafid,
                      int nly, int* key2d, int* keyx, int* keyy) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  int bx = (int)floor(x[j] * (double)nx);
  int by = (int)floor(y[j] * (double)ny);
  bx = min(max(bx, 0), nx - 1);
  by = min(max(by, 0), ny - 1);
  key2d[j] = leafid[leafx[bx] * nly + leafy[by]];
  keyx[j] = bx;
  keyy[j] = by;
}

void bin_points(cudaStream_t st, const double* x, const double* y, int M, int nx, int ny, const int* leafx,
                const int* leafy, const int* leafid, int nly, int* key2d, int* keyx, int* keyy) {
  k_bin<<<(M + 255) / 256, 256, 0, st>>>(x, y, M, nx, ny, leafx, leafy, leafid, nly, key2d, keyx, keyy);
  NH_LAUNCH_CK();
}

constexpr int CHUNK = 256;

__global__ void k_hist(const int* __restrict__ keys, int M, int nkeys, int* __restrict__ hist) {
  extern __shared__ int sh[];
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) sh[k] = 0;
  __syncthreads();
  const int j = blockIdx.x * CHUNK + threadIdx.x;
  if (j < M) atomicAdd(&sh[keys[j]], 1);
  __syncthreads();
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) hist[(size_t)blockIdx.x * nkeys + k] = sh[k];
}

__global__ void k_colscan(int* __restrict__ hist, int nchunk, int nkeys, int* __restrict__ total) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nkeys) return;
  int s = 0;
  for (int c = 0; c < nchunk; ++c) {
    const int v = hist[(size_t)c * nkeys + k];
    hist[(size_t)c * nkeys + k] = s;
    s += v;
  }
  total[k] = s;
}

__global__ void k_keyscan(const int* __restrict__ total, int nkeys, int* __restrict__ start) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (nkeys + 1023) / 1024;
  const int a = t * per, b = min(a + per, nkeys);
  int s = 0;
  for (int k = a; k < b; ++k) s += total[k];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < 1024; ++i) { const int v = part[i]; part[i] = run; run += v; }
  }
  __syncthreads();
  s = part[t];
  for (int k = a; k < b; ++k) { start[k] = s; s += total[k]; }
}

__global__ void k_scatter(const int* __restrict__ keys, int M, int nkeys, const int* __restrict__ hist,
                          const int* __restrict__ start, int* __restrict__ perm) {
  __shared__ int kk[CHUNK];
  const int j = blockIdx.x * CHUNK + threadIdx.x;
  kk[threadIdx.x] = j < M ? keys[j] : -1;
  __syncthreads();
  if (j >= M) return;
  const int key = kk[threadIdx.x];
  int r = 0;
  for (int t = 0; t < (int)threadIdx.x; ++t) r += (kk[t] == key);
  perm[start[key] + hist[(size_t)blockIdx.x * nkeys + key] + r] = j;
}

void counting_sort(cudaStream_t st, Arena& ar, const int* keys, int M, int nkeys, int* perm, int* counts) {
  const int nchunk = (M + CHUNK - 1) / CHUNK;
  auto mk = ar.mark();
  int* hist = ar.arr<int>((size_t)nchunk * nkeys);
  int* start = ar.arr<int>(nkeys);
  const size_t sm = (size_t)nkeys * sizeof(int);
  if (sm > 48 * 1024) NH_CK(cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_hist<<<nchunk, CHUNK, sm, st>>>(keys, M, nkeys, hist);
  NH_LAUNCH_CK();
  k_colscan<<<(nkeys + 255) / 256, 256, 0, st>>>(hist, nchunk, nkeys, counts);
  NH_LAUNCH_CK();
  k_keyscan<<<1, 1024, 0, st>>>(counts, nkeys, start);
  NH_LAUNCH_CK();
  k_scatter<<<nchunk, CHUNK, 0, st>>>(keys, M, nkeys, hist, start, perm);
  NH_LAUNCH_CK();
  ar.release(mk);
}

__global__ void k_permd(const double* __restrict__ in, const int* __restrict__ perm, int M, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) out[i] = in[perm[i]];
}
void permute_double(cudaStream_t st, const double* in, const int* perm, int M, double* out) {
  k_permd<<<(M + 255) / 256, 256, 0, st>>>(in, perm, M, out);
  NH_LAUNCH_CK();
}
__global__ void k_invp(const int* __restrict__ perm, int M, int* __restrict__ inv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) inv[perm[i]] = i;
}
void inverse_perm(cudaStream_t st, const int* perm, int M, int* inv) {
  k_invp<<<(M + 255) / 256, 256, 0, st>>>(perm, M, inv);
  NH_LAUNCH_CK();
}
__global__ void k_compose(const int* __restrict__ a, const int* __restrict__ b, int M, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) out[i] = a[b[i]];
}
void compose(cudaStream_t st, const int* a, const int* b, int M, int* out) {
  k_compose<<<(M + 255) / 256, 256, 0, st>>>(a, b, M, out);
  NH_LAUNCH_CK();
}

template <typename RS, typename RD>
__global__ void k_convert_gather(const cplx<RS>* __restrict__ src, int lds, const int* __restrict__ idx, int m, int n,
                                 cplx<RD>* __restrict__ dst, int ldd, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (i >= m || q >= n) return;
  const int si = idx ? idx[i] : i;
  const cplx<RS> v = src[(size_t)si + (size_t)q * lds];
  dst[(size_t)i + (size_t)q * ldd] = mkc((RD)(scale * (double)v.x), (RD)(scale * (double)v.y));
}
template <typename RS, typename RD>
void convert_gather(cudaStream_t st, const cplx<RS>* src, int lds, const int* idx, int m, int n, cplx<RD>* dst,
                    int ldd, double scale) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((m + 255) / 256, n);
  k_convert_gather<RS, RD><<<grid, 256, 0, st>>>(src, lds, idx, m, n, dst, ldd, scale);
  NH_LAUNCH_CK();
}
template <typename RS, typename RD>
__global__ void k_convert_scatter(const cplx<RS>* __restrict__ src, int lds, const int* __restrict__ idx, int m,
                                  int n, cplx<RD>* __restrict__ dst, int ldd, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (i >= m || q >= n) return;
  const int di = idx ? idx[i] : i;
  const cplx<RS> v = src[(size_t)i + (size_t)q * lds];
  dst[(size_t)di + (size_t)q * ldd] = mkc((RD)(scale * (double)v.x), (RD)(scale * (double)v.y));
}
template <typename RS, typename RD>
void convert_scatter(cudaStream_t st, const cplx<RS>* src, int lds, const int* idx, int m, int n, cplx<RD>* dst,
                     int ldd, double scale) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((m + 255) / 256, n);
  k_convert_scatter<RS, RD><<<grid, 256, 0, st>>>(src, lds, idx, m, n, dst, ldd, scale);
  NH_LAUNCH_CK();
}
#define NH_INST_CONV(RS, RD)                                                                              \
  template void convert_gather<RS, RD>(cudaStream_t, const cplx<RS>*, int, const int*, int, int, cplx<RD>*, \
                                       int, double);                                                     \
  template void convert_scatter<RS, RD>(cudaStream_t, const cplx<RS>*, int, const int*, int, int, cplx<RD>*, \
                                        int, double);
NH_INST_CONV(double, double)
NH_INST_CONV(double, float)
NH_INST_CONV(float, double)
NH_INST_CONV(float, float)

__global__ void k_axpy2(int m, int n, double alpha, const double2* __restrict__ x, int ldx, double2* __restrict__ y,
                        int ldy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (i >= m) return;
  double2& o = y[(size_t)i + (size_t)q * ldy];
  const double2 v = x[(size_t)i + (size_t)q * ldx];
  o.x += alpha * v.x;
  o.y += alpha * v.y;
}
void axpy2(cudaStream_t st, int m, int n, double alpha, const double2* x, int ldx, double2* y, int ldy) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((m + 255) / 256, n);
  k_axpy2<<<grid, 256, 0, st>>>(m, n, alpha, x, ldx, y, ldy);
  NH_LAUNCH_CK();
}

__global__ void k_colnorm2(int m, const double2* __restrict__ x, int ldx, double* __restrict__ out) {
  __shared__ double sh[32];
  const double2* c = x + (size_t)blockIdx.x * ldx;
  double s = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += abs2(c[i]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
  }
}
void colnorm2(cudaStream_t st, int m, int n, const double2* x, int ldx, double* out) {
  if (n <= 0) return;
  k_colnorm2<<<n, 256, 0, st>>>(m, x, ldx, out);
  NH_LAUNCH_CK();
}


// Derivative weights of the exact map: column k = kx*ny + ky of A is exp(-2 pi i (kx x + ky y)),
// so d/dx_j A(j,k) = -2 pi i kx A(j,k).  wx(k, q) = -2 pi i kx c(k, q), wy likewise with ky.
__global__ void k_deriv_weights(int nx, int ny, const double2* __restrict__ c, int ldc, double2* __restrict__ wx,
                                double2* __restrict__ wy, int ldw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (k >= nx * ny) return;
  const double2 v = c[(size_t)k + (size_t)q * ldc];
  const double tx = 6.283185307179586 * (double)(k / ny), ty = 6.283185307179586 * (double)(k % ny);
  // -i * t * (a + i b) = t * (b - i a)
  wx[(size_t)k + (size_t)q * ldw] = make_double2(tx * v.y, -tx * v.x);
  wy[(size_t)k + (size_t)q * ldw] = make_double2(ty * v.y, -ty * v.x);
}
void deriv_weights(cudaStream_t st, int nx, int ny, int s, const double2* c, int ldc, double2* wx, double2* wy,
                   int ldw) {
  if (s <= 0 || nx * ny <= 0) return;
  dim3 grid((nx * ny + 255) / 256, s);
  k_deriv_weights<<<grid, 256, 0, st>>>(nx, ny, c, ldc, wx, wy, ldw);
  NH_LAUNCH_CK();
}

// gx_j = sum_q Re[ -conj(lam_jq) Dx_jq + conj(Mx_jq) r_jq ], gy likewise: the point-coordinate
// gradient of a real loss of the least-squares solution (one thread per point).
__global__ void k_grad_combine(int M, int s, const double2* __restrict__ lam, int ldl, const double2* __restrict__ dxc,
                               const double2* __restrict__ dyc, const double2* __restrict__ dxm,
                               const double2* __restrict__ dym, const double2* __restrict__ r, int lde,
                               double* __restrict__ gx, double* __restrict__ gy) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  double ax = 0, ay = 0;
  for (int q = 0; q < s; ++q) {
    const double2 l = lam[(size_t)j + (size_t)q * ldl];
    const size_t e = (size_t)j + (size_t)q * lde;
    const double2 rr = r[e], a = dxc[e], b = dyc[e], u = dxm[e], v = dym[e];
    // Re(conj(z) w) = z.x w.x + z.y w.y
    ax += -(l.x * a.x + l.y * a.y) + (u.x * rr.x + u.y * rr.y);
    ay += -(l.x * b.x + l.y * b.y) + (v.x * rr.x + v.y * rr.y);
  }
  gx[j] = ax;
  gy[j] = ay;
}
void grad_combine(cudaStream_t st, int M, int s, const double2* lam, int ldl, const double2* dxc, const double2* dyc,
                  const double2* dxm, const double2* dym, const double2* r, int lde, double* gx, double* gy) {
  if (M <= 0) return;
  k_grad_combine<<<(M + 255) / 256, 256, 0, st>>>(M, s, lam, ldl, dxc, dyc, dxm, dym, r, lde, gx, gy);
  NH_LAUNCH_CK();
}


// y(:, q) = a[q] * x(:, q) + b[q] * y(:, q) (x may be NULL: y = b y), per-column coefficients.
__global__ void k_axpby_cols(int m, const double* __restrict__ a, const double2* __restrict__ x, int ldx,
                             const double* __restrict__ b, double2* __restrict__ y, int ldy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (i >= m) return;
  double2* yp = y + (size_t)i + (size_t)q * ldy;
  double2 v = make_double2(b[q] * yp->x, b[q] * yp->y);
  if (x) {
    const double2 xv = x[(size_t)i + (size_t)q * ldx];
    v.x += a[q] * xv.x;
    v.y += a[q] * xv.y;
  }
  *yp = v;
}
void axpby_cols(cudaStream_t st, int m, int n, const double* a, const double2* x, int ldx, const double* b, double2* y,
                int ldy) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((m + 255) / 256, n);
  k_axpby_cols<<<grid, 256, 0, st>>>(m, a, x, ldx, b, y, ldy);
  NH_LAUNCH_CK();
}

}  // namespace nh
