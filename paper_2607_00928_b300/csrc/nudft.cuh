// NUDFT-specific kernels: kernel-entry evaluation of the transformed 1D matrices, twiddle
// tables for the exact apply, point binning (stable counting sort) and DFT matrices.
#pragma once
#include "la.cuh"

namespace nh {

// Psi(gamma, xi) = (1/n) sum_l (gamma/xi)^l = exp(-i pi (n-1) t) sin(pi n t) / (n sin(pi t)),
// t = x - k/n reduced to [-1/2, 1/2); Psi = 1 at t = 0 (the entries of the transformed 1D matrix).
__device__ __forceinline__ double2 psi_entry(double x, int k, int n) {
  double t = x - (double)k / (double)n;
  t -= floor(t + 0.5);
  if (t == 0.0) return make_double2(1.0, 0.0);
  double sn, cn, s1, c1, sp, cp;
  sincospi((double)n * t, &sn, &cn);
  sincospi(t, &s1, &c1);
  sincospi((double)(n - 1) * t, &sp, &cp);
  const double r = sn / ((double)n * s1);
  return make_double2(r * cp, -r * sp);
}

// out(i, k) = Psi(x[i], k0 + k; n), i < m, k < nk.
template <typename R> struct PsiD {
  const double* x; int m; int k0, nk, n; cplx<R>* out; int ld;
};
template <typename R> void psi_eval(Ops<R>& ops, const std::vector<PsiD<R>>& d);

// tab(j, k) = exp(-2 pi i k x_j), j < M, k < n (FP64)
void twiddle_table(cudaStream_t st, const double* x, int M, int n, double2* tab);
// out_j(q) = sum_k A(j, k) T(j, k) for every column q of T (T has M rows, nk cols per column block)
void rowdot(cudaStream_t st, const double2* A, int lda, const double2* T, int ldt, int M, int nk, int nrhs,
            double2* out, int ldo);
// out(j, q) -= sum_k A(j, k) T(j, k + q nk): FP32 operands and sum, subtracted from the FP64 out
void rowdot_sub32(cudaStream_t st, const float2* A, int lda, const float2* T, int ldt, int M, int nk, int nrhs,
                  double2* out, int ldo);
// Z(j, k + q n) = (FP32) f(j, q) * conj(A(j, k)) for k < n, q < nrhs
void scale_rows_conj32(cudaStream_t st, const float2* A, int lda, const double2* f, int ldf, int M, int n, int nrhs,
                       float2* Z, int ldz);
// Z(j, k) = f_j * conj(A(j, k)) for k < n
void scale_rows_conj(cudaStream_t st, const double2* A, int lda, const double2* f, int M, int n, double2* Z,
                     int ldz);
void scale_rows_conj_multi(cudaStream_t st, const double2* A, int lda, const double2* f, int ldf, int M, int n,
                           int nrhs, double2* Z, int ldz);
// F(k, l) = exp(sign * 2 pi i k l / n) * scale, n x n
template <typename R> void dft_matrix(cudaStream_t st, int n, int sign, double scale, cplx<R>* F);

// Stable counting sort of keys[0..M) in [0, nkeys): perm[pos] = j, counts[key] (device).
void counting_sort(cudaStream_t st, Arena& ar, const int* keys, int M, int nkeys, int* perm, int* counts);
// keys: key2d (product-tree leaf: leafid[lx * nly + ly] for the 1D leaves lx, ly of the point's
// bins), keyx (x bin), keyy (y bin)
void bin_points(cudaStream_t st, const double* x, const double* y, int M, int nx, int ny, const int* leafx,
                const int* leafy, const int* leafid, int nly, int* key2d, int* keyx, int* keyy);
// out[i] = in[perm[i]] (double), out_pos[i] = inv[perm[i]]
void permute_double(cudaStream_t st, const double* in, const int* perm, int M, double* out);
void inverse_perm(cudaStream_t st, const int* perm, int M, int* inv);
void compose(cudaStream_t st, const int* a, const int* b, int M, int* out);   // out[i] = a[b[i]]
// complex precision conversion with row gather: dst(i, q) = (R) src(idx ? idx[i] : i, q) * scale
template <typename RS, typename RD>
void convert_gather(cudaStream_t st, const cplx<RS>* src, int lds, const int* idx, int m, int n, cplx<RD>* dst,
                    int ldd, double scale);
// dst(idx[i], q) = src(i, q) (scatter), with precision conversion and scale
template <typename RS, typename RD>
void convert_scatter(cudaStream_t st, const cplx<RS>* src, int lds, const int* idx, int m, int n, cplx<RD>* dst,
                     int ldd, double scale);
// y(:, q) += alpha * x(:, q) in double
void axpy2(cudaStream_t st, int m, int n, double alpha, const double2* x, int ldx, double2* y, int ldy);
// per-column sums of |x|^2 (double), out[q]
void colnorm2(cudaStream_t st, int m, int n, const double2* x, int ldx, double* out);
// y(:, q) = a[q] x(:, q) + b[q] y(:, q) with device coefficient arrays a, b (x may be NULL)
void axpby_cols(cudaStream_t st, int m, int n, const double* a, const double2* x, int ldx, const double* b, double2* y,
                int ldy);
// wx(k, q) = -2 pi i kx c(k, q), wy(k, q) = -2 pi i ky c(k, q), k = kx * ny + ky
void deriv_weights(cudaStream_t st, int nx, int ny, int s, const double2* c, int ldc, double2* wx, double2* wy,
                   int ldw);
// gx_j = sum_q Re[-conj(lam) dxc + conj(dxm) r], gy_j likewise (all M x s, ld lde except lam)
void grad_combine(cudaStream_t st, int M, int s, const double2* lam, int ldl, const double2* dxc, const double2* dyc,
                  const double2* dxm, const double2* dym, const double2* r, int lde, double* gx, double* gy);

}  // namespace nh
