// Householder QR with column pivoting: kernels shared by the truncated SVD (la.cu) and the
// sketch-pivoted blocked QR (qrcp.cu).
#pragma once
#include "common.cuh"

namespace nh {

// Householder QR with column pivoting (Businger-Golub): before step k the column of largest
// remaining norm is swapped to position k.  Partial norms are downdated after every step and
// recomputed when cancellation makes the downdate unreliable (the LAPACK xLAQP2 rule).  Used to
// precondition the one-sided Jacobi SVD: on R^* of a pivoted QR the Jacobi sweeps converge
// even for strongly graded matrices.
template <typename R> struct QpD {
  cplx<R>* A; int lda, m, n;
  int* perm;       // perm[i] = original column at position i
  R* vn1; R* vn2;  // partial norms and norms at the last recomputation
  cplx<R>* v;      // reflector of the current step (m entries)
  R* tau;          // tau of the current step
};

template <typename R> __global__ void __launch_bounds__(256) k_qp_init(const QpD<R>* __restrict__ ds) {
  const QpD<R> d = ds[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + warp;
  if (j >= d.n) return;
  R s = 0;
  for (int i = lane; i < d.m; i += 32) s += abs2(d.A[(size_t)i + (size_t)j * d.lda]);
  s = warp_sum(s);
  if (lane == 0) { d.perm[j] = j; d.vn1[j] = sqrt(s); d.vn2[j] = sqrt(s); }
}

// step k, part 1: pivot, swap, reflector (one CTA per matrix)
template <typename R> __global__ void __launch_bounds__(256) k_qp_pivot(const QpD<R>* __restrict__ ds, int k) {
  const QpD<R> d = ds[blockIdx.x];
  if (k >= min(d.m, d.n)) return;
  __shared__ R bv[256];
  __shared__ int bi[256];
  __shared__ R red[32];
  __shared__ int jp_s;
  __shared__ cplx<R> v0_s;
  __shared__ R nrm_s, tau_s;
  const int tid = threadIdx.x;
  R best = -1;
  int bj = k;
  for (int j = k + tid; j < d.n; j += 256) {
    const R v = d.vn1[j];
    if (v > best) { best = v; bj = j; }
  }
  bv[tid] = best;
  bi[tid] = bj;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) {
      const R a = bv[tid], b = bv[tid + o];
      const int ia = bi[tid], ib = bi[tid + o];
      if (b > a || (b == a && ib < ia)) { bv[tid] = b; bi[tid] = ib; }
    }
    __syncthreads();
  }
  if (tid == 0) jp_s = bi[0];
  __syncthreads();
  const int jp = jp_s;
  if (jp != k) {
    cplx<R>* a = d.A + (size_t)k * d.lda;
    cplx<R>* b = d.A + (size_t)jp * d.lda;
    for (int i = tid; i < d.m; i += 256) { const cplx<R> t = a[i]; a[i] = b[i]; b[i] = t; }
    if (tid == 0) {
      const int tp = d.perm[k]; d.perm[k] = d.perm[jp]; d.perm[jp] = tp;
      R t = d.vn1[k]; d.vn1[k] = d.vn1[jp]; d.vn1[jp] = t;
      t = d.vn2[k]; d.vn2[k] = d.vn2[jp]; d.vn2[jp] = t;
    }
  }
  __syncthreads();
  cplx<R>* x = d.A + (size_t)k * d.lda;
  R s = 0;
  for (int i = k + tid; i < d.m; i += 256) s += abs2(x[i]);
  s = warp_sum(s);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    R t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    const R nrm = sqrt(t);
    const cplx<R> a0 = x[k];
    const R aa = sqrt(abs2(a0));
    const cplx<R> ph = aa > R(0) ? mkc(a0.x / aa, a0.y / aa) : mkc(R(1), R(0));
    if (nrm == R(0)) {
      v0_s = mkc(R(0), R(0));
      tau_s = R(0);                          // nothing to annihilate: H = I
    } else {
      v0_s = a0 + nrm * ph;
      tau_s = R(2) / (R(1) + (t - aa * aa) / abs2(v0_s));
    }
    nrm_s = nrm;
    *d.tau = tau_s;
    x[k] = (nrm > R(0)) ? mkc(-nrm * ph.x, -nrm * ph.y) : a0;
    d.v[k] = mkc(R(1), R(0));
  }
  __syncthreads();
  const cplx<R> v0 = v0_s;
  const R v0a2 = abs2(v0);
  for (int i = k + 1 + tid; i < d.m; i += 256) {
    const cplx<R> xv = x[i];
    d.v[i] = (v0a2 > R(0)) ? mkc((xv.x * v0.x + xv.y * v0.y) / v0a2, (xv.y * v0.x - xv.x * v0.y) / v0a2)
                           : mkc(R(0), R(0));
    x[i] = mkc(R(0), R(0));
  }
}

// step k, part 2: apply the reflector to columns k+1.. and downdate their norms (warp per column)
template <typename R> __global__ void __launch_bounds__(256) k_qp_update(const QpD<R>* __restrict__ ds, int k, R tol3z) {
  const QpD<R> d = ds[blockIdx.y];
  if (k >= min(d.m, d.n)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = k + 1 + blockIdx.x * 8 + warp;
  if (j >= d.n) return;
  const R tau = *d.tau;
  cplx<R>* y = d.A + (size_t)j * d.lda;
  if (tau != R(0)) {
    cplx<R> w = czero<R>();
    for (int i = k + lane; i < d.m; i += 32) cfmac(w, d.v[i], y[i]);
    w.x = warp_sum(w.x);
    w.y = warp_sum(w.y);
    w = tau * w;
    for (int i = k + lane; i < d.m; i += 32) y[i] = y[i] - d.v[i] * w;
  }
  __syncwarp();
  R vn1 = d.vn1[j];
  if (vn1 != R(0)) {
    const R a = sqrt(abs2(y[k])) / vn1;
    R temp = fmax(R(0), (R(1) + a) * (R(1) - a));
    const R ratio = vn1 / d.vn2[j];
    if (temp * ratio * ratio <= tol3z) {
      R s = 0;
      for (int i = k + 1 + lane; i < d.m; i += 32) s += abs2(y[i]);
      s = warp_sum(s);
      vn1 = sqrt(s);
      if (lane == 0) { d.vn1[j] = vn1; d.vn2[j] = vn1; }
    } else if (lane == 0) {
      d.vn1[j] = vn1 * sqrt(temp);
    }
  }
}

// Step k, part 2, for columns of at most 256*EPT rows: one CTA per column, the column held in
// registers, so each trailing entry is read once and written once per step (the warp-per-column
// kernel above reads it twice).  Same reflector application and norm downdate.
template <typename R> __device__ __forceinline__ cplx<R> block_csum(cplx<R> v, cplx<R>* red) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  cplx<R> t = czero<R>();
#pragma unroll
  for (int w = 0; w < 8; ++w) t = t + red[w];
  __syncthreads();
  return t;
}

template <typename R, int EPT>
__global__ void __launch_bounds__(256) k_qp_update_cta(const QpD<R>* __restrict__ ds, int k, R tol3z) {
  const QpD<R> d = ds[blockIdx.y];
  if (k >= min(d.m, d.n)) return;
  const int j = k + 1 + blockIdx.x;
  if (j >= d.n) return;
  __shared__ cplx<R> red[8];
  __shared__ cplx<R> yk_s;
  const R tau = *d.tau;
  cplx<R>* y = d.A + (size_t)j * d.lda;
  const int tid = threadIdx.x;
  cplx<R> yv[EPT];
  cplx<R> w = czero<R>();
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = k + tid + 256 * e;
    yv[e] = i < d.m ? y[i] : czero<R>();
    if (i < d.m) cfmac(w, d.v[i], yv[e]);
  }
  if (tau != R(0)) {
    w = tau * block_csum<R>(w, red);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int i = k + tid + 256 * e;
      if (i < d.m) {
        yv[e] = yv[e] - d.v[i] * w;
        y[i] = yv[e];
      }
    }
  }
  if (tid == 0) yk_s = yv[0];
  R vn1 = d.vn1[j];                      // every thread reads the norms before thread 0 updates them
  const R vn2 = d.vn2[j];
  __syncthreads();
  if (vn1 != R(0)) {
    const R a = sqrt(abs2(yk_s)) / vn1;
    const R temp = fmax(R(0), (R(1) + a) * (R(1) - a));
    const R ratio = vn1 / vn2;
    if (temp * ratio * ratio <= tol3z) {
      cplx<R> s = czero<R>();
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = k + tid + 256 * e;
        if (i > k && i < d.m) s.x += abs2(yv[e]);
      }
      vn1 = sqrt(block_csum<R>(s, red).x);
      if (tid == 0) { d.vn1[j] = vn1; d.vn2[j] = vn1; }
    } else if (tid == 0) {
      d.vn1[j] = vn1 * sqrt(temp);
    }
  }
}

}  // namespace nh
