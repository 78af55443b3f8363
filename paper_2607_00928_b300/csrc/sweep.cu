// Streaming application of stored Householder factors to a few right-hand sides: the inner step
// of the URV solve sweeps (Sec. 2.3: Omega^*, P^* on the way up; the root QR; Q_v on the way
// down) and of their adjoint.  For a block of b <= 256 reflectors V_b with compact-WY factor T,
//   Q^* C = C - V_b (T^* (V_b^* C)),   Q C = C - V_b (T (V_b^* C)),
// so each block is two streaming passes over V_b (one reduction over its rows, one update of C's
// rows) around a tiny b x b product.  With s right-hand sides the passes do 4 s real FMAs per
// complex entry of V (64 per 8 bytes at s = 16): no matrix unit is needed, and generic GEMM tiles
// would leave most of a 64 x 64 output tile empty while the long row reduction of V_b^* C ran on a
// handful of CTAs.  (Measured on a 65536-row block: 1.4-1.6 TB/s, issue and latency bound at one or
// two CTAs per SM rather than bandwidth bound.)  Four kernels per block step:
//   1. k_wy_part:   partial V_b^* C over one slab of rows per CTA; thread t owns reflector column
//                   t; V and C tiles are double-buffered in shared memory with cp.async.  A node
//                   with a single slab writes W1 = V_b^* C directly;
//   2. k_wy_reduce: W1 = the sum of a node's partials in a fixed order (deterministic), four
//                   lanes per element;
//   3. k_wy_tmul:   W2 = T^* W1 (Q^* C) or T W1 (Q C); a few CTAs per node, one slice of rows each;
//   4. k_wy_update: C -= V_b W2; two threads per row (one per half of the reflectors), W2 in
//                   shared memory.
// Blocks are applied in increasing order for Q^* C and in decreasing order for Q C.  Every node of
// a level (and every chunk of S columns of its right-hand sides) shares the same four launches
// per block step.  Rows above a block's first reflector are untouched (the vectors are zero
// there) and are skipped.
#include <algorithm>
#include <cstring>

#include "la.cuh"

namespace nh {

namespace {
constexpr int WY_T = 256;       // threads per CTA = widest reflector block
constexpr int WY_MID = 8;       // CTAs per node in k_wy_tmul
constexpr int WY_TARGET = 4 * 148;   // aim for about four CTAs per SM in k_wy_part
}  // namespace

// rows per shared-memory tile of k_wy_part (keeps two buffers of 256 columns near 70 KB)
template <typename R> struct WyTile { static constexpr int TR = 16; };
template <> struct WyTile<double> { static constexpr int TR = 8; };

template <typename R> struct WyD {
  const cplx<R>* V;   // reflectors of this block, from its first row (row j0 of the factor)
  const cplx<R>* T;   // the block's compact-WY T (b x b, upper triangular, leading dimension ldt)
  cplx<R>* C;         // right-hand-side rows j0.. of this chunk of columns
  int ldv, ldt, ldc;
  int m, b, s;        // rows from j0, reflectors in the block, columns in this chunk (<= S)
  int rows;           // rows per slab in k_wy_part (a multiple of the tile height)
  int nparts;         // slabs
  int pre_p, pre_u, pre_r;   // first CTA of this descriptor in k_wy_part / k_wy_update / k_wy_reduce
  int part0;          // first partial slot (nparts > 1)
};

// descriptor owning CTA t of a launch, from the exclusive CTA prefix field F (0: part, 1: update,
// 2: reduce); descriptors with no CTAs in that launch repeat the next prefix and are skipped
template <typename R, int F> __device__ __forceinline__ int wy_pre(const WyD<R>& d) {
  return F == 0 ? d.pre_p : (F == 1 ? d.pre_u : d.pre_r);
}
template <typename R, int F>
__device__ __forceinline__ int wy_find(const WyD<R>* ds, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (wy_pre<R, F>(ds[mid]) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void wy_cp(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void wy_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void wy_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename R, int S>
__global__ void __launch_bounds__(WY_T) k_wy_part(const WyD<R>* __restrict__ ds, int nd, cplx<R>* __restrict__ part,
                                                 cplx<R>* __restrict__ w1) {
  constexpr int TR = WyTile<R>::TR, VS = TR + 1;
  const int di = wy_find<R, 0>(ds, nd, blockIdx.x);
  const WyD<R> d = ds[di];
  const int slab = blockIdx.x - d.pre_p;
  const int r0 = slab * d.rows, r1 = min(d.m, r0 + d.rows);
  const int t = threadIdx.x;
  extern __shared__ __align__(16) unsigned char wy_raw[];
  cplx<R>* Vs = reinterpret_cast<cplx<R>*>(wy_raw);          // [2][WY_T][VS]
  cplx<R>* Cs = Vs + 2 * WY_T * VS;                           // [2][TR][S]
  // columns q >= s are never copied: zero them once so the unused accumulators stay finite
  for (int e = t; e < 2 * TR * S; e += WY_T) Cs[e] = czero<R>();
  __syncthreads();
  auto issue = [&](int rb, int buf) {
    const int nr = min(TR, r1 - rb);
    cplx<R>* vb = Vs + buf * WY_T * VS;
    for (int e = t; e < TR * WY_T; e += WY_T) {       // consecutive threads -> consecutive rows
      const int row = e % TR, col = e / TR;
      if (row < nr && col < d.b) wy_cp(vb + col * VS + row, d.V + (size_t)(rb + row) + (size_t)col * d.ldv, sizeof(cplx<R>));
    }
    cplx<R>* cb = Cs + buf * TR * S;
    for (int e = t; e < TR * S; e += WY_T) {
      const int row = e % TR, q = e / TR;
      if (row < nr && q < d.s) wy_cp(cb + row * S + q, d.C + (size_t)(rb + row) + (size_t)q * d.ldc, sizeof(cplx<R>));
    }
    wy_commit();
  };
  cplx<R> acc[S];
#pragma unroll
  for (int q = 0; q < S; ++q) acc[q] = czero<R>();
  const int ntile = (r1 - r0 + TR - 1) / TR;
  if (ntile > 0) issue(r0, 0);
  for (int it = 0; it < ntile; ++it) {
    const int rb = r0 + it * TR, nr = min(TR, r1 - rb), buf = it & 1;
    if (it + 1 < ntile) { issue(rb + TR, buf ^ 1); wy_wait<1>(); } else { wy_wait<0>(); }
    __syncthreads();
    if (t < d.b) {
      const cplx<R>* vb = Vs + buf * WY_T * VS + t * VS;
      const cplx<R>* cb = Cs + buf * TR * S;
      for (int r = 0; r < nr; ++r) {
        const cplx<R> x = vb[r];
#pragma unroll
        for (int q = 0; q < S; ++q) cfmac(acc[q], x, cb[r * S + q]);
      }
    }
    __syncthreads();
  }
  cplx<R>* out = (d.nparts == 1) ? w1 + (size_t)di * WY_T * S : part + ((size_t)d.part0 + slab) * WY_T * S;
  if (t < d.b) {
#pragma unroll
    for (int q = 0; q < S; ++q) out[t * S + q] = acc[q];
  }
}

// W1 = sum of the node's partials, 64 elements of W1 per CTA: four lanes per element each sum the
// slabs p = lane (mod 4) (several loads in flight), then the four lane sums are added in a fixed
// order -- deterministic
template <typename R, int S>
__global__ void __launch_bounds__(WY_T) k_wy_reduce(const WyD<R>* __restrict__ ds, int nd,
                                                   const cplx<R>* __restrict__ part, cplx<R>* __restrict__ w1) {
  const int di = wy_find<R, 2>(ds, nd, blockIdx.x);
  const WyD<R> d = ds[di];
  const int el = threadIdx.x & 63, pl = threadIdx.x >> 6;
  const int e = (blockIdx.x - d.pre_r) * 64 + el;
  __shared__ cplx<R> acc4[4][64];
  cplx<R> sum = czero<R>();
  if (e < d.b * S) {
    const cplx<R>* pp = part + (size_t)d.part0 * WY_T * S + e;
    int p = pl;
    for (; p + 12 < d.nparts; p += 16) {
      const cplx<R> a0 = pp[(size_t)p * WY_T * S], a1 = pp[(size_t)(p + 4) * WY_T * S];
      const cplx<R> a2 = pp[(size_t)(p + 8) * WY_T * S], a3 = pp[(size_t)(p + 12) * WY_T * S];
      sum = sum + a0;
      sum = sum + a1;
      sum = sum + a2;
      sum = sum + a3;
    }
    for (; p < d.nparts; p += 4) sum = sum + pp[(size_t)p * WY_T * S];
  }
  acc4[pl][el] = sum;
  __syncthreads();
  if (pl == 0 && e < d.b * S) w1[(size_t)di * WY_T * S + e] = ((acc4[0][el] + acc4[1][el]) + acc4[2][el]) + acc4[3][el];
}

// W2 rows of slice blockIdx.x % WY_MID of node blockIdx.x / WY_MID: op(T) W1, op = ^* (conj) or none
template <typename R, int S>
__global__ void __launch_bounds__(WY_T) k_wy_tmul(const WyD<R>* __restrict__ ds, const cplx<R>* __restrict__ w1,
                                                 cplx<R>* __restrict__ w2, int conj) {
  const int di = blockIdx.x / WY_MID;
  const WyD<R> d = ds[di];
  const int per = (d.b + WY_MID - 1) / WY_MID, i0 = (blockIdx.x % WY_MID) * per, i1 = min(d.b, i0 + per);
  extern __shared__ __align__(16) unsigned char wy_raw[];
  cplx<R>* W1 = reinterpret_cast<cplx<R>*>(wy_raw);   // b x S
  const cplx<R>* src = w1 + (size_t)di * WY_T * S;
  for (int e = threadIdx.x; e < d.b * S; e += WY_T) W1[e] = src[e];
  __syncthreads();
  cplx<R>* out = w2 + (size_t)di * WY_T * S;
  for (int e = threadIdx.x; e < (i1 - i0) * S; e += WY_T) {
    const int i = i0 + e / S, q = e % S;
    cplx<R> acc = czero<R>();
    if (conj) {   // (T^* W1)(i) = sum_{j <= i} conj(T(j, i)) W1(j)
      const cplx<R>* tc = d.T + (size_t)i * d.ldt;
      for (int j = 0; j <= i; ++j) cfmac(acc, tc[j], W1[j * S + q]);
    } else {      // (T W1)(i) = sum_{j >= i} T(i, j) W1(j)
      for (int j = i; j < d.b; ++j) cfma(acc, d.T[(size_t)i + (size_t)j * d.ldt], W1[j * S + q]);
    }
    out[i * S + q] = acc;
  }
}

// C(r, :) -= V(r, :) W2 for 128 rows per CTA: thread t takes row t % 128 and half t / 128 of the
// reflector columns (eight loads in flight); the halves are added through shared memory.
template <typename R, int S>
__global__ void __launch_bounds__(WY_T) k_wy_update(const WyD<R>* __restrict__ ds, int nd,
                                                   const cplx<R>* __restrict__ w2) {
  const int di = wy_find<R, 1>(ds, nd, blockIdx.x);
  const WyD<R> d = ds[di];
  const int rl = threadIdx.x & 127, half = threadIdx.x >> 7;
  const int r = (blockIdx.x - d.pre_u) * 128 + rl;
  extern __shared__ __align__(16) unsigned char wy_raw[];
  cplx<R>* W2 = reinterpret_cast<cplx<R>*>(wy_raw);   // b x S
  cplx<R>* Hs = W2 + WY_T * S;                       // 128 x S: the second half's sums
  const cplx<R>* src = w2 + (size_t)di * WY_T * S;
  for (int e = threadIdx.x; e < d.b * S; e += WY_T) W2[e] = src[e];
  __syncthreads();
  cplx<R> acc[S];
#pragma unroll
  for (int q = 0; q < S; ++q) acc[q] = czero<R>();
  const int hb = (d.b + 1) / 2, i0 = half * hb, i1 = min(d.b, i0 + hb);
  if (r < d.m) {
    const cplx<R>* v = d.V + r;
    int i = i0;
    for (; i + 8 <= i1; i += 8) {
      cplx<R> x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = v[(size_t)(i + u) * d.ldv];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int q = 0; q < S; ++q) cfma(acc[q], x[u], W2[(i + u) * S + q]);
    }
    for (; i < i1; ++i) {
      const cplx<R> x = v[(size_t)i * d.ldv];
#pragma unroll
      for (int q = 0; q < S; ++q) cfma(acc[q], x, W2[i * S + q]);
    }
  }
  if (half == 1) {
#pragma unroll
    for (int q = 0; q < S; ++q) Hs[rl * S + q] = acc[q];
  }
  __syncthreads();
  if (half == 0 && r < d.m) {
#pragma unroll
    for (int q = 0; q < S; ++q)
      if (q < d.s) {
        cplx<R>& c = d.C[(size_t)r + (size_t)q * d.ldc];
        c = c - (acc[q] + Hs[rl * S + q]);
      }
  }
}

template <typename R>
template <int S>
void Ops<R>::apply_q_stream_s(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj) {
  constexpr int TR = WyTile<R>::TR;
  auto bw = [](const QFac<R>& q) { return q.Tg ? GW : NB; };
  static_assert(GW <= WY_T && NB <= WY_T, "one reflector column per thread");
  // (factor, column chunk) pairs
  struct Job { int i, c0, s; };
  std::vector<Job> jobs;
  int pmax = 0;
  for (size_t i = 0; i < Q.size(); ++i) {
    if (Q[i].k <= 0 || C[i].n <= 0) continue;
    NH_REQUIRE(C[i].m >= Q[i].m, ST_EINVAL, "apply_q_stream: C has fewer rows than Q");
    for (int c0 = 0; c0 < C[i].n; c0 += S) jobs.push_back({(int)i, c0, std::min(S, C[i].n - c0)});
    pmax = std::max(pmax, (Q[i].k + bw(Q[i]) - 1) / bw(Q[i]));
  }
  if (jobs.empty()) return;
  // plan every step first: descriptors and the largest partial-slot count
  std::vector<std::vector<WyD<R>>> steps(pmax);
  std::vector<int> np(pmax), nu(pmax), nr(pmax);
  size_t maxslots = 1;
  for (int st = 0; st < pmax; ++st) {
    long total = 0;
    for (const Job& jb : jobs) {
      const QFac<R>& q = Q[jb.i];
      const int nb = (q.k + bw(q) - 1) / bw(q);
      if (st < nb) total += q.m - (conj ? st : nb - 1 - st) * bw(q);
    }
    const int rows_all = (int)std::max<long>(8L * TR, ((total + WY_TARGET - 1) / WY_TARGET + TR - 1) / TR * TR);
    int slot = 0, p_cta = 0, u_cta = 0, r_cta = 0;
    for (const Job& jb : jobs) {
      const QFac<R>& q = Q[jb.i];
      const int B = bw(q), nb = (q.k + B - 1) / B;
      if (st >= nb) continue;
      const int p = conj ? st : (nb - 1 - st);
      const int j0 = p * B, mm = q.m - j0;
      WyD<R> w;
      w.V = q.V + (size_t)j0 + (size_t)j0 * q.ldv;
      w.T = (q.Tg ? q.Tg : q.Tp) + (size_t)p * B * B;
      w.C = C[jb.i].p + j0 + (size_t)jb.c0 * C[jb.i].ld;
      w.ldv = q.ldv; w.ldt = B; w.ldc = C[jb.i].ld;
      w.m = mm; w.b = std::min(B, q.k - j0); w.s = jb.s;
      // at most 256 slabs per node keeps the partial sums small next to V
      w.rows = std::max(rows_all, ((mm + 255) / 256 + TR - 1) / TR * TR);
      w.nparts = (mm + w.rows - 1) / w.rows;
      w.pre_p = p_cta; w.pre_u = u_cta; w.pre_r = r_cta; w.part0 = slot;
      p_cta += w.nparts;
      u_cta += (mm + 127) / 128;
      if (w.nparts > 1) {
        slot += w.nparts;
        r_cta += (w.b * S + 63) / 64;
      }
      steps[st].push_back(w);
    }
    np[st] = p_cta; nu[st] = u_cta; nr[st] = r_cta;
    maxslots = std::max(maxslots, (size_t)slot);
  }
  auto mk = ar_->mark();
  const size_t per = (size_t)WY_T * S * sizeof(cplx<R>);
  cplx<R>* part = (cplx<R>*)ar_->alloc(maxslots * per);
  cplx<R>* w1 = (cplx<R>*)ar_->alloc(jobs.size() * per);
  cplx<R>* w2 = (cplx<R>*)ar_->alloc(jobs.size() * per);
  const size_t smem_p = (2 * (size_t)WY_T * (TR + 1) + 2 * (size_t)TR * S) * sizeof(cplx<R>);
  const size_t smem_u = per + (size_t)128 * S * sizeof(cplx<R>);
  static const bool attr = [&] {   // once per template instance (thread-safe static initialisation)
    NH_CK(cudaFuncSetAttribute(k_wy_part<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
    NH_CK(cudaFuncSetAttribute(k_wy_tmul<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_u));
    NH_CK(cudaFuncSetAttribute(k_wy_update<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_u));
    return true;
  }();
  (void)attr;
  for (int st = 0; st < pmax; ++st) {
    const std::vector<WyD<R>>& d = steps[st];
    if (d.empty()) continue;
    const WyD<R>* dd = (const WyD<R>*)stage(d.data(), d.size() * sizeof(WyD<R>));
    const int nd = (int)d.size();
    k_wy_part<R, S><<<np[st], WY_T, smem_p, st_>>>(dd, nd, part, w1);
    NH_LAUNCH_CK();
    if (nr[st] > 0) {
      k_wy_reduce<R, S><<<nr[st], WY_T, 0, st_>>>(dd, nd, part, w1);
      NH_LAUNCH_CK();
      count();
    }
    k_wy_tmul<R, S><<<nd * WY_MID, WY_T, smem_u, st_>>>(dd, w1, w2, conj ? 1 : 0);
    NH_LAUNCH_CK();
    k_wy_update<R, S><<<nu[st], WY_T, smem_u, st_>>>(dd, nd, w2);
    NH_LAUNCH_CK();
    count(3);
  }
  ar_->release(mk);
}

template <typename R>
void Ops<R>::apply_q_stream(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj) {
  int smax = 0;
  for (size_t i = 0; i < Q.size(); ++i)
    if (Q[i].k > 0) smax = std::max(smax, C[i].n);
  if (smax <= 1) apply_q_stream_s<1>(Q, C, conj);
  else if (smax <= 4) apply_q_stream_s<4>(Q, C, conj);
  else if (smax <= 8) apply_q_stream_s<8>(Q, C, conj);
  else apply_q_stream_s<16>(Q, C, conj);
}

template <typename R>
void Ops<R>::apply_q_sweep(const std::vector<QFac<R>>& Q, const std::vector<Mat<R>>& C, bool conj) {
  const char* e = getenv("NH_SWEEP_STREAM");   // "0": the generic blocked GEMM path
  if (!e || atoi(e) != 0) apply_q_stream(Q, C, conj);
  else apply_q_left(Q, C, conj);
}

template void Ops<double>::apply_q_stream(const std::vector<QFac<double>>&, const std::vector<Mat<double>>&, bool);
template void Ops<float>::apply_q_stream(const std::vector<QFac<float>>&, const std::vector<Mat<float>>&, bool);
template void Ops<double>::apply_q_sweep(const std::vector<QFac<double>>&, const std::vector<Mat<double>>&, bool);
template void Ops<float>::apply_q_sweep(const std::vector<QFac<float>>&, const std::vector<Mat<float>>&, bool);

}  // namespace nh
