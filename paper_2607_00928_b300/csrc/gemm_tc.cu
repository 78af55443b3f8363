// Complex FP32 GEMM on the 5th-generation tensor cores (tcgen05.mma, kind::tf32) with the
// 3xTF32 split, for the FP32 generator products of the mixed-precision path (Sec. 2.2-2.3:
// F B G^*, P^* B Q, U2 B V2^*, the URV trailing updates).
//
// Every FP32 operand x is split as x = hi + lo, hi = tf32(x), lo = tf32(x - hi) (both rounded to
// nearest; x - hi is exact in FP32); each real product X Y is formed as
// Xhi Yhi + Xhi Ylo + Xlo Yhi, which keeps FP32-level accuracy.  A complex product needs four
// real ones:  Cr += Ar Br - Ai Bi,  Ci += Ar Bi + Ai Br,  so one k = 8 step of a tile is 12 MMAs
// (the -Ai Bi ones through the A-negate bit of the instruction descriptor).
//
// The tensor core's FP32 accumulation truncates, so an error that grows linearly with k builds
// up in a long accumulation (measured: about 1.5e-8 k relative).  The k range is therefore cut
// into chunks of 64: the MMAs of one chunk accumulate in a chunk accumulator in tensor memory,
// which the epilogue warps then add (FP32, round to nearest) into a running total kept in a
// second tensor-memory region.  The error is then that of a 64-term tensor-core sum, about 1e-6
// relative for any k, below the CUDA-core FP32 kernel's.
//
// Two passes:
//  1. pack: op(A) (m x k) and op(B)^T (n x k) are split into four planes (re hi, re lo, im hi,
//     im lo) and written tile by tile, zero padded, in exactly the shared-memory image the MMA
//     reads: the canonical K-major layout without swizzle (8-row x 16-byte core matrices).  One
//     packed block covers 128 rows x 8 k: 4 planes of 128 x 8 x 4 bytes.  The blocks of one row
//     tile are contiguous along k.  Packing removes every alignment and ragged-edge case from the
//     main kernel and does the conjugation.
//  2. gemm: one CTA of six warps per 128 x 128 output tile.  Warp 4 (one lane) streams packed A
//     and B blocks into a ring of shared-memory stages with cp.async.bulk (TMA bulk copies,
//     completion counted on the stage's "full" mbarrier); warp 5 (one lane) waits for a full
//     stage, issues its 12 MMAs and commits them to the stage's "empty" mbarrier, which releases
//     the stage to the producer, and to the chunk barrier at the end of a chunk.  Warps 0-3 drain
//     each chunk into the total (tcgen05.ld / tcgen05.st) and release the chunk accumulator to
//     the MMA warp; after the last chunk they apply alpha, beta and write C.  Every wait is
//     bounded: a wait that runs out sets g_tc_error and the CTA stops issuing, waits (bounded)
//     for its copies and MMAs in flight, frees its tensor memory and returns without writing C.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "la.cuh"
#include "tc.cuh"

namespace nh {

namespace {
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 8;
constexpr int TC_KC = 8;                                   // k blocks (of 8) per accumulation chunk
constexpr int TC_STAGES = 6;
constexpr int TC_BLK = 4 * 128 * TC_BK * 4;                // 16 KB: one packed 128-row block
constexpr int TC_STAGE = 2 * TC_BLK;                       // A block + B block
constexpr int TC_SMEM = TC_STAGES * TC_STAGE + 1024;       // + alignment slack
constexpr int TC_THREADS = 192;                            // warps 0-3 drain / epilogue, 4 producer, 5 MMA
constexpr uint32_t TC_TMEM_COLS = 512;                     // chunk Cr, Ci; total Cr, Ci (128 each)
}  // namespace

__device__ int g_tc_error;

// ------------------------------------------------------------------------------------- packing
// P(r, k) = op(X) element: kcontig ? X[k + r*ld] : X[r + k*ld], conjugated when conj.
struct PackD {
  const float2* X;
  unsigned char* out;   // tiles_r * ktiles blocks of 4 * 128 * 8 * 4 bytes
  int rows, k, ld;
  int kcontig, conj;
  int tiles_r, ktiles;
};


// One CTA of 256 threads per packed block; thread (kq, r) writes row r, k quad kq of each plane
// as one 16-byte store.
__global__ void __launch_bounds__(256) k_tc_pack(const PackD* __restrict__ ds, const int* __restrict__ pre, int np) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const PackD d = ds[lo];
  const int b = blockIdx.x - pre[lo];
  const int tr = b / d.ktiles, tk = b - tr * d.ktiles;
  constexpr int R = 128;
  const int r = threadIdx.x % R, kq = threadIdx.x / R;
  const int gr = tr * R + r;
  const int gk0 = tk * TC_BK + kq * 4;
  uint32_t p[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int gk = gk0 + e;
    float2 v = make_float2(0.f, 0.f);
    if (gr < d.rows && gk < d.k)
      v = d.kcontig ? d.X[(size_t)gk + (size_t)gr * d.ld] : d.X[(size_t)gr + (size_t)gk * d.ld];
    if (d.conj) v.y = -v.y;
    tc_split(v.x, p[0][e], p[1][e]);
    tc_split(v.y, p[2][e], p[3][e]);
  }
  unsigned char* blk = d.out + (size_t)b * (4 * R * TC_BK * 4);
  const uint32_t off = tc_kmajor(r, kq * 4, 256);   // one packed block: 8 k, so 8-row groups are 256 B apart
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<uint4*>(blk + q * (R * TC_BK * 4) + off) = make_uint4(p[q][0], p[q][1], p[q][2], p[q][3]);
}

// ------------------------------------------------------------------------------------- gemm
struct TcProb {
  const unsigned char* Ap;   // tiles_m * ktiles packed A blocks
  const unsigned char* Bp;   // tiles_n * ktiles packed B blocks (128 rows = output columns each)
  float2* C;
  int m, n, ldc, ktiles, tiles_m;
  float alpha, beta;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const TcProb* __restrict__ ds, const int* __restrict__ pre, int np) {
  constexpr int S = TC_STAGES;
  extern __shared__ unsigned char tc_raw[];
  __shared__ uint64_t full[S], empty[S], chunk_full, chunk_free, mma_done;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const uint32_t raw_s = tc_smem_u32(tc_raw);
  unsigned char* sm = tc_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const TcProb g = ds[lo];
  const int lt = blockIdx.x - pre[lo];
  const int tm = lt % g.tiles_m, tn = lt / g.tiles_m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(&tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&chunk_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(tc_smem_u32(&chunk_free)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&mma_done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  const int KT = g.ktiles;
  const int NCH = (KT + TC_KC - 1) / TC_KC;
  volatile int* abort_v = &abort_flag;

  if (warp == 4) {
    if (lane == 0) {
      // producer: packed A block (tm, kt) and B block (tn, kt) into stage kt % S
      const unsigned char* a0 = g.Ap + (size_t)tm * KT * TC_BLK;
      const unsigned char* b0 = g.Bp + (size_t)tn * KT * TC_BLK;
      int issued = 0;
      for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % S;
        if (kt >= S && !tc_wait(&empty[s], (uint32_t)(((kt / S) - 1) & 1))) { *abort_v = 1; break; }
        if (*abort_v) break;
        unsigned char* st = sm + s * TC_STAGE;
        tc_expect(&full[s], (uint32_t)TC_STAGE);
        tc_bulk(st, a0 + (size_t)kt * TC_BLK, TC_BLK, &full[s]);
        tc_bulk(st + TC_BLK, b0 + (size_t)kt * TC_BLK, TC_BLK, &full[s]);
        issued = kt + 1;
      }
      // every copy issued must have landed before the CTA can exit: wait for the last fill of
      // each stage (a no-op when the MMA warp already consumed it)
      for (int kt = (issued > S ? issued - S : 0); kt < issued; ++kt)
        if (!tc_wait(&full[kt % S], (uint32_t)((kt / S) & 1))) *abort_v = 1;
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // MMA issuer: chunk accumulator in columns [0, 256) (Cr, Ci)
      const uint32_t idp = tc_idesc(TC_BM, TC_BN, false), idn = tc_idesc(TC_BM, TC_BN, true);
      const uint32_t cr = tmem, ci = tmem + TC_BN;
      constexpr uint32_t PL = 128 * TC_BK * 4;   // plane bytes
      for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % S, c = kt / TC_KC, kc = kt - c * TC_KC;
        if (kc == 0 && c > 0 && !tc_wait(&chunk_free, (uint32_t)((c - 1) & 1))) { *abort_v = 1; break; }
        if (!tc_wait(&full[s], (uint32_t)((kt / S) & 1))) { *abort_v = 1; break; }
        if (*abort_v) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a = tc_smem_u32(sm + s * TC_STAGE), b = a + TC_BLK;
        const uint64_t arh = tc_desc(a, 256), arl = tc_desc(a + PL, 256), aih = tc_desc(a + 2 * PL, 256),
                       ail = tc_desc(a + 3 * PL, 256);
        const uint64_t brh = tc_desc(b, 256), brl = tc_desc(b + PL, 256), bih = tc_desc(b + 2 * PL, 256),
                       bil = tc_desc(b + 3 * PL, 256);
        const uint32_t f = kc == 0 ? 0u : 1u;
        tc_mma(cr, arh, brh, idp, f);
        tc_mma(cr, arh, brl, idp, 1u);
        tc_mma(cr, arl, brh, idp, 1u);
        tc_mma(cr, aih, bih, idn, 1u);
        tc_mma(cr, aih, bil, idn, 1u);
        tc_mma(cr, ail, bih, idn, 1u);
        tc_mma(ci, arh, bih, idp, f);
        tc_mma(ci, arh, bil, idp, 1u);
        tc_mma(ci, arl, bih, idp, 1u);
        tc_mma(ci, aih, brh, idp, 1u);
        tc_mma(ci, aih, brl, idp, 1u);
        tc_mma(ci, ail, brh, idp, 1u);
        tc_commit(&empty[s]);                                   // the stage is free once these MMAs read it
        if (kc == TC_KC - 1 || kt == KT - 1) tc_commit(&chunk_full);   // the chunk is complete
      }
      tc_commit(&mma_done);                                     // every MMA issued above is complete
    }
  } else {
    // warps 0-3: lane t of warp w owns row 32 w + t of the tile (tensor-memory lane 32 w + t)
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t tot = lane_addr + 2 * TC_BN;                 // running total: columns [256, 512)
    for (int c = 0; c + 1 < NCH; ++c) {
      bool ok = tc_wait(&chunk_full, (uint32_t)(c & 1));
      if (!ok || *abort_v) { *abort_v = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int c0 = 0; c0 < 2 * TC_BN; c0 += 16) {
        uint32_t v[16], t[16];
        tc_ld16(lane_addr + (uint32_t)c0, v);
        if (c > 0) tc_ld16(tot + (uint32_t)c0, t);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c > 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(t[j]));
        }
        tc_st16(tot + (uint32_t)c0, v);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      tc_arrive(&chunk_free);
    }
    // last chunk (or none): total + chunk, alpha, beta, store C
    bool ok = true;
    if (NCH > 0) ok = tc_wait(&chunk_full, (uint32_t)((NCH - 1) & 1));
    if (!ok) *abort_v = 1;
    ok = ok && !*abort_v;
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int r = tm * TC_BM + warp * 32 + lane;
      const int col0 = tn * TC_BN;
      for (int c0 = 0; c0 < TC_BN; c0 += 16) {
        if (col0 + c0 >= g.n) break;
        uint32_t vr[16], vi[16], tr[16], ti[16];
        tc_ld16(lane_addr + (uint32_t)c0, vr);
        tc_ld16(lane_addr + (uint32_t)(TC_BN + c0), vi);
        if (NCH > 1) {
          tc_ld16(tot + (uint32_t)c0, tr);
          tc_ld16(tot + (uint32_t)(TC_BN + c0), ti);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (r < g.m) {
          // every load of the 16 columns is issued before the first store, so the C reads of a
          // beta != 0 update overlap instead of waiting out one memory latency per column
          float2* cp = g.C + (size_t)r + (size_t)(col0 + c0) * g.ldc;
          const int nc = min(16, g.n - col0 - c0);
          float2 old[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) old[j] = (g.beta != 0.f && j < nc) ? cp[(size_t)j * g.ldc] : make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (j >= nc) break;
            float2 acc = make_float2(0.f, 0.f);
            if (NCH > 0) acc = make_float2(__uint_as_float(vr[j]), __uint_as_float(vi[j]));
            if (NCH > 1) acc = make_float2(acc.x + __uint_as_float(tr[j]), acc.y + __uint_as_float(ti[j]));
            cp[(size_t)j * g.ldc] = g.alpha * acc + g.beta * old[j];
          }
        }
      }
    }
  }
  // MMAs in flight complete before the tensor memory is freed
  __syncwarp();
  const bool fin = tc_wait(&mma_done, 0u);
  const int good = __syncthreads_and(fin && !*abort_v);
  if (!good && tid == 0) atomicExch(&g_tc_error, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ------------------------------------------------------------------------------------- host
bool gemm_tc_enabled() {
  const char* e = std::getenv("NH_GEMM_TC");
  return !(e && std::strcmp(e, "0") == 0);
}

int gemm_tc_run(const std::vector<GemmD<float>>& d, int cls, Arena& ar, cudaStream_t st,
                void* (*stage)(void*, const void*, size_t), void* ctx) {
  if (d.empty()) return 0;
  const bool ta = cls >= 2, tb = (cls & 1) != 0;
  std::vector<PackD> pk;
  std::vector<int> prek, pre;
  std::vector<TcProb> pr;
  int nk = 0, nt = 0;
  for (const auto& g : d) {
    const int kt = (g.k + TC_BK - 1) / TC_BK;
    const int tmn = (g.m + TC_BM - 1) / TC_BM, tnn = (g.n + TC_BN - 1) / TC_BN;
    TcProb p;
    p.C = g.C; p.m = g.m; p.n = g.n; p.ldc = g.ldc; p.ktiles = kt; p.tiles_m = tmn;
    p.alpha = g.alpha; p.beta = g.beta;
    p.Ap = p.Bp = nullptr;
    if (kt > 0) {
      unsigned char* Ap = (unsigned char*)ar.alloc((size_t)tmn * kt * TC_BLK);
      unsigned char* Bp = (unsigned char*)ar.alloc((size_t)tnn * kt * TC_BLK);
      // A: P(r, k) = op(A)(r, k); k is contiguous when op(A) reads A transposed
      pk.push_back({g.A, Ap, g.m, g.k, g.lda, ta ? 1 : 0, g.opA == OP_C ? 1 : 0, tmn, kt});
      prek.push_back(nk);
      nk += tmn * kt;
      // B: P(r, k) = op(B)(k, r); k is contiguous when op(B) reads B as stored
      pk.push_back({g.B, Bp, g.n, g.k, g.ldb, tb ? 0 : 1, g.opB == OP_C ? 1 : 0, tnn, kt});
      prek.push_back(nk);
      nk += tnn * kt;
      p.Ap = Ap; p.Bp = Bp;
    }
    pr.push_back(p);
    pre.push_back(nt);
    nt += tmn * tnn;
  }
  int launches = 1;
  if (nk > 0) {
    auto* dpk = (PackD*)stage(ctx, pk.data(), pk.size() * sizeof(PackD));
    auto* dpr = (int*)stage(ctx, prek.data(), prek.size() * sizeof(int));
    k_tc_pack<<<nk, 256, 0, st>>>(dpk, dpr, (int)pk.size());
    NH_LAUNCH_CK();
    launches++;
  }
  auto* dpb = (TcProb*)stage(ctx, pr.data(), pr.size() * sizeof(TcProb));
  auto* dpre = (int*)stage(ctx, pre.data(), pre.size() * sizeof(int));
  NH_CK(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  k_gemm_tc<<<nt, TC_THREADS, TC_SMEM, st>>>(dpb, dpre, (int)pr.size());
  NH_LAUNCH_CK();
  return launches;
}

int gemm_tc_error(bool reset) {
  int v = 0;
  NH_CK(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)));
  if (reset && v) {
    const int z = 0;
    NH_CK(cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int)));
  }
  return v;
}

}  // namespace nh
