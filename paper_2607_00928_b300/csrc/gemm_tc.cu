// Complex FP32 GEMM on the 5th-generation tensor cores (tcgen05.mma, kind::tf32) with the
// 3xTF32 split, for the FP32 generator products of the mixed-precision path.
//
// Every FP32 operand x is split as x = hi + lo, hi = tf32(x) (round to nearest), lo = x - hi
// (exact in FP32); each real product X Y is formed as Xhi Yhi + Xhi Ylo + Xlo Yhi, which keeps
// FP32-level accuracy.  A complex product needs four real ones:
//   Cr += Ar Br - Ai Bi,   Ci += Ar Bi + Ai Br,
// so one 128 x 128 x 8 step of the tile is 12 MMAs (the -Ai Bi ones through the A-negate bit of
// the instruction descriptor).  The two accumulators live in tensor memory (2 x 128 columns).
//
// Per CTA (128 threads): one 128 x 128 output tile of one problem.  The k loop stages 16-deep
// slices of A and B through shared memory (two stages), split into hi/lo planes of real and
// imaginary parts, in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices).  One thread issues the MMAs and commits them to the stage's mbarrier; the stage is
// refilled once that mbarrier reports the MMAs that read it complete.  Every wait is bounded: a
// wait that runs out sets g_tc_error, the CTA waits (bounded) for its MMAs in flight, frees its
// tensor memory and returns without writing C.
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "la.cuh"

namespace nh {

namespace {
constexpr int TC_BM = 128, TC_BN = 128, TC_KT = 16, TC_THREADS = 128;
constexpr int TC_PLANE_A = TC_BM * TC_KT * 4;                       // bytes of one operand plane
constexpr int TC_PLANE_B = TC_BN * TC_KT * 4;
constexpr int TC_STAGE = 4 * TC_PLANE_A + 4 * TC_PLANE_B;           // Ar_hi, Ar_lo, Ai_hi, Ai_lo, then B's
constexpr int TC_SMEM = 2 * TC_STAGE + 1024;                        // two stages + alignment slack
constexpr uint32_t TC_TMEM_COLS = 2 * TC_BN;                        // Cr, Ci
constexpr int TC_SBO = (TC_KT / 4) * 128;                           // bytes between 8-row core groups
constexpr int TC_LBO = 128;                                         // bytes between core matrices along k
constexpr long long TC_SPIN = 1LL << 22;                            // try_wait attempts per wait

// kind::tf32 instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = TC_BN.
constexpr uint32_t tc_idesc(bool negate_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (negate_a ? (1u << 13) : 0u) | ((uint32_t)(TC_BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}
}  // namespace

__device__ int g_tc_error;

// problem of tile t: last i with pre[i] <= t (exclusive tile prefix)
__device__ __forceinline__ int tc_find_prob(const int* pre, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a rows x TC_KT plane in the canonical no-swizzle K-major layout
__device__ __forceinline__ uint32_t tc_kmajor(int r, int k) {
  return (uint32_t)((r >> 3) * TC_SBO + (k >> 2) * TC_LBO + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1,
// base offset 0, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(TC_LBO >> 4) << 16) | ((uint64_t)(TC_SBO >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void tc_split(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(x - __uint_as_float(hi)));   // x - hi is exact in FP32
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = tc_smem_u32(bar);
  for (long long it = 0; it < TC_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc3(const GemmD<float>* __restrict__ ds,
                                                           const int* __restrict__ pre, int np) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ uint64_t bar[3];          // two stage barriers and the final one
  __shared__ uint32_t tslot;
  const uint32_t raw_s = tc_smem_u32(tc_raw);
  unsigned char* sm = tc_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  const int pi = tc_find_prob(pre, np, blockIdx.x);
  const GemmD<float> g = ds[pi];
  const int lt = blockIdx.x - pre[pi];
  const int tiles_m = (g.m + TC_BM - 1) / TC_BM;
  const int row0 = (lt % tiles_m) * TC_BM, col0 = (lt / tiles_m) * TC_BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(&tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&bar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;

  const float sa = g.opA == OP_C ? -1.f : 1.f, sb = g.opB == OP_C ? -1.f : 1.f;
  const int ktiles = (g.k + TC_KT - 1) / TC_KT;
  const uint32_t id_pos = tc_idesc(false), id_neg = tc_idesc(true);
  int ok = 1;
  for (int kt = 0; kt < ktiles; ++kt) {
    const int s = kt & 1;
    unsigned char* st = sm + s * TC_STAGE;
    if (kt >= 2) ok = tc_wait(&bar[s], (uint32_t)(((kt - 2) >> 1) & 1));   // MMAs of tile kt-2 read this stage
    ok = __syncthreads_and(ok);
    if (!ok) break;
    const int k0 = kt * TC_KT;
#pragma unroll 4
    for (int q = 0; q < TC_BM * TC_KT / TC_THREADS; ++q) {
      const int e = tid + q * TC_THREADS;
      int i, kk;
      if (!TA) { i = e % TC_BM; kk = e / TC_BM; } else { kk = e % TC_KT; i = e / TC_KT; }
      const int gi = row0 + i, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gi < g.m && gk < g.k) v = !TA ? g.A[(size_t)gi + (size_t)gk * g.lda] : g.A[(size_t)gk + (size_t)gi * g.lda];
      uint32_t rh, rl, ih, il;
      tc_split(v.x, rh, rl);
      tc_split(sa * v.y, ih, il);
      const uint32_t o = tc_kmajor(i, kk);
      *(uint32_t*)(st + 0 * TC_PLANE_A + o) = rh;
      *(uint32_t*)(st + 1 * TC_PLANE_A + o) = rl;
      *(uint32_t*)(st + 2 * TC_PLANE_A + o) = ih;
      *(uint32_t*)(st + 3 * TC_PLANE_A + o) = il;
    }
#pragma unroll 4
    for (int q = 0; q < TC_BN * TC_KT / TC_THREADS; ++q) {
      const int e = tid + q * TC_THREADS;
      int j, kk;
      if (!TB) { kk = e % TC_KT; j = e / TC_KT; } else { j = e % TC_BN; kk = e / TC_BN; }
      const int gj = col0 + j, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gj < g.n && gk < g.k) v = !TB ? g.B[(size_t)gk + (size_t)gj * g.ldb] : g.B[(size_t)gj + (size_t)gk * g.ldb];
      uint32_t rh, rl, ih, il;
      tc_split(v.x, rh, rl);
      tc_split(sb * v.y, ih, il);
      const uint32_t o = tc_kmajor(j, kk);
      unsigned char* b0 = st + 4 * TC_PLANE_A;
      *(uint32_t*)(b0 + 0 * TC_PLANE_B + o) = rh;
      *(uint32_t*)(b0 + 1 * TC_PLANE_B + o) = rl;
      *(uint32_t*)(b0 + 2 * TC_PLANE_B + o) = ih;
      *(uint32_t*)(b0 + 3 * TC_PLANE_B + o) = il;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy stores -> tensor core
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = tc_smem_u32(st), b0 = a0 + 4 * TC_PLANE_A;
      const uint32_t cr = tmem, ci = tmem + TC_BN;
#pragma unroll
      for (int ks = 0; ks < TC_KT / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 2 * TC_LBO;                 // 8 k = two core matrices
        const uint64_t arh = tc_desc(a0 + 0 * TC_PLANE_A + ko), arl = tc_desc(a0 + 1 * TC_PLANE_A + ko);
        const uint64_t aih = tc_desc(a0 + 2 * TC_PLANE_A + ko), ail = tc_desc(a0 + 3 * TC_PLANE_A + ko);
        const uint64_t brh = tc_desc(b0 + 0 * TC_PLANE_B + ko), brl = tc_desc(b0 + 1 * TC_PLANE_B + ko);
        const uint64_t bih = tc_desc(b0 + 2 * TC_PLANE_B + ko), bil = tc_desc(b0 + 3 * TC_PLANE_B + ko);
        const uint32_t first = (kt == 0 && ks == 0) ? 0u : 1u;
        tc_mma(cr, arh, brh, id_pos, first);
        tc_mma(cr, arh, brl, id_pos, 1u);
        tc_mma(cr, arl, brh, id_pos, 1u);
        tc_mma(cr, aih, bih, id_neg, 1u);
        tc_mma(cr, aih, bil, id_neg, 1u);
        tc_mma(cr, ail, bih, id_neg, 1u);
        tc_mma(ci, arh, bih, id_pos, first);
        tc_mma(ci, arh, bil, id_pos, 1u);
        tc_mma(ci, arl, bih, id_pos, 1u);
        tc_mma(ci, aih, brh, id_pos, 1u);
        tc_mma(ci, aih, brl, id_pos, 1u);
        tc_mma(ci, ail, brh, id_pos, 1u);
      }
      tc_commit(&bar[s]);
    }
  }
  // every MMA issued so far (none if a wait ran out before the first tile) completes before the
  // accumulators are read or the tensor memory is freed
  if (tid == 0) tc_commit(&bar[2]);
  const int fin = __syncthreads_and(tc_wait(&bar[2], 0u));
  if (!ok || !fin) {
    if (tid == 0) atomicExch(&g_tc_error, 1);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int r = row0 + warp * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < TC_BN; c0 += 16) {
      uint32_t vr[16], vi[16];
      tc_ld16(lane_addr + (uint32_t)c0, vr);
      tc_ld16(lane_addr + (uint32_t)(TC_BN + c0), vi);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < g.m) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = col0 + c0 + j;
          if (c >= g.n) break;
          float2* cp = g.C + (size_t)r + (size_t)c * g.ldc;
          const float2 acc = ktiles > 0 ? make_float2(__uint_as_float(vr[j]), __uint_as_float(vi[j]))
                                        : make_float2(0.f, 0.f);
          float2 v = g.alpha * acc;
          if (g.beta != 0.f) v = v + g.beta * (*cp);
          *cp = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

bool gemm_tc_enabled() {
  const char* e = std::getenv("NH_GEMM_TC");
  return e && std::strcmp(e, "1") == 0;
}

void gemm_tc_launch(int cls, const GemmD<float>* dd, const int* dp, int np, int tiles, cudaStream_t st) {
  if (tiles <= 0) return;
  auto go = [&](auto kern) {
    NH_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    kern<<<tiles, TC_THREADS, TC_SMEM, st>>>(dd, dp, np);
    NH_LAUNCH_CK();
  };
  switch (cls) {
    case 0: go(k_gemm_tc3<false, false>); break;
    case 1: go(k_gemm_tc3<false, true>); break;
    case 2: go(k_gemm_tc3<true, false>); break;
    default: go(k_gemm_tc3<true, true>); break;
  }
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
