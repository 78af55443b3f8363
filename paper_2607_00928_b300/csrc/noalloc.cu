// Exact forward apply f = A c (Eq. 1) that allocates no device memory.
//
// Who needs it: callers that must not allocate device memory while they run.  A serving loop
// that reserves all device memory up front at start-up has nothing left for a workspace; a host
// application whose own allocator owns the device (a framework's caching pool) cannot have a
// library allocate behind its back; and latency-bound request paths cannot afford cudaMalloc,
// which may synchronise the device and has no bounded cost.  Instead of asking for workspace,
// this entry point works in one fixed, file-scope device array that every GPU loading the
// library holds until exit.
//
// Contract: the array is shared by all calls in the process.  Calls that overlap on the GPU
// (different streams, or several host threads) race on it; serialise them.  Every byte a call
// reads from the array is written earlier by the same call, so leftovers from the previous call
// never leak into a result.  The call returns once its work is queued on the caller's stream.
#include <cstring>
#include <mutex>

#include "../../include/nudft2_hss.h"
#include "la.cuh"
#include "nudft.cuh"

namespace nh {

// 64 MiB: holds the two twiddle tables and at least one right-hand side of the intermediate
// product for M * (2*nx + ny) <= ~4.19e6, e.g. M = 32768 points with nx = ny = 42, or
// M = 8192 with nx = ny = 170.
constexpr size_t kNoAllocBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr size_t kHeader = 4096;   // descriptor + tile prefix at the start of the array

// Writes the GEMM descriptor and its tile prefix into the array (kernel argument -> device).
__global__ void k_noalloc_header(GemmD<double> g) {
  GemmD<double>* d = reinterpret_cast<GemmD<double>*>(g_noalloc_scratch);
  int* pre = reinterpret_cast<int*>(g_noalloc_scratch + 1024);
  if (threadIdx.x == 0) {
    *d = g;
    *pre = 0;
  }
}

// Device address of the array for the current device, looked up once per device.  In host
// code the symbol name is only a host-side stand-in, so the address must come from the runtime.
static unsigned char* scratch_address() {
  static std::mutex mu;
  static unsigned char* addr[256] = {nullptr};
  int dev = 0;
  NH_CK(cudaGetDevice(&dev));
  NH_REQUIRE(dev >= 0 && dev < 256, ST_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    NH_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = static_cast<unsigned char*>(p);
  }
  return addr[dev];
}

}  // namespace nh

using namespace nh;
extern thread_local std::string nudft2_err_tls;   // defined in api.cu

extern "C" nudft2_status nudft2_exact_fwd_noalloc(const double* d_x, const double* d_y, int64_t M, int nx, int ny,
                                                  const void* d_c, int64_t ldc, int nrhs, void* d_f, int64_t ldf,
                                                  void* stream) {
  try {
    NH_REQUIRE(d_x && d_y && d_c && d_f && M >= 1 && nx >= 1 && ny >= 1 && nrhs >= 0, ST_EINVAL,
               "exact_fwd_noalloc: bad arguments");
    const int64_t N = (int64_t)nx * ny;
    NH_REQUIRE(ldc >= N && ldf >= M, ST_EINVAL, "exact_fwd_noalloc: leading dimension too small");
    NH_REQUIRE(M < (1LL << 31) && ldf < (1LL << 31), ST_EINVAL, "exact_fwd_noalloc: M and ldf must be below 2^31");
    const size_t tab = (size_t)M * (nx + ny) * sizeof(double2);
    const size_t per_rhs = (size_t)M * nx * sizeof(double2);
    NH_REQUIRE(kHeader + tab + per_rhs <= kNoAllocBytes, ST_EINVAL,
               "exact_fwd_noalloc: M*(2*nx+ny)*16 bytes exceeds the 64 MiB fixed workspace");
    NH_REQUIRE(ldc == N, ST_EINVAL, "exact_fwd_noalloc: coefficients must be contiguous (ldc == nx*ny)");
    if (nrhs == 0) {
      nudft2_err_tls.clear();
      return NUDFT2_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = scratch_address();
    auto* desc = reinterpret_cast<GemmD<double>*>(base);
    auto* pre = reinterpret_cast<int*>(base + 1024);
    auto* Ax = reinterpret_cast<double2*>(base + kHeader);
    auto* Ay = Ax + (size_t)M * nx;
    auto* T = Ay + (size_t)M * ny;
    const int chunk = (int)std::min<size_t>((size_t)nrhs, (kNoAllocBytes - kHeader - tab) / per_rhs);
    twiddle_table(st, d_x, (int)M, nx, Ax);
    twiddle_table(st, d_y, (int)M, ny, Ay);
    for (int q0 = 0; q0 < nrhs; q0 += chunk) {
      const int qs = std::min(chunk, nrhs - q0);
      // T (M x nx*qs) = Ay (M x ny) * C (ny x nx*qs): the inner sum over ky of Eq. 1
      GemmD<double> g{Ay, static_cast<const double2*>(d_c) + (size_t)q0 * ldc, T, (int)M, nx * qs, ny, (int)M, ny,
                      (int)M, OP_N, OP_N, 1.0, 0.0};
      k_noalloc_header<<<1, 32, 0, st>>>(g);
      NH_LAUNCH_CK();
      gemm_launch_raw(desc, pre, 1, gemm_tiles(g), st);
      // f_j = sum_kx Ax(j, kx) T(j, kx): the outer sum
      rowdot(st, Ax, (int)M, T, (int)M, (int)M, nx, qs, static_cast<double2*>(d_f) + (size_t)q0 * ldf, (int)ldf);
    }
    nudft2_err_tls.clear();
    return NUDFT2_OK;
  } catch (Error& e) {
    nudft2_err_tls = e.what();
    return (nudft2_status)e.code;
  } catch (std::exception& e) {
    nudft2_err_tls = e.what();
    return NUDFT2_ECUDA;
  }
}
