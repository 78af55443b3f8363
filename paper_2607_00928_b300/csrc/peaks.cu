// Arithmetic peaks of the GPU the library runs on, measured: the denominators of the rooflines
// of the CUDA-core kernels (FP32 FFMA for the mixed-precision factorization, FP64 DFMA for the
// exact apply and the FP64 path).  Each thread runs 8 independent FMA chains; enough CTAs are
// launched to fill every SM several times over.
#include <algorithm>

#include "../../include/nudft2_hss.h"
#include "common.cuh"

namespace nh {

template <typename R> __global__ void __launch_bounds__(256) k_fma_peak(R* out, int iters, R a, R b) {
  R x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (R)(threadIdx.x + j) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  R s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (R)12345.678) out[0] = s;   // keeps the chains live; never true for these inputs
}

template <typename R> static double fma_peak(cudaStream_t st) {
  int dev = 0, sms = 0;
  NH_CK(cudaGetDevice(&dev));
  NH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  R* out = nullptr;
  NH_CK(cudaMallocAsync(&out, sizeof(R), st));
  const int blocks = sms * 16, threads = 256;
  const int iters = sizeof(R) == 8 ? 1 << 12 : 1 << 16;
  cudaEvent_t e0, e1;
  NH_CK(cudaEventCreate(&e0));
  NH_CK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {   // the first run warms the clocks up
    NH_CK(cudaEventRecord(e0, st));
    k_fma_peak<R><<<blocks, threads, 0, st>>>(out, iters, (R)0.999999, (R)1e-7);
    NH_LAUNCH_CK();
    NH_CK(cudaEventRecord(e1, st));
    NH_CK(cudaEventSynchronize(e1));
    float ms = 0;
    NH_CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  NH_CK(cudaFreeAsync(out, st));
  NH_CK(cudaStreamSynchronize(st));
  return 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
}

}  // namespace nh

using namespace nh;
extern thread_local std::string nudft2_err_tls;   // defined in api.cu

extern "C" nudft2_status nudft2_peak_fma(int prec, double* tflops, void* stream) {
  try {
    NH_REQUIRE(tflops && (prec == NUDFT2_FP64 || prec == NUDFT2_MIXED), ST_EINVAL, "peak_fma: bad arguments");
    *tflops = prec == NUDFT2_FP64 ? fma_peak<double>((cudaStream_t)stream) : fma_peak<float>((cudaStream_t)stream);
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
