// Shared device/host helpers: complex arithmetic on double2/float2, error handling,
// a stream-ordered device arena, and the matrix view used by every batched operation.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <atomic>
#include <stdexcept>
#include <string>
#include <vector>

namespace nh {

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ERANK = 4,
       ST_ETIMEOUT = 5, ST_ESTATE = 6, ST_ENOTIMPL = 7 };

#define NH_CK(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      throw ::nh::Error(e_ == cudaErrorMemoryAllocation ? ::nh::ST_ENOMEM              \
                                                        : ::nh::ST_ECUDA,             \
                        std::string(#call) + ": " + cudaGetErrorString(e_) +         \
                            " @" + __FILE__ + ":" + std::to_string(__LINE__));       \
    }                                                                                 \
  } while (0)
#define NH_LAUNCH_CK() NH_CK(cudaGetLastError())
#define NH_REQUIRE(cond, code, msg)                     \
  do {                                                  \
    if (!(cond)) throw ::nh::Error((code), (msg));      \
  } while (0)

// ------------------------------------------------------------------ complex types
template <typename R> struct CT;
template <> struct CT<double> { using type = double2; };
template <> struct CT<float> { using type = float2; };
template <typename R> using cplx = typename CT<R>::type;

__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
template <typename R> __host__ __device__ __forceinline__ cplx<R> czero() { return mkc(R(0), R(0)); }

__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

__host__ __device__ __forceinline__ double2 conj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 conj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float abs2(float2 a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ matrix view (column major)
template <typename R> struct Mat {
  cplx<R>* p = nullptr;
  int m = 0, n = 0, ld = 1;
  __host__ __device__ cplx<R>* at(int i, int j) const { return p + (size_t)i + (size_t)j * ld; }
  Mat block(int i0, int j0, int mm, int nn) const {
    Mat b;
    b.p = (mm > 0 && nn > 0) ? at(i0, j0) : p;
    b.m = mm; b.n = nn; b.ld = ld;
    return b;
  }
  size_t bytes() const { return (size_t)ld * n * sizeof(cplx<R>); }
};

// ------------------------------------------------------------------ injected allocation failures
// Host-side fault injection for tests: when armed with k > 0, the k-th device-memory request of the
// arenas from then on fails with ENOMEM (once), exactly as an exhausted device would report it.
inline std::atomic<long long>& fault_alloc_countdown() {
  static std::atomic<long long> c{0};
  return c;
}
inline void fault_alloc_check() {
  auto& c = fault_alloc_countdown();
  if (c.load(std::memory_order_relaxed) > 0 && c.fetch_sub(1) == 1)
    throw Error(ST_ENOMEM, "device allocation failed (injected by nudft2_test_fail_alloc)");
}

// ------------------------------------------------------------------ stream-ordered arena
// Large chunks come from cudaMallocAsync on the owning stream; sub-allocations are bump
// pointers with 256-byte alignment.  mark()/release() give stack-like scratch lifetimes.
class Arena {
 public:
  // dedicated_large: an arena that is never marked or released (long-lived storage) gives every
  // allocation of at least a quarter chunk its own device block, so that large blocks do not
  // leave the unused tails of partly filled chunks behind.
  explicit Arena(size_t chunk = (size_t)256 << 20, bool dedicated_large = false)
      : chunk_(chunk), dedicated_(dedicated_large) {}
  ~Arena() { free_all(); }
  void set_stream(cudaStream_t s) { st_ = s; }
  // While frozen (during CUDA-graph capture) the arena may only reuse chunks it already owns.
  void freeze(bool f) { frozen_ = f; }
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    if (dedicated_ && bytes >= chunk_ / 4) {
      if (frozen_) throw Error(ST_ENOMEM, "arena is frozen during graph capture and has no room left");
      fault_alloc_check();
      void* p = nullptr;
      NH_CK(cudaMallocAsync(&p, bytes, st_));
      big_.push_back({p, bytes});
      total_ += bytes;
      return p;
    }
    if (cur_ < chunks_.size()) {
      // try current chunk, then later (already allocated) chunks
      while (cur_ < chunks_.size()) {
        Chunk& c = chunks_[cur_];
        if (c.used + bytes <= c.size) {
          void* p = (char*)c.p + c.used;
          c.used += bytes;
          total_ += bytes;
          return p;
        }
        cur_++;
      }
    }
    if (frozen_) throw Error(ST_ENOMEM, "arena is frozen during graph capture and has no room left");
    // Every chunk from the stack top on was tried and none fits.  Trailing chunks that hold
    // nothing (used == 0: all their allocations were released) are handed back before growing, so
    // that scratch of varying large sizes does not pile up as dedicated chunks.  The frees are
    // stream-ordered: work still queued on the memory completes first.
    while (!chunks_.empty() && chunks_.back().used == 0) {
      cudaFreeAsync(chunks_.back().p, st_);
      chunks_.pop_back();
    }
    size_t sz = bytes > chunk_ ? bytes : chunk_;
    fault_alloc_check();
    void* p = nullptr;
    NH_CK(cudaMallocAsync(&p, sz, st_));
    chunks_.push_back({p, sz, bytes});
    cur_ = chunks_.size() - 1;
    total_ += bytes;
    return p;
  }
  template <typename R> Mat<R> mat(int m, int n, bool zero = false) {
    Mat<R> a;
    a.m = m; a.n = n; a.ld = m > 0 ? m : 1;
    a.p = (cplx<R>*)alloc((size_t)a.ld * (n > 0 ? n : 1) * sizeof(cplx<R>));
    if (zero) NH_CK(cudaMemsetAsync(a.p, 0, (size_t)a.ld * (n > 0 ? n : 1) * sizeof(cplx<R>), st_));
    return a;
  }
  template <typename T> T* arr(size_t n, bool zero = false) {
    T* p = (T*)alloc(n * sizeof(T));
    if (zero) NH_CK(cudaMemsetAsync(p, 0, n * sizeof(T), st_));
    return p;
  }
  struct Mark { size_t chunk, used, total; };
  Mark mark() const {
    if (chunks_.empty()) return {0, 0, 0};
    return {cur_, chunks_[cur_].used, total_};
  }
  void release(const Mark& mk) {
    if (chunks_.empty()) return;
    for (size_t i = mk.chunk + 1; i < chunks_.size(); ++i) chunks_[i].used = 0;
    if (mk.chunk < chunks_.size()) chunks_[mk.chunk].used = mk.used;
    cur_ = mk.chunk;
    total_ = mk.total;
  }
  void free_all() {
    for (auto& c : chunks_) cudaFreeAsync(c.p, st_);
    for (auto& b : big_) cudaFreeAsync(b.first, st_);
    big_.clear();
    chunks_.clear();
    cur_ = 0;
    total_ = 0;
  }
  size_t reserved() const {
    size_t s = 0;
    for (auto& c : chunks_) s += c.size;
    for (auto& b : big_) s += b.second;
    return s;
  }
  size_t used() const { return total_; }

 private:
  struct Chunk { void* p; size_t size; size_t used; };
  std::vector<Chunk> chunks_;
  std::vector<std::pair<void*, size_t>> big_;   // dedicated blocks (dedicated_large arenas)
  size_t cur_ = 0, chunk_, total_ = 0;
  bool dedicated_ = false;
  cudaStream_t st_ = 0;
  bool frozen_ = false;
};

// Pinned host memory that stays valid as long as the object lives: descriptors uploaded while a
// CUDA graph is captured are copied from here at every replay.
// Allocating pinned memory is not allowed while a stream is being captured, so reserve() takes
// one block up front (outside the capture) and alloc() sub-allocates from it; only when the
// reservation is used up does alloc() fall back to a fresh cudaMallocHost.
class PinnedPool {
 public:
  ~PinnedPool() { for (void* p : blocks_) cudaFreeHost(p); }
  void reserve(size_t bytes) {
    void* p = nullptr;
    NH_CK(cudaMallocHost(&p, bytes > 0 ? bytes : 1));
    blocks_.push_back(p);
    base_ = (char*)p;
    cap_ = bytes;
    off_ = 0;
  }
  void* alloc(size_t bytes) {
    bytes = (bytes + 15) & ~(size_t)15;
    if (base_ && off_ + bytes <= cap_) {
      void* p = base_ + off_;
      off_ += bytes;
      return p;
    }
    void* p = nullptr;
    NH_CK(cudaMallocHost(&p, bytes > 0 ? bytes : 1));
    blocks_.push_back(p);
    return p;
  }
 private:
  std::vector<void*> blocks_;
  char* base_ = nullptr;
  size_t cap_ = 0, off_ = 0;
};

}  // namespace nh
