// Shared host/device plumbing of the library: status handling, the device
// memory arena of a plan, the canonical constants and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hlc.h"

namespace hlc {

// ---------------------------------------------------------------------------
// Status and messages.
// ---------------------------------------------------------------------------

void set_error(const char* fmt, ...);
void clear_error();

struct Status {
  int code = HLC_OK;
  bool ok() const { return code == HLC_OK; }
};

#define HLC_TRY(expr)                 \
  do {                                \
    int _rc = (expr);                 \
    if (_rc != HLC_OK) return _rc;    \
  } while (0)

#define HLC_CUDA(call)                                                      \
  do {                                                                      \
    cudaError_t _e = (call);                                                \
    if (_e != cudaSuccess) {                                                \
      ::hlc::set_error("%s failed at %s:%d: %s", #call, __FILE__, __LINE__, \
                       cudaGetErrorString(_e));                             \
      return _e == cudaErrorMemoryAllocation ? HLC_ENOMEM : HLC_ECUDA;      \
    }                                                                       \
  } while (0)

extern std::atomic<unsigned long long> g_launches;  // kernels launched so far

#define HLC_LAUNCH_CHECK()                                                  \
  do {                                                                      \
    ::hlc::g_launches.fetch_add(1, std::memory_order_relaxed);              \
    cudaError_t _e = cudaGetLastError();                                    \
    if (_e != cudaSuccess) {                                                \
      ::hlc::set_error("kernel launch failed at %s:%d: %s", __FILE__,       \
                       __LINE__, cudaGetErrorString(_e));                   \
      return HLC_ECUDA;                                                     \
    }                                                                       \
  } while (0)

// ---------------------------------------------------------------------------
// Device error word: kernels record problems here instead of trapping.
// ---------------------------------------------------------------------------
enum DevErr : int {
  DERR_NONE = 0,
  DERR_INPUT = 1,     // non-finite RA/Dec or |Dec| > 90
  DERR_TIMEOUT = 2,   // a bounded spin-wait gave up
  DERR_OVERFLOW = 4,  // an output buffer was too small (host retries)
  DERR_BOUNDS = 8,    // an index check failed (skipped access)
  DERR_BUCKET = 16,   // an output bucket exceeded the in-block sort (host re-orders)
};

// ---------------------------------------------------------------------------
// Allocation: the caller's allocator, or stream-ordered cudaMallocAsync.
// ---------------------------------------------------------------------------
struct Allocator {
  hlc_alloc_fn alloc = nullptr;
  hlc_dealloc_fn dealloc = nullptr;
  void* ctx = nullptr;
  cudaStream_t stream = nullptr;
};

// Owns a list of device buffers; released together.
class Arena {
 public:
  explicit Arena(const Allocator& a) : a_(a) {}
  ~Arena() { release(); }
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;

  // Allocate bytes (rounded up to 256); nullptr with the error set on failure.
  void* get(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (a_.alloc) {
      p = a_.alloc(bytes, a_.ctx);
      if (!p) set_error("device allocator callback returned NULL for %zu bytes", bytes);
    } else {
      cudaError_t e = cudaMallocAsync(&p, bytes, a_.stream);
      if (e != cudaSuccess) {
        set_error("cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        cudaGetLastError();
        p = nullptr;
      }
    }
    if (p) bufs_.push_back(p);
    return p;
  }
  template <typename T>
  T* get_n(size_t n) {
    return static_cast<T*>(get(n * sizeof(T)));
  }
  void release() {
    for (void* p : bufs_) {
      if (a_.dealloc)
        a_.dealloc(p, a_.ctx);
      else
        cudaFreeAsync(p, a_.stream);
    }
    bufs_.clear();
  }
  // Free one buffer early (must have come from this arena).
  void drop(void* p) {
    for (size_t i = 0; i < bufs_.size(); ++i)
      if (bufs_[i] == p) {
        if (a_.dealloc)
          a_.dealloc(p, a_.ctx);
        else
          cudaFreeAsync(p, a_.stream);
        bufs_.erase(bufs_.begin() + i);
        return;
      }
  }
  cudaStream_t stream() const { return a_.stream; }
  const Allocator& allocator() const { return a_; }

 private:
  Allocator a_;
  std::vector<void*> bufs_;
};

#define HLC_ALLOC(arena, ptr, T, n)                                    \
  do {                                                                 \
    (ptr) = (arena).get_n<T>(n);                                       \
    if (!(ptr)) return HLC_ENOMEM;                                     \
  } while (0)

// ---------------------------------------------------------------------------
// Canonical constants (one copy per process, derived at load).
// ---------------------------------------------------------------------------
struct Canon {
  double s[10];  // sin Taylor terms in degrees
  double c[11];  // cos Taylor terms in degrees
};

void derive_trig_coefficients(double sin_c[10], double cos_c[11]);
const Canon& canon();
int ensure_device_tables();  // uploads constant tables to the current device

// ---------------------------------------------------------------------------
// Small device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Test hook: every bounded device wait gives up after its spin limit shifted
// right by d_spin_shift (0, the default, keeps the production limits; set
// through hlc_test_spin_shift).
__device__ int d_spin_shift = 0;
__device__ __forceinline__ long long spin_limit(long long base) { return base >> d_spin_shift; }

// Streaming multiprocessors of the current device (queried once per device;
// grids are sized in multiples of it).
inline unsigned num_sms() {
  static std::atomic<unsigned> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 148u;
  }
  unsigned v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 148;
    }
    v = (unsigned)n;
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// Blocks for n items of `block` threads, at most `cap` (0: 64 per SM).
inline unsigned grid_for(uint64_t n, int block, unsigned cap = 0) {
  if (cap == 0) cap = num_sms() * 64u;
  uint64_t g = (n + block - 1) / block;
  if (g == 0) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace hlc
