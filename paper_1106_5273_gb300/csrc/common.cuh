// Internal definitions shared by the CUDA translation units of the FMM.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/fmm_vortex.h"

namespace fmm {

// Kernel launches issued by this library (all host threads).
extern std::atomic<int64_t> g_launches;

constexpr int kMaxLevel = 21;      // 63-bit Morton keys, 3 bits per level (Sec. 3.2)
constexpr int kPMax = 16;          // expansion degrees 0..15
constexpr int kNCoefMax = kPMax * kPMax;
constexpr int kTile = 64;          // target cells per M2L tile
constexpr int kImageZero = 13;     // image index of the zero shift, (ox+1)*9+(oy+1)*3+(oz+1)

#define FMM_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return FMM_E_CUDA;      \
  } while (0)

#define FMM_TRY(expr)                              \
  do {                                             \
    int r_ = (expr);                               \
    if (r_ != FMM_OK) return r_;                   \
  } while (0)

// A device-byte budget shared by a group of host threads (the serving loop
// installs one on its worker threads with set_thread_budget).  Every DBuf
// allocation made by such a thread is charged to it before cudaMalloc is
// called and refused (FMM_E_NOMEM) if the charge would take the bytes held
// past the limit; the buffer returns its bytes to the same budget when it is
// released, whichever thread releases it.
struct ByteBudget {
  std::atomic<int64_t> held{0};
  std::atomic<int64_t> peak{0};
  std::atomic<int64_t> refusals{0};
  int64_t limit = 0;
  bool charge(int64_t b) {
    int64_t cur = held.load();
    do {
      if (cur + b > limit) {
        ++refusals;
        last_refused() = b;
        return false;
      }
    } while (!held.compare_exchange_weak(cur, cur + b));
    int64_t pk = peak.load();
    while (cur + b > pk && !peak.compare_exchange_weak(pk, cur + b)) {
    }
    return true;
  }
  void credit(int64_t b) { held -= b; }
  // size of the last allocation this host thread had refused
  static int64_t& last_refused() {
    static thread_local int64_t v = 0;
    return v;
  }
};
inline ByteBudget*& thread_budget() {
  static thread_local ByteBudget* b = nullptr;
  return b;
}
inline void set_thread_budget(ByteBudget* b) { thread_budget() = b; }

// Device buffer that only grows.
struct DBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  ByteBudget* owner = nullptr;  // budget charged with `bytes` (nullptr: none)
  int ensure(size_t need) {
    if (need <= bytes) return FMM_OK;
    size_t nb = need + need / 4 + 256;
    ByteBudget* bb = thread_budget();
    if (bb && !bb->charge((int64_t)nb)) return FMM_E_NOMEM;  // the old buffer stays
    release();
    if (cudaMalloc(&ptr, nb) != cudaSuccess) {
      ptr = nullptr;
      if (bb) bb->credit((int64_t)nb);
      return FMM_E_NOMEM;
    }
    bytes = nb;
    owner = bb;
    return FMM_OK;
  }
  // Grow to at least `need` bytes keeping the current contents.
  int grow_copy(size_t need, cudaStream_t st) {
    if (need <= bytes) return FMM_OK;
    void* np = nullptr;
    size_t nb = need + need / 4 + 256;
    ByteBudget* bb = thread_budget();
    if (bb && !bb->charge((int64_t)nb)) return FMM_E_NOMEM;
    if (cudaMalloc(&np, nb) != cudaSuccess) {
      if (bb) bb->credit((int64_t)nb);
      return FMM_E_NOMEM;
    }
    if (ptr) {
      if (cudaMemcpyAsync(np, ptr, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        cudaFree(np);
        if (bb) bb->credit((int64_t)nb);
        return FMM_E_CUDA;
      }
    }
    release();
    ptr = np;
    bytes = nb;
    owner = bb;
    return FMM_OK;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    if (owner) owner->credit((int64_t)bytes);
    ptr = nullptr;
    bytes = 0;
    owner = nullptr;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(ptr); }
};

// Real-packed index of coefficient (n, m>=0, part 0=Re 1=Im): degree n owns
// [n^2, (n+1)^2) as [Re m0, Re m1, Im m1, ..., Re mn, Im mn].
__host__ __device__ inline int ridx(int n, int m, int part) {
  return n * n + (m == 0 ? 0 : 2 * m - 1 + part);
}

}  // namespace fmm

