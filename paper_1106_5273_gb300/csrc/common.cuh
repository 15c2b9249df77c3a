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

// Device buffer that only grows.
struct DBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  int ensure(size_t need) {
    if (need <= bytes) return FMM_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    size_t nb = need + need / 4 + 256;
    if (cudaMalloc(&ptr, nb) != cudaSuccess) return FMM_E_NOMEM;
    bytes = nb;
    return FMM_OK;
  }
  // Grow to at least `need` bytes keeping the current contents.
  int grow_copy(size_t need, cudaStream_t st) {
    if (need <= bytes) return FMM_OK;
    void* np = nullptr;
    size_t nb = need + need / 4 + 256;
    if (cudaMalloc(&np, nb) != cudaSuccess) return FMM_E_NOMEM;
    if (ptr) {
      if (cudaMemcpyAsync(np, ptr, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return FMM_E_CUDA;
      if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_E_CUDA;
      cudaFree(ptr);
    }
    ptr = np;
    bytes = nb;
    return FMM_OK;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
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

