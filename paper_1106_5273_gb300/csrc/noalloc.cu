// Allocation-free Morton ordering: the spatial sort of the hot path (cube,
// 63-bit Morton keys, stable LSD radix sort) with all of its scratch in one
// file-scope device array.
//
// For callers that cannot call cudaMalloc: code that runs under a memory
// manager owning every device allocation (a framework's caching allocator, a
// fixed device-memory budget) and code that must not trigger the implicit
// device-wide synchronization that cudaMalloc / cudaFree can cause.  The
// plan-based entry points allocate and grow a workspace; this one allocates
// nothing.  The paper has no counterpart of this entry point.
//
// The scratch array below exists on every GPU that loads the library, for the
// life of the process.  In host code its name is only a host-side stand-in,
// not a device address: the device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <atomic>

#include "fmm_internal.cuh"

namespace fmm {
size_t scan_scratch_words(int64_t n);
int radix_sort_u64_raw(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int bit_begin,
                       int bit_end, int* in_second, uint32_t* hist, uint32_t* scan_tmp, cudaStream_t s);
int morton_keys_raw(int64_t n, const float* pos, int periodic, const double* box_min, double box_len,
                    uint64_t* keys, uint32_t* idx, double* partials, double* box, cudaStream_t s);
}  // namespace fmm

namespace {

constexpr int64_t kMaxN = FMM_NOALLOC_MAX_N;
constexpr int64_t kTiles = (kMaxN + 4095) / 4096;
// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffBox = 0;                                                   // 4 doubles
constexpr size_t kOffPart = 256;                                                // 1024 x 6 doubles
constexpr size_t kOffKeys = align256(kOffPart + 1024 * 6 * sizeof(double));     // kMaxN u64
constexpr size_t kOffVals = align256(kOffKeys + kMaxN * sizeof(uint64_t));      // kMaxN u32
constexpr size_t kOffHist = align256(kOffVals + kMaxN * sizeof(uint32_t));      // 256 x kTiles u32
constexpr size_t kOffScan = align256(kOffHist + 256 * kTiles * sizeof(uint32_t));
constexpr size_t kScanWords = 4096;                                             // >= scan_scratch_words(256 * kTiles)
constexpr size_t kScratchBytes = align256(kOffScan + kScanWords * sizeof(uint32_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// Device address of the scratch array, per device.  Atomic so that two host
// threads making their first call on one device at once do not race: both
// look the same address up and store it (release), readers load it (acquire).
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

}  // namespace

extern "C" int fmm_morton_order_noalloc(int64_t n, const float* pos, int periodic, const double* box_min,
                                        double box_len, uint64_t* keys_out, uint32_t* order_out, void* stream) {
  using namespace fmm;
  if (n < 0) return FMM_E_INVAL;
  if (n > kMaxN) return FMM_E_CAPACITY;  // beyond the static scratch
  if (n > 0 && (!pos || !keys_out || !order_out)) return FMM_E_INVAL;
  if (periodic && (!box_min || !(box_len > 0.0))) return FMM_E_INVAL;
  if (n == 0) return FMM_OK;
  if (fmm::scan_scratch_words(256 * kTiles) > kScanWords) return FMM_E_CAPACITY;
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FMM_E_INVAL;
  unsigned char* base = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!base) {
    // set-up, once per device, with that device current
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return FMM_E_CUDA;
    base = static_cast<unsigned char*>(ptr);
    g_scratch_addr[dev].store(base, std::memory_order_release);
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* box = reinterpret_cast<double*>(base + kOffBox);
  double* part = reinterpret_cast<double*>(base + kOffPart);
  uint64_t* keys_alt = reinterpret_cast<uint64_t*>(base + kOffKeys);
  uint32_t* vals_alt = reinterpret_cast<uint32_t*>(base + kOffVals);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
  uint32_t* scan = reinterpret_cast<uint32_t*>(base + kOffScan);
  FMM_TRY(morton_keys_raw(n, pos, periodic, box_min, box_len, keys_out, order_out, part, box, s));
  int second = 0;
  FMM_TRY(radix_sort_u64_raw(keys_out, order_out, keys_alt, vals_alt, n, 0, 63, &second, hist, scan, s));
  if (second) {  // an odd number of passes would leave the result in the scratch halves
    FMM_CUDA_TRY(cudaMemcpyAsync(keys_out, keys_alt, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(order_out, vals_alt, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  return FMM_OK;
}
