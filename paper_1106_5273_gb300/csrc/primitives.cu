// Device-wide exclusive scan and stable LSD radix sort (keys u64, values u32).
//
// Used by the Morton sort (Sec. 3.2), the tree build, the traversal output
// compaction and the grouping of P2P / M2L lists.  Both are deterministic:
// the scan is a fixed-order reduction, the sort is stable.
#include "primitives.cuh"

namespace fmm {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ inline uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t x = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0u;
    uint32_t xi = warp_incl_scan(x);
    s_warp[lane] = xi - x;
    if (lane == 31) s_warp[32] = xi;
  }
  __syncthreads();
  uint32_t r = inc - v + s_warp[w];
  total = s_warp[32];
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t s_warp[33];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
    if (idx < n) acc += in[idx];
  }
  uint32_t total;
  block_excl_scan(acc, s_warp, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_apply(const uint32_t* in, int64_t n, uint32_t* out,
                             const uint32_t* __restrict__ offs, uint32_t* __restrict__ total_out) {
  __shared__ uint32_t s_warp[33];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v[kScanItems];
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
    v[i] = idx < n ? in[idx] : 0u;
    acc += v[i];
  }
  uint32_t total;
  uint32_t pre = block_excl_scan(acc, s_warp, total);
  uint32_t off = offs ? offs[blockIdx.x] : 0u;
  pre += off;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
    if (idx < n) out[idx] = pre;
    pre += v[i];
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = off + total;
}

}  // namespace

static void scan_rec(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, uint32_t* tmp,
                     cudaStream_t s) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb <= 1) {
    ++g_launches;
    k_scan_apply<<<1, kScanThreads, 0, s>>>(in, n, out, nullptr, total_dev);
    return;
  }
  uint32_t* sums = tmp;
  ++g_launches;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  scan_rec(sums, sums, nb, nullptr, tmp + nb + 1, s);
  ++g_launches;
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, out, sums, total_dev);
}

// Exclusive scan of n u32 values (in may equal out).  If total_dev is given,
// the sum of all values is written there.  tmp is grown as needed.
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, DBuf& tmp,
                       cudaStream_t s) {
  if (n <= 0) {
    if (total_dev) FMM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s));
    return FMM_OK;
  }
  size_t need = 0;
  for (int64_t m = n;;) {
    int64_t nb = (m + kScanTile - 1) / kScanTile;
    if (nb <= 1) break;
    need += (size_t)(nb + 1);
    m = nb;
  }
  FMM_TRY(tmp.ensure((need + 1) * sizeof(uint32_t)));
  scan_rec(in, out, n, total_dev, tmp.as<uint32_t>(), s);
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

// ---------------------------------------------------------- three scans ---
// Exclusive scans of three u32 arrays of one length in the same passes (the
// traversal's per-pair M2L, P2P and push counts).  Each array is scanned
// exactly as exclusive_scan_u32 scans it.

namespace {

struct Scan3Ptrs {
  const uint32_t* in[3];
  uint32_t* out[3];
};

__global__ void k_scan3_reduce(Scan3Ptrs a, int64_t n, uint32_t* __restrict__ sums, int64_t ld) {
  __shared__ uint32_t s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
      if (idx < n) acc += a.in[c][idx];
    }
    uint32_t total;
    block_excl_scan(acc, s_warp, total);
    if (threadIdx.x == 0) sums[c * ld + blockIdx.x] = total;
  }
}

__global__ void k_scan3_apply(Scan3Ptrs a, int64_t n, const uint32_t* __restrict__ offs, int64_t ld,
                              uint32_t* __restrict__ total_out) {
  __shared__ uint32_t s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    uint32_t v[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
      v[i] = idx < n ? a.in[c][idx] : 0u;
      acc += v[i];
    }
    uint32_t total;
    uint32_t pre = block_excl_scan(acc, s_warp, total);
    const uint32_t off = offs ? offs[c * ld + blockIdx.x] : 0u;
    pre += off;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
      if (idx < n) a.out[c][idx] = pre;
      pre += v[i];
    }
    if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) total_out[c] = off + total;
  }
}

}  // namespace

int exclusive_scan3_u32(const uint32_t* const in[3], uint32_t* const out[3], int64_t n, uint32_t* total_dev,
                        DBuf& tmp, DBuf& tmp2, cudaStream_t s) {
  if (n <= 0) {
    if (total_dev) FMM_CUDA_TRY(cudaMemsetAsync(total_dev, 0, 3 * sizeof(uint32_t), s));
    return FMM_OK;
  }
  Scan3Ptrs a;
  for (int c = 0; c < 3; ++c) {
    a.in[c] = in[c];
    a.out[c] = out[c];
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb <= 1) {
    ++g_launches;
    k_scan3_apply<<<1, kScanThreads, 0, s>>>(a, n, nullptr, 0, total_dev);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
  }
  // block sums of the three arrays, scanned in place by the one-array scan
  const int64_t ld = nb + 1;
  FMM_TRY(tmp.ensure((size_t)(3 * ld) * sizeof(uint32_t) + 64));
  uint32_t* sums = tmp.as<uint32_t>();
  ++g_launches;
  k_scan3_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(a, n, sums, ld);
  if (nb <= kScanTile) {  // the three block-sum arrays in one single-block pass (in place)
    Scan3Ptrs b;
    for (int c = 0; c < 3; ++c) {
      b.in[c] = sums + c * ld;
      b.out[c] = sums + c * ld;
    }
    ++g_launches;
    k_scan3_apply<<<1, kScanThreads, 0, s>>>(b, nb, nullptr, 0, nullptr);
  } else {
    for (int c = 0; c < 3; ++c) FMM_TRY(exclusive_scan_u32(sums + c * ld, sums + c * ld, nb, nullptr, tmp2, s));
  }
  ++g_launches;
  k_scan3_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(a, n, sums, ld, total_dev);
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

// ------------------------------------------------------------------ sort ---

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRows = 16;
constexpr int kSortTile = kSortThreads * kSortRows;  // 4096 keys per tile

__global__ void k_sort_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int ntiles,
                            uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRows; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: rows of 256 keys in order; within a row, warps in order;
// within a warp, lanes in order.  Element order = (row, warp, lane).
__global__ void k_sort_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                               uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                               int shift, int ntiles, const uint32_t* __restrict__ offs) {
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_w[8][256];
  __shared__ uint32_t s_base[256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  s_run[tid] = 0;
  s_base[tid] = offs[(size_t)tid * ntiles + blockIdx.x];
  const uint32_t lt_mask = (1u << lane) - 1u;
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRows; ++r) {
    int64_t i = base + r * kSortThreads + tid;
    bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0ull;
    uint32_t val = valid ? vin[i] : 0u;
    int d = valid ? (int)((key >> shift) & 0xff) : 256;
#pragma unroll
    for (int q = 0; q < 8; ++q) s_w[q][tid] = 0;
    __syncthreads();
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) s_w[w][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = s_run[tid];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t c = s_w[q][tid];
        s_w[q][tid] = acc;
        acc += c;
      }
      s_run[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = s_base[d] + s_w[w][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

__global__ void k_iota(uint32_t* v, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

}  // namespace

int iota_u32(uint32_t* v, int64_t n, cudaStream_t s) {
  if (n <= 0) return FMM_OK;
  ++g_launches;
  k_iota<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, n);
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

// Sort (keys, vals) by key bits [bit_begin, bit_end).  Input in (k0,v0);
// on return *in_second says whether the result is in (k1,v1).
int radix_sort_u64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int bit_begin,
                   int bit_end, int* in_second, DBuf& hist, DBuf& scan_tmp, cudaStream_t s, uint64_t vary) {
  *in_second = 0;
  if (n <= 1) return FMM_OK;
  int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  FMM_TRY(hist.ensure((size_t)256 * ntiles * sizeof(uint32_t)));
  uint64_t* ka = k0;
  uint64_t* kb = k1;
  uint32_t* va = v0;
  uint32_t* vb = v1;
  for (int shift = bit_begin; shift < bit_end; shift += 8) {
    const int w = bit_end - shift < 8 ? bit_end - shift : 8;
    if (((vary >> shift) & ((1ull << w) - 1ull)) == 0ull) continue;  // constant digit: identity pass
    ++g_launches;
    k_sort_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, hist.as<uint32_t>());
    FMM_TRY(exclusive_scan_u32(hist.as<uint32_t>(), hist.as<uint32_t>(), (int64_t)256 * ntiles, nullptr,
                               scan_tmp, s));
    ++g_launches;
    k_sort_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, ntiles, hist.as<uint32_t>());
    FMM_CUDA_TRY(cudaGetLastError());
    uint64_t* tk = ka;
    ka = kb;
    kb = tk;
    uint32_t* tv = va;
    va = vb;
    vb = tv;
    *in_second ^= 1;
  }
  return FMM_OK;
}

}  // namespace fmm

namespace fmm {

// Variants of the scan and sort above that take their scratch as raw device
// pointers (for callers that provide all memory): scan_tmp must hold
// scan_scratch_words(n) words, hist 256 * ceil(n/4096) words.
size_t scan_scratch_words(int64_t n) {
  size_t need = 0;
  for (int64_t m = n;;) {
    int64_t nb = (m + kScanTile - 1) / kScanTile;
    if (nb <= 1) break;
    need += (size_t)(nb + 1);
    m = nb;
  }
  return need + 1;
}

int radix_sort_u64_raw(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int bit_begin,
                       int bit_end, int* in_second, uint32_t* hist, uint32_t* scan_tmp, cudaStream_t s) {
  *in_second = 0;
  if (n <= 1) return FMM_OK;
  int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  uint64_t* ka = k0;
  uint64_t* kb = k1;
  uint32_t* va = v0;
  uint32_t* vb = v1;
  for (int shift = bit_begin; shift < bit_end; shift += 8) {
    ++g_launches;
    k_sort_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, hist);
    scan_rec(hist, hist, (int64_t)256 * ntiles, nullptr, scan_tmp, s);
    ++g_launches;
    k_sort_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, ntiles, hist);
    FMM_CUDA_TRY(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
    *in_second ^= 1;
  }
  return FMM_OK;
}

}  // namespace fmm
