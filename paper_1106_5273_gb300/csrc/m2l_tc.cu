// M2L on the 5th-generation tensor cores (tcgen05), BF16x3 split products
// with FP32 accumulation in tensor memory (Sec. 3.1 M2L, batched per
// translation vector).
//
// A step applies one translation operator T (P x P, P = p^2) to the
// multipoles of the 64 source cells paired with a tile of 64 target cells:
//   D[128 x 192] += T[128 x K] . B[K x 192],  B column (comp, slot) = M~ of
// the slot's source for that potential component (zero if the slot has no
// source under this translation).  T = T_hi + T_lo and B = B_hi + B_lo in
// BF16; D accumulates T_hi B_hi + T_hi B_lo + T_lo B_hi (the lo.lo term is
// below FP32 resolution of the sum).  The K chunks from m2l_split_chunks on
// (source degrees 8 and up) take T_hi B_hi only: under the MAC their terms
// are at most theta^8 / (1 - theta) of the leading one, which keeps the
// 2^-8 error of one BF16 product there under 7e-6 for theta <= 0.42.  D lives in TMEM for all steps of the
// tile; each target local expansion is written once.  P > 128 output rows
// take a second CTA per tile (blockIdx.y = block of 128 rows), which gathers
// the same B and its own rows of T.
//
// Per stage (one step, one 64-wide K chunk): A (T hi/lo, pre-swizzled in
// global memory in the 128B-swizzle K-major layout) arrives by two 1-D bulk
// copies on mbarrier fullA; 8 producer warps gather the B rows (128 B each)
// and store them swizzled, then arrive on fullB; one thread issues the MMAs
// and commits them to the stage's empty barrier.  One stage per CTA and two
// CTAs per SM (81 KB of shared memory and 256 TMEM columns each): while one
// CTA waits on its gathers and barriers the other's MMAs keep the tensor pipe
// busy.  The producers load a stage's rows into registers before they wait
// for its buffer.  Measured at 2M blobs: 5.6 ms, against 6.6 ms without the
// early loads and 7.8 ms for two stages in one CTA per SM.  When a step has
// two K chunks and the second takes one product (p = 9, 10 at theta <= 0.42)
// the stage holds the whole step instead (three operator blocks of the rows
// below P and three B blocks, 111 KB at p = 10, still two CTAs per SM), so
// the operator-copy latency is paid once per step.  Every wait is
// bounded; on expiry the kernel records FMM_E_TIMEOUT, waits (bounded) for
// its own bulk copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kN = 3 * kTile;                               // 192 columns
constexpr int kStages = 1;  // pipeline stages per CTA (the loop also runs with 2)
constexpr int kProducerWarps = 8;
constexpr int kProducers = kProducerWarps * 32;
constexpr int kThreads = kProducers + 32;                   // + control warp
constexpr uint32_t kABytes = 128 * 128;                     // 128 rows x 64 bf16
constexpr uint32_t kBBytes = kN * 128;                      // 192 rows x 64 bf16
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;  // 80 KB
constexpr uint32_t kBarOff = kStages * kStageBytes;
constexpr int kTmemCols = 256;
constexpr long long kSpin = 1ll << 24;
constexpr int kGather = (2 * kN * 8) / kProducers;          // 16-byte items per producer thread (12)
// Work items of one-problem plans: S = steps / kItemTarget (about four items
// per concurrent CTA, 2 per SM x 152 SMs) clamped to [kItemMinSteps,
// kItemMaxSteps], then raised if needed so that there are at most kItemsMax
// items.  The upper clamp is for accuracy as much as for balance: the FP32
// accumulation of the tensor memory over a whole tile's steps (thousands of
// MMAs into one sum) measured 4x the M2L error of sums over at most a few
// hundred steps added in FP32 afterwards.
constexpr int64_t kItemMinSteps = 64;
constexpr int64_t kItemMaxSteps = 256;
constexpr int64_t kItemTarget = 4 * 2 * 152;
constexpr int64_t kItemsMax = 1 << 15;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t tx) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(tx)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the limit is reached (the caller aborts).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          long long limit = kSpin) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023) == 1023 && *abort) return false;
  }
  *abort = 1;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptors: D f32, both operands K-major, N = 192, M = 128;
// kind::f16 with A and B BF16 (format 1), kind::tf32 with A and B TF32 (format 2).
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) | ((128u >> 4) << 24);

template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  if (KIND == 0)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(kIdescBf16), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(kIdescTf32), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// KIND 0: BF16 operands (64 per 128-byte row, K step 16); KIND 1: TF32 (32
// per row, K step 8).  Tb / Mb hold 128-byte rows: a K chunk of one operator
// row or one (cell, hi/lo, component) multipole row.
// items == nullptr: CTA x runs all steps of tile x and writes its local
// expansions.  Otherwise CTA x runs work item x (tile, first step, end step,
// partial slot) of *nitems: a tile's steps in runs of at most S; a tile split
// into several items writes each item's D to its partial slot, summed later
// by k_m2l_combine.
template <int KIND, bool M2>
__global__ void __launch_bounds__(kThreads, 2)
    k_m2l_tc(const int2* __restrict__ tile_range, const int4* __restrict__ items, const uint32_t* __restrict__ nitems,
             const int* __restrict__ tfirst, const int* __restrict__ st_slot, const int* __restrict__ st_src,
             const uint8_t* __restrict__ Tb, const uint8_t* __restrict__ Mb, int P, int nkc, int nkc3, int ksteps_last,
             int nrh,
             const int* __restrict__ tcell, float* __restrict__ L, float* __restrict__ partial,
             int* __restrict__ flag) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  int tile = blockIdx.x, pslot = -1;
  int2 rg;
  if (items) {
    if (blockIdx.x >= *nitems) return;  // beyond the items of this evaluation
    const int4 w = items[blockIdx.x];
    tile = w.x;
    rg = make_int2(w.y, w.z);
    pslot = w.w;
  } else {
    rg = tile_range[tile];
  }
  const int rh = blockIdx.y;  // block of 128 output rows
  if (rg.y <= rg.x) return;  // no M2L for this tile: the whole CTA leaves before any barrier
  // Only the operator rows below P are copied (whole 8-row swizzle groups):
  // the rows above feed only output rows that the epilogue never stores.
  const uint32_t arows = (uint32_t)min(128, ((P - rh * 128) + 7) & ~7);
  const uint32_t abytes = arows * 128u;
  // M2 (two K chunks, the second with one product, P <= 128): the stage holds
  // a whole step, A buffers of abytes (chunk 0 hi, chunk 0 lo, chunk 1 hi;
  // the MMA's rows past arows read the next buffer and feed discarded output
  // rows) followed by the B buffers (chunk 0 hi, chunk 0 lo, chunk 1 hi).
  const uint32_t abuf = M2 ? abytes : kABytes;
  const uint32_t stage_bytes = M2 ? 3u * abuf + 3u * kBBytes : kStageBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + stage_bytes);
  // bars: fullA[2], fullB[2], empty[2], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
  volatile int* abort = reinterpret_cast<volatile int*>(bars + 9);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  auto fullA = [&](int s) { return bar0 + 8u * (uint32_t)s; };
  auto fullB = [&](int s) { return bar0 + 8u * (uint32_t)(2 + s); };
  auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(4 + s); };
  const uint32_t done = bar0 + 8u * 6u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(fullA(s), 1);
      mbar_init(fullB(s), kProducers);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == kProducerWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int niter = M2 ? (rg.y - rg.x) : (rg.y - rg.x) * nkc;

  if (M2 && warp < kProducerWarps) {
    // ---- producers, whole step per stage: 16-byte chunk j = t % 8 of rows
    // n = t/8 + 32k (k = 0..5) of the three B buffers
    const int j = threadIdx.x & 7, r0 = threadIdx.x >> 3;
    constexpr int G = 18;
    for (int it = 0; it < niter; ++it) {
      const uint32_t ph = (uint32_t)it & 1u;
      const int st = rg.x + it;
      const int srcA = __ldg(st_src + (size_t)st * kTile + r0), srcB = __ldg(st_src + (size_t)st * kTile + r0 + 32);
      uint4 v[G];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int bsel = q / 6, k = q % 6;  // buffer: chunk 0 hi, chunk 0 lo, chunk 1 hi
        const int h = bsel == 1 ? 1 : 0, kc = bsel == 2 ? 1 : 0;
        const int src = (k & 1) ? srcB : srcA;
        v[q] = make_uint4(0u, 0u, 0u, 0u);
        if (src >= 0)
          v[q] = __ldg(reinterpret_cast<const uint4*>(Mb + ((((size_t)src * 2 + h) * 3 + (k >> 1)) * nkc + kc) * 128) +
                       j);
      }
      if (!mbar_wait(empty(0), ph ^ 1u, abort)) break;
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int bsel = q / 6, n = r0 + 32 * (q % 6);
        *reinterpret_cast<uint4*>(smem + 3 * abuf + bsel * kBBytes + n * 128 + ((j ^ (n & 7)) << 4)) = v[q];
      }
      fence_proxy_async();
      mbar_arrive(fullB(0));
    }
  } else if (M2 && lane == 0 && warp == kProducerWarps) {
    // ---- control thread, whole step per stage: three operator copies, then
    // 12 MMAs for chunk 0 (three products) and ksteps_last for chunk 1 (hi x hi)
    int issued = 0, consumed = 0;
    bool ok = true;
    const size_t chunk = (size_t)128 * 128;  // bytes of one (operator, hi/lo, K chunk) block (nrh == 1)
    for (int it = 0; it < niter; ++it) {
      const uint32_t ph = (uint32_t)it & 1u;
      if (!mbar_wait(empty(0), ph ^ 1u, abort)) {
        ok = false;
        break;
      }
      const size_t key = (size_t)st_slot[rg.x + it];
      const uint32_t a0 = sbase;
      mbar_arrive_tx(fullA(0), 3u * abytes);
      bulk_g2s(a0, Tb + ((key * 2 + 0) * nkc + 0) * chunk, abytes, fullA(0));
      bulk_g2s(a0 + abuf, Tb + ((key * 2 + 1) * nkc + 0) * chunk, abytes, fullA(0));
      bulk_g2s(a0 + 2 * abuf, Tb + ((key * 2 + 0) * nkc + 1) * chunk, abytes, fullA(0));
      issued = it + 1;
      if (!mbar_wait(fullA(0), ph, abort)) {
        ok = false;
        break;
      }
      consumed = it + 1;
      if (!mbar_wait(fullB(0), ph, abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t b0 = a0 + 3 * abuf;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t off = (uint32_t)kk * 32u;
        umma<KIND>(tmem, sw128_desc(a0 + off), sw128_desc(b0 + off), (it > 0 || kk > 0) ? 1u : 0u);
        umma<KIND>(tmem, sw128_desc(a0 + off), sw128_desc(b0 + kBBytes + off), 1u);
        umma<KIND>(tmem, sw128_desc(a0 + abuf + off), sw128_desc(b0 + off), 1u);
      }
      for (int kk = 0; kk < ksteps_last; ++kk) {
        const uint32_t off = (uint32_t)kk * 32u;
        umma<KIND>(tmem, sw128_desc(a0 + 2 * abuf + off), sw128_desc(b0 + 2 * kBBytes + off), 1u);
      }
      umma_commit(empty(0));
    }
    if (ok) {
      umma_commit(done);
    } else {
      *abort = 1;
      volatile int never = 0;
      for (int it = consumed; it < issued; ++it) mbar_wait(fullA(0), (uint32_t)it & 1u, &never);
      umma_commit(done);
      mbar_wait(done, 0u, &never);
      atomicExch(flag, FMM_E_TIMEOUT);
    }
  } else if (M2) {
    // the other lanes of the control warp go straight to the teardown
  } else if (warp < kProducerWarps) {
    // ---- producers: thread t stores 16-byte chunk j = t % 8 of rows n = t/8 + 32k
    // (k = 0..5) of both halves, i.e. of the sources in slots t/8 and t/8 + 32;
    // the rows are loaded before the stage's buffer is waited for.
    static_assert(kGather == 12 && kProducers == 256 && kN == 192, "producer row mapping");
    const int j = threadIdx.x & 7, r0 = threadIdx.x >> 3;
    for (int it = 0; it < niter; ++it) {
      const int stage = it % kStages;
      const uint32_t ph = (uint32_t)(it / kStages) & 1u;
      const int st = rg.x + it / nkc, kc = it % nkc;
      const bool lo = kc < nkc3;  // chunks from nkc3 on take the hi.hi product only
      const int srcA = __ldg(st_src + (size_t)st * kTile + r0), srcB = __ldg(st_src + (size_t)st * kTile + r0 + 32);
      uint4 v[kGather];
#pragma unroll
      for (int q = 0; q < kGather; ++q) {
        const int h = q / 6, k = q % 6;
        const int src = (k & 1) ? srcB : srcA;
        v[q] = make_uint4(0u, 0u, 0u, 0u);
        if (src >= 0 && (h == 0 || lo))
          v[q] = __ldg(reinterpret_cast<const uint4*>(Mb + ((((size_t)src * 2 + h) * 3 + (k >> 1)) * nkc + kc) * 128) +
                       j);
      }
      if (!mbar_wait(empty(stage), ph ^ 1u, abort)) break;
#pragma unroll
      for (int q = 0; q < kGather; ++q) {
        const int h = q / 6, n = r0 + 32 * (q % 6);
        if (h == 0 || lo)
          *reinterpret_cast<uint4*>(smem + stage * kStageBytes + 2 * kABytes + h * kBBytes + n * 128 +
                                    ((j ^ (n & 7)) << 4)) = v[q];
      }
      fence_proxy_async();
      mbar_arrive(fullB(stage));
    }
  } else if (lane == 0) {
    // ---- control thread: operator copies and MMAs
    int issued = 0;  // A copies issued for iterations [0, issued)
    auto issue_A = [&](int it) -> bool {
      const int stage = it % kStages;
      const uint32_t ph = (uint32_t)(it / kStages) & 1u;
      if (!mbar_wait(empty(stage), ph ^ 1u, abort)) return false;
      const int st = rg.x + it / nkc, kc = it % nkc;
      const size_t key = (size_t)st_slot[st];
      const size_t chunk = (size_t)nrh * 128 * 128, row0 = (size_t)rh * 128 * 128;  // bytes
      const uint8_t* hi = Tb + ((key * 2 + 0) * nkc + kc) * chunk + row0;
      const uint8_t* lo = Tb + ((key * 2 + 1) * nkc + kc) * chunk + row0;
      const uint32_t a0 = sbase + stage * kStageBytes;
      const bool with_lo = kc < nkc3;
      mbar_arrive_tx(fullA(stage), with_lo ? 2 * abytes : abytes);
      bulk_g2s(a0, hi, abytes, fullA(stage));
      if (with_lo) bulk_g2s(a0 + kABytes, lo, abytes, fullA(stage));
      issued = it + 1;
      return true;
    };
    // operator copies run kStages - 1 iterations ahead of the MMAs
    constexpr int kAhead = kStages - 1;
    bool ok = true;
    for (int k = 0; ok && k < kAhead && k < niter; ++k) ok = issue_A(k);
    int consumed = 0;  // iterations whose A copy was observed complete
    for (int it = 0; ok && it < niter; ++it) {
      const int stage = it % kStages;
      const uint32_t ph = (uint32_t)(it / kStages) & 1u;
      if (it + kAhead < niter && !issue_A(it + kAhead)) {
        ok = false;
        break;
      }
      if (!mbar_wait(fullA(stage), ph, abort)) {
        ok = false;
        break;
      }
      consumed = it + 1;
      if (!mbar_wait(fullB(stage), ph, abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int kc = it % nkc;
      const int ks = (kc == nkc - 1) ? ksteps_last : 4;
      const uint32_t a_hi = sbase + stage * kStageBytes, a_lo = a_hi + kABytes;
      const uint32_t b_hi = a_hi + 2 * kABytes, b_lo = b_hi + kBBytes;
      const bool three = kc < nkc3;
      for (int kk = 0; kk < ks; ++kk) {
        const uint32_t off = (uint32_t)kk * 32u;
        umma<KIND>(tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), (it > 0 || kk > 0) ? 1u : 0u);
        if (three) {
          umma<KIND>(tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), 1u);
          umma<KIND>(tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), 1u);
        }
      }
      umma_commit(empty(stage));
    }
    if (ok) {
      umma_commit(done);
    } else {
      *abort = 1;
      // let our own in-flight bulk copies land and our MMAs finish before
      // the tensor memory is freed and the CTA exits
      volatile int never = 0;
      for (int it = consumed; it < issued; ++it)
        mbar_wait(fullA(it % kStages), (uint32_t)(it / kStages) & 1u, &never);
      umma_commit(done);
      mbar_wait(done, 0u, &never);
      atomicExch(flag, FMM_E_TIMEOUT);
    }
  }
  // ---- epilogue: warps 0-3 own TMEM lanes 0-127 (rows = output coefficients)
  if (warp < 4) {
    if (mbar_wait(done, 0u, abort)) {
      tc_fence_after();
      const int first = tfirst[tile];
      const int ncell = tfirst[tile + 1] - first;
      const int r = rh * 128 + warp * 32 + lane;  // output coefficient of this TMEM lane
      float* pdst = pslot >= 0 ? partial + ((size_t)pslot * nrh + rh) * (size_t)kN * 128 : nullptr;
#pragma unroll 1
      for (int cb = 0; cb < kN / 16; ++cb) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = cb * 16 + i;
          const int comp = n / kTile, slot = n % kTile;
          if (pdst) pdst[(size_t)n * 128 + warp * 32 + lane] = v[i];  // [column][row of the block]
          else if (r < P && slot < ncell) L[((size_t)tcell[first + slot] * 3 + comp) * P + r] = v[i];
        }
      }
    } else {
      atomicExch(flag, FMM_E_TIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kProducerWarps) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---- work items (one-problem plans): runs of at most S steps per CTA

__global__ void k_m2l_item_count(const int2* __restrict__ tr, int ntiles, int S, uint32_t* __restrict__ cnt,
                                 uint32_t* __restrict__ pcnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const int c = tr[t].y - tr[t].x;
  const uint32_t k = c > 0 ? (uint32_t)((c + S - 1) / S) : 0u;
  cnt[t] = k;
  pcnt[t] = k > 1 ? k : 0u;
}

__global__ void k_m2l_item_fill(const int2* __restrict__ tr, int ntiles, int S, const uint32_t* __restrict__ cnt,
                                const uint32_t* __restrict__ ioff, const uint32_t* __restrict__ poff,
                                int4* __restrict__ items) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const uint32_t k = cnt[t];
  for (uint32_t q = 0; q < k; ++q) {
    const int s0 = tr[t].x + (int)q * S;
    items[ioff[t] + q] = make_int4(t, s0, min(s0 + S, tr[t].y), k > 1 ? (int)(poff[t] + q) : -1);
  }
}

// Local expansions of the split tiles: the partial sums of their items, added
// in item order (a fixed order, so the result is deterministic).
__global__ void k_m2l_combine(const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ poff,
                              const int* __restrict__ tfirst, const int* __restrict__ tcell, int P, int nrh,
                              const float* __restrict__ partial, float* __restrict__ L) {
  const int t = blockIdx.x;
  const uint32_t k = cnt[t];
  if (k <= 1) return;
  const int first = tfirst[t], ncell = tfirst[t + 1] - first;
  const size_t per = (size_t)nrh * kN * 128;  // floats per partial slot
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < nrh * kN * 128; e += gridDim.y * blockDim.x) {
    const int r = e & 127, n = (e >> 7) % kN, rh = e / (kN * 128);
    const int row = rh * 128 + r, slot = n % kTile, comp = n / kTile;
    if (row >= P || slot >= ncell) continue;
    float acc = 0.f;
    for (uint32_t q = 0; q < k; ++q) acc += partial[(size_t)(poff[t] + q) * per + (size_t)e];
    L[((size_t)tcell[first + slot] * 3 + comp) * P + row] = acc;
  }
}

// Self-test of the bounded wait above: one thread waits on a barrier that
// either completes (arrive = 1: it arrives first) or that nothing completes
// (arrive = 0), polling at most `spins` times; FMM_OK or FMM_E_TIMEOUT.
__global__ void k_wait_selftest(long long spins, int arrive, int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    const uint32_t b = smem_u32(&bar);
    abort_flag = 0;
    mbar_init(b, 1);
    if (arrive) mbar_arrive(b);
    *status = mbar_wait(b, 0u, &abort_flag, spins) ? FMM_OK : FMM_E_TIMEOUT;
  }
}

}  // namespace

int m2l_tensor(fmm_plan p, cudaStream_t s) {
  if (p->n_steps == 0) return FMM_OK;
  const int kind = p->tc_kind;
  const int ksteps = (p->P + m2l_kstep(kind) - 1) / m2l_kstep(kind);
  const int nkc = m2l_kchunks(p->P, kind);
  const int last = ksteps - 4 * (nkc - 1);
  const int nkc3 = m2l_split_chunks(p->P, kind, p->prm.theta, p->prm.m2l_mode & FMM_M2L_FULL_SPLIT);
  const size_t sh = (size_t)kBarOff + 128 + 1024;
  static bool attr_set[2] = {false, false};
  if (!attr_set[kind]) {
    FMM_CUDA_TRY(cudaFuncSetAttribute(kind ? k_m2l_tc<1, false> : k_m2l_tc<0, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    attr_set[kind] = true;
  }
  const int nrh = m2l_rowblocks(p->P);
  // A whole step per stage when it has two BF16 K chunks, the second with one
  // product, in one block of output rows, and two such CTAs still fit an SM
  // (p = 9 and 10 at theta <= 0.42): one operator-copy latency per step
  // instead of one per chunk.
  bool m2 = false;
  size_t sh2 = 0;
  if (kind == 0 && nkc == 2 && nkc3 == 1 && nrh == 1 && !(p->prm.m2l_mode & FMM_M2L_CHUNK_STAGES)) {
    const size_t arows = (size_t)std::min(128, (p->P + 7) & ~7);
    sh2 = 3 * arows * 128 + 3 * (size_t)kBBytes + 128 + 1024;
    static int m2_ok = -1;  // 1: two CTAs per SM at the largest stage (P = 128 rows would not fit)
    static size_t m2_sh = 0;
    if (m2_ok < 0 || m2_sh != sh2) {
      // Two CTAs per SM by shared memory (each with the per-block reserve) and
      // registers, from the device and kernel attributes; the occupancy query
      // reports one CTA per SM for both forms of this kernel, although two
      // run (ncu: 17.5 of 18 warps active per SM).  Two such CTAs need the
      // largest shared-memory carveout.
      int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0;
      cudaFuncAttributes fa{};
      m2_ok = cudaGetDevice(&dev) == cudaSuccess &&
                      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ==
                          cudaSuccess &&
                      cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
                      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
                      cudaFuncGetAttributes(&fa, k_m2l_tc<0, true>) == cudaSuccess &&
                      cudaFuncSetAttribute(k_m2l_tc<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh2) ==
                          cudaSuccess &&
                      cudaFuncSetAttribute(k_m2l_tc<0, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) ==
                          cudaSuccess &&
                      2 * (sh2 + (size_t)resv + fa.sharedSizeBytes) <= (size_t)smem_sm &&
                      2 * (size_t)fa.numRegs * kThreads <= (size_t)regs_sm
                  ? 1
                  : 0;
      cudaGetLastError();
      m2_sh = sh2;
    }
    m2 = m2_ok == 1;
  }
  p->m2l_stage_chunks = m2 ? 2 : 1;
  const int nt = (int)p->ntiles;
  const int T = 256;
  // One-problem plans split the tiles into work items of at most S steps:
  // with Alg. 1's printed rule the coarse target tiles collect many more
  // steps than the rest, and one CTA per tile left a long tail (and long
  // tensor-memory sums).  Batches keep one CTA per tile: their tiles mix
  // problems, and items cut at fixed step counts would make a problem's sums
  // depend on the other problems of the batch.
  const int4* items = nullptr;
  const uint32_t* nitems = nullptr;
  uint32_t *cnt = nullptr, *poff = nullptr;
  unsigned grid = (unsigned)nt;
  if (!p->batched) {
    int64_t S = std::min(kItemMaxSteps, std::max(kItemMinSteps, (p->n_steps + kItemTarget - 1) / kItemTarget));
    S = std::max(S, (p->n_steps + kItemsMax - 1) / kItemsMax);
    const int64_t max_items = nt + p->n_steps / S + 1;
    const int64_t max_split = 2 * (p->n_steps / S) + 1;
    const size_t b_items = (size_t)max_items * sizeof(int4), b_arr = (size_t)(nt + 1) * sizeof(uint32_t);
    FMM_TRY(p->m2l_items.ensure(b_items + 4 * b_arr + 64));
    FMM_TRY(p->m2l_partial.ensure((size_t)max_split * nrh * kN * 128 * sizeof(float)));
    uint8_t* base = p->m2l_items.as<uint8_t>();
    int4* it = reinterpret_cast<int4*>(base);
    cnt = reinterpret_cast<uint32_t*>(base + b_items);
    uint32_t* pcnt = cnt + (nt + 1);
    uint32_t* ioff = pcnt + (nt + 1);
    poff = ioff + (nt + 1);
    uint32_t* totals = poff + (nt + 1);  // [0] items, [1] partial slots
    const unsigned gt = (unsigned)((nt + T - 1) / T);
    ++g_launches;
    k_m2l_item_count<<<gt, T, 0, s>>>(p->tile_range.as<int2>(), nt, (int)S, cnt, pcnt);
    FMM_TRY(exclusive_scan_u32(cnt, ioff, nt, totals, p->scan_tmp, s));
    FMM_TRY(exclusive_scan_u32(pcnt, poff, nt, totals + 1, p->scan_tmp, s));
    ++g_launches;
    k_m2l_item_fill<<<gt, T, 0, s>>>(p->tile_range.as<int2>(), nt, (int)S, cnt, ioff, poff, it);
    FMM_CUDA_TRY(cudaGetLastError());
    items = it;
    nitems = totals;
    grid = (unsigned)max_items;
  }
  ++g_launches;
  const dim3 g3(grid, (unsigned)nrh);
  if (m2)
    k_m2l_tc<0, true><<<g3, kThreads, sh2, s>>>(p->tile_range.as<int2>(), items, nitems, p->tile_first.as<int>(),
                                                p->st_slot.as<int>(), p->st_src.as<int>(), p->Tbf.as<uint8_t>(),
                                                p->Mbf.as<uint8_t>(), p->P, nkc, nkc3, last, nrh,
                                                p->tile_cells.as<int>(), p->L.as<float>(), p->m2l_partial.as<float>(),
                                                p->flags.as<int>());
  else if (kind)
    k_m2l_tc<1, false><<<g3, kThreads, sh, s>>>(p->tile_range.as<int2>(), items, nitems, p->tile_first.as<int>(),
                                         p->st_slot.as<int>(), p->st_src.as<int>(), p->Tbf.as<uint8_t>(),
                                         p->Mbf.as<uint8_t>(), p->P, nkc, nkc3, last, nrh, p->tile_cells.as<int>(),
                                         p->L.as<float>(), p->m2l_partial.as<float>(), p->flags.as<int>());
  else
    k_m2l_tc<0, false><<<g3, kThreads, sh, s>>>(p->tile_range.as<int2>(), items, nitems, p->tile_first.as<int>(),
                                         p->st_slot.as<int>(), p->st_src.as<int>(), p->Tbf.as<uint8_t>(),
                                         p->Mbf.as<uint8_t>(), p->P, nkc, nkc3, last, nrh, p->tile_cells.as<int>(),
                                         p->L.as<float>(), p->m2l_partial.as<float>(), p->flags.as<int>());
  FMM_CUDA_TRY(cudaGetLastError());
  if (items) {
    ++g_launches;
    // a tile's D block over 8 CTAs (the split tiles are a few hundred)
    k_m2l_combine<<<dim3((unsigned)nt, 8), T, 0, s>>>(cnt, poff, p->tile_first.as<int>(), p->tile_cells.as<int>(),
                                                      p->P, nrh, p->m2l_partial.as<float>(), p->L.as<float>());
    FMM_CUDA_TRY(cudaGetLastError());
  }
  return FMM_OK;
}

}  // namespace fmm

extern "C" int fmm_selftest_bounded_wait(int64_t spins, int arrive, void* stream) {
  if (spins < 1 || spins > fmm::kSpin || (arrive != 0 && arrive != 1)) return FMM_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int* d = nullptr;
  int h = FMM_E_CUDA;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return FMM_E_NOMEM;
  ++fmm::g_launches;
  fmm::k_wait_selftest<<<1, 32, 0, s>>>((long long)spins, arrive, d);
  if (cudaGetLastError() == cudaSuccess && cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess) {
  } else {
    h = FMM_E_CUDA;
  }
  cudaFree(d);
  return h;
}
