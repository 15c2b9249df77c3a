// Device-wide primitives: exclusive scan (u32) and stable LSD radix sort.
#pragma once
#include "common.cuh"

namespace fmm {
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, DBuf& tmp,
                       cudaStream_t s);
// Exclusive scans of three arrays of length n in shared passes; total_dev[3]
// (if given) receives the three sums.  tmp holds the block sums, tmp2 the
// scratch of their scans when n exceeds 16M.
int exclusive_scan3_u32(const uint32_t* const in[3], uint32_t* const out[3], int64_t n, uint32_t* total_dev,
                        DBuf& tmp, DBuf& tmp2, cudaStream_t s);
int iota_u32(uint32_t* v, int64_t n, cudaStream_t s);
// vary: the key bits that differ between keys (if known); a pass whose 8-bit
// digit is the same in every key is the identity and is skipped.
int radix_sort_u64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int bit_begin,
                   int bit_end, int* in_second, DBuf& hist, DBuf& scan_tmp, cudaStream_t s,
                   uint64_t vary = ~0ull);
}  // namespace fmm
