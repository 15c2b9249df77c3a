// Dual-tree traversal (Sec. 3.3, Algorithms 1-2) and list grouping.
//
// Algorithm 1 pops a pair (A, B), splits the larger cell -- the larger cube,
// i.e. the coarser level; on equal cubes its ELSE branch, the source B
// (fmm_params.split_tie = FMM_SPLIT_TARGET takes A instead); the other cell
// when that one is a leaf -- and calls Algorithm 2
// on every child pair: M2L if the FMM MAC holds (R_A + R_B < theta |X_A-X_B|)
// and the pair is at least k_sigma sigma_max apart (the far field uses the
// singular kernel), else P2P if both are leaves, else push.  Here the stack
// is a breadth-first frontier processed in two passes per level (classify,
// then emit at scanned offsets) by one cooperative kernel for all levels, so
// the emitted lists have a fixed order and the host reads their sizes once.  Periodic: the traversal starts
// from (root, root + o L) for the 27 o in {-1,0,1}^3.  The MAC is evaluated
// in FP64 with explicitly rounded operations in a fixed order.
//
// Outputs: P2P entries grouped by target leaf (CSR), and M2L entries grouped
// into steps = (tile of 64 consecutive target cells of one level, translation
// key), each step carrying the source cell of every tile slot (or -1).
#include <algorithm>
#include <climits>
#include <cstring>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

struct TravArgs {
  const double* center;
  const double* radius;
  const float4* cf;  // FP32 copies of centre and radius
  const int* nchild;
  const int* child;
  const int* level;
  const int* cseg;    // batch: problem of each cell (nullptr: one problem, the scalars below)
  const SegMac* sm;   // batch: per-problem shift and MAC constants
  const int* begin;   // particle range of each cell (the leaf-pair cost rule)
  const int* end;
  long long p2p_pair_max;  // leaf pairs with n_A n_B <= this do P2P before the MAC (0: never)
  int split_tie;           // FMM_SPLIT_SOURCE / FMM_SPLIT_TARGET: the cell split on equal cubes
  double theta, ksig, smax, blen;
  float thetaf, ksf, blenf, slack0;  // slack0 = 2e-6 * (largest coordinate magnitude + box length)
};

// The MAC exactly as the oracle evaluates it: FP64, explicitly rounded, fixed order.
__device__ inline bool mac_fp64(const TravArgs& t, int a, int b, int o, double blen, double smax) {
  double sh[3] = {(double)(o / 9 - 1) * blen, (double)((o / 3) % 3 - 1) * blen, (double)(o % 3 - 1) * blen};
  double dx = __dsub_rn(t.center[3 * a], __dadd_rn(t.center[3 * b], sh[0]));
  double dy = __dsub_rn(t.center[3 * a + 1], __dadd_rn(t.center[3 * b + 1], sh[1]));
  double dz = __dsub_rn(t.center[3 * a + 2], __dadd_rn(t.center[3 * b + 2], sh[2]));
  double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double dist = __dsqrt_rn(d2);
  double sr = __dadd_rn(t.radius[a], t.radius[b]);
  return sr < __dmul_rn(t.theta, dist) && __dsub_rn(dist, sr) >= __dmul_rn(t.ksig, smax);
}

// FP32 screen with a bound on its rounding error (centres and radii rounded
// to FP32, shift, differences, square root: well below slack); only pairs
// inside the slack of a decision boundary take the FP64 test, so every
// decision equals the FP64 one.
__device__ inline int interact(const TravArgs& t, int a, int b, int o) {
  double blen = t.blen, smax = t.smax;
  float blenf = t.blenf, ksf = t.ksf, slack0 = t.slack0;
  if (t.cseg) {  // both cells belong to one problem
    const SegMac m = t.sm[t.cseg[a]];
    blen = m.blen;
    smax = m.smax;
    blenf = m.blenf;
    ksf = m.ksf;
    slack0 = m.slack0;
  }
  const bool leaves = t.nchild[a] == 0 && t.nchild[b] == 0;
  if (leaves && t.p2p_pair_max > 0 &&
      (long long)(t.end[a] - t.begin[a]) * (long long)(t.end[b] - t.begin[b]) <= t.p2p_pair_max)
    return 1;  // cost rule (Alg. 2): few particles in both, P2P whatever the MAC says
  const float4 A = t.cf[a], B = t.cf[b];
  const float sx = (float)(o / 9 - 1) * blenf, sy = (float)((o / 3) % 3 - 1) * blenf,
              sz = (float)(o % 3 - 1) * blenf;
  const float dx = A.x - (B.x + sx), dy = A.y - (B.y + sy), dz = A.z - (B.z + sz);
  const float d = sqrtf(dx * dx + dy * dy + dz * dz);
  const float sr = A.w + B.w;
  const float slack = slack0 + 1e-6f * (d + sr + ksf);
  const float v1 = t.thetaf * d - sr;  // M2L needs v1 > 0
  const float v2 = d - sr - ksf;       // and v2 >= 0
  bool m2l;
  if (v1 <= -slack || v2 <= -slack) m2l = false;
  else if (v1 > slack && v2 > slack) m2l = true;
  else m2l = mac_fp64(t, a, b, o, blen, smax);
  if (m2l) return 0;                                          // M2L
  if (leaves) return 1;                                       // P2P
  return 2;                                                   // push
}

// An M2L pair record in 8 bytes: (target, source | image << 27).  Cells are
// fewer than 2^27 (checked before the traversal) and images fewer than 32.
constexpr int kPairSrcBits = 27;
__device__ __forceinline__ int2 pack_m2l(int a, int b, int img) { return make_int2(a, b | (img << kPairSrcBits)); }
__device__ __forceinline__ int m2l_src(int2 v) { return v.y & ((1 << kPairSrcBits) - 1); }
__device__ __forceinline__ int m2l_img(int2 v) { return (int)((unsigned)v.y >> kPairSrcBits); }

// Initial pairs (root r, root r + o L) for every root (one per problem) and
// image, in (root, image) order; one CTA, order-preserving compaction.
__global__ void __launch_bounds__(1024) k_trav_init(TravArgs t, int nroot, int nimg, int img0, int4* fr, int2* m2l,
                                                    int4* p2p, uint32_t* cnt) {
  __shared__ uint32_t wsum[3][32];
  __shared__ uint32_t base[3];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < 3) base[tid] = 0;
  __syncthreads();
  const int total = nroot * nimg;
  for (int c0 = 0; c0 < total; c0 += 1024) {
    const int q = c0 + tid;
    int ty = -1;
    int4 v = make_int4(0, 0, 0, 0);
    if (q < total) {
      const int r = q / nimg, o = img0 + q % nimg;
      ty = interact(t, r, r, o);
      v = make_int4(r, r, o, 0);
    }
    uint32_t rank[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const unsigned b = __ballot_sync(0xffffffffu, ty == k);
      rank[k] = __popc(b & ((1u << lane) - 1u));
      if (lane == 0) wsum[k][w] = __popc(b);
    }
    __syncthreads();
    if (tid < 3) {  // exclusive scan of the warp totals
      uint32_t acc = base[tid];
      for (int i = 0; i < 32; ++i) {
        const uint32_t x = wsum[tid][i];
        wsum[tid][i] = acc;
        acc += x;
      }
      base[tid] = acc;
    }
    __syncthreads();
    if (ty == 0) m2l[wsum[0][w] + rank[0]] = pack_m2l(v.x, v.y, v.z);
    else if (ty == 1) p2p[wsum[1][w] + rank[1]] = v;
    else if (ty == 2) fr[wsum[2][w] + rank[2]] = v;
    __syncthreads();
  }
  if (tid < 3) cnt[tid] = base[tid];
}

__device__ inline void split_of(const TravArgs& t, int a, int b, bool& split_a, int& c0, int& nc) {
  // A's cube larger than B's <=> A on the coarser level (equal levels: split_tie)
  split_a = t.level[a] < t.level[b] || (t.split_tie == FMM_SPLIT_TARGET && t.level[a] == t.level[b]);
  if (split_a && t.nchild[a] == 0) split_a = false;
  else if (!split_a && t.nchild[b] == 0) split_a = true;
  int s = split_a ? a : b;
  c0 = t.child[s];
  nc = t.nchild[s];
}

// ---- The frontier loop as one cooperative kernel.
//
// All levels of the frontier in one launch: the blocks own contiguous ranges
// of the frontier; per level they classify their pairs (phase A), meet at a
// grid barrier, take their output offsets from the block totals and emit the
// children in item order (phase B), and meet again.  The lists come out in
// the same order as the level-by-level kernels above (item order, children in
// digit order), with no host round trip per level.  Every block is resident
// (cooperative launch); each barrier wait is bounded and gives up with
// FMM_E_TIMEOUT.  When a level's output would outgrow a buffer the blocks
// stop together before writing it and save where they are (the lists so far
// and that level's frontier stay in place); the host grows the buffers,
// keeping their contents, and relaunches the kernel, which resumes at that
// level.

constexpr int kTravThreads = 256;
constexpr int kTravMaxIter = 128;         // > 2 x the 22 levels a pair can descend
constexpr long long kGridSpin = 1ll << 24;

// state[]: 0 nm, 1 np, 2 nf, 3 overflow, 4 need_m, 5 need_p, 6 need_f, 7 iterations,
// 8 barrier arrivals, 9 barrier generation, 10 abort
struct TravState {
  uint32_t nm, np, nf, cur_b, overflow, need_m, need_p, need_f, iters, bar_count, bar_gen, abort;
};

__device__ bool grid_barrier(TravState* st, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = &st->bar_gen;
    volatile uint32_t* ab = &st->abort;
    const uint32_t g = *gen;
    __threadfence();
    if (atomicAdd(&st->bar_count, 1u) == nblocks - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      for (long long i = 0; *gen == g; ++i) {
        if (*ab) break;
        if (i > kGridSpin) {
          atomicExch(&st->abort, 1u);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ((volatile uint32_t*)&st->abort)[0] == 0u;
}

// Exclusive block scan of three counts (thread order); returns the block totals.
__device__ inline void block_scan3(uint32_t v[3], uint32_t tot[3]) {
  __shared__ uint32_t ws[3][kTravThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    inc[k] = v[k];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc[k], o);
      if (lane >= o) inc[k] += y;
    }
    if (lane == 31) ws[k][w] = inc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint32_t before = 0, all = 0;
    for (int i = 0; i < kTravThreads / 32; ++i) {
      const uint32_t x = ws[k][i];
      if (i < w) before += x;
      all += x;
    }
    v[k] = before + inc[k] - v[k];
    tot[k] = all;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kTravThreads) k_trav_loop(TravArgs t, int4* __restrict__ frA, int4* __restrict__ frB,
                                                            const uint32_t* __restrict__ cnt0, int2* __restrict__ m2l,
                                                            int4* __restrict__ p2p, uint32_t* __restrict__ mask,
                                                            uint32_t* __restrict__ blk, TravState* st, uint32_t cap_fr,
                                                            uint32_t cap_m, uint32_t cap_p, int resume) {
  __shared__ uint32_t red[3][kTravThreads / 32];
  __shared__ uint32_t bases[6];
  const unsigned G = gridDim.x, b = blockIdx.x;
  // first launch: the initial pairs of k_trav_init; a resumed launch: the saved state
  uint32_t nm = resume ? st->nm : cnt0[0], np = resume ? st->np : cnt0[1], nf = resume ? st->nf : cnt0[2];
  const bool start_b = resume && st->cur_b;
  int iter = resume ? (int)st->iters : 0;
  int4* cur = start_b ? frB : frA;
  int4* nxt = start_b ? frA : frB;
  bool stopped = false;
  for (; nf > 0 && iter < kTravMaxIter; ++iter) {
    const uint32_t chunk = (nf + G - 1) / G;
    const uint32_t i0 = min(nf, b * chunk), i1 = min(nf, i0 + chunk);
    // phase A: classify the block's pairs, block totals
    uint32_t c[3] = {0u, 0u, 0u};
    for (uint32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const int4 pr = cur[i];
      bool sa;
      int c0, ncc;
      split_of(t, pr.x, pr.y, sa, c0, ncc);
      uint32_t msk = 0;
      for (int q = 0; q < ncc; ++q) {
        const int ch = c0 + q;
        const int ty = sa ? interact(t, ch, pr.y, pr.z) : interact(t, pr.x, ch, pr.z);
        msk |= (uint32_t)ty << (2 * q);
        c[ty] += 1u;
      }
      mask[i] = msk | ((uint32_t)ncc << 16);
    }
    {
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint32_t x = c[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][w] = x;
      }
      __syncthreads();
      if (threadIdx.x < 3) {
        uint32_t x = 0;
        for (int i = 0; i < kTravThreads / 32; ++i) x += red[threadIdx.x][i];
        blk[3 * b + threadIdx.x] = x;
      }
    }
    if (!grid_barrier(st, G)) return;
    // offsets of this block (sum of the earlier blocks) and the level totals
    if (threadIdx.x < 6) bases[threadIdx.x] = 0u;
    __syncthreads();
    {
      uint32_t pre[3] = {0u, 0u, 0u}, all[3] = {0u, 0u, 0u};
      for (unsigned j = threadIdx.x; j < G; j += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const uint32_t x = ((volatile uint32_t*)blk)[3 * j + k];
          all[k] += x;
          if (j < b) pre[k] += x;
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        atomicAdd(&bases[k], pre[k]);
        atomicAdd(&bases[3 + k], all[k]);
      }
    }
    __syncthreads();
    const uint32_t tm = bases[3], tp = bases[4], tf = bases[5];
    // every block sees the same totals, so they all stop here together when a
    // buffer is too small for this level's output (nothing of it written yet)
    if ((uint64_t)nm + tm > cap_m || (uint64_t)np + tp > cap_p || tf > cap_fr) {
      if (b == 0 && threadIdx.x == 0) {
        st->overflow = 1u;
        st->need_m = nm + tm;
        st->need_p = np + tp;
        st->need_f = tf;
      }
      stopped = true;
      break;
    }
    // phase B: emit in item order
    uint32_t run[3] = {nm + bases[0], np + bases[1], bases[2]};
    for (uint32_t base = i0; base < i1; base += blockDim.x) {
      const uint32_t i = base + threadIdx.x;
      uint32_t msk = 0, ncc = 0;
      uint32_t v[3] = {0u, 0u, 0u};
      if (i < i1) {
        msk = mask[i];
        ncc = msk >> 16;
        for (uint32_t q = 0; q < ncc; ++q) v[(msk >> (2 * q)) & 3u] += 1u;
      }
      uint32_t tot[3];
      block_scan3(v, tot);
      if (i < i1) {
        const int4 pr = cur[i];
        bool sa;
        int c0, ncn;
        split_of(t, pr.x, pr.y, sa, c0, ncn);
        uint32_t im = run[0] + v[0], ip = run[1] + v[1], iff = run[2] + v[2];
        for (uint32_t q = 0; q < ncc; ++q) {
          const int ch = c0 + (int)q;
          const int4 val = sa ? make_int4(ch, pr.y, pr.z, 0) : make_int4(pr.x, ch, pr.z, 0);
          const uint32_t ty = (msk >> (2 * q)) & 3u;
          if (ty == 0) m2l[im++] = pack_m2l(val.x, val.y, val.z);
          else if (ty == 1) p2p[ip++] = val;
          else nxt[iff++] = val;
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) run[k] += tot[k];
    }
    nm += tm;
    np += tp;
    nf = tf;
    int4* sw = cur;
    cur = nxt;
    nxt = sw;
    if (!grid_barrier(st, G)) return;
  }
  if (b == 0 && threadIdx.x == 0) {  // where the lists stand (and, if stopped, where to resume)
    st->nm = nm;
    st->np = np;
    st->nf = nf;
    st->cur_b = cur == frB ? 1u : 0u;
    st->iters = (uint32_t)iter;
    if (!stopped) st->overflow = 0u;
  }
}

// ---- P2P CSR

__global__ void k_p2p_keys(const int4* __restrict__ raw, int n, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = (uint64_t)raw[i].x;
  vals[i] = (uint32_t)i;
}

__global__ void k_p2p_gather(const int4* __restrict__ raw, const uint32_t* __restrict__ order, int n,
                             int2* __restrict__ out, const int* __restrict__ begin, const int* __restrict__ end,
                             unsigned long long* __restrict__ pairs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt = 0;
  if (i < n) {
    int4 v = raw[order[i]];
    out[i] = make_int2(v.y, v.z);
    cnt = (unsigned long long)(end[v.x] - begin[v.x]) * (unsigned long long)(end[v.y] - begin[v.y]);
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(pairs, cnt);
}

__device__ inline int lower_bound_key(const uint64_t* a, int n, uint64_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void k_p2p_offsets(const int* __restrict__ leaves, int nl, const uint64_t* __restrict__ skeys, int n,
                              int2* __restrict__ off) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  uint64_t a = (uint64_t)leaves[i];
  off[i] = make_int2(lower_bound_key(skeys, n, a), lower_bound_key(skeys, n, a + 1));
}

// ---- M2L steps

// Integer cell coordinates of a level-l cell (the bits above 3l hold the problem).
__device__ inline void cell_ijk(uint64_t key, int l, long long ijk[3]) {
  uint64_t k = key & ((1ull << (3 * l)) - 1ull);
  long long r[3] = {0, 0, 0};
  for (int b = 0; b < kMaxLevel; ++b) {
    r[0] |= (long long)((k >> (3 * b + 2)) & 1ull) << b;
    r[1] |= (long long)((k >> (3 * b + 1)) & 1ull) << b;
    r[2] |= (long long)((k >> (3 * b)) & 1ull) << b;
  }
  ijk[0] = r[0];
  ijk[1] = r[1];
  ijk[2] = r[2];
}

// Integer coordinates of every cell, 21 bits each (x | y << 21 | z << 42).
__global__ void k_cell_ijk(const int* __restrict__ level, const uint64_t* __restrict__ ckey, int nc,
                           uint64_t* __restrict__ ijk) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  long long r[3];
  cell_ijk(ckey[c], level[c], r);
  ijk[c] = (uint64_t)r[0] | ((uint64_t)r[1] << 21) | ((uint64_t)r[2] << 42);
}

// Translation key of every M2L pair, and the field ranges of the keys
// (delta, tx, ty, tz; min and max in rng[2q], rng[2q + 1]) for their compact
// encoding.
__global__ void k_m2l_keys(const int2* __restrict__ raw, int n, const int* __restrict__ level,
                           const uint64_t* __restrict__ cijk, uint64_t* __restrict__ keys, int* __restrict__ rng,
                           int* __restrict__ flag) {
  int lo[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX}, hi[4] = {INT_MIN, INT_MIN, INT_MIN, INT_MIN};
  // grid-stride over the pairs: few blocks, so few atomics on the 8 range words
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int2 pr = raw[i];
    const int va = pr.x, vb = m2l_src(pr), vz = m2l_img(pr);
    int la = level[va], lb = level[vb];
    int lf = la > lb ? la : lb;
    const uint64_t pa = cijk[va], pb = cijk[vb];
    const long long ia[3] = {(long long)(pa & 0x1FFFFFull), (long long)((pa >> 21) & 0x1FFFFFull),
                             (long long)(pa >> 42)};
    const long long ib[3] = {(long long)(pb & 0x1FFFFFull), (long long)((pb >> 21) & 0x1FFFFFull),
                             (long long)(pb >> 42)};
    int o[3] = {vz / 9 - 1, (vz / 3) % 3 - 1, vz % 3 - 1};
    long long t[3];
    bool ok = true;
    for (int q = 0; q < 3; ++q) {
      t[q] = (2 * ia[q] + 1) * (1ll << (lf - la)) - (2 * ib[q] + 1) * (1ll << (lf - lb)) -
             (long long)o[q] * (1ll << (lf + 1));
      if (t[q] > kKeyLim || t[q] < -kKeyLim) ok = false;
    }
    if (!ok) atomicExch(flag, FMM_E_DEPTH);
    const uint64_t k = m2l_key_encode(la - lb, t[0], t[1], t[2]);
    keys[i] = k;
    const int f[4] = {(int)(k >> 57) - 32, (int)key_field(k, 38), (int)key_field(k, 19), (int)key_field(k, 0)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lo[q] = min(lo[q], f[q]);
      hi[q] = max(hi[q], f[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = min(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = max(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
  }
  __shared__ int slo[4][32], shi[4][32];
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 4; ++q) {
      slo[q][w] = lo[q];
      shi[q][w] = hi[q];
    }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    int l = INT_MAX, h = INT_MIN;
    for (int k = 0; k < nw; ++k) {
      l = min(l, slo[q][k]);
      h = max(h, shi[q][k]);
    }
    if (l <= h) {
      atomicMin(&rng[2 * q], l);
      atomicMax(&rng[2 * q + 1], h);
    }
  }
}

// Limits of the binned step build: compact keys of at most 22 bits (a 16 MB
// flag table) and at most 2^28 (tile, translation) bins (two 1 GB tables;
// 512^3 blobs need ~1.2e8); beyond either the steps come from the sort.
constexpr int kBinKeyBits = 22;
constexpr int64_t kBinMax = 1ll << 28;

struct KeyPack {
  int lo[4];
  int shift[4];  // bit position of each field in the compact key
  int width[4];  // bits of each field
  int bits;      // total compact key bits
};

__device__ inline uint64_t compact_key(uint64_t k, const KeyPack& kp) {
  const int f[4] = {(int)(k >> 57) - 32, (int)key_field(k, 38), (int)key_field(k, 19), (int)key_field(k, 0)};
  uint64_t c = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) c |= (uint64_t)(f[q] - kp.lo[q]) << kp.shift[q];
  return c;
}

// (tile, compact key) sort keys of the M2L pairs: a run of equal keys is one
// step.  A target has at most one source per translation, so the pairs of a
// step have distinct slots and their order within the run does not matter.
__global__ void k_step_keys2(const int2* __restrict__ raw, const uint64_t* __restrict__ fkeys, int n,
                             const int* __restrict__ ctile, KeyPack kp, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t tile = (uint64_t)(ctile[raw[i].x] / kTile);
  keys[i] = (tile << kp.bits) | compact_key(fkeys[i], kp);
  vals[i] = (uint32_t)i;
}

// Binned step build.  With K = 2^bits compact keys, the translations present
// are flagged in a K-table; its scan numbers them in compact-key order (the
// operator slots).  The (tile, slot) bins present are flagged in a second
// table, whose scan numbers the steps in (tile, compact key) order: the same
// steps, slots and order as the sort of k_step_keys2.
__global__ void k_key_mark(const uint64_t* __restrict__ fkeys, int n, KeyPack kp, uint32_t* __restrict__ kflag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) kflag[compact_key(fkeys[i], kp)] = 1u;
}

// Slot of every flagged compact key -> its full translation key.
__global__ void k_key_unpack(const uint32_t* __restrict__ kflag, const uint32_t* __restrict__ kslot, int64_t K,
                             KeyPack kp, uint64_t* __restrict__ ukeys) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K || !kflag[c]) return;
  int f[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) f[q] = (int)((c >> kp.shift[q]) & ((1ll << kp.width[q]) - 1)) + kp.lo[q];
  ukeys[kslot[c]] = m2l_key_encode(f[0], f[1], f[2], f[3]);
}

// bin of pair i = tile * nkeys + slot; flags the bin and keeps it per pair.
__global__ void k_bin_mark(const int2* __restrict__ raw, const uint64_t* __restrict__ fkeys, int n,
                           const int* __restrict__ ctile, KeyPack kp, const uint32_t* __restrict__ kslot, int nkeys,
                           uint32_t* __restrict__ bflag, uint32_t* __restrict__ pbin) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t b = (uint32_t)(ctile[raw[i].x] / kTile) * (uint32_t)nkeys + kslot[compact_key(fkeys[i], kp)];
  bflag[b] = 1u;
  pbin[i] = b;
}

__global__ void k_bin_steps(const uint32_t* __restrict__ bflag, const uint32_t* __restrict__ bstep, int64_t nb,
                            int nkeys, int* __restrict__ st_tile, int* __restrict__ st_slot) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !bflag[b]) return;
  st_tile[bstep[b]] = (int)(b / nkeys);
  st_slot[bstep[b]] = (int)(b % nkeys);
}

__global__ void k_bin_fill(const int2* __restrict__ raw, const uint32_t* __restrict__ pbin, int n,
                           const uint32_t* __restrict__ bstep, const int* __restrict__ ctile,
                           int* __restrict__ st_src) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int2 v = raw[i];
  st_src[(size_t)bstep[pbin[i]] * kTile + (ctile[v.x] % kTile)] = m2l_src(v);
}

__global__ void k_step_write2(const uint64_t* __restrict__ k, const uint32_t* __restrict__ idx, int n,
                              const uint32_t* __restrict__ f, const uint32_t* __restrict__ e,
                              const int2* __restrict__ raw, const uint64_t* __restrict__ fkeys,
                              const int* __restrict__ ctile, int kbits, int* __restrict__ st_tile,
                              uint64_t* __restrict__ st_ckey, uint64_t* __restrict__ st_fkey,
                              int* __restrict__ st_src) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t s = e[i] + f[i] - 1u;
  const uint64_t key = k[i];
  if (f[i]) {
    st_tile[s] = (int)(key >> kbits);
    st_ckey[s] = key & ((1ull << kbits) - 1ull);
    st_fkey[s] = fkeys[idx[i]];
  }
  const int2 v = raw[idx[i]];
  st_src[(size_t)s * kTile + (ctile[v.x] % kTile)] = m2l_src(v);
}

__global__ void k_step_slots(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sidx, int ns,
                             const uint32_t* __restrict__ f, const uint32_t* __restrict__ e,
                             const uint64_t* __restrict__ st_fkey, uint64_t* __restrict__ ukeys,
                             int* __restrict__ st_slot) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  const uint32_t slot = e[i] + f[i] - 1u;
  if (f[i]) ukeys[slot] = st_fkey[sidx[i]];
  st_slot[sidx[i]] = (int)slot;
}

__global__ void k_copy_u64_iota(const uint64_t* __restrict__ in, int n, uint64_t* __restrict__ out,
                                uint32_t* __restrict__ idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    out[i] = in[i];
    idx[i] = (uint32_t)i;
  }
}

__global__ void k_unique_flags(const uint64_t* __restrict__ k, int n, uint32_t* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

// Tiles group the cells of one level and one child octant (in Morton order),
// at most 64 per tile: cells at the same octant position have the same
// relative interaction lists in a uniform region, so a tile's steps are
// nearly full; a tile never mixes octants, so a coarse level is split into
// its octants instead of one long tile.
__global__ void k_tile_order_keys(const int* __restrict__ level, const uint64_t* __restrict__ ckey, int nc,
                                  uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                  int* __restrict__ gcount) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int oct = (int)(ckey[c] & 7ull);
  // the sort is stable, so cells of a group keep their (Morton) index order
  keys[c] = ((uint64_t)level[c] << 3) | (uint64_t)oct;
  vals[c] = (uint32_t)c;
  atomicAdd(&gcount[level[c] * 8 + oct], 1);
}

// gofs[g] = first sorted position of (level, octant) group g, gtile[g] = its
// first tile.
__global__ void k_cell_tiles(int nc, int ntiles, const uint32_t* __restrict__ order, const int* __restrict__ level,
                             const uint64_t* __restrict__ ckey, const int* __restrict__ gofs,
                             const int* __restrict__ gtile, int* __restrict__ ctile, int* __restrict__ tcell,
                             int* __restrict__ tfirst) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nc) return;
  const int c = (int)order[q];
  const int g = level[c] * 8 + (int)(ckey[c] & 7ull);
  const int r = q - gofs[g];
  const int t = gtile[g] + r / kTile;
  ctile[c] = t * kTile + r % kTile;
  tcell[q] = c;
  if (r % kTile == 0) tfirst[t] = q;
  if (q == 0) tfirst[ntiles] = nc;
}

__global__ void k_step_flags(const uint64_t* __restrict__ k, int n, uint32_t* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void k_tile_ranges(const int* __restrict__ st_tile, int ns, int2* __restrict__ tr) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  int t = st_tile[s];
  if (s == 0 || st_tile[s - 1] != t) tr[t].x = s;
  if (s == ns - 1 || st_tile[s + 1] != t) tr[t].y = s + 1;
}

// Per-problem constants of a batch, with the arithmetic of the one-problem
// path: MAC slack and near-field class margin 2e-6 (largest |coordinate| of
// the cube + side), k_sigma sigma_max, image shift = side (periodic only).
__global__ void k_seg_tables(int nseg, const double* __restrict__ box, const unsigned int* __restrict__ smax_bits,
                             const float* __restrict__ sig, double ksig, int periodic, SegMac* __restrict__ mac,
                             SegP2P* __restrict__ pp) {
  const int sg = blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  const double* b = box + 4 * sg;
  double cmax = 0.0;
  for (int q = 0; q < 3; ++q) cmax = fmax(cmax, fmax(fabs(b[q]), fabs(__dadd_rn(b[q], b[3]))));
  const double margin = __dmul_rn(2e-6, __dadd_rn(cmax, b[3]));
  const double smax = (double)__uint_as_float(smax_bits[sg]);
  const double blen = periodic ? b[3] : 0.0;
  SegMac m;
  m.blen = blen;
  m.smax = smax;
  m.blenf = (float)blen;
  m.ksf = (float)__dmul_rn(ksig, smax);
  m.slack0 = (float)margin;
  m.pad = 0.f;
  mac[sg] = m;
  SegP2P q;
  q.sigma = sig ? sig[sg] : 1.f;
  q.smax = (float)smax;
  q.blen = (float)blen;
  q.margin = (float)margin;
  q.dip[0] = q.dip[1] = q.dip[2] = 0.f;
  q.pad = 0.f;
  pp[sg] = q;
}

int bits_for(int64_t v) {
  int b = 1;
  while (b < 63 && (1ll << b) <= v) ++b;
  return (b + 7) / 8 * 8;
}

}  // namespace

int segment_tables(fmm_plan p, int per_particle_sigma, cudaStream_t s) {
  const int S = p->nseg;
  ++g_launches;
  k_seg_tables<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(
      S, p->seg_box.as<double>(), p->seg_smax.as<unsigned int>(), per_particle_sigma ? nullptr : p->seg_sig.as<float>(),
      (double)p->prm.sigma_sep, p->prm.periodic, p->seg_mac.as<SegMac>(), p->seg_p2p.as<SegP2P>());
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

int traverse(fmm_plan p, double smax, cudaStream_t s) {
  const int T = 256;
  const int nc = (int)p->ncells;
  if (p->ncells >= (1ll << kPairSrcBits)) return FMM_E_CAPACITY;  // the 8-byte M2L pair record
  TravArgs ta;
  ta.center = p->c_center.as<double>();
  ta.radius = p->c_radius.as<double>();
  ta.cf = p->c_cf.as<float4>();
  ta.nchild = p->c_nchild.as<int>();
  ta.begin = p->c_begin.as<int>();
  ta.end = p->c_end.as<int>();
  ta.p2p_pair_max = p->prm.p2p_pair_max;
  ta.split_tie = p->prm.split_tie;
  ta.child = p->c_child.as<int>();
  ta.level = p->c_level.as<int>();
  ta.cseg = nullptr;
  ta.sm = nullptr;
  ta.theta = (double)p->prm.theta;
  ta.ksig = (double)p->prm.sigma_sep;
  ta.smax = smax;
  ta.blen = p->prm.periodic ? p->prm.box_len : 0.0;
  ta.thetaf = (float)ta.theta;
  if (p->batched) {
    ta.cseg = p->c_seg.as<int>();
    ta.sm = p->seg_mac.as<SegMac>();
    ta.ksf = ta.blenf = ta.slack0 = 0.f;
  } else {
    double hbox[4];
    FMM_CUDA_TRY(cudaMemcpyAsync(hbox, p->scal.as<double>() + kScalBox, sizeof(hbox), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    double cmax = 0.0;
    for (int q = 0; q < 3; ++q) cmax = std::max(cmax, std::max(std::fabs(hbox[q]), std::fabs(hbox[q] + hbox[3])));
    ta.ksf = (float)(ta.ksig * ta.smax);
    ta.blenf = (float)ta.blen;
    ta.slack0 = (float)(2e-6 * (cmax + hbox[3]));
    p->cf_margin = 2e-6 * (cmax + hbox[3]);
  }
  const int nimg = p->prm.periodic ? 27 : 1;
  const int img0 = p->prm.periodic ? 0 : kImageZero;
  uint32_t* hc = reinterpret_cast<uint32_t*>(p->pinned);
  uint32_t* dcnt = reinterpret_cast<uint32_t*>(p->scal.as<double>() + kScalCount);

  // Frontier loop: one cooperative launch for all levels; the host reads the
  // list sizes once.  A launch that stops because a buffer is too small is
  // resumed after the buffers grew (their contents kept).
  // Starting capacities: from the cell count, at least what the plan's
  // earlier evaluations needed (so a plan that saw its problem once runs one
  // launch).
  int64_t cap_fr = p->cap_fr0 > 0 ? p->cap_fr0 : std::max<int64_t>({1024, 16 * (int64_t)nc, p->hw_fr});
  int64_t cap_m = p->cap_m0 > 0 ? p->cap_m0 : std::max<int64_t>({1024, 64 * (int64_t)nc, p->hw_m});
  int64_t cap_p = p->cap_p0 > 0 ? p->cap_p0 : std::max<int64_t>({1024, 32 * (int64_t)nc, p->hw_p});
  // the initial pairs (one per root and image) always fit
  const int64_t ninit = (int64_t)(p->batched ? p->nseg : 1) * nimg;
  cap_fr = std::max(cap_fr, ninit);
  cap_m = std::max(cap_m, ninit);
  cap_p = std::max(cap_p, ninit);
  static int grid_blocks[64] = {0};
  const int dev = p->device >= 0 && p->device < 64 ? p->device : 0;
  if (!grid_blocks[dev]) {
    int sms = 0, per_sm = 0;
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trav_loop, kTravThreads, 0));
    grid_blocks[dev] = std::max(1, sms * std::min(per_sm, 4));
  }
  const unsigned G = (unsigned)grid_blocks[dev];
  FMM_TRY(p->fr0.ensure(cap_fr * sizeof(int4)));
  FMM_TRY(p->fr1.ensure(cap_fr * sizeof(int4)));
  FMM_TRY(p->m2l_raw.ensure(cap_m * sizeof(int2)));
  FMM_TRY(p->p2p_raw.ensure(cap_p * sizeof(int4)));
  FMM_TRY(p->tmask.ensure(cap_fr * sizeof(uint32_t)));
  FMM_TRY(p->tscan0.ensure((size_t)(3 * G + 8) * sizeof(uint32_t)));
  FMM_TRY(p->tscan1.ensure(sizeof(TravState) + 64));
  TravState* dst = p->tscan1.as<TravState>();
  FMM_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(TravState), s));
  ++g_launches;
  k_trav_init<<<1, 1024, 0, s>>>(ta, p->batched ? p->nseg : 1, nimg, img0, p->fr0.as<int4>(), p->m2l_raw.as<int2>(),
                                 p->p2p_raw.as<int4>(), dcnt);
  int64_t nm = 0, np = 0;
  for (int launch = 0;; ++launch) {
    p->trav_runs = launch + 1;
    if (launch > 64) return FMM_E_CAPACITY;
    int4* a0 = p->fr0.as<int4>();
    int4* a1 = p->fr1.as<int4>();
    int2* am = p->m2l_raw.as<int2>();
    int4* ap = p->p2p_raw.as<int4>();
    uint32_t* msk = p->tmask.as<uint32_t>();
    uint32_t* blk = p->tscan0.as<uint32_t>();
    uint32_t cf = (uint32_t)cap_fr, cm = (uint32_t)cap_m, cp = (uint32_t)cap_p;
    int resume = launch > 0 ? 1 : 0;
    void* args[] = {&ta, &a0, &a1, &dcnt, &am, &ap, &msk, &blk, &dst, &cf, &cm, &cp, &resume};
    ++g_launches;
    FMM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_trav_loop, dim3(G), dim3(kTravThreads), args, 0, s));
    TravState hs;
    FMM_CUDA_TRY(cudaMemcpyAsync(hc, dst, sizeof(TravState), cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    memcpy(&hs, hc, sizeof(TravState));
    if (hs.abort) return FMM_E_TIMEOUT;
    if (hs.overflow) {  // grow what was too small (x1.25, contents kept) and resume
      if ((int64_t)hs.need_m > cap_m) cap_m = (int64_t)hs.need_m + hs.need_m / 4 + 1024;
      if ((int64_t)hs.need_p > cap_p) cap_p = (int64_t)hs.need_p + hs.need_p / 4 + 1024;
      if ((int64_t)hs.need_f > cap_fr) cap_fr = (int64_t)hs.need_f + hs.need_f / 4 + 1024;
      if (cap_fr > 0x7fffffff || cap_m > 0x7fffffff || cap_p > 0x7fffffff) return FMM_E_CAPACITY;
      FMM_TRY(p->m2l_raw.grow_copy(cap_m * sizeof(int2), s));
      FMM_TRY(p->p2p_raw.grow_copy(cap_p * sizeof(int4), s));
      FMM_TRY(p->fr0.grow_copy(cap_fr * sizeof(int4), s));
      FMM_TRY(p->fr1.grow_copy(cap_fr * sizeof(int4), s));
      FMM_TRY(p->tmask.ensure(cap_fr * sizeof(uint32_t)));
      FMM_CUDA_TRY(cudaMemsetAsync(&dst->overflow, 0, sizeof(uint32_t), s));
      continue;
    }
    if (hs.nf != 0) return FMM_E_CAPACITY;  // deeper than kTravMaxIter levels of the frontier
    nm = hs.nm;
    np = hs.np;
    break;
  }
  p->hw_m = std::max<int64_t>(p->hw_m, nm + nm / 8);
  p->hw_p = std::max<int64_t>(p->hw_p, np + np / 8);
  p->hw_fr = std::max<int64_t>(p->hw_fr, cap_fr);
  p->n_m2l = nm;
  p->n_p2p = np;

  // ---- P2P: group by target leaf
  {
    const int n = (int)np;
    FMM_TRY(p->lk0.ensure((n + 1) * sizeof(uint64_t)));
    FMM_TRY(p->lk1.ensure((n + 1) * sizeof(uint64_t)));
    FMM_TRY(p->lv0.ensure((n + 1) * sizeof(uint32_t)));
    FMM_TRY(p->lv1.ensure((n + 1) * sizeof(uint32_t)));
    FMM_TRY(p->p2p_sorted.ensure((n + 1) * sizeof(int2)));
    FMM_TRY(p->p2p_off.ensure((p->nleaves + 1) * sizeof(int2)));
    unsigned g = (unsigned)((n + T - 1) / T);
    ++g_launches;
    k_p2p_keys<<<g, T, 0, s>>>(p->p2p_raw.as<int4>(), n, p->lk0.as<uint64_t>(), p->lv0.as<uint32_t>());
    int second = 0;
    FMM_TRY(radix_sort_u64(p->lk0.as<uint64_t>(), p->lv0.as<uint32_t>(), p->lk1.as<uint64_t>(),
                           p->lv1.as<uint32_t>(), n, 0, bits_for(nc), &second, p->sort_hist, p->scan_tmp, s));
    uint64_t* sk = second ? p->lk1.as<uint64_t>() : p->lk0.as<uint64_t>();
    uint32_t* sv = second ? p->lv1.as<uint32_t>() : p->lv0.as<uint32_t>();
    unsigned long long* dpairs = reinterpret_cast<unsigned long long*>(p->scal.as<double>() + kScalCount + 2);
    FMM_CUDA_TRY(cudaMemsetAsync(dpairs, 0, sizeof(unsigned long long), s));
    ++g_launches;
    k_p2p_gather<<<g, T, 0, s>>>(p->p2p_raw.as<int4>(), sv, n, p->p2p_sorted.as<int2>(), p->c_begin.as<int>(),
                                 p->c_end.as<int>(), dpairs);
    ++g_launches;
    k_p2p_offsets<<<(unsigned)((p->nleaves + T - 1) / T), T, 0, s>>>(p->leaves.as<int>(), (int)p->nleaves, sk, n,
                                                                     p->p2p_off.as<int2>());
    FMM_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(p->pinned) + 64, dpairs, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
  }

  // ---- M2L: keys, unique operators, steps per (tile, key)
  {
    const int n = (int)nm;
    // tiles: at most 64 cells of one (level, octant) group each
    constexpr int kGroups = (kMaxLevel + 1) * 8;
    FMM_TRY(p->c_tile.ensure((nc + 1) * sizeof(int)));
    FMM_TRY(p->tile_cells.ensure((nc + 1) * sizeof(int)));
    FMM_TRY(p->tile_groups.ensure(3 * kGroups * sizeof(int)));
    FMM_TRY(p->lk0.ensure((nc + 1) * sizeof(uint64_t)));
    FMM_TRY(p->lk1.ensure((nc + 1) * sizeof(uint64_t)));
    FMM_TRY(p->lv0.ensure((nc + 1) * sizeof(uint32_t)));
    FMM_TRY(p->lv1.ensure((nc + 1) * sizeof(uint32_t)));
    {
      int* gcount = p->tile_groups.as<int>();
      int* gofs = gcount + kGroups;
      int* gtile = gofs + kGroups;
      FMM_CUDA_TRY(cudaMemsetAsync(gcount, 0, kGroups * sizeof(int), s));
      unsigned gc = (unsigned)((nc + T - 1) / T);
      ++g_launches;
      k_tile_order_keys<<<gc, T, 0, s>>>(p->c_level.as<int>(), p->c_key.as<uint64_t>(), nc, p->lk0.as<uint64_t>(),
                                         p->lv0.as<uint32_t>(), gcount);
      int second = 0;
      FMM_TRY(radix_sort_u64(p->lk0.as<uint64_t>(), p->lv0.as<uint32_t>(), p->lk1.as<uint64_t>(),
                             p->lv1.as<uint32_t>(), nc, 0, 8, &second, p->sort_hist, p->scan_tmp, s));
      uint32_t* ord = second ? p->lv1.as<uint32_t>() : p->lv0.as<uint32_t>();
      int* hg = reinterpret_cast<int*>(reinterpret_cast<char*>(p->pinned) + 1024);  // counts, then offsets
      FMM_CUDA_TRY(cudaMemcpyAsync(hg, gcount, kGroups * sizeof(int), cudaMemcpyDeviceToHost, s));
      FMM_CUDA_TRY(cudaStreamSynchronize(s));
      int* hofs = hg + kGroups;
      int* htile = hofs + kGroups;
      int cells = 0, tiles = 0;
      for (int g = 0; g < kGroups; ++g) {
        hofs[g] = cells;
        htile[g] = tiles;
        cells += hg[g];
        tiles += (hg[g] + kTile - 1) / kTile;
      }
      p->ntiles = tiles;
      FMM_CUDA_TRY(cudaMemcpyAsync(gofs, hofs, 2 * kGroups * sizeof(int), cudaMemcpyHostToDevice, s));
      FMM_TRY(p->tile_first.ensure((p->ntiles + 1) * sizeof(int)));
      ++g_launches;
      k_cell_tiles<<<gc, T, 0, s>>>(nc, (int)p->ntiles, ord, p->c_level.as<int>(), p->c_key.as<uint64_t>(), gofs,
                                    gtile, p->c_tile.as<int>(), p->tile_cells.as<int>(), p->tile_first.as<int>());
    }
    FMM_TRY(p->tile_range.ensure((p->ntiles + 1) * sizeof(int2)));
    FMM_CUDA_TRY(cudaMemsetAsync(p->tile_range.ptr, 0, (p->ntiles + 1) * sizeof(int2), s));
    p->n_keys = 0;
    p->n_steps = 0;
    if (n > 0) {
      FMM_TRY(p->lk0.ensure((n + 1) * sizeof(uint64_t)));
      FMM_TRY(p->lk1.ensure((n + 1) * sizeof(uint64_t)));
      FMM_TRY(p->lv0.ensure((n + 1) * sizeof(uint32_t)));
      FMM_TRY(p->lv1.ensure((n + 1) * sizeof(uint32_t)));
      FMM_TRY(p->m2l_key.ensure((n + 1) * sizeof(uint64_t)));
      FMM_TRY(p->tcount.ensure((n + 1) * sizeof(uint32_t)));
      FMM_TRY(p->tscan0.ensure((n + 1) * sizeof(uint32_t)));
      unsigned g = (unsigned)((n + T - 1) / T);
      int* flag = p->flags.as<int>();
      // 1. full translation keys and their field ranges
      ++g_launches;
      FMM_TRY(p->c_ijk.ensure((size_t)(nc + 1) * sizeof(uint64_t)));
      ++g_launches;
      k_cell_ijk<<<(unsigned)((nc + T - 1) / T), T, 0, s>>>(p->c_level.as<int>(), p->c_key.as<uint64_t>(), nc,
                                                           p->c_ijk.as<uint64_t>());
      int* drng = reinterpret_cast<int*>(p->scal.as<double>() + kScalCount + 8);
      const int init[8] = {INT_MAX, INT_MIN, INT_MAX, INT_MIN, INT_MAX, INT_MIN, INT_MAX, INT_MIN};
      int* hr = reinterpret_cast<int*>(reinterpret_cast<char*>(p->pinned) + 256);
      memcpy(hr, init, sizeof(init));
      FMM_CUDA_TRY(cudaMemcpyAsync(drng, hr, sizeof(init), cudaMemcpyHostToDevice, s));
      k_m2l_keys<<<std::min<unsigned>(g, 2048u), T, 0, s>>>(p->m2l_raw.as<int2>(), n, p->c_level.as<int>(),
                                                            p->c_ijk.as<uint64_t>(), p->m2l_key.as<uint64_t>(), drng,
                                                            flag);
      FMM_CUDA_TRY(cudaMemcpyAsync(hr, drng, sizeof(init), cudaMemcpyDeviceToHost, s));
      FMM_CUDA_TRY(cudaStreamSynchronize(s));
      KeyPack kp;
      int sh = 0;
      for (int q = 3; q >= 0; --q) {
        kp.lo[q] = hr[2 * q];
        int range = hr[2 * q + 1] - hr[2 * q];
        int b = 0;
        while ((1ll << b) <= (long long)range) ++b;
        kp.shift[q] = sh;
        kp.width[q] = b;
        sh += b;
      }
      kp.bits = sh;
      int tb = 1;
      while ((1ll << tb) < (long long)p->ntiles) ++tb;
      if (tb + kp.bits > 63) return FMM_E_DEPTH;
      const int64_t K = 1ll << kp.bits;
      bool binned = false;
      if (kp.bits <= kBinKeyBits && !(p->prm.m2l_mode & FMM_M2L_SORT_STEPS)) {
        // 2'. the steps from flag tables (no sort) when the tables are small
        FMM_TRY(p->bin_flag.ensure((size_t)(K + 1) * sizeof(uint32_t)));
        FMM_TRY(p->bin_scan.ensure((size_t)(K + 1) * sizeof(uint32_t)));
        uint32_t* kflag = p->bin_flag.as<uint32_t>();
        uint32_t* kslot = p->bin_scan.as<uint32_t>();
        FMM_CUDA_TRY(cudaMemsetAsync(kflag, 0, (size_t)K * sizeof(uint32_t), s));
        ++g_launches;
        k_key_mark<<<g, T, 0, s>>>(p->m2l_key.as<uint64_t>(), n, kp, kflag);
        FMM_TRY(exclusive_scan_u32(kflag, kslot, K, dcnt, p->scan_tmp, s));
        FMM_CUDA_TRY(cudaMemcpyAsync(hc, dcnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t nkeys = hc[0];
        const int64_t nb = nkeys * (int64_t)p->ntiles;
        if (nb <= kBinMax) {
          binned = true;
          p->n_keys = nkeys;
          FMM_TRY(p->ukeys.ensure((size_t)(nkeys + 1) * sizeof(uint64_t)));
          ++g_launches;
          k_key_unpack<<<(unsigned)((K + T - 1) / T), T, 0, s>>>(kflag, kslot, K, kp, p->ukeys.as<uint64_t>());
          // the key tables stay live: bins go to bin_flag2 / bin_scan2
          FMM_TRY(p->bin_flag2.ensure((size_t)(nb + 1) * sizeof(uint32_t)));
          FMM_TRY(p->bin_scan2.ensure((size_t)(nb + 1) * sizeof(uint32_t)));
          uint32_t* bflag = p->bin_flag2.as<uint32_t>();
          uint32_t* bstep = p->bin_scan2.as<uint32_t>();
          uint32_t* pbin = p->lv0.as<uint32_t>();
          FMM_CUDA_TRY(cudaMemsetAsync(bflag, 0, (size_t)nb * sizeof(uint32_t), s));
          ++g_launches;
          k_bin_mark<<<g, T, 0, s>>>(p->m2l_raw.as<int2>(), p->m2l_key.as<uint64_t>(), n, p->c_tile.as<int>(), kp,
                                     kslot, (int)nkeys, bflag, pbin);
          FMM_TRY(exclusive_scan_u32(bflag, bstep, nb, dcnt, p->scan_tmp, s));
          FMM_CUDA_TRY(cudaMemcpyAsync(hc, dcnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
          FMM_CUDA_TRY(cudaStreamSynchronize(s));
          p->n_steps = hc[0];
          const int64_t ns = p->n_steps;
          FMM_TRY(p->st_tile.ensure((ns + 1) * sizeof(int)));
          FMM_TRY(p->st_slot.ensure((ns + 1) * sizeof(int)));
          FMM_TRY(p->st_src.ensure((ns + 1) * kTile * sizeof(int)));
          FMM_CUDA_TRY(cudaMemsetAsync(p->st_src.ptr, 0xff, (ns + 1) * kTile * sizeof(int), s));
          ++g_launches;
          k_bin_steps<<<(unsigned)((nb + T - 1) / T), T, 0, s>>>(bflag, bstep, nb, (int)nkeys, p->st_tile.as<int>(),
                                                                 p->st_slot.as<int>());
          ++g_launches;
          k_bin_fill<<<g, T, 0, s>>>(p->m2l_raw.as<int2>(), pbin, n, bstep, p->c_tile.as<int>(),
                                     p->st_src.as<int>());
          ++g_launches;
          k_tile_ranges<<<(unsigned)((ns + T - 1) / T), T, 0, s>>>(p->st_tile.as<int>(), (int)ns,
                                                                  p->tile_range.as<int2>());
          FMM_CUDA_TRY(cudaGetLastError());
        }
      }
      if (!binned) {
        // 2. sort pairs by (tile, compact key): consecutive runs are the steps
        ++g_launches;
        k_step_keys2<<<g, T, 0, s>>>(p->m2l_raw.as<int2>(), p->m2l_key.as<uint64_t>(), n, p->c_tile.as<int>(), kp,
                                     p->lk0.as<uint64_t>(), p->lv0.as<uint32_t>());
        int second = 0;
        FMM_TRY(radix_sort_u64(p->lk0.as<uint64_t>(), p->lv0.as<uint32_t>(), p->lk1.as<uint64_t>(),
                               p->lv1.as<uint32_t>(), n, 0, tb + kp.bits, &second, p->sort_hist, p->scan_tmp, s));
        uint64_t* sk = second ? p->lk1.as<uint64_t>() : p->lk0.as<uint64_t>();
        uint32_t* sv = second ? p->lv1.as<uint32_t>() : p->lv0.as<uint32_t>();
        ++g_launches;
        k_step_flags<<<g, T, 0, s>>>(sk, n, p->tcount.as<uint32_t>());
        FMM_TRY(exclusive_scan_u32(p->tcount.as<uint32_t>(), p->tscan0.as<uint32_t>(), n, dcnt, p->scan_tmp, s));
        FMM_CUDA_TRY(cudaMemcpyAsync(hc, dcnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        p->n_steps = hc[0];
        const int64_t ns = p->n_steps;
        FMM_TRY(p->st_tile.ensure((ns + 1) * sizeof(int)));
        FMM_TRY(p->st_slot.ensure((ns + 1) * sizeof(int)));
        FMM_TRY(p->st_src.ensure((ns + 1) * kTile * sizeof(int)));
        FMM_TRY(p->st_ckey.ensure((ns + 1) * sizeof(uint64_t)));
        FMM_TRY(p->st_fkey.ensure((ns + 1) * sizeof(uint64_t)));
        FMM_CUDA_TRY(cudaMemsetAsync(p->st_src.ptr, 0xff, (ns + 1) * kTile * sizeof(int), s));
        ++g_launches;
        k_step_write2<<<g, T, 0, s>>>(sk, sv, n, p->tcount.as<uint32_t>(), p->tscan0.as<uint32_t>(),
                                      p->m2l_raw.as<int2>(), p->m2l_key.as<uint64_t>(), p->c_tile.as<int>(), kp.bits,
                                      p->st_tile.as<int>(),
                                      p->st_ckey.as<uint64_t>(), p->st_fkey.as<uint64_t>(), p->st_src.as<int>());
        ++g_launches;
        k_tile_ranges<<<(unsigned)((ns + T - 1) / T), T, 0, s>>>(p->st_tile.as<int>(), (int)ns, p->tile_range.as<int2>());
        // 3. distinct translations among the steps -> operator slots
        FMM_TRY(p->ukeys.ensure((ns + 1) * sizeof(uint64_t)));
        unsigned gs = (unsigned)((ns + T - 1) / T);
        ++g_launches;
        k_copy_u64_iota<<<gs, T, 0, s>>>(p->st_ckey.as<uint64_t>(), (int)ns, p->lk0.as<uint64_t>(), p->lv0.as<uint32_t>());
        FMM_TRY(radix_sort_u64(p->lk0.as<uint64_t>(), p->lv0.as<uint32_t>(), p->lk1.as<uint64_t>(),
                               p->lv1.as<uint32_t>(), ns, 0, std::max(kp.bits, 1), &second, p->sort_hist, p->scan_tmp,
                               s));
        sk = second ? p->lk1.as<uint64_t>() : p->lk0.as<uint64_t>();
        sv = second ? p->lv1.as<uint32_t>() : p->lv0.as<uint32_t>();
        ++g_launches;
        k_unique_flags<<<gs, T, 0, s>>>(sk, (int)ns, p->tcount.as<uint32_t>());
        FMM_TRY(exclusive_scan_u32(p->tcount.as<uint32_t>(), p->tscan0.as<uint32_t>(), ns, dcnt, p->scan_tmp, s));
        ++g_launches;
        k_step_slots<<<gs, T, 0, s>>>(sk, sv, (int)ns, p->tcount.as<uint32_t>(), p->tscan0.as<uint32_t>(),
                                      p->st_fkey.as<uint64_t>(), p->ukeys.as<uint64_t>(), p->st_slot.as<int>());
        FMM_CUDA_TRY(cudaMemcpyAsync(hc, dcnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        FMM_CUDA_TRY(cudaStreamSynchronize(s));
        p->n_keys = hc[0];
        FMM_CUDA_TRY(cudaGetLastError());
      }
    }
  }
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  p->p2p_pairs = (int64_t) * reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(p->pinned) + 64);
  return FMM_OK;
}

}  // namespace fmm
