// Morton keys, sort, octree build, cell centres and radii (Sec. 3.2).
//
// Keys: positions normalised into the cube in FP64, 21 bits per axis
// interleaved (bit b of x, y, z at 3b+2, 3b+1, 3b), stable LSD radix sort of
// (key, index).  Cells: level by level, a cell splits while it holds more than
// ncrit particles and its level is below 21; children are the non-empty
// octants in digit order, so every level is stored in Morton order.
// Expansion centre = geometric cube centre, radius = largest FP64 distance
// from the centre to a particle of the cell.  Every FP64 expression uses
// explicitly rounded operations (no contraction) in a fixed order, so the MAC
// decisions built on them are reproducible.
#include <cstring>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

__global__ void k_bbox_partial(const float* __restrict__ pos, int64_t n, double* __restrict__ part) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double v = (double)pos[3 * i + a];
      lo[a] = fmin(lo[a], v);
      hi[a] = fmax(hi[a], v);
    }
  }
  __shared__ double s[6][256];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s[a][threadIdx.x] = lo[a];
    s[3 + a][threadIdx.x] = hi[a];
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        s[a][threadIdx.x] = fmin(s[a][threadIdx.x], s[a][threadIdx.x + o]);
        s[3 + a][threadIdx.x] = fmax(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + o]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// Free-space cube: centre of the bounding box, half side = longest extent/2
// times (1 + 2^-10) (0.5 if all points coincide).
__device__ inline void cube_from_bounds(const double lo[3], const double hi[3], double* box) {
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) ext = fmax(ext, __dsub_rn(hi[a], lo[a]));
  double half = __dmul_rn(__dmul_rn(ext, 0.5), 1.0 + 0.0009765625);
  if (half == 0.0) half = 0.5;
  for (int a = 0; a < 3; ++a) box[a] = __dsub_rn(__dmul_rn(__dadd_rn(lo[a], hi[a]), 0.5), half);
  box[3] = __dmul_rn(half, 2.0);
}

__global__ void k_bbox_final(const double* __restrict__ part, int nb, double* __restrict__ box) {
  if (threadIdx.x != 0) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], part[b * 6 + a]);
      hi[a] = fmax(hi[a], part[b * 6 + 3 + a]);
    }
  cube_from_bounds(lo, hi, box);
}

// One CTA per problem of a batch: its cube (same arithmetic as above; min and
// max are exact, so the cube equals the one of the problem on its own).
__global__ void __launch_bounds__(256) k_bbox_seg(const float* __restrict__ pos, const int* __restrict__ off,
                                                  double* __restrict__ box) {
  const int sg = blockIdx.x;
  const int b = off[sg], e = off[sg + 1];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double v = (double)pos[3 * (int64_t)i + a];
      lo[a] = fmin(lo[a], v);
      hi[a] = fmax(hi[a], v);
    }
  }
  __shared__ double sh[6][256];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    sh[a][threadIdx.x] = lo[a];
    sh[3 + a][threadIdx.x] = hi[a];
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        sh[a][threadIdx.x] = fmin(sh[a][threadIdx.x], sh[a][threadIdx.x + o]);
        sh[3 + a][threadIdx.x] = fmax(sh[3 + a][threadIdx.x], sh[3 + a][threadIdx.x + o]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double l[3] = {sh[0][0], sh[1][0], sh[2][0]}, h[3] = {sh[3][0], sh[4][0], sh[5][0]};
    cube_from_bounds(l, h, box + 4 * sg);
  }
}

// Largest sigma of each problem (float bits; sigma > 0 orders like its bits).
__global__ void __launch_bounds__(256) k_sigma_max_seg(const float* __restrict__ sig, const int* __restrict__ off,
                                                       unsigned int* __restrict__ out) {
  const int sg = blockIdx.x;
  float m = 0.f;
  for (int i = off[sg] + threadIdx.x; i < off[sg + 1]; i += blockDim.x) m = fmaxf(m, sig[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh[w]);
    out[sg] = __float_as_uint(fmaxf(m, sh[0]));
  }
}

// Problem of particle i: the largest s with off[s] <= i.
__device__ inline int seg_of(const int* __restrict__ off, int nseg, int64_t i) {
  int lo = 0, hi = nseg;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)off[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_set_box(double x, double y, double z, double len, double* box) {
  box[0] = x;
  box[1] = y;
  box[2] = z;
  box[3] = len;
}

__device__ inline uint64_t spread3(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

__device__ inline uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

// Cell coordinate floor((x - bmin) f) with f = 2^kbits / L rounded once (one
// FP64 division per particle rather than one per coordinate), clamped.
__device__ inline uint64_t quantize_axis(float x, double bmin, double f, double scale) {
  double k = floor(__dmul_rn(__dsub_rn((double)x, bmin), f));
  if (!(k >= 0.0)) k = 0.0;
  if (k > scale - 1.0) k = scale - 1.0;
  return (uint64_t)k;
}

// kbits Morton bits per axis; a batch puts the problem index above them.
// span (if given) gathers the AND and the OR of all keys (one atomic each per
// warp): their XOR marks the key bits that vary.
__global__ void k_keys(const float* __restrict__ pos, int64_t n, const double* __restrict__ box,
                       const int* __restrict__ off, int nseg, int kbits, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ idx, unsigned long long* __restrict__ span) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long ka = ~0ull, ko = 0ull;
  if (i < n) {
    const int sg = off ? seg_of(off, nseg, i) : 0;
    const double* b = box + 4 * sg;
    const double scale = ldexp(1.0, kbits), f = __ddiv_rn(scale, b[3]);
    uint64_t kx = quantize_axis(pos[3 * i + 0], b[0], f, scale);
    uint64_t ky = quantize_axis(pos[3 * i + 1], b[1], f, scale);
    uint64_t kz = quantize_axis(pos[3 * i + 2], b[2], f, scale);
    const uint64_t k = ((uint64_t)sg << (3 * kbits)) | (spread3(kx) << 2) | (spread3(ky) << 1) | spread3(kz);
    keys[i] = k;
    idx[i] = (uint32_t)i;
    ka = ko = k;
  }
  if (!span) return;
  for (int o = 16; o > 0; o >>= 1) {
    ka &= __shfl_xor_sync(0xffffffffu, ka, o);
    ko |= __shfl_xor_sync(0xffffffffu, ko, o);
  }
  if ((threadIdx.x & 31) == 0 && (int64_t)blockIdx.x * blockDim.x + threadIdx.x < n) {
    atomicAnd(&span[0], ka);
    atomicOr(&span[1], ko);
  }
}

// Sorted position i of a batch lies in its problem's input range.
__global__ void k_permute(const float* __restrict__ pos, const float* __restrict__ gam,
                          const float* __restrict__ sig, float sig_u, const float* __restrict__ seg_sig,
                          const int* __restrict__ off, int nseg, const uint32_t* __restrict__ idx,
                          int64_t n, float4* __restrict__ A, float4* __restrict__ B) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t j = idx[i];
  float s = sig ? sig[j] : (seg_sig ? seg_sig[seg_of(off, nseg, i)] : sig_u);
  A[i] = make_float4(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], s);
  B[i] = make_float4(gam[3 * j], gam[3 * j + 1], gam[3 * j + 2], 0.f);
}

__global__ void k_sigma_max(const float* __restrict__ sig, int64_t n, unsigned int* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, sig[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // sigma > 0: order of bits = order of values
}

// Root cells at level 0: one per problem (key = problem index).
__global__ void k_roots(int nroot, const int* __restrict__ off, int n, int* begin, int* end, int* level, int* parent,
                        uint64_t* key) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nroot) return;
  begin[r] = off ? off[r] : 0;
  end[r] = off ? off[r + 1] : n;
  level[r] = 0;
  parent[r] = -1;
  key[r] = (uint64_t)r;
}

__device__ inline int lower_bound_u64(const uint64_t* a, int lo, int hi, uint64_t v) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One group of 8 lanes per cell: lane d finds the first particle of child
// digit d (a binary search in the cell's sorted keys, d = 1..7; lane 0 holds
// the cell's begin), so the 7 searches run side by side instead of one after
// the other.  The bounds are kept in bnd[8 * (c - lb) + d] for k_split_write.
__global__ void k_split_count(const uint64_t* __restrict__ skeys, const int* __restrict__ begin,
                              const int* __restrict__ end, const uint64_t* __restrict__ key, int lb, int le,
                              int l, int kbits, int ncrit, uint32_t* __restrict__ cnt, int* __restrict__ bnd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = lb + (t >> 3), d = t & 7;
  const bool live = c < le;
  int b = 0, e = 0;
  bool split = false;
  if (live) {
    b = begin[c];
    e = end[c];
    split = e - b > ncrit && l < kbits;
  }
  int bd = b;
  if (split && d > 0) {
    const int shift = 3 * (kbits - 1 - l);
    bd = lower_bound_u64(skeys, b, e, ((key[c] << 3) | (uint64_t)d) << shift);
  }
  // lane d's child is non-empty when the next bound (lane d + 1, or the end) is larger
  const int nb = __shfl_down_sync(0xffffffffu, bd, 1, 8);
  const int next = d == 7 ? e : nb;
  const unsigned grp = (threadIdx.x & 31) & ~7u;
  const unsigned m = __ballot_sync(0xffffffffu, split && next > bd);
  if (!live) return;
  bnd[8 * (c - lb) + d] = bd;
  if (d == 0) cnt[c - lb] = (uint32_t)__popc((m >> grp) & 0xffu);
}

__global__ void k_split_write(int* __restrict__ begin, int* __restrict__ end, int* __restrict__ level,
                              int* __restrict__ parent, int* __restrict__ child, int* __restrict__ nchild,
                              uint64_t* __restrict__ key, int lb, int le, int l, const uint32_t* __restrict__ cnt,
                              const uint32_t* __restrict__ off, const int* __restrict__ bnd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = lb + (t >> 3), d = t & 7;
  const bool live = c < le;
  uint32_t k = 0;
  int bd = 0, e = 0;
  if (live) {
    k = cnt[c - lb];
    bd = bnd[8 * (c - lb) + d];
    e = end[c];
  }
  const int nb = __shfl_down_sync(0xffffffffu, bd, 1, 8);
  const int next = d == 7 ? e : nb;
  const bool mine = live && k > 0 && next > bd;
  const unsigned grp = (threadIdx.x & 31) & ~7u;
  const unsigned m = (__ballot_sync(0xffffffffu, mine) >> grp) & 0xffu;
  if (!live) return;
  const int first = le + (int)off[c - lb];
  if (d == 0) {
    nchild[c] = (int)k;
    child[c] = k ? first : -1;
  }
  if (!mine) return;
  const int o = first + __popc(m & ((1u << d) - 1u));  // children in digit order
  begin[o] = bd;
  end[o] = next;
  level[o] = l + 1;
  parent[o] = c;
  key[o] = (key[c] << 3) | (uint64_t)d;
}

// Cell key = problem index above the 3l level-local Morton bits.
__global__ void k_centers(const int* __restrict__ level, const uint64_t* __restrict__ key, int nc,
                          const double* __restrict__ box, double* __restrict__ center,
                          unsigned long long* __restrict__ r2bits, int* __restrict__ cseg) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int l = level[c];
  const uint64_t kf = key[c];
  const int sg = (int)(kf >> (3 * l));
  const uint64_t k = kf & ((1ull << (3 * l)) - 1ull);
  const double* b = box + 4 * sg;
  double a = __dmul_rn(b[3], ldexp(1.0, -l));
  uint32_t ijk[3] = {compact3(k >> 2), compact3(k >> 1), compact3(k)};
#pragma unroll
  for (int q = 0; q < 3; ++q) center[3 * c + q] = __dadd_rn(b[q], __dmul_rn((double)ijk[q] + 0.5, a));
  r2bits[c] = 0ull;
  if (cseg) cseg[c] = sg;
}

__global__ void k_leaf_flags(const int* __restrict__ nchild, int nc, uint32_t* __restrict__ f) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) f[c] = nchild[c] == 0 ? 1u : 0u;
}

__global__ void k_leaf_list(const int* __restrict__ nchild, int nc, const uint32_t* __restrict__ off,
                            int* __restrict__ leaves) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc && nchild[c] == 0) leaves[off[c]] = c;
}

__global__ void k_leaf_of(const int* __restrict__ leaves, int nl, const int* __restrict__ begin,
                          const int* __restrict__ end, int* __restrict__ leaf_of) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= nl) return;
  int c = leaves[w];
  for (int i = begin[c] + lane; i < end[c]; i += 32) leaf_of[i] = c;
}

// r^2 of every particle about every ancestor centre; max via 64-bit atomics
// (non-negative doubles order like their bit patterns), one atomic per
// distinct cell per warp.
__global__ void k_radius(const float4* __restrict__ A, int64_t n, const int* __restrict__ leaf_of,
                         const int* __restrict__ parent, const double* __restrict__ center,
                         unsigned long long* __restrict__ r2bits) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = i < n;
  int c = valid ? leaf_of[i] : -1;
  float4 a = valid ? A[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  // all lanes walk until every lane is done
  while (__any_sync(0xffffffffu, c >= 0)) {
    unsigned long long v = 0ull;
    if (c >= 0) {
      double dx = __dsub_rn((double)a.x, center[3 * c]);
      double dy = __dsub_rn((double)a.y, center[3 * c + 1]);
      double dz = __dsub_rn((double)a.z, center[3 * c + 2]);
      double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      v = (unsigned long long)__double_as_longlong(d2);
    }
    unsigned peers = __match_any_sync(0xffffffffu, c);
    unsigned long long m = v;
    // max over peers
    for (int o = 0; o < 32; ++o) {
      unsigned long long t = __shfl_sync(0xffffffffu, v, o);
      if ((peers >> o) & 1u) m = m > t ? m : t;
    }
    int leader = __ffs(peers) - 1;
    if (c >= 0 && (int)(threadIdx.x & 31) == leader) atomicMax(&r2bits[c], m);
    c = c >= 0 ? parent[c] : -1;
  }
}

__global__ void k_radius_final(const unsigned long long* __restrict__ r2bits, int nc, const double* __restrict__ center,
                               double* __restrict__ R, float4* __restrict__ cf) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double r = __dsqrt_rn(__longlong_as_double((long long)r2bits[c]));
  R[c] = r;
  cf[c] = make_float4((float)center[3 * c], (float)center[3 * c + 1], (float)center[3 * c + 2], (float)r);
}

}  // namespace

int grow_cells(fmm_plan p, int64_t need, cudaStream_t s) {
  size_t ni = (size_t)need;
  FMM_TRY(p->c_begin.grow_copy(ni * sizeof(int), s));
  FMM_TRY(p->c_end.grow_copy(ni * sizeof(int), s));
  FMM_TRY(p->c_level.grow_copy(ni * sizeof(int), s));
  FMM_TRY(p->c_parent.grow_copy(ni * sizeof(int), s));
  FMM_TRY(p->c_child.grow_copy(ni * sizeof(int), s));
  FMM_TRY(p->c_nchild.grow_copy(ni * sizeof(int), s));
  FMM_TRY(p->c_key.grow_copy(ni * sizeof(uint64_t), s));
  return FMM_OK;
}

// Octree over the sorted keys (one root per problem), centres, leaves, radii.
static int tree_from_sorted(fmm_plan p, int64_t n, int nroot, const int* off, const double* box, int kbits,
                            bool with_seg, cudaStream_t s) {
  const int T = 256;
  unsigned nb = (unsigned)((n + T - 1) / T);
  int64_t cap = std::max<int64_t>(64, 4 * n / std::max(1, p->prm.ncrit) + 64 + 2 * (int64_t)nroot);
  if ((int64_t)(p->c_begin.bytes / sizeof(int)) < cap) FMM_TRY(grow_cells(p, cap, s));
  ++g_launches;
  k_roots<<<(unsigned)((nroot + T - 1) / T), T, 0, s>>>(nroot, off, (int)n, p->c_begin.as<int>(), p->c_end.as<int>(),
                                                         p->c_level.as<int>(), p->c_parent.as<int>(),
                                                         p->c_key.as<uint64_t>());
  p->level_begin.assign(1, 0);
  int lb = 0, le = nroot;
  uint32_t* hcount = reinterpret_cast<uint32_t*>(p->pinned);
  for (int l = 0;; ++l) {
    p->level_begin.push_back(le);
    int ncl = le - lb;
    FMM_TRY(p->tcount.ensure((size_t)(ncl + 1) * sizeof(uint32_t)));
    FMM_TRY(p->tscan0.ensure((size_t)(ncl + 1) * sizeof(uint32_t)));
    FMM_TRY(p->tscan1.ensure((size_t)(8 * (int64_t)ncl + 8) * sizeof(int)));  // child bounds (free until the traversal)
    unsigned g = (unsigned)((8 * (int64_t)ncl + T - 1) / T);
    ++g_launches;
    k_split_count<<<g, T, 0, s>>>(p->skeys, p->c_begin.as<int>(), p->c_end.as<int>(), p->c_key.as<uint64_t>(),
                                  lb, le, l, kbits, p->prm.ncrit, p->tcount.as<uint32_t>(), p->tscan1.as<int>());
    FMM_TRY(exclusive_scan_u32(p->tcount.as<uint32_t>(), p->tscan0.as<uint32_t>(), ncl,
                               p->tscan0.as<uint32_t>() + ncl, p->scan_tmp, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(hcount, p->tscan0.as<uint32_t>() + ncl, sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t nnew = hcount[0];
    if (le + nnew > (int64_t)(p->c_begin.bytes / sizeof(int))) FMM_TRY(grow_cells(p, 2 * (le + nnew), s));
    ++g_launches;
    k_split_write<<<g, T, 0, s>>>(p->c_begin.as<int>(), p->c_end.as<int>(), p->c_level.as<int>(),
                                  p->c_parent.as<int>(), p->c_child.as<int>(), p->c_nchild.as<int>(),
                                  p->c_key.as<uint64_t>(), lb, le, l, p->tcount.as<uint32_t>(),
                                  p->tscan0.as<uint32_t>(), p->tscan1.as<int>());
    FMM_CUDA_TRY(cudaGetLastError());
    if (nnew == 0) break;
    lb = le;
    le = (int)(le + nnew);
  }
  // level_begin has one entry per level plus the end
  const int nc = p->level_begin.back();
  p->ncells = nc;
  p->nlevels = (int)p->level_begin.size() - 1;

  // ---- centres, leaves, radii
  FMM_TRY(p->c_center.ensure((size_t)nc * 3 * sizeof(double)));
  FMM_TRY(p->c_radius2.ensure((size_t)nc * sizeof(unsigned long long)));
  FMM_TRY(p->c_radius.ensure((size_t)nc * sizeof(double)));
  FMM_TRY(p->leaves.ensure((size_t)(nc + 1) * sizeof(int)));
  FMM_TRY(p->tcount.ensure((size_t)(nc + 1) * sizeof(uint32_t)));
  FMM_TRY(p->tscan0.ensure((size_t)(nc + 1) * sizeof(uint32_t)));
  int* cseg = nullptr;
  if (with_seg) {
    FMM_TRY(p->c_seg.ensure((size_t)nc * sizeof(int)));
    cseg = p->c_seg.as<int>();
  }
  unsigned gc = (unsigned)((nc + T - 1) / T);
  ++g_launches;
  k_centers<<<gc, T, 0, s>>>(p->c_level.as<int>(), p->c_key.as<uint64_t>(), nc, box, p->c_center.as<double>(),
                             p->c_radius2.as<unsigned long long>(), cseg);
  ++g_launches;
  k_leaf_flags<<<gc, T, 0, s>>>(p->c_nchild.as<int>(), nc, p->tcount.as<uint32_t>());
  FMM_TRY(exclusive_scan_u32(p->tcount.as<uint32_t>(), p->tscan0.as<uint32_t>(), nc, p->tscan0.as<uint32_t>() + nc,
                             p->scan_tmp, s));
  ++g_launches;
  k_leaf_list<<<gc, T, 0, s>>>(p->c_nchild.as<int>(), nc, p->tscan0.as<uint32_t>(), p->leaves.as<int>());
  FMM_CUDA_TRY(cudaMemcpyAsync(hcount, p->tscan0.as<uint32_t>() + nc, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  p->nleaves = hcount[0];
  ++g_launches;
  k_leaf_of<<<(unsigned)((p->nleaves * 32 + T - 1) / T), T, 0, s>>>(p->leaves.as<int>(), (int)p->nleaves,
                                                                   p->c_begin.as<int>(), p->c_end.as<int>(),
                                                                   p->leaf_of.as<int>());
  ++g_launches;
  k_radius<<<nb, T, 0, s>>>(p->sortA.as<float4>(), n, p->leaf_of.as<int>(), p->c_parent.as<int>(),
                            p->c_center.as<double>(), p->c_radius2.as<unsigned long long>());
  ++g_launches;
  FMM_TRY(p->c_cf.ensure((size_t)nc * sizeof(float4)));
  k_radius_final<<<gc, T, 0, s>>>(p->c_radius2.as<unsigned long long>(), nc, p->c_center.as<double>(),
                                  p->c_radius.as<double>(), p->c_cf.as<float4>());
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

// Keys, sort, permutation into sorted SoA, octree, centres, radii.
int build_tree(fmm_plan p, int64_t n, const float* pos, const float* gam, const float* sig, float sig_u,
               cudaStream_t s) {
  const int T = 256;
  unsigned nb = (unsigned)((n + T - 1) / T);
  double* box = p->scal.as<double>();
  p->batched = 0;
  p->nseg = 1;
  p->kbits = kMaxLevel;
  if (p->prm.periodic) {
    ++g_launches;
    k_set_box<<<1, 1, 0, s>>>(p->prm.box_min[0], p->prm.box_min[1], p->prm.box_min[2], p->prm.box_len, box);
  } else {
    int parts = (int)std::min<int64_t>(1024, (n + 255) / 256);
    FMM_TRY(p->scan_tmp.ensure((size_t)parts * 6 * sizeof(double)));
    ++g_launches;
    k_bbox_partial<<<parts, 256, 0, s>>>(pos, n, p->scan_tmp.as<double>());
    ++g_launches;
    k_bbox_final<<<1, 32, 0, s>>>(p->scan_tmp.as<double>(), parts, box);
  }
  // sigma max (uniform: the value itself)
  unsigned int* smax = reinterpret_cast<unsigned int*>(box + 8);
  if (sig) {
    FMM_CUDA_TRY(cudaMemsetAsync(smax, 0, sizeof(unsigned int), s));
    int parts = (int)std::min<int64_t>(1024, (n + 255) / 256);
    ++g_launches;
    k_sigma_max<<<parts, 256, 0, s>>>(sig, n, smax);
  }
  uint64_t* k0 = p->keys0.as<uint64_t>();
  uint64_t* k1 = p->keys1.as<uint64_t>();
  uint32_t* v0 = p->vals0.as<uint32_t>();
  uint32_t* v1 = p->vals1.as<uint32_t>();
  unsigned long long* span = reinterpret_cast<unsigned long long*>(box + kScalKeySpan);
  FMM_CUDA_TRY(cudaMemsetAsync(span, 0xff, sizeof(unsigned long long), s));
  FMM_CUDA_TRY(cudaMemsetAsync(span + 1, 0, sizeof(unsigned long long), s));
  ++g_launches;
  k_keys<<<nb, T, 0, s>>>(pos, n, box, nullptr, 1, kMaxLevel, k0, v0, span);
  FMM_CUDA_TRY(cudaGetLastError());
  // sort passes over digits that no key changes are skipped (a lattice leaves
  // its low bits constant)
  unsigned long long* hspan = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(p->pinned) + 512);
  FMM_CUDA_TRY(cudaMemcpyAsync(hspan, span, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  const uint64_t vary = hspan[0] ^ hspan[1];
  int second = 0;
  FMM_TRY(radix_sort_u64(k0, v0, k1, v1, n, 0, 63, &second, p->sort_hist, p->scan_tmp, s, vary));
  p->skeys = second ? k1 : k0;
  p->sidx = second ? v1 : v0;
  ++g_launches;
  k_permute<<<nb, T, 0, s>>>(pos, gam, sig, sig_u, nullptr, nullptr, 1, p->sidx, n, p->sortA.as<float4>(),
                             p->sortB.as<float4>());
  FMM_CUDA_TRY(cudaGetLastError());
  return tree_from_sorted(p, n, 1, nullptr, box, kMaxLevel, false, s);
}

// Problem tables of a batch to the device (ranges, sigma, periodic cubes).
int upload_segments(fmm_plan p, const SegSpec& sg, cudaStream_t s) {
  const int S = sg.nseg;
  const size_t b_off = (size_t)(S + 1) * sizeof(int), b_sig = (size_t)S * sizeof(float),
               b_box = (size_t)S * 4 * sizeof(double);
  const size_t need = b_box + b_off + 2 * b_sig + 64;
  if (p->seg_pinned_bytes < need) {
    if (p->seg_pinned) cudaFreeHost(p->seg_pinned);
    p->seg_pinned = nullptr;
    p->seg_pinned_bytes = 0;
    if (cudaMallocHost(&p->seg_pinned, need) != cudaSuccess) return FMM_E_NOMEM;
    p->seg_pinned_bytes = need;
  }
  char* h = reinterpret_cast<char*>(p->seg_pinned);
  double* hbox = reinterpret_cast<double*>(h);
  int* hoff = reinterpret_cast<int*>(h + b_box);
  float* hsig = reinterpret_cast<float*>(h + b_box + b_off);
  unsigned int* hsm = reinterpret_cast<unsigned int*>(h + b_box + b_off + b_sig);
  memcpy(hoff, sg.h_off, b_off);
  FMM_TRY(p->seg_off.ensure(b_off));
  FMM_TRY(p->seg_box.ensure(b_box));
  FMM_TRY(p->seg_smax.ensure((size_t)S * sizeof(unsigned int)));
  FMM_TRY(p->seg_mac.ensure((size_t)S * sizeof(SegMac)));
  FMM_TRY(p->seg_p2p.ensure((size_t)S * sizeof(SegP2P)));
  FMM_CUDA_TRY(cudaMemcpyAsync(p->seg_off.ptr, hoff, b_off, cudaMemcpyHostToDevice, s));
  if (sg.h_box) {
    memcpy(hbox, sg.h_box, b_box);
    FMM_CUDA_TRY(cudaMemcpyAsync(p->seg_box.ptr, hbox, b_box, cudaMemcpyHostToDevice, s));
  }
  if (sg.h_sigma) {
    memcpy(hsig, sg.h_sigma, b_sig);
    memcpy(hsm, sg.h_sigma, b_sig);  // sigma > 0: its bits are the max of one value
    FMM_TRY(p->seg_sig.ensure(b_sig));
    FMM_CUDA_TRY(cudaMemcpyAsync(p->seg_sig.ptr, hsig, b_sig, cudaMemcpyHostToDevice, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(p->seg_smax.ptr, hsm, b_sig, cudaMemcpyHostToDevice, s));
  }
  return FMM_OK;
}

// A forest of independent problems: problem index above kBatchBits Morton
// bits per axis, one root per problem, each problem its own cube and sigma.
int build_forest(fmm_plan p, int64_t n, const float* pos, const float* gam, const float* sig, const SegSpec& sg,
                 cudaStream_t s) {
  const int T = 256;
  const int S = sg.nseg;
  unsigned nb = (unsigned)((n + T - 1) / T);
  p->batched = 1;
  p->nseg = S;
  p->kbits = kBatchBits;
  FMM_TRY(upload_segments(p, sg, s));
  const int* off = p->seg_off.as<int>();
  double* box = p->seg_box.as<double>();
  if (!sg.h_box) {
    ++g_launches;
    k_bbox_seg<<<S, 256, 0, s>>>(pos, off, box);
  }
  if (sig) {
    ++g_launches;
    k_sigma_max_seg<<<S, 256, 0, s>>>(sig, off, p->seg_smax.as<unsigned int>());
  }
  uint64_t* k0 = p->keys0.as<uint64_t>();
  uint64_t* k1 = p->keys1.as<uint64_t>();
  uint32_t* v0 = p->vals0.as<uint32_t>();
  uint32_t* v1 = p->vals1.as<uint32_t>();
  unsigned long long* span = reinterpret_cast<unsigned long long*>(p->scal.as<double>() + kScalKeySpan);
  FMM_CUDA_TRY(cudaMemsetAsync(span, 0xff, sizeof(unsigned long long), s));
  FMM_CUDA_TRY(cudaMemsetAsync(span + 1, 0, sizeof(unsigned long long), s));
  ++g_launches;
  k_keys<<<nb, T, 0, s>>>(pos, n, box, off, S, kBatchBits, k0, v0, span);
  FMM_CUDA_TRY(cudaGetLastError());
  unsigned long long* hspan = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(p->pinned) + 512);
  FMM_CUDA_TRY(cudaMemcpyAsync(hspan, span, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  int sbits = 0;
  while ((1 << sbits) < S) ++sbits;
  int second = 0;
  FMM_TRY(radix_sort_u64(k0, v0, k1, v1, n, 0, 3 * kBatchBits + sbits, &second, p->sort_hist, p->scan_tmp, s,
                         hspan[0] ^ hspan[1]));
  p->skeys = second ? k1 : k0;
  p->sidx = second ? v1 : v0;
  ++g_launches;
  k_permute<<<nb, T, 0, s>>>(pos, gam, sig, 0.f, sig ? nullptr : p->seg_sig.as<float>(), off, S, p->sidx, n,
                             p->sortA.as<float4>(), p->sortB.as<float4>());
  FMM_CUDA_TRY(cudaGetLastError());
  return tree_from_sorted(p, n, S, off, box, kBatchBits, true, s);
}

}  // namespace fmm

namespace fmm {

// Cube and Morton keys into caller-provided memory (same arithmetic as
// build_tree): partials holds 1024*6 doubles, box 4 doubles.
int morton_keys_raw(int64_t n, const float* pos, int periodic, const double* box_min, double box_len,
                    uint64_t* keys, uint32_t* idx, double* partials, double* box, cudaStream_t s) {
  if (periodic) {
    ++g_launches;
    k_set_box<<<1, 1, 0, s>>>(box_min[0], box_min[1], box_min[2], box_len, box);
  } else {
    int parts = (int)std::min<int64_t>(1024, (n + 255) / 256);
    ++g_launches;
    k_bbox_partial<<<parts, 256, 0, s>>>(pos, n, partials);
    ++g_launches;
    k_bbox_final<<<1, 32, 0, s>>>(partials, parts, box);
  }
  ++g_launches;
  k_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, box, nullptr, 1, kMaxLevel, keys, idx, nullptr);
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

}  // namespace fmm
