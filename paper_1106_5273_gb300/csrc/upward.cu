// Upward pass (Sec. 3.1): P2M at the leaves, M2M from the deepest level up,
// then the BF16 hi/lo split of every multipole for the tensor-core M2L.
// Three potentials (one per component of gamma) share the expansions.
#include <cuda_bf16.h>

#include "expansions.cuh"
#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kP2MThreads = 64;  // particles per pass of k_p2m (one per thread)
constexpr int kP2MRows = 4;      // output rows per thread: P <= 256 (p <= 16)

// One CTA per leaf; threads own coefficients r = tid, tid + 128.
__global__ void __launch_bounds__(kP2MThreads) k_p2m(const int* __restrict__ leaves, const int* __restrict__ begin,
                                                     const int* __restrict__ end, const int* __restrict__ level,
                                                     const double* __restrict__ center,
                                                     const double* __restrict__ box, const int* __restrict__ cseg,
                                                     const float4* __restrict__ A, const float4* __restrict__ B,
                                                     int p, float* __restrict__ M) {
  extern __shared__ float sm[];
  const int P = p * p;
  const int PS = P | 1;                          // odd row stride: the per-thread row stores hit distinct banks
  float* sR = sm;                                // [kP2MThreads][PS] conj(R~) real-packed
  float4* sG = reinterpret_cast<float4*>(sm + ((kP2MThreads * PS + 3) & ~3));  // [kP2MThreads]
  const int leaf = leaves[blockIdx.x];
  const int b = begin[leaf], e = end[leaf];
  const double a = box[4 * (cseg ? cseg[leaf] : 0) + 3] * ldexp(1.0, -level[leaf]);
  const float inv_a = (float)(1.0 / a);
  const double cx = center[3 * leaf], cy = center[3 * leaf + 1], cz = center[3 * leaf + 2];
  const int t = threadIdx.x;
  float acc[3][kP2MRows];
#pragma unroll
  for (int q = 0; q < kP2MRows; ++q) acc[0][q] = acc[1][q] = acc[2][q] = 0.f;
  for (int c0 = b; c0 < e; c0 += kP2MThreads) {
    // one particle per thread: the regular solid harmonics R~_n^m by the
    // recurrences in registers (the diagonal m = n, then up each column m),
    // stored conjugated in real-packed order
    const int j = c0 + t;
    float* row = sR + t * PS;
    if (j < e) {
      const float4 x = A[j];
      const float4 g = B[j];
      const float X = (float)((double)x.x - cx) * inv_a;
      const float Y = (float)((double)x.y - cy) * inv_a;
      const float Z = (float)((double)x.z - cz) * inv_a;
      const float r2 = X * X + Y * Y + Z * Z;
      float dre = 1.f, dim = 0.f;  // R~_m^m
      for (int m = 0; m < p; ++m) {
        if (m > 0) {
          const float f = sqrtf((2.f * m - 1.f) / (2.f * m));
          const float nr = f * (dre * X - dim * Y), ni = f * (dre * Y + dim * X);
          dre = nr;
          dim = ni;
        }
        float r1r = 0.f, r1i = 0.f, r0r = dre, r0i = dim;  // R~_{n-1}^m, R~_n^m
        for (int n = m; n < p; ++n) {
          if (n > m) {
            const float inv = rsqrtf((float)((n + m) * (n - m)));
            const float aa = (2.f * n - 1.f) * Z;
            float vr = aa * r0r, vi = aa * r0i;
            if (n - 2 >= m) {
              const float bb = r2 * sqrtf((float)((n + m - 1) * (n - m - 1)));
              vr -= bb * r1r;
              vi -= bb * r1i;
            }
            r1r = r0r;
            r1i = r0i;
            r0r = vr * inv;
            r0i = vi * inv;
          }
          if (m == 0) {
            row[n * n] = r0r;
          } else {
            row[n * n + 2 * m - 1] = r0r;
            row[n * n + 2 * m] = -r0i;
          }
        }
      }
      sG[t] = make_float4(g.x, g.y, g.z, 0.f);
    } else {
      for (int r = 0; r < P; ++r) row[r] = 0.f;
      sG[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    // M_c[r] += sum over the chunk's particles of gamma_c R~*[r]
    const int cnt = min(kP2MThreads, e - c0);
#pragma unroll
    for (int q = 0; q < kP2MRows; ++q) {
      const int r = t + kP2MThreads * q;
      if (r >= P) break;
      for (int jj = 0; jj < cnt; ++jj) {
        const float v = sR[jj * PS + r];
        const float4 gg = sG[jj];
        acc[0][q] = fmaf(gg.x, v, acc[0][q]);
        acc[1][q] = fmaf(gg.y, v, acc[1][q]);
        acc[2][q] = fmaf(gg.z, v, acc[2][q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kP2MRows; ++q) {
    const int r = t + kP2MThreads * q;
    if (r >= P) break;
    for (int c = 0; c < 3; ++c) M[((size_t)leaf * 3 + c) * P + r] = acc[c][q];
  }
}

// One CTA per cell of the level; leaves keep their P2M result.  The cell's
// expansion is the sum, in child order, of each child's term.
__global__ void __launch_bounds__(128) k_m2m(int lb, const int* __restrict__ child, const int* __restrict__ nchild,
                                             const uint64_t* __restrict__ ckey, const float* __restrict__ opT, int P,
                                             float* __restrict__ M) {
  extern __shared__ float sMc[];  // [3][P]
  const int c = lb + blockIdx.x;
  const int nch = nchild[c];
  if (nch == 0) return;
  float acc[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int q = 0; q < nch; ++q) {
    const int ch = child[c] + q;
    const int oct = (int)(ckey[ch] & 7ull);
    for (int i = threadIdx.x; i < 3 * P; i += blockDim.x) sMc[i] = M[(size_t)ch * 3 * P + i];
    __syncthreads();
    const float* W = opT + (size_t)oct * P * P;
    for (int h = 0; h < 2; ++h) {
      int r = threadIdx.x + 128 * h;
      if (r >= P) break;
      // the child's term, then added to the sum of the earlier children's
      // (the order and rounding of k_m2m8)
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 8
      for (int k = 0; k < P; ++k) {
        float w = W[(size_t)k * P + r];
        a0 = fmaf(w, sMc[k], a0);
        a1 = fmaf(w, sMc[P + k], a1);
        a2 = fmaf(w, sMc[2 * P + k], a2);
      }
      if (q == 0) {
        acc[0][h] = a0;
        acc[1][h] = a1;
        acc[2][h] = a2;
      } else {
        acc[0][h] += a0;
        acc[1][h] += a1;
        acc[2][h] += a2;
      }
    }
    __syncthreads();
  }
  for (int h = 0; h < 2; ++h) {
    int r = threadIdx.x + 128 * h;
    if (r >= P) break;
    for (int cc = 0; cc < 3; ++cc) M[((size_t)c * 3 + cc) * P + r] = acc[cc][h];
  }
}

// The same for levels of few cells (the upper levels, where one CTA per cell
// walking its children one after the other is a latency chain).  Each of the
// cell's children has its own group of 128 threads (thread = output row):
// the group applies the child's octant operator to the child's expansion,
// and the cell's expansion is the sum of the children's terms in child
// order (a fixed order, so the result is deterministic).
constexpr int kM2MGroup = 128;
constexpr int kM2MWide = 1024;  // levels of at least this many cells use k_m2m (one 128-thread CTA per cell)
__global__ void __launch_bounds__(8 * kM2MGroup) k_m2m8(int lb, const int* __restrict__ child,
                                                       const int* __restrict__ nchild,
                                                       const uint64_t* __restrict__ ckey,
                                                       const float* __restrict__ opT, int P, float* __restrict__ M) {
  extern __shared__ float sm[];
  float* sMc = sm;               // [8][3][P] the children's expansions
  float* sPart = sm + 8 * 3 * P;  // [8][3][P] each child's term
  const int c = lb + blockIdx.x;
  const int nch = nchild[c];
  if (nch == 0) return;
  const int g = threadIdx.x / kM2MGroup, t = threadIdx.x % kM2MGroup;
  const int cb = child[c];
  for (int i = threadIdx.x; i < nch * 3 * P; i += blockDim.x) sMc[i] = M[(size_t)cb * 3 * P + i];
  __syncthreads();
  if (g < nch) {
    const int oct = (int)(ckey[cb + g] & 7ull);
    const float* W = opT + (size_t)oct * P * P;
    const float* x = sMc + g * 3 * P;
    for (int h = 0; h < 2; ++h) {
      const int r = t + kM2MGroup * h;
      if (r >= P) break;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 8
      for (int k = 0; k < P; ++k) {
        const float w = W[(size_t)k * P + r];
        a0 = fmaf(w, x[k], a0);
        a1 = fmaf(w, x[P + k], a1);
        a2 = fmaf(w, x[2 * P + k], a2);
      }
      sPart[(g * 3 + 0) * P + r] = a0;
      sPart[(g * 3 + 1) * P + r] = a1;
      sPart[(g * 3 + 2) * P + r] = a2;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * P; e += blockDim.x) {
    float acc = sPart[e];
    for (int q = 1; q < nch; ++q) acc += sPart[q * 3 * P + e];
    M[(size_t)c * 3 * P + e] = acc;
  }
}

// Round an FP32 value to TF32 (10 stored mantissa bits, to nearest, ties to
// even) in its 32-bit container; the low 13 bits end up zero.
__device__ __forceinline__ float round_tf32_m(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;  // inf / nan
  u += 0x0FFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xFFFFE000u);
}

// Mtf[cell][hi/lo][comp][kpad] TF32 halves, zero beyond P (kpad = 32 x K chunks).
__global__ void k_split_tf32(const float* __restrict__ M, int64_t ncell, int P, int kpad, float* __restrict__ Mtf) {
  int64_t total = ncell * 3 * kpad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(i % kpad);
    int64_t cc = i / kpad;  // cell*3 + comp
    int64_t cell = cc / 3;
    int comp = (int)(cc % 3);
    float v = k < P ? M[cc * P + k] : 0.f;
    const float hi = round_tf32_m(v);
    Mtf[((cell * 2 + 0) * 3 + comp) * kpad + k] = hi;
    Mtf[((cell * 2 + 1) * 3 + comp) * kpad + k] = round_tf32_m(v - hi);
  }
}

// Mbf[cell][hi/lo][comp][kpad], zero beyond P (kpad = 64 x K chunks).
__global__ void k_split_bf16(const float* __restrict__ M, int64_t ncell, int P, int kpad,
                             __nv_bfloat16* __restrict__ Mbf) {
  int64_t total = ncell * 3 * kpad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(i % kpad);
    int64_t cc = i / kpad;  // cell*3 + comp
    int64_t cell = cc / 3;
    int comp = (int)(cc % 3);
    float v = k < P ? M[cc * P + k] : 0.f;
    __nv_bfloat16 hi = __float2bfloat16(v);
    __nv_bfloat16 lo = __float2bfloat16(v - __bfloat162float(hi));
    Mbf[((cell * 2 + 0) * 3 + comp) * kpad + k] = hi;
    Mbf[((cell * 2 + 1) * 3 + comp) * kpad + k] = lo;
  }
}

}  // namespace

int upward_pass(fmm_plan p, cudaStream_t s) {
  const int P = p->P, pp = p->prm.p;
  const int nc = (int)p->ncells;
  FMM_TRY(p->M.ensure((size_t)nc * 3 * P * sizeof(float)));
  const size_t sh = ((size_t)((kP2MThreads * (P | 1) + 3) & ~3) + 4 * kP2MThreads) * sizeof(float);
  if (sh > 48 * 1024) FMM_CUDA_TRY(cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  ++g_launches;
  k_p2m<<<(unsigned)p->nleaves, kP2MThreads, sh, s>>>(p->leaves.as<int>(), p->c_begin.as<int>(), p->c_end.as<int>(),
                                              p->c_level.as<int>(), p->c_center.as<double>(),
                                              p->batched ? p->seg_box.as<double>() : p->scal.as<double>(),
                                              p->batched ? p->c_seg.as<int>() : nullptr,
                                              p->sortA.as<float4>(), p->sortB.as<float4>(), pp, p->M.as<float>());
  FMM_CUDA_TRY(cudaGetLastError());
  const size_t sh_m2m = (size_t)2 * 8 * 3 * P * sizeof(float);  // 48 KB at P = 256
  if (sh_m2m > 48 * 1024)
    FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2m8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_m2m));
  for (int l = p->nlevels - 2; l >= 0; --l) {
    int lb = p->level_begin[l], le = p->level_begin[l + 1];
    ++g_launches;
    if (le - lb >= kM2MWide)
      k_m2m<<<le - lb, 128, 3 * P * sizeof(float), s>>>(lb, p->c_child.as<int>(), p->c_nchild.as<int>(),
                                                        p->c_key.as<uint64_t>(), p->m2m_T.as<float>(), P,
                                                        p->M.as<float>());
    else
      k_m2m8<<<le - lb, 8 * kM2MGroup, 2 * 8 * 3 * P * sizeof(float), s>>>(
          lb, p->c_child.as<int>(), p->c_nchild.as<int>(), p->c_key.as<uint64_t>(), p->m2m_T.as<float>(), P,
          p->M.as<float>());
  }
  FMM_CUDA_TRY(cudaGetLastError());
  if (p->last_tc) {
    // 128 bytes per K chunk of each (cell, hi/lo, component) row
    const int nkc = m2l_kchunks(P, p->tc_kind);
    FMM_TRY(p->Mbf.ensure((size_t)nc * 2 * 3 * nkc * 128));
    ++g_launches;
    if (p->tc_kind)
      k_split_tf32<<<2048, 256, 0, s>>>(p->M.as<float>(), nc, P, 32 * nkc, p->Mbf.as<float>());
    else
      k_split_bf16<<<2048, 256, 0, s>>>(p->M.as<float>(), nc, P, 64 * nkc, p->Mbf.as<__nv_bfloat16>());
    FMM_CUDA_TRY(cudaGetLastError());
  }
  return FMM_OK;
}

}  // namespace fmm
