// Upward pass (Sec. 3.1): P2M at the leaves, M2M from the deepest level up,
// then the BF16 hi/lo split of every multipole for the tensor-core M2L.
// Three potentials (one per component of gamma) share the expansions.
#include <cuda_bf16.h>

#include "expansions.cuh"
#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kP2MChunk = 32;

// One CTA per leaf; threads own coefficients r = tid, tid + 128.
__global__ void __launch_bounds__(128) k_p2m(const int* __restrict__ leaves, const int* __restrict__ begin,
                                             const int* __restrict__ end, const int* __restrict__ level,
                                             const double* __restrict__ center, const double* __restrict__ box,
                                             const int* __restrict__ cseg,
                                             const float4* __restrict__ A, const float4* __restrict__ B, int p,
                                             float* __restrict__ M) {
  extern __shared__ float sm[];
  const int P = p * p;
  const int NC = p * (p + 1) / 2;
  float* sR = sm;                       // [32][P] conj(R~) real-packed
  float* sG = sR + kP2MChunk * P;       // [32][3]
  float* sRe = sG + kP2MChunk * 3;      // [32][NC] scratch
  float* sIm = sRe + kP2MChunk * NC;    // [32][NC]
  const int leaf = leaves[blockIdx.x];
  const int b = begin[leaf], e = end[leaf];
  const double a = box[4 * (cseg ? cseg[leaf] : 0) + 3] * ldexp(1.0, -level[leaf]);
  const float inv_a = (float)(1.0 / a);
  const double cx = center[3 * leaf], cy = center[3 * leaf + 1], cz = center[3 * leaf + 2];
  float acc[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int c0 = b; c0 < e; c0 += kP2MChunk) {
    const int t = threadIdx.x;
    if (t < kP2MChunk) {
      int j = c0 + t;
      float* re = sRe + t * NC;
      float* im = sIm + t * NC;
      float* row = sR + t * P;
      if (j < e) {
        float4 x = A[j];
        float4 g = B[j];
        float yx = (float)((double)x.x - cx) * inv_a;
        float yy = (float)((double)x.y - cy) * inv_a;
        float yz = (float)((double)x.z - cz) * inv_a;
        regular_table_f(yx, yy, yz, p, re, im);
        for (int n = 0; n < p; ++n) {
          row[n * n] = re[n * (n + 1) / 2];
          for (int m = 1; m <= n; ++m) {
            row[n * n + 2 * m - 1] = re[n * (n + 1) / 2 + m];
            row[n * n + 2 * m] = -im[n * (n + 1) / 2 + m];
          }
        }
        sG[3 * t] = g.x;
        sG[3 * t + 1] = g.y;
        sG[3 * t + 2] = g.z;
      } else {
        for (int r = 0; r < P; ++r) row[r] = 0.f;
        sG[3 * t] = sG[3 * t + 1] = sG[3 * t + 2] = 0.f;
      }
    }
    __syncthreads();
    const int cnt = min(kP2MChunk, e - c0);
    for (int q = 0; q < 2; ++q) {
      int r = threadIdx.x + 128 * q;
      if (r >= P) break;
      for (int jj = 0; jj < cnt; ++jj) {
        float v = sR[jj * P + r];
        acc[0][q] = fmaf(sG[3 * jj], v, acc[0][q]);
        acc[1][q] = fmaf(sG[3 * jj + 1], v, acc[1][q]);
        acc[2][q] = fmaf(sG[3 * jj + 2], v, acc[2][q]);
      }
    }
    __syncthreads();
  }
  for (int q = 0; q < 2; ++q) {
    int r = threadIdx.x + 128 * q;
    if (r >= P) break;
    for (int c = 0; c < 3; ++c) M[((size_t)leaf * 3 + c) * P + r] = acc[c][q];
  }
}

// One CTA per cell of the level; leaves keep their P2M result.
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
#pragma unroll 8
      for (int k = 0; k < P; ++k) {
        float w = W[(size_t)k * P + r];
        acc[0][h] = fmaf(w, sMc[k], acc[0][h]);
        acc[1][h] = fmaf(w, sMc[P + k], acc[1][h]);
        acc[2][h] = fmaf(w, sMc[2 * P + k], acc[2][h]);
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
  const int NC = pp * (pp + 1) / 2;
  size_t sh = (size_t)(kP2MChunk * P + kP2MChunk * 3 + 2 * kP2MChunk * NC) * sizeof(float);
  if (sh > 48 * 1024) FMM_CUDA_TRY(cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  ++g_launches;
  k_p2m<<<(unsigned)p->nleaves, 128, sh, s>>>(p->leaves.as<int>(), p->c_begin.as<int>(), p->c_end.as<int>(),
                                              p->c_level.as<int>(), p->c_center.as<double>(),
                                              p->batched ? p->seg_box.as<double>() : p->scal.as<double>(),
                                              p->batched ? p->c_seg.as<int>() : nullptr,
                                              p->sortA.as<float4>(), p->sortB.as<float4>(), pp, p->M.as<float>());
  FMM_CUDA_TRY(cudaGetLastError());
  for (int l = p->nlevels - 2; l >= 0; --l) {
    int lb = p->level_begin[l], le = p->level_begin[l + 1];
    ++g_launches;
    k_m2m<<<le - lb, 128, 3 * P * sizeof(float), s>>>(lb, p->c_child.as<int>(), p->c_nchild.as<int>(),
                                                      p->c_key.as<uint64_t>(), p->m2m_T.as<float>(), P,
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
