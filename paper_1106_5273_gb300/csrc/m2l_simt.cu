// M2L on CUDA cores, FP32 (Sec. 3.1; the reference path for the tensor-core
// kernel).  Work is grouped into steps: one step = one 64-cell target tile
// of a level and one translation operator T (P x P), applied to the
// multipoles of the tile's source cells:  L[:, t] += T M[:, src(t)].  One CTA
// owns a tile, accumulates all its steps in registers and writes each target
// local expansion once (no atomics, fixed summation order).
#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int kRC = 32;  // output rows per pass

__global__ void __launch_bounds__(192) k_m2l_simt(const int2* __restrict__ tile_range, const int* __restrict__ tfirst,
                                                  const int* __restrict__ st_slot, const int* __restrict__ st_src,
                                                  const float* __restrict__ T32, const float* __restrict__ M, int P,
                                                  const int* __restrict__ tcell, float* __restrict__ L) {
  extern __shared__ float sT[];  // [kRC][P]
  const int tile = blockIdx.x;
  const int2 rg = tile_range[tile];
  if (rg.y <= rg.x) return;
  const int first = tfirst[tile];
  const int ncell = tfirst[tile + 1] - first;
  const int comp = threadIdx.x / kTile, slot = threadIdx.x % kTile;
  for (int r0 = 0; r0 < P; r0 += kRC) {
    const int nr = min(kRC, P - r0);
    float acc[kRC];
#pragma unroll
    for (int i = 0; i < kRC; ++i) acc[i] = 0.f;
    for (int st = rg.x; st < rg.y; ++st) {
      const float* T = T32 + (size_t)st_slot[st] * P * P;
      for (int i = threadIdx.x; i < nr * P; i += blockDim.x) sT[i] = T[(size_t)r0 * P + i];
      __syncthreads();
      const int src = st_src[(size_t)st * kTile + slot];
      if (src >= 0) {
        const float* m = M + ((size_t)src * 3 + comp) * P;
        for (int k = 0; k < P; ++k) {
          const float b = m[k];
#pragma unroll
          for (int i = 0; i < kRC; ++i) acc[i] = fmaf(sT[i * P + k], b, acc[i]);
        }
      }
      __syncthreads();
    }
    if (slot < ncell) {
      float* out = L + ((size_t)tcell[first + slot] * 3 + comp) * P + r0;
      for (int i = 0; i < nr; ++i) out[i] = acc[i];
    }
  }
}

}  // namespace

int m2l_simt(fmm_plan p, cudaStream_t s) {
  if (p->n_steps == 0) return FMM_OK;
  size_t sh = (size_t)kRC * p->P * sizeof(float);
  if (sh > 48 * 1024) FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  ++g_launches;
  k_m2l_simt<<<(unsigned)p->ntiles, 3 * kTile, sh, s>>>(p->tile_range.as<int2>(), p->tile_first.as<int>(),
                                                         p->st_slot.as<int>(),
                                                         p->st_src.as<int>(), p->T32.as<float>(), p->M.as<float>(),
                                                         p->P, p->tile_cells.as<int>(), p->L.as<float>());
  FMM_CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

}  // namespace fmm
