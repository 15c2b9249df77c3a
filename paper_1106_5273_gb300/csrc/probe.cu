// FP32 throughput probe: the rate the FMA pipe sustains on independent FFMA2
// chains, timed with CUDA events.  It measures the ceiling the P2P kernel's
// roofline fraction is read against (the derived peak counts 128 FP32 lanes
// per SM at the maximum clock; this is what the pipe delivers).
#include "fmm_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_ffma2_probe(float* __restrict__ out, float seed) {
  float2 v[kChains];
  const float2 a = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = make_float2(seed + threadIdx.x + c, seed - c);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], a, b);
  }
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += v[c].x + v[c].y;
  if (acc == 12345.678f) out[blockIdx.x] = acc;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int fmm_probe_fp32_rate(int32_t launches, double* tflops, double* ms_per_launch, void* stream) {
  if (launches < 1 || launches > 1000 || !tflops) return FMM_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  FMM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)sms * 8;  // 8 CTAs of 256 threads per SM: 64 warps
  fmm::DBuf out;
  FMM_TRY(out.ensure(grid * sizeof(float)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FMM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FMM_E_CUDA;
  if (rc == FMM_OK) {
    k_ffma2_probe<<<grid, 256, 0, s>>>(out.as<float>(), 1.0f);  // warm-up
    cudaEventRecord(e0, s);
    for (int l = 0; l < launches; ++l) k_ffma2_probe<<<grid, 256, 0, s>>>(out.as<float>(), 1.0f + l);
    cudaEventRecord(e1, s);
    fmm::g_launches += launches + 1;
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = FMM_E_CUDA;
  }
  if (rc == FMM_OK) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = (double)grid * 256 * kChains * kIters * 4.0 * launches;  // FFMA2 = 2 FMAs = 4 flops
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_per_launch) *ms_per_launch = ms / launches;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  out.release();
  return rc;
}
