// Velocity at separate target points (Sec. 4.3 compares the kinetic energy
// spectrum of the vortex-method field with the spectral method's, which needs
// the velocity on grid points that are not particles).  The targets enter the
// plan's tree as blobs of zero strength behind the sources, so the FMM of
// fmm_eval_velocity_stretching evaluates the field there unchanged: a zero
// strength contributes nothing to any sum.  Velocity only (the stretching of
// a zero strength is zero).
#include "fmm_internal.cuh"

using namespace fmm;

namespace {

// Largest source core width (one CTA, fixed-order reduction): the targets get
// it, so sigma_max -- and with it the far-field separation and the pair
// classes -- is that of the sources alone.
__global__ void __launch_bounds__(1024) k_sigma_fill(const float* __restrict__ src_sigma, int64_t ns,
                                                     float* __restrict__ tgt_sigma, int64_t nt) {
  __shared__ float sh[1024];
  float m = 0.f;
  for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) m = fmaxf(m, src_sigma[i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  const float v = sh[0];
  for (int64_t i = threadIdx.x; i < nt; i += blockDim.x) tgt_sigma[i] = v;
}

}  // namespace

extern "C" int fmm_eval_targets(fmm_plan p, int64_t ns, const float* src_pos, const float* src_gamma,
                                const float* src_sigma, float sigma_uniform, int64_t nt, const float* tgt_pos,
                                float* vel, void* stream) {
  if (!p || ns < 0 || nt < 0 || ns + nt > p->n_max) return FMM_E_INVAL;
  if ((ns > 0 && (!src_pos || !src_gamma)) || (nt > 0 && (!tgt_pos || !vel))) return FMM_E_INVAL;
  if (!src_sigma && !(sigma_uniform > 0.f)) return FMM_E_INVAL;
  if (nt == 0) return FMM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (ns == 0) {  // no sources: the field is zero
    FMM_CUDA_TRY(cudaMemsetAsync(vel, 0, (size_t)nt * 12, s));
    return FMM_OK;
  }
  const int64_t n = ns + nt;
  const size_t b3 = (size_t)n * 3 * sizeof(float);
  FMM_CUDA_TRY(cudaSetDevice(p->device));
  FMM_TRY(p->t_pos.ensure(b3));
  FMM_TRY(p->t_gam.ensure(b3));
  FMM_TRY(p->t_vel.ensure(b3));
  float* pos = p->t_pos.as<float>();
  float* gam = p->t_gam.as<float>();
  float* sig = nullptr;
  FMM_CUDA_TRY(cudaMemcpyAsync(pos, src_pos, (size_t)ns * 12, cudaMemcpyDeviceToDevice, s));
  FMM_CUDA_TRY(cudaMemcpyAsync(gam, src_gamma, (size_t)ns * 12, cudaMemcpyDeviceToDevice, s));
  FMM_CUDA_TRY(cudaMemcpyAsync(pos + 3 * ns, tgt_pos, (size_t)nt * 12, cudaMemcpyDeviceToDevice, s));
  FMM_CUDA_TRY(cudaMemsetAsync(gam + 3 * ns, 0, (size_t)nt * 12, s));
  if (src_sigma) {
    FMM_TRY(p->t_sig.ensure((size_t)n * sizeof(float)));
    sig = p->t_sig.as<float>();
    FMM_CUDA_TRY(cudaMemcpyAsync(sig, src_sigma, (size_t)ns * 4, cudaMemcpyDeviceToDevice, s));
    ++g_launches;
    k_sigma_fill<<<1, 1024, 0, s>>>(src_sigma, ns, sig + ns, nt);
    FMM_CUDA_TRY(cudaGetLastError());
  }
  // a point target has no core width of its own: the source rule applies
  const int rule = p->prm.sigma_rule;
  p->prm.sigma_rule = FMM_SIGMA_SOURCE;
  const int rc = fmm_eval_velocity_stretching(p, n, pos, gam, sig, sigma_uniform, p->t_vel.as<float>(), nullptr, stream);
  p->prm.sigma_rule = rule;
  p->reuse_ok = 0;  // the tree holds the targets too: no strength-only re-evaluation
  FMM_TRY(rc);
  FMM_CUDA_TRY(cudaMemcpyAsync(vel, p->t_vel.as<float>() + 3 * ns, (size_t)nt * 12, cudaMemcpyDeviceToDevice, s));
  return FMM_OK;
}
