// Leaf-size autotuner for the batched and serving forms.  The leaf capacity
// ncrit sets the work split of the method: the P2P tile (one or two targets
// per lane, the source chunks per leaf pair) against the number of cells,
// M2L tiles and translation operators.  The best value depends on p, the
// particle distribution and the problem sizes, so it is measured: each
// candidate evaluates the caller's sample batch on a plan of its own, timed
// by CUDA events on the caller's stream.  Host code; the evaluations run in
// the kernels of fmm_eval_batch.
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

extern "C" int fmm_autotune_ncrit(const fmm_params* base, int32_t nprob, const int64_t* offsets, const float* pos,
                                  const float* gamma, const float* sigma_prob, const double* boxes,
                                  const int32_t* candidates, int32_t ncand, int32_t reps, int32_t* best_ncrit,
                                  double* ms_out, void* stream) {
  if (!base || !offsets || !candidates || !best_ncrit || nprob < 1 || nprob > FMM_BATCH_MAX || ncand < 1 ||
      reps < 1 || reps > 100)
    return FMM_E_INVAL;
  for (int c = 0; c < ncand; ++c)
    if (candidates[c] < 1 || candidates[c] > 4096) return FMM_E_INVAL;
  const int64_t n = offsets[nprob];
  if (n < 1 || !pos || !gamma || !sigma_prob) return FMM_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // both outputs are produced, so the timed work is the full evaluation
  fmm::DBuf vel, dg;
  struct Release {
    fmm::DBuf *a, *b;
    ~Release() {
      a->release();
      b->release();
    }
  } release_on_exit{&vel, &dg};
  FMM_TRY(vel.ensure((size_t)n * 3 * sizeof(float)));
  FMM_TRY(dg.ensure((size_t)n * 3 * sizeof(float)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FMM_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FMM_E_CUDA;
  }
  float* dv = vel.as<float>();
  float* ds = dg.as<float>();
  int rc = FMM_OK;
  double best = -1.0;
  for (int c = 0; c < ncand && rc == FMM_OK; ++c) {
    fmm_params q = *base;
    q.ncrit = candidates[c];
    fmm_plan p = nullptr;
    if ((rc = fmm_plan_create(&q, n, &p)) != FMM_OK) break;
    // warm-up: sizes the workspace and fills the plan's operator cache
    rc = fmm_eval_batch(p, nprob, offsets, pos, gamma, nullptr, sigma_prob, boxes, dv, ds, stream);
    float ms = 0.f;
    if (rc == FMM_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = FMM_E_CUDA;
    for (int r = 0; r < reps && rc == FMM_OK; ++r)
      rc = fmm_eval_batch(p, nprob, offsets, pos, gamma, nullptr, sigma_prob, boxes, dv, ds, stream);
    if (rc == FMM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = FMM_E_CUDA;
    fmm_plan_destroy(p);
    if (rc != FMM_OK) break;
    const double per = (double)ms / reps;
    if (ms_out) ms_out[c] = per;
    if (best < 0.0 || per < best) {
      best = per;
      *best_ncrit = candidates[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  return rc;
}
