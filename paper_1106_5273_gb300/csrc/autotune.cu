// Autotuner for the batched and serving forms.  The leaf capacity ncrit sets
// the work split of the method (the source chunks per leaf pair, against the
// number of cells, M2L tiles and translation operators) and the P2P tile (one
// or two targets per lane) how a leaf's targets map onto a warp.  The best
// values depend on p, the particle distribution and the problem sizes, so
// they are measured: each candidate evaluates the caller's sample batch on a
// plan of its own, timed by CUDA events on the caller's stream.  Host code;
// the evaluations run in the kernels of fmm_eval_batch.
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

extern "C" int fmm_autotune_plan(const fmm_params* base, int32_t nprob, const int64_t* offsets, const float* pos,
                                 const float* gamma, const float* sigma_prob, const double* boxes,
                                 const int32_t* ncrit_cand, int32_t n_ncrit, const int32_t* tpl_cand, int32_t n_tpl,
                                 int32_t reps, int32_t* best_ncrit, int32_t* best_tpl, double* ms_out,
                                 void* stream) {
  if (!base || !offsets || !ncrit_cand || !tpl_cand || !best_ncrit || nprob < 1 || nprob > FMM_BATCH_MAX ||
      n_ncrit < 1 || n_tpl < 1 || reps < 1 || reps > 100)
    return FMM_E_INVAL;
  for (int c = 0; c < n_ncrit; ++c)
    if (ncrit_cand[c] < 1 || ncrit_cand[c] > 4096) return FMM_E_INVAL;
  for (int c = 0; c < n_tpl; ++c)
    if (tpl_cand[c] < 0 || tpl_cand[c] > 2) return FMM_E_INVAL;
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
  for (int c = 0; c < n_ncrit && rc == FMM_OK; ++c) {
    for (int t = 0; t < n_tpl && rc == FMM_OK; ++t) {
      fmm_params q = *base;
      q.ncrit = ncrit_cand[c];
      q.p2p_tpl = tpl_cand[t];
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
      if (ms_out) ms_out[c * n_tpl + t] = per;
      if (best < 0.0 || per < best) {
        best = per;
        *best_ncrit = ncrit_cand[c];
        if (best_tpl) *best_tpl = tpl_cand[t];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  return rc;
}

extern "C" int fmm_autotune_ncrit(const fmm_params* base, int32_t nprob, const int64_t* offsets, const float* pos,
                                  const float* gamma, const float* sigma_prob, const double* boxes,
                                  const int32_t* candidates, int32_t ncand, int32_t reps, int32_t* best_ncrit,
                                  double* ms_out, void* stream) {
  if (!base) return FMM_E_INVAL;
  const int32_t tpl = base->p2p_tpl;
  return fmm_autotune_plan(base, nprob, offsets, pos, gamma, sigma_prob, boxes, candidates, ncand, &tpl, 1, reps,
                           best_ncrit, nullptr, ms_out, stream);
}
