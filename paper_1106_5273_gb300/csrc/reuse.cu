// Re-evaluation with new strengths on an unchanged tree, and its capture as a
// CUDA graph.
//
// The vortex method re-initialises its particles onto the same positions
// every step, so the tree built for them can be kept (Sec. 3.4: the
// partitioning is done once and the tree structure reused).  Here the plan
// keeps, from its last full evaluation, the sorted positions and core widths,
// the octree, both interaction lists and the M2L operators; a new set of
// strengths then needs only the steps that depend on them: gather the
// strengths into the sorted order, P2M/M2M, M2L (+ the periodic lattice
// operator), L2L/L2P and P2P with the combine -- a fixed sequence of kernel
// launches with fixed shapes, no host synchronization and no allocation.
// That sequence is what fmm_graph_capture records once and fmm_graph_launch
// replays.
#include <cstring>

#include "fmm_internal.cuh"

using namespace fmm;

namespace {

__global__ void k_gather_gamma(const float* __restrict__ gam, const uint32_t* __restrict__ idx, int64_t n,
                               float4* __restrict__ B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t j = idx[i];
  B[i] = make_float4(gam[3 * j], gam[3 * j + 1], gam[3 * j + 2], 0.f);
}

}  // namespace

struct fmm_graph_s {
  fmm_plan plan = nullptr;
  int64_t epoch = 0;
  int64_t launches = 0;  // kernel launches recorded in the graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace fmm {

// Every buffer below was sized by the full evaluation that set reuse_ok, so
// no ensure() in the launchers allocates.
int eval_strengths(fmm_plan p, const float* gam, float* vel, float* dg, cudaStream_t s) {
  if (!p->reuse_ok) return FMM_E_INVAL;
  const int64_t n = p->last_n;
  if (n > 0 && !gam) return FMM_E_INVAL;
  if (n == 0) return FMM_OK;
  FMM_CUDA_TRY(cudaMemsetAsync(p->flags.ptr, 0, sizeof(int) * 4, s));
  ++g_launches;
  k_gather_gamma<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gam, p->sidx, n, p->sortB.as<float4>());
  FMM_CUDA_TRY(cudaGetLastError());
  FMM_TRY(upward_pass(p, s));
  FMM_TRY(dipole_pass(p, n, s));
  const size_t lbytes = (size_t)p->ncells * 3 * p->P * sizeof(float);
  FMM_CUDA_TRY(cudaMemsetAsync(p->L.ptr, 0, lbytes, s));
  if (p->last_tc) FMM_TRY(m2l_tensor(p, s));
  else FMM_TRY(m2l_simt(p, s));
  FMM_TRY(apply_lattice(p, s));
  FMM_TRY(downward_pass(p, n, s));
  FMM_TRY(p2p_near(p, n, p->reuse_sig_u, p->reuse_ps, p->reuse_smax, vel, dg, s));
  return FMM_OK;
}

}  // namespace fmm

extern "C" {

int fmm_eval_strengths(fmm_plan p, const float* gamma, float* vel, float* dgamma, void* stream) {
  if (!p) return FMM_E_INVAL;
  FMM_CUDA_TRY(cudaSetDevice(p->device));
  return eval_strengths(p, gamma, vel, dgamma, (cudaStream_t)stream);
}

int fmm_plan_status(fmm_plan p, void* stream) {
  if (!p) return FMM_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  FMM_CUDA_TRY(cudaSetDevice(p->device));
  FMM_CUDA_TRY(cudaMemcpyAsync(p->pinned, p->flags.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  int hf = 0;
  memcpy(&hf, p->pinned, sizeof(int));
  return hf;
}

int fmm_graph_capture(fmm_plan p, const float* gamma, float* vel, float* dgamma, fmm_graph* out) {
  if (!p || !out) return FMM_E_INVAL;
  if (!p->reuse_ok || p->last_n == 0 || !gamma) return FMM_E_INVAL;
  FMM_CUDA_TRY(cudaSetDevice(p->device));
  fmm_graph g = new (std::nothrow) fmm_graph_s();
  if (!g) return FMM_E_NOMEM;
  g->plan = p;
  g->epoch = p->epoch;
  cudaStream_t cs = nullptr;
  int rc = FMM_OK;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = FMM_E_CUDA;
  if (rc == FMM_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = FMM_E_CUDA;
  if (rc == FMM_OK) {
    const int64_t l0 = g_launches;
    const int erc = eval_strengths(p, gamma, vel, dgamma, cs);
    g->launches = g_launches - l0;
    g_launches -= g->launches;  // counted when the graph is launched
    // always end the capture, also after an error, so the stream is usable
    const cudaError_t ce = cudaStreamEndCapture(cs, &g->graph);
    if (erc != FMM_OK) rc = erc;
    else if (ce != cudaSuccess || !g->graph) rc = FMM_E_CUDA;
  }
  if (rc == FMM_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = FMM_E_CUDA;
  if (cs) cudaStreamDestroy(cs);
  if (rc != FMM_OK) {
    fmm_graph_destroy(g);
    cudaGetLastError();
    return rc;
  }
  *out = g;
  return FMM_OK;
}

int fmm_graph_launch(fmm_graph g, void* stream) {
  if (!g || !g->exec || !g->plan) return FMM_E_INVAL;
  if (g->plan->epoch != g->epoch || !g->plan->reuse_ok) return FMM_E_INVAL;  // the plan was re-evaluated
  FMM_CUDA_TRY(cudaSetDevice(g->plan->device));
  FMM_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  g_launches += g->launches;
  return FMM_OK;
}

int64_t fmm_graph_kernel_count(fmm_graph g) { return g ? g->launches : 0; }

void fmm_graph_destroy(fmm_graph g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

}  // extern "C"
