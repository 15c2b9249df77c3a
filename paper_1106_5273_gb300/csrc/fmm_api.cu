// C ABI (include/fmm_vortex.h): plan management and the evaluation sequence
//   tree (keys, sort, octree, radii) -> P2M/M2M -> traversal -> M2L
//   (+ periodic lattice) -> L2L/L2P -> P2P + combine,
// every step a kernel on the caller's stream (Sec. 3.1, Algorithms 1-2).
#include <cmath>
#include <cstdio>
#include <cstring>

#include "fmm_internal.cuh"

using namespace fmm;

namespace fmm {
std::atomic<int64_t> g_launches{0};
}

namespace {

int check_params(const fmm_params* q) {
  if (!q) return FMM_E_INVAL;
  if (q->p < 1 || q->p > kPMax) return FMM_E_INVAL;
  if (!(q->theta > 0.f && q->theta < 1.f)) return FMM_E_INVAL;
  if (q->ncrit < 1 || q->ncrit > 4096) return FMM_E_INVAL;
  if (q->periodic != 0 && q->periodic != 1) return FMM_E_INVAL;
  if (q->periodic && (q->images < 1 || q->images > 8 || !(q->box_len > 0.0))) return FMM_E_INVAL;
  if (!(q->sigma_sep >= 0.f)) return FMM_E_INVAL;
  if (q->m2l_mode & ~(3 | FMM_M2L_SORT_STEPS | FMM_M2L_FULL_SPLIT | FMM_M2L_CHUNK_STAGES)) return FMM_E_INVAL;
  if (q->outputs & ~(FMM_OUT_VELOCITY | FMM_OUT_STRETCHING | FMM_OUT_STRETCHING_TRANSPOSE)) return FMM_E_INVAL;
  if (q->sigma_rule != FMM_SIGMA_SOURCE && q->sigma_rule != FMM_SIGMA_MIXED) return FMM_E_INVAL;
  if (q->p2p_pair_max < 0) return FMM_E_INVAL;
  if (q->split_tie != FMM_SPLIT_SOURCE && q->split_tie != FMM_SPLIT_TARGET) return FMM_E_INVAL;
  if (q->p2p_tpl < 0 || q->p2p_tpl > 2) return FMM_E_INVAL;
  return FMM_OK;
}

std::vector<DBuf*> plan_buffers(fmm_plan p) {
  return {&p->m2m_T, &p->l2l_T, &p->l2p_tab, &p->lattice, &p->keys0, &p->keys1, &p->vals0, &p->vals1,
          &p->sortA, &p->sortB, &p->far_u, &p->far_s, &p->leaf_of, &p->in_pos, &p->in_gam, &p->in_sig,
          &p->out_vel, &p->out_dg, &p->c_begin, &p->c_end, &p->c_level, &p->c_parent, &p->c_child,
          &p->c_nchild, &p->c_key, &p->c_center, &p->c_radius2, &p->c_radius, &p->dip_part, &p->c_cf, &p->c_tile,
          &p->tile_cells, &p->tile_first, &p->tile_groups, &p->c_ijk, &p->t_pos, &p->t_gam, &p->t_sig, &p->t_vel, &p->leaves, &p->M, &p->L, &p->Mbf, &p->fr0, &p->fr1, &p->tcount, &p->tmask,
          &p->tscan0, &p->tscan1, &p->tscan2, &p->p2p_raw, &p->m2l_raw, &p->lk0, &p->lk1, &p->lv0, &p->lv1,
          &p->p2p_sorted, &p->p2p_off, &p->m2l_key, &p->m2l_slot, &p->ukeys, &p->T32, &p->Tbf,
          &p->tmiss_keys, &p->tmiss_slots, &p->tslot_map, &p->st_tile, &p->st_slot, &p->st_src, &p->bin_flag, &p->bin_scan, &p->bin_flag2, &p->bin_scan2, &p->st_ckey,
          &p->st_fkey, &p->m2l_items, &p->m2l_partial, &p->tile_range, &p->scan_tmp, &p->sort_hist, &p->scal,
          &p->flags, &p->seg_off, &p->seg_box, &p->seg_sig, &p->seg_smax, &p->seg_mac, &p->seg_p2p, &p->c_seg};
}

struct Timer {
  fmm_plan p;
  cudaStream_t s;
  int k = 0;
  void mark() { mark_on(s); }
  void mark_on(cudaStream_t st) {
    if (p->timing && k < 8) cudaEventRecord(p->ev[k++], st);
  }
};

// The plan's second stream and its fork / join events (created on the plan's
// device by its first evaluation).
int ensure_aux_stream(fmm_plan p) {
  if (p->s_up) return FMM_OK;
  FMM_CUDA_TRY(cudaStreamCreateWithFlags(&p->s_up, cudaStreamNonBlocking));
  FMM_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  FMM_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  return FMM_OK;
}

// sg: nullptr for one problem, else the (non-empty) problems of a batch.
int eval_device(fmm_plan p, int64_t n, const float* pos, const float* gam, const float* sig, float sig_u, float* vel,
                float* dg, cudaStream_t s, const SegSpec* sg = nullptr) {
  if (n < 0 || n > p->n_max) return FMM_E_INVAL;
  if (n > 0 && (!pos || !gam)) return FMM_E_INVAL;
  if (!sg && !sig && !(sig_u > 0.f)) return FMM_E_INVAL;
  memset(&p->stats, 0, sizeof(p->stats));
  p->last_n = n;
  p->reuse_ok = 0;
  ++p->epoch;
  p->ncells = p->nleaves = 0;
  p->n_p2p = p->n_m2l = p->n_keys = p->n_steps = p->p2p_pairs = 0;
  p->level_begin.clear();
  if (n == 0) return FMM_OK;
  FMM_CUDA_TRY(cudaSetDevice(p->device));
  FMM_CUDA_TRY(cudaMemsetAsync(p->flags.ptr, 0, sizeof(int) * 4, s));
  const int m2l_kind = p->prm.m2l_mode & 3;
  p->last_tc = (m2l_kind == FMM_M2L_SIMT) ? 0 : p->tc_ok;
  if ((m2l_kind == FMM_M2L_TENSOR || m2l_kind == FMM_M2L_TENSOR_TF32) && !p->tc_ok) return FMM_E_INVAL;
  Timer tm{p, s};
  tm.mark();
  if (sg) FMM_TRY(build_forest(p, n, pos, gam, sig, *sg, s));
  else FMM_TRY(build_tree(p, n, pos, gam, sig, sig_u, s));
  tm.mark();
  // Fork: P2M / M2M on the plan's second stream while the traversal (which
  // reads only the tree) runs on the caller's stream; join before M2L.
  FMM_TRY(ensure_aux_stream(p));
  FMM_CUDA_TRY(cudaEventRecord(p->ev_fork, s));
  FMM_CUDA_TRY(cudaStreamWaitEvent(p->s_up, p->ev_fork, 0));
  {
    int urc = upward_pass(p, p->s_up);
    if (urc == FMM_OK) urc = dipole_pass(p, n, p->s_up);
    if (urc != FMM_OK) {
      cudaStreamSynchronize(p->s_up);
      return urc;
    }
  }
  tm.mark_on(p->s_up);
  FMM_CUDA_TRY(cudaEventRecord(p->ev_join, p->s_up));
  // from here on an early return must not leave the upward pass running
  struct JoinOnExit {
    fmm_plan p;
    cudaStream_t s;
    bool joined = false;
    ~JoinOnExit() {
      if (!joined) cudaStreamSynchronize(p->s_up);
    }
  } join_guard{p, s};
  double smax = (double)sig_u;
  if (sg) {
    FMM_TRY(segment_tables(p, sig ? 1 : 0, s));
  } else if (sig) {
    unsigned int bits = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&bits, p->scal.as<double>() + kScalSigma, sizeof(unsigned int),
                                 cudaMemcpyDeviceToHost, s));
    FMM_CUDA_TRY(cudaStreamSynchronize(s));
    float f;
    memcpy(&f, &bits, sizeof(f));
    smax = (double)f;
  }
  FMM_TRY(traverse(p, smax, s));
  FMM_TRY(build_m2l_operators(p, s));
  tm.mark();
  FMM_CUDA_TRY(cudaStreamWaitEvent(s, p->ev_join, 0));
  join_guard.joined = true;
  const int nc = (int)p->ncells;
  FMM_TRY(p->L.ensure((size_t)nc * 3 * p->P * sizeof(float)));
  FMM_CUDA_TRY(cudaMemsetAsync(p->L.ptr, 0, (size_t)nc * 3 * p->P * sizeof(float), s));
  if (p->last_tc) FMM_TRY(m2l_tensor(p, s));
  else FMM_TRY(m2l_simt(p, s));
  FMM_TRY(apply_lattice(p, s));
  tm.mark();
  FMM_TRY(downward_pass(p, n, s));
  tm.mark();
  FMM_TRY(p2p_near(p, n, sig_u, sig ? 1 : 0, smax, vel, dg, s));
  tm.mark();
  // error flags raised by kernels
  int hf = 0;
  FMM_CUDA_TRY(cudaMemcpyAsync(p->pinned, p->flags.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(p->pinned) + 128, p->scal.as<double>() + kScalCount + 4,
                               3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  memcpy(&hf, p->pinned, sizeof(int));
  unsigned long long cls[3];
  memcpy(cls, reinterpret_cast<char*>(p->pinned) + 128, sizeof(cls));
  if (hf != 0) return hf;
  p->reuse_ok = 1;
  p->reuse_ps = sig ? 1 : 0;
  p->reuse_sig_u = sig_u;
  p->reuse_smax = smax;
  fmm_stats& st = p->stats;
  st.n = n;
  st.ncells = p->ncells;
  st.nleaves = p->nleaves;
  st.nlevels = p->nlevels;
  st.m2l_tensor = p->last_tc;
  st.p2p_cell_pairs = p->n_p2p;
  st.p2p_pairs = p->p2p_pairs;
  st.m2l_pairs = p->n_m2l;
  st.m2l_steps = p->n_steps;
  st.m2l_keys = p->n_keys;
  st.m2l_built = p->n_built;
  st.traversal_runs = p->trav_runs;
  st.m2l_split_coefs =
      p->last_tc ? std::min<int64_t>(p->P, (int64_t)4 * m2l_kstep(p->tc_kind) *
                                                m2l_split_chunks(p->P, p->tc_kind, p->prm.theta,
                                                                 p->prm.m2l_mode & FMM_M2L_FULL_SPLIT))
                  : 0;
  st.m2l_stage_chunks = p->last_tc ? p->m2l_stage_chunks : 0;
  st.p2p_pairs_near = (int64_t)cls[0];
  st.p2p_pairs_mid = (int64_t)cls[1];
  st.p2p_pairs_far = (int64_t)cls[2];
  if (p->timing && tm.k == 7) {
    float ms[6];
    for (int i = 0; i < 6; ++i) cudaEventElapsedTime(&ms[i], p->ev[i], p->ev[i + 1]);
    st.ms_tree = ms[0];
    st.ms_upward = ms[1];
    float trav = 0.f;  // the traversal starts with the upward pass (they overlap)
    cudaEventElapsedTime(&trav, p->ev[1], p->ev[3]);
    st.ms_traverse = trav;
    st.ms_m2l = ms[3];
    st.ms_downward = ms[4];
    st.ms_p2p = ms[5];
    float tot = 0.f;
    cudaEventElapsedTime(&tot, p->ev[0], p->ev[6]);
    st.ms_total = tot;
  }
  return FMM_OK;
}

}  // namespace

extern "C" {

void fmm_params_default(fmm_params* q) {
  if (!q) return;
  memset(q, 0, sizeof(*q));
  q->p = 10;
  q->theta = 0.4f;
  q->ncrit = 64;
  q->periodic = 0;
  q->images = 3;
  q->box_min[0] = q->box_min[1] = q->box_min[2] = 0.0;
  q->box_len = 1.0;
  q->sigma_sep = 5.0f;
  q->outputs = FMM_OUT_VELOCITY | FMM_OUT_STRETCHING;
  q->sigma_rule = FMM_SIGMA_SOURCE;
  q->p2p_pair_max = 0;
  q->split_tie = FMM_SPLIT_SOURCE;
  q->m2l_mode = FMM_M2L_AUTO;
}

const char* fmm_strerror(int code) {
  switch (code) {
    case FMM_OK: return "ok";
    case FMM_E_INVAL: return "invalid argument";
    case FMM_E_NOMEM: return "out of memory";
    case FMM_E_CAPACITY: return "internal list capacity exceeded";
    case FMM_E_TIMEOUT: return "bounded device wait timed out";
    case FMM_E_DEPTH: return "translation vector outside the encodable range";
    case FMM_E_CUDA: return "CUDA runtime error";
    default: return "unknown error";
  }
}

int fmm_plan_create(const fmm_params* prm, int64_t n_max, fmm_plan* out) {
  if (!out || n_max < 0 || n_max > 0x7fffffffll) return FMM_E_INVAL;
  FMM_TRY(check_params(prm));
  fmm_plan p = new (std::nothrow) fmm_plan_s();
  if (!p) return FMM_E_NOMEM;
  p->prm = *prm;
  p->n_max = n_max;
  p->P = prm->p * prm->p;
  p->Kpad = 128;
  p->tc_ok = 1;  // tcgen05 M2L: one CTA per 128 output rows (two for p > 11)
  p->tc_kind = (prm->m2l_mode & 3) == FMM_M2L_TENSOR_TF32 ? 1 : 0;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return FMM_E_CUDA;
  }
  int rc = FMM_OK;
  size_t nn = (size_t)std::max<int64_t>(n_max, 1);
  do {
    if ((rc = build_constant_operators(p)) != FMM_OK) break;
    if ((rc = p->keys0.ensure(nn * 8)) || (rc = p->keys1.ensure(nn * 8)) || (rc = p->vals0.ensure(nn * 4)) ||
        (rc = p->vals1.ensure(nn * 4)) || (rc = p->sortA.ensure(nn * 16)) || (rc = p->sortB.ensure(nn * 16)) ||
        (rc = p->leaf_of.ensure(nn * 4)) || (rc = p->scal.ensure(64 * sizeof(double))) ||
        (rc = p->flags.ensure(16 * sizeof(int))))
      break;
    if (cudaMallocHost(&p->pinned, 4096) != cudaSuccess) {
      rc = FMM_E_NOMEM;
      break;
    }
    for (int i = 0; i < 8; ++i) cudaEventCreate(&p->ev[i]);
    p->have_events = 1;
    cudaMemset(p->scal.ptr, 0, 64 * sizeof(double));
    if (cudaDeviceSynchronize() != cudaSuccess) rc = FMM_E_CUDA;
  } while (0);
  if (rc != FMM_OK) {
    fmm_plan_destroy(p);
    return rc;
  }
  *out = p;
  return FMM_OK;
}

void fmm_plan_destroy(fmm_plan p) {
  if (!p) return;
  cudaDeviceSynchronize();
  for (DBuf* b : plan_buffers(p)) b->release();
  if (p->pinned) cudaFreeHost(p->pinned);
  if (p->seg_pinned) cudaFreeHost(p->seg_pinned);
  if (p->have_events)
    for (int i = 0; i < 8; ++i) cudaEventDestroy(p->ev[i]);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->s_up) cudaStreamDestroy(p->s_up);
  delete p;
}

int64_t fmm_plan_device_bytes(fmm_plan p) {
  if (!p) return 0;
  int64_t t = 0;
  for (DBuf* b : plan_buffers(p)) t += (int64_t)b->bytes;
  return t;
}

int fmm_eval_batch(fmm_plan p, int32_t nprob, const int64_t* offsets, const float* pos, const float* gam,
                   const float* sig, const float* sigma_prob, const double* boxes, float* vel, float* dg,
                   void* stream) {
  if (!p || nprob < 0 || nprob > FMM_BATCH_MAX || (nprob > 0 && !offsets)) return FMM_E_INVAL;
  if (nprob == 0) return eval_device(p, 0, pos, gam, sig, 1.f, vel, dg, (cudaStream_t)stream);
  if (offsets[0] != 0) return FMM_E_INVAL;
  for (int i = 0; i < nprob; ++i)
    if (offsets[i + 1] < offsets[i]) return FMM_E_INVAL;
  const int64_t n = offsets[nprob];
  if (n > p->n_max) return FMM_E_INVAL;
  if (n == 0) return eval_device(p, 0, pos, gam, sig, 1.f, vel, dg, (cudaStream_t)stream);
  if (!sig && !sigma_prob) return FMM_E_INVAL;
  if (p->prm.periodic && !boxes) return FMM_E_INVAL;
  // the non-empty problems, in order
  std::vector<int> off(1, 0);
  std::vector<float> sg_sig;
  std::vector<double> sg_box;
  for (int i = 0; i < nprob; ++i) {
    if (offsets[i + 1] == offsets[i]) continue;
    if (!sig) {
      if (!(sigma_prob[i] > 0.f) || !std::isfinite(sigma_prob[i])) return FMM_E_INVAL;
      sg_sig.push_back(sigma_prob[i]);
    }
    if (p->prm.periodic) {
      if (!(boxes[4 * i + 3] > 0.0)) return FMM_E_INVAL;
      for (int q = 0; q < 4; ++q) sg_box.push_back(boxes[4 * i + q]);
    }
    off.push_back((int)offsets[i + 1]);
  }
  SegSpec spec;
  spec.nseg = (int)off.size() - 1;
  spec.h_off = off.data();
  spec.h_sigma = sig ? nullptr : sg_sig.data();
  spec.h_box = p->prm.periodic ? sg_box.data() : nullptr;
  return eval_device(p, n, pos, gam, sig, 0.f, vel, dg, (cudaStream_t)stream, spec.nseg > 0 ? &spec : nullptr);
}

int fmm_eval_velocity_stretching(fmm_plan p, int64_t n, const float* pos, const float* gam, const float* sig,
                                 float sig_u, float* vel, float* dg, void* stream) {
  if (!p) return FMM_E_INVAL;
  return eval_device(p, n, pos, gam, sig, sig_u, vel, dg, (cudaStream_t)stream);
}

int fmm_eval_velocity_stretching_host(fmm_plan p, int64_t n, const float* pos, const float* gam, const float* sig,
                                      float sig_u, float* vel, float* dg, void* stream) {
  if (!p || n < 0 || n > p->n_max) return FMM_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  size_t b3 = (size_t)std::max<int64_t>(n, 1) * 3 * sizeof(float);
  FMM_TRY(p->in_pos.ensure(b3));
  FMM_TRY(p->in_gam.ensure(b3));
  FMM_TRY(p->out_vel.ensure(b3));
  FMM_TRY(p->out_dg.ensure(b3));
  if (sig) FMM_TRY(p->in_sig.ensure((size_t)std::max<int64_t>(n, 1) * sizeof(float)));
  if (n > 0) {
    FMM_CUDA_TRY(cudaMemcpyAsync(p->in_pos.ptr, pos, (size_t)n * 12, cudaMemcpyHostToDevice, s));
    FMM_CUDA_TRY(cudaMemcpyAsync(p->in_gam.ptr, gam, (size_t)n * 12, cudaMemcpyHostToDevice, s));
    if (sig) FMM_CUDA_TRY(cudaMemcpyAsync(p->in_sig.ptr, sig, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  }
  FMM_TRY(eval_device(p, n, p->in_pos.as<float>(), p->in_gam.as<float>(), sig ? p->in_sig.as<float>() : nullptr,
                      sig_u, vel ? p->out_vel.as<float>() : nullptr, dg ? p->out_dg.as<float>() : nullptr, s));
  if (n > 0) {
    if (vel) FMM_CUDA_TRY(cudaMemcpyAsync(vel, p->out_vel.ptr, (size_t)n * 12, cudaMemcpyDeviceToHost, s));
    if (dg) FMM_CUDA_TRY(cudaMemcpyAsync(dg, p->out_dg.ptr, (size_t)n * 12, cudaMemcpyDeviceToHost, s));
  }
  FMM_CUDA_TRY(cudaStreamSynchronize(s));
  return FMM_OK;
}

int fmm_direct_velocity_stretching(int64_t n, const float* pos, const float* gam, const float* sig, float sig_u,
                                   float* vel, float* dg, void* stream) {
  if (n < 0 || (n > 0 && (!pos || !gam))) return FMM_E_INVAL;
  if (!sig && !(sig_u > 0.f)) return FMM_E_INVAL;
  if (n == 0) return FMM_OK;
  return p2p_direct_all(n, pos, gam, sig, sig_u, vel, dg, (cudaStream_t)stream);
}

int64_t fmm_kernel_launch_count(void) { return fmm::g_launches; }

int fmm_lattice_operator(int32_t p, int32_t images, int32_t on_device, double* out) {
  if (p < 1 || p > kPMax || images < 1 || images > 8 || !out) return FMM_E_INVAL;
  const size_t bytes = (size_t)p * p * p * p * sizeof(double);
  if (!on_device) return lattice_operator_host(p, images, out);
  DBuf A;
  int rc = A.ensure(bytes);
  if (rc == FMM_OK) rc = lattice_operator_device(p, images, A.as<double>(), 0);
  if (rc == FMM_OK && cudaMemcpy(out, A.ptr, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) rc = FMM_E_CUDA;
  A.release();
  return rc;
}

int fmm_plan_set_list_capacity(fmm_plan p, int64_t frontier, int64_t m2l, int64_t p2p) {
  if (!p || frontier < 0 || m2l < 0 || p2p < 0) return FMM_E_INVAL;
  p->cap_fr0 = frontier;
  p->cap_m0 = m2l;
  p->cap_p0 = p2p;
  return FMM_OK;
}

int fmm_plan_set_timing(fmm_plan p, int enable) {
  if (!p) return FMM_E_INVAL;
  p->timing = enable ? 1 : 0;
  return FMM_OK;
}

int fmm_plan_get_stats(fmm_plan p, fmm_stats* out) {
  if (!p || !out) return FMM_E_INVAL;
  *out = p->stats;
  return FMM_OK;
}

int fmm_plan_get_order(fmm_plan p, uint32_t* order, uint64_t* keys) {
  if (!p) return FMM_E_INVAL;
  FMM_CUDA_TRY(cudaDeviceSynchronize());
  int64_t n = p->last_n;
  if (n == 0) return FMM_OK;
  if (order) FMM_CUDA_TRY(cudaMemcpy(order, p->sidx, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (keys) FMM_CUDA_TRY(cudaMemcpy(keys, p->skeys, n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  return FMM_OK;
}

int fmm_plan_get_cells(fmm_plan p, int32_t* begin, int32_t* end, int32_t* level, int32_t* parent,
                       int32_t* child_begin, int32_t* nchild, double* center, double* radius) {
  if (!p) return FMM_E_INVAL;
  FMM_CUDA_TRY(cudaDeviceSynchronize());
  size_t nc = (size_t)p->ncells;
  if (nc == 0) return FMM_OK;
  if (begin) FMM_CUDA_TRY(cudaMemcpy(begin, p->c_begin.ptr, nc * 4, cudaMemcpyDeviceToHost));
  if (end) FMM_CUDA_TRY(cudaMemcpy(end, p->c_end.ptr, nc * 4, cudaMemcpyDeviceToHost));
  if (level) FMM_CUDA_TRY(cudaMemcpy(level, p->c_level.ptr, nc * 4, cudaMemcpyDeviceToHost));
  if (parent) FMM_CUDA_TRY(cudaMemcpy(parent, p->c_parent.ptr, nc * 4, cudaMemcpyDeviceToHost));
  if (child_begin) FMM_CUDA_TRY(cudaMemcpy(child_begin, p->c_child.ptr, nc * 4, cudaMemcpyDeviceToHost));
  if (nchild) FMM_CUDA_TRY(cudaMemcpy(nchild, p->c_nchild.ptr, nc * 4, cudaMemcpyDeviceToHost));
  if (center) FMM_CUDA_TRY(cudaMemcpy(center, p->c_center.ptr, nc * 24, cudaMemcpyDeviceToHost));
  if (radius) FMM_CUDA_TRY(cudaMemcpy(radius, p->c_radius.ptr, nc * 8, cudaMemcpyDeviceToHost));
  return FMM_OK;
}

int fmm_plan_get_lists(fmm_plan p, int32_t* p2p, int32_t* m2l) {
  if (!p) return FMM_E_INVAL;
  FMM_CUDA_TRY(cudaDeviceSynchronize());
  if (p2p && p->n_p2p) {
    std::vector<int4> h(p->n_p2p);
    FMM_CUDA_TRY(cudaMemcpy(h.data(), p->p2p_raw.ptr, p->n_p2p * sizeof(int4), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < p->n_p2p; ++i) {
      p2p[3 * i] = h[i].x;
      p2p[3 * i + 1] = h[i].y;
      p2p[3 * i + 2] = h[i].z;
    }
  }
  if (m2l && p->n_m2l) {  // 8-byte records: (target, source | image << 27)
    std::vector<int2> h(p->n_m2l);
    FMM_CUDA_TRY(cudaMemcpy(h.data(), p->m2l_raw.ptr, p->n_m2l * sizeof(int2), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < p->n_m2l; ++i) {
      m2l[3 * i] = h[i].x;
      m2l[3 * i + 1] = h[i].y & ((1 << 27) - 1);
      m2l[3 * i + 2] = (int32_t)((uint32_t)h[i].y >> 27);
    }
  }
  return FMM_OK;
}

}  // extern "C"
