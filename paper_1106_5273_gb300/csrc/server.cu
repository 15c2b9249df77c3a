// Serving loop over the batched evaluation: request queue, worker threads
// with their own streams and device-resident plans, continuous batching by
// (p, periodic) class in arrival order, and admission by a device-memory
// budget.  Host code only; every step of an evaluation runs in the kernels of
// fmm_eval_batch / fmm_eval_velocity_stretching.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fmm_internal.cuh"

namespace {

// Workspace model of a class (bytes an evaluation of n particles adds to a
// fresh plan): fixed + per_particle * n.  Until measured: 256 MiB (translation
// operator cache, lists of a small tree) + 2 KiB per particle.
constexpr double kDefaultFixed = 256.0 * 1048576.0;
constexpr double kDefaultPerParticle = 2048.0;
constexpr int64_t kSmallBatch = 65536;           // batches below this size measure the fixed part
constexpr int64_t kPlanBytesPerCapacity = 64;    // allocated at plan creation per particle of n_max
constexpr int64_t kIoBytesPerParticle = 48;      // pos, gamma, vel, dgamma staging

struct Model {
  double fixed = kDefaultFixed, per = kDefaultPerParticle;
  bool have_small = false, have_big = false;
};

struct Req {
  fmm_request r;
  fmm_request_result res;
  bool done = false;
  int retries = 0;  // batches of this request refused by the byte budget
};

constexpr int kMaxRetries = 4;

struct PlanRec {
  fmm_plan plan = nullptr;
  int64_t base = 0;       // device bytes right after creation
  int64_t n_seen = 0;     // largest batch evaluated with it
};

struct Worker {
  int id = 0;
  std::thread th;
  cudaStream_t stream = nullptr;
  std::map<int, PlanRec> plans;  // class -> plan
  fmm::DBuf d_pos, d_gam, d_vel, d_dg;
  int64_t held = 0;   // device bytes accounted to this worker (plans + staging)
  bool busy = false;
};

int class_of(const fmm_request& r) { return r.p * 2 + (r.periodic ? 1 : 0); }

int64_t plan_bytes(fmm_plan p) { return p ? fmm_plan_device_bytes(p) : 0; }

}  // namespace

struct fmm_server_s {
  fmm_server_params prm;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Req> reqs;
  int64_t next_ticket = 1;
  bool stop = false;
  std::vector<Worker*> workers;
  int64_t held_total = 0;
  std::map<int, Model> model;  // workspace model by class, learned from evaluations
  std::map<int, int> tuned;    // autotuned leaf capacity by class (server ncrit = 0)
  int mem_waiters = 0;
  int probing = 0;  // a first batch of a class is running
  fmm_server_counters ctr{};
  // every device byte the workers allocate is charged here first; an
  // allocation past hbm_budget_bytes fails (FMM_E_NOMEM) instead of happening
  fmm::ByteBudget budget;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Plans are created for max_batch_particles (or the one larger request) and
// kept, so evaluations do not reallocate.
int64_t new_plan_capacity(fmm_server S, int64_t n) { return std::max<int64_t>(n, S->prm.max_batch_particles); }

// Bytes a worker will hold after running a batch of `n` particles of class c:
// its other plans, this class's plan (creation bytes + the workspace model)
// and the staging buffers.
Model initial_model(fmm_server S) {
  Model m;
  if (S->prm.model_bytes_per_particle > 0) m.per = (double)S->prm.model_bytes_per_particle;
  return m;
}

int64_t projected(fmm_server S, Worker* W, int c, int64_t n) {
  const Model m = S->model.count(c) ? S->model[c] : initial_model(S);
  int64_t other_plans = 0, cur = 0, base = kPlanBytesPerCapacity * new_plan_capacity(S, n);
  for (auto& kv : W->plans) {
    if (kv.first == c) {
      cur = plan_bytes(kv.second.plan);
      if (kv.second.plan->n_max >= n) base = kv.second.base;
    } else {
      other_plans += plan_bytes(kv.second.plan);
    }
  }
  const int64_t io = std::max<int64_t>((int64_t)W->d_pos.bytes * 4, n * kIoBytesPerParticle);
  return other_plans + std::max<int64_t>(cur, base + (int64_t)(m.fixed + m.per * (double)n)) + io;
}

void recount(fmm_server S, Worker* W) {
  int64_t h = (int64_t)(W->d_pos.bytes + W->d_gam.bytes + W->d_vel.bytes + W->d_dg.bytes);
  for (auto& kv : W->plans) h += plan_bytes(kv.second.plan);
  S->held_total += h - W->held;
  W->held = h;
  S->ctr.peak_bytes = std::max(S->ctr.peak_bytes, S->held_total);
}

// Free an idle worker's plans except class `keep` (-1: all).  Caller holds the lock.
void drop_plans(fmm_server S, Worker* W, int keep) {
  for (auto it = W->plans.begin(); it != W->plans.end();) {
    if (it->first == keep) {
      ++it;
      continue;
    }
    fmm_plan_destroy(it->second.plan);
    it = W->plans.erase(it);
  }
  recount(S, W);
}

constexpr int32_t kTuneCandidates[] = {32, 48, 64, 96, 128, 192, 256};

// One batch on the worker's stream; the lock is not held.  ncrit = 0: the
// class has no tuned leaf capacity yet; this batch measures it (*ncrit_out).
int run_batch(fmm_server S, Worker* W, std::vector<fmm_request>& rs, int64_t ntot, PlanRec* rec, int ncrit,
              int* ncrit_out) {
  const cudaStream_t st = W->stream;
  fmm_plan& plan = rec->plan;
  const fmm_request& r0 = rs[0];
  fmm_params q;
  fmm_params_default(&q);
  q.p = r0.p;
  q.theta = S->prm.theta;
  // ncrit: the leaf capacity, with an autotuned P2P tile in bits 16 and up
  q.ncrit = ncrit > 0 ? (ncrit & 0xffff) : 64;
  q.p2p_tpl = ncrit > 0 ? (ncrit >> 16) : 0;
  q.sigma_sep = S->prm.sigma_sep;
  q.images = S->prm.images;
  q.m2l_mode = S->prm.m2l_mode;
  q.periodic = r0.periodic ? 1 : 0;
  if (r0.periodic) {
    for (int k = 0; k < 3; ++k) q.box_min[k] = r0.box[k];
    q.box_len = r0.box[3];
  }
  *ncrit_out = ncrit;
  const size_t b3 = (size_t)std::max<int64_t>(ntot, 1) * 3 * sizeof(float);
  FMM_TRY(W->d_pos.ensure(b3));
  FMM_TRY(W->d_gam.ensure(b3));
  FMM_TRY(W->d_vel.ensure(b3));
  FMM_TRY(W->d_dg.ensure(b3));
  std::vector<int64_t> off(rs.size() + 1, 0);
  std::vector<float> sig(rs.size());
  std::vector<double> box(rs.size() * 4);
  for (size_t k = 0; k < rs.size(); ++k) {
    off[k + 1] = off[k] + rs[k].n;
    sig[k] = rs[k].sigma;
    for (int q = 0; q < 4; ++q) box[4 * k + q] = rs[k].box[q];
  }
  float* dp = W->d_pos.as<float>();
  float* dg = W->d_gam.as<float>();
  float* dv = W->d_vel.as<float>();
  float* ds = W->d_dg.as<float>();
  for (size_t k = 0; k < rs.size(); ++k) {
    if (rs[k].n == 0) continue;
    FMM_CUDA_TRY(cudaMemcpyAsync(dp + 3 * off[k], rs[k].pos, (size_t)rs[k].n * 12, cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(dg + 3 * off[k], rs[k].gamma, (size_t)rs[k].n * 12, cudaMemcpyHostToDevice, st));
  }
  if (ncrit == 0 && ntot > 0) {  // first batch of the class: measure leaf capacity and P2P tile on it
    int32_t best = 64, best_tpl = 0;
    const int32_t tpls[2] = {1, 2};
    FMM_TRY(fmm_autotune_plan(&q, (int32_t)rs.size(), off.data(), dp, dg, sig.data(),
                              r0.periodic ? box.data() : nullptr, kTuneCandidates,
                              (int32_t)(sizeof(kTuneCandidates) / sizeof(kTuneCandidates[0])), tpls, 2, 1, &best,
                              &best_tpl, nullptr, st));
    q.ncrit = best;
    q.p2p_tpl = best_tpl;
    *ncrit_out = best | (best_tpl << 16);
  }
  if (plan && (plan->n_max < ntot || plan->prm.ncrit != q.ncrit || plan->prm.p2p_tpl != q.p2p_tpl)) {
    fmm_plan_destroy(plan);
    plan = nullptr;
  }
  if (!plan) {
    rec->n_seen = 0;
    FMM_TRY(fmm_plan_create(&q, new_plan_capacity(S, ntot), &plan));
    rec->base = plan_bytes(plan);
  }
  if (S->prm.batching) {
    FMM_TRY(fmm_eval_batch(plan, (int32_t)rs.size(), off.data(), dp, dg, nullptr, sig.data(),
                           r0.periodic ? box.data() : nullptr, dv, ds, st));
  } else {
    if (r0.periodic) {  // the one-problem path takes the cube from the plan
      for (int k = 0; k < 3; ++k) plan->prm.box_min[k] = r0.box[k];
      plan->prm.box_len = r0.box[3];
    }
    FMM_TRY(fmm_eval_velocity_stretching(plan, ntot, dp, dg, nullptr, r0.sigma, dv, ds, st));
  }
  for (size_t k = 0; k < rs.size(); ++k) {
    if (rs[k].n == 0) continue;
    if (rs[k].vel)
      FMM_CUDA_TRY(cudaMemcpyAsync(rs[k].vel, dv + 3 * off[k], (size_t)rs[k].n * 12, cudaMemcpyDeviceToHost, st));
    if (rs[k].dgamma)
      FMM_CUDA_TRY(cudaMemcpyAsync(rs[k].dgamma, ds + 3 * off[k], (size_t)rs[k].n * 12, cudaMemcpyDeviceToHost, st));
  }
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  return FMM_OK;
}

void worker_loop(fmm_server S, Worker* W) {
  cudaSetDevice(S->device);
  fmm::set_thread_budget(&S->budget);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
    if (S->queue.empty()) {
      if (S->stop) break;
      continue;
    }
    // ---- form a batch: the oldest request, then later ones of its class.
    // Requests that an idle worker can start right away are left to it: a
    // batch takes at most (queued requests - idle other workers), so batches
    // form only from requests that would otherwise wait (below saturation a
    // small request does not wait behind a large one in the same batch).
    int idle_others = 0;
    for (Worker* o : S->workers) idle_others += (o != W && !o->busy) ? 1 : 0;
    const int max_prob =
        S->prm.batching ? std::max(1, std::min(S->prm.max_batch_problems, (int)S->queue.size() - idle_others)) : 1;
    const int64_t budget = S->prm.hbm_budget_bytes;
    std::vector<int64_t> batch;
    int64_t ntot = 0;
    int c = -1;
    bool waited = false;
    for (;;) {
      batch.clear();
      ntot = 0;
      if (S->queue.empty()) break;
      c = class_of(S->reqs[S->queue.front()].r);
      const int64_t others = S->held_total - W->held;
      for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        const fmm_request& q = S->reqs[*it].r;
        if (class_of(q) != c) continue;
        if (!batch.empty()) {
          if ((int)batch.size() >= max_prob || ntot + q.n > S->prm.max_batch_particles) break;
          if (others + projected(S, W, c, ntot + q.n) > budget) break;
        }
        batch.push_back(*it);
        ntot += q.n;
        if (!S->prm.batching) break;
      }
      // the first batch of a class runs alone, so that its footprint is
      // measured before anything is admitted on the strength of it
      bool busy_other = false;
      for (Worker* o : S->workers) busy_other |= (o != W && o->busy);
      if (S->probing || (!S->model.count(c) && busy_other)) {
        if (!waited) ++S->ctr.memory_waits;
        waited = true;
        S->cv_done.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      if (others + projected(S, W, c, ntot) <= budget) break;
      // the oldest request alone does not fit: free the idle plans of every
      // idle worker (this one keeps its plan of the class), then wait for the
      // busy ones, or give up when nothing else holds memory
      bool busy = false;
      for (Worker* o : S->workers) {
        if (o == W) continue;
        if (o->busy) busy = true;
        else if (!o->plans.empty()) drop_plans(S, o, -1);
      }
      if (S->held_total - W->held + projected(S, W, c, ntot) <= budget) continue;
      drop_plans(S, W, c);
      if (S->held_total - W->held + projected(S, W, c, ntot) <= budget) continue;
      if (!busy) {
        // Nothing else runs and nothing else is held: the request goes ahead
        // alone whatever the projection says.  The byte budget decides on its
        // actual allocations; a request it keeps refusing completes with
        // FMM_E_NOMEM (the refusal path after the batch).
        drop_plans(S, W, -1);
        break;
      }
      if (!waited) ++S->ctr.memory_waits;
      waited = true;
      ++S->mem_waiters;
      S->cv_done.wait_for(lk, std::chrono::milliseconds(20));
      --S->mem_waiters;
    }
    if (batch.empty()) continue;
    for (int64_t t : batch) S->queue.erase(std::find(S->queue.begin(), S->queue.end(), t));
    std::vector<fmm_request> rs;
    const double ts = S->now();
    for (int64_t t : batch) {
      Req& rq = S->reqs[t];
      rq.res.t_start = ts;
      rs.push_back(rq.r);
    }
    // reserve the projected bytes while the batch runs
    const int64_t proj = projected(S, W, c, ntot);
    S->held_total += proj - W->held;
    W->held = proj;
    S->ctr.peak_bytes = std::max(S->ctr.peak_bytes, S->held_total);
    W->busy = true;
    const bool probe = !S->model.count(c);
    if (probe) S->probing = 1;
    PlanRec rec = W->plans.count(c) ? W->plans[c] : PlanRec();
    const int ncrit = S->prm.ncrit > 0 ? S->prm.ncrit : (S->tuned.count(c) ? S->tuned[c] : 0);
    int ncrit_used = ncrit;
    lk.unlock();
    int rc = run_batch(S, W, rs, ntot, &rec, ncrit, &ncrit_used);
    lk.lock();
    if (rc == FMM_E_NOMEM && ntot > 0) {
      // An allocation of this batch was refused by the byte budget (or the
      // device is out of memory): the class's footprint was underestimated.
      // What the batch had allocated plus the refused allocation bounds its
      // need from below; the class's per-particle need is raised past that
      // (and by at least 25%), every idle plan is freed, and the requests go
      // back to the front of the queue, where the next batch is formed with
      // the larger need (fewer requests, or a wait for the other workers).
      // A request counts a refusal only when no other worker was running;
      // after kMaxRetries such refusals it completes with FMM_E_NOMEM.
      bool others_busy = false;
      for (Worker* o : S->workers) others_busy |= (o != W && o->busy);
      W->busy = false;
      if (probe) S->probing = 0;
      const int64_t grown = plan_bytes(rec.plan) - rec.base + fmm::ByteBudget::last_refused();
      if (rec.plan) W->plans[c] = rec;
      else W->plans.erase(c);
      Model& m = S->model.count(c) ? S->model[c] : (S->model[c] = initial_model(S));
      const double per_lb = ((double)grown - (m.have_small ? m.fixed : 0.0)) / (double)ntot;
      m.per = std::max(m.per * 1.25, 1.1 * per_lb);
      m.have_big = true;
      for (Worker* o : S->workers)
        if (o == W || !o->busy) drop_plans(S, o, -1);
      std::vector<int64_t> again;
      const double td = S->now();
      for (int64_t t : batch) {
        Req& rq = S->reqs[t];
        if (others_busy || ++rq.retries <= kMaxRetries) {
          again.push_back(t);
          continue;
        }
        rq.res.status = FMM_E_NOMEM;
        rq.res.batch_problems = (int32_t)batch.size();
        rq.res.batch_particles = ntot;
        rq.res.worker = W->id;
        rq.res.t_done = td;
        rq.done = true;
      }
      S->queue.insert(S->queue.begin(), again.begin(), again.end());
      ++S->ctr.memory_waits;
      S->cv_done.notify_all();
      S->cv_work.notify_all();
      continue;
    }
    if (rc == FMM_OK && ncrit_used > 0 && !S->tuned.count(c)) S->tuned[c] = ncrit_used;
    W->busy = false;
    if (probe) S->probing = 0;
    if (rec.plan) W->plans[c] = rec;
    else W->plans.erase(c);
    if (rc == FMM_OK && rec.plan && ntot > 0 && ntot >= rec.n_seen) {
      // the largest batch this plan has seen sets its workspace: small batches
      // bound the fixed part, large ones the part per particle (upper envelope)
      const double ws = (double)(plan_bytes(rec.plan) - rec.base);
      Model& m = S->model[c];
      if (ntot < kSmallBatch) {
        m.fixed = m.have_small ? std::max(m.fixed, ws) : ws;
        m.have_small = true;
      } else {
        const double b = (ws - (m.have_small ? m.fixed : 0.0)) / (double)ntot;
        m.per = m.have_big ? std::max(m.per, b) : std::max(b, 0.0);
        m.have_big = true;
        if (!m.have_small) m.fixed = 0.0;
      }
      W->plans[c].n_seen = ntot;
    }
    recount(S, W);
    if (S->mem_waiters > 0) drop_plans(S, W, -1);
    const double td = S->now();
    for (int64_t t : batch) {
      Req& rq = S->reqs[t];
      rq.res.status = rc;
      rq.res.batch_problems = (int32_t)batch.size();
      rq.res.batch_particles = ntot;
      rq.res.worker = W->id;
      rq.res.t_done = td;
      rq.done = true;
    }
    ++S->ctr.batches;
    S->ctr.requests += (int64_t)batch.size();
    S->ctr.particles += ntot;
    S->cv_done.notify_all();
  }
}

int check_request(const fmm_request* r) {
  if (!r || r->n < 0 || r->n > 0x7fffffffll || r->p < 1 || r->p > fmm::kPMax) return FMM_E_INVAL;
  if (!(r->sigma > 0.f) || !(r->sigma < 3.0e38f)) return FMM_E_INVAL;
  if (r->n > 0 && (!r->pos || !r->gamma)) return FMM_E_INVAL;
  if (r->periodic != 0 && r->periodic != 1) return FMM_E_INVAL;
  if (r->periodic && !(r->box[3] > 0.0)) return FMM_E_INVAL;
  return FMM_OK;
}

}  // namespace

extern "C" {

void fmm_server_params_default(fmm_server_params* q) {
  if (!q) return;
  memset(q, 0, sizeof(*q));
  q->workers = 2;
  q->batching = 1;
  q->hbm_budget_bytes = 64ll << 30;
  q->max_batch_particles = 16ll << 20;
  q->max_batch_problems = 4096;
  q->theta = 0.5f;
  q->ncrit = 64;
  q->sigma_sep = 5.f;
  q->images = 3;
  q->m2l_mode = FMM_M2L_AUTO;
}

int fmm_server_create(const fmm_server_params* prm, fmm_server* out) {
  if (!prm || !out) return FMM_E_INVAL;
  if (prm->workers < 1 || prm->workers > 16 || (prm->batching != 0 && prm->batching != 1)) return FMM_E_INVAL;
  if (prm->hbm_budget_bytes <= 0 || prm->max_batch_particles < 1) return FMM_E_INVAL;
  if (prm->max_batch_problems < 1 || prm->max_batch_problems > FMM_BATCH_MAX) return FMM_E_INVAL;
  fmm_params q;
  fmm_params_default(&q);
  q.theta = prm->theta;
  q.ncrit = prm->ncrit == 0 ? 64 : prm->ncrit;  // 0: autotuned per class
  q.sigma_sep = prm->sigma_sep;
  q.images = prm->images;
  q.m2l_mode = prm->m2l_mode;
  if (!(q.theta > 0.f && q.theta < 1.f) || q.ncrit < 1 || q.ncrit > 4096 || !(q.sigma_sep >= 0.f) ||
      q.images < 1 || q.images > 8 || (q.m2l_mode & ~(3 | FMM_M2L_SORT_STEPS | FMM_M2L_FULL_SPLIT | FMM_M2L_CHUNK_STAGES)))
    return FMM_E_INVAL;
  if (prm->model_bytes_per_particle < 0) return FMM_E_INVAL;
  fmm_server S = new (std::nothrow) fmm_server_s();
  if (!S) return FMM_E_NOMEM;
  S->prm = *prm;
  S->budget.limit = prm->hbm_budget_bytes;
  S->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return FMM_E_CUDA;
  }
  for (int w = 0; w < prm->workers; ++w) {
    Worker* W = new Worker();
    W->id = w;
    if (cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete W;
      fmm_server_destroy(S);
      return FMM_E_CUDA;
    }
    S->workers.push_back(W);
  }
  for (Worker* W : S->workers) W->th = std::thread(worker_loop, S, W);
  *out = S;
  return FMM_OK;
}

int fmm_server_submit(fmm_server S, const fmm_request* req, int64_t* ticket) {
  if (!S || !ticket) return FMM_E_INVAL;
  FMM_TRY(check_request(req));
  std::lock_guard<std::mutex> g(S->mu);
  if (S->stop) return FMM_E_INVAL;
  const int64_t t = S->next_ticket++;
  Req& rq = S->reqs[t];
  rq.r = *req;
  memset(&rq.res, 0, sizeof(rq.res));
  rq.res.t_submit = S->now();
  S->queue.push_back(t);
  *ticket = t;
  S->cv_work.notify_one();
  return FMM_OK;
}

int fmm_server_wait(fmm_server S, int64_t ticket, double timeout_s, fmm_request_result* out) {
  if (!S || !out) return FMM_E_INVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FMM_E_INVAL;
  auto ready = [&] { return S->reqs[ticket].done; };
  if (timeout_s < 0) S->cv_done.wait(lk, ready);
  else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return FMM_E_TIMEOUT;
  *out = S->reqs[ticket].res;
  S->reqs.erase(ticket);
  return FMM_OK;
}

double fmm_server_clock(fmm_server S) { return S ? S->now() : 0.0; }

int fmm_server_get_counters(fmm_server S, fmm_server_counters* out) {
  if (!S || !out) return FMM_E_INVAL;
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->ctr;
  out->peak_bytes = S->budget.peak.load();  // allocated bytes, never above the budget
  return FMM_OK;
}

void fmm_server_destroy(fmm_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (Worker* W : S->workers)
    if (W->th.joinable()) W->th.join();
  for (Worker* W : S->workers) {
    for (auto& kv : W->plans) fmm_plan_destroy(kv.second.plan);
    W->d_pos.release();
    W->d_gam.release();
    W->d_vel.release();
    W->d_dg.release();
    if (W->stream) cudaStreamDestroy(W->stream);
    delete W;
  }
  delete S;
}

}  // extern "C"
