// Serving engine: a request loop with HBM-budget admission and continuous
// batching over Levenberg-Marquardt solves (the serving form of the solver).
//
// Requests (grid warps / Poisson edits, mesh deformations) are queued by
// opt_server_submit_*; each opt_server_step
//   1. admits queued requests in arrival order while their estimated device
//      footprint fits in the budget (planning = opt_problem_create_*),
//   2. resets the new members' scalars and copies their unknowns in,
//   3. runs ONE LM outer iteration (PCGInit, `inner` PCG iterations, trial
//      energy, gain-ratio decision, conditional update) for every member in
//      one launch per phase (the batched kernels), so requests admitted at
//      different times overlap on the device,
//   4. reads the members' scalars and retires those that converged (relative
//      energy change below rel_tol after an accepted step) or reached the
//      outer-iteration cap: their unknowns are written back, their report is
//      stored for opt_server_poll, and their memory returns to the budget.
// Every member follows exactly the LM sequence of opt_solve_lm with the same
// parameters, so its result equals the one-at-a-time solve up to float
// rounding (batch reductions run per problem in the same order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "opt_gb300.h"
#include "opt_internal.cuh"
#include "opt_problem.h"

using namespace optgb;

namespace {

struct ServeReq {
  uint64_t ticket = 0;
  bool graph = false;
  opt_grid_desc gd{};
  opt_graph_desc md{};
  size_t est_bytes = 0;
  opt_problem* pb = nullptr;
  std::vector<double> hist;
  int outer_seen = 0;   // LM outer iterations done at the last step
  opt_report rep{};
  opt_status status = OPT_OK;
  int state = 0;   // 0 queued, 1 active, 2 finished
};

__global__ void k_serve_reset(Scalars* s, double lambda0) { scalars_reset(s, lambda0); }

size_t round32(size_t v) { return (v + 31) / 32 * 32; }

constexpr int kServeMaxRounds = 64;   // cap of opt_server_set_max_rounds

// Device bytes a planned problem allocates (planes, tables, reduction slots).
size_t estimate_grid(const opt_grid_desc& d, int tile_w) {
  const bool warp = d.kind == OPT_ARAP_WARP_2D;
  const size_t tw = tile_w ? tile_w : (d.W >= 128 ? 128 : 32);
  const size_t pl = ((size_t)d.W + tw - 1) / tw * tw * (size_t)d.H;
  // 128-pixel tiles also hold the single-reduction PCG's z and w buffers
  // (12 planes for a warp, 16 for Poisson)
  const size_t planes = warp ? (tw == 128 ? 38 : 24) : (tw == 128 ? 46 : 30);
  const size_t tiles = ((size_t)d.W + tw - 1) / tw * ((size_t)(d.H + 7) / 8);
  return planes * pl * 4 + (d.mask ? pl : 0) + tiles * 64 + (size_t)d.n_handles * 16 + (1 << 16);
}
size_t estimate_graph(const opt_graph_desc& d) {
  const size_t pl = round32((size_t)d.V);
  // 48 planes + the 3 + 2 float4 records per vertex, edges (sorted copy,
  // in-edge sources and positions), row pointers
  return 68 * pl * 4 + (size_t)d.E * 16 + 8 * pl + (size_t)d.n_handles * 16 + (1 << 16);
}

}  // namespace

struct opt_server {
  size_t budget = 0, used = 0;
  int max_active = 0;                // 0: admission by the budget alone
  int max_rounds = 1;                // LM outer iterations per step when no request waits
  opt_solve_params prm{};
  cudaStream_t st = nullptr;
  std::mutex mu;
  std::deque<ServeReq*> queue;
  std::vector<RoundRec> rbuf;        // round records of the last step
  std::vector<ServeReq*> active;
  std::unordered_map<uint64_t, std::unique_ptr<ServeReq>> reqs;
  uint64_t next_ticket = 1;
  opt_batch* batch = nullptr;
  bool dirty = true;
  opt_status inject = OPT_OK;        // test hook: the next batch rebuild fails with this status
  std::vector<Scalars> sbuf;

  ~opt_server() {
    if (batch) opt_batch_destroy(batch);
    for (auto& kv : reqs)
      if (kv.second->pb) opt_problem_destroy(kv.second->pb);
    if (st) cudaStreamDestroy(st);
  }
};

namespace {

opt_status submit(opt_server* s, ServeReq* r, uint64_t* ticket) {
  if (r->est_bytes > s->budget) return OPT_ERR_BUDGET;
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  if (ticket) *ticket = r->ticket;
  s->queue.push_back(r);
  s->reqs[r->ticket].reset(r);
  return OPT_OK;
}

void finish(opt_server* s, ServeReq* r, opt_status st) {
  r->status = st;
  r->state = 2;
  if (r->pb) {
    opt_problem_destroy(r->pb);
    r->pb = nullptr;
  }
  s->used -= std::min(s->used, r->est_bytes);
}

// Copies the member's working unknowns back to the caller's planes.
opt_status write_back(opt_problem* pb, cudaStream_t st) {
  return copy_planes_out(pb, pb->user_x, pb->x, pb->nx, st);
}

opt_status copy_in(opt_problem* pb, cudaStream_t st) {
  return copy_planes_in(pb, pb->x, pb->user_x, pb->nx, st);
}

// A rebuild or a round failed: every active request ends with `st` (its
// memory returns to the budget) and the batch is dropped, so the next step
// starts over from the queue instead of retrying the same rebuild forever.
opt_status fail_active(opt_server* s, opt_status st) {
  cudaStreamSynchronize(s->st);
  (void)cudaGetLastError();
  if (s->batch) {
    opt_batch_destroy(s->batch);
    s->batch = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (ServeReq* r : s->active) finish(s, r, st);
  s->active.clear();
  s->dirty = true;
  return st;
}

}  // namespace

extern "C" {

opt_status opt_server_create(size_t hbm_budget_bytes, const opt_solve_params* params, opt_server** out) {
  if (!out) return OPT_ERR_INVALID_ARG;
  *out = nullptr;
  if (hbm_budget_bytes == 0) return OPT_ERR_INVALID_ARG;
  std::unique_ptr<opt_server> s(new opt_server());
  if (params) s->prm = *params;
  else opt_solve_params_default(&s->prm);
  if (s->prm.outer < 1 || s->prm.inner < 0 || s->prm.materialized || s->prm.pcg_form < 0 || s->prm.pcg_form > 1)
    return OPT_ERR_INVALID_ARG;
  s->budget = hbm_budget_bytes;
  if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    return OPT_ERR_CUDA;
  }
  *out = s.release();
  return OPT_OK;
}

opt_status opt_server_destroy(opt_server* s) {
  if (!s) return OPT_OK;
  cudaStreamSynchronize(s->st);
  delete s;
  return OPT_OK;
}

opt_status opt_server_submit_grid(opt_server* s, const opt_grid_desc* d, uint64_t* ticket) {
  if (!s || !d || d->W < 1 || d->H < 1) return OPT_ERR_INVALID_ARG;
  ServeReq* r = new ServeReq();
  r->gd = *d;
  r->est_bytes = estimate_grid(*d, s->prm.tile_w);
  const opt_status st = submit(s, r, ticket);
  if (st != OPT_OK) delete r;
  return st;
}

opt_status opt_server_submit_graph(opt_server* s, const opt_graph_desc* d, uint64_t* ticket) {
  if (!s || !d || d->V < 1 || d->E < 0) return OPT_ERR_INVALID_ARG;
  ServeReq* r = new ServeReq();
  r->graph = true;
  r->md = *d;
  r->est_bytes = estimate_graph(*d);
  const opt_status st = submit(s, r, ticket);
  if (st != OPT_OK) delete r;
  return st;
}

opt_status opt_server_step(opt_server* s, int32_t* n_active, int32_t* n_queued) {
  if (!s) return OPT_ERR_INVALID_ARG;
  auto counts = [&](opt_status st) {
    if (n_active) *n_active = (int32_t)s->active.size();
    if (n_queued) {
      std::lock_guard<std::mutex> lk(s->mu);
      *n_queued = (int32_t)s->queue.size();
    }
    return st;
  };
  // 1. admission in arrival order under the budget
  std::vector<ServeReq*> admit;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->queue.empty() && s->used + s->queue.front()->est_bytes <= s->budget &&
           (s->max_active <= 0 || s->active.size() + admit.size() < (size_t)s->max_active)) {
      ServeReq* r = s->queue.front();
      s->queue.pop_front();
      s->used += r->est_bytes;
      admit.push_back(r);
    }
  }
  for (ServeReq* r : admit) {
    opt_status st = r->graph ? opt_problem_create_graph(&r->md, &s->prm, &r->pb)
                             : opt_problem_create_grid(&r->gd, &s->prm, &r->pb);
    if (st != OPT_OK) {
      std::lock_guard<std::mutex> lk(s->mu);
      finish(s, r, st);
      continue;
    }
    if (copy_in(r->pb, s->st) != OPT_OK) {
      std::lock_guard<std::mutex> lk(s->mu);
      finish(s, r, OPT_ERR_CUDA);
      continue;
    }
    k_serve_reset<<<1, 1, 0, s->st>>>(r->pb->d_s, s->prm.lambda0);
    r->state = 1;
    s->active.push_back(r);
    s->dirty = true;
  }
  // 2. one LM outer iteration of every member
  if (!s->active.empty()) {
    if (s->dirty) {
      cudaStreamSynchronize(s->st);
      if (s->batch) {
        opt_batch_destroy(s->batch);
        s->batch = nullptr;
      }
      std::vector<opt_problem*> ps;
      for (ServeReq* r : s->active) ps.push_back(r->pb);
      opt_status st = s->inject;
      s->inject = OPT_OK;
      if (st == OPT_OK) st = opt_batch_create(ps.data(), (int)ps.size(), &s->batch);
      if (st == OPT_OK) st = batch_prepare_round(s->batch, s->prm);
      if (st != OPT_OK) return counts(fail_active(s, st));
      s->dirty = false;
    }
    // One round when requests are waiting (they are admitted at the next
    // step); otherwise as many rounds as the admitted request closest to its
    // iteration cap has left (at most max_rounds), so that a lightly loaded
    // server does not synchronise after every outer iteration.  A member that
    // converges earlier idles through the remaining rounds (its kernels skip
    // finished problems).
    int rounds = 1, cap = 1;
    bool waiting;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      waiting = !s->queue.empty();
      cap = s->max_rounds;
    }
    if (!waiting && cap > 1) {
      int left = cap;
      for (const ServeReq* r : s->active) left = std::min(left, s->prm.outer - r->outer_seen);
      rounds = std::max(1, left);
    }
    if (batch_reserve_rounds(s->batch, rounds) != OPT_OK) rounds = 1;
    for (int k = 0; k < rounds; ++k) batch_enqueue_lm_round(s->batch, s->prm, s->st, k);
    if (cudaGetLastError() != cudaSuccess) return counts(fail_active(s, OPT_ERR_CUDA));
    const size_t n = s->active.size();
    s->sbuf.resize(n);
    s->rbuf.resize((size_t)rounds * n);
    opt_status st = batch_read_scalars(s->batch, s->sbuf.data(), s->rbuf.data(), rounds, s->st);
    if (st != OPT_OK) return counts(fail_active(s, st));
    // 3. the energies of the rounds each member ran; retire converged / capped members
    std::vector<ServeReq*> keep;
    for (size_t i = 0; i < n; ++i) {
      ServeReq* r = s->active[i];
      const Scalars& t = s->sbuf[i];
      const int live = std::min(rounds, std::max(0, t.outer_done - r->outer_seen));
      for (int k = 0; k < live; ++k) r->hist.push_back(s->rbuf[(size_t)k * n + i].E);
      r->outer_seen = t.outer_done;
      const bool capped = t.outer_done >= s->prm.outer;
      if (!t.done && !capped && !t.nonfinite && !t.timeout && !t.misaligned) {
        keep.push_back(r);
        continue;
      }
      // the final energy: after the member's last decision
      const RoundRec last = live > 0 ? s->rbuf[(size_t)(live - 1) * n + i]
                                     : RoundRec{t.E, t.E_trial, t.accept, t.outer_done};
      if (live == 0) r->hist.push_back(t.E);
      const double Ef = last.accept ? last.E_trial : last.E;
      r->hist.push_back(Ef);
      r->rep.outer_done = t.outer_done;
      r->rep.pcg_done = t.pcg_iters;
      r->rep.accepted = t.accepted_total;
      r->rep.converged = t.converged;
      r->rep.E0 = r->hist.front();
      r->rep.E_final = Ef;
      r->rep.lambda_final = t.lambda;
      r->rep.ms = 0.f;
      opt_status ws = write_back(r->pb, s->st);
      cudaStreamSynchronize(s->st);
      std::lock_guard<std::mutex> lk(s->mu);
      finish(s, r, t.timeout ? OPT_ERR_TIMEOUT : t.misaligned ? OPT_ERR_CUDA : (t.nonfinite ? OPT_ERR_NUMERIC : ws));
      s->dirty = true;
    }
    s->active.swap(keep);
  }
  return counts(OPT_OK);
}

opt_status opt_server_inject_rebuild_failure(opt_server* s, opt_status status) {
  if (!s || status == OPT_OK) return OPT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->inject = status;
  return OPT_OK;
}

opt_status opt_server_set_max_rounds(opt_server* s, int32_t max_rounds) {
  if (!s || max_rounds < 1 || max_rounds > kServeMaxRounds) return OPT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_rounds = max_rounds;
  return OPT_OK;
}

opt_status opt_server_set_max_active(opt_server* s, int32_t max_active) {
  if (!s || max_active < 0) return OPT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_active = max_active;
  return OPT_OK;
}

opt_status opt_server_poll(opt_server* s, uint64_t ticket, opt_report* report) {
  if (!s) return OPT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return OPT_ERR_INVALID_ARG;
  ServeReq* r = it->second.get();
  if (r->state != 2) return OPT_ERR_NOT_READY;
  const opt_status st = r->status;
  if (report) {
    double* h = report->E_history;
    *report = r->rep;
    report->E_history = h;
    if (h) std::memcpy(h, r->hist.data(), r->hist.size() * sizeof(double));
  }
  s->reqs.erase(it);
  return st;
}

}  // extern "C"
