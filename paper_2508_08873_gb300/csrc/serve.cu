// Continuous-batching Parareal server.
//
// The low-rank coarse solvers depend only on the operator and the time grid,
// not on the source term or the initial value (Sec. 2.1; Remark
// rem:affine_g_n), so built coarse handles stay resident and serve a stream of
// requests (new u0, new f).  A worker thread runs "ticks"; each tick
//   1. admits queued requests into free slots (slot memory is reserved per
//      coarse handle up to the HBM budget; requests wait in the queue when no
//      slot is free),
//   2. for the newly admitted requests: uploads u0, g, c, computes b_i = F_i 0
//      for all their intervals in one launch and runs their initial coarse
//      sweeps in one batched launch,
//   3. for every active request: one Parareal iteration -- the fine solves of
//      all their unconverged intervals in ONE propagator launch (a system map
//      (slot, interval) addresses each request's vectors), then all their
//      coarse sweeps in one batched launch (one cluster per request),
//   4. reads back the per-request bounds and retires the requests that met
//      their tolerance or iteration cap (copying the iterate to the host).
// Requests arriving while others are on the GPU join at the next tick, so
// their work shares launches with the requests in flight.  Every kernel is
// deterministic per system, so a request's result does not depend on the mix
// beyond the rounding of the launch configuration chosen for the batch size.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace lrp;
using Clock = std::chrono::steady_clock;

struct lrp_ctx : public Ctx {};
struct lrp_operator : public Operator {};
struct lrp_coarse : public Coarse {};

namespace {

struct Request {
  uint64_t ticket = 0;
  Coarse* co = nullptr;
  std::vector<double> u0, g, c;   // g: Qmax x n, c: (N*M) x Qmax (zero padded)
  int Q = 0, K = 0;
  double tol = 0.0;
  Clock::time_point t_submit, t_admit, t_done;
  int slot = -1, k = 0;
  bool admitted = false, done = false, fetched = false;
  int status = LRP_OK;
  double bound = 0.0, scale = 0.0;
  std::vector<double> result;
};

struct Group {
  Coarse* co = nullptr;
  int n = 0, N = 0, M = 0, Qmax = 0, slots = 0;
  size_t su = 0, sF = 0, sg = 0, sc = 0, snorm = 0;   // per-slot strides (doubles)
  int rows = 0, nsl = 0;                               // coarse-sweep slices
  size_t scw = 0;                                      // per-slot sweep workspace (doubles)
  DevBuf u, F, b, g, c, norms, summ, dargs, dmap, cw, cnt;
  std::vector<int> free;
  std::vector<Request*> active;
};

}  // namespace

struct lrp_server {
  lrp_ctx* ctx = nullptr;           // the server's own context (stream, memory)
  int max_slots = 64, Qmax = 4;
  size_t budget = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::unordered_map<const Coarse*, std::unique_ptr<Group>> groups;
  uint64_t next_ticket = 1;
  bool stop = false;
  int active_total = 0;
  size_t queue_cap = 100000;
  // statistics
  unsigned long long completed = 0, ticks = 0, launches = 0;
  double busy_ms = 0.0;
  lrp_status worker_error = LRP_OK;
  std::string worker_msg;
};

namespace {

lrp_status make_group(lrp_server* S, Coarse* co, Group** out) {
  Ctx* c = S->ctx;
  auto G = std::make_unique<Group>();
  G->co = co;
  G->n = co->op->n;
  G->N = co->N;
  G->M = co->M;
  G->Qmax = S->Qmax;
  const size_t n = G->n, N = G->N;
  G->su = (N + 1) * n;
  G->sF = N * n;
  G->sg = (size_t)G->Qmax * n;
  G->sc = N * G->M * (size_t)G->Qmax;
  G->snorm = 3 * (N + 1);
  G->rows = sweep_rows(c);
  G->nsl = (G->n + G->rows - 1) / G->rows;
  G->scw = sweep_ws_doubles(G->N, G->nsl, std::max(co->R, 1));
  const size_t per_slot = 8 * (G->su + 2 * G->sF + G->sg + G->sc + G->snorm + 2 + G->scw + 1) +
                          sizeof(SweepArgs) + 8 * N;
  // slots by free HBM: at most half of what the device has free, and the budget
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  size_t cap = freeb / 2;
  if (S->budget) cap = std::min(cap, S->budget);
  int slots = (int)std::min<size_t>((size_t)S->max_slots, cap / std::max<size_t>(per_slot, 1));
  if (slots < 1) return set_err(c, LRP_ENOMEM, "no HBM for a single request slot");
  G->slots = slots;
  lrp_status s;
  if ((s = dev_alloc(c, G->u, 8 * G->su * slots))) return s;
  if ((s = dev_alloc(c, G->F, 8 * G->sF * slots))) return s;
  if ((s = dev_alloc(c, G->b, 8 * G->sF * slots))) return s;
  if ((s = dev_alloc(c, G->g, 8 * std::max<size_t>(G->sg, 1) * slots))) return s;
  if ((s = dev_alloc(c, G->c, 8 * std::max<size_t>(G->sc, 1) * slots))) return s;
  if ((s = dev_alloc(c, G->norms, 8 * G->snorm * slots))) return s;
  if ((s = dev_alloc(c, G->summ, 16 * (size_t)slots))) return s;
  if ((s = dev_alloc(c, G->dargs, sizeof(SweepArgs) * (size_t)slots))) return s;
  if ((s = dev_alloc(c, G->dmap, 8 * N * (size_t)slots))) return s;
  if ((s = dev_alloc(c, G->cw, 8 * G->scw * slots))) return s;
  if ((s = dev_alloc(c, G->cnt, 2 * sizeof(unsigned) * slots))) return s;
  cudaMemsetAsync(G->cnt.ptr, 0, G->cnt.bytes, c->stream);
  for (int i = slots - 1; i >= 0; --i) G->free.push_back(i);
  *out = G.get();
  S->groups[co] = std::move(G);
  return LRP_OK;
}

SweepArgs slot_args(Group* G, int slot, int first, int initial) {
  Coarse* co = G->co;
  SweepArgs a;
  const int f32 = co->prec == LRP_PREC_MIXED;
  a.N = G->N;
  a.n = G->n;
  a.R = std::max(co->R, 1);
  a.first = first;
  a.initial = initial;
  a.u = G->u.as<double>() + (size_t)slot * G->su;
  a.F = (initial ? G->b.as<double>() : G->F.as<double>()) + (size_t)slot * G->sF;
  a.U = f32 ? co->U32.ptr : co->U.ptr;
  a.S = f32 ? co->S32.ptr : co->S.ptr;
  a.V = f32 ? co->V32.ptr : co->V.ptr;
  a.K = co->Kc.as<double>();
  a.f32 = f32;
  a.delta = co->delta;
  a.eps = co->eps;
  a.rows = G->rows;
  a.nsl = G->nsl;
  a.cw = G->cw.as<double>() + (size_t)slot * G->scw;
  a.cnt = G->cnt.as<unsigned>() + 2 * (size_t)slot;
  double* nr = G->norms.as<double>() + (size_t)slot * G->snorm;
  a.du = nr;
  a.unorm = nr + (G->N + 1);
  a.bound = initial ? nullptr : nr + 2 * (G->N + 1);
  a.summary = G->summ.as<double>() + 2 * (size_t)slot;
  return a;
}

// One batched sweep launch for `list` (slot, first, initial) of group G.
lrp_status batch_sweep(lrp_server* S, Group* G, const std::vector<Request*>& list, int initial) {
  if (list.empty()) return LRP_OK;
  Ctx* c = S->ctx;
  std::vector<SweepArgs> h(list.size());
  for (size_t i = 0; i < list.size(); ++i)
    h[i] = slot_args(G, list[i]->slot, initial ? 0 : list[i]->k, initial);
  lrp_status s = coarse_sweep(c, h.data(), G->dargs.as<SweepArgs>(), (int)h.size());
  // the host array must outlive the (pageable, so synchronous-for-host) copy
  cudaStreamSynchronize(c->stream);
  return s;
}

lrp_status tick_group(lrp_server* S, Group* G, std::vector<Request*>& fresh) {
  Ctx* c = S->ctx;
  Coarse* co = G->co;
  Operator* op = const_cast<Operator*>(co->op);
  const int n = G->n, N = G->N, M = G->M;
  lrp_status s;
  cudaError_t e;
  // ---- admission: inputs, b_i, initial sweeps --------------------------------
  if (!fresh.empty()) {
    std::vector<int> map;
    for (Request* r : fresh) {
      double* u = G->u.as<double>() + (size_t)r->slot * G->su;
      e = cudaMemcpyAsync(u, r->u0.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
      if (!e && r->Q > 0) {
        e = cudaMemcpyAsync(G->g.as<double>() + (size_t)r->slot * G->sg, r->g.data(), 8 * G->sg,
                            cudaMemcpyHostToDevice, c->stream);
        if (!e)
          e = cudaMemcpyAsync(G->c.as<double>() + (size_t)r->slot * G->sc, r->c.data(), 8 * G->sc,
                              cudaMemcpyHostToDevice, c->stream);
        for (int i = 0; i < N; ++i) { map.push_back(r->slot); map.push_back(i); }
      } else if (!e) {
        e = cudaMemsetAsync(G->b.as<double>() + (size_t)r->slot * G->sF, 0, 8 * G->sF, c->stream);
      }
      if (e) return cuda_err(c, e, "request upload");
    }
    if (!map.empty()) {
      e = cudaMemcpyAsync(G->dmap.ptr, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice,
                          c->stream);
      if (e) return cuda_err(c, e, "map upload");
      PropIn in;                      // zero initial values
      PropOut out;
      out.y = G->b.ptr;
      out.ldy = n;
      out.map = G->dmap.as<int>();
      out.slot_stride = (long)G->sF;
      PropSrc src;
      src.Q = G->Qmax;
      src.g = G->g.as<double>();
      src.c = G->c.as<double>();
      src.cstride = (long)M * G->Qmax;
      src.map = G->dmap.as<int>();
      src.c_slot_stride = (long)G->sc;
      src.g_slot_stride = (long)G->sg;
      if ((s = propagate_any(c, op, co->dt, M, 0, (int)map.size() / 2, 0, in, out, src)))
        return s;
      cudaStreamSynchronize(c->stream);   // the host map must outlive its upload
    }
    if ((s = batch_sweep(S, G, fresh, 1))) return s;
  }
  // ---- one Parareal iteration for every active request -------------------------
  std::vector<Request*> run;
  std::vector<int> map;
  for (Request* r : G->active)
    if (r->k < r->K) {
      run.push_back(r);
      for (int i = r->k; i < N; ++i) { map.push_back(r->slot); map.push_back(i); }
    }
  if (!map.empty()) {
    e = cudaMemcpyAsync(G->dmap.ptr, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice,
                        c->stream);
    if (e) return cuda_err(c, e, "map upload");
    PropIn in;
    in.x = G->u.ptr;
    in.x_f64 = 1;
    in.ldx = n;
    in.map = G->dmap.as<int>();
    in.slot_stride = (long)G->su;
    PropOut out;
    out.y = G->F.ptr;
    out.ldy = n;
    out.map = G->dmap.as<int>();
    out.slot_stride = (long)G->sF;
    PropSrc src;
    src.Q = G->Qmax;
    src.g = G->g.as<double>();
    src.c = G->c.as<double>();
    src.cstride = (long)M * G->Qmax;
    src.map = G->dmap.as<int>();
    src.c_slot_stride = (long)G->sc;
    src.g_slot_stride = (long)G->sg;
    // requests without a source use zero-padded g/c; skip the source when none has one
    bool any_src = false;
    for (Request* r : run) any_src |= r->Q > 0;
    if (!any_src) src.Q = 0;
    if ((s = propagate_any(c, op, co->dt, M, 0, (int)map.size() / 2, 0, in, out, src)))
      return s;
    cudaStreamSynchronize(c->stream);
    if ((s = batch_sweep(S, G, run, 0))) return s;
    for (Request* r : run) r->k += 1;
  }
  return LRP_OK;
}

void worker_main(lrp_server* S) {
  cudaSetDevice(S->ctx->device);
  std::vector<double> summ;
  while (true) {
    std::unordered_map<Group*, std::vector<Request*>> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || S->active_total > 0; });
      if (S->stop) break;
      // admit FIFO into free slots
      for (auto it = S->queue.begin(); it != S->queue.end();) {
        Request* r = *it;
        Group* G = nullptr;
        auto gi = S->groups.find(r->co);
        if (gi == S->groups.end()) {
          lrp_status s = make_group(S, r->co, &G);
          if (s) {
            r->status = s;
            r->done = true;
            r->t_done = Clock::now();
            it = S->queue.erase(it);
            S->cv_done.notify_all();
            continue;
          }
        } else {
          G = gi->second.get();
        }
        if (G->free.empty()) { ++it; continue; }
        r->slot = G->free.back();
        G->free.pop_back();
        r->admitted = true;
        r->t_admit = Clock::now();
        G->active.push_back(r);
        fresh[G].push_back(r);
        S->active_total += 1;
        it = S->queue.erase(it);
      }
    }
    auto t0 = Clock::now();
    lrp_status st = LRP_OK;
    std::vector<Group*> gl;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& kv : S->groups)
        if (!kv.second->active.empty()) gl.push_back(kv.second.get());
    }
    for (Group* G : gl) {
      std::vector<Request*> fr = fresh[G];
      if ((st = tick_group(S, G, fr))) break;
    }
    // ---- read back bounds, retire converged requests -------------------------
    std::vector<std::pair<Group*, Request*>> retire;
    for (Group* G : gl) {
      summ.resize(2 * (size_t)G->slots);
      if (!st) {
        cudaError_t e = cudaMemcpyAsync(summ.data(), G->summ.ptr, 16 * (size_t)G->slots,
                                        cudaMemcpyDeviceToHost, S->ctx->stream);
        if (!e) e = cudaStreamSynchronize(S->ctx->stream);
        if (e) st = cuda_err(S->ctx, e, "server tick");
      }
      for (Request* r : G->active) {
        if (st) { r->status = st; retire.push_back({G, r}); continue; }
        r->bound = summ[2 * r->slot];
        r->scale = summ[2 * r->slot + 1];
        bool conv = r->k >= 1 && r->tol > 0 && r->bound <= r->tol * r->scale;
        if (conv || r->k >= r->K) {
          r->status = (r->tol > 0 && !conv) ? LRP_ENOTCONV : LRP_OK;
          retire.push_back({G, r});
        }
      }
    }
    for (auto& gr : retire) {
      Group* G = gr.first;
      Request* r = gr.second;
      r->result.resize((size_t)G->su);
      if (!st)
        cudaMemcpyAsync(r->result.data(), G->u.as<double>() + (size_t)r->slot * G->su, 8 * G->su,
                        cudaMemcpyDeviceToHost, S->ctx->stream);
    }
    if (!retire.empty()) cudaStreamSynchronize(S->ctx->stream);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& gr : retire) {
        Group* G = gr.first;
        Request* r = gr.second;
        r->done = true;
        r->t_done = Clock::now();
        G->free.push_back(r->slot);
        G->active.erase(std::find(G->active.begin(), G->active.end(), r));
        S->active_total -= 1;
        S->completed += 1;
      }
      if (st) { S->worker_error = st; S->worker_msg = S->ctx->last_error; }
      S->ticks += 1;
      S->busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
    if (!retire.empty()) S->cv_done.notify_all();
  }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

lrp_status lrp_server_create(lrp_ctx* ctx, int max_slots, int max_terms, size_t hbm_budget_bytes,
                             lrp_server** out) {
  if (!ctx || !out || max_slots < 1 || max_terms < 0) return LRP_EINVAL;
  auto S = std::make_unique<lrp_server>();
  lrp_status s = lrp_create(&S->ctx, ctx->device, hbm_budget_bytes);
  if (s) return s;
  S->max_slots = max_slots;
  S->Qmax = max_terms;
  S->budget = hbm_budget_bytes;
  lrp_server* raw = S.get();
  raw->worker = std::thread(worker_main, raw);
  *out = S.release();
  return LRP_OK;
}

void lrp_server_destroy(lrp_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  S->groups.clear();
  lrp_ctx* c = S->ctx;
  S->reqs.clear();
  delete S;
  lrp_destroy(c);
}

lrp_status lrp_server_submit(lrp_server* S, const lrp_coarse* co, const double* u0, int Q,
                             const double* g, const double* c, int K_max, double tol,
                             uint64_t* ticket) {
  if (!S || !co || !u0 || !ticket || Q < 0 || K_max < 0) return LRP_EINVAL;
  if (Q > S->Qmax) return LRP_EINVAL;
  if (Q > 0 && (!g || !c)) return LRP_EINVAL;
  if (co->op->ctx->device != S->ctx->device) return LRP_EINVAL;
  auto r = std::make_unique<Request>();
  Coarse* cc = const_cast<lrp_coarse*>(co);
  const int n = cc->op->n, N = cc->N, M = cc->M, Qm = S->Qmax;
  r->co = cc;
  r->Q = Q;
  r->K = std::min(K_max, N);
  r->tol = tol;
  r->u0.assign(u0, u0 + n);
  if (Q > 0) {
    r->g.assign((size_t)Qm * n, 0.0);
    std::memcpy(r->g.data(), g, sizeof(double) * (size_t)Q * n);
    r->c.assign((size_t)N * M * Qm, 0.0);
    for (size_t j = 0; j < (size_t)N * M; ++j)
      for (int q = 0; q < Q; ++q) r->c[j * Qm + q] = c[j * Q + q];
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queue.size() >= S->queue_cap) return LRP_EBUSY;
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    S->queue.push_back(r.get());
    S->reqs[r->ticket] = std::move(r);
  }
  S->cv_work.notify_one();
  return LRP_OK;
}

static lrp_status fetch(lrp_server* S, Request* r, double* u_out, lrp_request_info* info) {
  if (u_out && !r->result.empty())
    std::memcpy(u_out, r->result.data(), sizeof(double) * r->result.size());
  if (info) {
    info->k_done = r->k;
    info->status = r->status;
    info->final_bound = r->bound;
    info->scale = r->scale;
    info->queue_ms = std::chrono::duration<double, std::milli>(
                         (r->admitted ? r->t_admit : r->t_done) - r->t_submit).count();
    info->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  }
  lrp_status st = (lrp_status)r->status;
  S->reqs.erase(r->ticket);
  return st;
}

lrp_status lrp_server_poll(lrp_server* S, uint64_t ticket, double* u_out, lrp_request_info* info) {
  if (!S) return LRP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return LRP_EINVAL;
  if (!it->second->done) return LRP_PENDING;
  return fetch(S, it->second.get(), u_out, info);
}

lrp_status lrp_server_wait(lrp_server* S, uint64_t ticket, double timeout_s, double* u_out,
                           lrp_request_info* info) {
  if (!S) return LRP_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return LRP_EINVAL;
  Request* r = it->second.get();
  auto pred = [&] { return r->done || S->worker_error != LRP_OK; };
  if (timeout_s > 0) {
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return LRP_ETIMEOUT;
  } else {
    S->cv_done.wait(lk, pred);
  }
  if (!r->done) return S->worker_error;
  return fetch(S, r, u_out, info);
}

lrp_status lrp_server_stats_get(lrp_server* S, lrp_server_stats* st) {
  if (!S || !st) return LRP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  st->completed = S->completed;
  st->queued = S->queue.size();
  st->active = S->active_total;
  st->ticks = S->ticks;
  st->busy_ms = S->busy_ms;
  st->slots = 0;
  for (auto& kv : S->groups) st->slots += kv.second->slots;
  st->error = S->worker_error;
  return LRP_OK;
}

}  // extern "C"
