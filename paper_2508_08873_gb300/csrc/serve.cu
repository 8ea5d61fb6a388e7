// Continuous-batching Parareal server.
//
// The low-rank coarse solvers depend only on the operator and the time grid,
// not on the source term or the initial value (Sec. 2.1; Remark
// rem:affine_g_n), so built coarse handles stay resident and serve a stream of
// requests (new u0, new f).  Requests on one coarse handle form a group with
// its own worker thread and its own stream, whose CUDA priority grows as the
// group's requests get cheaper (fewer row-steps per fine solve), so that
// short requests are not held behind long ones of another handle: the GPU
// gives the higher-priority stream's blocks the SMs as the running blocks
// retire.  An optional latency target per handle turns away (LRP_EBUSY)
// requests whose estimated latency, from the group's measured service time
// and completion rate, would exceed it.  A group's worker runs "ticks"; each
// tick
//   1. admits queued requests into free slots (slot memory is reserved per
//      coarse handle up to the HBM budget; requests wait in the queue when no
//      slot is free),
//   2. for the newly admitted requests: uploads u0, g, c, computes b_i = F_i 0
//      for all their intervals in one launch and runs their initial coarse
//      sweeps in one batched launch,
//   3. for every active request: one Parareal iteration -- the fine solves of
//      all their unconverged intervals in shared propagator launches of at
//      most SERVE_LAUNCH_ROW_STEPS work each (a system map (slot, interval)
//      addresses each request's vectors; the bound lets a higher-priority
//      group's kernels in between), then all their coarse sweeps in one
//      batched launch (one cluster per request),
//   4. reads back the per-request bounds and retires the requests that met
//      their tolerance or iteration cap (copying the iterate to the host).
// Requests arriving while others are on the GPU join at the next tick, so
// their work shares launches with the requests in flight.  Every kernel is
// deterministic per system, so a request's result does not depend on the mix
// beyond the rounding of the launch configuration chosen for the batch size.
#include <algorithm>
#include <chrono>
#include <cmath>
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
  unsigned long long tick_admit = 0;   // the group's tick count at admission
  bool admitted = false, done = false, fetched = false;
  int status = LRP_OK;
  double bound = 0.0, scale = 0.0;
  std::vector<double> result;
};

struct Group {
  Coarse* co = nullptr;
  Ctx* gctx = nullptr;                                 // own stream (priority) and memory
  int n = 0, N = 0, M = 0, Qmax = 0, slots = 0, priority = 0;
  size_t su = 0, sF = 0, sg = 0, sc = 0, snorm = 0;   // per-slot strides (doubles)
  int rows = 0, nsl = 0;                               // coarse-sweep slices
  size_t scw = 0;                                      // per-slot sweep workspace (doubles)
  DevBuf u, F, b, g, c, norms, summ, dargs, dmap, cw, cnt;
  std::vector<int> free;
  std::vector<Request*> active;
  // under the server mutex
  std::deque<Request*> queue;
  std::condition_variable cv;
  std::thread worker;
  double target_ms = 0.0;          // latency target (0: none)
  // latency model: a request spends svc_ticks ticks in a slot (EWMA over
  // finished requests, about its iteration count whatever the load); a tick
  // with A requests active takes t0 + t1 A ms (least squares over the ticks,
  // exponentially forgetting)
  double svc_ticks = 0.0;
  double sw = 0.0, sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
  int n_est = 0;
  unsigned long long ticks = 0, completed = 0;
  double busy_ms = 0.0;
  ~Group() {
    for (DevBuf* d : {&u, &F, &b, &g, &c, &norms, &summ, &dargs, &dmap, &cw, &cnt}) d->release();
    ctx_release(gctx);
  }
};

}  // namespace

struct lrp_server {
  lrp_ctx* ctx = nullptr;           // the server's context (device)
  int max_slots = 64, Qmax = 4;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::unordered_map<const Coarse*, std::unique_ptr<Group>> groups;
  std::unordered_map<const Coarse*, double> targets;
  uint64_t next_ticket = 1;
  bool stop = false;
  int active_total = 0;
  size_t queued_total = 0, queue_cap = 100000;
  lrp_status worker_error = LRP_OK;
  std::string worker_msg;
};

namespace {

// CUDA stream priority of a group: the highest for requests of at most 1e5
// row-steps per fine solve (n N M), one level lower per factor of ten.
int group_priority(const Coarse* co) {
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest)) { cudaGetLastError(); return 0; }
  const double cost = (double)co->op->n * co->N * co->M;
  const int lvl = std::max(0, (int)std::floor(std::log10(std::max(cost, 1.0))) - 5);
  return std::min(least, greatest + lvl);
}

lrp_status make_group(lrp_server* S, Coarse* co, Group** out) {
  auto G = std::make_unique<Group>();
  G->priority = group_priority(co);
  G->gctx = ctx_create(S->ctx->device, S->budget, G->priority);
  if (!G->gctx) return set_err(S->ctx, LRP_ECUDA, "server group: stream creation failed");
  Ctx* c = G->gctx;
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
  if (slots < 1) return set_err(S->ctx, LRP_ENOMEM, "no HBM for a single request slot");
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
  if (cudaStreamSynchronize(c->stream)) return cuda_err(S->ctx, cudaGetLastError(), "server group");
  for (int i = slots - 1; i >= 0; --i) G->free.push_back(i);
  auto t = S->targets.find(co);
  if (t != S->targets.end()) G->target_ms = t->second;
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
  (void)S;
  if (list.empty()) return LRP_OK;
  Ctx* c = G->gctx;
  std::vector<SweepArgs> h(list.size());
  for (size_t i = 0; i < list.size(); ++i)
    h[i] = slot_args(G, list[i]->slot, initial ? 0 : list[i]->k, initial);
  lrp_status s = coarse_sweep(c, h.data(), G->dargs.as<SweepArgs>(), (int)h.size());
  // the host array must outlive the (pageable, so synchronous-for-host) copy
  cudaStreamSynchronize(c->stream);
  return s;
}

// Fine-solve work of one propagator launch of the server, in row-steps
// (systems x n x M): about 1.5 ms of FP64 fine solves on GB300.  A tick's
// fine solves go out in launches of at most this much work, so that the
// higher-priority stream of a group with cheaper requests gets the SMs
// between them instead of waiting for one launch over every request in
// flight (with 50 adr1d requests of 64 intervals, a single launch would run
// for ~40 ms).
constexpr double SERVE_LAUNCH_ROW_STEPS = 128.0 * 4096.0 * 256.0;

// propagate_any over nsys mapped systems in launches of at most
// SERVE_LAUNCH_ROW_STEPS row-steps; the maps of in, out and src (2 ints per
// system) are offset per launch
static lrp_status propagate_chunked(Ctx* c, Operator* op, double dt, int M, int nsys,
                                    const PropIn& in, const PropOut& out, const PropSrc& src) {
  const double per = (double)op->n * std::max(M, 1);
  const int chunk = std::max(1, (int)std::min<double>(nsys, SERVE_LAUNCH_ROW_STEPS / per));
  for (int s0 = 0; s0 < nsys; s0 += chunk) {
    const int cnt = std::min(chunk, nsys - s0);
    PropIn i2 = in;
    PropOut o2 = out;
    PropSrc r2 = src;
    if (i2.map) i2.map += 2 * s0;
    if (o2.map) o2.map += 2 * s0;
    if (r2.map) r2.map += 2 * s0;
    lrp_status st = propagate_any(c, op, dt, M, 0, cnt, 0, i2, o2, r2);
    if (st) return st;
  }
  return LRP_OK;
}

lrp_status tick_group(lrp_server* S, Group* G, std::vector<Request*>& fresh) {
  Ctx* c = G->gctx;
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
      if ((s = propagate_chunked(c, op, co->dt, M, (int)map.size() / 2, in, out, src)))
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
    if ((s = propagate_chunked(c, op, co->dt, M, (int)map.size() / 2, in, out, src)))
      return s;
    cudaStreamSynchronize(c->stream);
    if ((s = batch_sweep(S, G, run, 0))) return s;
    for (Request* r : run) r->k += 1;
  }
  return LRP_OK;
}

// The worker of one group: admit from the group's queue into free slots,
// run a tick, retire finished requests, update the estimates.
void group_main(lrp_server* S, Group* G) {
  cudaSetDevice(S->ctx->device);
  Ctx* c = G->gctx;
  std::vector<double> summ;
  while (true) {
    std::vector<Request*> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      G->cv.wait(lk, [&] { return S->stop || !G->queue.empty() || !G->active.empty(); });
      if (S->stop) break;
      while (!G->queue.empty() && !G->free.empty()) {
        Request* r = G->queue.front();
        G->queue.pop_front();
        S->queued_total -= 1;
        r->slot = G->free.back();
        G->free.pop_back();
        r->admitted = true;
        r->t_admit = Clock::now();
        r->tick_admit = G->ticks;
        G->active.push_back(r);
        fresh.push_back(r);
        S->active_total += 1;
      }
    }
    auto t0 = Clock::now();
    const double active_in_tick = (double)G->active.size();
    lrp_status st = tick_group(S, G, fresh);
    // ---- read back bounds, retire converged requests -------------------------
    std::vector<Request*> retire;
    summ.resize(2 * (size_t)G->slots);
    if (!st) {
      cudaError_t e = cudaMemcpyAsync(summ.data(), G->summ.ptr, 16 * (size_t)G->slots,
                                      cudaMemcpyDeviceToHost, c->stream);
      if (!e) e = cudaStreamSynchronize(c->stream);
      if (e) st = cuda_err(c, e, "server tick");
    }
    for (Request* r : G->active) {
      if (st) { r->status = st; retire.push_back(r); continue; }
      r->bound = summ[2 * r->slot];
      r->scale = summ[2 * r->slot + 1];
      bool conv = r->k >= 1 && r->tol > 0 && r->bound <= r->tol * r->scale;
      if (conv || r->k >= r->K) {
        r->status = (r->tol > 0 && !conv) ? LRP_ENOTCONV : LRP_OK;
        retire.push_back(r);
      }
    }
    for (Request* r : retire) {
      r->result.resize((size_t)G->su);
      if (!st)
        cudaMemcpyAsync(r->result.data(), G->u.as<double>() + (size_t)r->slot * G->su, 8 * G->su,
                        cudaMemcpyDeviceToHost, c->stream);
    }
    if (!retire.empty()) cudaStreamSynchronize(c->stream);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const auto now = Clock::now();
      const double tick = std::chrono::duration<double, std::milli>(now - t0).count();
      for (Request* r : retire) {
        r->done = true;
        r->t_done = now;
        G->free.push_back(r->slot);
        G->active.erase(std::find(G->active.begin(), G->active.end(), r));
        S->active_total -= 1;
        G->completed += 1;
        const double svc = (double)(G->ticks - r->tick_admit + 1);
        G->svc_ticks = G->n_est ? 0.8 * G->svc_ticks + 0.2 * svc : svc;
        G->n_est += 1;
      }
      const double f = 0.97;   // forgetting factor of the tick-time fit
      G->sw = f * G->sw + 1.0;
      G->sx = f * G->sx + active_in_tick;
      G->sy = f * G->sy + tick;
      G->sxx = f * G->sxx + active_in_tick * active_in_tick;
      G->sxy = f * G->sxy + active_in_tick * tick;
      G->ticks += 1;
      G->busy_ms += tick;
      if (st && S->worker_error == LRP_OK) { S->worker_error = st; S->worker_msg = c->last_error; }
    }
    if (!retire.empty() || st) S->cv_done.notify_all();
  }
}

// Estimated latency (ms) of a request submitted to G now: with A = the
// requests active or queued plus this one, the tick time at min(A, slots)
// active requests from the fitted line, times the request's ticks in a slot,
// times the waves of slots the queue needs; 0 while the group has no
// finished request.
double estimate_ms(const lrp_server* S, const Group* G) {
  (void)S;
  if (!G->n_est || G->sw <= 0.0) return 0.0;
  const double mx = G->sx / G->sw, my = G->sy / G->sw;
  const double var = G->sxx / G->sw - mx * mx;
  double t1 = var > 1e-9 ? (G->sxy / G->sw - mx * my) / var : 0.0;
  t1 = std::max(t1, 0.0);
  const double t0 = std::max(my - t1 * mx, 0.0);
  const long A = (long)G->queue.size() + (long)G->active.size() + 1;
  const long running = std::min<long>(A, G->slots);
  const long waves = (A + G->slots - 1) / G->slots;
  return G->svc_ticks * (t0 + t1 * (double)running) * (double)waves;
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
  *out = S.release();
  return LRP_OK;
}

void lrp_server_destroy(lrp_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (auto& kv : S->groups) kv.second->cv.notify_all();
  }
  for (auto& kv : S->groups)
    if (kv.second->worker.joinable()) kv.second->worker.join();
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
  if (Q > 0 && source_samples(co->op) != 1)
    return set_err(S->ctx, LRP_EINVAL, "served requests take sources with backward-Euler fine steps");
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
  Group* G = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return LRP_EINVAL;
    if (S->queued_total >= S->queue_cap) return LRP_EBUSY;
    auto gi = S->groups.find(cc);
    if (gi == S->groups.end()) {
      cudaSetDevice(S->ctx->device);
      lrp_status s = make_group(S, cc, &G);
      if (s) {
        S->groups.erase(cc);
        return s;
      }
      G->worker = std::thread(group_main, S, G);
    } else {
      G = gi->second.get();
    }
    if (G->target_ms > 0.0 && estimate_ms(S, G) > G->target_ms) return LRP_EBUSY;
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    G->queue.push_back(r.get());
    S->queued_total += 1;
    S->reqs[r->ticket] = std::move(r);
  }
  G->cv.notify_one();
  return LRP_OK;
}

lrp_status lrp_server_set_latency_target(lrp_server* S, const lrp_coarse* co, double target_ms) {
  if (!S || !co || !(target_ms >= 0.0)) return LRP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  const Coarse* cc = co;
  S->targets[cc] = target_ms;
  auto gi = S->groups.find(cc);
  if (gi != S->groups.end()) gi->second->target_ms = target_ms;
  return LRP_OK;
}

lrp_status lrp_server_estimate(lrp_server* S, const lrp_coarse* co, double* latency_ms) {
  if (!S || !co || !latency_ms) return LRP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto gi = S->groups.find(static_cast<const Coarse*>(co));
  *latency_ms = gi == S->groups.end() ? 0.0 : estimate_ms(S, gi->second.get());
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
  st->completed = 0;
  st->ticks = 0;
  st->busy_ms = 0.0;
  st->slots = 0;
  for (auto& kv : S->groups) {
    st->completed += kv.second->completed;
    st->ticks += kv.second->ticks;
    st->busy_ms += kv.second->busy_ms;
    st->slots += kv.second->slots;
  }
  st->queued = S->queued_total;
  st->active = S->active_total;
  st->error = S->worker_error;
  return LRP_OK;
}

}  // extern "C"
