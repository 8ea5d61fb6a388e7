// C ABI of the library (include/lrp.h): contexts, operators, the batched fine
// propagator, the coarse-solver build (randomized SVD, Sec. 2.1) and the
// Parareal solve (Eq. def_Parareal).  Host code only orchestrates kernels;
// every arithmetic step of the method runs on the device.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

using namespace lrp;

struct lrp_ctx : public Ctx {};
struct lrp_operator : public Operator {};
struct lrp_coarse : public Coarse {};

namespace lrp {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
lrp_status set_err(Ctx* c, lrp_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

lrp_status cuda_err(Ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_err(c, LRP_ENOMEM, m);
  return set_err(c, LRP_ECUDA, m);
}

DevBuf::~DevBuf() { release(); }

static void pool_drain(Ctx* c);

void ctx_retain(Ctx* c) { if (c) c->refs += 1; }

void ctx_release(Ctx* c) {
  if (!c || --c->refs > 0) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (DevBuf* b : {&c->kws, &c->kstat, &c->bws, &c->irws, &c->irstat, &c->triws}) b->release();
  pool_drain(c);
  for (auto& kv : c->timers)
    for (auto& pr : kv.second.pairs) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete static_cast<lrp_ctx*>(c);
}

// Buffers are released before the context reference is dropped.
Operator::~Operator() {
  Ctx* c = ctx;
  plans.clear();
  cplans.clear();
  splans.clear();
  for (auto& b : a64) b.release();
  for (auto& b : a32) b.release();
  ctx_release(c);
}

Coarse::~Coarse() {
  Ctx* c = ctx;
  for (DevBuf* b : {&U, &S, &V, &U32, &S32, &V32, &Kc, &ws_u, &ws_F, &ws_b, &ws_norm, &ws_d, &ws_g,
                     &ws_c, &ws_cw, &ws_cnt, &ws_args, &ws_flag, &ws_bh, &ws_argv})
    b->release();
  if (h_stat) cudaFreeHost(h_stat);
  ctx_release(c);
}

// Buffers go back to the context's pool (the memory stays allocated and
// counted in in_use) unless the pool is full.  Users of a buffer finish in
// stream order before it is released: every path synchronises the
// context's stream before dropping temporaries.
void DevBuf::release() {
  if (ptr) {
    bool kept = false;
    if (ctx) {
      std::lock_guard<std::mutex> lk(ctx->pool_mu);
      if (ctx->pool_bytes + bytes <= ctx->pool_cap) {
        ctx->pool.emplace(bytes, ptr);
        ctx->pool_bytes += bytes;
        kept = true;
      }
    }
    if (!kept) {
      cudaFree(ptr);
      if (ctx) ctx->in_use -= bytes;
    }
  }
  ptr = nullptr;
  bytes = 0;
}

static void pool_drain(Ctx* c) {
  std::lock_guard<std::mutex> lk(c->pool_mu);
  for (auto& kv : c->pool) {
    cudaFree(kv.second);
    c->in_use -= kv.first;
  }
  c->pool.clear();
  c->pool_bytes = 0;
}

lrp_status dev_alloc(Ctx* c, DevBuf& b, size_t bytes) {
  b.release();
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  {
    // reuse a pooled block of at least `bytes` and at most twice that
    std::lock_guard<std::mutex> lk(c->pool_mu);
    auto it = c->pool.lower_bound(bytes);
    if (it != c->pool.end() && it->first <= 2 * bytes) {
      b.ctx = c;
      b.ptr = it->second;
      b.bytes = it->first;
      c->pool_bytes -= it->first;
      c->pool.erase(it);
      return LRP_OK;
    }
  }
  if (c->budget && c->in_use + bytes > c->budget) {
    pool_drain(c);
    if (c->in_use + bytes > c->budget)
      return set_err(c, LRP_ENOMEM, "HBM budget of the context exceeded");
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    pool_drain(c);
    e = cudaMalloc(&p, bytes);
  }
  if (e) { cudaGetLastError(); return cuda_err(c, e, "cudaMalloc"); }
  b.ctx = c;
  b.ptr = p;
  b.bytes = bytes;
  c->in_use += bytes;
  return LRP_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) { cudaGetLastError(); return false; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void timer_begin(Ctx* c, const char* fam, cudaEvent_t* ev) {
  *ev = nullptr;
  if (!c->timing) return;
  cudaEventCreate(ev);
  cudaEventRecord(*ev, c->stream);
}

void timer_end(Ctx* c, const char* fam, cudaEvent_t ev) {
  c->launches += 1;
  if (!c->timing || !ev) return;
  cudaEvent_t e2;
  cudaEventCreate(&e2);
  cudaEventRecord(e2, c->stream);
  c->timers[fam].pairs.emplace_back(ev, e2);
}

// copy `bytes` from a host or device pointer into a device buffer
static lrp_status to_device(Ctx* c, void* dst, const void* src, size_t bytes) {
  if (!bytes) return LRP_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream);
  return e ? cuda_err(c, e, "copy to device") : LRP_OK;
}

static lrp_status from_device(Ctx* c, void* dst, const void* src, size_t bytes) {
  if (!bytes) return LRP_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream);
  if (e) return cuda_err(c, e, "copy from device");
  if (!is_device_ptr(dst)) {
    e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_err(c, e, "synchronize");
  }
  return LRP_OK;
}

// A device view of caller data: the pointer itself when it is device memory,
// else a temporary device copy.
struct DevView {
  const void* p = nullptr;
  DevBuf tmp;
};
static lrp_status device_view(Ctx* c, const void* src, size_t bytes, DevView& v) {
  if (!src || !bytes) { v.p = nullptr; return LRP_OK; }
  if (is_device_ptr(src)) { v.p = src; return LRP_OK; }
  lrp_status s = dev_alloc(c, v.tmp, bytes);
  if (s) return s;
  if ((s = to_device(c, v.tmp.ptr, src, bytes))) return s;
  v.p = v.tmp.ptr;
  return LRP_OK;
}

}  // namespace lrp

// ===========================================================================
// context
// ===========================================================================
namespace lrp {
Ctx* ctx_create(int device, size_t hbm_budget_bytes, int priority) {
  if (cudaSetDevice(device)) { cudaGetLastError(); return nullptr; }
  auto* c = new lrp_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaStreamCreateWithPriority(&c->own_stream, cudaStreamNonBlocking, priority)) {
    cudaGetLastError();
    delete c;
    return nullptr;
  }
  c->stream = c->own_stream;
  return c;
}
}  // namespace lrp

extern "C" {

const char* lrp_status_string(lrp_status s) {
  switch (s) {
    case LRP_OK: return "ok";
    case LRP_EINVAL: return "invalid argument";
    case LRP_ENOMEM: return "out of device memory or HBM budget";
    case LRP_ENOTCONV: return "not converged within the iteration cap";
    case LRP_EBREAKDOWN: return "breakdown (zero pivot)";
    case LRP_ETIMEOUT: return "device wait timed out";
    case LRP_ECUDA: return "CUDA error";
    case LRP_EBUSY: return "queue full";
  }
  return "unknown status";
}

lrp_status lrp_create(lrp_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return LRP_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e || device < 0 || device >= ndev) { cudaGetLastError(); return LRP_ECUDA; }
  e = cudaSetDevice(device);
  if (e) return LRP_ECUDA;
  auto* c = new lrp_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
  if (e) { delete c; return LRP_ECUDA; }
  c->stream = c->own_stream;
  *out = c;
  return LRP_OK;
}

void lrp_destroy(lrp_ctx* c) {
  if (!c) return;
  ctx_release(c);   // freed now, or when its last operator / coarse handle goes
}

lrp_status lrp_set_stream(lrp_ctx* c, void* s) {
  if (!c) return LRP_EINVAL;
  c->stream = s ? (cudaStream_t)s : c->own_stream;
  return LRP_OK;
}

void* lrp_get_stream(lrp_ctx* c) { return c ? (void*)c->stream : nullptr; }

lrp_status lrp_synchronize(lrp_ctx* c) {
  if (!c) return LRP_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e ? cuda_err(c, e, "synchronize") : LRP_OK;
}

const char* lrp_last_error(lrp_ctx* c) { return c ? c->last_error.c_str() : ""; }

size_t lrp_bytes_in_use(lrp_ctx* c) { return c ? c->in_use.load() : 0; }

long lrp_launch_count(lrp_ctx* c) { return c ? c->launches : 0; }

lrp_status lrp_set_param(lrp_ctx* c, const char* name, int value) {
  if (!c || !name) return LRP_EINVAL;
  std::string k(name);
  if (k == "sweep_rows") {
    if (value != 0 && (value < 128 || value > 2048 || (value & (value - 1)))) return LRP_EINVAL;
    c->p_sweep_rows = value;
  } else if (k == "tri_cluster") {
    if (value < 0 || value > 8) return LRP_EINVAL;
    c->p_tri_cluster = value;
  } else if (k == "tri_warp") {
    if (value < 0 || value > 2) return LRP_EINVAL;
    c->p_tri_warp = value;
  } else if (k == "tri_spt") {
    if (value != 0 && value != 1 && value != 2) return LRP_EINVAL;
    c->p_tri_spt = value;
  } else if (k == "tri_chunk") {
    if (value != 0 && value != 8 && value != 16) return LRP_EINVAL;
    c->p_tri_chunk = value;
  } else if (k == "orth_tc") {
    if (value != 0 && value != 1) return LRP_EINVAL;
    c->p_orth_tc = value;
  } else if (k == "tri_wchunk") {
    if (value != 0 && (value < 8 || value > 16)) return LRP_EINVAL;
    c->p_tri_wchunk = value;
  } else if (k == "tri_wsplit") {
    if (value < 0 || value > 1) return LRP_EINVAL;
    c->p_tri_wsplit = value;
  } else if (k == "tri_wblock") {
    if (value < 0 || value > 2) return LRP_EINVAL;
    c->p_tri_wblock = value;
  } else if (k == "tri_wtoep") {
    if (value < 0 || value > 2) return LRP_EINVAL;
    c->p_tri_wtoep = value;
  } else if (k == "tri_group") {
    if (value < 0 || value > 16) return LRP_EINVAL;
    c->p_tri_group = value;
  } else if (k == "orth_cluster") {
    if (value < -1 || value > 16 || (value > 0 && (value & (value - 1)))) return LRP_EINVAL;
    c->p_orth_cluster = value;
  } else if (k == "krylov_cluster") {
    if (value < 0 || value > 16 || (value & (value - 1))) return LRP_EINVAL;
    c->p_krylov_cluster = value;
  } else if (k == "queue_cluster") {
    if (value < 0 || value > 16 || (value & (value - 1))) return LRP_EINVAL;
    c->p_queue_cluster = value;
  } else if (k == "krylov_onchip") {
    if (value != 0 && value != 2) return LRP_EINVAL;
    c->p_krylov_onchip = value;
  } else if (k == "krylov_block") {
    if (value != 0 && value != 4) return LRP_EINVAL;
    c->p_krylov_block = value;
  } else if (k == "krylov_block_clusters") {
    if (value < 0 || value > 1024) return LRP_EINVAL;
    c->p_krylov_block_clusters = value;
  } else if (k == "krylov_refine") {
    if (value < 0 || value > 2) return LRP_EINVAL;
    c->p_krylov_refine = value;
  } else if (k == "krylov_refine_digits") {
    if (value < 0 || value > 7) return LRP_EINVAL;
    c->p_krylov_refine_digits = value;
  } else if (k == "krylov_stage") {
    if (value != 0 && value != 1) return LRP_EINVAL;
    c->p_krylov_stage = value;
  } else if (k == "tri_refine") {
    if (value != 0 && value != 1) return LRP_EINVAL;
    c->p_tri_refine = value;
  } else if (k == "tri_refine_rounds") {
    if (value < 1 || value > 3) return LRP_EINVAL;
    c->p_tri_refine_rounds = value;
  } else if (k == "tri_refine_cluster") {
    if (value != 0 && value != 1) return LRP_EINVAL;
    c->p_tri_refine_cluster = value;
  } else {
    return set_err(c, LRP_EINVAL, "unknown parameter");
  }
  return LRP_OK;
}

lrp_status lrp_get_param(lrp_ctx* c, const char* name, int* value) {
  if (!c || !name || !value) return LRP_EINVAL;
  std::string k(name);
  if (k == "sweep_rows") *value = c->p_sweep_rows;
  else if (k == "tri_cluster") *value = c->p_tri_cluster;
  else if (k == "queue_cluster") *value = c->p_queue_cluster;
  else if (k == "krylov_cluster") *value = c->p_krylov_cluster;
  else if (k == "krylov_onchip") *value = c->p_krylov_onchip;
  else if (k == "krylov_onchip_rows") *value = c->oc_last[0];
  else if (k == "krylov_onchip_cs") *value = c->oc_last[1];
  else if (k == "krylov_onchip_clusters") *value = c->oc_last[2];
  else if (k == "krylov_block") *value = c->p_krylov_block;
  else if (k == "krylov_block_clusters") *value = c->p_krylov_block_clusters;
  else if (k == "krylov_refine") *value = c->p_krylov_refine;
  else if (k == "krylov_refine_digits") *value = c->p_krylov_refine_digits;
  else if (k == "krylov_stage") *value = c->p_krylov_stage;
  else if (k == "tri_refine") *value = c->p_tri_refine;
  else if (k == "tri_refine_rounds") *value = c->p_tri_refine_rounds;
  else if (k == "tri_refine_cluster") *value = c->p_tri_refine_cluster;
  else if (k == "krylov_block_last_systems") *value = c->bk_last[0];
  else if (k == "krylov_block_last_cs") *value = c->bk_last[1];
  else if (k == "krylov_block_last_clusters") *value = c->bk_last[2];
  else if (k == "orth_cluster") *value = c->p_orth_cluster;
  else if (k == "tri_spt") *value = c->p_tri_spt;
  else if (k == "tri_warp") *value = c->p_tri_warp;
  else if (k == "tri_chunk") *value = c->p_tri_chunk;
  else if (k == "tri_group") *value = c->p_tri_group;
  else if (k == "tri_wchunk") *value = c->p_tri_wchunk;
  else if (k == "tri_wsplit") *value = c->p_tri_wsplit;
  else if (k == "tri_wblock") *value = c->p_tri_wblock;
  else if (k == "tri_wtoep") *value = c->p_tri_wtoep;
  else if (k == "orth_tc") *value = c->p_orth_tc;
  else return set_err(c, LRP_EINVAL, "unknown parameter");
  return LRP_OK;
}

lrp_status lrp_set_kernel_timing(lrp_ctx* c, int enable) {
  if (!c) return LRP_EINVAL;
  c->timing = enable != 0;
  return LRP_OK;
}

lrp_status lrp_kernel_time(lrp_ctx* c, const char* fam, int* launches, double* total_ms) {
  if (!c || !fam) return LRP_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "synchronize");
  auto it = c->timers.find(fam);
  int nl = 0;
  double tot = 0.0;
  if (it != c->timers.end()) {
    KernelTimer& t = it->second;
    for (auto& pr : t.pairs) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      t.total_ms += ms;
      t.launches += 1;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    t.pairs.clear();
    nl = t.launches;
    tot = t.total_ms;
  }
  if (launches) *launches = nl;
  if (total_ms) *total_ms = tot;
  return LRP_OK;
}

lrp_status lrp_reset_kernel_time(lrp_ctx* c) {
  if (!c) return LRP_EINVAL;
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->timers)
    for (auto& pr : kv.second.pairs) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  c->timers.clear();
  return LRP_OK;
}

// ===========================================================================
// operators
// ===========================================================================
lrp_status lrp_operator_tridiag(lrp_ctx* c, int n, const double* lo, const double* di,
                                const double* up, lrp_operator** out) {
  if (!c || !out || !lo || !di || !up) return LRP_EINVAL;
  if (n < 2 || n > 16384) return set_err(c, LRP_EINVAL, "tridiagonal size must be 2..16384");
  cudaSetDevice(c->device);
  auto op = std::make_unique<lrp_operator>();
  op->ctx = c;
  ctx_retain(c);
  op->kind = 0;
  op->n = n;
  const double* src[3] = {lo, di, up};
  for (int k = 0; k < 3; ++k) {
    lrp_status s = dev_alloc(c, op->a64[k], sizeof(double) * n);
    if (s) return s;
    if ((s = to_device(c, op->a64[k].ptr, src[k], sizeof(double) * n))) return s;
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "operator upload");
  // constant coefficients (lo[1..n-1], di, up[0..n-2] each one value): the
  // one-warp kernel has a variant for them
  {
    std::vector<double> h(3 * (size_t)n);
    for (int k = 0; k < 3; ++k) {
      e = cudaMemcpy(h.data() + (size_t)k * n, op->a64[k].ptr, sizeof(double) * n, cudaMemcpyDeviceToHost);
      if (e) return cuda_err(c, e, "operator read-back");
    }
    const double* hl = h.data();
    const double* hd = hl + n;
    const double* hu = hd + n;
    bool toep = true;
    for (int i = 1; i < n && toep; ++i) toep = hl[i] == hl[1] && hd[i] == hd[0] && hu[i - 1] == hu[0];
    op->toeplitz = toep;
    op->tlo = hl[1];
    op->tdi = hd[0];
    op->tup = hu[0];
  }
  *out = op.release();
  return LRP_OK;
}

void lrp_operator_free(lrp_operator* op) {
  if (!op) return;
  cudaSetDevice(op->ctx->device);
  cudaStreamSynchronize(op->ctx->stream);
  delete op;
}

int lrp_operator_size(const lrp_operator* op) { return op ? op->n : 0; }

unsigned long long lrp_operator_krylov_iterations(const lrp_operator* op) {
  return op ? op->krylov_iters.load() : 0ULL;
}

lrp_status lrp_operator_set_krylov(lrp_operator* op, double rtol_f64, double rtol_f32,
                                   int max_iter) {
  if (!op || !(rtol_f64 > 0) || !(rtol_f32 > 0) || max_iter < 0) return LRP_EINVAL;
  op->rtol64 = rtol_f64;
  op->rtol32 = rtol_f32;
  op->max_iter = max_iter;
  return LRP_OK;
}

}  // extern "C"

// ===========================================================================
// propagation dispatch
// ===========================================================================
namespace lrp {
lrp_status stencil_propagate(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys,
                             int prec, const PropIn& in, const PropOut& out, const PropSrc& src);

StepCoef step_coefficients(int stepper) {
  // Butcher tableaus of the two SDIRK methods of Sec. 4 (effect of the time
  // discretisation): SDIRK2 with gamma = 1, a21 = -1, b = (1/2, 1/2);
  // SDIRK2-L with gamma = (2 - sqrt 2)/2, a21 = 1 - gamma, b = (1 - gamma, gamma)
  double g = 1.0, a21 = -1.0, b1 = 0.5, b2 = 0.5;
  if (stepper == LRP_STEP_SDIRK2_L) {
    g = (2.0 - std::sqrt(2.0)) / 2.0;
    a21 = 1.0 - g;
    b1 = 1.0 - g;
    b2 = g;
  }
  StepCoef sc;
  sc.gamma = g;
  sc.su = 1.0 - a21 / g;
  sc.s1 = a21 / g;
  sc.bu = 1.0 - b1 / g - b2 / g + b2 * a21 / (g * g);
  sc.b1 = b1 / g - b2 * a21 / (g * g);
  sc.b2 = b2 / g;
  return sc;
}

// Source samples per fine step: the two stage times of an SDIRK step, else
// the step end.
int source_samples(const Operator* op) { return op->stepper != 0 ? 2 : 1; }

lrp_status propagate_any(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys, int prec,
                         const PropIn& in, const PropOut& out, const PropSrc& src) {
  if (op->kind == 2) return tri_td_propagate(c, op, dt, M, adjoint, nsys, prec, in, out, src);
  if (op->kind == 0 && op->stepper != 0) {
    // SDIRK fine steps: two solves with B = I + gamma dt A per step on the
    // one-CTA-per-system kernel; a source brings two samples per step (the
    // stage times), src.cstride counts them
    const double dtg = dt * step_coefficients(op->stepper).gamma;
    // chunks of at most 8 rows (three chunk states in registers); one CTA per
    // system while its factors fit in shared memory, else a 4-CTA cluster
    const int m = op->n >= 32 ? 8 : 4;
    const int P = (op->n + m - 1) / m;
    int L = 0;
    while ((1 << L) < P) ++L;
    const size_t one_cta = (size_t)(prec == 0 ? 8 : 4) * ((size_t)5 * m * P + (size_t)(2 * L + 1) * P + 3 * P);
    if (one_cta > 200 * 1024 && m == 8 && (P + 3) / 4 >= 32 && (P + 3) / 4 <= 256) {
      ClPlan* cp = nullptr;
      lrp_status s = tri_get_cluster_plan(c, op, dtg, adjoint, 4, 8, &cp);
      if (s) return s;
      return tri_propagate_cluster(c, cp, M, nsys, prec, 1, in, out, src, op->stepper);
    }
    TriPlan* plan = nullptr;
    lrp_status s = tri_get_plan(c, op, dtg, adjoint, &plan, m);
    if (s) return s;
    return tri_propagate(c, op, plan, M, nsys, prec, in, out, src);
  }
  if (op->kind == 0 && tri_ir_applies(c, op, prec, adjoint, M, in, src))
    return tri_propagate_ir(c, op, dt, M, nsys, in, out);
  if (op->kind == 0) {
    // Small batches of long systems: spread every system over a cluster of
    // C CTAs (chunks of m rows, spt systems per thread) so that more SMs take
    // part; otherwise one CTA per system.
    int C = 1, m = 16, spt = 1;
    auto fits = [&](int cc, int mm) {
      int P = (op->n + mm - 1) / mm;
      int Pc = (P + cc - 1) / cc;
      return Pc >= 32 && Pc <= 256 && Pc * cc <= 1024;
    };
    if (c->p_tri_cluster > 1) {
      C = c->p_tri_cluster;
      m = c->p_tri_chunk ? c->p_tri_chunk : 16;
      spt = c->p_tri_spt ? c->p_tri_spt : 1;
      if (!fits(C, m)) C = 1;
    } else if (c->p_tri_cluster == 0 && op->n >= 2048) {
      // measured on GB300 (adr1d, n = 4095, 64 systems, FP64): 4 CTAs with
      // 8-row chunks 1.13 ms, 2 CTAs with 16-row chunks 1.26 ms, one CTA per
      // system 1.90 ms; clusters beyond the resident ones run in a second wave.
      // Systems too long for one CTA's shared memory always take a cluster.
      const int m1 = op->n >= 1024 ? 32 : 16;
      const int P1 = (op->n + m1 - 1) / m1;
      int L1 = 0;
      while ((1 << L1) < P1) ++L1;
      const size_t one_cta = (size_t)(prec == 0 ? 8 : 4) *
                             ((size_t)5 * m1 * P1 + (size_t)(2 * L1 + 1) * P1 + 3 * (size_t)P1);
      const bool small_batch = nsys * 2 <= c->num_sms;
      const bool must = (one_cta > 220 * 1024 || P1 > 512) && !(prec == 1 && op->n <= 4096);
      if (small_batch || must) {
        // block kernel (FP32, or the one-warp kernel disabled): measured on
        // GB300 (n = 4095, FP64): 4-CTA clusters of 8-row chunks 1.26 ms per
        // 256 steps, 8-CTA 1.10-1.26, 2-CTA 1.35, 3/5/6/7-CTA up to 1.7 (their
        // clusters do not all fit at once)
        const int cand[4][2] = {{4, 8}, {8, 8}, {2, 16}, {4, 16}};
        for (auto& cm : cand)
          if (fits(cm[0], cm[1])) { C = cm[0]; m = cm[1]; break; }
      }
      if (c->p_tri_chunk) m = c->p_tri_chunk;
      if (c->p_tri_spt) spt = c->p_tri_spt;
      if (C > 1 && !fits(C, m)) { C = 1; }
    }
    // FP64 batches of up to ~7 warps per SM sub-partition with 256 < n <=
    // 4096: the one-warp-per-CTA cluster kernel (factors in registers, no
    // block barrier, 32 chunks per CTA).  Its time per step is the FP64 issue
    // of the warps sharing a sub-partition (~80 cycles per FP64 warp
    // instruction on GB300), so the chunk length MM (8..16 rows) trades the
    // number of warps, n / (32 MM) per system, against the interface work
    // per row.  Measured on GB300 (n = 4095, 256 steps, ms; wpp8 = warps per
    // sub-partition with 8-row chunks):
    //   systems  wpp8   MM=8   9      10     11     12     13     14     15     16
    //   16       0.42   0.653  0.661  0.718  0.743  0.808  0.813  0.852  0.922  0.972
    //   24       0.63   0.686  0.674  0.722  0.743  0.823  0.814  0.852  0.929  0.979
    //   32       0.84   0.697  0.692  0.735  0.749  0.827  0.815  0.855  0.934  0.982
    //   40       1.05   0.742  0.768  0.747  0.767  0.830  0.815  0.854  0.941  0.987
    //   44       1.16   0.813  0.845  0.814  0.766  0.827  0.843  0.883  0.941  0.984
    //   48       1.26   0.897  0.845  0.892  0.852  0.852  0.845  0.886  0.976  0.987
    //   52       1.37   0.916  0.877  0.896  0.856  0.915  0.844  0.886  0.976  1.010
    //   56       1.47   1.028  0.951  0.908  0.856  0.917  0.845  0.886  0.976  1.016
    //   60       1.58   1.029  0.971  0.914  0.956  0.926  0.961  1.021  0.976  1.027
    //   64       1.68   1.079  1.102  1.031  0.957  0.938  0.964  1.023  1.096  1.027
    //   80       2.11   1.706  1.742  1.177  1.088  1.166  1.076  1.140  1.097  1.160
    //   96       2.53   1.754  1.773  1.869  1.272  1.327  1.215  1.287  1.231  1.274
    //   128      3.37   2.100  2.060  1.977  2.011  2.170  2.178  2.300  2.445  1.634
    //   160      4.21   2.825  2.842  2.355  2.218  2.281  2.190  2.316  2.459  2.596
    //   192      5.05   3.160  3.129  3.040  2.499  2.569  2.435  2.580  2.618  2.599
    //   256      6.74   4.110  4.136  4.194  3.440  3.575  3.544  3.749  3.962  2.904
    // (the block kernel takes 1.30 ms from 40 to 64 systems and the one-CTA
    // kernel 3.80 ms at 192 and 256; beyond ~7 warps per sub-partition the
    // one-CTA kernel is faster: 5.94 against 6.51 ms at 512 systems).
    const int Cw8 = ((op->n + 7) / 8 + 31) / 32;
    const double wpp = (double)nsys * Cw8 / (4.0 * c->num_sms);   // warps per sub-partition, 8-row chunks
    // (n = 511 and 1023, 16 systems, 64 steps: 0.162 / 0.167 ms against 0.254 /
    // 0.267 ms for the one-CTA kernel; n = 255, one CTA: 0.160 against 0.146)
    const bool warp_auto = c->p_tri_warp == 0 && Cw8 >= 2 && Cw8 <= 16 && wpp <= 7.0;
    if ((warp_auto || c->p_tri_warp == 2) && prec == 0 && c->p_tri_wblock != 1 && c->p_tri_cluster == 0 &&
        c->p_tri_chunk == 0 && c->p_tri_spt == 0) {
      int mw = c->p_tri_wchunk;
      if (!mw)
        mw = wpp <= 1.1 ? 8 : wpp <= 1.2 ? 11 : wpp <= 1.5 ? 13 : wpp <= 1.75 ? 12
           : wpp <= 2.8 ? 13 : wpp <= 3.8 ? 16 : wpp <= 5.5 ? 13 : 16;
      int Cw = ((op->n + mw - 1) / mw + 31) / 32;
      if (Cw < 2 && c->p_tri_wchunk == 0) {
        mw = 8;
        Cw = Cw8;
      }
      // constant-coefficient operators without a source: the Toeplitz
      // variant (two FP64 instructions per row for the chunk solve instead of
      // three), on the chunk length nearest the rule's (the larger on a tie)
      // for which n mod MM is 0 or MM - 1
      // Measured on GB300 (n = 4095, 256 steps, ms per launch, general kernel
      // in brackets; chunk lengths 8, 9, 13, 15, 16 are the ones with n mod
      // MM in {0, MM - 1}): 16 systems MM = 8 0.664 (0.662); 40 systems
      // MM = 9 0.723 (MM = 8 0.739); 48-56 systems MM = 13 0.765 (0.814-0.843);
      // 60 systems MM = 15 0.826 (MM = 12 0.950); 64 systems MM = 13 0.863
      // (0.954); 96 systems MM = 15 1.041 (1.217); 128 systems MM = 16 1.412
      // (1.633).
      ToepCoef tz{};
      if (op->toeplitz && src.Q == 0 && c->p_tri_wtoep != 2) {
        if (!c->p_tri_wchunk)
          mw = wpp <= 0.55 ? 8 : wpp <= 1.1 ? 9 : wpp <= 1.5 ? 13 : wpp <= 1.6 ? 15
             : wpp <= 1.75 ? 13 : wpp <= 2.8 ? 15 : wpp <= 3.8 ? 16 : wpp <= 5.5 ? 13 : 16;
        int best = 0;
        for (int d = 0; d <= 8 && !best; ++d) {
          const int cands[2] = {mw + d, mw - d};
          for (int cand : cands)
            if (!best && cand >= 8 && cand <= 16 && (op->n % cand == 0 || (op->n + 1) % cand == 0) &&
                (c->p_tri_wchunk == 0 || cand == mw))
              best = cand;
        }
        if (best) {
          const int Cb = ((op->n + best - 1) / best + 31) / 32;
          if (Cb >= 1 && Cb <= 16) {
            tri_toeplitz_coef(op, dt, adjoint, M, best, &tz);
            if (tz.on) { mw = best; Cw = Cb; }
          }
        }
      }
      if (c->p_tri_wtoep == 1 && !tz.on)
        return set_err(c, LRP_EINVAL, "constant-coefficient kernel not applicable");
      if (Cw >= 1 && Cw <= 16) {
        ClPlan* cp = nullptr;
        lrp_status s = tri_get_cluster_plan(c, op, dt, adjoint, Cw, mw, &cp, 1);
        if (s) return s;
        return tri_propagate_cluster(c, cp, M, nsys, prec, 1, in, out, src, 0, tz.on ? &tz : nullptr);
      }
    }
    // FP32 batches (the sketches), and FP64 on request: one system per CTA
    // of C warps (k_tri_block_w), the one-warp kernel's steps with the
    // exchange through shared memory; chunks of 8, 12 or 16 rows.  Measured
    // on GB300 (FP32, 256 steps, ms per launch; the register-chunk kernel
    // k_tri_propagate_rc in brackets): n = 4095, 1536 systems: 16-row chunks
    // 0.731, 12-row 1.265, 8-row 1.255 (1.012); 192 systems: 0.143 (0.289);
    // n = 255, 64 steps, 1536 systems: 8-row 0.032, 16-row 0.035 (0.062).
    // In FP64 it does not beat the one-CTA kernel (n = 4095, 1536 systems:
    // 17.86 against 17.78 ms) and runs only on request.
    {
      const int wc = c->p_tri_wchunk;
      const int mb = (wc == 8 || wc == 12 || wc == 16) ? wc : op->n >= 1024 ? 16 : 8;
      const int Cb = ((op->n + mb - 1) / mb + 31) / 32;
      const bool blk_auto = c->p_tri_wblock == 0 && prec == 1 && C == 1 && c->p_tri_cluster == 0 &&
                            c->p_tri_chunk == 0 && c->p_tri_spt == 0;
      // Constant-coefficient batches without a source (FP64, and the FP32
      // ones that take no cluster): the block variant of the
      // constant-coefficient kernel, on the longest chunk
      // length with n mod MM in {0, MM - 1}, 2 to 8 warps per system and the
      // warps at least three quarters full.  Measured on GB300 (ms per
      // launch, the one-CTA-per-system kernel in brackets): n = 4095, 256
      // steps: 300 systems 2.81 (3.80), 1536 systems 15.35 (17.74), 3072
      // systems 29.3 (32.5); n = 1023, 64 steps, 512 systems: 0.326 (0.372);
      // a single half-full warp per system (n = 255) is slower: 0.213 (0.144).
      if ((prec == 0 || C == 1) && op->toeplitz && src.Q == 0 && c->p_tri_wtoep != 2 &&
          c->p_tri_wblock != 2 && c->p_tri_cluster == 0 && c->p_tri_chunk == 0 && c->p_tri_spt == 0) {
        for (int mm = 16; mm >= 8; --mm) {
          if ((wc && mm != wc) || (op->n % mm != 0 && (op->n + 1) % mm != 0)) continue;
          const int chunks = (op->n + mm - 1) / mm;
          const int Ct = (chunks + 31) / 32;
          if (Ct < 2 || Ct > 8 || 4 * chunks < 3 * 32 * Ct) continue;
          ToepCoef tzb{};
          tri_toeplitz_coef(op, dt, adjoint, M, mm, &tzb, prec);
          if (!tzb.on) continue;
          ClPlan* cp = nullptr;
          lrp_status s = tri_get_cluster_plan(c, op, dt, adjoint, Ct, mm, &cp, 1);
          if (s) return s;
          return tri_propagate_warp_block(c, cp, M, nsys, prec, in, out, src, &tzb);
        }
      }
      if ((blk_auto || c->p_tri_wblock == 1) && Cb >= 1 && Cb <= 16) {
        ClPlan* cp = nullptr;
        lrp_status s = tri_get_cluster_plan(c, op, dt, adjoint, Cb, mb, &cp, 1);
        if (s) return s;
        return tri_propagate_warp_block(c, cp, M, nsys, prec, in, out, src);
      }
    }
    if (C > 1) {
      ClPlan* cp = nullptr;
      lrp_status s = tri_get_cluster_plan(c, op, dt, adjoint, C, m, &cp);
      if (s) return s;
      return tri_propagate_cluster(c, cp, M, nsys, prec, spt, in, out, src);
    }
    // FP32 with n in [256, 4096]: chunks of 16 rows keep the factors in
    // registers (k_tri_propagate_rc)
    const int m_req = (prec == 1 && op->n >= 256 && op->n <= 4096) ? 16 : 0;
    TriPlan* plan = nullptr;
    lrp_status s = tri_get_plan(c, op, dt, adjoint, &plan, m_req);
    if (s) return s;
    return tri_propagate(c, op, plan, M, nsys, prec, in, out, src);
  }
  return stencil_propagate(c, op, dt, M, adjoint, nsys, prec, in, out, src);
}
}  // namespace lrp

extern "C" {

lrp_status lrp_propagate(lrp_ctx* c, const lrp_operator* opc, double dt, int M, int adjoint,
                         int nvec, const double* x_in, double* x_out, int Q, const double* g,
                         const double* cv, lrp_precision prec) {
  if (!c || !opc || !x_out || nvec < 0 || M < 0 || !(dt > 0) || Q < 0) return LRP_EINVAL;
  if (adjoint && Q > 0) return set_err(c, LRP_EINVAL, "the adjoint propagates the linear part only");
  if (Q > 0 && (!g || !cv)) return LRP_EINVAL;
  if (nvec == 0) return LRP_OK;
  cudaSetDevice(c->device);
  Operator* op = const_cast<lrp_operator*>(opc);
  const int n = op->n;
  size_t vb = sizeof(double) * (size_t)nvec * n;
  DevView xin, gv, cvv;
  lrp_status s;
  if ((s = device_view(c, x_in, vb, xin))) return s;
  if ((s = device_view(c, g, sizeof(double) * (size_t)Q * n, gv))) return s;
  const int sps = source_samples(op);
  if ((s = device_view(c, cv, sizeof(double) * (size_t)nvec * M * sps * Q, cvv))) return s;
  bool out_dev = is_device_ptr(x_out);
  DevBuf tmp_out;
  void* dout = x_out;
  if (!out_dev) {
    if ((s = dev_alloc(c, tmp_out, vb))) return s;
    dout = tmp_out.ptr;
  }
  PropIn in;
  in.x = xin.p;
  in.x_f64 = 1;
  in.ldx = n;
  in.ncol = std::max(nvec, 1);   // time-dependent operators: every vector from t = 0
  PropOut o;
  o.y = dout;
  o.y_f64 = 1;
  o.ldy = n;
  PropSrc src;
  src.Q = Q;
  src.g = (const double*)gv.p;
  src.c = (const double*)cvv.p;
  src.cstride = (long)M * sps * Q;
  if ((s = propagate_any(c, op, dt, M, adjoint, nvec, prec == LRP_PREC_MIXED ? 1 : 0, in, o, src)))
    return s;
  if (!out_dev) {
    if ((s = from_device(c, x_out, dout, vb))) return s;
  } else {
    cudaError_t e = cudaStreamSynchronize(c->stream);  // temporaries are freed on return
    if (e) return cuda_err(c, e, "propagate");
  }
  return LRP_OK;
}

lrp_status lrp_gaussian(lrp_ctx* c, uint64_t seed, int interval, int ncol, int n,
                        lrp_precision prec, double* out) {
  if (!c || !out || ncol < 0 || n < 0 || interval < 0) return LRP_EINVAL;
  cudaSetDevice(c->device);
  size_t bytes = sizeof(double) * (size_t)ncol * n;
  bool dev = is_device_ptr(out);
  DevBuf tmp;
  double* d = out;
  lrp_status s;
  if (!dev) {
    if ((s = dev_alloc(c, tmp, bytes))) return s;
    d = tmp.as<double>();
  }
  if ((s = gaussian(c, seed, interval, ncol, n, prec == LRP_PREC_MIXED, d))) return s;
  if (!dev) return from_device(c, out, d, bytes);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e ? cuda_err(c, e, "gaussian") : LRP_OK;
}

// ===========================================================================
// coarse solvers: randomized SVD of every interval (Sec. 2.1)
// ===========================================================================
lrp_status lrp_build_coarse(lrp_ctx* c, const lrp_operator* opc, double dt, int M, int N,
                            int rank, int oversample, uint64_t seed, lrp_precision prec,
                            lrp_coarse** out) {
  return lrp_build_coarse_ex(c, opc, dt, M, N, rank, oversample, seed, prec, 0, out);
}

lrp_status lrp_build_coarse_ex(lrp_ctx* c, const lrp_operator* opc, double dt, int M, int N,
                               int rank, int oversample, uint64_t seed, lrp_precision prec,
                               int flags, lrp_coarse** out) {
  if (!c || !opc || !out || !(dt > 0) || M < 1 || N < 1 || rank < 0 || oversample < 0 ||
      (flags & ~LRP_BUILD_INDEPENDENT_ADJOINT))
    return LRP_EINVAL;
  const bool two_sided = (flags & LRP_BUILD_INDEPENDENT_ADJOINT) != 0;
  const int ell = rank + oversample;
  if (ell < 1) return set_err(c, LRP_EINVAL, "rank + oversample must be >= 1");
  if (rank > 64 || ell > 128) return set_err(c, LRP_EINVAL, "rank <= 64 and rank+oversample <= 128");
  cudaSetDevice(c->device);
  Operator* op = const_cast<lrp_operator*>(opc);
  const int n = op->n;
  if (ell > n) return set_err(c, LRP_EINVAL, "rank + oversample exceeds the dimension");
  if ((op->kind == 2 || op->kind == 3) && (long)N * M > op->nJ)
    return set_err(c, LRP_EINVAL, "N * M exceeds the time grid of the operator");
  auto co = std::make_unique<lrp_coarse>();
  co->ctx = c;
  ctx_retain(c);
  co->op = op;
  co->dt = dt;
  co->M = M;
  co->N = N;
  co->R = rank;
  co->p = oversample;
  co->ell = ell;
  co->seed = seed;
  co->prec = prec;
  const int f32 = prec == LRP_PREC_MIXED;
  const size_t es = f32 ? 4 : 8;
  const size_t blk = (size_t)N * ell * n;
  DevBuf Y, Z, Rw, Rz, rw, rv, sv, Psi, Phi, st, Rid;
  lrp_status s;
  if ((s = dev_alloc(c, Y, blk * es))) return s;
  if ((s = dev_alloc(c, Z, blk * es))) return s;
  if ((s = dev_alloc(c, Rw, sizeof(double) * N * ell * ell))) return s;
  if ((s = dev_alloc(c, Rz, sizeof(double) * N * ell * ell))) return s;
  if ((s = dev_alloc(c, rw, sizeof(int) * N))) return s;
  if ((s = dev_alloc(c, rv, sizeof(int) * N))) return s;
  if ((s = dev_alloc(c, sv, sizeof(double) * N * ell))) return s;
  if ((s = dev_alloc(c, Psi, sizeof(double) * N * ell * ell))) return s;
  if ((s = dev_alloc(c, Phi, sizeof(double) * N * ell * ell))) return s;
  if ((s = dev_alloc(c, st, sizeof(int)))) return s;
  if ((s = dev_alloc(c, Rid, sizeof(int) * N))) return s;
  cudaMemsetAsync(st.ptr, 0, sizeof(int), c->stream);
  const double tau = f32 ? 2e-5 : 1e-13;
  // workspace of the tensor-core orthonormalisation (FP32 sketches)
  DevBuf ows, tcc;
  if ((s = dev_alloc(c, tcc, 2 * sizeof(int)))) return s;
  cudaMemsetAsync(tcc.ptr, 0, 2 * sizeof(int), c->stream);
  if (orth_tc_applies(c, ell, !f32))
    if ((s = dev_alloc(c, ows, orth_tc_workspace(c, N, ell, n)))) return s;
  auto orth = [&](void* X, double* Rc, int* rk, int which) {
    return orth_auto(c, N, ell, n, X, !f32, tau, Rc, rk, ows.ptr, ows.bytes, st.as<int>(),
                     tcc.as<int>() + which);
  };
  // step 1: Y = F' Omega, Omega generated in the kernel (N*ell systems)
  PropIn in;
  in.gen = 1;
  in.seed = seed;
  in.ncol = ell;
  in.interval0 = 0;
  PropOut o;
  o.y = Y.ptr;
  o.y_f64 = !f32;
  o.ldy = n;
  PropSrc nosrc;
  if ((s = propagate_any(c, op, dt, M, 0, N * ell, f32, in, o, nosrc))) return s;
  if (two_sided) {
    // F'^* on 2 l independent random vectors psi (Philox stream 3), with no
    // dependence on the forward sketch; Q = orth(Y); X^T = Z (Psi^T Q)^+T;
    // Vh = orth(X^T) with X = Rz^T Vh, so the small SVD below is that of X.
    const int ell2 = 2 * ell;
    DevBuf Z2, Bb, Cb;
    if ((s = dev_alloc(c, Z2, (size_t)N * ell2 * n * es))) return s;
    if ((s = dev_alloc(c, Bb, sizeof(double) * (size_t)N * ell2 * ell))) return s;
    if ((s = dev_alloc(c, Cb, sizeof(double) * (size_t)N * ell2 * ell))) return s;
    PropIn ina;
    ina.gen = 1;
    ina.seed = seed;
    ina.stream = 3;
    ina.ncol = ell2;
    ina.interval0 = 0;
    PropOut oa;
    oa.y = Z2.ptr;
    oa.y_f64 = !f32;
    oa.ldy = n;
    if ((s = propagate_any(c, op, dt, M, 1, N * ell2, f32, ina, oa, nosrc))) return s;
    if ((s = orth(Y.ptr, Rw.as<double>(), rw.as<int>(), 0))) return s;
    if ((s = two_sided_core(c, N, ell, ell2, n, seed, f32, Y.ptr, rw.as<int>(), Z2.ptr, Z.ptr,
                            Bb.as<double>(), Cb.as<double>(), st.as<int>())))
      return s;
    if ((s = orth(Z.ptr, Rz.as<double>(), rv.as<int>(), 1))) return s;
    cudaStreamSynchronize(c->stream);    // Z2, Bb, Cb are released here
  } else {
  // step 2: W = orth(Y), in place
  if ((s = orth(Y.ptr, Rw.as<double>(), rw.as<int>(), 0))) return s;
  // step 3: Z = F'^* W
  PropIn in2;
  in2.x = Y.ptr;
  in2.x_f64 = !f32;
  in2.ldx = n;
  in2.ncol = ell;               // system s is column s % ell of interval s / ell
  PropOut o2;
  o2.y = Z.ptr;
  o2.y_f64 = !f32;
  o2.ldy = n;
  if ((s = propagate_any(c, op, dt, M, 1, N * ell, f32, in2, o2, nosrc))) return s;
  // step 4: Vh = orth(Z) in place; M_ij = (z_i, v_j) = Rz[j][i]
  if ((s = orth(Z.ptr, Rz.as<double>(), rv.as<int>(), 1))) return s;
  }
  // step 5: SVD of M
  if ((s = small_svd(c, N, ell, Rz.as<double>(), rv.as<int>(), sv.as<double>(), Psi.as<double>(),
                     Phi.as<double>(), st.as<int>())))
    return s;
  // R_i and S on the device, then the lift (step 6) and the chain matrices
  // of the sweep; the host reads ranks, singular values and statuses once,
  // at the end
  const int Rm = std::max(rank, 1);
  if ((s = dev_alloc(c, co->U, sizeof(double) * N * Rm * (size_t)n))) return s;
  if ((s = dev_alloc(c, co->V, sizeof(double) * N * Rm * (size_t)n))) return s;
  if ((s = dev_alloc(c, co->S, sizeof(double) * N * Rm))) return s;
  if ((s = dev_alloc(c, co->U32, sizeof(float) * N * Rm * (size_t)n))) return s;
  if ((s = dev_alloc(c, co->V32, sizeof(float) * N * Rm * (size_t)n))) return s;
  if ((s = dev_alloc(c, co->S32, sizeof(float) * N * Rm))) return s;
  const bool ltc = lift_tc_applies(c, ell, rank, !f32);
  if (!ltc) {
    // the SIMT lift writes the rows below R_i only
    cudaMemsetAsync(co->U.ptr, 0, co->U.bytes, c->stream);
    cudaMemsetAsync(co->V.ptr, 0, co->V.bytes, c->stream);
    cudaMemsetAsync(co->U32.ptr, 0, co->U32.bytes, c->stream);
    cudaMemsetAsync(co->V32.ptr, 0, co->V32.bytes, c->stream);
  }
  k_finish_ranks<<<(N + 127) / 128, 128, 0, c->stream>>>(N, rank, ell, rw.as<int>(), rv.as<int>(),
                                                         sv.as<double>(), Rid.as<int>(),
                                                         co->S.as<double>(), co->S32.as<float>());
  ++c->launches;
  if (ltc) {
    if ((s = lift_tc(c, N, ell, rank, n, Y.as<float>(), Z.as<float>(), Psi.as<double>(),
                     Phi.as<double>(), Rid.as<int>(), co->U.as<double>(), co->V.as<double>(),
                     co->U32.as<float>(), co->V32.as<float>(), st.as<int>())))
      return s;
  } else if ((s = lift(c, N, ell, rank, n, Y.ptr, Z.ptr, !f32, Psi.as<double>(), Phi.as<double>(),
                       Rid.as<int>(), co->U.as<double>(), co->V.as<double>(), co->U32.as<float>(),
                       co->V32.as<float>()))) {
    return s;
  }
  if ((s = coarse_chain(c, co.get()))) return s;
  co->rank_w.resize(N);
  co->rank_v.resize(N);
  co->sigma.resize((size_t)N * ell);
  int svd_status = 0;
  int tc_counts[2] = {0, 0};
  cudaMemcpyAsync(co->rank_w.data(), rw.ptr, sizeof(int) * N, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(co->rank_v.data(), rv.ptr, sizeof(int) * N, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(co->sigma.data(), sv.ptr, sizeof(double) * N * ell, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(&svd_status, st.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(tc_counts, tcc.ptr, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "build_coarse");
  co->orth_tc_w = tc_counts[0];
  co->orth_tc_v = tc_counts[1];
  if (svd_status & 4) return set_err(c, LRP_EBREAKDOWN, "tensor-core orthonormalisation or lift failed");
  if (svd_status & 2) return set_err(c, LRP_EBREAKDOWN, "rank-deficient two-sided sketch core");
  if (svd_status) return set_err(c, LRP_ENOTCONV, "Jacobi SVD did not converge");
  // R_i, sigma_{R_i+1}, delta, eps (as k_finish_ranks)
  co->Ri.resize(N);
  co->delta = 0.0;
  co->eps = 0.0;
  for (int i = 0; i < N; ++i) {
    int kk = std::min(co->rank_w[i], co->rank_v[i]);
    int Ri = std::min(rank, kk);
    co->Ri[i] = Ri;
    const double* si = &co->sigma[(size_t)i * ell];
    for (int r = kk; r < ell; ++r) co->sigma[(size_t)i * ell + r] = 0.0;
    double s1 = kk > 0 ? si[0] : 0.0;
    // sigma_{R_i+1} from the oversampled SVD; when deflation left no (R_i+1)-th
    // value, the dropped directions were below tau * sigma_1
    double sn = (kk > Ri) ? si[Ri] : tau * s1;
    co->delta = std::max(co->delta, s1);
    co->eps = std::max(co->eps, sn);
  }
  *out = co.release();
  return LRP_OK;
}

void lrp_coarse_free(lrp_coarse* co) {
  if (!co) return;
  cudaSetDevice(co->ctx->device);
  cudaStreamSynchronize(co->ctx->stream);
  delete co;
}

lrp_status lrp_coarse_orth_method(const lrp_coarse* co, int* tc_w, int* tc_v) {
  if (!co) return LRP_EINVAL;
  if (tc_w) *tc_w = co->orth_tc_w;
  if (tc_v) *tc_v = co->orth_tc_v;
  return LRP_OK;
}

lrp_status lrp_coarse_info(const lrp_coarse* co, int* R_i, int* rank_w, int* rank_v,
                           double* sigma, double* delta, double* eps) {
  if (!co) return LRP_EINVAL;
  const int N = co->N;
  if (R_i) std::memcpy(R_i, co->Ri.data(), sizeof(int) * N);
  if (rank_w) std::memcpy(rank_w, co->rank_w.data(), sizeof(int) * N);
  if (rank_v) std::memcpy(rank_v, co->rank_v.data(), sizeof(int) * N);
  if (sigma) std::memcpy(sigma, co->sigma.data(), sizeof(double) * N * co->ell);
  if (delta) *delta = co->delta;
  if (eps) *eps = co->eps;
  return LRP_OK;
}

lrp_status lrp_coarse_factors(const lrp_coarse* co, int interval, double* U, double* S,
                              double* V) {
  if (!co || interval < 0 || interval >= co->N) return LRP_EINVAL;
  Ctx* c = co->ctx;
  const int n = co->op->n, Rm = std::max(co->R, 1), Ri = co->Ri[interval];
  size_t off = (size_t)interval * Rm * n;
  lrp_status s;
  if (U && (s = from_device(c, U, co->U.as<double>() + off, sizeof(double) * Ri * n))) return s;
  if (V && (s = from_device(c, V, co->V.as<double>() + off, sizeof(double) * Ri * n))) return s;
  if (S && (s = from_device(c, S, co->S.as<double>() + (size_t)interval * Rm, sizeof(double) * Ri)))
    return s;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e ? cuda_err(c, e, "coarse_factors") : LRP_OK;
}

// ---- checkpoint: export / import of a coarse handle ------------------------
lrp_status lrp_coarse_export(const lrp_coarse* co, int* meta_i, double* meta_d, uint64_t* seed,
                             int* R_i, int* rank_w, int* rank_v, double* sigma, double* U,
                             double* S, double* V) {
  if (!co || !meta_i || !meta_d) return LRP_EINVAL;
  Ctx* c = co->ctx;
  const int n = co->op->n, N = co->N, Rm = std::max(co->R, 1);
  meta_i[0] = co->M; meta_i[1] = N; meta_i[2] = co->R; meta_i[3] = co->p; meta_i[4] = n;
  meta_i[5] = (int)co->prec;
  meta_d[0] = co->dt; meta_d[1] = co->delta; meta_d[2] = co->eps;
  if (seed) *seed = co->seed;
  if (R_i) std::memcpy(R_i, co->Ri.data(), sizeof(int) * N);
  if (rank_w) std::memcpy(rank_w, co->rank_w.data(), sizeof(int) * N);
  if (rank_v) std::memcpy(rank_v, co->rank_v.data(), sizeof(int) * N);
  if (sigma) std::memcpy(sigma, co->sigma.data(), sizeof(double) * (size_t)N * co->ell);
  lrp_status s;
  if (U && (s = from_device(c, U, co->U.ptr, sizeof(double) * (size_t)N * Rm * n))) return s;
  if (V && (s = from_device(c, V, co->V.ptr, sizeof(double) * (size_t)N * Rm * n))) return s;
  if (S && (s = from_device(c, S, co->S.ptr, sizeof(double) * (size_t)N * Rm))) return s;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e ? cuda_err(c, e, "coarse export") : LRP_OK;
}

__global__ static void k_copy_f32(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b[k] = (float)a[k];
}

lrp_status lrp_coarse_import(lrp_ctx* c, const lrp_operator* opc, const int* meta_i,
                             const double* meta_d, uint64_t seed, const int* R_i,
                             const int* rank_w, const int* rank_v, const double* sigma,
                             const double* U, const double* S, const double* V,
                             lrp_coarse** out) {
  if (!c || !opc || !meta_i || !meta_d || !R_i || !rank_w || !rank_v || !sigma || !U || !S || !V ||
      !out)
    return LRP_EINVAL;
  if (meta_i[4] != opc->n || meta_i[1] < 1 || meta_i[2] < 0 || meta_i[3] < 0 || meta_i[0] < 1)
    return set_err(c, LRP_EINVAL, "checkpoint does not match the operator");
  cudaSetDevice(c->device);
  auto co = std::make_unique<lrp_coarse>();
  co->ctx = c;
  ctx_retain(c);
  co->op = const_cast<lrp_operator*>(opc);
  co->M = meta_i[0]; co->N = meta_i[1]; co->R = meta_i[2]; co->p = meta_i[3];
  co->ell = co->R + co->p;
  co->prec = (lrp_precision)meta_i[5];
  co->dt = meta_d[0]; co->delta = meta_d[1]; co->eps = meta_d[2];
  co->seed = seed;
  const int N = co->N, n = opc->n, Rm = std::max(co->R, 1);
  co->Ri.assign(R_i, R_i + N);
  co->rank_w.assign(rank_w, rank_w + N);
  co->rank_v.assign(rank_v, rank_v + N);
  co->sigma.assign(sigma, sigma + (size_t)N * co->ell);
  const size_t nf = (size_t)N * Rm * n, ns = (size_t)N * Rm;
  lrp_status s;
  if ((s = dev_alloc(c, co->U, 8 * nf))) return s;
  if ((s = dev_alloc(c, co->V, 8 * nf))) return s;
  if ((s = dev_alloc(c, co->S, 8 * ns))) return s;
  if ((s = dev_alloc(c, co->U32, 4 * nf))) return s;
  if ((s = dev_alloc(c, co->V32, 4 * nf))) return s;
  if ((s = dev_alloc(c, co->S32, 4 * ns))) return s;
  if ((s = to_device(c, co->U.ptr, U, 8 * nf))) return s;
  if ((s = to_device(c, co->V.ptr, V, 8 * nf))) return s;
  if ((s = to_device(c, co->S.ptr, S, 8 * ns))) return s;
  k_copy_f32<<<(unsigned)((nf + 255) / 256), 256, 0, c->stream>>>(co->U.as<double>(), co->U32.as<float>(), nf);
  k_copy_f32<<<(unsigned)((nf + 255) / 256), 256, 0, c->stream>>>(co->V.as<double>(), co->V32.as<float>(), nf);
  k_copy_f32<<<(unsigned)((ns + 255) / 256), 256, 0, c->stream>>>(co->S.as<double>(), co->S32.as<float>(), ns);
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_err(c, e, "coarse import");
  if ((s = coarse_chain(c, co.get()))) return s;
  e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "coarse import");
  *out = co.release();
  return LRP_OK;
}

// ===========================================================================
// Parareal solve (Eq. def_Parareal in the delta form of Remark rem:affine_g_n)
// ===========================================================================
lrp_status lrp_parareal_solve(lrp_ctx* c, const lrp_coarse* coc, const double* u0, int Q,
                              const double* g, const double* cv, int K_max, double tol,
                              double* u_out, double* bound_out, int* k_done,
                              lrp_solve_stats* stats) {
  if (!c || !coc || !u0 || !u_out || Q < 0 || K_max < 0) return LRP_EINVAL;
  if (Q > 0 && (!g || !cv)) return LRP_EINVAL;
  cudaSetDevice(c->device);
  lrp_coarse* co = const_cast<lrp_coarse*>(coc);
  Operator* op = const_cast<Operator*>(co->op);
  const int n = op->n, N = co->N, M = co->M, Rm = std::max(co->R, 1);
  const int K = std::min(K_max, N);
  lrp_status s;
  // workspace
  if (!co->ws_u.ptr) {
    if ((s = dev_alloc(c, co->ws_u, sizeof(double) * (size_t)(N + 1) * n))) return s;
    if ((s = dev_alloc(c, co->ws_F, sizeof(double) * (size_t)N * n))) return s;
    if ((s = dev_alloc(c, co->ws_b, sizeof(double) * (size_t)N * n))) return s;
    if ((s = dev_alloc(c, co->ws_norm, sizeof(double) * (size_t)(3 * (N + 1) + 2)))) return s;
  }
  // (the batched solver allocates the buffers above for its handles, not these)
  if (!co->ws_flag.ptr) {
    if ((s = dev_alloc(c, co->ws_flag, 2 * sizeof(int)))) return s;
    if ((s = dev_alloc(c, co->ws_bh, sizeof(double) * (size_t)(N + 1) * (N + 1)))) return s;
    if ((s = dev_alloc(c, co->ws_argv, sizeof(SweepArgs) * (size_t)(N + 1)))) return s;
  }
  if (!co->h_stat) {
    cudaError_t eh = cudaMallocHost(&co->h_stat, 2 * 32);
    if (eh) return cuda_err(c, eh, "pinned status slots");
  }
  double* du = co->ws_norm.as<double>();
  double* unorm = du + (N + 1);
  double* bnd = unorm + (N + 1);
  double* summ = bnd + (N + 1);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  // inputs
  if ((s = to_device(c, co->ws_u.ptr, u0, sizeof(double) * n))) return s;
  DevView gv, cvv;
  if ((s = device_view(c, g, sizeof(double) * (size_t)Q * n, gv))) return s;
  const int sps = source_samples(co->op);
  if ((s = device_view(c, cv, sizeof(double) * (size_t)N * M * sps * Q, cvv))) return s;
  const int f32 = co->prec == LRP_PREC_MIXED;
  // b_i = F_i 0 for all intervals in one launch (Eq. F_n_affine)
  PropSrc src;
  src.Q = Q;
  src.g = (const double*)gv.p;
  src.c = (const double*)cvv.p;
  src.cstride = (long)M * sps * Q;
  int evals = 0;
  if (Q > 0) {
    PropIn zin;               // zero initial values
    zin.x = nullptr;
    PropOut bo;
    bo.y = co->ws_b.ptr;
    bo.ldy = n;
    cudaMemsetAsync(co->ws_b.ptr, 0, co->ws_b.bytes, c->stream);
    if ((s = propagate_any(c, op, co->dt, M, 0, N, 0, zin, bo, src))) return s;
    evals = 1;
  } else {
    cudaMemsetAsync(co->ws_b.ptr, 0, co->ws_b.bytes, c->stream);
  }
  const int rows = sweep_rows(c);
  if ((s = coarse_sweep_workspace(c, co, rows))) return s;
  SweepArgs a;
  a.N = N;
  a.n = n;
  a.R = Rm;
  a.u = co->ws_u.as<double>();
  a.U = f32 ? co->U32.ptr : co->U.ptr;
  a.S = f32 ? co->S32.ptr : co->S.ptr;
  a.V = f32 ? co->V32.ptr : co->V.ptr;
  a.K = co->Kc.as<double>();
  a.f32 = f32;
  a.rows = rows;
  a.nsl = (n + rows - 1) / rows;
  a.cw = co->ws_cw.as<double>();
  a.cnt = co->ws_cnt.as<unsigned>();
  a.delta = co->delta;
  a.eps = co->eps;
  a.du = du;
  a.unorm = unorm;
  a.summary = summ;
  // initial coarse sweep u^0_{i+1} = G_i u^0_i
  a.first = 0;
  a.initial = 1;
  a.F = co->ws_b.as<double>();
  a.bound = nullptr;
  SweepArgs* dargs = co->ws_args.as<SweepArgs>();
  if ((s = coarse_sweep(c, &a, dargs, 1))) return s;
  // Iterations are enqueued in batches without waiting for the stopping test:
  // the sweep of iteration k sets a device flag when the tolerance is met and
  // every later kernel of the solve then returns at once.  The host reads the
  // flag of batch j only after batch j + 1 is enqueued, so the GPU does not
  // idle between iterations.
  int* dflag = co->ws_flag.as<int>();        // [0] stop, [1] k_done
  cudaMemsetAsync(dflag, 0, 2 * sizeof(int), c->stream);
  struct HostStat { double sum[2]; int flag[2]; };
  HostStat* hst = static_cast<HostStat*>(co->h_stat);
  cudaEvent_t bev[2];
  cudaEventCreateWithFlags(&bev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&bev[1], cudaEventDisableTiming);
  int k = 0, converged = 0, k_run = 0, slot = 0, pending = 0;
  double hsum[2] = {0.0, 0.0};
  a.initial = 0;
  a.F = co->ws_F.as<double>();
  a.stop = dflag;
  a.k_done = dflag + 1;
  a.tol = tol;
  auto read_slot = [&](int sl) -> lrp_status {
    cudaError_t ee = cudaEventSynchronize(bev[sl]);
    if (ee) return cuda_err(c, ee, "parareal iteration");
    hsum[0] = hst[sl].sum[0];
    hsum[1] = hst[sl].sum[1];
    k_run = hst[sl].flag[1];
    if (hst[sl].flag[0]) converged = 1;
    return LRP_OK;
  };
  // the sweep arguments of every iteration, uploaded once
  std::vector<SweepArgs> hv((size_t)std::max(K, 1));
  for (int kk = 0; kk < K; ++kk) {
    hv[kk] = a;
    hv[kk].first = kk;
    hv[kk].iter = kk + 1;
    hv[kk].bound = co->ws_bh.as<double>() + (size_t)kk * (N + 1);
  }
  SweepArgs* dv = co->ws_argv.as<SweepArgs>();
  if (K > 0) {
    cudaError_t eu = cudaMemcpyAsync(dv, hv.data(), sizeof(SweepArgs) * K, cudaMemcpyHostToDevice,
                                     c->stream);
    if (eu) return cuda_err(c, eu, "sweep arguments");
  }
  // batches of 1, 2, then 4 iterations: a solve that converges after one or
  // two iterations runs few no-op launches, a long one keeps 4 in flight
  int batch = 1;
  while (k < K && !converged) {
    const int kb = std::min(K, k + batch);
    batch = std::min(4, 2 * batch);
    for (; k < kb; ++k) {
      const int first = k;          // F u^k_i for i < k equals the previous value
      PropIn in;
      in.x = co->ws_u.as<double>() + (size_t)first * n;
      in.x_f64 = 1;
      in.ldx = n;
      in.stop = dflag;
      in.interval0 = first;          // system s is interval first + s
      PropOut o;
      o.y = co->ws_F.as<double>() + (size_t)first * n;
      o.y_f64 = 1;
      o.ldy = n;
      PropSrc sk = src;
      if (Q > 0) sk.c = src.c + (size_t)first * M * sps * Q;
      if ((s = propagate_any(c, op, co->dt, M, 0, N - first, 0, in, o, sk))) return s;
      if ((s = coarse_sweep_ex(c, &hv[k], dv + k, 1, 0))) return s;
    }
    cudaMemcpyAsync(hst[slot].sum, summ, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(hst[slot].flag, dflag, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaEventRecord(bev[slot], c->stream);
    if (pending && (s = read_slot(slot ^ 1))) return s;
    pending = 1;
    slot ^= 1;
  }
  if (pending && (s = read_slot(slot ^ 1))) return s;
  cudaEventDestroy(bev[0]);
  cudaEventDestroy(bev[1]);
  k = k_run;
  evals += k;
  if (bound_out && k > 0)
    if ((s = from_device(c, bound_out, co->ws_bh.ptr, sizeof(double) * (size_t)k * (N + 1)))) return s;
  if ((s = from_device(c, u_out, co->ws_u.ptr, sizeof(double) * (size_t)(N + 1) * n))) return s;
  cudaEventRecord(e1, c->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e) return cuda_err(c, e, "parareal solve");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (k_done) *k_done = k;
  if (stats) {
    stats->k_done = k;
    stats->fine_evals = evals;
    stats->converged = converged;
    stats->final_bound = hsum[0];
    stats->scale = hsum[1];
    stats->device_ms = ms;
  }
  if (tol > 0 && !converged) return set_err(c, LRP_ENOTCONV, "tolerance not met within K_max");
  return LRP_OK;
}

lrp_status lrp_fine_solution(lrp_ctx* c, const lrp_operator* opc, double dt, int M, int N,
                             const double* u0, int Q, const double* g, const double* cv,
                             double* u_out) {
  if (!c || !opc || !u0 || !u_out || N < 1 || M < 1 || !(dt > 0) || Q < 0) return LRP_EINVAL;
  if (Q > 0 && (!g || !cv)) return LRP_EINVAL;
  cudaSetDevice(c->device);
  Operator* op = const_cast<lrp_operator*>(opc);
  const int n = op->n;
  DevBuf u;
  lrp_status s;
  if ((s = dev_alloc(c, u, sizeof(double) * (size_t)(N + 1) * n))) return s;
  if ((s = to_device(c, u.ptr, u0, sizeof(double) * n))) return s;
  DevView gv, cvv;
  if ((s = device_view(c, g, sizeof(double) * (size_t)Q * n, gv))) return s;
  const int sps = source_samples(op);
  if ((s = device_view(c, cv, sizeof(double) * (size_t)N * M * sps * Q, cvv))) return s;
  if ((op->kind == 2 || op->kind == 3) && (long)N * M > op->nJ)
    return set_err(c, LRP_EINVAL, "N * M exceeds the time grid of the operator");
  for (int i = 0; i < N; ++i) {
    PropIn in;
    in.x = u.as<double>() + (size_t)i * n;
    in.ldx = n;
    in.interval0 = i;
    PropOut o;
    o.y = u.as<double>() + (size_t)(i + 1) * n;
    o.ldy = n;
    PropSrc src;
    src.Q = Q;
    src.g = (const double*)gv.p;
    src.c = Q > 0 ? (const double*)cvv.p + (size_t)i * M * sps * Q : nullptr;
    src.cstride = (long)M * sps * Q;
    if ((s = propagate_any(c, op, dt, M, 0, 1, 0, in, o, src))) return s;
  }
  return from_device(c, u_out, u.ptr, sizeof(double) * (size_t)(N + 1) * n);
}


// ===========================================================================
// Classical Parareal: one backward-Euler step of size M*dt as the coarse
// solver (the comparison method of the paper's numerical experiments)
// ===========================================================================
// u^k_{i+1} = F_i u^{k-1}_i + G_i'(u^k_i - u^{k-1}_i); the increment is stored
// for the next interval's coarse step and for the norms.
__global__ static void k_cls_update(const double* __restrict__ F, const double* __restrict__ y,
                                    double* __restrict__ u_next, double* __restrict__ d_out, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double nv = y ? F[k] + y[k] : F[k];
  d_out[k] = nv - u_next[k];
  u_next[k] = nv;
}

// Per interval m = 0..N: ||u_m||^2 and ||u^k_m - u^{k-1}_m||^2 (the increment
// of m >= first + 1 is in D[m - 1]), one CTA per interval, fixed-order sums.
__global__ static void k_cls_norms(const double* __restrict__ u, const double* __restrict__ D, int n,
                                   int first, double* __restrict__ out) {
  __shared__ double red[2][8];
  const int m = blockIdx.x;
  const bool hasd = m >= first + 1;
  double su = 0.0, sd = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double v = u[(size_t)m * n + k];
    su += v * v;
    if (hasd) {
      const double d = D[(size_t)(m - 1) * n + k];
      sd += d * d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    su += __shfl_xor_sync(0xffffffffu, su, o);
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][w] = su; red[1][w] = sd; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[0][q]; b += red[1][q]; }
    out[2 * m] = sqrt(a);
    out[2 * m + 1] = sqrt(b);
  }
}

lrp_status lrp_operator_set_stepper(lrp_operator* opc, int stepper) {
  if (!opc || stepper < LRP_STEP_BACKWARD_EULER || stepper > LRP_STEP_SDIRK2_L) return LRP_EINVAL;
  Operator* op = opc;
  if ((op->kind == 2 || op->kind == 3) && stepper != op->stepper)
    return set_err(op->ctx, LRP_EINVAL,
                   "a time-dependent operator keeps the stepper its coefficient rows were sampled for");
  op->stepper = stepper;
  return LRP_OK;
}

lrp_status lrp_parareal_solve_classical(lrp_ctx* c, const lrp_operator* opc, double dt, int M, int N,
                                        const double* u0, int Q, const double* g, const double* cv,
                                        int K_max, double tol, double* u_out, double* incr_out,
                                        int* k_done, lrp_solve_stats* stats) {
  if (!c || !opc || !u0 || !u_out || N < 1 || M < 1 || !(dt > 0) || Q < 0 || K_max < 0)
    return LRP_EINVAL;
  if (Q > 0 && (!g || !cv)) return LRP_EINVAL;
  cudaSetDevice(c->device);
  Operator* op = const_cast<lrp_operator*>(opc);
  if (op->kind == 2 || op->kind == 3)
    return set_err(c, LRP_EINVAL, "the classical comparator takes time-invariant operators");
  if (Q > 0 && source_samples(op) != 1)
    return set_err(c, LRP_EINVAL, "the classical comparator takes sources with backward-Euler fine steps");
  const int n = op->n;
  const int K = std::min(K_max, N);
  const double DT = dt * M;
  DevBuf u, F, D, y, nrm;
  lrp_status s;
  if ((s = dev_alloc(c, u, sizeof(double) * (size_t)(N + 1) * n))) return s;
  if ((s = dev_alloc(c, F, sizeof(double) * (size_t)N * n))) return s;
  if ((s = dev_alloc(c, D, sizeof(double) * (size_t)N * n))) return s;
  if ((s = dev_alloc(c, y, sizeof(double) * (size_t)n))) return s;
  if ((s = dev_alloc(c, nrm, sizeof(double) * 2 * (size_t)(N + 1)))) return s;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  if ((s = to_device(c, u.ptr, u0, sizeof(double) * n))) return s;
  DevView gv, cvv;
  if ((s = device_view(c, g, sizeof(double) * (size_t)Q * n, gv))) return s;
  if ((s = device_view(c, cv, sizeof(double) * (size_t)N * M * Q, cvv))) return s;
  // initial coarse sweep u^0_{i+1} = G_i u^0_i: one step of size M*dt, the
  // source sampled at the interval's end t_{i+1}
  for (int i = 0; i < N; ++i) {
    PropIn in;
    in.x = u.as<double>() + (size_t)i * n;
    in.ldx = n;
    PropOut o;
    o.y = u.as<double>() + (size_t)(i + 1) * n;
    o.ldy = n;
    PropSrc src;
    src.Q = Q;
    src.g = (const double*)gv.p;
    src.c = Q > 0 ? (const double*)cvv.p + ((size_t)(i + 1) * M - 1) * Q : nullptr;
    src.cstride = Q;
    if ((s = propagate_any(c, op, DT, 1, 0, 1, 0, in, o, src))) return s;
  }
  PropSrc srcf;
  srcf.Q = Q;
  srcf.g = (const double*)gv.p;
  srcf.c = (const double*)cvv.p;
  srcf.cstride = (long)M * Q;
  int k = 0, converged = 0;
  double last_inc = 0.0;
  std::vector<double> hn(2 * (size_t)(N + 1));
  const unsigned nb = (unsigned)((n + 255) / 256);
  while (k < K) {
    const int first = k;
    PropIn in;
    in.x = u.as<double>() + (size_t)first * n;
    in.ldx = n;
    PropOut o;
    o.y = F.as<double>() + (size_t)first * n;
    o.ldy = n;
    PropSrc sk = srcf;
    if (Q > 0) sk.c = srcf.c + (size_t)first * M * Q;
    if ((s = propagate_any(c, op, dt, M, 0, N - first, 0, in, o, sk))) return s;
    // sequential correction; the increment at `first` is 0
    for (int i = first; i < N; ++i) {
      const double* yi = nullptr;
      if (i > first) {
        PropIn gin;
        gin.x = D.as<double>() + (size_t)(i - 1) * n;
        gin.ldx = n;
        PropOut go;
        go.y = y.ptr;
        go.ldy = n;
        PropSrc none;
        if ((s = propagate_any(c, op, DT, 1, 0, 1, 0, gin, go, none))) return s;
        yi = y.as<double>();
      }
      k_cls_update<<<nb, 256, 0, c->stream>>>(F.as<double>() + (size_t)i * n, yi,
                                              u.as<double>() + (size_t)(i + 1) * n,
                                              D.as<double>() + (size_t)i * n, n);
      c->launches += 1;
    }
    k_cls_norms<<<N + 1, 256, 0, c->stream>>>(u.as<double>(), D.as<double>(), n, first, nrm.as<double>());
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(hn.data(), nrm.ptr, sizeof(double) * hn.size(), cudaMemcpyDeviceToHost,
                                c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_err(c, e, "classical parareal iteration");
    ++k;
    double umax = 0.0, dmax = 0.0;
    for (int m = 0; m <= N; ++m) {
      umax = std::max(umax, hn[2 * m]);
      dmax = std::max(dmax, hn[2 * m + 1]);
    }
    last_inc = umax > 0.0 ? dmax / umax : dmax;
    if (incr_out) incr_out[k - 1] = last_inc;
    if (tol > 0 && last_inc <= tol) { converged = 1; break; }
  }
  if ((s = from_device(c, u_out, u.ptr, sizeof(double) * (size_t)(N + 1) * n))) return s;
  cudaEventRecord(e1, c->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e) return cuda_err(c, e, "classical parareal");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (k_done) *k_done = k;
  if (stats) {
    stats->k_done = k;
    stats->fine_evals = k;
    stats->converged = converged;
    stats->final_bound = last_inc;
    stats->scale = 1.0;
    stats->device_ms = ms;
  }
  if (tol > 0 && !converged) return set_err(c, LRP_ENOTCONV, "tolerance not met within K_max");
  return LRP_OK;
}

}  // extern "C"
