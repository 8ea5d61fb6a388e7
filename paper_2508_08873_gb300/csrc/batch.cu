// Many independent 2D problems of uneven grid sizes at once (the "batched
// uneven sizes" workload: independent advection-diffusion problems on grids
// drawn from a few sizes).
//
// lrp_build_coarse_batch runs the randomized SVD of every interval of every
// problem with each propagation stage as ONE persistent launch over a device
// work queue of (problem, system) items, largest grids first
// (k_krylov_queue), and the whole build -- forward sketch, orthonormalisation,
// adjoint sketch, orthonormalisation, small SVDs, ranks, lift -- captured into
// one CUDA graph and launched once; the host reads ranks, singular values and
// solver status once at the end.  lrp_parareal_solve_batch runs the Parareal
// iterations of all problems with the fine solves of all unconverged
// intervals of all problems in one queue launch per iteration and the coarse
// sweeps batched per grid size.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

using namespace lrp;

struct lrp_ctx : public Ctx {};
struct lrp_operator : public Operator {};
struct lrp_coarse : public Coarse {};

namespace lrp {

// ranks -> R_i and S (FP64 and FP32), one thread per interval
__global__ void k_finish_ranks(int N, int R, int ell, const int* __restrict__ rw,
                               const int* __restrict__ rv, const double* __restrict__ sv,
                               int* __restrict__ Ri, double* __restrict__ S, float* __restrict__ S32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int kk = min(rw[i], rv[i]);
  int r = min(R, kk);
  Ri[i] = r;
  const int Rm = max(R, 1);
  for (int j = 0; j < Rm; ++j) {
    double v = j < r ? sv[(size_t)i * ell + j] : 0.0;
    S[(size_t)i * Rm + j] = v;
    S32[(size_t)i * Rm + j] = (float)v;
  }
}

}  // namespace lrp

namespace {

struct BuildScratch {
  DevBuf Y, Z, Rw, Rz, rw, rv, sv, Psi, Phi, st, Rid;
  DevBuf ows, ost;    // tensor-core orthonormalisation workspace; status, counts of W, V^ intervals
};

}  // namespace

extern "C" {

lrp_status lrp_build_coarse_batch(lrp_ctx* c, int count, lrp_operator* const* ops, double dt,
                                  int M, int N, int rank, int oversample, uint64_t seed,
                                  lrp_precision prec, lrp_coarse** out) {
  if (!c || count < 1 || !ops || !out || !(dt > 0) || M < 1 || N < 1 || rank < 0 || oversample < 0)
    return LRP_EINVAL;
  const int ell = rank + oversample;
  if (ell < 1 || rank > 64 || ell > 128) return set_err(c, LRP_EINVAL, "bad rank / oversample");
  cudaSetDevice(c->device);
  const int f32 = prec == LRP_PREC_MIXED ? 1 : 0;
  const size_t es = f32 ? 4 : 8;
  for (int p = 0; p < count; ++p) {
    out[p] = nullptr;
    if (!ops[p] || ops[p]->kind != 1) return set_err(c, LRP_EINVAL, "batched builds take 5-point operators");
    if (ops[p]->stepper != 0)
      return set_err(c, LRP_EINVAL, "batched builds take backward-Euler fine steps");
    if (ell > ops[p]->n) return set_err(c, LRP_EINVAL, "rank + oversample exceeds a dimension");
  }
  lrp_status s;
  // ---- plans, handles and scratch (all allocations before the capture) -------
  std::vector<StencilPlan*> pf(count), pa(count);
  std::vector<std::unique_ptr<lrp_coarse>> co(count);
  std::vector<BuildScratch> sc(count);
  int maxn = 0, bicg = 0;
  for (int p = 0; p < count; ++p) {
    Operator* op = ops[p];
    if ((s = stencil_plan(c, op, dt, 0, &pf[p]))) return s;
    if ((s = stencil_plan(c, op, dt, 1, &pa[p]))) return s;
    maxn = std::max(maxn, op->n + 2 * op->mx);
    bicg |= op->symmetric ? 0 : 1;
    co[p] = std::make_unique<lrp_coarse>();
    Coarse* q = co[p].get();
    q->ctx = c;
    ctx_retain(c);
    q->op = op;
    q->dt = dt; q->M = M; q->N = N; q->R = rank; q->p = oversample; q->ell = ell;
    q->seed = seed; q->prec = prec;
    const size_t n = op->n, Rm = std::max(rank, 1);
    BuildScratch& b = sc[p];
    if ((s = dev_alloc(c, b.Y, (size_t)N * ell * n * es))) return s;
    if ((s = dev_alloc(c, b.Z, (size_t)N * ell * n * es))) return s;
    if ((s = dev_alloc(c, b.Rw, 8 * (size_t)N * ell * ell))) return s;
    if ((s = dev_alloc(c, b.Rz, 8 * (size_t)N * ell * ell))) return s;
    if ((s = dev_alloc(c, b.rw, 4 * (size_t)N))) return s;
    if ((s = dev_alloc(c, b.rv, 4 * (size_t)N))) return s;
    if ((s = dev_alloc(c, b.sv, 8 * (size_t)N * ell))) return s;
    if ((s = dev_alloc(c, b.Psi, 8 * (size_t)N * ell * ell))) return s;
    if ((s = dev_alloc(c, b.Phi, 8 * (size_t)N * ell * ell))) return s;
    if ((s = dev_alloc(c, b.st, 4))) return s;
    if ((s = dev_alloc(c, b.Rid, 4 * (size_t)N))) return s;
    if ((s = dev_alloc(c, b.ost, 3 * sizeof(int)))) return s;
    cudaMemsetAsync(b.ost.ptr, 0, 3 * sizeof(int), c->stream);
    if (orth_tc_applies(c, ell, !f32))
      if ((s = dev_alloc(c, b.ows, orth_tc_workspace(c, N, ell, (int)n)))) return s;
    if ((s = dev_alloc(c, q->U, 8 * N * Rm * n))) return s;
    if ((s = dev_alloc(c, q->V, 8 * N * Rm * n))) return s;
    if ((s = dev_alloc(c, q->S, 8 * N * Rm))) return s;
    if ((s = dev_alloc(c, q->U32, 4 * N * Rm * n))) return s;
    if ((s = dev_alloc(c, q->V32, 4 * N * Rm * n))) return s;
    if ((s = dev_alloc(c, q->S32, 4 * N * Rm))) return s;
  }
  // queue items: (problem, system), problems with larger grids first
  std::vector<int> order(count);
  for (int p = 0; p < count; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ops[a]->n > ops[b]->n; });
  const int nsys = N * ell;
  std::vector<int> items;
  items.reserve((size_t)2 * count * nsys);
  for (int p : order)
    for (int j = 0; j < nsys; ++j) { items.push_back(p); items.push_back(j); }
  const int nitems = (int)(items.size() / 2);
  // problem descriptors: forward (generated Omega -> Y), adjoint (W -> Z)
  DevBuf d_items, d_fwd, d_adj, d_cnt, d_stat, ws;
  if ((s = dev_alloc(c, d_items, sizeof(int) * items.size()))) return s;
  if ((s = dev_alloc(c, d_fwd, sizeof(KryArgs) * count))) return s;
  if ((s = dev_alloc(c, d_adj, sizeof(KryArgs) * count))) return s;
  if ((s = dev_alloc(c, d_cnt, 2 * sizeof(unsigned int)))) return s;
  if ((s = dev_alloc(c, d_stat, 16 * (size_t)count))) return s;   // per problem: iterations, status
  const int cs = c->p_queue_cluster > 0 ? c->p_queue_cluster : 4;
  const int nclu = krylov_queue_clusters(c, f32, cs);
  const size_t nvec = krylov_queue_nvec(bicg);
  const size_t ws_stride = ((nvec * maxn * es + 255) / 256) * 256;
  if ((s = dev_alloc(c, ws, ws_stride * nclu))) return s;
  std::vector<KryArgs> hf(count), ha(count);
  for (int p = 0; p < count; ++p) {
    Operator* op = ops[p];
    KryArgs a{};
    a.mx = op->mx; a.my = op->my; a.n = op->n; a.M = M; a.nsys = nsys;
    a.bicg = op->symmetric ? 0 : 1;
    a.dt = dt;
    a.rtol = f32 ? op->rtol32 : op->rtol64;
    a.max_iter = op->max_iter;
    a.nvec = (int)nvec;
    a.iters = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_stat.ptr) + 16 * p);
    a.status = reinterpret_cast<int*>(static_cast<char*>(d_stat.ptr) + 16 * p + 8);
    KryArgs b = a;
    a.B = stencil_B(pf[p], op, f32);
    a.Bs = stencil_Bs(pf[p], op, f32);
    a.in.gen = 1; a.in.seed = seed; a.in.ncol = ell; a.in.interval0 = 0;
    a.out.y = sc[p].Y.ptr; a.out.y_f64 = !f32; a.out.ldy = op->n;
    b.B = stencil_B(pa[p], op, f32);
    b.Bs = stencil_Bs(pa[p], op, f32);
    b.in.x = sc[p].Y.ptr; b.in.x_f64 = !f32; b.in.ldx = op->n;
    b.out.y = sc[p].Z.ptr; b.out.y_f64 = !f32; b.out.ldy = op->n;
    hf[p] = a;
    ha[p] = b;
  }
  cudaError_t e = cudaMemcpyAsync(d_items.ptr, items.data(), sizeof(int) * items.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemcpyAsync(d_fwd.ptr, hf.data(), sizeof(KryArgs) * count, cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemcpyAsync(d_adj.ptr, ha.data(), sizeof(KryArgs) * count, cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemsetAsync(d_stat.ptr, 0, d_stat.bytes, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "batch build setup");
  const double tau = f32 ? 2e-5 : 1e-13;
  // ---- the whole build as one captured CUDA graph ----------------------------
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e) return cuda_err(c, e, "begin capture");
  auto capture_body = [&]() -> lrp_status {
    lrp_status r;
    cudaMemsetAsync(d_cnt.ptr, 0, 2 * sizeof(unsigned int), c->stream);
    if ((r = krylov_queue_launch(c, f32, d_fwd.as<KryArgs>(), d_items.as<int>(), nitems,
                                 d_cnt.as<unsigned int>(), ws.ptr, ws_stride, cs, nclu)))
      return r;
    for (int p = 0; p < count; ++p)
      if ((r = orth_auto(c, N, ell, ops[p]->n, sc[p].Y.ptr, !f32, tau, sc[p].Rw.as<double>(),
                         sc[p].rw.as<int>(), sc[p].ows.ptr, sc[p].ows.bytes, sc[p].ost.as<int>(),
                         sc[p].ost.as<int>() + 1)))
        return r;
    if ((r = krylov_queue_launch(c, f32, d_adj.as<KryArgs>(), d_items.as<int>(), nitems,
                                 d_cnt.as<unsigned int>() + 1, ws.ptr, ws_stride, cs, nclu)))
      return r;
    for (int p = 0; p < count; ++p) {
      if ((r = orth_auto(c, N, ell, ops[p]->n, sc[p].Z.ptr, !f32, tau, sc[p].Rz.as<double>(),
                         sc[p].rv.as<int>(), sc[p].ows.ptr, sc[p].ows.bytes, sc[p].ost.as<int>(),
                         sc[p].ost.as<int>() + 2)))
        return r;
      cudaMemsetAsync(sc[p].st.ptr, 0, 4, c->stream);
      if ((r = small_svd(c, N, ell, sc[p].Rz.as<double>(), sc[p].rv.as<int>(), sc[p].sv.as<double>(),
                         sc[p].Psi.as<double>(), sc[p].Phi.as<double>(), sc[p].st.as<int>())))
        return r;
      Coarse* q = co[p].get();
      k_finish_ranks<<<(N + 127) / 128, 128, 0, c->stream>>>(
          N, rank, ell, sc[p].rw.as<int>(), sc[p].rv.as<int>(), sc[p].sv.as<double>(),
          sc[p].Rid.as<int>(), q->S.as<double>(), q->S32.as<float>());
      cudaMemsetAsync(q->U.ptr, 0, q->U.bytes, c->stream);
      cudaMemsetAsync(q->V.ptr, 0, q->V.bytes, c->stream);
      if (lift_tc_applies(c, ell, rank, !f32)) {
        if ((r = lift_tc(c, N, ell, rank, ops[p]->n, sc[p].Y.as<float>(), sc[p].Z.as<float>(),
                         sc[p].Psi.as<double>(), sc[p].Phi.as<double>(), sc[p].Rid.as<int>(),
                         q->U.as<double>(), q->V.as<double>(), q->U32.as<float>(),
                         q->V32.as<float>(), sc[p].ost.as<int>())))
          return r;
      } else if ((r = lift(c, N, ell, rank, ops[p]->n, sc[p].Y.ptr, sc[p].Z.ptr, !f32,
                           sc[p].Psi.as<double>(), sc[p].Phi.as<double>(), sc[p].Rid.as<int>(),
                           q->U.as<double>(), q->V.as<double>(), q->U32.as<float>(),
                           q->V32.as<float>()))) {
        return r;
      }
    }
    return LRP_OK;
  };
  lrp_status cap = capture_body();
  e = cudaStreamEndCapture(c->stream, &graph);
  if (cap) { if (graph) cudaGraphDestroy(graph); return cap; }
  if (e) return cuda_err(c, e, "end capture");
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (!e) e = cudaGraphLaunch(exec, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (e) return cuda_err(c, e, "batched build graph");
  // chain matrices of the coarse sweep (allocating, so outside the graph)
  for (int p = 0; p < count; ++p) {
    lrp_status r = coarse_chain(c, co[p].get());
    if (r) return r;
  }
  // ---- ranks, singular values, status ------------------------------------------
  std::vector<unsigned long long> hs(2 * (size_t)count, 0);
  e = cudaMemcpy(hs.data(), d_stat.ptr, 16 * (size_t)count, cudaMemcpyDeviceToHost);
  if (e) return cuda_err(c, e, "batch build status");
  for (int p = 0; p < count; ++p) {
    Coarse* q = co[p].get();
    q->rank_w.resize(N);
    q->rank_v.resize(N);
    q->sigma.resize((size_t)N * ell);
    q->Ri.resize(N);
    int svd_st = 0;
    int orth_st[3] = {0, 0, 0};
    e = cudaMemcpy(q->rank_w.data(), sc[p].rw.ptr, 4 * N, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(q->rank_v.data(), sc[p].rv.ptr, 4 * N, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(q->sigma.data(), sc[p].sv.ptr, 8 * (size_t)N * ell, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(q->Ri.data(), sc[p].Rid.ptr, 4 * N, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(&svd_st, sc[p].st.ptr, 4, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(orth_st, sc[p].ost.ptr, 3 * sizeof(int), cudaMemcpyDeviceToHost);
    if (e) return cuda_err(c, e, "batch build results");
    if (orth_st[0]) return set_err(c, LRP_EBREAKDOWN, "tensor-core orthonormalisation or lift failed");
    q->orth_tc_w = orth_st[1];
    q->orth_tc_v = orth_st[2];
    if (svd_st) return set_err(c, LRP_ENOTCONV, "Jacobi SVD did not converge");
    q->delta = q->eps = 0.0;
    for (int i = 0; i < N; ++i) {
      int kk = std::min(q->rank_w[i], q->rank_v[i]);
      for (int r = kk; r < ell; ++r) q->sigma[(size_t)i * ell + r] = 0.0;
      double s1 = kk > 0 ? q->sigma[(size_t)i * ell] : 0.0;
      double sn = kk > q->Ri[i] ? q->sigma[(size_t)i * ell + q->Ri[i]] : tau * s1;
      q->delta = std::max(q->delta, s1);
      q->eps = std::max(q->eps, sn);
    }
  }
  int bad = -1, kbad = 0;
  for (int p = 0; p < count; ++p) {
    ops[p]->krylov_iters += hs[2 * p];
    const int kst = (int)(hs[2 * p + 1] & 0xffffffffu);
    if (kst && (bad < 0 || (kst & 2) > (kbad & 2))) { bad = p; kbad = kst; }
  }
  for (int p = 0; p < count; ++p) out[p] = co[p].release();
  if (kbad & 2)
    return set_err(c, LRP_EBREAKDOWN, "Krylov breakdown in a batched build (problem " +
                                          std::to_string(bad) + ")");
  if (kbad & 1)
    return set_err(c, LRP_ENOTCONV, "Krylov iteration cap reached in a batched build (problem " +
                                        std::to_string(bad) + ")");
  return LRP_OK;
}

lrp_status lrp_parareal_solve_batch(lrp_ctx* c, int count, lrp_coarse* const* cos,
                                    const double* const* u0, int K_max, double tol,
                                    double* const* u_out, int* k_done) {
  if (!c || count < 1 || !cos || !u0 || !u_out || K_max < 0) return LRP_EINVAL;
  cudaSetDevice(c->device);
  const int N = cos[0]->N, M = cos[0]->M;
  int bicg = 0, maxn = 0;
  for (int p = 0; p < count; ++p) {
    if (!cos[p] || !u0[p] || !u_out[p] || cos[p]->N != N || cos[p]->M != M ||
        cos[p]->op->kind != 1 || cos[p]->R != cos[0]->R || cos[p]->prec != cos[0]->prec)
      return set_err(c, LRP_EINVAL, "batched solves need 2D coarse handles with equal N, M, R, precision");
    bicg |= cos[p]->op->symmetric ? 0 : 1;
    maxn = std::max(maxn, cos[p]->op->n + 2 * cos[p]->op->mx);
  }
  const int K = std::min(K_max, N);
  lrp_status s;
  cudaError_t e;
  std::vector<StencilPlan*> pf(count);
  for (int p = 0; p < count; ++p) {
    Coarse* q = cos[p];
    Operator* op = const_cast<Operator*>(q->op);
    const int n = op->n;
    if ((s = stencil_plan(c, op, q->dt, 0, &pf[p]))) return s;
    if (!q->ws_u.ptr) {
      if ((s = dev_alloc(c, q->ws_u, 8 * (size_t)(N + 1) * n))) return s;
      if ((s = dev_alloc(c, q->ws_F, 8 * (size_t)N * n))) return s;
      if ((s = dev_alloc(c, q->ws_b, 8 * (size_t)N * n))) return s;
      if ((s = dev_alloc(c, q->ws_norm, 8 * (size_t)(3 * (N + 1) + 2)))) return s;
    }
    if ((s = coarse_sweep_workspace(c, q, sweep_rows(c)))) return s;
    e = cudaMemcpyAsync(q->ws_u.ptr, u0[p], 8 * (size_t)n, cudaMemcpyDefault, c->stream);
    if (!e) e = cudaMemsetAsync(q->ws_b.ptr, 0, q->ws_b.bytes, c->stream);
    if (e) return cuda_err(c, e, "batch solve input");
  }
  const int cs = c->p_queue_cluster > 0 ? c->p_queue_cluster : 4;
  // FP64 fine steps by in-kernel iterative refinement (FP32 Krylov
  // corrections) unless krylov_refine = 2
  const int qprec = c->p_krylov_refine == 2 ? 0 : 2;
  const int nclu = krylov_queue_clusters(c, qprec, cs);
  const size_t nvec = krylov_queue_nvec(bicg);
  const size_t ws_one = qprec == 2 ? krylov_queue_ir_bytes(maxn) : nvec * maxn * 8;
  const size_t ws_stride = ((ws_one + 255) / 256) * 256;
  // Queue items interval-major, intervals N-1 down to 0 and within an
  // interval the problems largest grid first: iteration k (intervals >= k)
  // is the prefix of count (N - k) items.  Per problem: a stop flag and
  // k_done (set by its sweeps, read by its queue items), and the Krylov
  // iteration count and status.
  std::vector<int> order(count);
  for (int p = 0; p < count; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return cos[a]->op->n > cos[b]->op->n; });
  std::vector<int> items;
  items.reserve(2 * (size_t)count * N);
  for (int i = N - 1; i >= 0; --i)
    for (int p : order) { items.push_back(p); items.push_back(i); }
  DevBuf ws, d_items, d_probs, d_cnt, d_stat, d_flag, d_args;
  if ((s = dev_alloc(c, ws, ws_stride * nclu))) return s;
  if ((s = dev_alloc(c, d_items, sizeof(int) * items.size()))) return s;
  if ((s = dev_alloc(c, d_probs, sizeof(KryArgs) * count))) return s;
  if ((s = dev_alloc(c, d_cnt, sizeof(unsigned int) * (size_t)(K + 1)))) return s;
  if ((s = dev_alloc(c, d_stat, 16 * (size_t)count))) return s;
  if ((s = dev_alloc(c, d_flag, 2 * sizeof(int) * (size_t)count))) return s;
  if ((s = dev_alloc(c, d_args, sizeof(SweepArgs) * (size_t)count * (K + 1)))) return s;
  int* dflag = d_flag.as<int>();
  std::vector<KryArgs> hp(count);
  for (int p = 0; p < count; ++p) {
    Coarse* q = cos[p];
    Operator* op = const_cast<Operator*>(q->op);
    KryArgs a{};
    a.mx = op->mx; a.my = op->my; a.n = op->n; a.M = M; a.nsys = N;
    a.bicg = op->symmetric ? 0 : 1;
    a.dt = q->dt; a.rtol = op->rtol64; a.max_iter = op->max_iter; a.nvec = (int)nvec;
    a.B = stencil_B(pf[p], op, 0);
    a.Bs = stencil_Bs(pf[p], op, 0);
    a.B32 = stencil_B(pf[p], op, 1);
    a.Bs32 = stencil_Bs(pf[p], op, 1);
    a.rtol_in = c->p_krylov_refine_digits > 0 ? std::pow(10.0, -c->p_krylov_refine_digits) : 1e-3;
    a.in.x = q->ws_u.ptr; a.in.x_f64 = 1; a.in.ldx = op->n;
    a.in.stop = dflag + 2 * p;
    a.out.y = q->ws_F.ptr; a.out.y_f64 = 1; a.out.ldy = op->n;
    a.iters = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_stat.ptr) + 16 * p);
    a.status = reinterpret_cast<int*>(static_cast<char*>(d_stat.ptr) + 16 * p + 8);
    hp[p] = a;
  }
  // sweep arguments: the initial sweep, then iteration k = 0..K-1
  const int rows = sweep_rows(c);
  std::vector<SweepArgs> hv((size_t)count * (K + 1));
  for (int k = -1; k < K; ++k)
    for (int p = 0; p < count; ++p) {
      Coarse* q = cos[p];
      const int f32 = q->prec == LRP_PREC_MIXED;
      const bool initial = k < 0;
      SweepArgs a;
      a.N = N; a.n = q->op->n; a.R = std::max(q->R, 1);
      a.first = initial ? 0 : k;
      a.initial = initial;
      a.u = q->ws_u.as<double>();
      a.F = initial ? q->ws_b.as<double>() : q->ws_F.as<double>();
      a.U = f32 ? q->U32.ptr : q->U.ptr;
      a.S = f32 ? q->S32.ptr : q->S.ptr;
      a.V = f32 ? q->V32.ptr : q->V.ptr;
      a.K = q->Kc.as<double>();
      a.f32 = f32;
      a.delta = q->delta; a.eps = q->eps;
      double* nr = q->ws_norm.as<double>();
      a.du = nr; a.unorm = nr + (N + 1); a.bound = initial ? nullptr : nr + 2 * (N + 1);
      a.summary = nr + 3 * (N + 1);
      a.rows = rows;
      a.nsl = (a.n + rows - 1) / rows;
      a.cw = q->ws_cw.as<double>();
      a.cnt = q->ws_cnt.as<unsigned>();
      if (!initial) {
        a.stop = dflag + 2 * p;
        a.k_done = dflag + 2 * p + 1;
        a.iter = k + 1;
        a.tol = tol;
      }
      hv[(size_t)(k + 1) * count + p] = a;
    }
  e = cudaMemcpyAsync(d_items.ptr, items.data(), sizeof(int) * items.size(),
                      cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemcpyAsync(d_probs.ptr, hp.data(), sizeof(KryArgs) * count,
                              cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemcpyAsync(d_args.ptr, hv.data(), sizeof(SweepArgs) * hv.size(),
                              cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemsetAsync(d_cnt.ptr, 0, d_cnt.bytes, c->stream);
  if (!e) e = cudaMemsetAsync(d_stat.ptr, 0, d_stat.bytes, c->stream);
  if (!e) e = cudaMemsetAsync(d_flag.ptr, 0, d_flag.bytes, c->stream);
  if (e) return cuda_err(c, e, "batch solve setup");
  SweepArgs* dargs = d_args.as<SweepArgs>();
  if ((s = coarse_sweep_ex(c, hv.data(), dargs, count, 0))) return s;
  // Iterations enqueued in batches of 1, 2, then 4 without waiting for the
  // stopping test; the flags of batch j are read after batch j + 1 is queued.
  int* hflag = nullptr;
  e = cudaMallocHost(&hflag, 2 * 2 * sizeof(int) * (size_t)count);
  if (e) return cuda_err(c, e, "pinned flags");
  cudaEvent_t bev[2];
  cudaEventCreateWithFlags(&bev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&bev[1], cudaEventDisableTiming);
  auto all_stopped = [&](int sl) {
    for (int p = 0; p < count; ++p)
      if (!hflag[(size_t)sl * 2 * count + 2 * p]) return false;
    return true;
  };
  int k = 0, batch = 1, slot = 0, pending = 0;
  bool done = false;
  s = LRP_OK;
  while (k < K && !done) {
    const int kb = std::min(K, k + batch);
    batch = std::min(4, 2 * batch);
    for (; k < kb && !s; ++k) {
      if ((s = krylov_queue_launch(c, qprec, d_probs.as<KryArgs>(), d_items.as<int>(), count * (N - k),
                                   d_cnt.as<unsigned int>() + k, ws.ptr, ws_stride, cs, nclu)))
        break;
      s = coarse_sweep_ex(c, &hv[(size_t)(k + 1) * count], dargs + (size_t)(k + 1) * count, count, 0);
    }
    if (s) break;
    e = cudaMemcpyAsync(hflag + (size_t)slot * 2 * count, dflag, 2 * sizeof(int) * count,
                        cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaEventRecord(bev[slot], c->stream);
    if (e) { s = cuda_err(c, e, "batch solve flags"); break; }
    if (pending) {
      e = cudaEventSynchronize(bev[slot ^ 1]);
      if (e) { s = cuda_err(c, e, "batch solve iteration"); break; }
      done = tol > 0 && all_stopped(slot ^ 1);
    }
    pending = 1;
    slot ^= 1;
  }
  e = cudaStreamSynchronize(c->stream);
  if (!s && e) s = cuda_err(c, e, "batch solve");
  std::vector<int> fl(2 * (size_t)count, 0);
  std::vector<unsigned long long> hs(2 * (size_t)count, 0);
  if (!s) {
    e = cudaMemcpy(fl.data(), dflag, 2 * sizeof(int) * count, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(hs.data(), d_stat.ptr, 16 * (size_t)count, cudaMemcpyDeviceToHost);
    if (e) s = cuda_err(c, e, "batch solve status");
  }
  cudaEventDestroy(bev[0]);
  cudaEventDestroy(bev[1]);
  cudaFreeHost(hflag);
  if (s) return s;
  int bad = -1, kbad = 0;
  for (int p = 0; p < count; ++p) {
    e = cudaMemcpy(u_out[p], cos[p]->ws_u.ptr, 8 * (size_t)(N + 1) * cos[p]->op->n, cudaMemcpyDefault);
    if (e) return cuda_err(c, e, "batch solve output");
    if (k_done) k_done[p] = K > 0 ? fl[2 * p + 1] : 0;
    const_cast<Operator*>(cos[p]->op)->krylov_iters += hs[2 * p];
    const int kst = (int)(hs[2 * p + 1] & 0xffffffffu);
    if (kst && (bad < 0 || (kst & 2) > (kbad & 2))) { bad = p; kbad = kst; }
  }
  if (kbad & 2)
    return set_err(c, LRP_EBREAKDOWN, "Krylov breakdown in a batched solve (problem " +
                                          std::to_string(bad) + ")");
  if (kbad & 1)
    return set_err(c, LRP_ENOTCONV, "Krylov iteration cap reached in a batched solve (problem " +
                                        std::to_string(bad) + ")");
  return LRP_OK;
}

}  // extern "C"
