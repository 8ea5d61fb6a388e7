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
#include <map>
#include <memory>
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
  if ((s = dev_alloc(c, d_stat, 16))) return s;
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
    a.iters = reinterpret_cast<unsigned long long*>(d_stat.ptr);
    a.status = reinterpret_cast<int*>(static_cast<char*>(d_stat.ptr) + 8);
    KryArgs b = a;
    a.B = stencil_B(pf[p], op, f32);
    a.in.gen = 1; a.in.seed = seed; a.in.ncol = ell; a.in.interval0 = 0;
    a.out.y = sc[p].Y.ptr; a.out.y_f64 = !f32; a.out.ldy = op->n;
    b.B = stencil_B(pa[p], op, f32);
    b.in.x = sc[p].Y.ptr; b.in.x_f64 = !f32; b.in.ldx = op->n;
    b.out.y = sc[p].Z.ptr; b.out.y_f64 = !f32; b.out.ldy = op->n;
    hf[p] = a;
    ha[p] = b;
  }
  cudaError_t e = cudaMemcpyAsync(d_items.ptr, items.data(), sizeof(int) * items.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemcpyAsync(d_fwd.ptr, hf.data(), sizeof(KryArgs) * count, cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemcpyAsync(d_adj.ptr, ha.data(), sizeof(KryArgs) * count, cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemsetAsync(d_stat.ptr, 0, 16, c->stream);
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
  unsigned long long hs[2] = {0, 0};
  cudaMemcpy(hs, d_stat.ptr, 16, cudaMemcpyDeviceToHost);
  for (int p = 0; p < count; ++p) {
    Coarse* q = co[p].get();
    q->rank_w.resize(N);
    q->rank_v.resize(N);
    q->sigma.resize((size_t)N * ell);
    q->Ri.resize(N);
    int svd_st = 0;
    cudaMemcpy(q->rank_w.data(), sc[p].rw.ptr, 4 * N, cudaMemcpyDeviceToHost);
    cudaMemcpy(q->rank_v.data(), sc[p].rv.ptr, 4 * N, cudaMemcpyDeviceToHost);
    cudaMemcpy(q->sigma.data(), sc[p].sv.ptr, 8 * (size_t)N * ell, cudaMemcpyDeviceToHost);
    cudaMemcpy(q->Ri.data(), sc[p].Rid.ptr, 4 * N, cudaMemcpyDeviceToHost);
    int orth_st[3] = {0, 0, 0};
    cudaMemcpy(&svd_st, sc[p].st.ptr, 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(orth_st, sc[p].ost.ptr, 3 * sizeof(int), cudaMemcpyDeviceToHost);
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
  for (int p = 0; p < count; ++p) ops[p]->krylov_iters += hs[0] / count;
  const int kst = (int)(hs[1] & 0xffffffffu);
  for (int p = 0; p < count; ++p) out[p] = co[p].release();
  if (kst & 2) return set_err(c, LRP_EBREAKDOWN, "Krylov breakdown in a batched build");
  if (kst & 1) return set_err(c, LRP_ENOTCONV, "Krylov iteration cap reached in a batched build");
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
    cudaMemcpyAsync(q->ws_u.ptr, u0[p], 8 * (size_t)n, cudaMemcpyDefault, c->stream);
    cudaMemsetAsync(q->ws_b.ptr, 0, q->ws_b.bytes, c->stream);
  }
  const int cs = c->p_queue_cluster > 0 ? c->p_queue_cluster : 4;
  const int nclu = krylov_queue_clusters(c, 0, cs);
  const size_t nvec = krylov_queue_nvec(bicg);
  const size_t ws_stride = ((nvec * maxn * 8 + 255) / 256) * 256;
  DevBuf ws, d_items, d_probs, d_cnt, d_stat;
  if ((s = dev_alloc(c, ws, ws_stride * nclu))) return s;
  if ((s = dev_alloc(c, d_items, sizeof(int) * 2 * (size_t)count * N))) return s;
  if ((s = dev_alloc(c, d_probs, sizeof(KryArgs) * count))) return s;
  if ((s = dev_alloc(c, d_cnt, sizeof(unsigned int)))) return s;
  if ((s = dev_alloc(c, d_stat, 16))) return s;
  cudaMemsetAsync(d_stat.ptr, 0, 16, c->stream);
  std::vector<KryArgs> hp(count);
  for (int p = 0; p < count; ++p) {
    Coarse* q = cos[p];
    Operator* op = const_cast<Operator*>(q->op);
    KryArgs a{};
    a.mx = op->mx; a.my = op->my; a.n = op->n; a.M = M; a.nsys = N;
    a.bicg = op->symmetric ? 0 : 1;
    a.dt = q->dt; a.rtol = op->rtol64; a.max_iter = op->max_iter; a.nvec = (int)nvec;
    a.B = stencil_B(pf[p], op, 0);
    a.in.x = q->ws_u.ptr; a.in.x_f64 = 1; a.in.ldx = op->n;
    a.out.y = q->ws_F.ptr; a.out.y_f64 = 1; a.out.ldy = op->n;
    a.iters = reinterpret_cast<unsigned long long*>(d_stat.ptr);
    a.status = reinterpret_cast<int*>(static_cast<char*>(d_stat.ptr) + 8);
    hp[p] = a;
  }
  cudaError_t e = cudaMemcpyAsync(d_probs.ptr, hp.data(), sizeof(KryArgs) * count,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e) return cuda_err(c, e, "batch solve setup");
  // all problems' sweeps in one pair of launches (equal N and precision)
  DevBuf d_args;
  if ((s = dev_alloc(c, d_args, sizeof(SweepArgs) * count))) return s;
  std::vector<int> kk(count, 0), active(count, 1);
  std::vector<double> summ(2);
  const int rows = sweep_rows(c);
  std::vector<SweepArgs> h;
  auto sweeps = [&](int initial) -> lrp_status {
    h.clear();
    for (int p = 0; p < count; ++p) {
      if (!initial && !active[p]) continue;
      Coarse* q = cos[p];
      const int f32 = q->prec == LRP_PREC_MIXED;
      SweepArgs a;
      a.N = N; a.n = q->op->n; a.R = std::max(q->R, 1);
      a.first = initial ? 0 : kk[p];
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
      h.push_back(a);
    }
    if (h.empty()) return LRP_OK;
    lrp_status r = coarse_sweep(c, h.data(), d_args.as<SweepArgs>(), (int)h.size());
    cudaStreamSynchronize(c->stream);      // host args outlive their upload
    return r;
  };
  if ((s = sweeps(1))) return s;
  int it = 0;
  while (it < K) {
    std::vector<int> items;
    for (int p = 0; p < count; ++p)
      if (active[p])
        for (int i = kk[p]; i < N; ++i) { items.push_back(p); items.push_back(i); }
    if (items.empty()) break;
    e = cudaMemcpyAsync(d_items.ptr, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice,
                        c->stream);
    if (!e) e = cudaMemsetAsync(d_cnt.ptr, 0, sizeof(unsigned int), c->stream);
    if (e) return cuda_err(c, e, "items");
    if ((s = krylov_queue_launch(c, 0, d_probs.as<KryArgs>(), d_items.as<int>(), (int)items.size() / 2,
                                 d_cnt.as<unsigned int>(), ws.ptr, ws_stride, cs, nclu)))
      return s;
    cudaStreamSynchronize(c->stream);
    if ((s = sweeps(0))) return s;
    ++it;
    for (int p = 0; p < count; ++p) {
      if (!active[p]) continue;
      kk[p] += 1;
      cudaMemcpy(summ.data(), cos[p]->ws_norm.as<double>() + 3 * (N + 1), 16, cudaMemcpyDeviceToHost);
      bool conv = tol > 0 && summ[0] <= tol * summ[1];
      if (conv || kk[p] >= K) active[p] = 0;
    }
  }
  for (int p = 0; p < count; ++p) {
    e = cudaMemcpy(u_out[p], cos[p]->ws_u.ptr, 8 * (size_t)(N + 1) * cos[p]->op->n, cudaMemcpyDefault);
    if (e) return cuda_err(c, e, "batch solve output");
    if (k_done) k_done[p] = kk[p];
  }
  unsigned long long hs[2] = {0, 0};
  cudaMemcpy(hs, d_stat.ptr, 16, cudaMemcpyDeviceToHost);
  const int kst = (int)(hs[1] & 0xffffffffu);
  if (kst & 2) return set_err(c, LRP_EBREAKDOWN, "Krylov breakdown in a batched solve");
  if (kst & 1) return set_err(c, LRP_ENOTCONV, "Krylov iteration cap reached in a batched solve");
  return LRP_OK;
}

}  // extern "C"
