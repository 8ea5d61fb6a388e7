// Sequential coarse sweep fused with the Parareal correction, in the delta
// form of Remark rem:affine_g_n:
//   u^k_{i+1} = F_i u^{k-1}_i + G_i'(u^k_i - u^{k-1}_i),  G_i' = U_i diag(S_i) V_i^T,
// and, for the initial sweep, u^0_{i+1} = b_i + G_i' u^0_i (Eq. def_Parareal
// with u^{-1} := 0).  The iterate is updated in place; the norms
// ||u^k_m - u^{k-1}_m|| and ||u^k_m|| are recorded on the way and the a
// posteriori bound eps sum_{m<n} delta^{n-m-1} ||u^k_m - u^{k-1}_m||
// (Eq. apost_bound) is evaluated by its recurrence B_n = delta B_{n-1} +
// eps ||u^k_{n-1} - u^{k-1}_{n-1}|| at the end.
//
// The sweep is sequential over intervals but each step is two skinny products
// with n x R factors, so one problem runs on a thread-block cluster: every CTA
// owns a contiguous slice of the n rows, computes partial V_i^T delta for its
// slice, and the partial sums are exchanged through distributed shared memory
// with one cluster barrier per interval (double-buffered).  All CTAs add the
// partials in the same order, so the result does not depend on timing.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace lrp {

// 4- or 8-byte asynchronous global->shared copies (cp.async, completion
// tracked per thread with commit/wait groups).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int SWEEP_THREADS = 256;
constexpr int SWEEP_MAXR = 64;
constexpr int SWEEP_MAXCS = 16;
constexpr size_t SWEEP_STAGE_MAX = 192 * 1024;   // dynamic smem when staging factors
constexpr size_t SWEEP_SMEM_MAX = 200 * 1024;

template <typename TF>
__device__ __forceinline__ void sweep_body(const SweepArgs& a) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int cs = (int)cl.num_blocks();
  const int n = a.n, R = a.R, N = a.N;
  const int nv = R + 2;                                 // R dots, ||delta||^2, ||u||^2
  extern __shared__ double dsm[];                       // delta of this CTA's rows
  __shared__ double red[SWEEP_THREADS / 32][SWEEP_MAXR + 2];
  // partial sums of every CTA, pushed here by their owners before the barrier
  // (remote stores), so that no remote read sits on the critical path
  __shared__ double gath[2][SWEEP_MAXCS][SWEEP_MAXR + 2];
  __shared__ double coef[SWEEP_MAXR + 2];
  __shared__ TF scoef[SWEEP_MAXR];                      // S_r * c_r in the apply type
  __shared__ TF sS[2][SWEEP_MAXR];                      // staged S of the next interval
  __shared__ double* rgath[SWEEP_MAXCS];                // gath[][][] of every CTA (DSMEM)
  const int per = (n + cs - 1) / cs;
  const int lo = crank * per, hi = min(n, lo + per), rows = max(0, hi - lo);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const TF* U = static_cast<const TF*>(a.U);
  const TF* S = static_cast<const TF*>(a.S);
  const TF* V = static_cast<const TF*>(a.V);
  // Optional staging of the next interval's factor slices and F slice in
  // shared memory (double-buffered cp.async), so that their load latency
  // overlaps the current interval's reductions and cluster barrier.
  const bool stage = a.stage != 0;
  // delta in the apply type: a separate FP32 copy in the mixed mode (so the
  // R dot products need no conversions), the FP64 array itself otherwise
  constexpr bool kSep = sizeof(TF) != sizeof(double);
  TF* dsT = kSep ? reinterpret_cast<TF*>(dsm + per) : reinterpret_cast<TF*>(dsm);
  TF* sU = reinterpret_cast<TF*>(dsm + per) + (kSep ? per + (per & 1) : 0);   // [2][R][per]
  TF* sV = sU + (size_t)2 * R * per;                          // [2][R][per]
  double* sF = reinterpret_cast<double*>(sV + (size_t)2 * R * per);   // [2][per]
  double* sO = sF + (size_t)2 * per;                          // [2][per] u^{k-1}_{iv+1}
  auto issue = [&](int iv, int b) {
    if (!stage || iv >= N) return;
    const TF* Ug = U + (size_t)iv * R * n + lo;
    const TF* Vg = V + (size_t)iv * R * n + lo;
    const double* Fg = a.F + (size_t)iv * n + lo;
    for (int r = 0; r < R; ++r) {                 // no integer division per element
      TF* du = sU + ((size_t)b * R + r) * per;
      TF* dv = sV + ((size_t)b * R + r) * per;
      const TF* gu = Ug + (size_t)r * n;
      const TF* gv = Vg + (size_t)r * n;
      for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        cp_async<sizeof(TF)>(du + i, gu + i);
        cp_async<sizeof(TF)>(dv + i, gv + i);
      }
    }
    const double* Og = a.u + (size_t)(iv + 1) * n + lo;
    for (int r = threadIdx.x; r < R; r += blockDim.x) cp_async<sizeof(TF)>(&sS[b][r], S + (size_t)iv * R + r);
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      cp_async<8>(sF + (size_t)b * per + i, Fg + i);
      if (!a.initial) cp_async<8>(sO + (size_t)b * per + i, Og + i);
    }
  };
  issue(a.first, 0);
  cp_async_commit();
  // distributed-shared-memory addresses of every CTA's partial sums, mapped once
  for (int q = threadIdx.x; q < cs; q += blockDim.x) rgath[q] = cl.map_shared_rank(&gath[0][0][0], q);
  cl.sync();   // every CTA of the cluster runs before any remote store into its shared memory
  // delta at the first interval: 0 (u^k_first == u^{k-1}_first), or u0 initially
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    double d0 = a.initial ? a.u[(size_t)a.first * n + lo + i] : 0.0;
    dsm[i] = d0;
    if (kSep) dsT[i] = (TF)d0;
  }
  if (crank == 0 && threadIdx.x == 0 && !a.initial)
    for (int m = 0; m <= a.first; ++m) a.du[m] = 0.0;
  __syncthreads();
  int buf = 0;
  // ||u^k_first||^2 of this thread's rows; later intervals carry it from the update
  TF acc_u_next = TF(0);
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    TF v = (TF)a.u[(size_t)a.first * n + lo + i];
    acc_u_next += v * v;
  }
  for (int iv = a.first; iv <= N; ++iv) {
    const int sb = (iv - a.first) & 1;      // staging buffer of this interval
    issue(iv + 1, sb ^ 1);
    cp_async_commit();
    cp_async_wait<1>();                     // this interval's slices have landed
    __syncthreads();
    // ---- partial reductions over this CTA's rows ---------------------------
    // norms for the bound in the apply type (FP32 in the mixed mode: FP64
    // instructions issue at 1/64 of the FP32 rate on GB300)
    TF acc_d = TF(0), acc_u = acc_u_next;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      TF d = dsT[i];
      acc_d += d * d;
    }
    acc_d = warp_sum<TF>(acc_d);
    acc_u = warp_sum<TF>(acc_u);
    if (lane == 0) { red[w][R] = (double)acc_d; red[w][R + 1] = (double)acc_u; }
    if (iv < N) {
      // one warp per factor row r: (V_iv[r], delta) over this CTA's rows
      const TF* Vi = stage ? sV + (size_t)sb * R * per : V + (size_t)iv * R * n + lo;
      const size_t ldv = stage ? (size_t)per : (size_t)n;
      for (int r = w; r < R; r += nw) {
        const TF* vr = Vi + (size_t)r * ldv;
        TF pr = TF(0);
        for (int i = lane; i < rows; i += 32) pr += vr[i] * dsT[i];
        pr = warp_sum<TF>(pr);
        if (lane == 0) {                   // push this CTA's partial dot to every CTA
          const int o = (buf * SWEEP_MAXCS + crank) * (SWEEP_MAXR + 2) + r;
          for (int q = 0; q < cs; ++q) rgath[q][o] = (double)pr;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double s = 0.0;
      for (int k = 0; k < nw; ++k) s += red[k][R + threadIdx.x];
      const int o = (buf * SWEEP_MAXCS + crank) * (SWEEP_MAXR + 2) + R + threadIdx.x;
      for (int q = 0; q < cs; ++q) rgath[q][o] = s;
    }
    cl.sync();
    if (threadIdx.x < nv) {
      double s = 0.0;
      if (iv < N || threadIdx.x >= R)
        for (int q = 0; q < cs; ++q) s += gath[buf][q][threadIdx.x];    // same order in every CTA
      coef[threadIdx.x] = s;
      if (threadIdx.x < R && iv < N)
        scoef[threadIdx.x] = (stage ? sS[sb][threadIdx.x] : S[(size_t)iv * R + threadIdx.x]) * (TF)s;
    }
    __syncthreads();
    if (crank == 0 && threadIdx.x == 0) {
      if (iv > a.first || a.initial) a.du[iv] = sqrt(coef[R]);
      a.unorm[iv] = sqrt(coef[R + 1]);
    }
    if (iv == N) break;
    // ---- u^k_{iv+1} = F_iv + U_iv (S_iv * c) on this CTA's rows ------------
    const TF* Ui = stage ? sU + (size_t)sb * R * per : U + (size_t)iv * R * n + lo;
    const size_t ldu = stage ? (size_t)per : (size_t)n;
    const double* Fi = stage ? sF + (size_t)sb * per : a.F + (size_t)iv * n + lo;
    double* un = a.u + (size_t)(iv + 1) * n + lo;
    acc_u_next = TF(0);
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      TF g = TF(0);
      for (int r = 0; r < R; ++r) g += Ui[(size_t)r * ldu + i] * scoef[r];
      double nv_ = Fi[i] + (double)g;
      double old = a.initial ? 0.0 : (stage ? sO[(size_t)sb * per + i] : un[i]);
      const double dn = nv_ - old;
      dsm[i] = dn;
      if (kSep) dsT[i] = (TF)dn;
      un[i] = nv_;
      const TF nt = (TF)nv_;
      acc_u_next += nt * nt;
    }
    buf ^= 1;
    __syncthreads();
  }
  // ---- bound recurrence and summary (one thread) ------------------------------
  if (crank == 0 && threadIdx.x == 0) {
    double B = 0.0, bmax = 0.0, umax = 0.0;
    for (int m = 0; m <= N; ++m) umax = fmax(umax, a.unorm[m]);
    if (a.bound) {
      a.bound[0] = 0.0;
      for (int m = 1; m <= N; ++m) {
        B = a.delta * B + a.eps * a.du[m - 1];
        a.bound[m] = B;
        bmax = fmax(bmax, B);
      }
    }
    a.summary[0] = bmax;
    a.summary[1] = umax;
  }
  cp_async_wait<0>();
  cl.sync();  // no CTA leaves while its shared memory may still be read
}

// One problem per launch.
template <typename TF>
__global__ void __launch_bounds__(SWEEP_THREADS) k_sweep(SweepArgs a) {
  sweep_body<TF>(a);
}

// A batch of problems (same n, R, staging), one cluster each: args[cluster].
template <typename TF>
__global__ void __launch_bounds__(SWEEP_THREADS) k_sweep_batch(const SweepArgs* __restrict__ args) {
  const SweepArgs a = args[blockIdx.x / cg::this_cluster().num_blocks()];
  sweep_body<TF>(a);
}

lrp_status coarse_sweep(Ctx* c, const SweepArgs& a) {
  if (a.R > SWEEP_MAXR) return set_err(c, LRP_EINVAL, "rank above 64 is not supported by the sweep");
  if ((size_t)((a.n + SWEEP_MAXCS - 1) / SWEEP_MAXCS) * (a.f32 ? 12 : 8) > SWEEP_SMEM_MAX)
    return set_err(c, LRP_EINVAL, "state dimension too large for the coarse sweep");
  int cs = 16;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  auto kern = a.f32 ? (void (*)(SweepArgs))k_sweep<float> : (void (*)(SweepArgs))k_sweep<double>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e) { cudaGetLastError(); cs = 8; }
  // small problems: fewer CTAs per cluster
  while (cs > 1 && (a.n + cs - 1) / cs < 64) cs >>= 1;
  if (c->p_sweep_cluster > 0) cs = c->p_sweep_cluster;
  while (cs < SWEEP_MAXCS && (size_t)((a.n + cs - 1) / cs) * (a.f32 ? 12 : 8) > SWEEP_SMEM_MAX) cs <<= 1;
  const size_t tf = a.f32 ? 4 : 8;
  auto dyn_for = [&](int csz, int stage) {
    size_t per = (size_t)((a.n + csz - 1) / csz);
    size_t b = sizeof(double) * per + (tf == 8 ? 0 : tf * (per + (per & 1)));
    if (stage) b += 4 * (size_t)a.R * per * tf + 4 * per * sizeof(double);
    return b;
  };
  SweepArgs aa = a;
  aa.stage = dyn_for(cs, 1) <= SWEEP_STAGE_MAX ? 1 : 0;
  size_t dyn = dyn_for(cs, aa.stage);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM_MAX);
  if (e) return cuda_err(c, e, "sweep smem attribute");
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(SWEEP_THREADS);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = c->stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaEvent_t ev = nullptr;
  timer_begin(c, "sweep", &ev);
  e = cudaLaunchKernelEx(&cfg, kern, aa);
  timer_end(c, "sweep", ev);
  if (e == cudaErrorInvalidValue || e == cudaErrorInvalidConfiguration) {
    // retry with a portable cluster size
    cudaGetLastError();
    cs = std::min(cs, 8);
    cfg.gridDim = dim3(cs);
    aa.stage = dyn_for(cs, 1) <= SWEEP_STAGE_MAX ? 1 : 0;
    cfg.dynamicSmemBytes = dyn_for(cs, aa.stage);
    attr[0].val.clusterDim.x = cs;
    e = cudaLaunchKernelEx(&cfg, kern, aa);
  }
  if (e) return cuda_err(c, e, "k_sweep launch");
  return LRP_OK;
}

lrp_status coarse_sweep_batch(Ctx* c, const SweepArgs& proto, SweepArgs* d_args, int nprob,
                              int* cs_out) {
  if (nprob <= 0) return LRP_OK;
  if (proto.R > SWEEP_MAXR) return set_err(c, LRP_EINVAL, "rank above 64 is not supported by the sweep");
  auto kern = proto.f32 ? (void (*)(const SweepArgs*))k_sweep_batch<float>
                        : (void (*)(const SweepArgs*))k_sweep_batch<double>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  int cs = e ? 8 : 16;
  if (e) cudaGetLastError();
  // several problems share the GPU: fewer CTAs per problem when many run
  while (cs > 1 && (size_t)nprob * cs > (size_t)c->num_sms) cs >>= 1;
  while (cs > 1 && (proto.n + cs - 1) / cs < 64) cs >>= 1;
  if (c->p_sweep_cluster > 0) cs = c->p_sweep_cluster;
  const size_t tf = proto.f32 ? 4 : 8;
  while (cs < SWEEP_MAXCS && (size_t)((proto.n + cs - 1) / cs) * (proto.f32 ? 12 : 8) > SWEEP_SMEM_MAX)
    cs <<= 1;
  const size_t per = (size_t)((proto.n + cs - 1) / cs);
  size_t dyn = sizeof(double) * per + (tf == 8 ? 0 : tf * (per + (per & 1)));
  const size_t dyn_stage = dyn + 4 * (size_t)proto.R * per * tf + 4 * per * sizeof(double);
  const int stage = dyn_stage <= SWEEP_STAGE_MAX ? 1 : 0;
  if (stage) dyn = dyn_stage;
  if (stage != proto.stage) return set_err(c, LRP_EINVAL, "sweep batch staging mismatch");
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM_MAX);
  if (e) return cuda_err(c, e, "sweep smem attribute");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(nprob * cs);
  cfg.blockDim = dim3(SWEEP_THREADS);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = c->stream;
  if (cs_out) *cs_out = cs;
  cudaEvent_t ev = nullptr;
  timer_begin(c, "sweep", &ev);
  e = cudaLaunchKernelEx(&cfg, kern, (const SweepArgs*)d_args);
  timer_end(c, "sweep", ev);
  if (e) return cuda_err(c, e, "k_sweep_batch launch");
  return LRP_OK;
}

// Staging decision of a batched sweep (the caller stores it in every
// problem's SweepArgs before copying them to the device).
int coarse_sweep_batch_stage(Ctx* c, const SweepArgs& proto, int nprob) {
  int cs = 16;
  while (cs > 1 && (size_t)nprob * cs > (size_t)c->num_sms) cs >>= 1;
  while (cs > 1 && (proto.n + cs - 1) / cs < 64) cs >>= 1;
  if (c->p_sweep_cluster > 0) cs = c->p_sweep_cluster;
  const size_t tf = proto.f32 ? 4 : 8;
  while (cs < SWEEP_MAXCS && (size_t)((proto.n + cs - 1) / cs) * (proto.f32 ? 12 : 8) > SWEEP_SMEM_MAX)
    cs <<= 1;
  const size_t per = (size_t)((proto.n + cs - 1) / cs);
  size_t dyn = sizeof(double) * per + (tf == 8 ? 0 : tf * (per + (per & 1)));
  return dyn + 4 * (size_t)proto.R * per * tf + 4 * per * sizeof(double) <= SWEEP_STAGE_MAX ? 1 : 0;
}

}  // namespace lrp
