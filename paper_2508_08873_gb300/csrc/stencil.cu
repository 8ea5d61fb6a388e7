// Batched backward-Euler propagator for 5-point stencil operators (2D): every
// implicit-Euler step (I + dt A) x_{j+1} = x_j + dt f(t_{j+1}) is solved by a
// Jacobi-preconditioned Krylov method warm-started from x_j -- conjugate
// gradients when A is symmetric, BiCGStab otherwise -- to the relative
// residual ||d - B x|| <= rtol ||d|| (d the step's right-hand side), with an
// iteration cap per step that raises a status instead of looping on.
//
// One system (one vector of one interval) runs on one thread-block cluster:
// the CTAs of the cluster own contiguous blocks of grid rows, the vectors live
// in a per-cluster workspace in global memory (L2-resident at these sizes) and
// every dot product is reduced across the cluster through distributed shared
// memory with the partial sums added in a fixed order, so the iteration count
// and the result of a system do not depend on which other systems share the
// launch.  Clusters loop over systems (persistent launch).  The adjoint
// propagation uses the transposed stencil, (B^T)_{p,q} = B_{q,p}.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace lrp {

constexpr int KRY_THREADS = 512;
constexpr int KRY_MAXCS = 16;
constexpr int KRY_MAXNV = 4;

// B = I + dt*A (adjoint: its transpose) with the couplings that leave the
// grid removed; dinv = 1 / diag.
__global__ void k_stencil_plan(int mx, int my, double dt, int adj, const double* __restrict__ C,
                               const double* __restrict__ W, const double* __restrict__ E,
                               const double* __restrict__ S, const double* __restrict__ N,
                               double* __restrict__ b64, float* __restrict__ b32) {
  const int n = mx * my;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int ix = p % mx, iy = p / mx;
  double c = 1.0 + dt * C[p], w, e, s, nn;
  if (!adj) {
    w = ix > 0 ? dt * W[p] : 0.0;
    e = ix < mx - 1 ? dt * E[p] : 0.0;
    s = iy > 0 ? dt * S[p] : 0.0;
    nn = iy < my - 1 ? dt * N[p] : 0.0;
  } else {
    w = ix > 0 ? dt * E[p - 1] : 0.0;
    e = ix < mx - 1 ? dt * W[p + 1] : 0.0;
    s = iy > 0 ? dt * N[p - mx] : 0.0;
    nn = iy < my - 1 ? dt * S[p + mx] : 0.0;
  }
  double v[6] = {c, w, e, s, nn, 1.0 / c};
  for (int k = 0; k < 6; ++k) {
    b64[(size_t)k * n + p] = v[k];
    b32[(size_t)k * n + p] = (float)v[k];
  }
}



struct ClRed {
  double part[2][KRY_MAXNV];
  double red[KRY_THREADS / 32][KRY_MAXNV];
  double gath[KRY_MAXCS][KRY_MAXNV];
  const double* rpart[KRY_MAXCS];   // part[][] of every CTA of the cluster (DSMEM), mapped once
};

// Map the partial-sum arrays of all CTAs of the cluster once per kernel.
__device__ __forceinline__ void cl_map(cg::cluster_group& cl, ClRed& sh) {
  for (int q = threadIdx.x; q < (int)cl.num_blocks(); q += blockDim.x)
    sh.rpart[q] = cl.map_shared_rank(&sh.part[0][0], q);
  __syncthreads();
}

// Cluster-wide sum of nv values (deterministic order); also a cluster barrier.
template <int NV>
__device__ __forceinline__ void cl_sum(cg::cluster_group& cl, double (&v)[NV], ClRed& sh, int& buf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh.red[w][i] = v[i];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sh.red[k][threadIdx.x];
    sh.part[buf][threadIdx.x] = s;
  }
  cl.sync();
  const int cs = (int)cl.num_blocks();
  for (int k = threadIdx.x; k < cs * NV; k += blockDim.x)
    sh.gath[k / NV][k % NV] = sh.rpart[k / NV][buf * KRY_MAXNV + k % NV];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (int q = 0; q < cs; ++q) s += sh.gath[q][i];
    v[i] = s;
  }
  buf ^= 1;
}

template <typename T>
__device__ __forceinline__ T stencil_apply(const T* __restrict__ B, int n, int mx, int k,
                                           const T* __restrict__ v) {
  int ix = k % mx;
  T acc = B[k] * v[k];
  if (ix > 0) acc += B[(size_t)n + k] * v[k - 1];
  if (ix < mx - 1) acc += B[(size_t)2 * n + k] * v[k + 1];
  if (k >= mx) acc += B[(size_t)3 * n + k] * v[k - mx];
  if (k + mx < n) acc += B[(size_t)4 * n + k] * v[k + mx];
  return acc;
}

// One system (vector `sys` of the problem described by `a`) on this cluster,
// using the workspace `ws` (a.nvec vectors of a.n values).
template <typename T>
__device__ __forceinline__ void krylov_system(const KryArgs& a, cg::cluster_group& cl, ClRed& sh,
                                              int& buf, int sys, T* ws,
                                              unsigned long long& my_iters, int& my_status) {
  const int cs = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int n = a.n, mx = a.mx;
  const int rows_per = (a.my + cs - 1) / cs;
  const int k0 = min(a.n, crank * rows_per * mx), k1 = min(a.n, (crank + 1) * rows_per * mx);
  const T* B = static_cast<const T*>(a.B);
  const T* Bd = B + (size_t)5 * n;                         // 1 / diag
  T* x = ws;
  T* r = ws + (size_t)n;
  T* p = ws + (size_t)2 * n;          // CG: p; BiCG: p
  T* q = ws + (size_t)3 * n;          // CG: q = B p; BiCG: v
  T* rh = ws + (size_t)4 * n;         // BiCG: r-hat
  T* ph = ws + (size_t)5 * n;         // BiCG: D^-1 p
  T* sv = ws + (size_t)6 * n;         // BiCG: s
  T* shh = ws + (size_t)7 * n;        // BiCG: D^-1 s
  T* tv = ws + (size_t)8 * n;         // BiCG: t = B D^-1 s
  const T dt = (T)a.dt;
    // ---- initial vector ----------------------------------------------------
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      T v = T(0);
      if (a.in.gen)
        v = gauss<T>(a.in.seed, 0u, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                     (uint32_t)(sys % a.in.ncol), (uint32_t)k);
      else if (a.in.x == nullptr)
        v = T(0);
      else if (a.in.x_f64)
        v = (T) static_cast<const double*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + k];
      else
        v = (T) static_cast<const float*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + k];
      x[k] = v;
    }
    cl.sync();
    const double* csys = a.src.Q > 0
        ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
    const double* gsys = (a.src.Q > 0 && a.src.map)
        ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
    for (int j = 0; j < a.M; ++j) {
      // ---- right-hand side d = x + dt f, residual r = d - B x --------------
      T red3t[3] = {T(0), T(0), T(0)};    // d.d, r.r, rho (per-thread partials in T)
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        T d = x[k];
        if (csys)
          for (int qq = 0; qq < a.src.Q; ++qq)
            d += dt * (T)csys[(size_t)j * a.src.Q + qq] * (T)gsys[(size_t)qq * n + k];
        T rk = d - stencil_apply(B, n, mx, k, x);
        r[k] = rk;
        red3t[0] += d * d;
        red3t[1] += rk * rk;
        if (a.bicg) {
          rh[k] = rk;
          p[k] = rk;
          red3t[2] += rk * rk;
        } else {
          T z = rk * Bd[k];
          p[k] = z;
          red3t[2] += rk * z;
        }
      }
      double red3[3] = {(double)red3t[0], (double)red3t[1], (double)red3t[2]};
      cl_sum<3>(cl, red3, sh, buf);
      const double tol2 = a.rtol * a.rtol * red3[0];
      double rr = red3[1], rho = red3[2];
      int it = 0;
      if (!a.bicg) {
        // ---- preconditioned conjugate gradients ----------------------------
        while (rr > tol2 && it < a.max_iter) {
          T pqt = T(0);
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            T qk = stencil_apply(B, n, mx, k, p);
            q[k] = qk;
            pqt += p[k] * qk;
          }
          double pq[1] = {(double)pqt};
          cl_sum<1>(cl, pq, sh, buf);
          if (!(pq[0] > 0.0)) { my_status |= 2; break; }
          const T alpha = (T)(rho / pq[0]);
          T rz0 = T(0), rz1 = T(0);
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            x[k] += alpha * p[k];
            T rk = r[k] - alpha * q[k];
            r[k] = rk;
            rz0 += rk * (rk * Bd[k]);
            rz1 += rk * rk;
          }
          double rz[2] = {(double)rz0, (double)rz1};
          cl_sum<2>(cl, rz, sh, buf);
          const T beta = (T)(rz[0] / rho);
          rho = rz[0];
          rr = rz[1];
          ++it;
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) p[k] = r[k] * Bd[k] + beta * p[k];
          cl.sync();
        }
      } else {
        // ---- BiCGStab with Jacobi right preconditioning ---------------------
        double rho_prev = rho;
        T alpha = T(1), omega = T(1);
        bool first = true;
        while (rr > tol2 && it < a.max_iter) {
          if (!first) {
            const T beta = (T)((rho / rho_prev) * ((double)alpha / (double)omega));
            for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x)
              p[k] = r[k] + beta * (p[k] - omega * q[k]);
          }
          first = false;
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) ph[k] = p[k] * Bd[k];
          cl.sync();
          T rvt = T(0);
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            T vk = stencil_apply(B, n, mx, k, ph);
            q[k] = vk;
            rvt += rh[k] * vk;
          }
          double rv[1] = {(double)rvt};
          cl_sum<1>(cl, rv, sh, buf);
          if (rv[0] == 0.0 || !isfinite(rv[0])) { my_status |= 2; break; }
          alpha = (T)(rho / rv[0]);
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            T s = r[k] - alpha * q[k];
            sv[k] = s;
            shh[k] = s * Bd[k];
          }
          cl.sync();
          T ts0 = T(0), ts1 = T(0);
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            T t = stencil_apply(B, n, mx, k, shh);
            tv[k] = t;
            ts0 += t * sv[k];
            ts1 += t * t;
          }
          double ts[2] = {(double)ts0, (double)ts1};
          cl_sum<2>(cl, ts, sh, buf);
          omega = ts[1] > 0.0 ? (T)(ts[0] / ts[1]) : T(0);
          T rr0 = T(0), rr1 = T(0);
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            x[k] += alpha * ph[k] + omega * shh[k];
            T rk = sv[k] - omega * tv[k];
            r[k] = rk;
            rr0 += rh[k] * rk;
            rr1 += rk * rk;
          }
          double rr2[2] = {(double)rr0, (double)rr1};
          cl_sum<2>(cl, rr2, sh, buf);
          rho_prev = rho;
          rho = rr2[0];
          rr = rr2[1];
          ++it;
          if (rr > tol2 && (omega == T(0) || rho == 0.0)) { my_status |= 2; break; }
        }
      }
      if (rr > tol2) my_status |= 1;
      my_iters += it;
      cl.sync();
    }
    // ---- store ---------------------------------------------------------------
    const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      if (a.out.y_f64)
        static_cast<double*>(a.out.y)[oy + k] = (double)x[k];
      else
        static_cast<float*>(a.out.y)[oy + k] = (float)x[k];
    }
    cl.sync();
}

template <typename T>
__global__ void __launch_bounds__(KRY_THREADS) k_krylov(KryArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ ClRed sh;
  const int cs = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int slot = blockIdx.x / cs, nslots = gridDim.x / cs;
  T* ws = static_cast<T*>(a.ws) + (size_t)slot * a.nvec * a.n;
  cl_map(cl, sh);
  int buf = 0;
  unsigned long long my_iters = 0;
  int my_status = 0;
  for (int sys = slot; sys < a.nsys; sys += nslots)
    krylov_system<T>(a, cl, sh, buf, sys, ws, my_iters, my_status);
  if (threadIdx.x == 0 && crank == 0) {
    if (my_iters) atomicAdd(a.iters, my_iters);
    if (my_status) atomicOr(a.status, my_status);
  }
}

// Many problems (different grids and operators) in one persistent launch: a
// device work queue of items (problem, system), largest grids first; each
// cluster takes the next item from a global counter (rank 0 draws it and
// the other CTAs read it through distributed shared memory).
template <typename T>
__global__ void __launch_bounds__(KRY_THREADS) k_krylov_queue(const KryArgs* __restrict__ probs,
                                                               const int* __restrict__ items,
                                                               int nitems,
                                                               unsigned int* __restrict__ counter,
                                                               void* ws_all, size_t ws_stride) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ ClRed sh;
  __shared__ int next_item;
  const int cs = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int slot = blockIdx.x / cs;
  T* ws = reinterpret_cast<T*>(static_cast<char*>(ws_all) + (size_t)slot * ws_stride);
  cl_map(cl, sh);
  int buf = 0;
  unsigned long long my_iters = 0;
  int my_status = 0;
  const KryArgs* last = nullptr;
  while (true) {
    if (crank == 0 && threadIdx.x == 0) next_item = (int)atomicAdd(counter, 1u);
    cl.sync();
    const int it = *cl.map_shared_rank(&next_item, 0);
    cl.sync();                        // rank 0 may overwrite next_item only after all read it
    if (it >= nitems) break;
    const KryArgs& a = probs[items[2 * it]];
    last = &a;
    krylov_system<T>(a, cl, sh, buf, items[2 * it + 1], ws, my_iters, my_status);
  }
  if (threadIdx.x == 0 && crank == 0 && last) {
    if (my_iters) atomicAdd(last->iters, my_iters);
    if (my_status) atomicOr(last->status, my_status);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
lrp_status stencil_plan(Ctx* c, Operator* op, double dt, int adjoint, StencilPlan** out) {
  std::lock_guard<std::mutex> plan_lock(op->plan_mu);
  for (auto& p : op->splans)
    if (p->dt == dt && p->adjoint == adjoint) { *out = p.get(); return LRP_OK; }
  auto pl = std::make_unique<StencilPlan>();
  pl->dt = dt;
  pl->adjoint = adjoint;
  lrp_status s;
  if ((s = dev_alloc(op->ctx, pl->b64, sizeof(double) * 6 * (size_t)op->n))) return s;
  if ((s = dev_alloc(op->ctx, pl->b32, sizeof(float) * 6 * (size_t)op->n))) return s;
  k_stencil_plan<<<(op->n + 255) / 256, 256, 0, c->stream>>>(
      op->mx, op->my, dt, adjoint, op->a64[0].as<double>(), op->a64[1].as<double>(),
      op->a64[2].as<double>(), op->a64[3].as<double>(), op->a64[4].as<double>(),
      pl->b64.as<double>(), pl->b32.as<float>());
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_err(c, e, "k_stencil_plan");
  *out = pl.get();
  op->splans.push_back(std::move(pl));
  return LRP_OK;
}

static int cluster_size_for(int mx, int my) {
  long n = (long)mx * my;
  int cs = 1;
  while (cs < KRY_MAXCS && n / cs > 8192 && (my + 2 * cs - 1) / (2 * cs) >= 1) cs *= 2;
  while (cs > 1 && (my + cs - 1) / cs * (cs - 1) >= my) cs /= 2;   // every CTA owns rows
  return cs;
}

lrp_status stencil_propagate(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys,
                             int prec, const PropIn& in, const PropOut& out, const PropSrc& src) {
  if (nsys <= 0) return LRP_OK;
  StencilPlan* plan = nullptr;
  lrp_status s = stencil_plan(c, op, dt, adjoint, &plan);
  if (s) return s;
  const int cs = cluster_size_for(op->mx, op->my);
  const int bicg = op->symmetric ? 0 : 1;
  const int nvec = bicg ? 9 : 4;
  auto kern = prec == 0 ? (void (*)(KryArgs))k_krylov<double> : (void (*)(KryArgs))k_krylov<float>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e) return cuda_err(c, e, "krylov cluster attribute");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(KRY_THREADS);
  cfg.gridDim = dim3(cs);
  cfg.stream = c->stream;
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e || max_clusters < 1) { cudaGetLastError(); max_clusters = std::max(1, c->num_sms / cs); }
  const int nclusters = std::min(nsys, max_clusters);
  cfg.gridDim = dim3(nclusters * cs);
  const size_t es = prec == 0 ? 8 : 4;
  const size_t need = (size_t)nclusters * nvec * op->n * es;
  if (op->kws.bytes < need)
    if ((s = dev_alloc(c, op->kws, need))) return s;
  if (!op->kstat.ptr)
    if ((s = dev_alloc(c, op->kstat, 16))) return s;
  cudaMemsetAsync(op->kstat.ptr, 0, 16, c->stream);
  KryArgs a{};
  a.mx = op->mx;
  a.my = op->my;
  a.n = op->n;
  a.M = M;
  a.nsys = nsys;
  a.bicg = bicg;
  a.dt = dt;
  a.rtol = prec == 0 ? op->rtol64 : op->rtol32;
  a.max_iter = op->max_iter;
  a.B = prec == 0 ? plan->b64.ptr : plan->b32.ptr;
  a.ws = op->kws.ptr;
  a.nvec = nvec;
  a.in = in;
  a.out = out;
  a.src = src;
  a.iters = reinterpret_cast<unsigned long long*>(op->kstat.ptr);
  a.status = reinterpret_cast<int*>(static_cast<char*>(op->kstat.ptr) + 8);
  const char* fam = prec == 0 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  e = cudaLaunchKernelEx(&cfg, kern, a);
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_krylov launch");
  unsigned long long hs[2] = {0, 0};
  e = cudaMemcpyAsync(hs, op->kstat.ptr, 16, cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "k_krylov");
  op->krylov_iters += hs[0];
  int st = (int)(hs[1] & 0xffffffffu);
  if (st & 2) return set_err(c, LRP_EBREAKDOWN, "Krylov breakdown in a 2D propagation");
  if (st & 1) return set_err(c, LRP_ENOTCONV, "Krylov iteration cap reached in a 2D propagation");
  return LRP_OK;
}

// ---- work-queue launches (batched problems of uneven size) -----------------
size_t krylov_queue_nvec(int bicg) { return bicg ? 9 : 4; }

int krylov_queue_clusters(Ctx* c, int prec, int cs) {
  auto kern = prec == 0 ? (void (*)(const KryArgs*, const int*, int, unsigned int*, void*, size_t))k_krylov_queue<double>
                        : (void (*)(const KryArgs*, const int*, int, unsigned int*, void*, size_t))k_krylov_queue<float>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(KRY_THREADS);
  cfg.gridDim = dim3(cs);
  int maxc = 0;
  if (cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg) != cudaSuccess || maxc < 1) {
    cudaGetLastError();
    maxc = std::max(1, c->num_sms / cs);
  }
  return maxc;
}

lrp_status krylov_queue_launch(Ctx* c, int prec, const KryArgs* d_probs, const int* d_items,
                               int nitems, unsigned int* d_counter, void* ws, size_t ws_stride,
                               int cs, int nclusters) {
  if (nitems <= 0) return LRP_OK;
  auto kern = prec == 0 ? (void (*)(const KryArgs*, const int*, int, unsigned int*, void*, size_t))k_krylov_queue<double>
                        : (void (*)(const KryArgs*, const int*, int, unsigned int*, void*, size_t))k_krylov_queue<float>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e) return cuda_err(c, e, "queue cluster attribute");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(KRY_THREADS);
  cfg.gridDim = dim3(nclusters * cs);
  cfg.stream = c->stream;
  const char* fam = prec == 0 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  e = cudaLaunchKernelEx(&cfg, kern, d_probs, d_items, nitems, d_counter, ws, ws_stride);
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_krylov_queue launch");
  return LRP_OK;
}

}  // namespace lrp

using namespace lrp;
struct lrp_operator : public Operator {};

extern "C" lrp_status lrp_operator_stencil5(lrp_ctx* cc, int mx, int my, const double* C,
                                            const double* W, const double* E, const double* S,
                                            const double* N, lrp_operator** out) {
  Ctx* c = reinterpret_cast<Ctx*>(cc);
  if (!c || !out || !C || !W || !E || !S || !N || mx < 1 || my < 1) return LRP_EINVAL;
  if ((long)mx * my > (1L << 26)) return set_err(c, LRP_EINVAL, "grid too large");
  cudaSetDevice(c->device);
  const int n = mx * my;
  auto* op = new lrp_operator();
  op->ctx = c;
  ctx_retain(c);
  op->kind = 1;
  op->mx = mx;
  op->my = my;
  op->n = n;
  const double* src[5] = {C, W, E, S, N};
  std::vector<double> h[5];
  for (int k = 0; k < 5; ++k) {
    h[k].resize(n);
    cudaError_t e = cudaMemcpy(h[k].data(), src[k], sizeof(double) * n, cudaMemcpyDefault);
    if (e) { delete op; return cuda_err(c, e, "stencil read"); }
    lrp_status s = dev_alloc(c, op->a64[k], sizeof(double) * n);
    if (s) { delete op; return s; }
    e = cudaMemcpyAsync(op->a64[k].ptr, h[k].data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                        c->stream);
    if (e) { delete op; return cuda_err(c, e, "stencil upload"); }
  }
  // symmetric (W_p = E_{p-1}, S_p = N_{p-mx} on interior couplings): CG, else BiCGStab
  bool sym = true;
  for (int p = 0; p < n && sym; ++p) {
    int ix = p % mx, iy = p / mx;
    if (ix > 0 && h[1][p] != h[2][p - 1]) sym = false;
    if (iy > 0 && h[3][p] != h[4][p - mx]) sym = false;
  }
  op->symmetric = sym;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) { delete op; return cuda_err(c, e, "stencil upload"); }
  *out = op;
  return LRP_OK;
}
