// Batched backward-Euler propagator for 5-point stencil operators (2D): every
// implicit-Euler step (I + dt A) x_{j+1} = x_j + dt f(t_{j+1}) is solved by a
// Jacobi-preconditioned Krylov method warm-started from x_j -- conjugate
// gradients when A is symmetric, BiCGStab otherwise -- to a relative
// residual rtol (d the step's right-hand side, D = diag(B)^-1): for CG the
// residual of the diagonally scaled system, ||D^1/2 (d - B x)|| <= rtol
// ||D^1/2 d||, for BiCGStab ||d - B x|| <= rtol ||d||; an iteration cap per
// step raises a status instead of looping on.  Symmetric operators whose
// grid fits one thread-block cluster's registers and shared memory run on
// the on-chip CG kernel instead (stencil_onchip.cuh).
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
// grid removed; dinv = 1 / diag.  Each of the 6 arrays has a zero pad of mx
// entries on both sides (row stride n + 2 mx), so that the stencil reads its
// four neighbours without bounds tests: couplings across the boundary are 0.
__global__ void k_stencil_plan(int mx, int my, double dt, int adj, const double* __restrict__ C,
                               const double* __restrict__ W, const double* __restrict__ E,
                               const double* __restrict__ S, const double* __restrict__ N,
                               double* __restrict__ b64, float* __restrict__ b32) {
  const int n = mx * my;
  const size_t ld = (size_t)n + 2 * mx;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  // time-dependent operators: grid row J takes step J's coefficients and plan
  const size_t J = blockIdx.y;
  C += J * n; W += J * n; E += J * n; S += J * n; N += J * n;
  b64 += J * 6 * ld;
  b32 += J * 6 * ld;
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
    b64[(size_t)k * ld + mx + p] = v[k];
    b32[(size_t)k * ld + mx + p] = (float)v[k];
  }
}

// The diagonally scaled step matrix of a symmetric operator, B^ = S^-1 B S^-1
// with S = diag(sqrt(c)), c the diagonal of B = I + dt A: [7][n + 2 mx] =
// west, east, south, north couplings of B^ (its diagonal is 1), 1/c,
// 1/sqrt(c), sqrt(c), with the layout and zero pads of the plan arrays.  The
// coupling of p to q is b_pq / sqrt(c_p c_q) for both directions, so B^ is
// symmetric bitwise when B is.
__global__ void k_stencil_plan_scaled(int mx, int my, const double* __restrict__ b64,
                                      double* __restrict__ s64, float* __restrict__ s32) {
  const int n = mx * my;
  const size_t ld = (size_t)n + 2 * mx;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const size_t J = blockIdx.y;   // time-dependent operators: step J
  b64 += J * 6 * ld;
  s64 += J * 7 * ld;
  s32 += J * 7 * ld;
  const size_t q = (size_t)mx + p;
  const double* c = b64;
  const double cp = c[q];
  const double w = b64[ld + q], e = b64[2 * ld + q], so = b64[3 * ld + q], no = b64[4 * ld + q];
  const int ix = p % mx, iy = p / mx;
  double v[7];
  v[0] = ix > 0 ? w / sqrt(cp * c[q - 1]) : 0.0;
  v[1] = ix < mx - 1 ? e / sqrt(cp * c[q + 1]) : 0.0;
  v[2] = iy > 0 ? so / sqrt(cp * c[q - mx]) : 0.0;
  v[3] = iy < my - 1 ? no / sqrt(cp * c[q + mx]) : 0.0;
  v[4] = 1.0 / cp;
  v[5] = 1.0 / sqrt(cp);
  v[6] = sqrt(cp);
  for (int k = 0; k < 7; ++k) {
    s64[(size_t)k * ld + q] = v[k];
    s32[(size_t)k * ld + q] = (float)v[k];
  }
}

// Cluster-wide reductions: per-warp sums in the working precision, per-CTA
// sums in FP64 pushed into every CTA's shared memory before the cluster
// barrier (remote stores), then one fixed-order sum over the CTAs per value.
struct ClRed {
  double red[KRY_THREADS / 32][KRY_MAXNV];
  double part[2][KRY_MAXCS][KRY_MAXNV];
  double tot[KRY_MAXNV];
  double* rpart[KRY_MAXCS];   // part[][][] of every CTA of the cluster (DSMEM), mapped once
};

__device__ __forceinline__ void cl_map(cg::cluster_group& cl, ClRed& sh) {
  for (int q = threadIdx.x; q < (int)cl.num_blocks(); q += blockDim.x)
    sh.rpart[q] = cl.map_shared_rank(&sh.part[0][0][0], q);
  __syncthreads();
}

// Sum of NV values over the cluster (deterministic order); also a cluster
// barrier.  v: per-thread partials in T on entry, cluster totals on exit.
template <typename T, int NV>
__device__ __forceinline__ void cl_sum(cg::cluster_group& cl, const T (&v)[NV], double (&out)[NV],
                                       ClRed& sh, int& buf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int cs = (int)cl.num_blocks(), crank = (int)cl.block_rank();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const T s = warp_sum<T>(v[i]);
    if (lane == 0) sh.red[w][i] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < NV * cs) {
    const int i = threadIdx.x % NV, q = threadIdx.x / NV;
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sh.red[k][i];
    sh.rpart[q][(buf * KRY_MAXCS + crank) * KRY_MAXNV + i] = s;
  }
  cl.sync();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int q = 0; q < cs; ++q) s += sh.part[buf][q][threadIdx.x];
    sh.tot[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = sh.tot[i];
  buf ^= 1;
}

// ---- staged stencil inputs (FP32 passes): the CTA's rows of the input vector
// of a stencil pass and one halo row on each side are brought into shared
// memory by one bulk asynchronous copy of the TMA engine (cp.async.bulk,
// completion on an mbarrier), and the pass reads the five points of its
// stencil from there.  Every thread orders its global stores of the vector
// before the copy (fence.proxy.async.global, then the cluster barrier that
// ends the producing pass); the issuing thread orders the previous pass's
// shared-memory reads of the tile before the copy that overwrites it
// (fence.proxy.async.shared::cta after the barrier).  Waits are bounded: a
// wait that gives up sets status bit 2 (LRP_ETIMEOUT) and the pass reads
// global memory instead, so that its result stays right.  Opt-in
// (krylov_stage = 1): measured on GB300 at 511^2 (FP32, 64 systems) it is
// bitwise equal to the unstaged kernel and no faster (CG 2.24 against 2.25 us
// per iteration and system, BiCGStab 7.09 against 6.95), the L1 cache already
// serving the stencil's reuse of neighbouring rows.
constexpr long KRY_SPIN = 1L << 20;   // polls of the mbarrier before giving up

__device__ __forceinline__ uint32_t kry_saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool kry_mbar_wait(uint32_t a, uint32_t parity) {
  for (long i = 0; i < KRY_SPIN; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void kry_fence_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Staging state of a CTA (its tile in dynamic shared memory and mbarrier).
struct KryStage {
  float* tile = nullptr;    // nullptr: no staging
  uint32_t bar = 0;         // shared address of the mbarrier
  uint32_t phase = 0;       // parity of the next phase (the same in every thread)
  bool failed = false;      // a wait gave up: no more staging in this launch
};

// Stage v[k0 - mx, k1 + mx) of a padded FP32 vector (v points past the pad);
// returns q with q[k] = v[k] over that range, or v itself when not staged.
// Called by every thread of the CTA at the same point, after a barrier that
// follows the stores of v.
__device__ __forceinline__ const float* kry_stage(KryStage& st, const float* v, int k0, int k1, int mx,
                                                  int& my_status) {
  if (!st.tile || st.failed || k1 <= k0) return v;
  const uintptr_t src = reinterpret_cast<uintptr_t>(v + (k0 - mx));
  const uintptr_t s0 = src & ~(uintptr_t)15;
  const int off = (int)((src - s0) / sizeof(float));
  const uint32_t bytes = (uint32_t)((((size_t)(k1 - k0 + 2 * mx) * sizeof(float) + (src - s0)) + 15) & ~(size_t)15);
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(st.bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            kry_saddr(st.tile)),
        "l"(reinterpret_cast<const void*>(s0)), "r"(bytes), "r"(st.bar)
        : "memory");
  }
  const bool ok = kry_mbar_wait(st.bar, st.phase) || kry_mbar_wait(st.bar, st.phase);
  st.phase ^= 1u;
  if (!ok) {
    st.failed = true;
    my_status |= 4;
    return v;
  }
  return st.tile + off - (k0 - mx);
}

// (B v)_k for the padded layouts: no bounds tests, boundary couplings are 0
// and the pads of v are 0.
template <typename T>
__device__ __forceinline__ T stencil_apply(const T* __restrict__ B, size_t ldb, int mx, int k,
                                           const T* __restrict__ v) {
  T acc = B[k] * v[k];
  acc += B[ldb + k] * v[k - 1];
  acc += B[2 * ldb + k] * v[k + 1];
  acc += B[3 * ldb + k] * v[k - mx];
  acc += B[4 * ldb + k] * v[k + mx];
  return acc;
}

// Loop over this CTA's points k in [k0, k1), KRY_UNROLL points per thread and
// round: the loads of all of them are issued before any of their arithmetic
// and stores (the passes only store to vectors they do not load at other
// points), so each thread keeps several L2 requests in flight.
constexpr int KRY_UNROLL = 4;
constexpr size_t KRY_STAGE_MAX = 100 * 1024;   // staging tile per CTA (two CTAs per SM)
template <typename Regs, typename Load, typename Comp>
__device__ __forceinline__ void for_points(int k0, int k1, Load load, Comp comp) {
  const int bd = blockDim.x;
  int kb = k0 + threadIdx.x;
  for (; kb + (KRY_UNROLL - 1) * bd < k1; kb += KRY_UNROLL * bd) {
    Regs g0 = load(kb), g1 = load(kb + bd), g2 = load(kb + 2 * bd), g3 = load(kb + 3 * bd);
    comp(kb, g0);
    comp(kb + bd, g1);
    comp(kb + 2 * bd, g2);
    comp(kb + 3 * bd, g3);
  }
  for (; kb < k1; kb += bd) comp(kb, load(kb));
}

// One system (vector `sys` of the problem described by `a`) on this cluster,
// using the workspace `ws` (a.nvec padded vectors of n + 2 mx values).
// SD: two-stage SDIRK steps.  TD: a time-dependent operator, every fine step
// its own plan (B, Bs advance by a.b_step, a.bs_step per step of the time
// grid); the system runs steps J0 .. J0 + M - 1 of its interval, the
// adjoint in reversed order.
template <typename T, bool SD = false, bool TD = false>
__device__ __forceinline__ void krylov_system(const KryArgs& a, cg::cluster_group& cl, ClRed& sh,
                                              int& buf, int sys, T* ws,
                                              unsigned long long& my_iters, int& my_status,
                                              KryStage* stg = nullptr) {
  const int cs = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int n = a.n, mx = a.mx;
  const size_t ldv = (size_t)n + 2 * mx;
  const size_t ldb = ldv;
  const int rows_per = (a.my + cs - 1) / cs;
  const int k0 = min(a.n, crank * rows_per * mx), k1 = min(a.n, (crank + 1) * rows_per * mx);
  const T* __restrict__ B = static_cast<const T*>(a.B);
  const T* __restrict__ Bd = B + 5 * ldb;             // 1 / diag (0 on the pads)
  const T* __restrict__ Bs = static_cast<const T*>(a.Bs);   // CG: scaled matrix (see KryArgs)
  long J0 = 0;
  if constexpr (TD) {
    // the interval of the system (system map of the input, else of the
    // output, else of the source; else interval0 + sys / ncol), its first step
    const int* imap = a.in.map ? a.in.map : a.out.map ? a.out.map : a.src.map;
    const int interval = imap ? imap[2 * sys + 1] : a.in.interval0 + sys / a.in.ncol;
    J0 = (long)interval * a.M;
    if (J0 < 0 || J0 + a.M > a.nJ) return;    // outside the time grid (checked on the host)
  }
  // TD: the plan of solve st of step j of the system (j in the order the
  // steps run): backward Euler: row J of the time grid; SDIRK: row 2J + s,
  // the operator at stage time s, solved stage 1 then 2 forward and stage 2
  // then 1 in the adjoint (the transposed step map)
  auto set_step = [&](int j, int st) {
    const long J = a.adj ? J0 + a.M - 1 - j : J0 + j;
    const long row = SD ? 2 * J + (a.adj ? 1 - st : st) : J;
    B = static_cast<const T*>(a.B) + row * a.b_step;
    Bd = B + 5 * ldb;
    if (a.Bs) Bs = static_cast<const T*>(a.Bs) + row * a.bs_step;
  };
  if constexpr (TD) set_step(0, 0);
  auto vec = [&](int v) { return ws + (size_t)v * ldv + mx; };
  T* x = vec(0);
  T* r = vec(1);
  T* p = vec(2);            // CG: p; BiCG: p
  T* q = vec(3);            // CG: q = B p; BiCG: v
  T* rh = vec(4);           // BiCG: r-hat
  T* ph = vec(5);           // BiCG: D^-1 p
  T* sv = vec(6);           // BiCG: s
  T* shh = vec(7);          // BiCG: D^-1 s
  T* tv = vec(8);           // BiCG: t = B D^-1 s
  T* u0v = SD ? vec(a.bicg ? 9 : 4) : nullptr;    // SDIRK: the state at the step start
  T* u1v = SD ? vec(a.bicg ? 10 : 5) : nullptr;   // SDIRK: the first stage value
  const T dt = (T)a.dt;
  struct St { T c0, c1, c2, c3, c4, v0, v1, v2, v3, v4; };   // stencil operands
  auto st_load = [&](int k, const T* v) {
    return St{B[k], B[ldb + k], B[2 * ldb + k], B[3 * ldb + k], B[4 * ldb + k],
              v[k], v[k - 1], v[k + 1], v[k - mx], v[k + mx]};
  };
  auto st_eval = [](const St& g) {
    T acc = g.c0 * g.v0;
    acc += g.c1 * g.v1;
    acc += g.c2 * g.v2;
    acc += g.c3 * g.v3;
    acc += g.c4 * g.v4;
    return acc;
  };
  // the input of a stencil pass, staged in shared memory where enabled (FP32)
  auto staged = [&](const T* v) -> const T* {
    if constexpr (std::is_same<T, float>::value) {
      if (stg) return kry_stage(*stg, v, k0, k1, mx, my_status);
    }
    return v;
  };
  // global stores of a vector that a later pass stages: ordered before the copy
  auto fence_stores = [&]() {
    if constexpr (std::is_same<T, float>::value) {
      if (stg && stg->tile) kry_fence_global();
    }
  };
  // zero pads of every workspace vector (the stencil reads them)
  for (int e = crank * blockDim.x + threadIdx.x; e < a.nvec * 2 * mx; e += cs * blockDim.x) {
    const int v = e / (2 * mx), o = e % (2 * mx);
    T* base = ws + (size_t)v * ldv;
    base[o < mx ? o : n + o] = T(0);       // [0, mx) and [n + mx, n + 2 mx)
  }
  // ---- initial vector ------------------------------------------------------
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    T v = T(0);
    if (a.in.gen)
      v = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                   (uint32_t)(sys % a.in.ncol), (uint32_t)k);
    else if (a.in.x == nullptr)
      v = T(0);
    else if (a.in.x_f64)
      v = (T) static_cast<const double*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + k];
    else
      v = (T) static_cast<const float*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + k];
    if (!a.bicg && a.M > 0) v *= Bs[6 * ldb + k];   // CG iterates in x^ = S x
    x[k] = v;
  }
  cl.sync();
  const double* csys = a.src.Q > 0
      ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
  const double* gsys = (a.src.Q > 0 && a.src.map)
      ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
  // one solve B x = d from the warm start x, d = au uv + a1 w1 + dt f (w1 may
  // be null; f the source sample fj; CG: the scaled vectors of the same
  // combination)
  auto solve = [&](T au, const T* uv, T a1, const T* w1, int fj) {
    // ---- right-hand side d, residual r = d - B x -------------------------
    T red3t[3] = {T(0), T(0), T(0)};    // d.d, r.r, rho
    for (int k = k0 + threadIdx.x; k < k1 && !a.bicg; k += blockDim.x) {
      // CG: d^ = (au u^ + a1 w1^) / c + dt f / sqrt(c), r = p = d^ - B^ x^
      T f = T(0);
      if (csys)
        for (int qq = 0; qq < a.src.Q; ++qq)
          f += (T)csys[(size_t)fj * a.src.Q + qq] * (T)gsys[(size_t)qq * n + k];
      T dv = au * uv[k];
      if (w1) dv += a1 * w1[k];
      // SD + TD: the stage vectors are kept unscaled (the scaling changes
      // with the stage's matrix), d^ = S^-1 (d + dt f)
      const T d = (SD && TD) ? Bs[5 * ldb + k] * (dv + dt * f)
                             : Bs[4 * ldb + k] * dv + dt * Bs[5 * ldb + k] * f;
      T bx = x[k];
      bx += Bs[k] * x[k - 1];
      bx += Bs[ldb + k] * x[k + 1];
      bx += Bs[2 * ldb + k] * x[k - mx];
      bx += Bs[3 * ldb + k] * x[k + mx];
      const T rk = d - bx;
      r[k] = rk;
      p[k] = rk;
      red3t[0] += d * d;
      red3t[1] += rk * rk;
      red3t[2] += rk * rk;
    }
    if (!a.bicg) fence_stores();
    for (int k = k0 + threadIdx.x; k < k1 && a.bicg; k += blockDim.x) {
      T d = au * uv[k];
      if (w1) d += a1 * w1[k];
      if (csys)
        for (int qq = 0; qq < a.src.Q; ++qq)
          d += dt * (T)csys[(size_t)fj * a.src.Q + qq] * (T)gsys[(size_t)qq * n + k];
      T rk = d - stencil_apply(B, ldb, mx, k, x);
      r[k] = rk;
      red3t[0] += d * d;
      red3t[1] += rk * rk;
      rh[k] = rk;
      p[k] = rk;
      red3t[2] += rk * rk;
    }
    double red3[3];
    cl_sum<T, 3>(cl, red3t, red3, sh, buf);
    const double tol2 = a.rtol * a.rtol * red3[0];
    double rr = red3[1], rho = red3[2];
    int it = 0;
    if (!a.bicg) {
      // ---- conjugate gradients on the diagonally scaled system ----------------
      // (Jacobi-preconditioned CG on B x = d: the same Krylov spaces and
      // scalars in exact arithmetic; B^ has a unit diagonal, so q = p + the
      // four scaled couplings, and the residual r^ = S^-1 r is the quantity
      // the stopping test measures: ||r^|| <= rtol ||d^||)
      struct Sc { T w, e, s, nn, v0, v1, v2, v3, v4; };
      while (rr > tol2 && it < a.max_iter) {
        T pqt[1] = {T(0)};
        const T* ps = staged(p);
        for_points<Sc>(k0, k1,
                       [&](int k) {
                         return Sc{Bs[k], Bs[ldb + k], Bs[2 * ldb + k], Bs[3 * ldb + k],
                                   ps[k], ps[k - 1], ps[k + 1], ps[k - mx], ps[k + mx]};
                       },
                       [&](int k, const Sc& g) {
                         T qk = g.v0;
                         qk += g.w * g.v1;
                         qk += g.e * g.v2;
                         qk += g.s * g.v3;
                         qk += g.nn * g.v4;
                         q[k] = qk;
                         pqt[0] += g.v0 * qk;
                       });
        double pq[1];
        cl_sum<T, 1>(cl, pqt, pq, sh, buf);
        if (!(pq[0] > 0.0)) { my_status |= 2; break; }
        const T alpha = (T)(rho / pq[0]);
        T rz[1] = {T(0)};
        struct Up { T x, p, r, q; };
        for_points<Up>(k0, k1,
                       [&](int k) { return Up{x[k], p[k], r[k], q[k]}; },
                       [&](int k, const Up& g) {
                         x[k] = g.x + alpha * g.p;
                         const T rk = g.r - alpha * g.q;
                         r[k] = rk;
                         rz[0] += rk * rk;
                       });
        double rzd[1];
        cl_sum<T, 1>(cl, rz, rzd, sh, buf);
        const T beta = (T)(rzd[0] / rho);
        rho = rzd[0];
        rr = rzd[0];
        ++it;
        struct Pu { T r, p; };
        for_points<Pu>(k0, k1, [&](int k) { return Pu{r[k], p[k]}; },
                       [&](int k, const Pu& g) { p[k] = g.r + beta * g.p; });
        fence_stores();
        cl.sync();
      }
    } else {
      // ---- BiCGStab with Jacobi right preconditioning ---------------------
      double rho_prev = rho;
      T alpha = T(1), omega = T(1);
      bool first = true;
      while (rr > tol2 && it < a.max_iter) {
        struct Pb { T r, p, q, d; };
        if (!first) {
          const T beta = (T)((rho / rho_prev) * ((double)alpha / (double)omega));
          for_points<Pb>(k0, k1, [&](int k) { return Pb{r[k], p[k], q[k], Bd[k]}; },
                         [&](int k, const Pb& g) {
                           const T pk = g.r + beta * (g.p - omega * g.q);
                           p[k] = pk;
                           ph[k] = pk * g.d;
                         });
        } else {
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) ph[k] = p[k] * Bd[k];
        }
        first = false;
        fence_stores();
        cl.sync();
        T rvt[1] = {T(0)};
        struct Sv { St s; T rh; };
        const T* phs = staged(ph);
        for_points<Sv>(k0, k1, [&](int k) { return Sv{st_load(k, phs), rh[k]}; },
                       [&](int k, const Sv& g) {
                         const T vk = st_eval(g.s);
                         q[k] = vk;
                         rvt[0] += g.rh * vk;
                       });
        double rv[1];
        cl_sum<T, 1>(cl, rvt, rv, sh, buf);
        if (rv[0] == 0.0 || !isfinite(rv[0])) { my_status |= 2; break; }
        alpha = (T)(rho / rv[0]);
        struct Ss { T r, q, d; };
        for_points<Ss>(k0, k1, [&](int k) { return Ss{r[k], q[k], Bd[k]}; },
                       [&](int k, const Ss& g) {
                         const T s = g.r - alpha * g.q;
                         sv[k] = s;
                         shh[k] = s * g.d;
                       });
        fence_stores();
        cl.sync();
        T tst[2] = {T(0), T(0)};
        struct Tv { St s; T sv; };
        const T* shs = staged(shh);
        for_points<Tv>(k0, k1, [&](int k) { return Tv{st_load(k, shs), sv[k]}; },
                       [&](int k, const Tv& g) {
                         const T t = st_eval(g.s);
                         tv[k] = t;
                         tst[0] += t * g.sv;
                         tst[1] += t * t;
                       });
        double ts[2];
        cl_sum<T, 2>(cl, tst, ts, sh, buf);
        omega = ts[1] > 0.0 ? (T)(ts[0] / ts[1]) : T(0);
        T rrt[2] = {T(0), T(0)};
        struct Xu { T x, ph, shh, sv, tv, rh; };
        for_points<Xu>(k0, k1,
                       [&](int k) { return Xu{x[k], ph[k], shh[k], sv[k], tv[k], rh[k]}; },
                       [&](int k, const Xu& g) {
                         x[k] = g.x + alpha * g.ph + omega * g.shh;
                         const T rk = g.sv - omega * g.tv;
                         r[k] = rk;
                         rrt[0] += g.rh * rk;
                         rrt[1] += rk * rk;
                       });
        double rr2[2];
        cl_sum<T, 2>(cl, rrt, rr2, sh, buf);
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
  };
  for (int j = 0; j < a.M; ++j) {
    if constexpr (TD && !SD) {
      if (j > 0) {
        // CG iterates in x^ = S_J x: rescale from the previous step's S
        const T* Bp = Bs;
        set_step(j, 0);
        if (!a.bicg) {
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x)
            x[k] = x[k] * Bp[5 * ldb + k] * Bs[6 * ldb + k];
          cl.sync();                             // the stencil reads neighbours' points
        }
      }
    }
    if constexpr (!SD) {
      solve(T(1), x, T(0), nullptr, j);        // backward Euler: d = x + dt f(t_{j+1})
    } else if constexpr (TD) {
      // SDIRK on a time-dependent operator: each stage solve on its own
      // matrix; u0v, u1v hold unscaled vectors and x (the Krylov iterate) is
      // rescaled to the diagonal of the matrix it is solved with (CG).  With
      // the combination coefficients remapped by the host, the same body runs
      // the adjoint: W2 = B2^-T v, W1 = B1^-T (b1 v + b2 s1 W2), v' = bu v +
      // b2 su W2 + W1.
      const bool cgs = !a.bicg;
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) u0v[k] = cgs ? x[k] * Bs[5 * ldb + k] : x[k];
      {
        const T* Bp = Bs;
        set_step(j, 0);
        if (cgs)
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x)
            x[k] = x[k] * Bp[5 * ldb + k] * Bs[6 * ldb + k];
      }
      cl.sync();
      solve(T(1), u0v, T(0), nullptr, 2 * j);
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) u1v[k] = cgs ? x[k] * Bs[5 * ldb + k] : x[k];
      {
        const T* Bp = Bs;
        set_step(j, 1);
        if (cgs)
          for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x)
            x[k] = x[k] * Bp[5 * ldb + k] * Bs[6 * ldb + k];
      }
      cl.sync();
      solve((T)a.su, u0v, (T)a.s1, u1v, 2 * j + 1);
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const T u2 = cgs ? x[k] * Bs[5 * ldb + k] : x[k];
        const T v = (T)a.bu * u0v[k] + (T)a.b1 * u1v[k] + (T)a.b2 * u2;
        x[k] = cgs ? v * Bs[6 * ldb + k] : v;
      }
      cl.sync();
    } else {
      // two-stage SDIRK with B = I + gamma dt A (dt here is gamma dt): stage
      // values U1 = B^-1 (u + gamma dt f_1), U2 = B^-1 (su u + s1 U1 + gamma dt f_2),
      // the new state bu u + b1 U1 + b2 U2 (the source at the stage times,
      // samples 2j and 2j + 1); every point is handled by the same thread in
      // these loops and in the right-hand side of the solves
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) u0v[k] = x[k];
      solve(T(1), u0v, T(0), nullptr, 2 * j);
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) u1v[k] = x[k];
      solve((T)a.su, u0v, (T)a.s1, u1v, 2 * j + 1);
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x)
        x[k] = (T)a.bu * u0v[k] + (T)a.b1 * u1v[k] + (T)a.b2 * x[k];
      cl.sync();
    }
  }
  // ---- store -----------------------------------------------------------------
  const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const T v = !a.bicg && a.M > 0 ? x[k] * Bs[5 * ldb + k] : x[k];   // CG: x = S^-1 x^
    if (a.out.y_f64)
      static_cast<double*>(a.out.y)[oy + k] = (double)v;
    else
      static_cast<float*>(a.out.y)[oy + k] = (float)v;
  }
  cl.sync();
}

template <typename T, bool SD = false, bool TD = false>
__global__ void __launch_bounds__(KRY_THREADS, 2) k_krylov(KryArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  cg::cluster_group cl = cg::this_cluster();
  __shared__ ClRed sh;
  __shared__ alignas(8) unsigned long long kbar;
  extern __shared__ __align__(16) unsigned char kry_dyn[];
  KryStage stg;
  KryStage* stp = nullptr;
  if constexpr (std::is_same<T, float>::value) {
    if (a.stage) {          // FP32 stencil inputs staged through dynamic shared memory
      stg.tile = reinterpret_cast<float*>(kry_dyn);
      stg.bar = kry_saddr(&kbar);
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(stg.bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      __syncthreads();
      stp = &stg;
    }
  }
  const int cs = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int slot = blockIdx.x / cs, nslots = gridDim.x / cs;
  T* ws = static_cast<T*>(a.ws) + (size_t)slot * a.nvec * ((size_t)a.n + 2 * a.mx);
  cl_map(cl, sh);
  cl.sync();   // every CTA runs before remote stores into its shared memory
  int buf = 0;
  unsigned long long my_iters = 0;
  int my_status = 0;
  for (int sys = slot; sys < a.nsys; sys += nslots)
    krylov_system<T, SD, TD>(a, cl, sh, buf, sys, ws, my_iters, my_status, stp);
  // a copy still in flight after a wait that gave up: wait for it (bounded)
  // before the CTA's shared memory goes away
  if (stp && stg.failed) kry_mbar_wait(stg.bar, stg.phase ^ 1u);
  if (threadIdx.x == 0 && crank == 0) {
    if (my_iters) atomicAdd(a.iters, my_iters);
    if (my_status) atomicOr(a.status, my_status);
  }
}

// ---------------------------------------------------------------------------
// FP64 steps by mixed-precision iterative refinement inside the kernel (the
// batched queue's fine solves): per step and round, the FP64 residual
// r = d - B x of the cluster's system and its norms (CG: scaled by 1/diag,
// BiCGStab: plain; and the rounding level of |d| + |B||x|), one cluster
// reduction, the test of the FP64 Krylov kernels (rtol, or the rounding
// level 8 u_64), then FP32 Krylov iterations on B e = r / sigma from e = 0
// to a.rtol_in and the FP64 update x += sigma e.  Workspace of a cluster:
// two FP64 vectors (x, d) and ten FP32 vectors, each padded like the others.
// ---------------------------------------------------------------------------
constexpr int IRK_ROUNDS = 60;
constexpr double IRK_FLOOR = 8.0;

__device__ __forceinline__ void krylov_system_ir(const KryArgs& a, cg::cluster_group& cl, ClRed& sh,
                                                 int& buf, int sys, void* ws_raw,
                                                 unsigned long long& my_iters, int& my_status) {
  const int cs = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int n = a.n, mx = a.mx;
  const size_t ldv = (size_t)n + 2 * mx;
  const size_t ldb = ldv;
  const int rows_per = (a.my + cs - 1) / cs;
  const int k0 = min(a.n, crank * rows_per * mx), k1 = min(a.n, (crank + 1) * rows_per * mx);
  const bool cgm = !a.bicg;
  const double* __restrict__ B64 = static_cast<const double*>(a.B);
  const float* __restrict__ B32 = static_cast<const float*>(a.B32);
  const float* __restrict__ Bd32 = B32 + 5 * ldb;
  const float* __restrict__ Bs32 = static_cast<const float*>(a.Bs32);
  double* x = static_cast<double*>(ws_raw) + mx;
  double* dv = x + ldv;
  float* fb = reinterpret_cast<float*>(static_cast<double*>(ws_raw) + 2 * ldv);
  auto fvec = [&](int v) { return fb + (size_t)v * ldv + mx; };
  float* rf = fvec(0);   // r / sigma
  float* ev = fvec(1);   // correction (CG: scaled)
  float* r = fvec(2);
  float* p = fvec(3);
  float* q = fvec(4);    // CG: B^ p; BiCG: v
  float* rh = fvec(5);
  float* ph = fvec(6);
  float* sv = fvec(7);
  float* shh = fvec(8);
  float* tv = fvec(9);
  // zero pads of the two FP64 and ten FP32 vectors (the stencils read them)
  for (int e = crank * blockDim.x + threadIdx.x; e < 12 * 2 * mx; e += cs * blockDim.x) {
    const int v = e / (2 * mx), o = e % (2 * mx);
    const size_t at = o < mx ? (size_t)o : (size_t)n + o;
    if (v < 2)
      static_cast<double*>(ws_raw)[(size_t)v * ldv + at] = 0.0;
    else
      fb[(size_t)(v - 2) * ldv + at] = 0.0f;
  }
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double v = 0.0;
    if (a.in.x != nullptr)
      v = a.in.x_f64 ? static_cast<const double*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + k]
                     : (double)static_cast<const float*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + k];
    x[k] = v;
  }
  const double* csys = a.src.Q > 0
      ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
  const double* gsys = (a.src.Q > 0 && a.src.map)
      ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
  const double rtol2 = a.rtol * a.rtol;
  const double floor2 = (IRK_FLOOR * 0x1p-53) * (IRK_FLOOR * 0x1p-53);
  const float rtol_in2 = (float)(a.rtol_in * a.rtol_in);
  // FP64 residual of point k: r, and |d| + |B||x|
  auto resid = [&](int k, double& ab) -> double {
    const double t0 = B64[k] * x[k], t1 = B64[ldb + k] * x[k - 1], t2 = B64[2 * ldb + k] * x[k + 1];
    const double t3 = B64[3 * ldb + k] * x[k - mx], t4 = B64[4 * ldb + k] * x[k + mx];
    const double d = dv[k];
    ab = fabs(d) + fabs(t0) + fabs(t1) + fabs(t2) + fabs(t3) + fabs(t4);
    return d - ((((t0 + t1) + t2) + t3) + t4);
  };
  for (int j = 0; j < a.M; ++j) {
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      double f = 0.0;
      if (csys)
        for (int qq = 0; qq < a.src.Q; ++qq) f += csys[(size_t)j * a.src.Q + qq] * gsys[(size_t)qq * n + k];
      dv[k] = x[k] + a.dt * f;
    }
    cl.sync();
    for (int round = 0;; ++round) {
      double red[3] = {0.0, 0.0, 0.0};
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        double ab;
        const double rk = resid(k, ab);
        const double w = cgm ? B64[5 * ldb + k] : 1.0;
        red[0] += rk * rk * w;
        red[1] += dv[k] * dv[k] * w;
        red[2] += ab * ab * w;
      }
      double tot[3];
      cl_sum<double, 3>(cl, red, tot, sh, buf);
      if (tot[0] <= rtol2 * tot[1] || tot[0] <= floor2 * tot[2]) break;
      if (round == IRK_ROUNDS || a.max_iter == 0) { my_status |= 1; break; }
      const double sig = sqrt(tot[0] / n);
      // the correction solve's right-hand side and first residual (e = 0)
      float rr0t[1] = {0.0f};
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        double ab;
        const float rs = (float)(resid(k, ab) / sig);
        rf[k] = rs;
        ev[k] = 0.0f;
        const float r0 = cgm ? rs * Bs32[5 * ldb + k] : rs;   // CG: S^-1 r
        r[k] = r0;
        p[k] = r0;
        if (!cgm) rh[k] = r0;
        rr0t[0] += r0 * r0;
      }
      double rr0[1];
      cl_sum<float, 1>(cl, rr0t, rr0, sh, buf);
      const double tol2 = (double)rtol_in2 * rr0[0];
      double rr = rr0[0], rho = rr0[0];
      int it = 0;
      if (cgm) {
        struct Sc { float w, e, s, nn, v0, v1, v2, v3, v4; };
        while (rr > tol2 && it < a.max_iter) {
          float pqt[1] = {0.0f};
          for_points<Sc>(k0, k1,
                         [&](int k) {
                           return Sc{Bs32[k], Bs32[ldb + k], Bs32[2 * ldb + k], Bs32[3 * ldb + k],
                                     p[k], p[k - 1], p[k + 1], p[k - mx], p[k + mx]};
                         },
                         [&](int k, const Sc& g) {
                           float qk = g.v0;
                           qk += g.w * g.v1;
                           qk += g.e * g.v2;
                           qk += g.s * g.v3;
                           qk += g.nn * g.v4;
                           q[k] = qk;
                           pqt[0] += g.v0 * qk;
                         });
          double pq[1];
          cl_sum<float, 1>(cl, pqt, pq, sh, buf);
          if (!(pq[0] > 0.0)) break;                  // the round ends; the FP64 test decides
          const float alpha = (float)(rho / pq[0]);
          float rz[1] = {0.0f};
          struct Up { float x, p, r, q; };
          for_points<Up>(k0, k1, [&](int k) { return Up{ev[k], p[k], r[k], q[k]}; },
                         [&](int k, const Up& g) {
                           ev[k] = g.x + alpha * g.p;
                           const float rk = g.r - alpha * g.q;
                           r[k] = rk;
                           rz[0] += rk * rk;
                         });
          double rzd[1];
          cl_sum<float, 1>(cl, rz, rzd, sh, buf);
          const float beta = (float)(rzd[0] / rho);
          rho = rzd[0];
          rr = rzd[0];
          ++it;
          struct Pu { float r, p; };
          for_points<Pu>(k0, k1, [&](int k) { return Pu{r[k], p[k]}; },
                         [&](int k, const Pu& g) { p[k] = g.r + beta * g.p; });
          cl.sync();
        }
      } else {
        struct St { float c0, c1, c2, c3, c4, v0, v1, v2, v3, v4; };
        auto st_load = [&](int k, const float* v) {
          return St{B32[k], B32[ldb + k], B32[2 * ldb + k], B32[3 * ldb + k], B32[4 * ldb + k],
                    v[k], v[k - 1], v[k + 1], v[k - mx], v[k + mx]};
        };
        auto st_eval = [](const St& g) {
          float acc = g.c0 * g.v0;
          acc += g.c1 * g.v1;
          acc += g.c2 * g.v2;
          acc += g.c3 * g.v3;
          acc += g.c4 * g.v4;
          return acc;
        };
        double rho_prev = rho;
        float alpha = 1.0f, omega = 1.0f;
        bool first = true;
        while (rr > tol2 && it < a.max_iter) {
          struct Pb { float r, p, q, d; };
          if (!first) {
            const float beta = (float)((rho / rho_prev) * ((double)alpha / (double)omega));
            for_points<Pb>(k0, k1, [&](int k) { return Pb{r[k], p[k], q[k], Bd32[k]}; },
                           [&](int k, const Pb& g) {
                             const float pk = g.r + beta * (g.p - omega * g.q);
                             p[k] = pk;
                             ph[k] = pk * g.d;
                           });
          } else {
            for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) ph[k] = p[k] * Bd32[k];
          }
          first = false;
          cl.sync();
          float rvt[1] = {0.0f};
          struct Sv { St s; float rh; };
          for_points<Sv>(k0, k1, [&](int k) { return Sv{st_load(k, ph), rh[k]}; },
                         [&](int k, const Sv& g) {
                           const float vk = st_eval(g.s);
                           q[k] = vk;
                           rvt[0] += g.rh * vk;
                         });
          double rv[1];
          cl_sum<float, 1>(cl, rvt, rv, sh, buf);
          if (rv[0] == 0.0 || !isfinite(rv[0])) break;
          alpha = (float)(rho / rv[0]);
          struct Ss { float r, q, d; };
          for_points<Ss>(k0, k1, [&](int k) { return Ss{r[k], q[k], Bd32[k]}; },
                         [&](int k, const Ss& g) {
                           const float sk = g.r - alpha * g.q;
                           sv[k] = sk;
                           shh[k] = sk * g.d;
                         });
          cl.sync();
          float tst[2] = {0.0f, 0.0f};
          struct Tv { St s; float sv; };
          for_points<Tv>(k0, k1, [&](int k) { return Tv{st_load(k, shh), sv[k]}; },
                         [&](int k, const Tv& g) {
                           const float t = st_eval(g.s);
                           tv[k] = t;
                           tst[0] += t * g.sv;
                           tst[1] += t * t;
                         });
          double ts[2];
          cl_sum<float, 2>(cl, tst, ts, sh, buf);
          omega = ts[1] > 0.0 ? (float)(ts[0] / ts[1]) : 0.0f;
          float rrt[2] = {0.0f, 0.0f};
          struct Xu { float x, ph, shh, sv, tv, rh; };
          for_points<Xu>(k0, k1,
                         [&](int k) { return Xu{ev[k], ph[k], shh[k], sv[k], tv[k], rh[k]}; },
                         [&](int k, const Xu& g) {
                           ev[k] = g.x + alpha * g.ph + omega * g.shh;
                           const float rk = g.sv - omega * g.tv;
                           r[k] = rk;
                           rrt[0] += g.rh * rk;
                           rrt[1] += rk * rk;
                         });
          double rr2[2];
          cl_sum<float, 2>(cl, rrt, rr2, sh, buf);
          rho_prev = rho;
          rho = rr2[0];
          rr = rr2[1];
          ++it;
          if (rr > tol2 && (omega == 0.0f || rho == 0.0)) break;
        }
      }
      my_iters += it;
      // x += sigma e (CG: e = S^-1 e^)
      for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const float e = cgm ? ev[k] * Bs32[5 * ldb + k] : ev[k];
        x[k] = fma(sig, (double)e, x[k]);
      }
      cl.sync();
    }
  }
  const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    if (a.out.y_f64)
      static_cast<double*>(a.out.y)[oy + k] = x[k];
    else
      static_cast<float*>(a.out.y)[oy + k] = (float)x[k];
  }
  cl.sync();
}

__global__ void __launch_bounds__(KRY_THREADS, 2) k_krylov_queue_ir(const KryArgs* __restrict__ probs,
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
  void* ws = static_cast<char*>(ws_all) + (size_t)slot * ws_stride;
  cl_map(cl, sh);
  cl.sync();   // every CTA runs before remote stores into its shared memory
  int buf = 0;
  while (true) {
    if (crank == 0 && threadIdx.x == 0) next_item = (int)atomicAdd(counter, 1u);
    cl.sync();
    const int it = *cl.map_shared_rank(&next_item, 0);
    cl.sync();                        // rank 0 may overwrite next_item only after all read it
    if (it >= nitems) break;
    const KryArgs& a = probs[items[2 * it]];
    if (a.in.stop && *a.in.stop) continue;   // the same flag for every CTA of the cluster
    unsigned long long my_iters = 0;
    int my_status = 0;
    krylov_system_ir(a, cl, sh, buf, items[2 * it + 1], ws, my_iters, my_status);
    if (threadIdx.x == 0 && crank == 0) {
      if (my_iters) atomicAdd(a.iters, my_iters);
      if (my_status) atomicOr(a.status, my_status);
    }
  }
}

// Many problems (different grids and operators) in one persistent launch: a
// device work queue of items (problem, system), largest grids first; each
// cluster takes the next item from a global counter (rank 0 draws it and
// the other CTAs read it through distributed shared memory).  The Krylov
// iterations and status of an item go to its own problem's counters; items
// of a problem whose stop flag (in.stop) is set are skipped.
template <typename T>
__global__ void __launch_bounds__(KRY_THREADS, 2) k_krylov_queue(const KryArgs* __restrict__ probs,
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
  cl.sync();   // every CTA runs before remote stores into its shared memory
  int buf = 0;
  while (true) {
    if (crank == 0 && threadIdx.x == 0) next_item = (int)atomicAdd(counter, 1u);
    cl.sync();
    const int it = *cl.map_shared_rank(&next_item, 0);
    cl.sync();                        // rank 0 may overwrite next_item only after all read it
    if (it >= nitems) break;
    const KryArgs& a = probs[items[2 * it]];
    if (a.in.stop && *a.in.stop) continue;   // the same flag for every CTA of the cluster
    unsigned long long my_iters = 0;
    int my_status = 0;
    krylov_system<T>(a, cl, sh, buf, items[2 * it + 1], ws, my_iters, my_status);
    if (threadIdx.x == 0 && crank == 0) {
      if (my_iters) atomicAdd(a.iters, my_iters);
      if (my_status) atomicOr(a.status, my_status);
    }
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
  const size_t ld = (size_t)op->n + 2 * op->mx;
  // time-dependent operators: one plan per fine step of the time grid, back to back
  const size_t steps = op->kind == 3 ? (size_t)op->nJ * (op->stepper ? 2 : 1) : 1;
  if ((s = dev_alloc(op->ctx, pl->b64, sizeof(double) * 6 * ld * steps))) return s;
  if ((s = dev_alloc(op->ctx, pl->b32, sizeof(float) * 6 * ld * steps))) return s;
  cudaMemsetAsync(pl->b64.ptr, 0, pl->b64.bytes, c->stream);
  cudaMemsetAsync(pl->b32.ptr, 0, pl->b32.bytes, c->stream);
  const dim3 pgrid((op->n + 255) / 256, (unsigned)steps);
  k_stencil_plan<<<pgrid, 256, 0, c->stream>>>(
      op->mx, op->my, dt, adjoint, op->a64[0].as<double>(), op->a64[1].as<double>(),
      op->a64[2].as<double>(), op->a64[3].as<double>(), op->a64[4].as<double>(),
      pl->b64.as<double>(), pl->b32.as<float>());
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_err(c, e, "k_stencil_plan");
  if (op->symmetric) {
    if ((s = dev_alloc(op->ctx, pl->bs64, sizeof(double) * 7 * ld * steps))) return s;
    if ((s = dev_alloc(op->ctx, pl->bs32, sizeof(float) * 7 * ld * steps))) return s;
    cudaMemsetAsync(pl->bs64.ptr, 0, pl->bs64.bytes, c->stream);
    cudaMemsetAsync(pl->bs32.ptr, 0, pl->bs32.bytes, c->stream);
    k_stencil_plan_scaled<<<pgrid, 256, 0, c->stream>>>(
        op->mx, op->my, pl->b64.as<double>(), pl->bs64.as<double>(), pl->bs32.as<float>());
    e = cudaGetLastError();
    if (e) return cuda_err(c, e, "k_stencil_plan_scaled");
  }
  // published only once filled: other contexts (a server's) may use it at once
  e = cudaStreamSynchronize(c->stream);
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

// Launch shape of k_krylov for a batch: the cluster size with the most CTAs in
// flight (the largest on a tie: fewest points per CTA, shortest iteration;
// clusters of 16 fit once per GPC, smaller ones pack the GPCs more densely),
// with the workspaces of the clusters in flight within 96 MB so that the
// Krylov vectors stay L2-resident (129 MB L2).
// Shared-memory bytes of the staging tile of a CTA for cc CTAs per cluster:
// its rows and one halo row on each side, plus 16 bytes of alignment slack
// (0 when staging is off or the tile would not leave two CTAs per SM).
static size_t krylov_stage_bytes(Ctx* c, const Operator* op, int prec, int cc) {
  if (prec != 1 || c->p_krylov_stage != 1) return 0;
  const long rows_per = (op->my + cc - 1) / cc;
  const size_t bytes = (((size_t)(rows_per + 2) * op->mx * 4 + 16) + 15) & ~(size_t)15;
  return bytes <= KRY_STAGE_MAX ? bytes : 0;
}

static void krylov_shape(Ctx* c, const Operator* op, int prec, int nvec, int nsys,
                         void (*kern)(KryArgs), int* cs_out, int* ncl_out,
                         size_t* stage_out = nullptr) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(KRY_THREADS);
  const int cs_max = cluster_size_for(op->mx, op->my);
  const size_t es_ = prec == 0 ? 8 : 4;
  const size_t ws_one = (size_t)nvec * ((size_t)op->n + 2 * op->mx) * es_;
  const int ws_cap = (int)std::max<size_t>(1, ((size_t)96 << 20) / ws_one);
  int cs = cs_max, nclusters = 1;
  long best = -1;
  for (int cc = cs_max; cc >= 1 && cc >= cs_max / 4; cc /= 2) {
    if (c->p_krylov_cluster > 0 && cc != std::min(c->p_krylov_cluster, cs_max)) continue;
    if ((op->my + cc - 1) / cc * (cc - 1) >= op->my && cc > 1) continue;   // every CTA owns rows
    attr[0].val.clusterDim.x = cc;
    cfg.gridDim = dim3(cc);
    cfg.dynamicSmemBytes = stage_out ? krylov_stage_bytes(c, op, prec, cc) : 0;
    int maxc = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg);
    if (e || maxc < 1) { cudaGetLastError(); maxc = std::max(1, c->num_sms / cc); }
    const int ncl = std::min(std::min(nsys, maxc), ws_cap);
    const long ctas = (long)ncl * cc;
    if (ctas > best) { best = ctas; cs = cc; nclusters = ncl; }
  }
  *cs_out = cs;
  *ncl_out = nclusters;
  if (stage_out) *stage_out = krylov_stage_bytes(c, op, prec, cs);
}

lrp_status krylov_f32_correction(Ctx* c, Operator* op, StencilPlan* plan, int nsys, KryArgs& a) {
  auto kern = (void (*)(KryArgs))k_krylov<float>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (!e) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KRY_STAGE_MAX);
  if (e) return cuda_err(c, e, "krylov kernel attributes");
  const int nvec = (int)krylov_queue_nvec(a.bicg);
  int cs = 1, ncl = 1;
  size_t stage = 0;
  krylov_shape(c, op, 1, nvec, nsys, kern, &cs, &ncl, &stage);
  a.stage = stage > 0;
  const size_t need = (size_t)ncl * nvec * ((size_t)op->n + 2 * op->mx) * 4;
  lrp_status s;
  if (c->kws.bytes < need)
    if ((s = dev_alloc(c, c->kws, need))) return s;
  a.B = stencil_B(plan, op, 1);
  a.Bs = stencil_Bs(plan, op, 1);
  a.ws = c->kws.ptr;
  a.nvec = nvec;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(KRY_THREADS);
  cfg.gridDim = dim3(ncl * cs);
  cfg.dynamicSmemBytes = stage;
  cfg.stream = c->stream;
  cudaEvent_t ev = nullptr;
  timer_begin(c, "propagate_f32", &ev);
  e = cudaLaunchKernelEx(&cfg, kern, a);
  timer_end(c, "propagate_f32", ev);
  if (e) return cuda_err(c, e, "k_krylov launch");
  return LRP_OK;
}

lrp_status stencil_propagate(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys,
                             int prec, const PropIn& in, const PropOut& out, const PropSrc& src) {
  if (nsys <= 0) return LRP_OK;
  // SDIRK steps solve with B = I + gamma dt A: the plan and the kernel's dt
  // are gamma dt (the source of a stage enters as gamma dt f); they run on
  // the kernel with its Krylov vectors in global memory
  const bool sdirk = op->stepper != 0;
  const StepCoef sc = sdirk ? step_coefficients(op->stepper) : StepCoef{1.0, 0, 0, 0, 0, 0};
  const double dtp = sdirk ? dt * sc.gamma : dt;
  StencilPlan* plan = nullptr;
  lrp_status s = stencil_plan(c, op, dtp, adjoint, &plan);
  if (s) return s;
  const int bicg = op->symmetric ? 0 : 1;
  const int nvec = (int)krylov_queue_nvec(bicg) + (sdirk ? 2 : 0);
  // time-dependent operators (kind 3) run on the kernel with its vectors in
  // global memory, every step on its own plan
  const bool td = op->kind == 3;
  if (td && adjoint && src.Q > 0) return set_err(c, LRP_EINVAL, "the adjoint acts on the linear part");
  if (td && !in.map && !out.map && !src.map) {
    const long last = (long)in.interval0 + (long)(nsys - 1) / std::max(in.ncol, 1);
    if (in.interval0 < 0 || (last + 1) * M > op->nJ)
      return set_err(c, LRP_EINVAL, "time-dependent operator: steps beyond its time grid");
  }
  const bool block = !sdirk && !td && stencil_block_applies(c, op, prec, nsys, M, src.Q);
  if (!block && stencil_refine_applies(c, op, prec, nsys)) {
    c->bk_last[0] = c->bk_last[1] = c->bk_last[2] = 0;
    c->oc_last[0] = c->oc_last[1] = c->oc_last[2] = 0;
    return stencil_propagate_refine(c, op, plan, M, nsys, in, out, src, adjoint);
  }
  if (!block) c->bk_last[0] = c->bk_last[1] = c->bk_last[2] = 0;
  const bool onchip = !sdirk && !block && stencil_onchip_applies(c, op, prec, nsys);
  if (!onchip) c->oc_last[0] = c->oc_last[1] = c->oc_last[2] = 0;
  using KrK = void (*)(KryArgs);
  auto kern = prec == 0 ? (sdirk ? (td ? (KrK)k_krylov<double, true, true> : (KrK)k_krylov<double, true>)
                           : td ? (KrK)k_krylov<double, false, true> : (KrK)k_krylov<double>)
                        : (sdirk ? (td ? (KrK)k_krylov<float, true, true> : (KrK)k_krylov<float, true>)
                           : td ? (KrK)k_krylov<float, false, true> : (KrK)k_krylov<float>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (!e && prec == 1)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KRY_STAGE_MAX);
  if (e) return cuda_err(c, e, "krylov kernel attributes");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(KRY_THREADS);
  cfg.stream = c->stream;
  int cs = 1, nclusters = 1;
  size_t stage = 0;
  krylov_shape(c, op, prec, nvec, nsys, kern, &cs, &nclusters, &stage);
  attr[0].val.clusterDim.x = cs;
  cfg.gridDim = dim3(nclusters * cs);
  cfg.dynamicSmemBytes = stage;
  const size_t es = prec == 0 ? 8 : 4;
  const size_t need = (size_t)nclusters * nvec * ((size_t)op->n + 2 * op->mx) * es;
  if (!onchip && !block && c->kws.bytes < need)
    if ((s = dev_alloc(c, c->kws, need))) return s;
  if (!c->kstat.ptr)
    if ((s = dev_alloc(c, c->kstat, 16))) return s;
  cudaMemsetAsync(c->kstat.ptr, 0, 16, c->stream);
  KryArgs a{};
  a.mx = op->mx;
  a.my = op->my;
  a.n = op->n;
  a.M = M;
  a.nsys = nsys;
  a.bicg = bicg;
  a.dt = dtp;
  a.stepper = op->stepper;
  a.su = sc.su;
  a.s1 = sc.s1;
  a.bu = sc.bu;
  a.b1 = sc.b1;
  a.b2 = sc.b2;
  a.rtol = prec == 0 ? op->rtol64 : op->rtol32;
  a.max_iter = op->max_iter;
  a.B = stencil_B(plan, op, prec);
  a.Bs = stencil_Bs(plan, op, prec);
  if (td) {
    a.b_step = 6 * ((long)op->n + 2 * op->mx);
    a.bs_step = 7 * ((long)op->n + 2 * op->mx);
    a.nJ = op->nJ;
    a.adj = adjoint;
    if (sdirk && adjoint) {
      // the transposed step map: W2 = B2^-T v, W1 = B1^-T (b1 v + b2 s1 W2),
      // v' = bu v + b2 su W2 + W1 (the kernel's stage body with these coefficients)
      a.su = sc.b1;
      a.s1 = sc.b2 * sc.s1;
      a.b1 = sc.b2 * sc.su;
      a.b2 = 1.0;
    }
  }
  a.ws = c->kws.ptr;
  a.nvec = nvec;
  a.in = in;
  a.out = out;
  a.src = src;
  a.iters = reinterpret_cast<unsigned long long*>(c->kstat.ptr);
  a.status = reinterpret_cast<int*>(static_cast<char*>(c->kstat.ptr) + 8);
  a.stage = stage > 0;
  if (block) {
    if ((s = stencil_propagate_block(c, op, plan, M, nsys, prec, a))) return s;
  } else if (onchip) {
    if ((s = stencil_propagate_onchip(c, op, plan, M, nsys, prec, a))) return s;
  } else {
    const char* fam = prec == 0 ? "propagate_f64" : "propagate_f32";
    cudaEvent_t ev = nullptr;
    timer_begin(c, fam, &ev);
    e = cudaLaunchKernelEx(&cfg, kern, a);
    timer_end(c, fam, ev);
    if (e) return cuda_err(c, e, "k_krylov launch");
  }
  unsigned long long hs[2] = {0, 0};
  e = cudaMemcpyAsync(hs, c->kstat.ptr, 16, cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "k_krylov");
  op->krylov_iters += hs[0];
  int st = (int)(hs[1] & 0xffffffffu);
  if (st & 4) return set_err(c, LRP_ETIMEOUT, "a bounded wait of a 2D propagator expired");
  if (st & 2) return set_err(c, LRP_EBREAKDOWN, "Krylov breakdown in a 2D propagation");
  if (st & 1) return set_err(c, LRP_ENOTCONV, "Krylov iteration cap reached in a 2D propagation");
  return LRP_OK;
}

// ---- work-queue launches (batched problems of uneven size) -----------------
size_t krylov_queue_nvec(int bicg) { return bicg ? 9 : 4; }

const void* stencil_B(const StencilPlan* pl, const Operator* op, int prec) {
  return prec == 0 ? (const void*)(pl->b64.as<double>() + op->mx)
                   : (const void*)(pl->b32.as<float>() + op->mx);
}

const void* stencil_Bs(const StencilPlan* pl, const Operator* op, int prec) {
  if (!op->symmetric) return nullptr;
  return prec == 0 ? (const void*)(pl->bs64.as<double>() + op->mx)
                   : (const void*)(pl->bs32.as<float>() + op->mx);
}

using QueueKern = void (*)(const KryArgs*, const int*, int, unsigned int*, void*, size_t);
static QueueKern queue_kernel(int prec) {
  return prec == 0 ? (QueueKern)k_krylov_queue<double>
       : prec == 1 ? (QueueKern)k_krylov_queue<float> : (QueueKern)k_krylov_queue_ir;
}

size_t krylov_queue_ir_bytes(int maxld) { return (size_t)maxld * (2 * 8 + 10 * 4); }

int krylov_queue_clusters(Ctx* c, int prec, int cs) {
  auto kern = queue_kernel(prec);
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
  auto kern = queue_kernel(prec);
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
  const char* fam = prec == 1 ? "propagate_f32" : "propagate_f64";
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

static lrp_status make_stencil5_td(Ctx* c, int mx, int my, int nJ, int stepper, const double* C,
                                   const double* W, const double* E, const double* S,
                                   const double* N, lrp_operator** out) {
  const long rows = (long)nJ * (stepper ? 2 : 1);
  if (rows > 65535) return set_err(c, LRP_EINVAL, "time-dependent operators take at most 65535 coefficient rows");
  if ((long)mx * my * rows > (1L << 28))
    return set_err(c, LRP_EINVAL, "time-dependent operator too large (mx my rows > 2^28)");
  cudaSetDevice(c->device);
  const int n = mx * my;
  auto* op = new lrp_operator();
  op->ctx = c;
  ctx_retain(c);
  op->kind = 3;
  op->mx = mx;
  op->my = my;
  op->n = n;
  op->nJ = nJ;
  op->stepper = stepper;
  const double* src[5] = {C, W, E, S, N};
  const size_t cnt = (size_t)rows * n;
  std::vector<double> h[5];
  for (int k = 0; k < 5; ++k) {
    h[k].resize(cnt);
    cudaError_t e = cudaMemcpy(h[k].data(), src[k], sizeof(double) * cnt, cudaMemcpyDefault);
    if (e) { delete op; return cuda_err(c, e, "stencil read"); }
    lrp_status s = dev_alloc(c, op->a64[k], sizeof(double) * cnt);
    if (s) { delete op; return s; }
    e = cudaMemcpyAsync(op->a64[k].ptr, h[k].data(), sizeof(double) * cnt, cudaMemcpyHostToDevice,
                        c->stream);
    if (e) { delete op; return cuda_err(c, e, "stencil upload"); }
  }
  // CG when every row's stencil is symmetric, else BiCGStab
  bool sym = true;
  for (size_t J = 0; J < (size_t)rows && sym; ++J) {
    const size_t o = J * n;
    for (int p = 0; p < n && sym; ++p) {
      int ix = p % mx, iy = p / mx;
      if (ix > 0 && h[1][o + p] != h[2][o + p - 1]) sym = false;
      if (iy > 0 && h[3][o + p] != h[4][o + p - mx]) sym = false;
    }
  }
  op->symmetric = sym;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) { delete op; return cuda_err(c, e, "stencil upload"); }
  *out = op;
  return LRP_OK;
}

extern "C" lrp_status lrp_operator_stencil5_td(lrp_ctx* cc, int mx, int my, int nJ, const double* C,
                                               const double* W, const double* E, const double* S,
                                               const double* N, lrp_operator** out) {
  Ctx* c = reinterpret_cast<Ctx*>(cc);
  if (!c || !out || !C || !W || !E || !S || !N || mx < 1 || my < 1 || nJ < 1) return LRP_EINVAL;
  return make_stencil5_td(c, mx, my, nJ, 0, C, W, E, S, N, out);
}

extern "C" lrp_status lrp_operator_stencil5_td_sdirk(lrp_ctx* cc, int mx, int my, int nJ,
                                                     int stepper, const double* C, const double* W,
                                                     const double* E, const double* S,
                                                     const double* N, lrp_operator** out) {
  Ctx* c = reinterpret_cast<Ctx*>(cc);
  if (!c || !out || !C || !W || !E || !S || !N || mx < 1 || my < 1 || nJ < 1) return LRP_EINVAL;
  if (stepper != LRP_STEP_SDIRK2 && stepper != LRP_STEP_SDIRK2_L)
    return set_err(c, LRP_EINVAL, "stage-sampled operators take an SDIRK stepper");
  return make_stencil5_td(c, mx, my, nJ, stepper, C, W, E, S, N, out);
}
