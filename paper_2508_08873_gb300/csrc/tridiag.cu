// Batched backward-Euler propagator for tridiagonal operators (the fine solver
// F_i, its linear part F_i' and adjoint F_i'^* of Sec. 2 / Sec. 4).
//
// Every implicit-Euler step solves (I + dt A) x_{j+1} = x_j + dt f(t_{j+1}).
// The matrix is the same for every step, interval and right-hand side, so it is
// factored once per (dt, direction) into a partitioned form and the per-step
// work is pure substitution:
//   * the n rows are cut into P chunks of m rows; the last row of each chunk is
//     an interface unknown y_t, the other m-1 rows are interior;
//   * interior rows: Thomas forward/backward substitution with precomputed
//     multipliers, giving g = A_int^{-1} d, and the precomputed "spikes" p, q
//     with x_int = g - p y_{t-1} - q y_t;
//   * the interface unknowns satisfy a P x P tridiagonal system whose matrix is
//     fixed; it is solved by parallel cyclic reduction with precomputed
//     elimination factors (log2 P levels of r_t -= k1 r_{t-s} + k2 r_{t+s}).
// One thread owns one chunk and keeps its m state values in registers for all
// M steps; only 2 values per thread cross shared memory per PCR level.  The
// factorisation is Gaussian elimination without pivoting, valid for the
// diagonally dominant I + dt A of the parabolic operators targeted here.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tri_common.cuh"

namespace lrp {

// ---------------------------------------------------------------------------
// Factorisation (one CTA of P threads, FP64).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_tri_factor(const double* __restrict__ lo, const double* __restrict__ di,
                             const double* __restrict__ up, int n, double dt, int adj, int m,
                             int P, int L, double* __restrict__ coef, float* __restrict__ coef32,
                             double* __restrict__ pcr, float* __restrict__ pcr32,
                             int* __restrict__ status) {
  extern __shared__ double sh[];
  double* sa = sh;            // alpha
  double* sb = sa + P;        // beta
  double* sc = sb + P;        // gamma
  double* sp0 = sc + P;       // p_t[0]
  double* sq0 = sp0 + P;      // q_t[0]
  const int t = threadIdx.x;
  const int mi = m - 1;       // interior rows
  const size_t MP = (size_t)m * P;
  double* cl = coef;
  double* cinv = coef + MP;
  double* cu = coef + 2 * MP;
  double* cp = coef + 3 * MP;
  double* cq = coef + 4 * MP;
  int bad = 0;
  double pl = 0.0, ql = 0.0, aE = 0.0, bE = 1.0, cE = 0.0;
  if (t < P) {
    const int r0 = t * m;
    // interior block: rows r0 .. r0+mi-1; eliminate without pivoting
    double piv = b_di(di, n, dt, r0);
    if (!(fabs(piv) > 0.0) || !isfinite(piv)) bad = 1;
    cl[t] = 0.0;
    cinv[t] = 1.0 / piv;
    for (int i = 1; i < mi; ++i) {
      int r = r0 + i;
      double mult = b_lo(lo, up, n, dt, adj, r) / piv;
      double bu_prev = b_up(lo, up, n, dt, adj, r - 1);
      piv = b_di(di, n, dt, r) - mult * bu_prev;
      if (!(fabs(piv) > 0.0) || !isfinite(piv)) bad = 1;
      cl[(size_t)i * P + t] = mult;
      cinv[(size_t)i * P + t] = 1.0 / piv;
    }
    for (int i = 0; i < mi; ++i)
      cu[(size_t)i * P + t] = (i < mi - 1) ? b_up(lo, up, n, dt, adj, r0 + i) * cinv[(size_t)i * P + t] : 0.0;
    // spikes: A_int p = bl(r0) e_0, A_int q = bu(r0+mi-1) e_{mi-1}
    const double left = b_lo(lo, up, n, dt, adj, r0);
    const double right = b_up(lo, up, n, dt, adj, r0 + mi - 1);
    double fp = left, fq = 0.0;           // forward elimination of both RHS
    cp[t] = fp;
    cq[t] = (mi == 1) ? right : 0.0;
    for (int i = 1; i < mi; ++i) {
      double mult = cl[(size_t)i * P + t];
      fp = 0.0 - mult * fp;
      fq = ((i == mi - 1) ? right : 0.0) - mult * fq;
      cp[(size_t)i * P + t] = fp;
      cq[(size_t)i * P + t] = fq;
    }
    double gp = 0.0, gq = 0.0;            // backward substitution
    for (int i = mi - 1; i >= 0; --i) {
      size_t k = (size_t)i * P + t;
      gp = cp[k] * cinv[k] - cu[k] * gp;
      gq = cq[k] * cinv[k] - cu[k] * gq;
      cp[k] = gp;
      cq[k] = gq;
    }
    pl = cp[(size_t)(mi - 1) * P + t];
    ql = cq[(size_t)(mi - 1) * P + t];
    const int e = r0 + mi;                // interface row
    aE = b_lo(lo, up, n, dt, adj, e);
    bE = b_di(di, n, dt, e);
    cE = b_up(lo, up, n, dt, adj, e);
    size_t k = (size_t)mi * P + t;
    cl[k] = aE;
    cinv[k] = bE;
    cu[k] = cE;
    cp[k] = 0.0;
    cq[k] = 0.0;
    sp0[t] = cp[t];
    sq0[t] = cq[t];
  }
  __syncthreads();
  if (t < P) {
    double pn = (t + 1 < P) ? sp0[t + 1] : 0.0;
    double qn = (t + 1 < P) ? sq0[t + 1] : 0.0;
    sa[t] = -aE * pl;
    sb[t] = bE - aE * ql - cE * pn;
    sc[t] = -cE * qn;
  }
  __syncthreads();
  // parallel cyclic reduction of the interface system: precompute factors
  for (int lev = 0, s = 1; lev < L; ++lev, s <<= 1) {
    double a = 0, b = 1, c = 0, k1 = 0, k2 = 0, na = 0, nb = 1, nc = 0;
    if (t < P) {
      a = sa[t]; b = sb[t]; c = sc[t];
      double a1 = 0, b1 = 1, c1 = 0, a2 = 0, b2 = 1, c2 = 0;
      if (t - s >= 0) { a1 = sa[t - s]; b1 = sb[t - s]; c1 = sc[t - s]; }
      if (t + s < P) { a2 = sa[t + s]; b2 = sb[t + s]; c2 = sc[t + s]; }
      k1 = (t - s >= 0) ? a / b1 : 0.0;
      k2 = (t + s < P) ? c / b2 : 0.0;
      na = -k1 * a1;
      nc = -k2 * c2;
      nb = b - k1 * c1 - k2 * a2;
      if (!(fabs(nb) > 0.0) || !isfinite(nb)) bad = 1;
      pcr[(size_t)lev * P + t] = k1;
      pcr[(size_t)(L + lev) * P + t] = k2;
    }
    __syncthreads();
    if (t < P) { sa[t] = na; sb[t] = nb; sc[t] = nc; }
    __syncthreads();
  }
  if (t < P) {
    if (!(fabs(sb[t]) > 0.0) || !isfinite(sb[t])) bad = 1;
    pcr[(size_t)(2 * L) * P + t] = 1.0 / sb[t];
  }
  __syncthreads();
  // FP32 copies
  for (size_t k = t; k < 5 * MP; k += blockDim.x) coef32[k] = (float)coef[k];
  for (size_t k = t; k < (size_t)(2 * L + 1) * P; k += blockDim.x) pcr32[k] = (float)pcr[k];
  if (bad) atomicOr(status, 1);
}

// ---------------------------------------------------------------------------
// Propagation kernel.  blockDim.x = P * G: G systems per CTA, one chunk per
// thread.  Systems are visited grid-stride; all threads take part in every
// barrier (inactive slots compute on zeros and do not store).
// ---------------------------------------------------------------------------
struct TriKArgs {
  int n, P, L, G, M, nsys;
  double dt;
  // two-stage SDIRK step (stepper != 0): with B = I + gamma dt A (the plan's
  // matrix), U1 = B^-1 u, U2 = B^-1 (su u + s1 U1), u_new = bu u + b1 U1 + b2 U2
  int stepper;
  double su, s1, bu, b1, b2;
  const void* coef;
  const void* pcr;
  PropIn in;
  PropOut out;
  PropSrc src;
};

// At most 512 threads per CTA, so that up to 128 registers per thread keep the
// whole chunk state (MM values) in registers.
template <typename T, int MM, bool SDIRK = false>
__global__ void __launch_bounds__(512) k_tri_propagate(TriKArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_coef = reinterpret_cast<T*>(smem_raw);                 // [5][MM][P]
  const int P = a.P, L = a.L, G = a.G;
  T* s_pcr = s_coef + 5 * MM * P;                             // [2L+1][P]
  T* s_x = s_pcr + (2 * L + 1) * P;                           // [G][3][P]
  const int nco = 5 * MM * P, npc = (2 * L + 1) * P;
  const T* gco = static_cast<const T*>(a.coef);
  const T* gpc = static_cast<const T*>(a.pcr);
  for (int k = threadIdx.x; k < nco; k += blockDim.x) s_coef[k] = gco[k];
  for (int k = threadIdx.x; k < npc; k += blockDim.x) s_pcr[k] = gpc[k];
  __syncthreads();

  const int t = threadIdx.x % P;
  const int gslot = threadIdx.x / P;
  T* xb = s_x + (size_t)gslot * 3 * P;
  const T* cl = s_coef;
  const T* ci = s_coef + MM * P;
  const T* cu = s_coef + 2 * MM * P;
  const T* cp = s_coef + 3 * MM * P;
  const T* cq = s_coef + 4 * MM * P;
  const T dt = (T)a.dt;
  const int n = a.n;
  const int r0 = t * MM;

  for (int base = blockIdx.x * G; base < a.nsys; base += gridDim.x * G) {
    const int sys = base + gslot;
    const bool active = sys < a.nsys;
    T x[MM];
    // ---- load the initial vector ---------------------------------------
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      int r = r0 + i;
      T v = T(0);
      if (active && r < n) {
        if (a.in.gen) {
          v = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                       (uint32_t)(sys % a.in.ncol), (uint32_t)r);
        } else if (a.in.x == nullptr) {
          v = T(0);                                   // zero initial value (b_i = F_i 0)
        } else if (a.in.x_f64) {
          v = (T) static_cast<const double*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
        } else {
          v = (T) static_cast<const float*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
        }
      }
      x[i] = v;
    }
    const double* csys = (active && a.src.Q > 0)
        ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
    const double* gsys = (active && a.src.Q > 0 && a.src.map)
        ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
    // one solve with B = I + dt A (the plan's matrix), in place on x
    auto solve = [&](T (&x)[MM]) {
      // interior forward elimination and back substitution: x[0..MM-2] := g
#pragma unroll
      for (int i = 1; i < MM - 1; ++i) x[i] -= cl[i * P + t] * x[i - 1];
      x[MM - 2] *= ci[(MM - 2) * P + t];
#pragma unroll
      for (int i = MM - 3; i >= 0; --i) x[i] = x[i] * ci[i * P + t] - cu[i * P + t] * x[i + 1];
      // interface right-hand side needs g_{t+1}[0]
      xb[2 * P + t] = x[0];
      __syncthreads();
      T gnext = (t + 1 < P) ? xb[2 * P + t + 1] : T(0);
      T r = x[MM - 1] - cl[(MM - 1) * P + t] * x[MM - 2] - cu[(MM - 1) * P + t] * gnext;
      // parallel cyclic reduction with precomputed factors
      int buf = 0;
      for (int lev = 0, s = 1; lev < L; ++lev, s <<= 1) {
        xb[buf * P + t] = r;
        __syncthreads();
        T rm = (t - s >= 0) ? xb[buf * P + t - s] : T(0);
        T rp = (t + s < P) ? xb[buf * P + t + s] : T(0);
        r = r - s_pcr[lev * P + t] * rm - s_pcr[(L + lev) * P + t] * rp;
        buf ^= 1;
      }
      T y = r * s_pcr[2 * L * P + t];
      xb[buf * P + t] = y;
      __syncthreads();
      T yl = (t > 0) ? xb[buf * P + t - 1] : T(0);
      // interior correction with the spikes
#pragma unroll
      for (int i = 0; i < MM - 1; ++i) x[i] = x[i] - cp[i * P + t] * yl - cq[i * P + t] * y;
      x[MM - 1] = y;
    };
    // ---- M time steps ------------------------------------------------------
    for (int j = 0; j < a.M; ++j) {
      if constexpr (!SDIRK) {
        // backward Euler with the source sampled at the step end
        if (csys) {
          for (int q = 0; q < a.src.Q; ++q) {
            T cq_ = dt * (T)csys[(size_t)j * a.src.Q + q];
            const double* gq = gsys + (size_t)q * n;
#pragma unroll
            for (int i = 0; i < MM; ++i) {
              int r = r0 + i;
              if (r < n) x[i] += cq_ * (T)gq[r];
            }
          }
        }
        solve(x);
      } else {
        // two-stage SDIRK, both stages with the same matrix B = I + gamma dt A;
        // the source of stage i, sampled at its stage time (two samples per
        // step), enters its right-hand side as gamma dt f_i (dt here is the
        // plan's gamma dt)
        auto add_source = [&](int stage) {
          if (!csys) return;
          for (int q = 0; q < a.src.Q; ++q) {
            T cq_ = dt * (T)csys[((size_t)j * 2 + stage) * a.src.Q + q];
            const double* gq = gsys + (size_t)q * n;
#pragma unroll
            for (int i = 0; i < MM; ++i) {
              int r = r0 + i;
              if (r < n) x[i] += cq_ * (T)gq[r];
            }
          }
        };
        T u[MM], u1[MM];
#pragma unroll
        for (int i = 0; i < MM; ++i) u[i] = x[i];
        add_source(0);
        solve(x);
#pragma unroll
        for (int i = 0; i < MM; ++i) {
          u1[i] = x[i];
          x[i] = (T)a.su * u[i] + (T)a.s1 * x[i];
        }
        add_source(1);
        solve(x);
#pragma unroll
        for (int i = 0; i < MM; ++i) x[i] = (T)a.bu * u[i] + (T)a.b1 * u1[i] + (T)a.b2 * x[i];
      }
    }
    // ---- store -------------------------------------------------------------
    if (active) {
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        int r = r0 + i;
        if (r < n) {
          const long o = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys) + r;
          if (a.out.y_f64)
            static_cast<double*>(a.out.y)[o] = (double)x[i];
          else
            static_cast<float*>(a.out.y)[o] = (float)x[i];
        }
      }
    }
    __syncthreads();
  }
}

// Register-resident variant: every thread keeps its chunk's factors (5 MM
// values) and its PCR factors in registers for the whole launch and advances
// SPT systems at once, so a step reads no factors from shared memory (the
// FP32 kernel above is bound by shared-memory bandwidth: 5 loads per
// row-step) and one set of barriers serves SPT systems.  FP32, MM = 16.
template <typename T, int MM, int LMAX, int SPT>
__global__ void __launch_bounds__(256) k_tri_propagate_rc(TriKArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = a.P, L = a.L;
  T* xb = reinterpret_cast<T*>(smem_raw);                  // [SPT][3][P]
  const int t = threadIdx.x;
  const T* gco = static_cast<const T*>(a.coef);
  const T* gpc = static_cast<const T*>(a.pcr);
  T cl[MM], ci[MM], cu[MM], cp[MM], cq[MM], k1[LMAX], k2[LMAX];
#pragma unroll
  for (int i = 0; i < MM; ++i) {
    cl[i] = gco[(size_t)(0 * MM + i) * P + t];
    ci[i] = gco[(size_t)(1 * MM + i) * P + t];
    cu[i] = gco[(size_t)(2 * MM + i) * P + t];
    cp[i] = gco[(size_t)(3 * MM + i) * P + t];
    cq[i] = gco[(size_t)(4 * MM + i) * P + t];
  }
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    k1[l] = l < L ? gpc[(size_t)l * P + t] : T(0);
    k2[l] = l < L ? gpc[(size_t)(L + l) * P + t] : T(0);
  }
  const T dinv = gpc[(size_t)(2 * L) * P + t];
  const T dt = (T)a.dt;
  const int n = a.n;
  const int r0 = t * MM;
  for (int base = blockIdx.x * SPT; base < a.nsys; base += gridDim.x * SPT) {
    T x[SPT][MM];
    const double* csys[SPT];
    const double* gsys[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int sys = base + s;
      const bool active = sys < a.nsys;
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        int r = r0 + i;
        T v = T(0);
        if (active && r < n) {
          if (a.in.gen)
            v = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                         (uint32_t)(sys % a.in.ncol), (uint32_t)r);
          else if (a.in.x == nullptr)
            v = T(0);
          else if (a.in.x_f64)
            v = (T) static_cast<const double*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
          else
            v = (T) static_cast<const float*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
        }
        x[s][i] = v;
      }
      csys[s] = (active && a.src.Q > 0)
          ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
      gsys[s] = (active && a.src.Q > 0 && a.src.map)
          ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
    }
    for (int j = 0; j < a.M; ++j) {
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        if (csys[s]) {
          for (int q = 0; q < a.src.Q; ++q) {
            T cq_ = dt * (T)csys[s][(size_t)j * a.src.Q + q];
            const double* gq = gsys[s] + (size_t)q * n;
#pragma unroll
            for (int i = 0; i < MM; ++i)
              if (r0 + i < n) x[s][i] += cq_ * (T)gq[r0 + i];
          }
        }
      }
#pragma unroll
      for (int i = 1; i < MM - 1; ++i)
#pragma unroll
        for (int s = 0; s < SPT; ++s) x[s][i] -= cl[i] * x[s][i - 1];
#pragma unroll
      for (int s = 0; s < SPT; ++s) x[s][MM - 2] *= ci[MM - 2];
#pragma unroll
      for (int i = MM - 3; i >= 0; --i)
#pragma unroll
        for (int s = 0; s < SPT; ++s) x[s][i] = x[s][i] * ci[i] - cu[i] * x[s][i + 1];
#pragma unroll
      for (int s = 0; s < SPT; ++s) xb[(s * 3 + 2) * P + t] = x[s][0];
      __syncthreads();
      T r[SPT];
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        T gnext = (t + 1 < P) ? xb[(s * 3 + 2) * P + t + 1] : T(0);
        r[s] = x[s][MM - 1] - cl[MM - 1] * x[s][MM - 2] - cu[MM - 1] * gnext;
      }
      int buf = 0;
#pragma unroll
      for (int lev = 0; lev < LMAX; ++lev) {
        if (lev < L) {
          const int sh = 1 << lev;
#pragma unroll
          for (int s = 0; s < SPT; ++s) xb[(s * 3 + buf) * P + t] = r[s];
          __syncthreads();
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            T rm = (t - sh >= 0) ? xb[(s * 3 + buf) * P + t - sh] : T(0);
            T rp = (t + sh < P) ? xb[(s * 3 + buf) * P + t + sh] : T(0);
            r[s] = r[s] - k1[lev] * rm - k2[lev] * rp;
          }
          buf ^= 1;
        }
      }
      T y[SPT];
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        y[s] = r[s] * dinv;
        xb[(s * 3 + buf) * P + t] = y[s];
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        const T yl = (t > 0) ? xb[(s * 3 + buf) * P + t - 1] : T(0);
#pragma unroll
        for (int i = 0; i < MM - 1; ++i) x[s][i] = x[s][i] - cp[i] * yl - cq[i] * y[s];
        x[s][MM - 1] = y[s];
      }
    }
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int sys = base + s;
      if (sys >= a.nsys) continue;
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        int r = r0 + i;
        if (r < n) {
          const long o = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys) + r;
          if (a.out.y_f64)
            static_cast<double*>(a.out.y)[o] = (double)x[s][i];
          else
            static_cast<float*>(a.out.y)[o] = (float)x[s][i];
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int choose_m(int n) {
  if (n >= 1024) return 32;
  if (n >= 256) return 16;
  if (n >= 32) return 8;
  return 4;
}

lrp_status tri_get_plan(Ctx* c, Operator* op, double dt, int adjoint, TriPlan** out, int m_req) {
  std::lock_guard<std::mutex> plan_lock(op->plan_mu);
  for (auto& p : op->plans)
    if (p->dt == dt && p->adjoint == adjoint && (m_req == 0 ? p->m == choose_m(op->n) : p->m == m_req)) {
      *out = p.get();
      return LRP_OK;
    }
  auto pl = std::make_unique<TriPlan>();
  pl->dt = dt;
  pl->adjoint = adjoint;
  pl->n = op->n;
  pl->m = m_req ? m_req : choose_m(op->n);
  pl->P = (op->n + pl->m - 1) / pl->m;
  if (pl->P > 512) return set_err(c, LRP_EINVAL, "tridiagonal operator too large (n > 16384)");
  int L = 0;
  while ((1 << L) < pl->P) ++L;
  pl->levels = L;
  size_t MP = (size_t)pl->m * pl->P;
  lrp_status s;
  if ((s = dev_alloc(op->ctx, pl->coef64, 5 * MP * 8))) return s;
  if ((s = dev_alloc(op->ctx, pl->coef32, 5 * MP * 4))) return s;
  if ((s = dev_alloc(op->ctx, pl->pcr64, (size_t)(2 * L + 1) * pl->P * 8))) return s;
  if ((s = dev_alloc(op->ctx, pl->pcr32, (size_t)(2 * L + 1) * pl->P * 4))) return s;
  if ((s = dev_alloc(op->ctx, pl->status, sizeof(int)))) return s;
  cudaError_t e = cudaMemsetAsync(pl->status.ptr, 0, sizeof(int), c->stream);
  if (e) return cuda_err(c, e, "memset");
  int threads = ((pl->P + 31) / 32) * 32;
  k_tri_factor<<<1, threads, 5 * pl->P * sizeof(double), c->stream>>>(
      op->a64[0].as<double>(), op->a64[1].as<double>(), op->a64[2].as<double>(), op->n, dt,
      adjoint, pl->m, pl->P, L, pl->coef64.as<double>(), pl->coef32.as<float>(),
      pl->pcr64.as<double>(), pl->pcr32.as<float>(), pl->status.as<int>());
  e = cudaGetLastError();
  if (e) return cuda_err(c, e, "k_tri_factor launch");
  int st = 0;
  e = cudaMemcpyAsync(&st, pl->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "k_tri_factor");
  if (st) return set_err(c, LRP_EBREAKDOWN, "zero pivot in the tridiagonal factorisation");
  *out = pl.get();
  op->plans.push_back(std::move(pl));
  return LRP_OK;
}

template <typename T, int MM>
static lrp_status launch_tri(Ctx* c, TriPlan* plan, TriKArgs& a, bool sdirk = false) {
  const int P = a.P;
  // up to 256 threads per CTA: two CTAs share an SM, so one CTA's barriers
  // overlap the other's arithmetic (c->p_tri_group overrides, tuning)
  int Gmax = std::max(1, (c->p_tri_group > 0 ? c->p_tri_group * P : 256) / P);
  if (P * Gmax > 512) Gmax = std::max(1, 512 / P);
  // spread small batches over the SMs before packing systems into a CTA
  int G = std::max(1, std::min(Gmax, a.nsys / std::max(1, c->num_sms)));
  a.G = G;
  size_t smem = sizeof(T) * ((size_t)5 * MM * P + (size_t)(2 * a.L + 1) * P + (size_t)G * 3 * P);
  // SDIRK instantiations only for chunks of up to 8 rows (three chunk states
  // in registers); the backward-Euler kernels are unchanged
  auto kern = (sdirk && MM <= 8) ? k_tri_propagate<T, (MM <= 8 ? MM : 8), true> : k_tri_propagate<T, MM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return cuda_err(c, e, "tri smem attribute");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P * G, smem);
  if (e) return cuda_err(c, e, "tri occupancy");
  if (per_sm < 1) return set_err(c, LRP_EINVAL, "tridiagonal kernel does not fit on an SM");
  int groups = (a.nsys + G - 1) / G;
  int grid = std::min(groups, per_sm * c->num_sms);
  const char* fam = sizeof(T) == 8 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  kern<<<grid, P * G, smem, c->stream>>>(a);
  e = cudaGetLastError();
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_tri_propagate launch");
  return LRP_OK;
}

template <typename T, int MM, int LMAX, int SPT>
static lrp_status launch_tri_rc(Ctx* c, TriKArgs& a) {
  const int P = a.P;
  const int G = SPT;                  // systems per CTA
  a.G = 1;
  size_t smem = sizeof(T) * (size_t)SPT * 3 * P;
  auto kern = k_tri_propagate_rc<T, MM, LMAX, SPT>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P, smem);
  if (e) return cuda_err(c, e, "tri rc occupancy");
  if (per_sm < 1) return set_err(c, LRP_EINVAL, "tridiagonal kernel does not fit on an SM");
  int groups = (a.nsys + G - 1) / G;
  int grid = std::min(groups, per_sm * c->num_sms);
  const char* fam = sizeof(T) == 8 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  kern<<<grid, P, smem, c->stream>>>(a);
  e = cudaGetLastError();
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_tri_propagate_rc launch");
  return LRP_OK;
}

lrp_status tri_propagate(Ctx* c, Operator* op, TriPlan* plan, int M, int nsys, int prec,
                         const PropIn& in, const PropOut& out, const PropSrc& src) {
  if (nsys <= 0) return LRP_OK;
  TriKArgs a{};
  a.stepper = op->stepper;
  if (op->stepper) {
    if (plan->m > 8) return set_err(c, LRP_EINVAL, "SDIRK propagation needs a plan of 8-row chunks");
    const StepCoef sc = step_coefficients(op->stepper);
    a.su = sc.su; a.s1 = sc.s1; a.bu = sc.bu; a.b1 = sc.b1; a.b2 = sc.b2;
  }
  const bool sd = a.stepper != 0;
  a.n = plan->n;
  a.P = plan->P;
  a.L = plan->levels;
  a.M = M;
  a.nsys = nsys;
  a.dt = plan->dt;
  a.in = in;
  a.out = out;
  a.src = src;
  if (prec == 0) {
    a.coef = plan->coef64.ptr;
    a.pcr = plan->pcr64.ptr;
    switch (plan->m) {
      case 4: return launch_tri<double, 4>(c, plan, a, sd);
      case 8: return launch_tri<double, 8>(c, plan, a, sd);
      case 16: return launch_tri<double, 16>(c, plan, a);
      default: return launch_tri<double, 32>(c, plan, a);
    }
  }
  a.coef = plan->coef32.ptr;
  a.pcr = plan->pcr32.ptr;
  if (plan->m == 16 && plan->P <= 256 && plan->levels <= 8 && a.stepper == 0) {
    // enough systems to fill the SMs with 4 per CTA, else 2 or 1
    if (nsys >= 4 * c->num_sms) return launch_tri_rc<float, 16, 8, 4>(c, a);
    if (nsys >= 2 * c->num_sms) return launch_tri_rc<float, 16, 8, 2>(c, a);
    return launch_tri_rc<float, 16, 8, 1>(c, a);
  }
  switch (plan->m) {
    case 4: return launch_tri<float, 4>(c, plan, a, sd);
    case 8: return launch_tri<float, 8>(c, plan, a, sd);
    case 16: return launch_tri<float, 16>(c, plan, a);
    default: return launch_tri<float, 32>(c, plan, a);
  }
}

// ---------------------------------------------------------------------------
// Launchers on caller-provided memory (used by the allocation-free entry
// point): the factorisation is written into `scratch` instead of buffers owned
// by an operator.  Layout of the scratch: coef64 [5][m][P] | pcr64
// [2L+1][P] | coef32 | pcr32 | status (int), each part 256-byte aligned.
// ---------------------------------------------------------------------------
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t tri_raw_scratch_bytes(int n) {
  int m = choose_m(n), P = (n + m - 1) / m, L = 0;
  while ((1 << L) < P) ++L;
  size_t MP = (size_t)m * P, Lp = (size_t)(2 * L + 1) * P;
  return align256(5 * MP * 8) + align256(Lp * 8) + align256(5 * MP * 4) + align256(Lp * 4) + 256;
}

lrp_status tri_raw_propagate(cudaStream_t stream, int num_sms, void* scratch, int n,
                             const double* lo, const double* di, const double* up, double dt,
                             int adjoint, int M, int nsys, int prec, const PropIn& in,
                             const PropOut& out, const PropSrc& src) {
  int m = choose_m(n), P = (n + m - 1) / m, L = 0;
  while ((1 << L) < P) ++L;
  size_t MP = (size_t)m * P, Lp = (size_t)(2 * L + 1) * P;
  char* base = static_cast<char*>(scratch);
  double* coef64 = reinterpret_cast<double*>(base);
  base += align256(5 * MP * 8);
  double* pcr64 = reinterpret_cast<double*>(base);
  base += align256(Lp * 8);
  float* coef32 = reinterpret_cast<float*>(base);
  base += align256(5 * MP * 4);
  float* pcr32 = reinterpret_cast<float*>(base);
  base += align256(Lp * 4);
  int* status = reinterpret_cast<int*>(base);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), stream);
  if (e) return LRP_ECUDA;
  int threads = ((P + 31) / 32) * 32;
  k_tri_factor<<<1, threads, 5 * P * sizeof(double), stream>>>(lo, di, up, n, dt, adjoint, m, P, L,
                                                              coef64, coef32, pcr64, pcr32, status);
  if (cudaGetLastError()) return LRP_ECUDA;
  int st = 0;
  e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (!e) e = cudaStreamSynchronize(stream);
  if (e) return LRP_ECUDA;
  if (st) return LRP_EBREAKDOWN;
  if (nsys <= 0) return LRP_OK;
  TriKArgs a{};
  a.n = n; a.P = P; a.L = L; a.M = M; a.nsys = nsys; a.dt = dt;
  a.in = in; a.out = out; a.src = src;
  a.coef = prec == 0 ? (const void*)coef64 : (const void*)coef32;
  a.pcr = prec == 0 ? (const void*)pcr64 : (const void*)pcr32;
  Ctx tmp;                       // stream and SM count for the shared launcher
  tmp.stream = stream;
  tmp.num_sms = num_sms;
  TriPlan* none = nullptr;
  if (prec == 0) {
    switch (m) {
      case 4: return launch_tri<double, 4>(&tmp, none, a);
      case 8: return launch_tri<double, 8>(&tmp, none, a);
      case 16: return launch_tri<double, 16>(&tmp, none, a);
      default: return launch_tri<double, 32>(&tmp, none, a);
    }
  }
  switch (m) {
    case 4: return launch_tri<float, 4>(&tmp, none, a);
    case 8: return launch_tri<float, 8>(&tmp, none, a);
    case 16: return launch_tri<float, 16>(&tmp, none, a);
    default: return launch_tri<float, 32>(&tmp, none, a);
  }
}

}  // namespace lrp
