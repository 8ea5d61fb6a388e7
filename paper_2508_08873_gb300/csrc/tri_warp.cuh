// Shared by the cluster tridiagonal propagators: the kernel arguments and the
// one-warp cluster kernel (instantiated in tridiag_warp.cu and tridiag_warp_nosplit.cu).
#pragma once
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace lrp {

constexpr int CL_MAXC = 16;
static_assert(CL_MAXC == 16, "the one-warp kernel splits the warp into two halves of CL_MAXC lanes");
constexpr int CLW_L = 5;    // PCR levels over the 31 local interface unknowns of a one-warp CTA

// Arguments of the cluster propagation kernels: cluster of C CTAs per system,
// blockDim = Pc (one chunk per thread).  Clusters loop over systems.
struct ClKArgs {
  int n, Pc, C, L, M, nsys;
  double dt;
  double su, s1, bu, b1, b2;   // two-stage SDIRK coefficients (see StepCoef)
  const void* coef;
  const void* lpcr;
  const void* spk;
  const void* sup;
  PropIn in;
  PropOut out;
  PropSrc src;
  ToepCoef tz;                 // constant-coefficient one-warp kernel
};

// One-warp cluster propagation, FP64 (chunks of 8..16 rows); S selects how
// the chunk-interior solve is split around the cluster barrier: S = 0 runs
// all of it between arrive and wait, S = 1 leaves its last (MM-2)/3
// backward rows after the wait (see the kernel).  Returns LRP_EINVAL for an
// unsupported plan.
template <int S>
lrp_status tri_launch_warp(Ctx* c, ClPlan* pl, ClKArgs& a);

// The constant-coefficient variant of the cluster kernel (a.tz.on, no
// source term, FP64), and of the one-CTA-per-system kernel (C <= 8; T =
// float or double).
lrp_status tri_launch_warp_toep(Ctx* c, ClPlan* pl, ClKArgs& a);
template <typename T>
lrp_status tri_launch_warp_block_toep(Ctx* c, ClPlan* pl, ClKArgs& a);

// One system per CTA of C warps (T = float or double; chunks of 8, 12 or 16
// rows), coefficients from a warp cluster plan (ClPlan with warp = 1) in T.
template <typename T>
lrp_status tri_launch_warp_block(Ctx* c, ClPlan* pl, ClKArgs& a);

#ifdef LRP_TRI_WARP_KERNEL
namespace cg = cooperative_groups;

__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// ---------------------------------------------------------------------------
// The steps of a system split over C units of one warp each (32 chunks per
// warp), each unit with its slice of the factorisation held in registers:
// the units are the one-warp CTAs of a cluster (k_tri_cluster_w, FP64: the
// Parareal fine solves) or the warps of one CTA (k_tri_block_w, FP32 or
// FP64: the sketches).  The local interface system of a unit is solved by
// parallel cyclic reduction with warp shuffles and the C x C super system by
// two warp sums, so a step needs one exchange of four values per unit and
// one barrier (cluster or block).  (Chunks of MM = 8..16 rows; C = 1..16.)
//
// Per step j the work splits into
//   * a chain through the cluster: interface row, PCR, publish, barrier,
//     super system, and the spike correction of rows 0 and MM-2 that the
//     next step's interface row reads;
//   * work off that chain: the chunk-interior solve of the next step and the
//     correction of the other rows.
// The spike correction x <- x - yl fp - y fq of a step is deferred into the
// next step, whose interior solve is then T x_local - yl T fp - y T fq (T is
// linear), so the interior solve does not wait for the barrier.  The loop is
// rotated so that the super system, the correction and the next step's PCR
// form one straight block (no branch between them: the compiler interleaves
// the independent FMAs of the correction with the PCR's shuffle chains), and
// the interior solve sits between the barrier's arrive and wait, except its
// last HLO backward rows, which follow the wait and run beside the super
// system's warp sums.
// ---------------------------------------------------------------------------
template <typename T, int MM, bool SRC, int HLO, class X>
__device__ __forceinline__ void warp_steps(const ClKArgs& a, X& xch, int c, int tl, int sys0,
                                           int dsys) {
  static_assert(HLO >= 0 && HLO <= MM - 2, "split row out of range");
  const int C = a.C;
  const int t = c * 32 + tl;
  const int n = a.n;
  const int r0 = t * MM;
  const unsigned FULL = 0xffffffffu;
  // ---- this thread's factors, in registers ---------------------------------
  const T* gco = static_cast<const T*>(a.coef) + (size_t)c * 5 * MM * 32;
  const T* gpc = static_cast<const T*>(a.lpcr) + (size_t)c * (2 * CLW_L + 1) * 32;
  const T* gsp = static_cast<const T*>(a.spk) + (size_t)c * 2 * 32;
  const T* gsu = static_cast<const T*>(a.sup);
  // pP, pQ hold T fp and T fq, the chunk-interior solve T applied to the two
  // spike vectors (the deferred correction)
  T fl[MM], fi[MM], fu[MM], pP[MM], pQ[MM];
#pragma unroll
  for (int i = 0; i < MM; ++i) {
    fl[i] = gco[(0 * MM + i) * 32 + tl];
    fi[i] = gco[(1 * MM + i) * 32 + tl];
    fu[i] = gco[(2 * MM + i) * 32 + tl];
    pP[i] = gco[(3 * MM + i) * 32 + tl];
    pQ[i] = gco[(4 * MM + i) * 32 + tl];
  }
  // the chunk-interior solve (rows 0..MM-2; row MM-1 is the interface row):
  // forward sweep, then the backward sweep in two parts, rows MM-3..HLO and
  // HLO-1..0; each backward row is one FMA on the chain (the scaling by the
  // inverse pivot is off it)
  auto fwd = [&](T* v) {
#pragma unroll
    for (int i = 1; i < MM - 1; ++i) v[i] = fmaT(-fl[i], v[i - 1], v[i]);
    v[MM - 2] *= fi[MM - 2];
  };
  auto bwd_hi = [&](T* v) {
#pragma unroll
    for (int i = MM - 3; i >= HLO; --i) v[i] = fmaT(-fu[i], v[i + 1], v[i] * fi[i]);
  };
  auto bwd_lo = [&](T* v) {
#pragma unroll
    for (int i = HLO - 1; i >= 0; --i) v[i] = fmaT(-fu[i], v[i + 1], v[i] * fi[i]);
  };
  fwd(pP); bwd_hi(pP); bwd_lo(pP);
  fwd(pQ); bwd_hi(pQ); bwd_lo(pQ);
  T k1[CLW_L], k2[CLW_L];
#pragma unroll
  for (int l = 0; l < CLW_L; ++l) {
    k1[l] = gpc[l * 32 + tl];
    k2[l] = gpc[(CLW_L + l) * 32 + tl];
  }
  const T dv = tl < 31 ? gpc[2 * CLW_L * 32 + tl] : T(0);
  const T p2 = gsp[tl], q2 = gsp[32 + tl];
  // super system: both half-warps form row q = tl mod 16 (q < C); the lower
  // half holds column q of inverse row c, the upper half column q of inverse
  // row c-1, so one product and four butterfly levels give Y_c and Y_{c-1}
  const int q = tl & (CL_MAXC - 1);
  const T sa = q < C ? gsu[6 * q + 0] : T(0);
  const T sc1 = q < C ? gsu[6 * q + 1] : T(0);
  const T sc2 = q < C ? gsu[6 * q + 2] : T(0);
  const T* minv = gsu + 6 * CL_MAXC;
  const T msel = q < C ? (tl < CL_MAXC ? minv[c * CL_MAXC + q]
                                       : (c > 0 ? minv[(c - 1) * CL_MAXC + q] : T(0)))
                       : T(0);
  const T dt = (T)a.dt;
  int pb = 0;
  for (int sys = sys0; sys < a.nsys; sys += dsys) {
    T x[MM];
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int r = r0 + i;
      T v = T(0);
      if (r < n) {
        if (a.in.gen)
          v = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                            (uint32_t)(sys % a.in.ncol), (uint32_t)r);
        else if (a.in.x == nullptr)
          v = T(0);
        else if (a.in.x_f64)
          v = (T)static_cast<const double*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
        else
          v = (T)static_cast<const float*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
      }
      x[i] = v;
    }
    if (a.M <= 0) {
      // no step: the output is the input
    } else {
      const double* csys = nullptr;
      const double* gsys = nullptr;
      if (SRC) {
        csys = a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys);
        gsys = a.src.map ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
      }
      // dt f(t_{j+1}) added to the right-hand side of step j on the interior
      // rows; the interface row's term is returned
      auto add_source = [&](int j) -> T {
        T sI = T(0);
        for (int qq = 0; qq < a.src.Q; ++qq) {
          const T cq_ = dt * (T)csys[(size_t)j * a.src.Q + qq];
          const double* gq = gsys + (size_t)qq * n;
#pragma unroll
          for (int i = 0; i < MM - 1; ++i)
            if (r0 + i < n) x[i] += cq_ * (T)gq[r0 + i];
          if (r0 + MM - 1 < n) sI += cq_ * (T)gq[r0 + MM - 1];
        }
        return sI;
      };
      T z0 = T(0), y = T(0), yl = T(0), v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
      // interface row and local PCR; reads x[0] (of the next lane), x[MM-2]
      // and x[MM-1]
      auto pcr = [&]() {
        T gnext = __shfl_down_sync(FULL, x[0], 1);
        if (tl == 31) gnext = T(0);
        T r = x[MM - 1] - fl[MM - 1] * x[MM - 2] - fu[MM - 1] * gnext;
        // local PCR over lanes 0..30 (lane 31 is the CTA's super unknown)
#pragma unroll
        for (int l = 0; l < CLW_L; ++l) {
          const T rm = __shfl_up_sync(FULL, r, 1 << l);
          const T rp = __shfl_down_sync(FULL, r, 1 << l);
          if (tl < 31) r = r - k1[l] * rm - k2[l] * rp;
        }
        z0 = r * dv;                           // 0 on lane 31 (dv = 0)
        // z0 of the first and last local unknown, the super row's r, the
        // first row of the first chunk
        v0 = __shfl_sync(FULL, z0, 0);
        v1 = __shfl_sync(FULL, z0, 30);
        v2 = __shfl_sync(FULL, r, 31);
        v3 = __shfl_sync(FULL, x[0], 0);
      };
      // publication of the CTA's four values: lane q stores into CTA q
      auto publish = [&]() {
        xch.publish(pb, c, tl, C, v0, v1, v2, v3);
      };
      // super system: lane q forms the right-hand side of unknown q; Y_c and
      // Y_{c-1} are rows of the precomputed inverse applied by warp sums
      auto super_solve = [&]() {
        T rhs = T(0);
        if (q < C) {
          const T* pq = xch.slot(pb, q);
          rhs = fmaT(-sa, pq[1], pq[2]);
          if (q + 1 < C) {
            const T* pn = xch.slot(pb, q + 1);
            rhs = fmaT(-sc2, pn[3], fmaT(-sc1, pn[0], rhs));
          }
        }
        T Ys = msel * rhs;
#pragma unroll
        for (int o = CL_MAXC / 2; o > 0; o >>= 1) Ys += __shfl_xor_sync(FULL, Ys, o);
        const T Yc = __shfl_sync(FULL, Ys, 0), Yl = __shfl_sync(FULL, Ys, CL_MAXC);
        y = (tl < 31) ? z0 - p2 * Yl - q2 * Yc : Yc;
        yl = __shfl_up_sync(FULL, y, 1);
        if (tl == 0) yl = Yl;
      };
      // x[0..MM-2]: the interior solution of the current step (spike
      // corrections of the previous step included); x[MM-1]: the right-hand
      // side of the interface row
      if (SRC) x[MM - 1] += add_source(0);
      fwd(x); bwd_hi(x); bwd_lo(x);
      pcr();
      publish();
      for (int j = 0; j + 1 < a.M; ++j) {
        xch.arrive();
        // while the barrier completes: the next step's interior solve on the
        // uncorrected interior values (its right-hand side x + dt f)
        T sI = T(0);                         // source of the interface row
        if (SRC) sI = add_source(j + 1);
        fwd(x);
        bwd_hi(x);
        xch.wait();
        super_solve();
        bwd_lo(x);
        // the deferred correction, through the next step's interior solve
        // (rows 0 and MM-2 feed the next interface row)
        x[0] = fmaT(-pP[0], yl, fmaT(-pQ[0], y, x[0]));
        x[MM - 2] = fmaT(-pP[MM - 2], yl, fmaT(-pQ[MM - 2], y, x[MM - 2]));
        x[MM - 1] = SRC ? y + sI : y;
        pb ^= 1;
        pcr();
#pragma unroll
        for (int i = 1; i < MM - 2; ++i) x[i] = fmaT(-pP[i], yl, fmaT(-pQ[i], y, x[i]));
        publish();
      }
      // the last step: its spike corrections with fp, fq themselves
      xch.arrive();
      xch.wait();
      super_solve();
#pragma unroll
      for (int i = 0; i < MM - 1; ++i)
        x[i] = x[i] - gco[(3 * MM + i) * 32 + tl] * yl - gco[(4 * MM + i) * 32 + tl] * y;
      x[MM - 1] = y;
      pb ^= 1;
    }
    const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int r = r0 + i;
      if (r < n) {
        if (a.out.y_f64)
          static_cast<double*>(a.out.y)[oy + r] = (double)x[i];
        else
          static_cast<float*>(a.out.y)[oy + r] = (float)x[i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Constant-coefficient variant (no source; FP64 on a cluster of one-warp
// CTAs per system, FP64 or FP32 on one CTA of warps per system).  Every
// chunk interior is the Toeplitz matrix T (lower a,
// diagonal d, upper c) of m = MM - 1 rows, or identity padding rows.  With
// the steady pivot dinf of the LU factorisation of tridiag(a, d, c),
//   T = L U + (d - dinf) e_0 e_0^T,  L = I + l E^T,  U = dinf (I + u E),
// so with S = dinf (L U)^{-1} (one forward and one backward sweep of one FMA
// per row: no division by a pivot) and phi = (L U)^{-1} e_0,
//   T^{-1} v = (L U)^{-1} v - kappa ((L U)^{-1} v)_0 phi,
//   kappa = (d - dinf) / (1 + (d - dinf) phi_0)        (Sherman-Morrison),
// and the left spike fp = T^{-1}(a_left e_0) = beta phi, beta = a_left (1 -
// kappa phi_0).  A step's interior solution is then
//   x = w - (kappa w_0 + beta yl) phi - y fq,   w = (L U)^{-1} b,
// two FMAs per row beside the two of the sweeps (the general kernel needs
// three for the solve).  The state is carried scaled: step j's quantities are
// dinf^(j+1) times the true ones, so that S replaces (L U)^{-1}; the
// interface row, PCR and super system take the scaling in their constants
// (the interface residual is formed divided by dinf), and every P steps the
// state is multiplied by rho = dinf^-P.  The step loop and its split around
// the barrier are those of warp_steps; the correction is deferred into the
// next step's sweeps through S phi and S fq.  (In FP32 the host sets dinf so
// that the swept matrix keeps the smallest eigenvalue of tridiag(a, d, c)
// exactly; see tri_toeplitz_coef.)
// ---------------------------------------------------------------------------
template <typename T, int MM, int HLO, class X>
__device__ __forceinline__ void warp_steps_toep(const ClKArgs& a, X& xch, int c, int tl, int sys0,
                                                int dsys, T* shc = nullptr) {
  static_assert(HLO >= 0 && HLO <= MM - 2, "split row out of range");
  const int C = a.C;
  const int t = c * 32 + tl;
  const int n = a.n;
  const int r0 = t * MM;
  const unsigned FULL = 0xffffffffu;
  const ToepCoef& z = a.tz;
  const T* gco = static_cast<const T*>(a.coef) + (size_t)c * 5 * MM * 32;
  const T* gpc = static_cast<const T*>(a.lpcr) + (size_t)c * (2 * CLW_L + 1) * 32;
  const T* gsp = static_cast<const T*>(a.spk) + (size_t)c * 2 * 32;
  const T* gsu = static_cast<const T*>(a.sup);
  // this lane's chunk: Toeplitz interior rows, or identity padding rows
  const bool real = r0 < n;
  const T l = real ? (T)z.l : T(0), u = real ? (T)z.u : T(0);
  auto s_fwd = [&](T* v) {
#pragma unroll
    for (int i = 1; i < MM - 1; ++i) v[i] = fmaT(-l, v[i - 1], v[i]);
  };
  auto s_bwd_hi = [&](T* v) {
#pragma unroll
    for (int i = MM - 3; i >= HLO; --i) v[i] = fmaT(-u, v[i + 1], v[i]);
  };
  auto s_bwd_lo = [&](T* v) {
#pragma unroll
    for (int i = HLO - 1; i >= 0; --i) v[i] = fmaT(-u, v[i + 1], v[i]);
  };
  // phi = (L U)^{-1} e_0 of a Toeplitz chunk (the same in every lane;
  // formed again for the last step rather than kept in registers)
  auto make_phi = [&](T* phi) {
#pragma unroll
    for (int i = 0; i < MM; ++i) phi[i] = i == 0 ? T(1) : T(0);
#pragma unroll
    for (int i = 1; i < MM - 1; ++i) phi[i] = fmaT(-(T)z.l, phi[i - 1], phi[i]);
#pragma unroll
    for (int i = MM - 3; i >= 0; --i) phi[i] = fmaT(-(T)z.u, phi[i + 1], phi[i]);
#pragma unroll
    for (int i = 0; i < MM - 1; ++i) phi[i] *= (T)z.idinf;
  };
  T phi[MM], sphi[MM], sq[MM];
  make_phi(phi);
  const T delta = (T)(z.d - z.dinf);
  const T kap_sys = delta / (T(1) + delta * phi[0]);
  const T kap = real ? kap_sys : T(0);
  const T beta = (real && r0 > 0) ? (T)z.a * (T(1) - kap_sys * phi[0]) : T(0);
  // S phi and S fq: the deferred correction.  With shc (the block kernel),
  // both live in shared memory: S phi is the same in every lane, and S fq
  // too, times qs = 0 for the lanes without a right coupling (padding, or
  // an interface row past the system); fq is then the fq of chunk 0
  // (identical in every chunk with a right coupling).
  const T qs = (real && r0 + MM - 1 < n) ? T(1) : T(0);
  const T* gq0 = static_cast<const T*>(a.coef) + 4 * MM * 32;   // chunk 0's fq
#pragma unroll
  for (int i = 0; i < MM - 1; ++i) {
    sphi[i] = phi[i];
    sq[i] = shc ? gq0[i * 32] : gco[(4 * MM + i) * 32 + tl];
  }
  if (shc) {
    const T lr = (T)z.l, ur = (T)z.u;
#pragma unroll
    for (int i = 1; i < MM - 1; ++i) {
      sphi[i] = fmaT(-lr, sphi[i - 1], sphi[i]);
      sq[i] = fmaT(-lr, sq[i - 1], sq[i]);
    }
#pragma unroll
    for (int i = MM - 3; i >= 0; --i) {
      sphi[i] = fmaT(-ur, sphi[i + 1], sphi[i]);
      sq[i] = fmaT(-ur, sq[i + 1], sq[i]);
    }
    if (threadIdx.x == 0)
#pragma unroll
      for (int i = 0; i < MM - 1; ++i) {
        shc[i] = sphi[i];
        shc[MM + i] = sq[i];
      }
    __syncthreads();
  } else {
    s_fwd(sphi); s_bwd_hi(sphi); s_bwd_lo(sphi);
    s_fwd(sq); s_bwd_hi(sq); s_bwd_lo(sq);
  }
  // the correction vectors of row i
  auto cphi = [&](int i) -> T { return shc ? shc[i] : sphi[i]; };
  auto cq = [&](int i) -> T { return shc ? shc[MM + i] : sq[i]; };
  // interface row (couplings aE to row MM-2 and cE to the next chunk's row
  // 0), divided by dinf, in terms of w: X_{MM-2} = w_{MM-2} - kappa phi_{MM-2}
  // w_0 and X'_0 = (1 - kappa phi_0) w'_0
  const T idinf = (T)z.idinf, dinf = (T)z.dinf;
  const T aE = gco[(0 * MM + MM - 1) * 32 + tl];
  const T cE = gco[(2 * MM + MM - 1) * 32 + tl];
  const T cA = aE * idinf;
  const T cK = aE * kap * phi[MM - 2] * idinf;
  const T cB = cE * (T(1) - kap_sys * phi[0]) * idinf;
  T k1[CLW_L], k2[CLW_L];
#pragma unroll
  for (int lv = 0; lv < CLW_L; ++lv) {
    k1[lv] = gpc[lv * 32 + tl];
    k2[lv] = gpc[(CLW_L + lv) * 32 + tl];
  }
  const T dv = tl < 31 ? gpc[2 * CLW_L * 32 + tl] * dinf : T(0);
  const T p2 = gsp[tl], q2 = gsp[32 + tl];
  const int q = tl & (CL_MAXC - 1);
  const T sa = q < C ? gsu[6 * q + 0] * idinf : T(0);
  const T sc1 = q < C ? gsu[6 * q + 1] * idinf : T(0);
  const T sc2 = q < C ? gsu[6 * q + 2] * (T(1) - kap_sys * phi[0]) * idinf : T(0);
  const T* minv = gsu + 6 * CL_MAXC;
  const T msel = q < C ? (tl < CL_MAXC ? minv[c * CL_MAXC + q]
                                       : (c > 0 ? minv[(c - 1) * CL_MAXC + q] : T(0))) * dinf
                       : T(0);
  int pb = 0;
  for (int sys = sys0; sys < a.nsys; sys += dsys) {
    T x[MM];
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int r = r0 + i;
      T v = T(0);
      if (r < n) {
        if (a.in.gen)
          v = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                            (uint32_t)(sys % a.in.ncol), (uint32_t)r);
        else if (a.in.x == nullptr)
          v = T(0);
        else if (a.in.x_f64)
          v = (T)static_cast<const double*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
        else
          v = (T)static_cast<const float*>(a.in.x)[sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) + r];
      }
      x[i] = v;
    }
    if (a.M > 0) {
      T z0 = T(0), y = T(0), yl = T(0), w0 = T(0), v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
      auto pcr = [&]() {
        T gnext = __shfl_down_sync(FULL, x[0], 1);
        if (tl == 31) gnext = T(0);
        T r = fmaT(-cB, gnext, fmaT(cK, x[0], fmaT(-cA, x[MM - 2], x[MM - 1])));
#pragma unroll
        for (int lv = 0; lv < CLW_L; ++lv) {
          const T rm = __shfl_up_sync(FULL, r, 1 << lv);
          const T rp = __shfl_down_sync(FULL, r, 1 << lv);
          if (tl < 31) r = r - k1[lv] * rm - k2[lv] * rp;
        }
        z0 = r * dv;
        v0 = __shfl_sync(FULL, z0, 0);
        v1 = __shfl_sync(FULL, z0, 30);
        v2 = __shfl_sync(FULL, r, 31);
        v3 = __shfl_sync(FULL, x[0], 0);
      };
      auto super_solve = [&]() {
        T rhs = T(0);
        if (q < C) {
          const T* pq = xch.slot(pb, q);
          rhs = fmaT(-sa, pq[1], pq[2]);
          if (q + 1 < C) {
            const T* pn = xch.slot(pb, q + 1);
            rhs = fmaT(-sc2, pn[3], fmaT(-sc1, pn[0], rhs));
          }
        }
        T Ys = msel * rhs;
#pragma unroll
        for (int o = CL_MAXC / 2; o > 0; o >>= 1) Ys += __shfl_xor_sync(FULL, Ys, o);
        const T Yc = __shfl_sync(FULL, Ys, 0), Yl = __shfl_sync(FULL, Ys, CL_MAXC);
        y = (tl < 31) ? z0 - p2 * Yl - q2 * Yc : Yc;
        yl = __shfl_up_sync(FULL, y, 1);
        if (tl == 0) yl = Yl;
      };
      // one step of the loop: the barrier of step j, the sweeps of step j+1,
      // the super system of step j and the deferred correction, the PCR of
      // step j+1; with resc, the state is rescaled by rho after the super
      // system
      auto body = [&](bool resc) {
        xch.arrive();
        w0 = x[0];
        s_fwd(x);
        s_bwd_hi(x);
        xch.wait();
        super_solve();
        s_bwd_lo(x);
        if (resc) {
          const T rho = (T)z.rho;
          y *= rho;
          yl *= rho;
          w0 *= rho;
#pragma unroll
          for (int i = 0; i < MM - 1; ++i) x[i] *= rho;
        }
        const T sc = fmaT(kap, w0, beta * yl);
        const T yq = shc ? qs * y : y;
        x[0] = fmaT(-sc, cphi(0), fmaT(-cq(0), yq, x[0]));
        x[MM - 2] = fmaT(-sc, cphi(MM - 2), fmaT(-cq(MM - 2), yq, x[MM - 2]));
        x[MM - 1] = y;
        pb ^= 1;
        pcr();
#pragma unroll
        for (int i = 1; i < MM - 2; ++i) x[i] = fmaT(-sc, cphi(i), fmaT(-cq(i), yq, x[i]));
        xch.publish(pb, c, tl, C, v0, v1, v2, v3);
      };
      s_fwd(x); s_bwd_hi(x); s_bwd_lo(x);
      pcr();
      xch.publish(pb, c, tl, C, v0, v1, v2, v3);
      // bodies j = 0 .. M-2; the one with (j + 1) % P == 0 rescales
      int j = 0;
      while (true) {
        const int jr = ((j + z.P) / z.P) * z.P - 1;
        const int jlim = min(jr, a.M - 1);
        for (; j < jlim; ++j) body(false);
        if (j >= a.M - 1) break;
        body(true);
        ++j;
      }
      // the last step: its correction with phi and fq themselves, then the
      // remaining scaling undone
      xch.arrive();
      xch.wait();
      super_solve();
      const T sc = fmaT(kap, x[0], beta * yl);
      const T fin = (T)z.fin;
      T phl[MM];
      make_phi(phl);
#pragma unroll
      for (int i = 0; i < MM - 1; ++i)
        x[i] = (x[i] - sc * phl[i] - gco[(4 * MM + i) * 32 + tl] * y) * fin;
      x[MM - 1] = y * fin;
      pb ^= 1;
    }
    const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int r = r0 + i;
      if (r < n) {
        if (a.out.y_f64)
          static_cast<double*>(a.out.y)[oy + r] = (double)x[i];
        else
          static_cast<float*>(a.out.y)[oy + r] = (float)x[i];
      }
    }
  }
}

// Exchange of the four published values per unit, between the one-warp CTAs
// of a cluster: lane q pushes into CTA q's shared memory; one cluster
// barrier (split into arrive and wait) per step
struct XchCluster {
  double (*pubg)[CL_MAXC][4];   // this CTA's receive buffers
  double* const* rpub;          // the receive buffers of the cluster's CTAs
  __device__ __forceinline__ void publish(int pb, int c, int tl, int C, double v0, double v1,
                                          double v2, double v3) {
    if (tl < C) {
      double* dst = rpub[tl] + (pb * CL_MAXC + c) * 4;
      dst[0] = v0; dst[1] = v1; dst[2] = v2; dst[3] = v3;
    }
  }
  __device__ __forceinline__ const double* slot(int pb, int q) const { return &pubg[pb][q][0]; }
  __device__ __forceinline__ void arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  }
  __device__ __forceinline__ void wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
};

// Exchange between the warps of one CTA: lane 0 of each warp writes its
// values into the CTA's buffer; one block barrier per step
template <typename T>
struct XchBlock {
  T (*pubg)[CL_MAXC][4];
  __device__ __forceinline__ void publish(int pb, int c, int tl, int, T v0, T v1, T v2, T v3) {
    if (tl == 0) {
      T* dst = &pubg[pb][c][0];
      dst[0] = v0; dst[1] = v1; dst[2] = v2; dst[3] = v3;
    }
  }
  __device__ __forceinline__ const T* slot(int pb, int q) const { return &pubg[pb][q][0]; }
  __device__ __forceinline__ void arrive() {}
  __device__ __forceinline__ void wait() { __syncthreads(); }
};

// FP64, one system per cluster of C one-warp CTAs (the Parareal fine solves)
template <int MM, bool SRC, int HLO>
__global__ void __launch_bounds__(32) k_tri_cluster_w(ClKArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double pubg[2][CL_MAXC][4];
  __shared__ double* rpub[CL_MAXC];
  const int C = a.C;
  const int c = (int)cl.block_rank();
  const int tl = threadIdx.x;
  if (tl < C) rpub[tl] = cl.map_shared_rank(&pubg[0][0][0], tl);
  __syncwarp();
  cl.sync();   // every CTA of the cluster runs before any remote store into its shared memory
  XchCluster xch{pubg, rpub};
  warp_steps<double, MM, SRC, HLO>(a, xch, c, tl, (int)blockIdx.x / C, (int)gridDim.x / C);
  cl.sync();  // no CTA leaves while others may still store into its shared memory
}

// FP64 constant-coefficient variant, one system per cluster of C one-warp CTAs
template <int MM, int HLO>
__global__ void __launch_bounds__(32) k_tri_cluster_wt(ClKArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double pubg[2][CL_MAXC][4];
  __shared__ double* rpub[CL_MAXC];
  const int C = a.C;
  const int c = (int)cl.block_rank();
  const int tl = threadIdx.x;
  if (tl < C) rpub[tl] = cl.map_shared_rank(&pubg[0][0][0], tl);
  __syncwarp();
  cl.sync();   // every CTA of the cluster runs before any remote store into its shared memory
  XchCluster xch{pubg, rpub};
  warp_steps_toep<double, MM, HLO>(a, xch, c, tl, (int)blockIdx.x / C, (int)gridDim.x / C);
  cl.sync();  // no CTA leaves while others may still store into its shared memory
}

// FP32 or FP64, one system per CTA of C warps (32 C chunks; C <= 16 in FP32,
// <= 8 in FP64): the same steps with the exchange through the CTA's shared
// memory and a block barrier, for batches large enough to fill the GPU with
// CTAs (the sketches)
template <typename T>
constexpr int blk_w_threads() { return sizeof(T) == 8 ? 256 : 512; }   // FP64: factors need > 128 registers

template <typename T, int MM, bool SRC, int HLO>
__global__ void __launch_bounds__(blk_w_threads<T>()) k_tri_block_w(ClKArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  __shared__ T pubg[2][CL_MAXC][4];
  XchBlock<T> xch{pubg};
  warp_steps<T, MM, SRC, HLO>(a, xch, (int)(threadIdx.x >> 5), (int)(threadIdx.x & 31),
                              (int)blockIdx.x, (int)gridDim.x);
}

// Constant-coefficient variant, one system per CTA of C warps (C <= 8):
// FP64, or FP32 at three CTAs per SM
template <typename T>
constexpr int blk_wt_min_ctas() { return sizeof(T) == 8 ? 1 : 3; }

template <typename T, int MM, int HLO>
__global__ void __launch_bounds__(256, blk_wt_min_ctas<T>()) k_tri_block_wt(ClKArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  __shared__ T pubg[2][CL_MAXC][4];
  __shared__ T shc[2 * MM];
  XchBlock<T> xch{pubg};
  warp_steps_toep<T, MM, HLO>(a, xch, (int)(threadIdx.x >> 5), (int)(threadIdx.x & 31),
                              (int)blockIdx.x, (int)gridDim.x, sizeof(T) == 4 ? shc : nullptr);
}

template <typename T, int MM>
static lrp_status launch_blk_wt(Ctx* c, ClPlan* pl, ClKArgs& a) {
  auto kern = k_tri_block_wt<T, MM, (MM - 2) / 3>;
  const int threads = 32 * pl->C;
  if (threads > 256) return set_err(c, LRP_EINVAL, "block warp kernel: at most 8 warps per system");
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e || per_sm < 1) { cudaGetLastError(); per_sm = 1; }
  const int grid = std::min(a.nsys, per_sm * c->num_sms);
  const char* fam = sizeof(T) == 8 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  kern<<<grid, threads, 0, c->stream>>>(a);
  e = cudaGetLastError();
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_tri_block_wt launch");
  return LRP_OK;
}

template <int MM, bool SRC, int HLO>
static lrp_status launch_cl_w(Ctx* c, ClPlan* pl, ClKArgs& a) {
  const int C = pl->C;
  auto kern = k_tri_cluster_w<MM, SRC, HLO>;
  cudaError_t e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e) return cuda_err(c, e, "cluster size 16 not available");
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(32);
  cfg.gridDim = dim3(C);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = c->stream;
  int maxc = 0;
  e = cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg);
  if (e || maxc < 1) { cudaGetLastError(); maxc = std::max(1, c->num_sms / C); }
  const int ncl = std::min(a.nsys, maxc);
  cfg.gridDim = dim3(ncl * C);
  cudaEvent_t ev = nullptr;
  timer_begin(c, "propagate_f64", &ev);
  e = cudaLaunchKernelEx(&cfg, kern, a);
  timer_end(c, "propagate_f64", ev);
  if (e) return cuda_err(c, e, "k_tri_cluster_w launch");
  return LRP_OK;
}

template <typename T, int MM, bool SRC, int HLO>
static lrp_status launch_blk_w(Ctx* c, ClPlan* pl, ClKArgs& a) {
  auto kern = k_tri_block_w<T, MM, SRC, HLO>;
  const int threads = 32 * pl->C;
  if (threads > blk_w_threads<T>())
    return set_err(c, LRP_EINVAL, "block warp kernel: too many warps per system for this precision");
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e || per_sm < 1) { cudaGetLastError(); per_sm = 1; }
  const int grid = std::min(a.nsys, per_sm * c->num_sms);
  const char* fam = sizeof(T) == 8 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  kern<<<grid, threads, 0, c->stream>>>(a);
  e = cudaGetLastError();
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_tri_block_w launch");
  return LRP_OK;
}

template <typename T>
lrp_status tri_launch_warp_block(Ctx* c, ClPlan* pl, ClKArgs& a) {
  const bool src = a.src.Q > 0;
  switch (pl->m) {
    case 16: return src ? launch_blk_w<T, 16, true, 4>(c, pl, a) : launch_blk_w<T, 16, false, 4>(c, pl, a);
    case 12: return src ? launch_blk_w<T, 12, true, 3>(c, pl, a) : launch_blk_w<T, 12, false, 3>(c, pl, a);
    case 8: return src ? launch_blk_w<T, 8, true, 2>(c, pl, a) : launch_blk_w<T, 8, false, 2>(c, pl, a);
    default: return set_err(c, LRP_EINVAL, "block warp kernel: chunk length 8, 12 or 16");
  }
}

template <int MM>
static lrp_status launch_cl_wt(Ctx* c, ClPlan* pl, ClKArgs& a) {
  const int C = pl->C;
  auto kern = k_tri_cluster_wt<MM, (MM - 2) / 3>;
  cudaError_t e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e) return cuda_err(c, e, "cluster size 16 not available");
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(32);
  cfg.gridDim = dim3(C);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = c->stream;
  int maxc = 0;
  e = cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg);
  if (e || maxc < 1) { cudaGetLastError(); maxc = std::max(1, c->num_sms / C); }
  const int ncl = std::min(a.nsys, maxc);
  cfg.gridDim = dim3(ncl * C);
  cudaEvent_t ev = nullptr;
  timer_begin(c, "propagate_f64", &ev);
  e = cudaLaunchKernelEx(&cfg, kern, a);
  timer_end(c, "propagate_f64", ev);
  if (e) return cuda_err(c, e, "k_tri_cluster_wt launch");
  return LRP_OK;
}

template <int MM, int S>
static lrp_status launch_cl_w_src(Ctx* c, ClPlan* pl, ClKArgs& a) {
  constexpr int HLO = S == 0 ? 0 : (MM - 2) / 3;
  if (a.src.Q > 0) return launch_cl_w<MM, true, HLO>(c, pl, a);
  return launch_cl_w<MM, false, HLO>(c, pl, a);
}

template <int S>
lrp_status tri_launch_warp(Ctx* c, ClPlan* pl, ClKArgs& a) {
  switch (pl->m) {
    case 16: return launch_cl_w_src<16, S>(c, pl, a);
    case 15: return launch_cl_w_src<15, S>(c, pl, a);
    case 14: return launch_cl_w_src<14, S>(c, pl, a);
    case 13: return launch_cl_w_src<13, S>(c, pl, a);
    case 12: return launch_cl_w_src<12, S>(c, pl, a);
    case 11: return launch_cl_w_src<11, S>(c, pl, a);
    case 10: return launch_cl_w_src<10, S>(c, pl, a);
    case 9: return launch_cl_w_src<9, S>(c, pl, a);
    case 8: return launch_cl_w_src<8, S>(c, pl, a);
    default: return set_err(c, LRP_EINVAL, "warp cluster chunk length out of range");
  }
}
#endif  // LRP_TRI_WARP_KERNEL

}  // namespace lrp
