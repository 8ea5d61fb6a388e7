// Backward-Euler propagator for time-dependent tridiagonal operators
// (Experiment 2 of Sec. 4: a conductivity varying in space and time, so that
// every fine step J has its own matrix B_J = I + dt A(t_{J+1}) and the fine
// solvers F_n of the intervals differ).
//
// No factorisation can be reused across steps, so each step is solved from
// its own coefficients by parallel cyclic reduction (PCR) in shared memory:
// one CTA per system, thread i owns row i (the CTA's P threads, a power of two
// >= n, pad the system with identity rows), and log2(P) levels each eliminate
// the couplings at distance s from every row, after which row i reads
// x_i = d_i / b_i.  PCR needs no pivoting for the diagonally dominant B_J of
// a diffusion operator.  The adjoint F_n'^* = B_{j0}^-T ... B_{j1}^-T runs the
// transposed steps in reversed order.  System s belongs to the interval given
// by the call's system map (of the input, else of the output, else of the
// source: calls with zero initial values map only their outputs), else to
// interval0 + s / ncol; its steps are interval * M .. interval * M + M - 1 of
// the operator's time grid.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lrp {

struct TdArgs {
  int n, nJ, M, adjoint, nsys, P;
  double dt;                 // SDIRK: gamma dt
  double su, s1, bu, b1, b2; // SDIRK: stage combination (see StepCoef; remapped for the adjoint)
  const double* lo;   // nJ x n: row J holds A(t_{J+1})
  const double* di;
  const double* up;
  PropIn in;
  PropOut out;
  PropSrc src;
};

// SD: two-stage SDIRK steps; the coefficient rows are then 2 per step, row
// 2J + s the operator at stage time s of step J.  The forward step solves
// with the stage-1 matrix, then the stage-2 matrix; the adjoint step (the
// transposed step map) solves with the transposed stage-2 matrix first, the
// host remapping the combination coefficients.
template <typename T, bool SD>
__global__ void __launch_bounds__(1024) k_tri_td(TdArgs a) {
  if (a.in.stop && *a.in.stop) return;
  extern __shared__ __align__(16) unsigned char td_smem[];
  const int P = a.P, n = a.n, i = threadIdx.x;
  T* sa = reinterpret_cast<T*>(td_smem);
  T* sib = sa + P;       // 1 / b of every row
  T* sc = sib + P;
  T* sd = sc + P;
  const T dt = (T)a.dt;
  const int* imap = a.in.map ? a.in.map : a.out.map ? a.out.map : a.src.map;
  for (int sys = blockIdx.x; sys < a.nsys; sys += gridDim.x) {
    const int interval = imap ? imap[2 * sys + 1] : a.in.interval0 + sys / a.in.ncol;
    const long j0 = (long)interval * a.M;
    if (j0 < 0 || j0 + a.M > a.nJ) continue;     // outside the time grid (checked on the host)
    T x = T(0);
    if (i < n) {
      if (a.in.gen)
        x = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                     (uint32_t)(sys % a.in.ncol), (uint32_t)i);
      else if (a.in.x != nullptr) {
        const long ox = sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys);
        x = a.in.x_f64 ? (T) static_cast<const double*>(a.in.x)[ox + i]
                       : (T) static_cast<const float*>(a.in.x)[ox + i];
      }
    }
    const double* csys = a.src.Q > 0
        ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
    const double* gsys = (a.src.Q > 0 && a.src.map)
        ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
    // one PCR solve with row `row` of the coefficients: (I + dt A_row) y = d
    // (or its transpose), thread i holding row i (identity rows beyond n)
    auto pcr = [&](long row, T dv) -> T {
      T av = T(0), bv = T(1), cv = T(0);
      if (i < n) {
        const double* lo = a.lo + row * n;
        const double* di = a.di + row * n;
        const double* up = a.up + row * n;
        // row i of B (or of its transpose): a x_{i-1} + b x_i + c x_{i+1}
        const double l = a.adjoint ? (i > 0 ? up[i - 1] : 0.0) : (i > 0 ? lo[i] : 0.0);
        const double u = a.adjoint ? (i + 1 < n ? lo[i + 1] : 0.0) : (i + 1 < n ? up[i] : 0.0);
        av = (T)(a.dt * l);
        bv = (T)(1.0 + a.dt * di[i]);
        cv = (T)(a.dt * u);
      } else {
        dv = T(0);
      }
      for (int s = 1; s < P; s <<= 1) {
        sa[i] = av;
        sib[i] = T(1) / bv;
        sc[i] = cv;
        sd[i] = dv;
        __syncthreads();
        T al = T(0), ga = T(0), am = T(0), cm = T(0), dm = T(0), ap = T(0), cp = T(0), dp = T(0);
        if (i - s >= 0) {
          al = -av * sib[i - s];
          am = sa[i - s];
          cm = sc[i - s];
          dm = sd[i - s];
        }
        if (i + s < P) {
          ga = -cv * sib[i + s];
          ap = sa[i + s];
          cp = sc[i + s];
          dp = sd[i + s];
        }
        av = al * am;
        cv = ga * cp;
        bv = bv + al * cm + ga * ap;
        dv = dv + al * dm + ga * dp;
        __syncthreads();
      }
      return dv / bv;
    };
    // dt f at source sample fj of this system (0 without a source)
    auto src = [&](int fj) -> T {
      T f = T(0);
      if (csys && i < n)
        for (int q = 0; q < a.src.Q; ++q)
          f += dt * (T)csys[(size_t)fj * a.src.Q + q] * (T)gsys[(size_t)q * n + i];
      return f;
    };
    for (int t = 0; t < a.M; ++t) {
      const long J = a.adjoint ? j0 + a.M - 1 - t : j0 + t;
      if constexpr (!SD) {
        x = pcr(J, x + src(t));
      } else {
        const long r1 = a.adjoint ? 2 * J + 1 : 2 * J, r2 = a.adjoint ? 2 * J : 2 * J + 1;
        const T u0 = x;
        const T U1 = pcr(r1, u0 + src(2 * t));
        const T U2 = pcr(r2, (T)a.su * u0 + (T)a.s1 * U1 + src(2 * t + 1));
        x = (T)a.bu * u0 + (T)a.b1 * U1 + (T)a.b2 * U2;
      }
    }
    if (i < n) {
      const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
      if (a.out.y_f64)
        static_cast<double*>(a.out.y)[oy + i] = (double)x;
      else
        static_cast<float*>(a.out.y)[oy + i] = (float)x;
    }
  }
}

lrp_status tri_td_propagate(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys,
                            int prec, const PropIn& in, const PropOut& out, const PropSrc& src) {
  if (nsys <= 0) return LRP_OK;
  if (adjoint && src.Q > 0) return set_err(c, LRP_EINVAL, "the adjoint acts on the linear part");
  if (!in.map && !out.map && !src.map) {
    const long last = (long)in.interval0 + (long)(nsys - 1) / std::max(in.ncol, 1);
    if (in.interval0 < 0 || (last + 1) * M > op->nJ)
      return set_err(c, LRP_EINVAL, "time-dependent operator: steps beyond its time grid");
  }
  TdArgs a;
  const bool sd = op->stepper != 0;
  const StepCoef sc = sd ? step_coefficients(op->stepper) : StepCoef{1.0, 0, 0, 0, 0, 0};
  a.su = sc.su;
  a.s1 = sc.s1;
  a.bu = sc.bu;
  a.b1 = sc.b1;
  a.b2 = sc.b2;
  if (sd && adjoint) {
    // the transposed step map bu I + b1 B1^-T + b2 su B2^-T + b2 s1 B1^-T B2^-T:
    // W2 = B2^-T v, W1 = B1^-T (b1 v + b2 s1 W2), v' = bu v + b2 su W2 + W1
    a.su = sc.b1;
    a.s1 = sc.b2 * sc.s1;
    a.b1 = sc.b2 * sc.su;
    a.b2 = 1.0;
  }
  a.n = op->n;
  a.nJ = op->nJ;
  a.M = M;
  a.adjoint = adjoint;
  a.nsys = nsys;
  int P = 32;
  while (P < op->n) P <<= 1;
  a.P = P;
  a.dt = sd ? dt * sc.gamma : dt;
  a.lo = op->a64[0].as<double>();
  a.di = op->a64[1].as<double>();
  a.up = op->a64[2].as<double>();
  a.in = in;
  a.out = out;
  a.src = src;
  const size_t smem = (size_t)4 * P * (prec == 0 ? 8 : 4);
  const int grid = std::min(nsys, c->num_sms * std::max(1, 2048 / P));
  const char* fam = prec == 0 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  if (prec == 0)
    (sd ? k_tri_td<double, true> : k_tri_td<double, false>)<<<grid, P, smem, c->stream>>>(a);
  else
    (sd ? k_tri_td<float, true> : k_tri_td<float, false>)<<<grid, P, smem, c->stream>>>(a);
  timer_end(c, fam, ev);
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_err(c, e, "k_tri_td launch");
  return LRP_OK;
}

}  // namespace lrp

using namespace lrp;
struct lrp_operator : public Operator {};

// rows = nJ (backward Euler) or 2 nJ (SDIRK: the two stage times of every step)
static lrp_status make_tridiag_td(Ctx* c, int n, int nJ, int stepper, const double* lo,
                                  const double* di, const double* up, lrp_operator** out) {
  if (n > 1024) return set_err(c, LRP_EINVAL, "time-dependent operators take n <= 1024");
  cudaSetDevice(c->device);
  auto* op = new lrp_operator();
  op->ctx = c;
  ctx_retain(c);
  op->kind = 2;
  op->n = n;
  op->nJ = nJ;
  op->stepper = stepper;
  const double* src[3] = {lo, di, up};
  const size_t bytes = sizeof(double) * (size_t)nJ * (stepper ? 2 : 1) * n;
  for (int k = 0; k < 3; ++k) {
    lrp_status s = dev_alloc(c, op->a64[k], bytes);
    if (s) { delete op; return s; }
    cudaError_t e = cudaMemcpyAsync(op->a64[k].ptr, src[k], bytes, cudaMemcpyDefault, c->stream);
    if (e) { delete op; return cuda_err(c, e, "time-dependent operator upload"); }
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) { delete op; return cuda_err(c, e, "time-dependent operator upload"); }
  *out = op;
  return LRP_OK;
}

extern "C" lrp_status lrp_operator_tridiag_td(lrp_ctx* cc, int n, int nJ, const double* lo,
                                              const double* di, const double* up,
                                              lrp_operator** out) {
  Ctx* c = reinterpret_cast<Ctx*>(cc);
  if (!c || !out || !lo || !di || !up || n < 2 || nJ < 1) return LRP_EINVAL;
  return make_tridiag_td(c, n, nJ, 0, lo, di, up, out);
}

extern "C" lrp_status lrp_operator_tridiag_td_sdirk(lrp_ctx* cc, int n, int nJ, int stepper,
                                                    const double* lo, const double* di,
                                                    const double* up, lrp_operator** out) {
  Ctx* c = reinterpret_cast<Ctx*>(cc);
  if (!c || !out || !lo || !di || !up || n < 2 || nJ < 1) return LRP_EINVAL;
  if (stepper != LRP_STEP_SDIRK2 && stepper != LRP_STEP_SDIRK2_L)
    return set_err(c, LRP_EINVAL, "stage-sampled operators take an SDIRK stepper");
  return make_tridiag_td(c, n, nJ, stepper, lo, di, up, out);
}
