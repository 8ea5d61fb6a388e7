// FP64 steps of 5-point operators by mixed-precision iterative refinement:
// every backward-Euler step (I + dt A) x = d, d = x_j + dt f(t_{j+1}) -- and
// every stage solve of an SDIRK step, (I + gamma dt A) x = d with d the
// stage's right-hand side -- is solved to the FP64 tolerance by rounds of
//   r = d - B x          (FP64, from the FP64 step matrix),
//   B e = r              (FP32, to a looser relative tolerance (1e-3), from
//                         e = 0: conjugate gradients on the on-chip kernel for
//                         symmetric operators, BiCGStab on the global-memory
//                         kernel otherwise),
//   x <- x + e           (FP64),
// until the residual meets the same test as the FP64 Krylov kernels -- for
// CG the diagonally scaled residual, ||D^1/2 (d - B x)|| <= rtol ||D^1/2 d||
// (D = diag(B)^-1), for BiCGStab the plain one (D = I) -- evaluated in FP64,
// or reaches its rounding level,
// ||D^1/2 (d - B x)|| <= IR_FLOOR u_64 ||D^1/2 (|d| + |B| |x|)|| (the residual
// of the true solution rounded to FP64 is of that size, so no iterate can do
// better; the Krylov kernels test their recursively updated residual, which
// can fall below it).  The FP32 solves run with every Krylov
// vector on chip, and GB300 executes FP32 at 64 times its FP64 rate, so the
// FP64 work of a step shrinks to one residual per round.
//
// Each round gains a factor of about rtol_inner + kappa u_32 on the residual
// (kappa the condition number of the scaled step matrix, u_32 the FP32 unit
// roundoff: the FP32 solve is exact only for the rounded matrix); a system
// stops as soon as its own residual passes, so that the rounds of a step only
// run the systems still above the tolerance.  The iterate is warm-started
// from x_j (an SDIRK stage from the previous stage value) as in the FP64
// kernels.  Systems are processed in batches of at most IR_BATCH with FP64
// workspaces of four vectors each (six with an SDIRK stepper).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lrp {

constexpr int IR_THREADS = 256;
constexpr int IR_PTS = 8;          // grid points per thread in the residual kernel
constexpr int IR_BATCH = 256;      // systems per batch (four FP64 vectors each)
constexpr int IR_MAX_ROUNDS = 60;  // refinement rounds per step before LRP_ENOTCONV
constexpr double IR_FLOOR = 8.0;   // rounding level of the residual, in units of u_64 (|d| + |B||x|)

// input vector of systems s0 .. s0 + cnt - 1 into X (cnt x n)
__global__ void k_ir_gather(PropIn in, int n, int s0, int cnt, double* __restrict__ X) {
  const long tot = (long)cnt * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), k = (int)(e % n), sys = s0 + s;
    double v = 0.0;
    if (in.gen)
      v = gauss<double>(in.seed, in.stream, (uint32_t)(in.interval0 + sys / in.ncol),
                        (uint32_t)(sys % in.ncol), (uint32_t)k);
    else if (in.x != nullptr) {
      const long o = sys_offset(in.map, in.slot_stride, in.ldx, sys) + k;
      v = in.x_f64 ? static_cast<const double*>(in.x)[o] : (double)static_cast<const float*>(in.x)[o];
    }
    X[e] = v;
  }
}

__global__ void k_ir_scatter(PropOut out, int n, int s0, int cnt, const double* __restrict__ X) {
  const long tot = (long)cnt * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), k = (int)(e % n);
    const long o = sys_offset(out.map, out.slot_stride, out.ldy, s0 + s) + k;
    if (out.y_f64)
      static_cast<double*>(out.y)[o] = X[e];
    else
      static_cast<float*>(out.y)[o] = (float)X[e];
  }
}

// right-hand side of a solve: D = au A + a1 W + dt f (W may be null; f the
// source sample `sample` of each system): backward Euler D = X + dt f(t_{j+1}),
// SDIRK stage s D = su U0 + s1 U1 + gamma dt f(stage time)
__global__ void k_ir_rhs(PropSrc src, int n, int s0, int cnt, int sample, double dt, double au,
                         const double* __restrict__ A, double a1, const double* __restrict__ W,
                         double* __restrict__ D) {
  const long tot = (long)cnt * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    const int s = (int)(e / n), k = (int)(e % n), sys = s0 + s;
    double f = 0.0;
    if (src.Q > 0) {
      const double* csys = src.c + sys_offset(src.map, src.c_slot_stride, src.cstride, sys);
      const double* gsys = src.map ? src.g + (long)src.map[2 * sys] * src.g_slot_stride : src.g;
      for (int q = 0; q < src.Q; ++q) f += csys[(size_t)sample * src.Q + q] * gsys[(size_t)q * n + k];
    }
    double d = au * A[e] + dt * f;
    if (W) d += a1 * W[e];
    D[e] = d;
  }
}

// SDIRK step end: X = bu U0 + b1 U1 + b2 X
__global__ void k_ir_combine(long tot, double bu, const double* __restrict__ U0, double b1,
                             const double* __restrict__ U1, double b2, double* __restrict__ X) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x)
    X[e] = bu * U0[e] + b1 * U1[e] + b2 * X[e];
}

// Residual of the listed systems (list[2 i] = system of the batch):
// r = D - B X into G (scaled for the FP32 correction solve by k_ir_scale),
// and per block the partial sums of r^T D r,
// d^T D d and a^T D a, a = |d| + |B| |x| (D = 1 / diag(B)), in a fixed order.
__global__ void __launch_bounds__(IR_THREADS) k_ir_resid(int mx, int my, int unit,
                                                        const double* __restrict__ B, long ldb,
                                                        long b_step,
                                                        const int* __restrict__ list,
                                                        const double* __restrict__ X,
                                                        const double* __restrict__ D,
                                                        double* __restrict__ G,
                                                        double* __restrict__ part) {
  const int n = mx * my;
  const int s = list[2 * blockIdx.y];
  const long base = (long)s * n;
  B += (long)list[2 * blockIdx.y + 1] * b_step;   // time-dependent operators: the step's plan
  const int k0 = blockIdx.x * IR_THREADS * IR_PTS;
  double rr = 0.0, dd = 0.0, aa = 0.0;
#pragma unroll
  for (int u = 0; u < IR_PTS; ++u) {
    const int k = k0 + u * IR_THREADS + threadIdx.x;
    if (k < n) {
      const int ix = k % mx, iy = k / mx;
      const double* x = X + base;
      double bx = B[k] * x[k];
      double ab = fabs(B[k] * x[k]);
      if (ix > 0) { const double t = B[ldb + k] * x[k - 1]; bx += t; ab += fabs(t); }
      if (ix < mx - 1) { const double t = B[2 * ldb + k] * x[k + 1]; bx += t; ab += fabs(t); }
      if (iy > 0) { const double t = B[3 * ldb + k] * x[k - mx]; bx += t; ab += fabs(t); }
      if (iy < my - 1) { const double t = B[4 * ldb + k] * x[k + mx]; bx += t; ab += fabs(t); }
      const double d = D[base + k];
      const double r = d - bx;
      const double dinv = unit ? 1.0 : B[5 * ldb + k];   // BiCGStab: the plain 2-norm
      G[base + k] = r;
      rr += r * r * dinv;
      dd += d * d * dinv;
      ab += fabs(d);
      aa += ab * ab * dinv;
    }
  }
  __shared__ double sh[3][IR_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
    aa += __shfl_xor_sync(0xffffffffu, aa, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = rr;
    sh[1][w] = dd;
    sh[2][w] = aa;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double a = 0.0;
    for (int i = 0; i < IR_THREADS / 32; ++i) a += sh[threadIdx.x][i];
    part[((long)blockIdx.y * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = a;
  }
}

// One warp per listed system: the residual test from the partial sums (fixed
// order); systems above both the tolerance and the rounding level go to the
// next list (cnt[0] counts them; their order does not affect any result),
// with the scale sigma = ||D^1/2 r|| / sqrt(n) of their residual (the FP32
// solve runs on r / sigma: a residual of a decayed state can lie below the
// FP32 range).
__global__ void k_ir_reduce(int nblk, int n, double rtol2, double floor2,
                            const int* __restrict__ list, const double* __restrict__ part,
                            int* __restrict__ next, int* __restrict__ cnt,
                            double* __restrict__ sigma) {
  const int i = blockIdx.x, lane = threadIdx.x;
  double rr = 0.0, dd = 0.0, aa = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    rr += part[((long)i * nblk + b) * 3];
    dd += part[((long)i * nblk + b) * 3 + 1];
    aa += part[((long)i * nblk + b) * 3 + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
    aa += __shfl_xor_sync(0xffffffffu, aa, o);
  }
  if (lane == 0 && rr > rtol2 * dd && rr > floor2 * aa) {
    const int at = atomicAdd(cnt, 1);
    next[2 * at] = list[2 * i];
    next[2 * at + 1] = list[2 * i + 1];
    sigma[list[2 * i]] = sqrt(rr / n);       // rr > 0 here
  }
}

// G <- G / (dt sigma) on the listed systems: the FP32 solve's source, whose
// right-hand side dt G is then r / sigma
__global__ void k_ir_scale(int n, double dt, const int* __restrict__ list,
                           const double* __restrict__ sigma, double* __restrict__ G) {
  const int s = list[2 * blockIdx.y];
  const long base = (long)s * n;
  const double f = 1.0 / (dt * sigma[s]);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    G[base + k] *= f;
}

// X += sigma E on the listed systems
__global__ void k_ir_apply(int n, const int* __restrict__ list, const double* __restrict__ sigma,
                           double* __restrict__ X, const double* __restrict__ E) {
  const int s = list[2 * blockIdx.y];
  const long base = (long)s * n;
  const double sg = sigma[s];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    X[base + k] = fma(sg, E[base + k], X[base + k]);
}

// every system of the batch into the list; its second entry is the row of
// the time grid of the system's step j (time-dependent operators: the
// interval of the system from the call's maps, else interval0 + s / ncol;
// the adjoint runs the steps in reversed order), else 0
__global__ void k_ir_list_all(int cnt, int* __restrict__ list, double* __restrict__ one, int td,
                              PropIn in, const int* __restrict__ omap, const int* __restrict__ smap,
                              int s0, int M, int j, int adj, int sd, int stage, long nrows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) {
    int row = 0;
    if (td) {
      const int sys = s0 + i;
      const int* imap = in.map ? in.map : omap ? omap : smap;
      const long J0 = (long)(imap ? imap[2 * sys + 1] : in.interval0 + sys / in.ncol) * M;
      const long J = adj ? J0 + M - 1 - j : J0 + j;
      // SDIRK: the operator at the stage time (rows 2J, 2J + 1; the adjoint
      // solves with the second stage's matrix first)
      const long r = sd ? 2 * J + (adj ? 1 - stage : stage) : J;
      // the callers' maps name intervals inside the time grid (checked where
      // they are made); a row outside it is never read
      row = (int)(r < 0 ? 0 : r >= nrows ? nrows - 1 : r);
    }
    list[2 * i] = i;
    list[2 * i + 1] = row;
  }
  if (i == 0) *one = 1.0;
}

bool stencil_refine_applies(Ctx* c, const Operator* op, int prec, int nsys) {
  if (prec != 0 || (op->kind != 1 && op->kind != 3)) return false;
  // time-dependent operators: symmetric ones, on the on-chip kernel's TD variant
  if (op->kind == 3 && !op->symmetric) return false;
  if (c->p_krylov_refine == 2) return false;
  // nonsymmetric operators: FP32 BiCGStab corrections on the global-memory
  // kernel (measured on GB300, adv2d nu = 0.01, dt = 1/4096, 64 systems, us
  // per system and step against FP64 BiCGStab: 511^2 207 / 556, 255^2 35 / 76)
  if (!op->symmetric) return true;
  return stencil_onchip_fits(c, op, 1, std::min(nsys, IR_BATCH));
}

lrp_status stencil_propagate_refine(Ctx* c, Operator* op, StencilPlan* plan, int M, int nsys,
                                    const PropIn& in, const PropOut& out, const PropSrc& src,
                                    int adjoint) {
  const int n = op->n;
  const int batch = std::min(nsys, IR_BATCH);
  const size_t vec = (size_t)batch * n;
  const int nblk = (n + IR_THREADS * IR_PTS - 1) / (IR_THREADS * IR_PTS);
  // X, D, G, E (FP64; SDIRK: U0, U1 too), partial sums, two system lists,
  // the counter, the constant 1
  const bool sd = op->stepper != 0;
  const size_t nv = sd ? 6 : 4;
  const size_t need = sizeof(double) * (nv * vec + (size_t)batch * nblk * 3 + (size_t)batch + 8) +
                      sizeof(int) * (4 * (size_t)batch + 8);
  lrp_status s;
  if (c->irws.bytes < need)
    if ((s = dev_alloc(c, c->irws, need))) return s;
  if (!c->irstat.ptr)
    if ((s = dev_alloc(c, c->irstat, 32))) return s;
  double* X = c->irws.as<double>();
  double* D = X + vec;
  double* G = D + vec;
  double* E = G + vec;
  double* U0 = E + vec;                       // SDIRK: the step's start state
  double* U1 = U0 + (sd ? vec : 0);           // SDIRK: the first stage value
  double* part = U1 + (sd ? vec : 0);
  double* sigma = part + (size_t)batch * nblk * 3;
  double* one = sigma + batch;
  int* listA = reinterpret_cast<int*>(one + 8);
  int* listB = listA + 2 * batch;
  int* cnt = listB + 2 * batch;
  cudaStream_t st = c->stream;
  // the inner FP32 solves: their iterations and status words
  unsigned long long* iters = reinterpret_cast<unsigned long long*>(c->irstat.ptr);
  int* istat = reinterpret_cast<int*>(static_cast<char*>(c->irstat.ptr) + 8);
  cudaMemsetAsync(c->irstat.ptr, 0, 32, st);
  const int bicg = op->symmetric ? 0 : 1;
  const int td = op->kind == 3 ? 1 : 0;       // every system on its own step's plan
  // SDIRK: each stage solve refined on its own stage matrix B = I + gamma dt A
  // (the plan's dt is gamma dt); the adjoint of a time-dependent operator runs
  // the transposed step map W2 = B2^-T v, W1 = B1^-T (b1 v + b2 s1 W2),
  // v' = bu v + b2 su W2 + W1 (the same stage body with these coefficients)
  StepCoef sc = sd ? step_coefficients(op->stepper) : StepCoef{1.0, 0, 0, 0, 0, 0};
  if (sd && td && adjoint) {
    const StepCoef f = sc;
    sc.su = f.b1;
    sc.s1 = f.b2 * f.s1;
    sc.b1 = f.b2 * f.su;
    sc.b2 = 1.0;
  }
  const double rtol2 = op->rtol64 * op->rtol64;
  const double floor2 = (IR_FLOOR * 0x1p-53) * (IR_FLOOR * 0x1p-53);
  // inner tolerance 1e-3 by default: measured on GB300 (diff2d, dt = 1/4096,
  // 128 systems, us per system and step for 1e-2 / 1e-3 / 1e-4 / 1e-5):
  // 511^2 2871 / 3194 / 3375 / 3106, 255^2 331 / 279 / 285 / 342,
  // 127^2 55 / 47 / 47 / 46
  const double rtol_in = c->p_krylov_refine_digits > 0 ? std::pow(10.0, -c->p_krylov_refine_digits)
                                                       : 1e-3;
  const long ldb = (long)n + 2 * op->mx;
  const double* B64 = plan->b64.as<double>() + op->mx;
  int* hcnt = nullptr;
  cudaError_t e = cudaMallocHost(&hcnt, sizeof(int));
  if (e) return cuda_err(c, e, "refinement counter");
  struct HostFree { int* p; ~HostFree() { if (p) cudaFreeHost(p); } } hf{hcnt};
  const int gsz = std::min<long>(4L * c->num_sms, ((long)vec + 255) / 256);
  const char* fam = "propagate_f64";
  bool notconv = false;
  for (int s0 = 0; s0 < nsys; s0 += batch) {
    const int cnt0 = std::min(batch, nsys - s0);
    k_ir_gather<<<gsz, 256, 0, st>>>(in, n, s0, cnt0, X);
    for (int j = 0; j < M && !notconv; ++j) {
      // the refinement rounds of one solve B x = D (x warm-started in X) for
      // every system of the batch, stage `stage` of step j
      auto solve = [&](int stage) -> lrp_status {
        k_ir_list_all<<<(cnt0 + 255) / 256, 256, 0, st>>>(cnt0, listA, one, td, in, out.map, src.map,
                                                          s0, M, j, adjoint, sd ? 1 : 0, stage,
                                                          (long)op->nJ * (sd ? 2 : 1));
        int nact = cnt0;
        int* cur = listA;
        int* nxt = listB;
        for (int round = 0;; ++round) {
          cudaEvent_t ev = nullptr;
          timer_begin(c, fam, &ev);
          k_ir_resid<<<dim3(nblk, nact), IR_THREADS, 0, st>>>(op->mx, op->my, bicg, B64, ldb,
                                                              td ? 6 * ldb : 0L, cur, X, D, G, part);
          cudaMemsetAsync(cnt, 0, sizeof(int), st);
          k_ir_reduce<<<nact, 32, 0, st>>>(nblk, n, rtol2, floor2, cur, part, nxt, cnt, sigma);
          timer_end(c, fam, ev);
          e = cudaMemcpyAsync(hcnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
          if (!e) e = cudaStreamSynchronize(st);
          if (!e) e = cudaGetLastError();
          if (e) return cuda_err(c, e, "refinement residual");
          nact = *hcnt;
          if (nact == 0) break;
          if (round == IR_MAX_ROUNDS || op->max_iter == 0) { notconv = true; break; }
          // the correction of every system still above the tolerance: FP32
          // CG on B e = dt G = r / sigma from e = 0 (zero input, the scaled
          // residual as the step's source), on chip
          std::swap(cur, nxt);
          k_ir_scale<<<dim3((n + 1023) / 1024, nact), 256, 0, st>>>(n, plan->dt, cur, sigma, G);
          KryArgs a{};
          a.mx = op->mx;
          a.my = op->my;
          a.n = n;
          a.M = 1;                       // TD: the list's second entry is the step's row (M = 1)
          a.nJ = op->nJ * (sd ? 2 : 1);  // rows of the time grid (two per step with SDIRK)
          a.adj = 0;
          a.nsys = nact;
          a.bicg = 0;
          a.dt = plan->dt;
          a.rtol = rtol_in;
          a.max_iter = op->max_iter;
          a.B = stencil_B(plan, op, 1);
          a.Bs = stencil_Bs(plan, op, 1);
          a.in.x = nullptr;
          a.in.ncol = 1;
          a.out.y = E;
          a.out.y_f64 = 1;
          a.out.map = cur;
          a.out.slot_stride = n;
          a.out.ldy = 0;
          a.src.Q = 1;
          a.src.g = G;
          a.src.c = one;
          a.src.cstride = 0;
          a.src.map = cur;
          a.src.c_slot_stride = 0;
          a.src.g_slot_stride = n;
          a.iters = iters;
          a.status = istat;
          a.bicg = bicg;
          if (bicg) {
            if ((s = krylov_f32_correction(c, op, plan, nact, a))) return s;
          } else if ((s = stencil_propagate_onchip(c, op, plan, 1, nact, 1, a))) {
            return s;
          }
          k_ir_apply<<<dim3((n + 1023) / 1024, nact), 256, 0, st>>>(n, cur, sigma, X, E);
        }
        return LRP_OK;
      };
      if (!sd) {
        k_ir_rhs<<<gsz, 256, 0, st>>>(src, n, s0, cnt0, j, plan->dt, 1.0, X, 0.0, nullptr, D);
        if ((s = solve(0))) return s;
      } else {
        // U1 = B1^-1 (U0 + gamma dt f_1), U2 = B2^-1 (su U0 + s1 U1 + gamma dt f_2),
        // X = bu U0 + b1 U1 + b2 U2 (coefficients remapped for the adjoint of a
        // time-dependent operator, whose step map is then the transposed one)
        e = cudaMemcpyAsync(U0, X, sizeof(double) * (size_t)cnt0 * n, cudaMemcpyDeviceToDevice, st);
        if (e) return cuda_err(c, e, "refinement stage copy");
        k_ir_rhs<<<gsz, 256, 0, st>>>(src, n, s0, cnt0, 2 * j, plan->dt, 1.0, U0, 0.0, nullptr, D);
        if ((s = solve(0))) return s;
        if (notconv) break;
        e = cudaMemcpyAsync(U1, X, sizeof(double) * (size_t)cnt0 * n, cudaMemcpyDeviceToDevice, st);
        if (e) return cuda_err(c, e, "refinement stage copy");
        k_ir_rhs<<<gsz, 256, 0, st>>>(src, n, s0, cnt0, 2 * j + 1, plan->dt, sc.su, U0, sc.s1, U1, D);
        if ((s = solve(1))) return s;
        if (notconv) break;
        k_ir_combine<<<gsz, 256, 0, st>>>((long)cnt0 * n, sc.bu, U0, sc.b1, U1, sc.b2, X);
      }
    }
    k_ir_scatter<<<gsz, 256, 0, st>>>(out, n, s0, cnt0, X);
    if (notconv) break;
  }
  unsigned long long hs[2] = {0, 0};
  e = cudaMemcpyAsync(hs, c->irstat.ptr, 16, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (!e) e = cudaGetLastError();
  if (e) return cuda_err(c, e, "refinement");
  op->krylov_iters += hs[0];
  const int stw = (int)(hs[1] & 0xffffffffu);
  if (stw & 2) return set_err(c, LRP_EBREAKDOWN, "Krylov breakdown in an FP32 correction solve");
  if (stw & 4) return set_err(c, LRP_ETIMEOUT, "a bounded wait of an FP32 correction solve expired");
  if (notconv) return set_err(c, LRP_ENOTCONV, "iterative refinement did not reach the FP64 tolerance");
  return LRP_OK;
}

}  // namespace lrp
