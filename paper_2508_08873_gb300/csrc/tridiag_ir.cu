// Near-FP64 backward-Euler steps (about 48 bits) of time-invariant
// tridiagonal operators from FP32 solves, for FP64 propagations that opt in:
// every step (I + dt A) x_{j+1} = x_j is solved by
//   y = B^-1 x_j             (FP32, the right-hand side rounded to FP32),
//   r = x_j - B y            (in pairs of FP32 numbers: products split
//                             exactly by FMA, sums by two-sum, B held as
//                             hi + lo pairs of its FP64 entries),
//   y <- y + B^-1 r          (FP32 solve of the correction, pair update),
// repeated `rounds` times per step, the state carried as an FP32 pair
// (about 48 bits).  GB300 issues FP32 at 64 times its FP64 rate, so the
// arithmetic of a step (two or three FP32 solves and one or two pair
// residuals) costs less FP32 issue than the single FP64 solve it replaces
// costs FP64 issue.  Each round gains a factor of about u_32 kappa(B) on the
// step's error; after R rounds the step error is about (u_32 kappa)^(R+1)
// plus the pair form of B, 2^-48, which enters every step alike (measured
// on the adr1d operator, n = 4095, 256 steps: 2.7e-12 from the FP64 kernels'
// result with one round, 1.4e-12 with two).
//
// One system per CTA of C warps (or, on request, per cluster of C one-warp
// CTAs), every warp 32 chunks of MM rows: the chunk solve, local PCR and
// C x C super system of the one-warp kernels, with the plan's FP32 factors,
// not deferred (each solve ends with its spike correction).  Constant
// coefficients (k_tri_irt): B's pair entries are three scalars and a lane's
// state and iterate stay in its registers; the rows beside a chunk come from
// the neighbouring lanes by shuffles and from the neighbouring warps through
// shared memory.  Variable coefficients (k_tri_ir): the state, the iterate
// and B's pair entries live in shared memory, stored chunk-transposed (row
// t MM + i at i W + t, W = 32 C chunks) so that the lanes of a warp touch
// consecutive words.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tri_warp.cuh"

namespace lrp {

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// the pair entries of B = I + dt A (lower, diagonal, upper; rows 0..n-1)
__global__ void k_tri_ir_coef(const double* __restrict__ lo, const double* __restrict__ di,
                              const double* __restrict__ up, int n, double dt,
                              float2* __restrict__ cB) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double v[3] = {dt * lo[r], 1.0 + dt * di[r], dt * up[r]};
  for (int k = 0; k < 3; ++k) {
    const float h = (float)v[k];
    cB[(size_t)k * n + r] = make_float2(h, (float)(v[k] - (double)h));
  }
}

struct IrArgs {
  const float2* cB;   // 3 x n pair entries of B
  int rounds;         // correction rounds per step (1..3)
};

// threads a CTA of the refined kernels may have (registers: the factors
// and, in the constant-coefficient kernel, the state of 5 MM rows a thread)
constexpr int ir_threads(int mm) { return mm == 16 ? 256 : mm == 12 ? 384 : 512; }

constexpr size_t ir_smem(int nr) {
  return sizeof(float) * 4 * (size_t)nr + sizeof(float2) * 3 * (size_t)nr;
}

template <int MM>
__global__ void __launch_bounds__(ir_threads(MM), 1) k_tri_ir(ClKArgs a, IrArgs ir) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  extern __shared__ __align__(16) unsigned char ir_dyn[];
  __shared__ float pubg[2][CL_MAXC][4];
  const int C = a.C, n = a.n;
  const int c = (int)(threadIdx.x >> 5), tl = (int)(threadIdx.x & 31);
  const int t = c * 32 + tl;
  const int r0 = t * MM;
  const int W = 32 * C;                        // chunks
  const int NR = W * MM;                       // rows with the padding rows
  const unsigned FULL = 0xffffffffu;
  // shared state: X (the step's start) and Y (its refined solution) as
  // pairs, and B's pair entries, row t MM + i at i W + t
  float* base = reinterpret_cast<float*>(ir_dyn);
  float* Xh = base;
  float* Xl = Xh + NR;
  float* Yh = Xl + NR;
  float* Yl = Yh + NR;
  float2* sB = reinterpret_cast<float2*>(base + 4 * NR);
  for (int i = threadIdx.x; i < 4 * NR; i += blockDim.x) base[i] = 0.f;
  for (int i = threadIdx.x; i < 3 * NR; i += blockDim.x) {
    const int k = i / NR, s = i - k * NR;      // s = iw W + tw
    const int r = (s % W) * MM + s / W;
    sB[i] = r < n ? ir.cB[(size_t)k * n + r] : make_float2(0.f, 0.f);
  }
  // this thread's factors (the warp plan's FP32 layout)
  const float* gco = static_cast<const float*>(a.coef) + (size_t)c * 5 * MM * 32;
  const float* gpc = static_cast<const float*>(a.lpcr) + (size_t)c * (2 * CLW_L + 1) * 32;
  const float* gsp = static_cast<const float*>(a.spk) + (size_t)c * 2 * 32;
  const float* gsu = static_cast<const float*>(a.sup);
  float fl[MM], fi[MM], fu[MM], fp[MM], fq[MM];
#pragma unroll
  for (int i = 0; i < MM; ++i) {
    fl[i] = gco[(0 * MM + i) * 32 + tl];
    fi[i] = gco[(1 * MM + i) * 32 + tl];
    fu[i] = gco[(2 * MM + i) * 32 + tl];
    fp[i] = gco[(3 * MM + i) * 32 + tl];
    fq[i] = gco[(4 * MM + i) * 32 + tl];
  }
  float k1[CLW_L], k2[CLW_L];
#pragma unroll
  for (int lv = 0; lv < CLW_L; ++lv) {
    k1[lv] = gpc[lv * 32 + tl];
    k2[lv] = gpc[(CLW_L + lv) * 32 + tl];
  }
  const float dv = tl < 31 ? gpc[2 * CLW_L * 32 + tl] : 0.f;
  const float p2 = gsp[tl], q2 = gsp[32 + tl];
  const int q = tl & (CL_MAXC - 1);
  const float sa = q < C ? gsu[6 * q + 0] : 0.f;
  const float sc1 = q < C ? gsu[6 * q + 1] : 0.f;
  const float sc2 = q < C ? gsu[6 * q + 2] : 0.f;
  const float* minv = gsu + 6 * CL_MAXC;
  const float msel = q < C ? (tl < CL_MAXC ? minv[c * CL_MAXC + q]
                                           : (c > 0 ? minv[(c - 1) * CL_MAXC + q] : 0.f))
                           : 0.f;
  int pb = 0;
  // B^-1 v for the whole system (v: this lane's chunk, v[MM-1] the
  // interface row); one block barrier
  auto solve = [&](float* v) {
#pragma unroll
    for (int i = 1; i < MM - 1; ++i) v[i] = __fmaf_rn(-fl[i], v[i - 1], v[i]);
    v[MM - 2] *= fi[MM - 2];
#pragma unroll
    for (int i = MM - 3; i >= 0; --i) v[i] = __fmaf_rn(-fu[i], v[i + 1], v[i] * fi[i]);
    float gnext = __shfl_down_sync(FULL, v[0], 1);
    if (tl == 31) gnext = 0.f;
    float r = v[MM - 1] - fl[MM - 1] * v[MM - 2] - fu[MM - 1] * gnext;
#pragma unroll
    for (int lv = 0; lv < CLW_L; ++lv) {
      const float rm = __shfl_up_sync(FULL, r, 1 << lv);
      const float rp = __shfl_down_sync(FULL, r, 1 << lv);
      if (tl < 31) r = r - k1[lv] * rm - k2[lv] * rp;
    }
    const float z0 = r * dv;
    const float v0 = __shfl_sync(FULL, z0, 0);
    const float v1 = __shfl_sync(FULL, z0, 30);
    const float v2 = __shfl_sync(FULL, r, 31);
    const float v3 = __shfl_sync(FULL, v[0], 0);
    if (tl == 0) {
      pubg[pb][c][0] = v0;
      pubg[pb][c][1] = v1;
      pubg[pb][c][2] = v2;
      pubg[pb][c][3] = v3;
    }
    __syncthreads();
    float rhs = 0.f;
    if (q < C) {
      rhs = __fmaf_rn(-sa, pubg[pb][q][1], pubg[pb][q][2]);
      if (q + 1 < C) rhs = __fmaf_rn(-sc2, pubg[pb][q + 1][3], __fmaf_rn(-sc1, pubg[pb][q + 1][0], rhs));
    }
    float Ys = msel * rhs;
#pragma unroll
    for (int o = CL_MAXC / 2; o > 0; o >>= 1) Ys += __shfl_xor_sync(FULL, Ys, o);
    const float Yc = __shfl_sync(FULL, Ys, 0), Ylft = __shfl_sync(FULL, Ys, CL_MAXC);
    const float y = (tl < 31) ? z0 - p2 * Ylft - q2 * Yc : Yc;
    float yl = __shfl_up_sync(FULL, y, 1);
    if (tl == 0) yl = Ylft;
    pb ^= 1;
#pragma unroll
    for (int i = 0; i < MM - 1; ++i) v[i] = __fmaf_rn(-fp[i], yl, __fmaf_rn(-fq[i], y, v[i]));
    v[MM - 1] = y;
  };
  // r = X - B Y of this lane's row i in pair arithmetic, rounded to FP32
  // (rows -1 and n carry no coupling: B's entries there are zero)
  auto resid = [&](int i) -> float {
    if (r0 + i >= n) return 0.f;
    const int me = i * W + t;
    const int dn = i > 0 ? me - W : (t > 0 ? (MM - 1) * W + t - 1 : -1);
    const int upi = i < MM - 1 ? me + W : (t + 1 < W ? t + 1 : -1);
    const float2 bl = sB[me], bd = sB[NR + me], bu = sB[2 * NR + me];
    const float yh = Yh[me];
    const float ym = dn >= 0 ? Yh[dn] : 0.f, yml = dn >= 0 ? Yl[dn] : 0.f;
    const float yp = upi >= 0 ? Yh[upi] : 0.f, ypl = upi >= 0 ? Yl[upi] : 0.f;
    const float p1 = __fmul_rn(bd.x, yh), e1 = __fmaf_rn(bd.x, yh, -p1);
    const float p2_ = __fmul_rn(bl.x, ym), e2 = __fmaf_rn(bl.x, ym, -p2_);
    const float p3 = __fmul_rn(bu.x, yp), e3 = __fmaf_rn(bu.x, yp, -p3);
    float sm = __fmaf_rn(bd.y, yh, __fmaf_rn(bl.y, ym, __fmul_rn(bu.y, yp)));
    sm = __fmaf_rn(bd.x, Yl[me], __fmaf_rn(bl.x, yml, __fmaf_rn(bu.x, ypl, sm)));
    float s, t1, t2, t3;
    two_sum(Xh[me], -p1, s, t1);
    two_sum(s, -p2_, s, t2);
    two_sum(s, -p3, s, t3);
    float tail = __fadd_rn(__fadd_rn(t1, t2), t3);
    tail = __fadd_rn(tail, Xl[me]);
    tail = __fsub_rn(tail, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, sm)));
    return __fadd_rn(s, tail);
  };
  __syncthreads();
  for (int sys = blockIdx.x; sys < a.nsys; sys += gridDim.x) {
    // the input as a pair
    const long ox = a.in.x ? sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) : 0;
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int rr = r0 + i;
      double v = 0.0;
      if (rr < n && a.in.x)
        v = a.in.x_f64 ? static_cast<const double*>(a.in.x)[ox + rr]
                       : (double)static_cast<const float*>(a.in.x)[ox + rr];
      const float h = (float)v;
      Xh[i * W + t] = h;
      Xl[i * W + t] = (float)(v - (double)h);
    }
    for (int j = 0; j < a.M; ++j) {
      float v[MM];
#pragma unroll
      for (int i = 0; i < MM; ++i) v[i] = Xh[i * W + t];
      solve(v);
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        Yh[i * W + t] = v[i];
        Yl[i * W + t] = 0.f;
      }
      __syncthreads();
      for (int k = 0; k < ir.rounds; ++k) {
#pragma unroll
        for (int i = 0; i < MM; ++i) v[i] = resid(i);
        solve(v);   // its barrier: every residual has read Y
#pragma unroll
        for (int i = 0; i < MM; ++i) {
          const int me = i * W + t;
          float s, e;
          two_sum(Yh[me], v[i], s, e);
          e = __fadd_rn(e, Yl[me]);
          const float h = __fadd_rn(s, e);
          Yh[me] = h;
          Yl[me] = __fsub_rn(e, __fsub_rn(h, s));
        }
        __syncthreads();
      }
      // the refined solution is the next step's start
      float* tp = Xh; Xh = Yh; Yh = tp;
      tp = Xl; Xl = Yl; Yl = tp;
    }
    const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int rr = r0 + i;
      if (rr < n) {
        const double v = (double)Xh[i * W + t] + (double)Xl[i * W + t];
        if (a.out.y_f64)
          static_cast<double*>(a.out.y)[oy + rr] = v;
        else
          static_cast<float*>(a.out.y)[oy + rr] = (float)v;
      }
    }
    __syncthreads();   // every row written out before the next system's input
  }
}

template <int MM>
lrp_status launch_ir(Ctx* c, ClPlan* pl, ClKArgs& a, IrArgs& ir) {
  auto kern = k_tri_ir<MM>;
  const int NR = 32 * pl->C * MM;
  const size_t smem = ir_smem(NR);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return cuda_err(c, e, "k_tri_ir smem attribute");
  const int grid = std::min(a.nsys, c->num_sms);
  cudaEvent_t ev = nullptr;
  timer_begin(c, "propagate_f64", &ev);
  kern<<<grid, 32 * pl->C, smem, c->stream>>>(a, ir);
  e = cudaGetLastError();
  timer_end(c, "propagate_f64", ev);
  if (e) return cuda_err(c, e, "k_tri_ir launch");
  return LRP_OK;
}


// Constant-coefficient operators: B's pair entries are three scalars, and the
// state and iterate stay in registers (a lane's rows; the rows next to its
// chunk come from the neighbouring lanes by shuffles and, at warp edges,
// through shared memory), so a residual row costs about 35 FP32
// instructions and no shared-memory traffic.
struct IrtCoef {
  float lh, ll, dh, dl, uh, ul;   // pairs of the lower, diagonal, upper entries
};

// Exchanges of the constant-coefficient steps between the C warps of one
// system: the four values of the super system (as in the one-warp kernels)
// and each warp's first and last row (the residual's neighbours across a warp
// edge).  sync() is the barrier after which both are visible.
// Warps of one CTA: shared memory and a block barrier.
struct IrtXchBlock {
  float (*pubg)[CL_MAXC][4];
  float (*edge)[4];                 // per warp: first row (hi, lo), last row (hi, lo)
  __device__ __forceinline__ void publish(int pb, int c, int tl, int, float v0, float v1, float v2,
                                          float v3) {
    if (tl == 0) {
      float* d = &pubg[pb][c][0];
      d[0] = v0; d[1] = v1; d[2] = v2; d[3] = v3;
    }
  }
  __device__ __forceinline__ float slot(int pb, int q, int k) const { return pubg[pb][q][k]; }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ void put_edges(int c, int tl, int, float fh, float fl_, float lh,
                                            float ll) {
    if (tl == 0) { edge[c][0] = fh; edge[c][1] = fl_; }
    if (tl == 31) { edge[c][2] = lh; edge[c][3] = ll; }
  }
  // the row before this warp's first (from warp c-1) and after its last
  __device__ __forceinline__ void get_edges(int c, int C, float& lh, float& ll, float& rh,
                                            float& rl) const {
    lh = c > 0 ? edge[c - 1][2] : 0.f;
    ll = c > 0 ? edge[c - 1][3] : 0.f;
    rh = c + 1 < C ? edge[c + 1][0] : 0.f;
    rl = c + 1 < C ? edge[c + 1][1] : 0.f;
  }
};

// One-warp CTAs of a cluster (one per SM where the cluster spreads): lanes
// store into the other CTAs' shared memory, one cluster barrier.
struct IrtXchCluster {
  float (*pubg)[CL_MAXC][4];        // this CTA's receive buffers
  float* const* rpub;               // the receive buffers of the cluster's CTAs
  float* eg;                        // this CTA's edges: [0..1] the row before, [2..3] after
  float* const* reg;                // the edges of the cluster's CTAs
  __device__ __forceinline__ void publish(int pb, int c, int tl, int C, float v0, float v1,
                                          float v2, float v3) {
    if (tl < C) {
      float* d = rpub[tl] + (pb * CL_MAXC + c) * 4;
      d[0] = v0; d[1] = v1; d[2] = v2; d[3] = v3;
    }
  }
  __device__ __forceinline__ float slot(int pb, int q, int k) const { return pubg[pb][q][k]; }
  __device__ __forceinline__ void sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
  __device__ __forceinline__ void put_edges(int c, int tl, int C, float fh, float fl_, float lh,
                                            float ll) {
    if (tl == 0 && c > 0) { reg[c - 1][2] = fh; reg[c - 1][3] = fl_; }
    if (tl == 31 && c + 1 < C) { reg[c + 1][0] = lh; reg[c + 1][1] = ll; }
  }
  __device__ __forceinline__ void get_edges(int c, int C, float& lh, float& ll, float& rh,
                                            float& rl) const {
    lh = c > 0 ? eg[0] : 0.f;
    ll = c > 0 ? eg[1] : 0.f;
    rh = c + 1 < C ? eg[2] : 0.f;
    rl = c + 1 < C ? eg[3] : 0.f;
  }
};

template <int MM, class X>
__device__ __forceinline__ void irt_steps(const ClKArgs& a, const IrtCoef& B, int rounds, X& xch,
                                          int c, int tl, int sys0, int dsys) {
  const int C = a.C, n = a.n;
  const int t = c * 32 + tl;
  const int r0 = t * MM;
  const unsigned FULL = 0xffffffffu;
  const float* gco = static_cast<const float*>(a.coef) + (size_t)c * 5 * MM * 32;
  const float* gpc = static_cast<const float*>(a.lpcr) + (size_t)c * (2 * CLW_L + 1) * 32;
  const float* gsp = static_cast<const float*>(a.spk) + (size_t)c * 2 * 32;
  const float* gsu = static_cast<const float*>(a.sup);
  float fl[MM], fi[MM], fu[MM], fp[MM], fq[MM];
#pragma unroll
  for (int i = 0; i < MM; ++i) {
    fl[i] = gco[(0 * MM + i) * 32 + tl];
    fi[i] = gco[(1 * MM + i) * 32 + tl];
    fu[i] = gco[(2 * MM + i) * 32 + tl];
    fp[i] = gco[(3 * MM + i) * 32 + tl];
    fq[i] = gco[(4 * MM + i) * 32 + tl];
  }
  float k1[CLW_L], k2[CLW_L];
#pragma unroll
  for (int lv = 0; lv < CLW_L; ++lv) {
    k1[lv] = gpc[lv * 32 + tl];
    k2[lv] = gpc[(CLW_L + lv) * 32 + tl];
  }
  const float dv = tl < 31 ? gpc[2 * CLW_L * 32 + tl] : 0.f;
  const float p2 = gsp[tl], q2 = gsp[32 + tl];
  const int q = tl & (CL_MAXC - 1);
  const float sa = q < C ? gsu[6 * q + 0] : 0.f;
  const float sc1 = q < C ? gsu[6 * q + 1] : 0.f;
  const float sc2 = q < C ? gsu[6 * q + 2] : 0.f;
  const float* minv = gsu + 6 * CL_MAXC;
  const float msel = q < C ? (tl < CL_MAXC ? minv[c * CL_MAXC + q]
                                           : (c > 0 ? minv[(c - 1) * CL_MAXC + q] : 0.f))
                           : 0.f;
  int pb = 0;
  // B^-1 v for the whole system (v: this lane's chunk, v[MM-1] the
  // interface row); one exchange and barrier
  auto solve = [&](float* v) {
#pragma unroll
    for (int i = 1; i < MM - 1; ++i) v[i] = __fmaf_rn(-fl[i], v[i - 1], v[i]);
    v[MM - 2] *= fi[MM - 2];
#pragma unroll
    for (int i = MM - 3; i >= 0; --i) v[i] = __fmaf_rn(-fu[i], v[i + 1], v[i] * fi[i]);
    float gnext = __shfl_down_sync(FULL, v[0], 1);
    if (tl == 31) gnext = 0.f;
    float r = v[MM - 1] - fl[MM - 1] * v[MM - 2] - fu[MM - 1] * gnext;
#pragma unroll
    for (int lv = 0; lv < CLW_L; ++lv) {
      const float rm = __shfl_up_sync(FULL, r, 1 << lv);
      const float rp = __shfl_down_sync(FULL, r, 1 << lv);
      if (tl < 31) r = r - k1[lv] * rm - k2[lv] * rp;
    }
    const float z0 = r * dv;
    const float v0 = __shfl_sync(FULL, z0, 0);
    const float v1 = __shfl_sync(FULL, z0, 30);
    const float v2 = __shfl_sync(FULL, r, 31);
    const float v3 = __shfl_sync(FULL, v[0], 0);
    xch.publish(pb, c, tl, C, v0, v1, v2, v3);
    xch.sync();
    float rhs = 0.f;
    if (q < C) {
      rhs = __fmaf_rn(-sa, xch.slot(pb, q, 1), xch.slot(pb, q, 2));
      if (q + 1 < C)
        rhs = __fmaf_rn(-sc2, xch.slot(pb, q + 1, 3), __fmaf_rn(-sc1, xch.slot(pb, q + 1, 0), rhs));
    }
    float Ys = msel * rhs;
#pragma unroll
    for (int o = CL_MAXC / 2; o > 0; o >>= 1) Ys += __shfl_xor_sync(FULL, Ys, o);
    const float Yc = __shfl_sync(FULL, Ys, 0), Ylft = __shfl_sync(FULL, Ys, CL_MAXC);
    const float y = (tl < 31) ? z0 - p2 * Ylft - q2 * Yc : Yc;
    float yl = __shfl_up_sync(FULL, y, 1);
    if (tl == 0) yl = Ylft;
    pb ^= 1;
#pragma unroll
    for (int i = 0; i < MM - 1; ++i) v[i] = __fmaf_rn(-fp[i], yl, __fmaf_rn(-fq[i], y, v[i]));
    v[MM - 1] = y;
  };
  float xh[MM], xl[MM], yh[MM], yl[MM];
  for (int sys = sys0; sys < a.nsys; sys += dsys) {
    const long ox = a.in.x ? sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys) : 0;
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int rr = r0 + i;
      double v = 0.0;
      if (rr < n && a.in.x)
        v = a.in.x_f64 ? static_cast<const double*>(a.in.x)[ox + rr]
                       : (double)static_cast<const float*>(a.in.x)[ox + rr];
      xh[i] = (float)v;
      xl[i] = (float)(v - (double)xh[i]);
    }
    for (int j = 0; j < a.M; ++j) {
      float v[MM];
#pragma unroll
      for (int i = 0; i < MM; ++i) v[i] = xh[i];
      solve(v);
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        yh[i] = v[i];
        yl[i] = 0.f;
      }
      for (int k = 0; k < rounds; ++k) {
        // the rows beside this lane's chunk: neighbouring lanes, and at the
        // warp's edges the neighbouring warps' rows
        xch.put_edges(c, tl, C, yh[0], yl[0], yh[MM - 1], yl[MM - 1]);
        xch.sync();
        float lh_ = __shfl_up_sync(FULL, yh[MM - 1], 1), ll_ = __shfl_up_sync(FULL, yl[MM - 1], 1);
        float rh_ = __shfl_down_sync(FULL, yh[0], 1), rl_ = __shfl_down_sync(FULL, yl[0], 1);
        float elh, ell, erh, erl;
        xch.get_edges(c, C, elh, ell, erh, erl);
        if (tl == 0) { lh_ = elh; ll_ = ell; }
        if (tl == 31) { rh_ = erh; rl_ = erl; }
        // r = X - B Y in pair arithmetic (rows past n: zero)
#pragma unroll
        for (int i = 0; i < MM; ++i) {
          const float ym = i > 0 ? yh[i - 1] : lh_, yml = i > 0 ? yl[i - 1] : ll_;
          const float yp = i < MM - 1 ? yh[i + 1] : rh_, ypl = i < MM - 1 ? yl[i + 1] : rl_;
          const float p1 = __fmul_rn(B.dh, yh[i]), e1 = __fmaf_rn(B.dh, yh[i], -p1);
          const float p2_ = __fmul_rn(B.lh, ym), e2 = __fmaf_rn(B.lh, ym, -p2_);
          const float p3 = __fmul_rn(B.uh, yp), e3 = __fmaf_rn(B.uh, yp, -p3);
          float sm = __fmaf_rn(B.dl, yh[i], __fmaf_rn(B.ll, ym, __fmul_rn(B.ul, yp)));
          sm = __fmaf_rn(B.dh, yl[i], __fmaf_rn(B.lh, yml, __fmaf_rn(B.uh, ypl, sm)));
          float s, t1, t2, t3;
          two_sum(xh[i], -p1, s, t1);
          two_sum(s, -p2_, s, t2);
          two_sum(s, -p3, s, t3);
          float tail = __fadd_rn(__fadd_rn(t1, t2), t3);
          tail = __fadd_rn(tail, xl[i]);
          tail = __fsub_rn(tail, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, sm)));
          v[i] = r0 + i < n ? __fadd_rn(s, tail) : 0.f;
        }
        solve(v);   // its barrier: every warp has read the edges
#pragma unroll
        for (int i = 0; i < MM; ++i) {
          float s, e;
          two_sum(yh[i], v[i], s, e);
          e = __fadd_rn(e, yl[i]);
          yh[i] = __fadd_rn(s, e);
          yl[i] = __fsub_rn(e, __fsub_rn(yh[i], s));
        }
      }
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        xh[i] = yh[i];
        xl[i] = yl[i];
      }
    }
    const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      const int rr = r0 + i;
      if (rr < n) {
        const double v = (double)xh[i] + (double)xl[i];
        if (a.out.y_f64)
          static_cast<double*>(a.out.y)[oy + rr] = v;
        else
          static_cast<float*>(a.out.y)[oy + rr] = (float)v;
      }
    }
  }
}

// one system per CTA of C warps
template <int MM>
__global__ void __launch_bounds__(ir_threads(MM), 1) k_tri_irt(ClKArgs a, IrtCoef B, int rounds) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  __shared__ float pubg[2][CL_MAXC][4];
  __shared__ float edge[CL_MAXC][4];
  IrtXchBlock xch{pubg, edge};
  irt_steps<MM>(a, B, rounds, xch, (int)(threadIdx.x >> 5), (int)(threadIdx.x & 31),
                (int)blockIdx.x, (int)gridDim.x);
}

// one system per cluster of C one-warp CTAs
template <int MM>
__global__ void __launch_bounds__(32) k_tri_irt_cl(ClKArgs a, IrtCoef B, int rounds) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  cg::cluster_group cl = cg::this_cluster();
  __shared__ float pubg[2][CL_MAXC][4];
  __shared__ float eg[4];
  __shared__ float* rpub[CL_MAXC];
  __shared__ float* reg[CL_MAXC];
  const int C = a.C;
  const int c = (int)cl.block_rank();
  const int tl = threadIdx.x;
  if (tl < 4) eg[tl] = 0.f;
  if (tl < C) {
    rpub[tl] = cl.map_shared_rank(&pubg[0][0][0], tl);
    reg[tl] = cl.map_shared_rank(&eg[0], tl);
  }
  __syncwarp();
  cl.sync();   // every CTA of the cluster runs before any remote store into its shared memory
  IrtXchCluster xch{pubg, rpub, eg, reg};
  irt_steps<MM>(a, B, rounds, xch, c, tl, (int)blockIdx.x / C, (int)gridDim.x / C);
  cl.sync();   // no CTA leaves while others may still store into its shared memory
}

template <int MM>
lrp_status launch_irt(Ctx* c, ClPlan* pl, ClKArgs& a, const IrtCoef& B, int rounds) {
  const int C = pl->C;
  cudaError_t e;
  cudaEvent_t ev = nullptr;
  if (c->p_tri_refine_cluster && C >= 2) {
    auto kern = k_tri_irt_cl<MM>;
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
    cfg.gridDim = dim3(std::min(a.nsys, maxc) * C);
    timer_begin(c, "propagate_f64", &ev);
    e = cudaLaunchKernelEx(&cfg, kern, a, B, rounds);
    timer_end(c, "propagate_f64", ev);
    if (e) return cuda_err(c, e, "k_tri_irt_cl launch");
    return LRP_OK;
  }
  const int grid = std::min(a.nsys, c->num_sms);
  timer_begin(c, "propagate_f64", &ev);
  k_tri_irt<MM><<<grid, 32 * C, 0, c->stream>>>(a, B, rounds);
  e = cudaGetLastError();
  timer_end(c, "propagate_f64", ev);
  if (e) return cuda_err(c, e, "k_tri_irt launch");
  return LRP_OK;
}

}  // namespace

// chunk length and warps per system of the refined FP32 path: the longest
// chunk (16, 12 or 8 rows; pref, when one of these, alone) whose 32 C chunks
// cover n within the warps a CTA of that chunk length may have
static bool tri_ir_shape(int n, int pref, int* mm, int* C) {
  for (int m : {16, 12, 8}) {
    if ((pref == 8 || pref == 12 || pref == 16) && m != pref) continue;
    const int cw = ((n + m - 1) / m + 31) / 32;
    if (cw >= 1 && 32 * cw <= ir_threads(m) && ir_smem(32 * cw * m) <= 200 * 1024) {
      *mm = m;
      *C = cw;
      return true;
    }
  }
  return false;
}

bool tri_ir_applies(Ctx* c, const Operator* op, int prec, int adjoint, int M, const PropIn& in,
                    const PropSrc& src) {
  if (c->p_tri_refine != 1) return false;
  if (prec != 0 || adjoint || M <= 0 || op->kind != 0 || op->stepper != 0 || src.Q > 0 || in.gen)
    return false;
  int mm = 0, C = 0;
  return op->n >= 64 && tri_ir_shape(op->n, c->p_tri_wchunk, &mm, &C);
}

lrp_status tri_propagate_ir(Ctx* c, Operator* op, double dt, int M, int nsys, const PropIn& in,
                            const PropOut& out) {
  if (nsys <= 0) return LRP_OK;
  int mm = 0, C = 0;
  if (!tri_ir_shape(op->n, c->p_tri_wchunk, &mm, &C)) return set_err(c, LRP_EINVAL, "refined FP32 tridiagonal: n out of range");
  ClPlan* pl = nullptr;
  lrp_status s = tri_get_cluster_plan(c, op, dt, 0, C, mm, &pl, 1);
  if (s) return s;
  const int rounds = std::min(3, std::max(1, c->p_tri_refine_rounds));
  ClKArgs a{};
  a.n = op->n;
  a.Pc = pl->Pc;
  a.C = pl->C;
  a.L = pl->L;
  a.M = M;
  a.nsys = nsys;
  a.dt = dt;
  a.in = in;
  a.out = out;
  a.coef = pl->b32[0].ptr;
  a.lpcr = pl->b32[1].ptr;
  a.spk = pl->b32[2].ptr;
  a.sup = pl->b32[3].ptr;
  if (op->toeplitz) {
    // B = I + dt A: three entries, as FP32 pairs
    const double v[3] = {dt * op->tlo, 1.0 + dt * op->tdi, dt * op->tup};
    float h[3], l[3];
    for (int k = 0; k < 3; ++k) {
      h[k] = (float)v[k];
      l[k] = (float)(v[k] - (double)h[k]);
    }
    const IrtCoef B{h[0], l[0], h[1], l[1], h[2], l[2]};
    switch (mm) {
      case 16: return launch_irt<16>(c, pl, a, B, rounds);
      case 12: return launch_irt<12>(c, pl, a, B, rounds);
      default: return launch_irt<8>(c, pl, a, B, rounds);
    }
  }
  const size_t need = sizeof(float2) * 3 * (size_t)op->n;
  if (c->triws.bytes < need)
    if ((s = dev_alloc(c, c->triws, need))) return s;
  float2* cB = c->triws.as<float2>();
  k_tri_ir_coef<<<(op->n + 255) / 256, 256, 0, c->stream>>>(
      op->a64[0].as<double>(), op->a64[1].as<double>(), op->a64[2].as<double>(), op->n, dt, cB);
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_err(c, e, "k_tri_ir_coef");
  IrArgs ir{cB, rounds};
  switch (mm) {
    case 16: return launch_ir<16>(c, pl, a, ir);
    case 12: return launch_ir<12>(c, pl, a, ir);
    default: return launch_ir<8>(c, pl, a, ir);
  }
}

}  // namespace lrp
