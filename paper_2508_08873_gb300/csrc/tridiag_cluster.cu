// Tridiagonal backward-Euler propagation with one system spread over a
// thread-block cluster of C CTAs (up to 16), for batches too small to fill
// the GPU with one CTA per system (the Parareal fine solves: one system per
// coarse interval, FP64).
//
// The partitioned solve of tridiag.cu is applied on two levels:
//   * rows -> chunks of m rows (one thread each): interior Thomas substitution
//     and spikes, leaving one interface unknown y_t per chunk;
//   * chunks -> C CTAs of Pc chunks: in every CTA the interface unknowns but
//     the last form a local tridiagonal system, solved by parallel cyclic
//     reduction with precomputed factors, whose solution is
//     z0 - P2 Y_{c-1} - Q2 Y_c in terms of the last interface unknowns Y_c of
//     the CTAs; these C unknowns satisfy a small tridiagonal "super" system
//     with a precomputed LU factorisation, which every CTA solves redundantly
//     after one exchange of 4 scalars per CTA through distributed shared
//     memory.
// So each implicit-Euler step costs one cluster barrier, and each CTA holds
// only its own slice of the factorisation in shared memory.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tri_common.cuh"
#include "tri_warp.cuh"

namespace cg = cooperative_groups;

namespace lrp {


// index helpers for the per-CTA layouts
__host__ __device__ __forceinline__ size_t cl_coef(int c, int k, int i, int tl, int m, int Pc) {
  return (((size_t)c * 5 + k) * m + i) * Pc + tl;
}

// ---------------------------------------------------------------------------
// Factorisation (one CTA of P threads, FP64).  Outputs (see ClPlan):
//   coef [C][5][m][Pc]; lpcr [C][2L+1][Pc]; spk [C][2][Pc]; sup [C][6].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_tri_factor_cl(const double* __restrict__ lo, const double* __restrict__ di,
                                const double* __restrict__ up, int n, double dt, int adj, int m,
                                int P, int C, int L, double* __restrict__ coef,
                                double* __restrict__ lpcr, double* __restrict__ spk,
                                double* __restrict__ sup, int* __restrict__ status) {
  extern __shared__ double sh[];
  double* ag = sh;             // interface system (whole system)
  double* bg = ag + P;
  double* cg_ = bg + P;
  double* p0 = cg_ + P;
  double* q0 = p0 + P;
  double* la = q0 + P;         // local PCR state
  double* lb = la + P;
  double* lc = lb + P;
  double* r1 = lc + P;
  double* r2 = r1 + P;
  double* cEs = r2 + P;
  const int t = threadIdx.x;
  const int Pc = P / C, Pl = Pc - 1;
  const int c = t / Pc, tl = t % Pc;
  const int mi = m - 1;
  int bad = 0;
  double pl = 0, ql = 0, aE = 0, bE = 1, cE = 0;
  if (t < P) {
    const int r0 = t * m;
    double piv = b_di(di, n, dt, r0);
    if (!(fabs(piv) > 0.0) || !isfinite(piv)) bad = 1;
    double* cl = coef + cl_coef(c, 0, 0, tl, m, Pc);
    double* ci = coef + cl_coef(c, 1, 0, tl, m, Pc);
    double* cu = coef + cl_coef(c, 2, 0, tl, m, Pc);
    double* cp = coef + cl_coef(c, 3, 0, tl, m, Pc);
    double* cq = coef + cl_coef(c, 4, 0, tl, m, Pc);
    cl[0] = 0.0;
    ci[0] = 1.0 / piv;
    for (int i = 1; i < mi; ++i) {
      int r = r0 + i;
      double mult = b_lo(lo, up, n, dt, adj, r) / piv;
      piv = b_di(di, n, dt, r) - mult * b_up(lo, up, n, dt, adj, r - 1);
      if (!(fabs(piv) > 0.0) || !isfinite(piv)) bad = 1;
      cl[(size_t)i * Pc] = mult;
      ci[(size_t)i * Pc] = 1.0 / piv;
    }
    for (int i = 0; i < mi; ++i)
      cu[(size_t)i * Pc] = (i < mi - 1) ? b_up(lo, up, n, dt, adj, r0 + i) * ci[(size_t)i * Pc] : 0.0;
    const double left = b_lo(lo, up, n, dt, adj, r0);
    const double right = b_up(lo, up, n, dt, adj, r0 + mi - 1);
    double fp = left, fq = (mi == 1) ? right : 0.0;
    cp[0] = fp;
    cq[0] = fq;
    for (int i = 1; i < mi; ++i) {
      double mult = cl[(size_t)i * Pc];
      fp = 0.0 - mult * fp;
      fq = ((i == mi - 1) ? right : 0.0) - mult * fq;
      cp[(size_t)i * Pc] = fp;
      cq[(size_t)i * Pc] = fq;
    }
    double gp = 0.0, gq = 0.0;
    for (int i = mi - 1; i >= 0; --i) {
      size_t k = (size_t)i * Pc;
      gp = cp[k] * ci[k] - cu[k] * gp;
      gq = cq[k] * ci[k] - cu[k] * gq;
      cp[k] = gp;
      cq[k] = gq;
    }
    pl = cp[(size_t)(mi - 1) * Pc];
    ql = cq[(size_t)(mi - 1) * Pc];
    const int e = r0 + mi;
    aE = b_lo(lo, up, n, dt, adj, e);
    bE = b_di(di, n, dt, e);
    cE = b_up(lo, up, n, dt, adj, e);
    size_t k = (size_t)mi * Pc;
    cl[k] = aE;
    ci[k] = bE;
    cu[k] = cE;
    cp[k] = 0.0;
    cq[k] = 0.0;
    p0[t] = cp[0];
    q0[t] = cq[0];
    cEs[t] = cE;
  }
  __syncthreads();
  if (t < P) {
    double pn = (t + 1 < P) ? p0[t + 1] : 0.0;
    double qn = (t + 1 < P) ? q0[t + 1] : 0.0;
    ag[t] = -aE * pl;
    bg[t] = bE - aE * ql - cE * pn;
    cg_[t] = -cE * qn;
  }
  __syncthreads();
  // ---- local PCR factors over each CTA's unknowns tl = 0 .. Pl-1 -------------
  if (t < P) {
    la[t] = (tl > 0 && tl < Pl) ? ag[t] : 0.0;
    lb[t] = (tl < Pl) ? bg[t] : 1.0;
    lc[t] = (tl < Pl - 1) ? cg_[t] : 0.0;
  }
  __syncthreads();
  double* lp = lpcr + (size_t)c * (2 * L + 1) * Pc;
  for (int lev = 0, s = 1; lev < L; ++lev, s <<= 1) {
    double na = 0, nb = 1, nc = 0, k1 = 0, k2 = 0;
    if (t < P && tl < Pl) {
      double a = la[t], b = lb[t], cc = lc[t];
      double a1 = 0, b1 = 1, c1 = 0, a2 = 0, b2 = 1, c2 = 0;
      bool hm = tl - s >= 0, hp = tl + s < Pl;
      if (hm) { a1 = la[t - s]; b1 = lb[t - s]; c1 = lc[t - s]; }
      if (hp) { a2 = la[t + s]; b2 = lb[t + s]; c2 = lc[t + s]; }
      k1 = hm ? a / b1 : 0.0;
      k2 = hp ? cc / b2 : 0.0;
      na = -k1 * a1;
      nc = -k2 * c2;
      nb = b - k1 * c1 - k2 * a2;
      if (!(fabs(nb) > 0.0) || !isfinite(nb)) bad = 1;
    }
    if (t < P) {
      lp[(size_t)lev * Pc + tl] = k1;
      lp[(size_t)(L + lev) * Pc + tl] = k2;
    }
    __syncthreads();
    if (t < P && tl < Pl) { la[t] = na; lb[t] = nb; lc[t] = nc; }
    __syncthreads();
  }
  if (t < P) {
    if (tl < Pl && (!(fabs(lb[t]) > 0.0) || !isfinite(lb[t]))) bad = 1;
    lp[(size_t)(2 * L) * Pc + tl] = (tl < Pl) ? 1.0 / lb[t] : 0.0;
  }
  // ---- spikes of the local systems: P2 (left coupling), Q2 (right) ----------
  if (t < P) {
    r1[t] = (tl == 0 && Pl > 0) ? ag[t] : 0.0;
    r2[t] = (tl == Pl - 1) ? cg_[t] : 0.0;
  }
  __syncthreads();
  for (int lev = 0, s = 1; lev < L; ++lev, s <<= 1) {
    double n1 = 0, n2 = 0;
    if (t < P && tl < Pl) {
      double k1 = lp[(size_t)lev * Pc + tl], k2 = lp[(size_t)(L + lev) * Pc + tl];
      double m1 = tl - s >= 0 ? r1[t - s] : 0.0, m2 = tl - s >= 0 ? r2[t - s] : 0.0;
      double p1 = tl + s < Pl ? r1[t + s] : 0.0, p2 = tl + s < Pl ? r2[t + s] : 0.0;
      n1 = r1[t] - k1 * m1 - k2 * p1;
      n2 = r2[t] - k1 * m2 - k2 * p2;
    }
    __syncthreads();
    if (t < P && tl < Pl) { r1[t] = n1; r2[t] = n2; }
    __syncthreads();
  }
  if (t < P) {
    double dv = (tl < Pl) ? lp[(size_t)(2 * L) * Pc + tl] : 0.0;
    spk[((size_t)c * 2 + 0) * Pc + tl] = r1[t] * dv;
    spk[((size_t)c * 2 + 1) * Pc + tl] = r2[t] * dv;
  }
  __syncthreads();
  // ---- super system over the last interface unknown of every CTA ------------
  if (t == 0) {
    double piv_prev = 1.0, gs_prev = 0.0;
    for (int cc = 0; cc < C; ++cc) {
      int tc = cc * Pc + Pc - 1;
      double P2l = spk[((size_t)cc * 2 + 0) * Pc + Pl - 1];
      double Q2l = spk[((size_t)cc * 2 + 1) * Pc + Pl - 1];
      double P2n = cc + 1 < C ? spk[((size_t)(cc + 1) * 2 + 0) * Pc + 0] : 0.0;
      double Q2n = cc + 1 < C ? spk[((size_t)(cc + 1) * 2 + 1) * Pc + 0] : 0.0;
      double as = -ag[tc] * P2l;
      double bs = bg[tc] - ag[tc] * Q2l - cg_[tc] * P2n;
      double gs = -cg_[tc] * Q2n;
      double mult = cc > 0 ? as / piv_prev : 0.0;
      double piv = bs - mult * gs_prev;
      if (!(fabs(piv) > 0.0) || !isfinite(piv)) bad = 1;
      double* su = sup + (size_t)cc * 6;
      su[0] = ag[tc];
      su[1] = cg_[tc];
      su[2] = cEs[tc];
      su[3] = mult;
      su[4] = 1.0 / piv;
      su[5] = gs;
      piv_prev = piv;
      gs_prev = gs;
    }
    // dense inverse of the C x C super system (columns: solves with e_p), so
    // that every step solves it with one short product per CTA
    double* minv = sup + 6 * CL_MAXC;
    for (int pcol = 0; pcol < C; ++pcol) {
      double w[CL_MAXC];
      for (int q = 0; q < C; ++q)
        w[q] = (q == pcol ? 1.0 : 0.0) - (q > 0 ? sup[(size_t)q * 6 + 3] * w[q - 1] : 0.0);
      double Y = 0.0;
      for (int q = C - 1; q >= 0; --q) {
        Y = (w[q] - (q + 1 < C ? sup[(size_t)q * 6 + 5] * Y : 0.0)) * sup[(size_t)q * 6 + 4];
        minv[q * CL_MAXC + pcol] = Y;
      }
    }
  }
  if (bad) atomicOr(status, 1);
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b[k] = (float)a[k];
}

// ---------------------------------------------------------------------------
// Propagation kernel: cluster of C CTAs per system, blockDim = Pc (one chunk
// per thread).  Clusters loop over systems.
// ---------------------------------------------------------------------------

// SPT systems per thread: a cluster advances SPT independent systems in
// lockstep, so that every thread has SPT independent dependency chains (FP64
// latency is exposed with one warp per scheduler) and the factors read from
// shared memory serve SPT systems.
template <typename T, int MM, int SPT, bool SDIRK = false>
__global__ void __launch_bounds__(256) k_tri_cluster(ClKArgs a) {
  if (a.in.stop && *a.in.stop) return;   // the iteration has stopped on the device
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Pc = a.Pc, L = a.L, C = a.C, Pl = Pc - 1;
  const int c = (int)cl.block_rank();
  T* s_coef = reinterpret_cast<T*>(smem_raw);            // [5][MM][Pc]
  T* s_pcr = s_coef + 5 * MM * Pc;                        // [2L+1][Pc]
  T* s_spk = s_pcr + (2 * L + 1) * Pc;                    // [2][Pc]
  T* s_sup = s_spk + 2 * Pc;                              // [C][6]
  T* xb = s_sup + 6 * CL_MAXC + CL_MAXC * CL_MAXC;        // [SPT][3][Pc]
  T* Ysh = xb + SPT * 3 * Pc;                             // [SPT][CL_MAXC]
  // values every CTA publishes for the super system, pushed into the shared
  // memory of all CTAs of the cluster before the barrier (no remote read on
  // the critical path after it): pubg[parity][system][cta][4]
  __shared__ double pubg[2][SPT][CL_MAXC][4];
  __shared__ double* rpub[CL_MAXC];
  {
    const T* gco = static_cast<const T*>(a.coef) + (size_t)c * 5 * MM * Pc;
    const T* gpc = static_cast<const T*>(a.lpcr) + (size_t)c * (2 * L + 1) * Pc;
    const T* gsp = static_cast<const T*>(a.spk) + (size_t)c * 2 * Pc;
    const T* gsu = static_cast<const T*>(a.sup);
    for (int k = threadIdx.x; k < 5 * MM * Pc; k += blockDim.x) s_coef[k] = gco[k];
    for (int k = threadIdx.x; k < (2 * L + 1) * Pc; k += blockDim.x) s_pcr[k] = gpc[k];
    for (int k = threadIdx.x; k < 2 * Pc; k += blockDim.x) s_spk[k] = gsp[k];
    for (int k = threadIdx.x; k < 6 * CL_MAXC + CL_MAXC * CL_MAXC; k += blockDim.x) s_sup[k] = gsu[k];
    for (int q = threadIdx.x; q < C; q += blockDim.x) rpub[q] = cl.map_shared_rank(&pubg[0][0][0][0], q);
  }
  cl.sync();   // every CTA of the cluster runs before any remote store into its shared memory
  const int tl = threadIdx.x;
  const int t = c * Pc + tl;
  const T* cl_ = s_coef;
  const T* ci = s_coef + MM * Pc;
  const T* cu = s_coef + 2 * MM * Pc;
  const T* cp = s_coef + 3 * MM * Pc;
  const T* cq = s_coef + 4 * MM * Pc;
  const T dt = (T)a.dt;
  const int n = a.n;
  const int r0 = t * MM;
  const int nclu = gridDim.x / C;
  int pb = 0;
  for (int base = (blockIdx.x / C) * SPT; base < a.nsys; base += nclu * SPT) {
    T x[SPT][MM];
    const double* csys[SPT];
    const double* gsys[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int sys = base + s;
      const bool act = sys < a.nsys;
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        int r = r0 + i;
        T v = T(0);
        if (act && r < n) {
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
      csys[s] = (act && a.src.Q > 0)
          ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
      gsys[s] = (act && a.src.Q > 0 && a.src.map)
          ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
    }
    // one solve with the plan's matrix, in place on x (one cluster barrier)
    auto solve = [&](T (&x)[SPT][MM]) {
      // interior forward elimination and back substitution (SPT chains)
#pragma unroll
      for (int i = 1; i < MM - 1; ++i) {
        const T l = cl_[i * Pc + tl];
#pragma unroll
        for (int s = 0; s < SPT; ++s) x[s][i] -= l * x[s][i - 1];
      }
      {
        const T iv = ci[(MM - 2) * Pc + tl];
#pragma unroll
        for (int s = 0; s < SPT; ++s) x[s][MM - 2] *= iv;
      }
#pragma unroll
      for (int i = MM - 3; i >= 0; --i) {
        const T iv = ci[i * Pc + tl], u = cu[i * Pc + tl];
#pragma unroll
        for (int s = 0; s < SPT; ++s) x[s][i] = x[s][i] * iv - u * x[s][i + 1];
      }
#pragma unroll
      for (int s = 0; s < SPT; ++s) xb[(s * 3 + 2) * Pc + tl] = x[s][0];
      __syncthreads();
      T r[SPT];
      const T aE = cl_[(MM - 1) * Pc + tl], cE = cu[(MM - 1) * Pc + tl];
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        T gnext = (tl + 1 < Pc) ? xb[(s * 3 + 2) * Pc + tl + 1] : T(0);
        r[s] = x[s][MM - 1] - aE * x[s][MM - 2] - cE * gnext;
      }
      // local parallel cyclic reduction (unknowns 0 .. Pl-1 of this CTA)
      int buf = 0;
      for (int lev = 0, sh = 1; lev < L; ++lev, sh <<= 1) {
#pragma unroll
        for (int s = 0; s < SPT; ++s) xb[(s * 3 + buf) * Pc + tl] = r[s];
        __syncthreads();
        if (tl < Pl) {
          const T k1 = s_pcr[lev * Pc + tl], k2 = s_pcr[(L + lev) * Pc + tl];
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            T rm = (tl - sh >= 0) ? xb[(s * 3 + buf) * Pc + tl - sh] : T(0);
            T rp = (tl + sh < Pl) ? xb[(s * 3 + buf) * Pc + tl + sh] : T(0);
            r[s] = r[s] - k1 * rm - k2 * rp;
          }
        }
        buf ^= 1;
      }
      T z0[SPT];
      const T dv = (tl < Pl) ? s_pcr[2 * L * Pc + tl] : T(0);
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        z0[s] = (tl < Pl) ? r[s] * dv : T(0);
        const int o = ((pb * SPT + s) * CL_MAXC + c) * 4;
        if (tl == 0) {
          for (int q = 0; q < C; ++q) { rpub[q][o + 0] = (double)z0[s]; rpub[q][o + 3] = (double)x[s][0]; }
        }
        if (tl == Pl - 1)
          for (int q = 0; q < C; ++q) rpub[q][o + 1] = (double)z0[s];
        if (tl == Pc - 1)
          for (int q = 0; q < C; ++q) rpub[q][o + 2] = (double)r[s];
      }
      cl.sync();
      if (tl < SPT * C) {
        // lane s*C + q forms the right-hand side of super unknown q of system
        // s, the C lanes of a system exchange them by shuffles and each
        // applies one row of the precomputed inverse
        const int s = tl / C, q = tl % C;
        const double* pq = &pubg[pb][s][q][0];
        double rhs = pq[2] - (double)s_sup[6 * q] * pq[1];
        if (q + 1 < C) {
          const double* pn = &pubg[pb][s][q + 1][0];
          rhs -= (double)s_sup[6 * q + 2] * pn[3] + (double)s_sup[6 * q + 1] * pn[0];
        }
        const unsigned mask = (SPT * C >= 32) ? 0xffffffffu : ((1u << (SPT * C)) - 1u);
        const T* minv = s_sup + 6 * CL_MAXC + q * CL_MAXC;
        double Y = 0.0;
#pragma unroll
        for (int pcol = 0; pcol < CL_MAXC; ++pcol) {
          if (pcol < C) {
            double rp = __shfl_sync(mask, rhs, s * C + pcol);
            Y += (double)minv[pcol] * rp;
          }
        }
        Ysh[s * CL_MAXC + q] = (T)Y;
      }
      __syncthreads();
      T y[SPT], Yl[SPT];
      const T p2 = s_spk[tl], q2 = s_spk[Pc + tl];
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        Yl[s] = c > 0 ? Ysh[s * CL_MAXC + c - 1] : T(0);
        const T Yc = Ysh[s * CL_MAXC + c];
        y[s] = (tl < Pl) ? z0[s] - p2 * Yl[s] - q2 * Yc : Yc;
        xb[(s * 3 + buf) * Pc + tl] = y[s];
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        const T yl = (tl > 0) ? xb[(s * 3 + buf) * Pc + tl - 1] : Yl[s];
#pragma unroll
        for (int i = 0; i < MM - 1; ++i) x[s][i] = x[s][i] - cp[i * Pc + tl] * yl - cq[i * Pc + tl] * y[s];
        x[s][MM - 1] = y[s];
      }
      pb ^= 1;
    };
    for (int j = 0; j < a.M; ++j) {
      if constexpr (!SDIRK) {
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
        solve(x);
      } else {
        // two-stage SDIRK, both stages with the same matrix B = I + gamma dt A;
        // the source of stage i, sampled at its stage time (two samples per
        // step), enters its right-hand side as gamma dt f_i (dt here is the
        // plan's gamma dt)
        auto add_source = [&](int stage) {
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            if (!csys[s]) continue;
            for (int q = 0; q < a.src.Q; ++q) {
              T cq_ = dt * (T)csys[s][((size_t)j * 2 + stage) * a.src.Q + q];
              const double* gq = gsys[s] + (size_t)q * n;
#pragma unroll
              for (int i = 0; i < MM; ++i)
                if (r0 + i < n) x[s][i] += cq_ * (T)gq[r0 + i];
            }
          }
        };
        T u[SPT][MM], u1[SPT][MM];
#pragma unroll
        for (int s = 0; s < SPT; ++s)
#pragma unroll
          for (int i = 0; i < MM; ++i) u[s][i] = x[s][i];
        add_source(0);
        solve(x);
#pragma unroll
        for (int s = 0; s < SPT; ++s)
#pragma unroll
          for (int i = 0; i < MM; ++i) {
            u1[s][i] = x[s][i];
            x[s][i] = (T)a.su * u[s][i] + (T)a.s1 * x[s][i];
          }
        add_source(1);
        solve(x);
#pragma unroll
        for (int s = 0; s < SPT; ++s)
#pragma unroll
          for (int i = 0; i < MM; ++i)
            x[s][i] = (T)a.bu * u[s][i] + (T)a.b1 * u1[s][i] + (T)a.b2 * x[s][i];
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
  cl.sync();  // remote reads of pub have finished before any CTA exits
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
lrp_status tri_get_cluster_plan(Ctx* c, Operator* op, double dt, int adjoint, int C, int m,
                                ClPlan** out, int warp) {
  const int CL_M = m;
  std::lock_guard<std::mutex> plan_lock(op->plan_mu);
  for (auto& p : op->cplans)
    if (p->dt == dt && p->adjoint == adjoint && p->C == C && p->m == m && p->warp == warp) {
      *out = p.get();
      return LRP_OK;
    }
  auto pl = std::make_unique<ClPlan>();
  pl->dt = dt;
  pl->adjoint = adjoint;
  pl->C = C;
  pl->n = op->n;
  pl->m = CL_M;
  pl->warp = warp;
  int P = (op->n + CL_M - 1) / CL_M;
  P = (P + C - 1) / C * C;
  if (warp) {
    // one warp per CTA: exactly 32 chunks of 8 rows per CTA (padding chunks
    // are identity rows)
    if (CL_M < 8 || CL_M > 16 || P > 32 * C)
      return set_err(c, LRP_EINVAL, "warp cluster plan out of range");
    P = 32 * C;
  }
  pl->P = P;
  pl->Pc = P / C;
  if (pl->Pc < 32 || pl->Pc > 256 || P > 1024)
    return set_err(c, LRP_EINVAL, "cluster tridiagonal plan out of range");
  int L = 0;
  while ((1 << L) < pl->Pc - 1) ++L;
  pl->L = L;
  const size_t ncoef = (size_t)5 * CL_M * P, npcr = (size_t)C * (2 * L + 1) * pl->Pc,
               nspk = (size_t)2 * P, nsup = 6 * CL_MAXC + CL_MAXC * CL_MAXC;
  pl->sz[0] = ncoef; pl->sz[1] = npcr; pl->sz[2] = nspk; pl->sz[3] = nsup;
  lrp_status s;
  for (int k = 0; k < 4; ++k) {
    if ((s = dev_alloc(op->ctx, pl->b64[k], pl->sz[k] * 8))) return s;
    if ((s = dev_alloc(op->ctx, pl->b32[k], pl->sz[k] * 4))) return s;
    cudaMemsetAsync(pl->b64[k].ptr, 0, pl->sz[k] * 8, c->stream);
  }
  if ((s = dev_alloc(op->ctx, pl->status, sizeof(int)))) return s;
  cudaMemsetAsync(pl->status.ptr, 0, sizeof(int), c->stream);
  int threads = ((P + 31) / 32) * 32;
  cudaError_t e0 = cudaFuncSetAttribute(k_tri_factor_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(11 * P * sizeof(double)));
  if (e0) return cuda_err(c, e0, "cluster factor smem attribute");
  k_tri_factor_cl<<<1, threads, 11 * P * sizeof(double), c->stream>>>(
      op->a64[0].as<double>(), op->a64[1].as<double>(), op->a64[2].as<double>(), op->n, dt,
      adjoint, CL_M, P, C, L, pl->b64[0].as<double>(), pl->b64[1].as<double>(),
      pl->b64[2].as<double>(), pl->b64[3].as<double>(), pl->status.as<int>());
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_err(c, e, "k_tri_factor_cl launch");
  for (int k = 0; k < 4; ++k)
    k_to_f32<<<(unsigned)((pl->sz[k] + 255) / 256), 256, 0, c->stream>>>(
        pl->b64[k].as<double>(), pl->b32[k].as<float>(), pl->sz[k]);
  int st = 0;
  e = cudaMemcpyAsync(&st, pl->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "k_tri_factor_cl");
  if (st) return set_err(c, LRP_EBREAKDOWN, "zero pivot in the tridiagonal factorisation");
  *out = pl.get();
  op->cplans.push_back(std::move(pl));
  return LRP_OK;
}

template <typename T, int MM, int SPT, bool SDIRK = false>
static lrp_status launch_cl(Ctx* c, ClPlan* pl, ClKArgs& a) {
  const int Pc = pl->Pc, L = pl->L, C = pl->C;
  size_t smem = sizeof(T) * ((size_t)5 * MM * Pc + (size_t)(2 * L + 1) * Pc + 2 * Pc +
                             6 * CL_MAXC + CL_MAXC * CL_MAXC + (size_t)SPT * 3 * Pc +
                             (size_t)SPT * CL_MAXC);
  auto kern = k_tri_cluster<T, MM, SPT, SDIRK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return cuda_err(c, e, "cluster tri smem attribute");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(Pc);
  cfg.gridDim = dim3(C);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  int maxc = 0;
  e = cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg);
  if (e || maxc < 1) { cudaGetLastError(); maxc = std::max(1, c->num_sms / C); }
  const int groups = (a.nsys + SPT - 1) / SPT;
  const int ncl = std::min(groups, maxc);
  cfg.gridDim = dim3(ncl * C);
  const char* fam = sizeof(T) == 8 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  e = cudaLaunchKernelEx(&cfg, kern, a);
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_tri_cluster launch");
  return LRP_OK;
}

lrp_status tri_propagate_warp_block(Ctx* c, ClPlan* pl, int M, int nsys, int prec,
                                    const PropIn& in, const PropOut& out, const PropSrc& src,
                                    const ToepCoef* tz) {
  if (nsys <= 0) return LRP_OK;
  if (!pl->warp) return set_err(c, LRP_EINVAL, "block warp kernel needs a warp plan");
  ClKArgs a{};
  a.n = pl->n;
  a.Pc = pl->Pc;
  a.C = pl->C;
  a.L = pl->L;
  a.M = M;
  a.nsys = nsys;
  a.dt = pl->dt;
  a.in = in;
  a.out = out;
  a.src = src;
  DevBuf* b = prec == 0 ? pl->b64 : pl->b32;
  a.coef = b[0].ptr;
  a.lpcr = b[1].ptr;
  a.spk = b[2].ptr;
  a.sup = b[3].ptr;
  if (tz && tz->on) {
    a.tz = *tz;
    return prec == 0 ? tri_launch_warp_block_toep<double>(c, pl, a)
                     : tri_launch_warp_block_toep<float>(c, pl, a);
  }
  return prec == 0 ? tri_launch_warp_block<double>(c, pl, a) : tri_launch_warp_block<float>(c, pl, a);
}

lrp_status tri_propagate_cluster(Ctx* c, ClPlan* pl, int M, int nsys, int prec, int spt,
                                 const PropIn& in, const PropOut& out, const PropSrc& src,
                                 int stepper, const ToepCoef* tz) {
  if (nsys <= 0) return LRP_OK;
  ClKArgs a{};
  a.n = pl->n;
  a.Pc = pl->Pc;
  a.C = pl->C;
  a.L = pl->L;
  a.M = M;
  a.nsys = nsys;
  a.dt = pl->dt;
  a.in = in;
  a.out = out;
  a.src = src;
  const int f = prec == 0 ? 0 : 1;
  DevBuf* b = f ? pl->b32 : pl->b64;
  a.coef = b[0].ptr;
  a.lpcr = b[1].ptr;
  a.spk = b[2].ptr;
  a.sup = b[3].ptr;
  if (stepper) {
    if (pl->warp || pl->m != 8) return set_err(c, LRP_EINVAL, "SDIRK cluster propagation needs 8-row chunks");
    const StepCoef sc = step_coefficients(stepper);
    a.su = sc.su; a.s1 = sc.s1; a.bu = sc.bu; a.b1 = sc.b1; a.b2 = sc.b2;
    return f ? launch_cl<float, 8, 1, true>(c, pl, a) : launch_cl<double, 8, 1, true>(c, pl, a);
  }
  if (pl->warp) {
    if (f || spt != 1) return set_err(c, LRP_EINVAL, "warp cluster kernel is FP64, one system per thread");
    if (tz && tz->on) {
      a.tz = *tz;
      return tri_launch_warp_toep(c, pl, a);
    }
    return c->p_tri_wsplit ? tri_launch_warp<1>(c, pl, a) : tri_launch_warp<0>(c, pl, a);
  }
  if (pl->m == 8) {
    if (spt == 2) return f ? launch_cl<float, 8, 2>(c, pl, a) : launch_cl<double, 8, 2>(c, pl, a);
    return f ? launch_cl<float, 8, 1>(c, pl, a) : launch_cl<double, 8, 1>(c, pl, a);
  }
  if (spt == 2) return f ? launch_cl<float, 16, 2>(c, pl, a) : launch_cl<double, 16, 2>(c, pl, a);
  return f ? launch_cl<float, 16, 1>(c, pl, a) : launch_cl<double, 16, 1>(c, pl, a);
}

}  // namespace lrp
