// Coarse sweep fused with the Parareal correction, in the delta form of
// Remark rem:affine_g_n:
//   u^k_{i+1} = F_i u^{k-1}_i + G_i'(u^k_i - u^{k-1}_i),  G_i' = U_i diag(S_i) V_i^T,
// and, for the initial sweep, u^0_{i+1} = b_i + G_i' u^0_i (Eq. def_Parareal
// with u^{-1} := 0), together with the norms ||u^k_m - u^{k-1}_m||, ||u^k_m||
// and the a posteriori bound of Eq. apost_bound through its recurrence
// B_n = delta B_{n-1} + eps ||u^k_{n-1} - u^{k-1}_{n-1}||.
//
// Evaluated in the coordinates of the low-rank factors.  With
// Delta_i = u^k_i - u^{k-1}_i and c_i = V_i^T Delta_i (an R-vector),
//   Delta_{i+1} = r_i + U_i diag(S_i) c_i,   r_i = F_i u^{k-1}_i - u^{k-1}_{i+1},
// so  c_{i+1} = V_{i+1}^T r_i + K_i c_i  with  K_i = V_{i+1}^T U_i diag(S_i).
// The K_i (R x R) depend only on the factors and are formed once per coarse
// handle.  The sequential dependence of the sweep is then an R-dimensional
// recurrence; everything of size n runs in parallel over all intervals:
//   1. project:  a_{i+1} = V_{i+1}^T r_i for every interval (all SMs);
//   2. recur:    c_{i+1} = a_{i+1} + K_i c_i (one CTA, R x R steps, in the
//                precision of the coarse apply);
//   3. apply:    u^k_{i+1} = F_i u^{k-1}_i + U_i (S_i * c_i) for every
//                interval, with the norms; then the bound recurrence.
// Steps 1+2 and 3+bound are one launch each: the CTA that finishes a launch's
// partial sums last (device-scope counter, no waiting) runs the sequential
// part.  Partial sums are per (interval, row slice) and are added in a fixed
// order, so results do not depend on scheduling or on which other problems
// share a launch.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace lrp {

constexpr int CSW_THREADS = 256;
constexpr int CSW_MAXROWS = 2048;    // rows per slice (upper limit)
constexpr int CSW_MAXR = 64;
constexpr int CSW_KBUF = 96 * 1024;  // bytes of K staged per chunk of the recurrence
constexpr int CSW_MAXN = 8192;       // intervals + 1 (norms staged in shared memory)
constexpr int CSW_RPT = 4;           // rows per thread in flight in the apply

// Workspace of one problem (doubles): a-partials [N][nsl][R], coefficients
// [N][R], norm partials [N+1][nsl][2].
__host__ __device__ inline size_t csw_coef(int N, int nsl, int R) { return (size_t)N * nsl * R; }
__host__ __device__ inline size_t csw_npart(int N, int nsl, int R) { return csw_coef(N, nsl, R) + (size_t)N * R; }
size_t sweep_ws_doubles(int N, int nsl, int R) { return csw_npart(N, nsl, R) + (size_t)(N + 1) * nsl * 2; }

int sweep_rows(Ctx* c) { return c->p_sweep_rows > 0 ? c->p_sweep_rows : 1024; }
int sweep_slices(Ctx* c, int n) { const int sl = sweep_rows(c); return (n + sl - 1) / sl; }

// The CTA that completes a launch's partial sums for its problem last: every
// CTA of the problem adds one to the counter after its partial sums are
// visible device-wide.  Returns true in exactly one CTA, which also resets the
// counter for the next launch.
__device__ __forceinline__ bool csw_last_cta(unsigned* cnt, unsigned total) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(cnt, 1u);
    last = (t == total - 1) ? 1 : 0;
    if (last) *cnt = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

// ---------------------------------------------------------------------------
// 1 + 2: projections and the coefficient recurrence.
// grid (slices, N, problems); blockIdx.y = j, the index of a_j.
// ---------------------------------------------------------------------------
template <typename TF>
__global__ void __launch_bounds__(CSW_THREADS) k_csw_project(const SweepArgs* __restrict__ args) {
  extern __shared__ __align__(16) unsigned char csw_smem[];
  __shared__ TF vs[CSW_MAXROWS];
  __shared__ TF cbuf[2][CSW_MAXR];
  const SweepArgs& a = args[blockIdx.z];
  if (a.stop && *a.stop) return;             // the iteration has stopped on the device
  const int j = blockIdx.y, sl = blockIdx.x;
  const int N = a.N, n = a.n, R = a.R, nsl = a.nsl;
  const int start = a.initial ? 0 : a.first;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* apart = a.cw;
  if (j < N && sl < nsl && (j > start || (a.initial && j == 0))) {
    const int lo = sl * a.rows, hi = min(n, lo + a.rows), rows = hi - lo;
    // the vector to project: u0 (initial, j = 0), else r_{j-1}
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      double v;
      if (j == 0) {
        v = a.u[lo + i];
      } else {
        v = a.F[(size_t)(j - 1) * n + lo + i];
        if (!a.initial) v -= a.u[(size_t)j * n + lo + i];
      }
      vs[i] = (TF)v;
    }
    __syncthreads();
    const TF* Vj = static_cast<const TF*>(a.V) + (size_t)j * R * n + lo;
    for (int r = w; r < R; r += nw) {
      const TF* vr = Vj + (size_t)r * n;
      TF acc = TF(0);
      for (int i = lane; i < rows; i += 32) acc += vr[i] * vs[i];
      acc = warp_sum<TF>(acc);
      if (lane == 0) apart[((size_t)j * nsl + sl) * R + r] = (double)acc;
    }
  }
  if (!csw_last_cta(&a.cnt[0], gridDim.x * gridDim.y)) return;
  // ---- the recurrence (this CTA only) ---------------------------------------
  double* coef = a.cw + csw_coef(N, nsl, R);
  // a_j is the fixed-order sum of its slice partials (summed where staged)
  auto a_sum = [&](int jj, int r) {
    double sum = 0.0;
    if (jj > start || a.initial)
      for (int q = 0; q < nsl; ++q) sum += __ldcg(&apart[((size_t)jj * nsl + q) * R + r]);
    return sum;
  };
  // c_start = a_start (initial: V_0^T u0) or 0; c_j = a_j + K_{j-1} c_{j-1}.
  // K_{j-1} and a_j of a chunk of steps are staged in shared memory, so the
  // sequential steps touch no global memory.
  // The recurrence runs in the precision of the coarse apply (TF: FP32 in
  // the mixed mode, where G' is applied in FP32; FP64 otherwise).
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const TF c0 = (TF)a_sum(start, r);
    cbuf[0][r] = c0;
    coef[(size_t)start * R + r] = (double)c0;
  }
  TF* sK = reinterpret_cast<TF*>(csw_smem);
  // K_j staged with row stride R + 1 (the one-warp recurrence reads a column
  // of K_j per FMA: rows r = 0..15 then fall in distinct banks)
  const int KS = R * (R + 1);
  const int kchunk = max(1, CSW_KBUF / (int)(sizeof(TF) * (KS + R)));
  TF* sA = sK + (size_t)kchunk * KS;
  const int t = threadIdx.x, rr = t >> 2, part = t & 3;
  int cb = 0;
  for (int j0 = start + 1; j0 < N; j0 += kchunk) {
    const int nk = min(kchunk, N - j0);
    __syncthreads();
    const double* Kg = a.K + (size_t)(j0 - 1) * R * R;
    // sixteen loads in flight per thread (this CTA stages alone while the
    // other CTAs of the launch have finished)
    const int nkr = nk * R * R;
    for (int k0 = threadIdx.x; k0 < nkr; k0 += 16 * blockDim.x) {
      double v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int k = k0 + u * blockDim.x;
        v[u] = k < nkr ? __ldcg(&Kg[k]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int k = k0 + u * blockDim.x;
        if (k < nkr) sK[(k / R) * (R + 1) + k % R] = (TF)v[u];
      }
    }
    const int na = nk * R;
    for (int k0 = threadIdx.x; k0 < na; k0 += 8 * blockDim.x) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u * blockDim.x;
        v[u] = k < na ? a_sum(j0 + k / R, k % R) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u * blockDim.x;
        if (k < na) sA[k] = (TF)v[u];
      }
    }
    __syncthreads();
    if (R <= 16) {
      // one warp, no block barrier: row r of K c on the two lanes r and
      // r + 16, lane group g taking columns q = g, g + 2, ...; c_q comes from
      // lane q by a shuffle; the two partial sums are added by one butterfly
      if (threadIdx.x < 32) {
        const int r = lane & 15, g = lane >> 4;
        TF cr = r < R ? cbuf[cb][r] : TF(0);
        for (int jj = 0; jj < nk; ++jj) {
          const TF* Kj = sK + (size_t)jj * KS + r * (R + 1);
          TF cq[8], kq[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int q = 2 * t + g;
            cq[t] = __shfl_sync(0xffffffffu, cr, q);
            kq[t] = (r < R && q < R) ? Kj[q] : TF(0);
          }
          TF acc = TF(0);
#pragma unroll
          for (int t = 0; t < 8; ++t) acc = fma(kq[t], cq[t], acc);
          acc += __shfl_xor_sync(0xffffffffu, acc, 16);
          if (r < R) cr = sA[(size_t)jj * R + r] + acc;
          __syncwarp();
          if (r < R && g == 0) sA[(size_t)jj * R + r] = cr;
        }
        if (r < R && g == 0) cbuf[cb][r] = cr;
      }
      __syncthreads();
    } else
    for (int jj = 0; jj < nk; ++jj) {
      const TF* Kj = sK + (size_t)jj * KS;
      // rows rr = 0..R-1 of K c, four threads per row (interleaved columns),
      // combined by shuffles in a fixed order
      for (int rb = 0; rb < R; rb += CSW_THREADS / 4) {
        const int r = rb + rr;
        TF acc = TF(0);
        if (r < R)
          for (int q = part; q < R; q += 4) acc = fma(Kj[r * (R + 1) + q], cbuf[cb][q], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (r < R && part == 0) {
          const TF cv = sA[(size_t)jj * R + r] + acc;
          cbuf[cb ^ 1][r] = cv;
          sA[(size_t)jj * R + r] = cv;
        }
      }
      cb ^= 1;
      __syncthreads();
    }
    for (int k = threadIdx.x; k < nk * R; k += blockDim.x) coef[(size_t)j0 * R + k] = (double)sA[k];
  }
}

// ---------------------------------------------------------------------------
// 3: apply, norms and the bound.  grid (slices, N + 1, problems);
// blockIdx.y - 1 = j, the interval whose end value u_{j+1} is formed
// (j = start - 1: only the norm of the unchanged u_start).
// ---------------------------------------------------------------------------
template <typename TF>
__global__ void __launch_bounds__(CSW_THREADS) k_csw_apply(const SweepArgs* __restrict__ args) {
  __shared__ TF sc[CSW_MAXR];
  __shared__ double red[CSW_THREADS / 32][2];
  const SweepArgs& a = args[blockIdx.z];
  if (a.stop && *a.stop) return;             // the iteration has stopped on the device
  const int j = (int)blockIdx.y - 1, sl = blockIdx.x;
  const int N = a.N, n = a.n, R = a.R, nsl = a.nsl;
  const int start = a.initial ? 0 : a.first;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* npart = a.cw + csw_npart(N, nsl, R);
  if (j < N && sl < nsl && j >= start - 1) {
    const int lo = sl * a.rows, hi = min(n, lo + a.rows), rows = hi - lo;
    TF accd = TF(0), accu = TF(0);
    if (j == start - 1) {
      const double* us = a.u + (size_t)start * n + lo;
      for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const TF v = (TF)us[i];
        accu += v * v;
      }
      if (a.initial) accd = accu;          // Delta_0 = u0 - 0
    } else {
      const double* coef = a.cw + csw_coef(N, nsl, R) + (size_t)j * R;
      const TF* S = static_cast<const TF*>(a.S) + (size_t)j * R;
      for (int r = threadIdx.x; r < R; r += blockDim.x) sc[r] = S[r] * (TF)__ldcg(&coef[r]);
      __syncthreads();
      const TF* Uj = static_cast<const TF*>(a.U) + (size_t)j * R * n + lo;
      const double* Fj = a.F + (size_t)j * n + lo;
      double* un = a.u + (size_t)(j + 1) * n + lo;
      // CSW_RPT rows per thread at once, so that all their loads are in flight
      for (int i0 = threadIdx.x; i0 < rows; i0 += CSW_RPT * blockDim.x) {
        TF g[CSW_RPT];
        double fv[CSW_RPT], ov[CSW_RPT];
#pragma unroll
        for (int k = 0; k < CSW_RPT; ++k) {
          const int i = i0 + k * blockDim.x;
          g[k] = TF(0);
          fv[k] = i < rows ? Fj[i] : 0.0;
          ov[k] = (i < rows && !a.initial) ? un[i] : 0.0;
        }
        for (int r = 0; r < R; ++r) {
          const TF sr = sc[r];
          const TF* ur = Uj + (size_t)r * n;
#pragma unroll
          for (int k = 0; k < CSW_RPT; ++k) {
            const int i = i0 + k * blockDim.x;
            if (i < rows) g[k] += ur[i] * sr;
          }
        }
#pragma unroll
        for (int k = 0; k < CSW_RPT; ++k) {
          const int i = i0 + k * blockDim.x;
          if (i < rows) {
            const double nv = fv[k] + (double)g[k];
            un[i] = nv;
            const TF d = (TF)(nv - ov[k]), u = (TF)nv;
            accd += d * d;
            accu += u * u;
          }
        }
      }
    }
    accd = warp_sum<TF>(accd);
    accu = warp_sum<TF>(accu);
    if (lane == 0) { red[w][0] = (double)accd; red[w][1] = (double)accu; }
    __syncthreads();
    if (threadIdx.x < 2) {
      double s = 0.0;
      for (int k = 0; k < nw; ++k) s += red[k][threadIdx.x];
      npart[((size_t)(j + 1) * nsl + sl) * 2 + threadIdx.x] = s;
    }
  }
  if (!csw_last_cta(&a.cnt[1], gridDim.x * gridDim.y)) return;
  // ---- norms, bound recurrence and summary (this CTA only) -------------------
  extern __shared__ double csw_nrm[];          // [2][N + 1]: ||Delta_m||, ||u_m||
  double* sdu = csw_nrm;
  double* sun = csw_nrm + (N + 1);
  double umax_t = 0.0;
  for (int m = threadIdx.x; m <= N; m += blockDim.x) {
    double dm = 0.0, um;
    if (m >= start) {
      double sd = 0.0, su = 0.0;
      for (int q = 0; q < nsl; ++q) {
        sd += __ldcg(&npart[((size_t)m * nsl + q) * 2 + 0]);
        su += __ldcg(&npart[((size_t)m * nsl + q) * 2 + 1]);
      }
      dm = sqrt(sd);
      um = sqrt(su);
      a.unorm[m] = um;
    } else {
      um = __ldcg(&a.unorm[m]);              // u^k_m = u^{k-1}_m for m < k
    }
    a.du[m] = dm;
    sdu[m] = dm;
    sun[m] = um;
    umax_t = fmax(umax_t, um);
  }
  umax_t = fmax(umax_t, __shfl_xor_sync(0xffffffffu, umax_t, 16));
  umax_t = fmax(umax_t, __shfl_xor_sync(0xffffffffu, umax_t, 8));
  umax_t = fmax(umax_t, __shfl_xor_sync(0xffffffffu, umax_t, 4));
  umax_t = fmax(umax_t, __shfl_xor_sync(0xffffffffu, umax_t, 2));
  umax_t = fmax(umax_t, __shfl_xor_sync(0xffffffffu, umax_t, 1));
  if (lane == 0) red[w][1] = umax_t;
  __syncthreads();
  // a posteriori bound B_m = delta B_{m-1} + eps ||Delta_{m-1}||, B_0 = 0, as
  // a scan over m in chunks of blockDim.x (Hillis-Steele within a chunk:
  // B_m += delta^d B_{m-d}), the carry delta^(m - m0 + 1) B_{m0-1} added
  // from the previous chunk; then the maximum over m
  double bmax_t = 0.0;
  if (a.bound) {
    double* sb = sun;                            // reused ([N + 1]): the scan buffer
    __syncthreads();
    double carry = 0.0;                          // B_{m0 - 1}
    for (int m0 = 1; m0 <= N; m0 += blockDim.x) {
      const int m = m0 + threadIdx.x;
      double v = m <= N ? a.eps * sdu[m - 1] : 0.0;
      __syncthreads();
      double dp = a.delta;                       // delta^d
      for (int d = 1; d < (int)blockDim.x; d <<= 1) {
        if (m <= N) sb[m] = v;
        __syncthreads();
        if (m <= N && threadIdx.x >= d) v = fma(dp, sb[m - d], v);
        __syncthreads();
        dp *= dp;
      }
      // add the carry: delta^(m - m0 + 1) B_{m0 - 1}
      double cp = 1.0, base = a.delta;
      for (int e = threadIdx.x + 1; e > 0; e >>= 1) {
        if (e & 1) cp *= base;
        base *= base;
      }
      v = fma(cp, carry, v);
      if (m <= N) {
        a.bound[m] = v;
        bmax_t = fmax(bmax_t, v);
        sb[m] = v;
      }
      __syncthreads();
      carry = sb[min(N, m0 + (int)blockDim.x - 1)];
    }
    if (threadIdx.x == 0) a.bound[0] = 0.0;
  }
  bmax_t = fmax(bmax_t, __shfl_xor_sync(0xffffffffu, bmax_t, 16));
  bmax_t = fmax(bmax_t, __shfl_xor_sync(0xffffffffu, bmax_t, 8));
  bmax_t = fmax(bmax_t, __shfl_xor_sync(0xffffffffu, bmax_t, 4));
  bmax_t = fmax(bmax_t, __shfl_xor_sync(0xffffffffu, bmax_t, 2));
  bmax_t = fmax(bmax_t, __shfl_xor_sync(0xffffffffu, bmax_t, 1));
  __syncthreads();
  if (lane == 0) red[w][0] = bmax_t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double umax = 0.0, bmax = 0.0;
    for (int k = 0; k < nw; ++k) {
      umax = fmax(umax, red[k][1]);
      bmax = fmax(bmax, red[k][0]);
    }
    a.summary[0] = bmax;
    a.summary[1] = umax;
    if (a.k_done) *a.k_done = a.iter;
    if (a.stop && a.tol > 0.0 && bmax <= a.tol * umax) *a.stop = 1;
  }
}

lrp_status coarse_sweep(Ctx* c, const SweepArgs* h, SweepArgs* d_args, int nprob) {
  return coarse_sweep_ex(c, h, d_args, nprob, 1);
}

lrp_status coarse_sweep_ex(Ctx* c, const SweepArgs* h, SweepArgs* d_args, int nprob, int upload) {
  if (nprob <= 0) return LRP_OK;
  const int f32 = h[0].f32, N = h[0].N;
  int nsl = 0;
  for (int p = 0; p < nprob; ++p) {
    const SweepArgs& a = h[p];
    if (a.R > CSW_MAXR) return set_err(c, LRP_EINVAL, "rank above 64 is not supported by the sweep");
    if (a.rows < 1 || a.rows > CSW_MAXROWS || a.nsl != (a.n + a.rows - 1) / a.rows)
      return set_err(c, LRP_EINVAL, "sweep slice layout");
    if (a.f32 != f32 || a.N != N) return set_err(c, LRP_EINVAL, "sweep batch mixes precisions or N");
    if (!a.cw || !a.cnt || (N > 1 && !a.K)) return set_err(c, LRP_EINVAL, "sweep workspace missing");
    nsl = std::max(nsl, a.nsl);
  }
  cudaError_t e = upload ? cudaMemcpyAsync(d_args, h, sizeof(SweepArgs) * nprob,
                                           cudaMemcpyHostToDevice, c->stream)
                         : cudaSuccess;
  if (e) return cuda_err(c, e, "sweep arguments");
  auto kp = f32 ? (void (*)(const SweepArgs*))k_csw_project<float>
                : (void (*)(const SweepArgs*))k_csw_project<double>;
  auto ka = f32 ? (void (*)(const SweepArgs*))k_csw_apply<float>
                : (void (*)(const SweepArgs*))k_csw_apply<double>;
  if (N + 1 > CSW_MAXN) return set_err(c, LRP_EINVAL, "too many intervals for the coarse sweep");
  e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, CSW_KBUF);
  if (!e) e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(double) * 2 * CSW_MAXN));
  if (e) return cuda_err(c, e, "sweep smem attribute");
  cudaEvent_t ev = nullptr;
  timer_begin(c, "sweep", &ev);
  kp<<<dim3(nsl, N, nprob), CSW_THREADS, CSW_KBUF, c->stream>>>(d_args);
  ka<<<dim3(nsl, N + 1, nprob), CSW_THREADS, sizeof(double) * 2 * (N + 1), c->stream>>>(d_args);
  timer_end(c, "sweep", ev);
  e = cudaGetLastError();
  if (e) return cuda_err(c, e, "coarse sweep launch");
  c->launches += 1;   // two kernels; launch_count counts one more here
  return LRP_OK;
}

// ---------------------------------------------------------------------------
// K_i = V_{i+1}^T U_i diag(S_i), i = 0..N-2, from the factors the coarse
// apply uses (FP32 copies in the mixed mode), accumulated in FP64: partial
// products over tiles of 64 rows, then a fixed-order sum over the tiles.
// ---------------------------------------------------------------------------
constexpr int CH_TILE = 64;
constexpr int CH_MAXSL = 64;

template <typename TF>
__global__ void __launch_bounds__(256) k_chain_partial(const TF* __restrict__ U, const TF* __restrict__ V,
                                                      int n, int R, int nslk, double* __restrict__ part) {
  extern __shared__ double ch_sm[];
  double* sV = ch_sm;                              // [R][CH_TILE + 1]
  double* sU = sV + (size_t)R * (CH_TILE + 1);     // [R][CH_TILE + 1]
  const int i = blockIdx.y, sl = blockIdx.x;
  const TF* Vn = V + (size_t)(i + 1) * R * n;
  const TF* Ui = U + (size_t)i * R * n;
  constexpr int MAXO = CSW_MAXR * CSW_MAXR / 256;
  double acc[MAXO];
#pragma unroll
  for (int k = 0; k < MAXO; ++k) acc[k] = 0.0;
  const int nout = R * R;
  for (int t0 = sl * CH_TILE; t0 < n; t0 += nslk * CH_TILE) {
    const int rows = min(CH_TILE, n - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < R * CH_TILE; k += blockDim.x) {
      const int r = k / CH_TILE, x = k % CH_TILE;
      sV[r * (CH_TILE + 1) + x] = x < rows ? (double)Vn[(size_t)r * n + t0 + x] : 0.0;
      sU[r * (CH_TILE + 1) + x] = x < rows ? (double)Ui[(size_t)r * n + t0 + x] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
      const int o = threadIdx.x + k * 256;
      if (o < nout) {
        const double* vr = sV + (o / R) * (CH_TILE + 1);
        const double* uq = sU + (o % R) * (CH_TILE + 1);
        double s = acc[k];
        for (int x = 0; x < CH_TILE; ++x) s = fma(vr[x], uq[x], s);
        acc[k] = s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < MAXO; ++k) {
    const int o = threadIdx.x + k * 256;
    if (o < nout) part[((size_t)i * nslk + sl) * nout + o] = acc[k];
  }
}

template <typename TF>
__global__ void k_chain_reduce(const double* __restrict__ part, const TF* __restrict__ S, int R,
                               int nslk, double* __restrict__ K) {
  const int i = blockIdx.x, nout = R * R;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nslk; ++q) s += part[((size_t)i * nslk + q) * nout + o];
    K[(size_t)i * nout + o] = s * (double)S[(size_t)i * R + (o % R)];
  }
}

lrp_status coarse_chain(Ctx* c, Coarse* co) {
  const int N = co->N, R = std::max(co->R, 1), n = co->op->n;
  if (R > CSW_MAXR) return set_err(c, LRP_EINVAL, "rank above 64 is not supported by the sweep");
  lrp_status s;
  const size_t nk = (size_t)std::max(N - 1, 1) * R * R;
  if ((s = dev_alloc(c, co->Kc, sizeof(double) * nk))) return s;
  cudaMemsetAsync(co->Kc.ptr, 0, co->Kc.bytes, c->stream);
  if (N < 2) return LRP_OK;
  const int f32 = co->prec == LRP_PREC_MIXED;
  const int nslk = std::min(CH_MAXSL, (n + CH_TILE - 1) / CH_TILE);
  DevBuf part;
  if ((s = dev_alloc(c, part, sizeof(double) * (size_t)(N - 1) * nslk * R * R))) return s;
  const size_t smem = sizeof(double) * 2 * R * (CH_TILE + 1);
  cudaError_t e;
  cudaEvent_t ev = nullptr;
  timer_begin(c, "lift", &ev);
  if (f32) {
    e = cudaFuncSetAttribute(k_chain_partial<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!e) {
      k_chain_partial<float><<<dim3(nslk, N - 1), 256, smem, c->stream>>>(
          co->U32.as<float>(), co->V32.as<float>(), n, R, nslk, part.as<double>());
      k_chain_reduce<float><<<N - 1, 256, 0, c->stream>>>(part.as<double>(), co->S32.as<float>(), R,
                                                         nslk, co->Kc.as<double>());
    }
  } else {
    e = cudaFuncSetAttribute(k_chain_partial<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!e) {
      k_chain_partial<double><<<dim3(nslk, N - 1), 256, smem, c->stream>>>(
          co->U.as<double>(), co->V.as<double>(), n, R, nslk, part.as<double>());
      k_chain_reduce<double><<<N - 1, 256, 0, c->stream>>>(part.as<double>(), co->S.as<double>(), R,
                                                          nslk, co->Kc.as<double>());
    }
  }
  timer_end(c, "lift", ev);
  c->launches += 1;   // two kernels
  if (!e) e = cudaGetLastError();
  if (e) return cuda_err(c, e, "coarse chain matrices");
  return LRP_OK;
}

lrp_status coarse_sweep_workspace(Ctx* c, Coarse* co, int rows) {
  const int N = co->N, R = std::max(co->R, 1), nsl = (co->op->n + rows - 1) / rows;
  const size_t need = sweep_ws_doubles(N, nsl, R) * sizeof(double);
  lrp_status s;
  if (!co->ws_cw.ptr || co->ws_cw.bytes < need) {
    co->ws_cw.release();
    if ((s = dev_alloc(c, co->ws_cw, need))) return s;
  }
  if (!co->ws_cnt.ptr) {
    if ((s = dev_alloc(c, co->ws_cnt, 2 * sizeof(unsigned)))) return s;
    cudaMemsetAsync(co->ws_cnt.ptr, 0, 2 * sizeof(unsigned), c->stream);
  }
  if (!co->ws_args.ptr) {
    if ((s = dev_alloc(c, co->ws_args, sizeof(SweepArgs)))) return s;
  }
  return LRP_OK;
}

}  // namespace lrp
