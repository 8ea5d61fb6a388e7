// Randomized-SVD finishing steps (Sec. 2.1, steps 2, 4, 5, 6):
//   * orthonormal bases of the sketches by classical Gram-Schmidt applied twice
//     ("twice is enough") with deflation of numerically dependent vectors;
//   * the small matrix M_ij = (F'^* w_i, v_j) read off the Gram-Schmidt
//     coefficients of the adjoint sketch, and its SVD by one-sided Jacobi
//     (Hestenes) in FP64 with a round-robin pair ordering;
//   * the lift of the leading R singular vectors to the bases.
// One CTA per coarse interval for the orthonormalisation and the SVD; the lift
// runs over (interval, row block).
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace lrp {

// ---------------------------------------------------------------------------
// CGS2 with deflation.  X: N blocks of ell rows of length n (row = vector).
// For input vector j: h = Q^T v, v -= Q h, twice; Rcoef[c][j] accumulates h;
// keep v / ||v|| as the next basis vector when ||v|| > tau * ||y_j||.
// ---------------------------------------------------------------------------
constexpr int ORTH_THREADS = 512;

// Warp sums stay in the vector's type (FP32 in the mixed mode: FP64 arithmetic
// runs at 1/64 of the FP32 rate on GB300); the per-warp results are combined
// in FP64.
template <typename T>
__device__ double block_sum(T v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double d = (double)warp_sum<T>(v);
  __syncthreads();
  if (lane == 0) red[w] = d;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

template <typename T>
__global__ void __launch_bounds__(ORTH_THREADS) k_cgs2(int ell, int n, T* __restrict__ X,
                                                        double tau, double* __restrict__ Rcoef,
                                                        int* __restrict__ rank,
                                                        const int* __restrict__ skip) {
  if (skip && skip[blockIdx.x]) return;
  extern __shared__ double sm[];
  const int nw = blockDim.x >> 5;
  double* red1 = sm;                // [nw] block-sum scratch
  T* hT = reinterpret_cast<T*>(red1 + nw);   // [ell] projection coefficients
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* B = X + (size_t)blockIdx.x * ell * n;
  double* Rc = Rcoef + (size_t)blockIdx.x * ell * ell;
  for (int k = threadIdx.x; k < ell * ell; k += blockDim.x) Rc[k] = 0.0;
  int r = 0;
  for (int j = 0; j < ell; ++j) {
    T* v = B + (size_t)j * n;
    T acc = T(0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i] * v[i];
    double nrm0 = sqrt(block_sum(acc, red1));
    for (int pass = 0; pass < 2; ++pass) {
      // one warp per basis vector c: lanes stride the rows, so the loads of
      // a warp are independent and the dot needs no cross-warp reduction
      for (int c = w; c < r; c += nw) {
        const T* q = B + (size_t)c * n;
        T pc = T(0);
#pragma unroll 4
        for (int i = lane; i < n; i += 32) pc += q[i] * v[i];
        pc = warp_sum<T>(pc);
        if (lane == 0) {
          hT[c] = pc;
          Rc[c * ell + j] += (double)pc;
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T s = v[i];
        for (int c = 0; c < r; ++c) s -= hT[c] * B[(size_t)c * n + i];
        v[i] = s;
      }
      __syncthreads();
    }
    acc = T(0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i] * v[i];
    double nrm = sqrt(block_sum(acc, red1));
    if (nrm0 > 0.0 && nrm > tau * nrm0) {
      T inv = (T)(1.0 / nrm);
      T* q = B + (size_t)r * n;
      for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] = v[i] * inv;
      if (threadIdx.x == 0) Rc[r * ell + j] = nrm;
      ++r;
    }
    __syncthreads();
  }
  for (int c = r; c < ell; ++c)
    for (int i = threadIdx.x; i < n; i += blockDim.x) B[(size_t)c * n + i] = T(0);
  if (threadIdx.x == 0) rank[blockIdx.x] = r;
}

// ---------------------------------------------------------------------------
// The same CGS2 with one interval per thread-block cluster and the interval's
// block held in shared memory: CTA q of the cluster keeps rows
// [q*per, (q+1)*per) of all ell vectors, dot products are summed over the
// cluster (per-CTA FP64 partials pushed into every CTA's shared memory before
// the cluster barrier, then added in a fixed order), and the update and
// normalisation touch only shared memory.  Three cluster sums per vector:
// ||y_j||^2 together with the first projection, the second projection, the
// norm after it.
// ---------------------------------------------------------------------------
constexpr int ORTHC_MAXC = 16;
constexpr int ORTHC_MAXV = 65;      // ell + 1 values per cluster sum

struct OrthRed {
  double red[ORTH_THREADS / 32];
  double part[2][ORTHC_MAXC][ORTHC_MAXV];
  double tot[ORTHC_MAXV];
  double* rpart[ORTHC_MAXC];
};

template <typename T>
__global__ void __launch_bounds__(ORTH_THREADS) k_cgs2_cl(int ell, int n, T* __restrict__ X,
                                                           double tau, double* __restrict__ Rcoef,
                                                           int* __restrict__ rank,
                                                           const int* __restrict__ skip) {
  cg::cluster_group cl = cg::this_cluster();
  // every CTA of a cluster serves the same interval, so a skipped interval
  // leaves the kernel before any cluster barrier
  if (skip && skip[blockIdx.x / cl.num_blocks()]) return;
  extern __shared__ __align__(16) unsigned char orth_smem[];
  __shared__ OrthRed sh;
  __shared__ T hT[ORTHC_MAXV];
  const int C = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int iv = blockIdx.x / C;
  const int per = (n + C - 1) / C;
  const int lo = min(n, q * per), rows = min(n, lo + per) - lo;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* sB = reinterpret_cast<T*>(orth_smem);           // [ell][per]
  T* B = X + (size_t)iv * ell * n;
  double* Rc = Rcoef + (size_t)iv * ell * ell;
  for (int k = threadIdx.x; k < ell * per; k += blockDim.x) {
    const int j = k / per, i = k % per;
    sB[k] = i < rows ? B[(size_t)j * n + lo + i] : T(0);
  }
  if (q == 0)
    for (int k = threadIdx.x; k < ell * ell; k += blockDim.x) Rc[k] = 0.0;
  for (int k = threadIdx.x; k < C; k += blockDim.x) sh.rpart[k] = cl.map_shared_rank(&sh.part[0][0][0], k);
  cl.sync();     // every CTA runs before remote stores into its shared memory
  int buf = 0;
  // cluster sum of nv values; vals[v] is set for v < nv by the caller's warps
  // through `partial` (lane 0 of a warp, or the block sum for slot `bslot`)
  auto push_and_sum = [&](int nv) {
    for (int k = threadIdx.x; k < nv * C; k += blockDim.x) {
      const int v = k % nv, dst = k / nv;
      sh.rpart[dst][(buf * ORTHC_MAXC + q) * ORTHC_MAXV + v] = sh.tot[v];
    }
    cl.sync();
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x < nv) {
      for (int k = 0; k < C; ++k) out += sh.part[buf][k][threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x < nv) sh.tot[threadIdx.x] = out;
    __syncthreads();
    buf ^= 1;
  };
  // per-CTA dots of v with basis vectors 0..r-1 into sh.tot[0..r-1] and,
  // when with_norm, ||v||^2 of this CTA's rows into sh.tot[r]
  auto local_dots = [&](const T* v, int r, bool with_norm) {
    for (int c = w; c < r; c += nw) {
      const T* qc = sB + (size_t)c * per;
      T pc = T(0);
      for (int i = lane; i < rows; i += 32) pc += qc[i] * v[i];
      pc = warp_sum<T>(pc);
      if (lane == 0) sh.tot[c] = (double)pc;
    }
    if (with_norm) {
      T a = T(0);
      for (int i = threadIdx.x; i < rows; i += blockDim.x) a += v[i] * v[i];
      a = warp_sum<T>(a);
      if (lane == 0) sh.red[w] = (double)a;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += sh.red[k];
        sh.tot[r] = s;
      }
    }
    __syncthreads();
  };
  auto subtract = [&](T* v, int r) {
    for (int c = threadIdx.x; c < r; c += blockDim.x) hT[c] = (T)sh.tot[c];
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      T s = v[i];
      for (int c = 0; c < r; ++c) s -= hT[c] * sB[(size_t)c * per + i];
      v[i] = s;
    }
    __syncthreads();
  };
  int r = 0;
  for (int j = 0; j < ell; ++j) {
    T* v = sB + (size_t)j * per;
    // ||y_j||^2 and the first projection in one cluster sum
    local_dots(v, r, true);
    push_and_sum(r + 1);
    const double nrm0 = sqrt(sh.tot[r]);
    if (q == 0)
      for (int c = threadIdx.x; c < r; c += blockDim.x) Rc[c * ell + j] += sh.tot[c];
    subtract(v, r);
    // second projection
    if (r > 0) {
      local_dots(v, r, false);
      push_and_sum(r);
      if (q == 0)
        for (int c = threadIdx.x; c < r; c += blockDim.x) Rc[c * ell + j] += sh.tot[c];
      subtract(v, r);
    }
    // norm after the projections
    local_dots(v, 0, true);
    push_and_sum(1);
    const double nrm = sqrt(sh.tot[0]);
    if (nrm0 > 0.0 && nrm > tau * nrm0) {
      const T inv = (T)(1.0 / nrm);
      T* qn = sB + (size_t)r * per;
      for (int i = threadIdx.x; i < rows; i += blockDim.x) qn[i] = v[i] * inv;
      if (q == 0 && threadIdx.x == 0) Rc[r * ell + j] = nrm;
      ++r;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < ell * per; k += blockDim.x) {
    const int j = k / per, i = k % per;
    if (i < rows) B[(size_t)j * n + lo + i] = j < r ? sB[k] : T(0);
  }
  if (q == 0 && threadIdx.x == 0) rank[iv] = r;
  cl.sync();     // no CTA leaves while others may still store into its shared memory
}

lrp_status orth_cgs2(Ctx* c, int N, int ell, int n, void* X, int x_f64, double tau,
                     double* Rcoef, int* rank, const int* skip) {
  if (N <= 0) return LRP_OK;
  // shared-memory cluster variant when the interval's block fits in at most
  // 16 CTAs of 200 KB (1D problems); the one-CTA kernel otherwise
  const size_t es = x_f64 ? 8 : 4;
  int C = 2;
  while (C <= ORTHC_MAXC && (size_t)ell * ((n + C - 1) / C) * es > 100 * 1024) C *= 2;
  if (c->p_orth_cluster > 0) C = c->p_orth_cluster;
  if (ell + 1 <= ORTHC_MAXV && C <= ORTHC_MAXC && c->p_orth_cluster >= 0 && n >= 64 * C) {
    const size_t smem = (size_t)ell * ((n + C - 1) / C) * es;
    cudaError_t e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(N * C);
    cfg.blockDim = dim3(ORTH_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaEvent_t ev = nullptr;
    if (x_f64) {
      e = cudaFuncSetAttribute(k_cgs2_cl<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (!e && C > 8) e = cudaFuncSetAttribute(k_cgs2_cl<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e) return cuda_err(c, e, "cgs2 cluster attributes");
      timer_begin(c, "orth", &ev);
      e = cudaLaunchKernelEx(&cfg, k_cgs2_cl<double>, ell, n, (double*)X, tau, Rcoef, rank, skip);
    } else {
      e = cudaFuncSetAttribute(k_cgs2_cl<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (!e && C > 8) e = cudaFuncSetAttribute(k_cgs2_cl<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e) return cuda_err(c, e, "cgs2 cluster attributes");
      timer_begin(c, "orth", &ev);
      e = cudaLaunchKernelEx(&cfg, k_cgs2_cl<float>, ell, n, (float*)X, tau, Rcoef, rank, skip);
    }
    timer_end(c, "orth", ev);
    return e ? cuda_err(c, e, "k_cgs2_cl") : LRP_OK;
  }
  const int nw = ORTH_THREADS / 32;
  size_t smem = sizeof(double) * ((size_t)ell + nw);
  cudaEvent_t ev = nullptr;
  timer_begin(c, "orth", &ev);
  if (x_f64)
    k_cgs2<double><<<N, ORTH_THREADS, smem, c->stream>>>(ell, n, (double*)X, tau, Rcoef, rank, skip);
  else
    k_cgs2<float><<<N, ORTH_THREADS, smem, c->stream>>>(ell, n, (float*)X, tau, Rcoef, rank, skip);
  cudaError_t e = cudaGetLastError();
  timer_end(c, "orth", ev);
  return e ? cuda_err(c, e, "k_cgs2") : LRP_OK;
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD of M (ell rows x kv columns), M[i][c] = Rz[c][i].
// Column pairs are rotated in round-robin order until a full sweep performs
// no rotation (|a_p.a_q| <= m eps sqrt(|a_p|^2 |a_q|^2)).  Eight lanes serve
// one pair, four pairs per warp: an FP64 warp instruction costs the same
// issue time on GB300 whatever the number of active lanes, so the rotation
// parameters (divisions and square roots) are computed once per eight lanes
// rather than once per warp.  The squared column norms are carried through
// the rotations (|a_p'|^2 = |a_p|^2 - t a_p.a_q, |a_q'|^2 = |a_q|^2 +
// t a_p.a_q) and recomputed from the columns at the start of every sweep,
// so a round needs one dot product per pair.  The angle's tangent is formed
// in FP32 (its divisions and square root cost FP64 issue slots otherwise);
// cos and sin are formed from it in FP64.
// ---------------------------------------------------------------------------
constexpr int SVD_THREADS = 512;    // launch: 32 * ceil(pairs / 4) threads
constexpr int SVD_MAX_SWEEPS = 60;

__global__ void __launch_bounds__(SVD_THREADS) k_jacobi(int ell, const double* __restrict__ Rz,
                                                         const int* __restrict__ rank_v,
                                                         double* __restrict__ s_out,
                                                         double* __restrict__ Psi,
                                                         double* __restrict__ Phi,
                                                         int* __restrict__ status) {
  extern __shared__ double sm[];
  const int iv = blockIdx.x;
  const int kv = rank_v[iv];
  const int m = ell;
  double* A = sm;                     // [kv][m] column-major (column c at c*m)
  double* Vw = A + (size_t)ell * m;   // [kv][kv] (column c at c*ell)
  double* nrm = Vw + (size_t)ell * ell;
  int* order = reinterpret_cast<int*>(nrm + ell);
  __shared__ int rotated;
  const double* Rzi = Rz + (size_t)iv * ell * ell;
  for (int k = threadIdx.x; k < ell * m; k += blockDim.x) {
    int c = k / m, i = k % m;
    A[k] = (c < kv) ? Rzi[(size_t)c * ell + i] : 0.0;
  }
  for (int k = threadIdx.x; k < ell * ell; k += blockDim.x)
    Vw[k] = ((k / ell) == (k % ell)) ? 1.0 : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int l8 = lane & 7;                        // lane within the pair's group
  const int slot = w * 4 + (lane >> 3);           // pair slot of this group
  const unsigned gmask = 0xffu << (lane & 24);    // the group's lanes
  const int nslots = (blockDim.x >> 5) * 4;
  const int kp = kv + (kv & 1);       // players, padded to even
  // convergence: every pair's cosine below m * eps (the usual one-sided
  // Jacobi threshold); a stricter eps keeps rotating on rounding noise
  const double eps = 2.220446049250313e-16 * m;
  const double eps2 = eps * eps;
  int sweep = 0, done = (kv < 2);
  while (!done && sweep < SVD_MAX_SWEEPS) {
    if (threadIdx.x == 0) rotated = 0;
    for (int c = threadIdx.x; c < kv; c += blockDim.x) {
      double t = 0.0;
      for (int i = 0; i < m; ++i) t = fma(A[(size_t)c * m + i], A[(size_t)c * m + i], t);
      nrm[c] = t;
    }
    __syncthreads();
    for (int rd = 0; rd < kp - 1; ++rd) {
      for (int pi = slot; pi < kp / 2; pi += nslots) {
        int p, q;
        if (pi == 0) { p = kp - 1; q = rd; }
        else { p = (rd + pi) % (kp - 1); q = (rd - pi + (kp - 1)) % (kp - 1); }
        if (p > q) { int tmp = p; p = q; q = tmp; }
        if (q >= kv) continue;
        double* ap = A + (size_t)p * m;
        double* aq = A + (size_t)q * m;
        double ga = 0.0;
        for (int i = l8; i < m; i += 8) ga = fma(ap[i], aq[i], ga);
        ga += __shfl_xor_sync(gmask, ga, 4);
        ga += __shfl_xor_sync(gmask, ga, 2);
        ga += __shfl_xor_sync(gmask, ga, 1);
        const double al = nrm[p], be = nrm[q];
        if (ga == 0.0 || ga * ga <= eps2 * (al * be)) continue;
        // zeta (dimensionless) in FP64, the tangent of the rotation angle
        // from it in FP32, cos and sin from the tangent in FP64: the rotation
        // is orthogonal to FP64 accuracy whatever the angle's accuracy, which
        // only sets how far a_p.a_q drops (a relative 1e-7 instead of 1e-16;
        // the sweeps go on until every pair passes the FP64 test)
        const double zeta = (be - al) / (2.0 * ga);
        double tt;
        if (fabs(zeta) < 1e15) {
          const float z = (float)zeta;
          tt = (double)(copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f))));
        } else {
          tt = 0.5 / zeta;
        }
        const double cs = rsqrt(fma(tt, tt, 1.0));
        const double sn = cs * tt;
        for (int i = l8; i < m; i += 8) {
          const double x = ap[i], y = aq[i];
          ap[i] = cs * x - sn * y;
          aq[i] = sn * x + cs * y;
        }
        double* vp = Vw + (size_t)p * ell;
        double* vq = Vw + (size_t)q * ell;
        for (int i = l8; i < kv; i += 8) {
          const double x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (l8 == 0) {
          nrm[p] = fma(-tt, ga, al);
          nrm[q] = fma(tt, ga, be);
          rotated = 1;
        }
      }
      __syncthreads();
    }
    ++sweep;
    done = !rotated;
    __syncthreads();
  }
  // singular values and descending order
  for (int c = threadIdx.x; c < ell; c += blockDim.x) {
    double t = 0.0;
    if (c < kv)
      for (int i = 0; i < m; ++i) t += A[(size_t)c * m + i] * A[(size_t)c * m + i];
    nrm[c] = sqrt(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < ell; ++c) order[c] = c;
    for (int a = 0; a < kv; ++a)
      for (int b = a + 1; b < kv; ++b)
        if (nrm[order[b]] > nrm[order[a]]) { int t = order[a]; order[a] = order[b]; order[b] = t; }
    if (!done) atomicOr(status, 1);
  }
  __syncthreads();
  double* so = s_out + (size_t)iv * ell;
  double* Ps = Psi + (size_t)iv * ell * ell;
  double* Ph = Phi + (size_t)iv * ell * ell;
  for (int k = threadIdx.x; k < ell * ell; k += blockDim.x) {
    int r = k / ell, i = k % ell;          // column r of the outputs
    double val_psi = 0.0, val_phi = 0.0;
    if (r < kv) {
      int c = order[r];
      double sc = nrm[c];
      val_psi = sc > 0.0 ? A[(size_t)c * m + i] / sc : 0.0;
      val_phi = (i < kv) ? Vw[(size_t)c * ell + i] : 0.0;
    }
    Ps[k] = val_psi;
    Ph[k] = val_phi;
  }
  for (int r = threadIdx.x; r < ell; r += blockDim.x) so[r] = (r < kv) ? nrm[order[r]] : 0.0;
}

lrp_status small_svd(Ctx* c, int N, int ell, const double* Rz, const int* rank_v, double* s,
                     double* Psi, double* Phi, int* status) {
  if (N <= 0) return LRP_OK;
  size_t smem = sizeof(double) * ((size_t)2 * ell * ell + ell) + sizeof(int) * ell;
  cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return cuda_err(c, e, "jacobi smem");
  cudaEvent_t ev = nullptr;
  timer_begin(c, "svd", &ev);
  const int pairs = std::max(1, (ell + 1) / 2);
  const int threads = std::min(SVD_THREADS, 32 * ((pairs + 3) / 4));
  k_jacobi<<<N, threads, smem, c->stream>>>(ell, Rz, rank_v, s, Psi, Phi, status);
  e = cudaGetLastError();
  timer_end(c, "svd", ev);
  return e ? cuda_err(c, e, "k_jacobi") : LRP_OK;
}

// ---------------------------------------------------------------------------
// Lift: U_i[r] = sum_j Psi_i[r][j] W_i[j], V_i[r] = sum_j Phi_i[r][j] Vh_i[j]
// for r < R_i (zero rows beyond).  grid = (row blocks, N).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_lift(int ell, int R, int n, const T* __restrict__ W, const T* __restrict__ Vh,
                       const double* __restrict__ Psi, const double* __restrict__ Phi,
                       const int* __restrict__ Ri, double* __restrict__ U, double* __restrict__ V,
                       float* __restrict__ U32, float* __restrict__ V32) {
  extern __shared__ double sm[];
  const int iv = blockIdx.y;
  double* sPsi = sm;                  // [R][ell]
  double* sPhi = sm + (size_t)R * ell;
  const int rk = Ri[iv];
  for (int k = threadIdx.x; k < R * ell; k += blockDim.x) {
    sPsi[k] = Psi[(size_t)iv * ell * ell + k];
    sPhi[k] = Phi[(size_t)iv * ell * ell + k];
  }
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const T* Wi = W + (size_t)iv * ell * n;
  const T* Vi = Vh + (size_t)iv * ell * n;
  for (int r = 0; r < R; ++r) {
    T u = T(0), v = T(0);               // the bases' precision (FP32 in the mixed mode)
    if (r < rk) {
      for (int j = 0; j < ell; ++j) {
        u += (T)sPsi[r * ell + j] * Wi[(size_t)j * n + row];
        v += (T)sPhi[r * ell + j] * Vi[(size_t)j * n + row];
      }
    }
    size_t o = ((size_t)iv * R + r) * n + row;
    U[o] = (double)u;
    V[o] = (double)v;
    U32[o] = (float)u;
    V32[o] = (float)v;
  }
}

lrp_status lift(Ctx* c, int N, int ell, int R, int n, const void* W, const void* Vh, int b_f64,
                const double* Psi, const double* Phi, const int* Ri, double* U, double* V,
                float* U32, float* V32) {
  if (N <= 0 || R <= 0) return LRP_OK;
  dim3 grid((n + 255) / 256, N);
  size_t smem = sizeof(double) * 2 * (size_t)R * ell;
  cudaEvent_t ev = nullptr;
  timer_begin(c, "lift", &ev);
  if (b_f64)
    k_lift<double><<<grid, 256, smem, c->stream>>>(ell, R, n, (const double*)W, (const double*)Vh,
                                                   Psi, Phi, Ri, U, V, U32, V32);
  else
    k_lift<float><<<grid, 256, smem, c->stream>>>(ell, R, n, (const float*)W, (const float*)Vh,
                                                  Psi, Phi, Ri, U, V, U32, V32);
  cudaError_t e = cudaGetLastError();
  timer_end(c, "lift", ev);
  return e ? cuda_err(c, e, "k_lift") : LRP_OK;
}

// ---------------------------------------------------------------------------
// Two-sided sketch (F'^* on independent random vectors psi_a, Philox stream 3):
//   B = Psi^T Q (2l x k), C = B (B^T B)^-1 (the least-squares solution map),
//   X^T = Z C (n x k), Z the adjoint sketch (2l x n, rows F'^T psi_a).
// ---------------------------------------------------------------------------
constexpr uint32_t PSI_STREAM = 3;

// B[iv][a][c] = (psi_a, q_c) for c < k = rank_w[iv] (0 beyond); psi_a
// regenerated in the sketch precision T, exactly as the adjoint propagation
// drew it.  grid (ell2, N).
template <typename T>
__global__ void __launch_bounds__(256) k_psi_dots(int ell2, int ell, int n, uint64_t seed,
                                                   const T* __restrict__ Q,
                                                   const int* __restrict__ rank_w,
                                                   double* __restrict__ B) {
  __shared__ double red[8][16];
  const int a = blockIdx.x, iv = blockIdx.y;
  const int k = rank_w[iv];
  const T* Qi = Q + (size_t)iv * ell * n;
  double* Bi = B + ((size_t)iv * ell2 + a) * ell;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c0 = 0; c0 < ell; c0 += 16) {
    T acc[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) acc[t] = T(0);
    if (c0 < k) {
      for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const T ps = gauss<T>(seed, PSI_STREAM, (uint32_t)iv, (uint32_t)a, (uint32_t)x);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (c0 + t < k) acc[t] += ps * Qi[(size_t)(c0 + t) * n + x];
      }
    }
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const T v = warp_sum<T>(acc[t]);
      if (lane == 0) red[w][t] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 16 && c0 + (int)threadIdx.x < ell) {
      double sum = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += red[q][threadIdx.x];
      Bi[c0 + threadIdx.x] = (c0 + (int)threadIdx.x < k) ? sum : 0.0;
    }
    __syncthreads();
  }
}

// C = B (B^T B)^-1 per interval (FP64, one CTA): Gram, Cholesky factor
// (right-looking, in shared memory), then two triangular solves per row of B.
__global__ void __launch_bounds__(256) k_lsq(int ell2, int ell, const double* __restrict__ B,
                                             const int* __restrict__ rank_w, double* __restrict__ Cm,
                                             int* __restrict__ status) {
  extern __shared__ double lsq_sm[];
  double* G = lsq_sm;                  // [ell][ell]
  const int iv = blockIdx.x, k = rank_w[iv];
  const double* Bi = B + (size_t)iv * ell2 * ell;
  double* Ci = Cm + (size_t)iv * ell2 * ell;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    double sum = 0.0;
    for (int a = 0; a < ell2; ++a) sum += Bi[(size_t)a * ell + i] * Bi[(size_t)a * ell + j];
    G[i * ell + j] = sum;
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = G[j * ell + j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      G[j * ell + j] = sqrt(fabs(d) > 0.0 ? fabs(d) : 1.0);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) G[i * ell + j] /= G[j * ell + j];
    __syncthreads();
    for (int e = threadIdx.x; e < (k - j - 1) * (k - j - 1); e += blockDim.x) {
      const int i = j + 1 + e / (k - j - 1), l = j + 1 + e % (k - j - 1);
      if (l <= i) G[i * ell + l] -= G[i * ell + j] * G[l * ell + j];
    }
    __syncthreads();
  }
  // row a of C: solve (L L^T) c = B[a]^T
  for (int a = threadIdx.x; a < ell2; a += blockDim.x) {
    double y[128];
    for (int i = 0; i < k; ++i) {
      double v = Bi[(size_t)a * ell + i];
      for (int l = 0; l < i; ++l) v -= G[i * ell + l] * y[l];
      y[i] = v / G[i * ell + i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double v = y[i];
      for (int l = i + 1; l < k; ++l) v -= G[l * ell + i] * y[l];
      y[i] = v / G[i * ell + i];
    }
    for (int i = 0; i < ell; ++i) Ci[(size_t)a * ell + i] = i < k ? y[i] : 0.0;
  }
  if (threadIdx.x == 0 && bad) atomicOr(status, 2);
}

// X^T = Z C: out[iv][c][x] = sum_a C[iv][a][c] Z[iv][a][x], c < ell (rows
// beyond the rank are 0 because C's columns are).  grid (row blocks, N).
template <typename T>
__global__ void __launch_bounds__(256) k_combine(int ell2, int ell, int n, const T* __restrict__ Z,
                                                 const double* __restrict__ Cm, T* __restrict__ out) {
  extern __shared__ double cmb_sm[];
  T* sC = reinterpret_cast<T*>(cmb_sm);            // [ell2][ell]
  const int iv = blockIdx.y;
  for (int e = threadIdx.x; e < ell2 * ell; e += blockDim.x) sC[e] = (T)Cm[(size_t)iv * ell2 * ell + e];
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const T* Zi = Z + (size_t)iv * ell2 * n;
  for (int c0 = 0; c0 < ell; c0 += 16) {
    T acc[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) acc[t] = T(0);
    for (int a = 0; a < ell2; ++a) {
      const T z = Zi[(size_t)a * n + x];
#pragma unroll
      for (int t = 0; t < 16; ++t)
        if (c0 + t < ell) acc[t] += sC[a * ell + c0 + t] * z;
    }
#pragma unroll
    for (int t = 0; t < 16; ++t)
      if (c0 + t < ell) out[((size_t)iv * ell + c0 + t) * n + x] = acc[t];
  }
}

lrp_status two_sided_core(Ctx* c, int N, int ell, int ell2, int n, uint64_t seed, int f32,
                          const void* Q, const int* rank_w, const void* Z, void* XT, double* Bbuf,
                          double* Cbuf, int* status) {
  if (ell > 128 || ell2 > 256) return set_err(c, LRP_EINVAL, "two-sided sketch too wide");
  cudaEvent_t ev = nullptr;
  timer_begin(c, "orth", &ev);
  const size_t smem_l = sizeof(double) * (size_t)ell * ell;
  cudaError_t e = cudaFuncSetAttribute(k_lsq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
  const size_t smem_c = (f32 ? 4 : 8) * (size_t)ell2 * ell;
  if (!e) {
    if (f32) {
      e = cudaFuncSetAttribute(k_combine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
      if (!e) {
        k_psi_dots<float><<<dim3(ell2, N), 256, 0, c->stream>>>(ell2, ell, n, seed, (const float*)Q, rank_w, Bbuf);
        k_lsq<<<N, 256, smem_l, c->stream>>>(ell2, ell, Bbuf, rank_w, Cbuf, status);
        k_combine<float><<<dim3((n + 255) / 256, N), 256, smem_c, c->stream>>>(ell2, ell, n, (const float*)Z,
                                                                              Cbuf, (float*)XT);
      }
    } else {
      e = cudaFuncSetAttribute(k_combine<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
      if (!e) {
        k_psi_dots<double><<<dim3(ell2, N), 256, 0, c->stream>>>(ell2, ell, n, seed, (const double*)Q, rank_w, Bbuf);
        k_lsq<<<N, 256, smem_l, c->stream>>>(ell2, ell, Bbuf, rank_w, Cbuf, status);
        k_combine<double><<<dim3((n + 255) / 256, N), 256, smem_c, c->stream>>>(ell2, ell, n, (const double*)Z,
                                                                               Cbuf, (double*)XT);
      }
    }
  }
  timer_end(c, "orth", ev);
  c->launches += 2;
  if (!e) e = cudaGetLastError();
  return e ? cuda_err(c, e, "two-sided sketch core") : LRP_OK;
}

// Sketch vectors of one interval, written as doubles.
template <typename T>
__global__ void k_gaussian(uint64_t seed, int interval, int ncol, int n, double* out) {
  long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long)ncol * n) return;
  int col = (int)(k / n), row = (int)(k % n);
  out[k] = (double)gauss<T>(seed, 0u, (uint32_t)interval, (uint32_t)col, (uint32_t)row);
}

lrp_status gaussian(Ctx* c, uint64_t seed, int interval, int ncol, int n, int f32, double* out) {
  long tot = (long)ncol * n;
  if (tot <= 0) return LRP_OK;
  int blocks = (int)((tot + 255) / 256);
  if (f32)
    k_gaussian<float><<<blocks, 256, 0, c->stream>>>(seed, interval, ncol, n, out);
  else
    k_gaussian<double><<<blocks, 256, 0, c->stream>>>(seed, interval, ncol, n, out);
  cudaError_t e = cudaGetLastError();
  return e ? cuda_err(c, e, "k_gaussian") : LRP_OK;
}

}  // namespace lrp
