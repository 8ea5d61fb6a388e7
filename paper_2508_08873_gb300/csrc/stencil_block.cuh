// Block conjugate gradients for the backward-Euler steps of a symmetric
// 5-point operator: S systems that share the step matrix are solved
// together, one block Krylov space for all of them (the sketch vectors of
// the randomized SVD of Sec. 2.1 meet the same matrix B in every step, and
// Sec. 2.2 notes that all R + p of them can be propagated at once; block
// solvers need fewer iterations than S separate ones, and the matrix
// coefficients are read once for all S).  The kernel template; the launch
// code is in stencil_block.cu.
//
// The iteration works on the diagonally scaled system B^ X^ = D^ (unit
// diagonal, S = diag(sqrt(c)), as in the single-system CG kernels) with the
// search directions made B^-orthonormal at every iteration.  With Z = B^ P,
//   G = P^T Z, H = P^T R, ZZ = Z^T Z, ZR = Z^T R   (one reduction)
//   G+ = the inverse of G on a pivoted subset of its columns (pivoted
//        Cholesky; a column whose Schur complement falls below thr times the
//        largest diagonal entry of G is left out, so that directions that
//        became dependent -- converged systems, or columns that the
//        propagation made nearly parallel -- drop out of that iteration)
//   C1 = G+ H,  E = ZR - ZZ C1 (= Z^T R_new),  C2 = G+ E
//   X += P C1,  R_new = R - Z C1,  P_new = R_new - P C2
// which, with T the factor of G+ = T T^T, is block CG with the directions
// P T: X += (P T)(P T)^T R, and P T is B^-orthogonalised against the new
// residual.  E comes from the Gram matrices of the old directions (the
// recurrence R_new = R - Z C1), so that one pass per iteration computes the
// update, the new directions, their product with B^ and all four Gram
// matrices, closed by a single cluster reduction.  A system counts as
// converged once ||r_s|| <= rtol ||d_s|| (the scaled system); the block
// iterates until all S have.
//
// One block runs on one thread-block cluster of cs CTAs: CTA c owns grid
// rows [c RB, c RB + RB), thread t owns grid columns 2t and 2t + 1 (PITCH / 2
// threads, PITCH >= mx), whose values it carries as pairs: in FP32 every
// multiply-add of the two columns is one packed instruction (fma.rn.f32x2),
// and a coefficient of the S x S algebra, stored twice side by side, is one
// 64-bit shared-memory load for both.  The block vectors X^, R (old and new)
// and P (old and new) live in a global-memory workspace of the cluster,
// laid out [row][s][PITCH] with two zero rows above and below the grid, so
// that one grid row of one block vector is S PITCH contiguous elements.  An
// iteration streams the rows of P, R and X^ (and the coupling row) that the
// CTA needs through a ring of DR shared-memory slots, each filled by the
// CTA's first thread with bulk asynchronous copies (cp.async.bulk,
// completion on an mbarrier of the slot) three rows ahead of their use: row
// q of the old directions enters the stencil of row q - 1, whose new
// residual and direction are computed and stored; the new directions of the
// last four rows stay in shared memory for the stencil of B^ P_new one row
// behind.  Every CTA also computes the new residual and direction of the
// row just above and just below its own (from old values that their owners
// do not change in the pass).  The S x S algebra runs on one warp of every
// CTA on the reduced totals, which every CTA receives bitwise equal, so that
// all CTAs take the same decisions.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace lrp {
namespace bk {

namespace cg = cooperative_groups;

constexpr int MAXCS = 16;         // CTAs per cluster
constexpr int PADR = 2;           // zero rows above and below every block vector
constexpr int DR = 6;             // ring slots
constexpr long SPIN = 1L << 20;   // polls of an mbarrier before giving up

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };


// Launch arguments.  cf: [rows + 2][PITCH] pairs (e^, n^) from grid row -1
// (the layout of the on-chip CG kernel); scl: three planes [rows + 2][PITCH]
// of 1/c, 1/sqrt(c), sqrt(c).  ws: per cluster slot, slot_elems elements:
// five block vectors X^, R0, R1, P0, P1 of (rows + 2 PADR) S PITCH elements.
struct Args {
  KryArgs k;
  const void* cf;
  const void* scl;
  int rows;
  void* ws;
  size_t slot_elems;
  double thr;
};

template <typename T, int S, int PITCH>
struct Smem {
  using T2 = typename V2<T>::t;
  static constexpr int NW = PITCH / 64;                      // warps (two columns per thread)
  static constexpr int NU = S * (S + 1) / 2;                 // upper triangle of a symmetric S x S
  static constexpr int NV = 2 * NU + 2 * S * S + S;          // G, ZZ, H, ZR, r.r
  static constexpr int OG = 0, OZZ = NU, OH = 2 * NU, OZR = 2 * NU + S * S, ORR = 2 * NU + 2 * S * S;
  alignas(16) T ring[DR][3][S][PITCH];   // per slot: one row of P (old), R (old), X^
  T2 cfr[DR][PITCH];         // per slot: the coupling row
  T pb[4][S][PITCH];         // new directions of the last four rows (row m in pb[m & 3])
  T red[NV][NW];             // per-warp partial sums
  T part[2][NV][MAXCS];      // per-CTA partials of every CTA (pushed by each CTA)
  T tot[NV];                 // cluster totals
  T A[S][S];                 // Schur complements of the pivoted Cholesky
  T L[S][S];                 // its columns: L[i][k] = entry of original row i in column k
  T C1[S][S], C2[S][S], E[S][S];
  T2 C1s[S][S], nC1s[S][S], nC2s[S][S];   // C1, -C1, -C2 with each entry twice (packed operands)
  T dinv[S];                 // 1 / L[piv[k]][k]
  T dd[S], rr[S];            // d^.d^ and r.r per system
  alignas(8) unsigned long long mbar[DR];
  int piv[S];
  int rank, go, brk;
};

LRP_DEV uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

LRP_DEV void mbar_init(uint32_t a) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}

// Poll the mbarrier for the given phase parity, at most SPIN times.
LRP_DEV bool mbar_wait(uint32_t a, uint32_t parity) {
  for (long i = 0; i < SPIN; ++i) {
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

LRP_DEV void mbar_expect(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on mbarrier a.
LRP_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint32_t a) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(a)
      : "memory");
}

// Generic-proxy stores to global memory before this point are ordered before
// later bulk copies that read them (the copies of the next pass).
LRP_DEV void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// Shared-memory reads of a slot before this point are ordered before the
// bulk copy that overwrites it.
LRP_DEV void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Cluster-wide sums of NV values, in a fixed order (lanes, warps, CTAs, each
// by the same butterfly), so that every CTA gets bitwise the same totals in
// sh.tot; also a cluster barrier, after which the global and shared memory
// writes made before it by any CTA of the cluster are visible.
template <typename T, int NV, typename SM>
LRP_DEV void cl_reduce(cg::cluster_group& cl, const T (&v)[NV], SM& sh, int& buf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cs = (int)cl.num_blocks(), crank = (int)cl.block_rank();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const T s = warp_sum<T>(v[i]);
    if (lane == 0) sh.red[i][w] = s;
  }
  __syncthreads();
  for (int i = w; i < NV; i += SM::NW) {
    const T s = warp_sum<T>(lane < SM::NW ? sh.red[i][lane] : T(0));
    if (lane < cs) *cl.map_shared_rank(&sh.part[buf][i][crank], lane) = s;
  }
  cl.sync();
  for (int i = w; i < NV; i += SM::NW) {
    const T s = warp_sum<T>(lane < cs ? sh.part[buf][i][lane] : T(0));
    if (lane == 0) sh.tot[i] = s;
  }
  __syncthreads();
  buf ^= 1;
}

// Index of M[i][j] (i <= j) in the packed upper triangle, row by row.
template <int S> LRP_DEV constexpr int up_idx(int i, int j) { return i * S - i * (i - 1) / 2 + (j - i); }
template <int S> LRP_DEV constexpr int sym_idx(int i, int j) { return i <= j ? up_idx<S>(i, j) : up_idx<S>(j, i); }

template <typename T> LRP_DEV T rsqrt_(T v);
template <> LRP_DEV float rsqrt_<float>(float v) { return 1.0f / sqrtf(v); }
template <> LRP_DEV double rsqrt_<double>(double v) { return 1.0 / sqrt(v); }

// Warp 0: pivoted Cholesky of G (the packed upper triangle g), thresholded
// at thr times its largest diagonal entry; fills sh.L, sh.piv, sh.dinv,
// sh.rank.  Lane i < S works on row i of the Schur complement.
template <typename T, int S, typename SM>
LRP_DEV void pchol(const T* g, T thr, SM& sh) {
  const int lane = threadIdx.x & 31;
  if (lane < S) {
#pragma unroll
    for (int m = 0; m < S; ++m) {
      sh.A[lane][m] = g[sym_idx<S>(lane, m)];
      sh.L[lane][m] = T(0);
    }
  }
  __syncwarp();
  T dmax = lane < S ? sh.A[lane][lane] : T(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  bool used = false;
  int r = 0;
#pragma unroll 1
  for (int k = 0; k < S; ++k) {
    // the largest remaining diagonal entry (the lowest lane on ties; NaN
    // entries never win, so that every lane agrees)
    T best = T(-1);
    if (lane < S && !used) {
      const T dv = sh.A[lane][lane];
      if (dv == dv) best = dv;
    }
    int j = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, j, o);
      if (ob > best || (ob == best && oj < j)) { best = ob; j = oj; }
    }
    if (!(best > thr * dmax)) break;
    const T is = rsqrt_<T>(best);
    const T l = (lane < S && !used) ? sh.A[lane][j] * is : T(0);
    if (lane < S) sh.L[lane][k] = lane == j ? best * is : l;
    if (lane == j) {
      used = true;
      sh.piv[k] = j;
      sh.dinv[k] = is;
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < S; ++m) {
      const T lm = __shfl_sync(0xffffffffu, l, m);
      if (lane < S) sh.A[lane][m] -= l * lm;
    }
    __syncwarp();
    ++r;
  }
  if (lane == 0) sh.rank = r;
  __syncwarp();
}

// Warp 0: out = G+ Mt, Mt an S x S matrix (Mt[t][s] at m[t * S + s]); lane
// s < S solves for column s: L11 y = Mt[piv, s], L11^T z = y,
// out[piv[k]][s] = z[k], the other rows 0.
template <typename T, int S, typename SM>
LRP_DEV void gplus_apply(const T* m, T (*out)[S], SM& sh) {
  const int lane = threadIdx.x & 31;
  const int r = sh.rank;
  if (lane < S) {
    T y[S], z[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
      y[k] = T(0);
      z[k] = T(0);
      if (k < r) {
        T v = m[sh.piv[k] * S + lane];
#pragma unroll
        for (int q = 0; q < k; ++q) v -= sh.L[sh.piv[k]][q] * y[q];
        y[k] = v * sh.dinv[k];
      }
    }
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
      if (k < r) {
        T v = y[k];
#pragma unroll
        for (int q = k + 1; q < S; ++q)
          if (q < r) v -= sh.L[sh.piv[q]][k] * z[q];
        z[k] = v * sh.dinv[k];
      }
    }
#pragma unroll
    for (int t = 0; t < S; ++t) out[t][lane] = T(0);
#pragma unroll
    for (int k = 0; k < S; ++k)
      if (k < r) out[sh.piv[k]][lane] = z[k];
  }
  __syncwarp();
}

// Warp 0, on the totals of a pass: the pivoted factor of G, C1 = G+ H,
// E = ZR - ZZ C1, C2 = G+ E, and C1, -C1, -C2 with each entry doubled for
// packed operands; brk when no direction is left.
template <typename T, int S, typename SM>
LRP_DEV void block_coefficients(T thr, SM& sh) {
  using T2 = typename SM::T2;
  const int lane = threadIdx.x & 31;
  pchol<T, S>(sh.tot + SM::OG, thr, sh);
  if (sh.rank == 0) {
    if (lane == 0) sh.brk = 1;
    __syncwarp();
    return;
  }
  gplus_apply<T, S>(sh.tot + SM::OH, sh.C1, sh);
  if (lane < S) {
#pragma unroll
    for (int t = 0; t < S; ++t) {
      T v = sh.tot[SM::OZR + t * S + lane];
#pragma unroll
      for (int u = 0; u < S; ++u) v -= sh.tot[SM::OZZ + sym_idx<S>(t, u)] * sh.C1[u][lane];
      sh.E[t][lane] = v;
    }
  }
  __syncwarp();
  gplus_apply<T, S>(&sh.E[0][0], sh.C2, sh);
  if (lane < S) {
#pragma unroll
    for (int t = 0; t < S; ++t) {
      sh.C1s[t][lane] = T2{sh.C1[t][lane], sh.C1[t][lane]};
      sh.nC1s[t][lane] = T2{-sh.C1[t][lane], -sh.C1[t][lane]};
      sh.nC2s[t][lane] = T2{-sh.C2[t][lane], -sh.C2[t][lane]};
    }
  }
  __syncwarp();
}

// ---- two adjacent columns as one value ----------------------------------------
// a * b + c on both halves: one packed instruction in FP32, two in FP64.
LRP_DEV float2 vfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "mov.b64 pc, {%6, %7};\n\tfma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
LRP_DEV double2 vfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}

// (e^, n^) of columns c and c + 1 (c even) as (e^ pair, n^ pair)
LRP_DEV void ld_cf_pair(const float2* p, float2& e, float2& n) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  e = make_float2(q.x, q.z);
  n = make_float2(q.y, q.w);
}
LRP_DEV void ld_cf_pair(const double2* p, double2& e, double2& n) {
  const double2 a = p[0], b = p[1];
  e = make_double2(a.x, b.x);
  n = make_double2(a.y, b.y);
}

// Gram accumulators: in FP32 one packed pair per entry (the two columns'
// partial sums, added at the end), in FP64 one scalar per entry (registers).
template <typename T> struct AccT;
template <> struct AccT<float> { using t = float2; };
template <> struct AccT<double> { using t = double; };
LRP_DEV void acc_add(float2& a, float2 x, float2 y) { a = vfma(x, y, a); }
LRP_DEV void acc_add(double& a, double2 x, double2 y) {
  a = fma(x.x, y.x, a);
  a = fma(x.y, y.y, a);
}
LRP_DEV float acc_val(float2 a) { return a.x + a.y; }
LRP_DEV double acc_val(double a) { return a; }
LRP_DEV void acc_zero(float2& a) { a = make_float2(0.f, 0.f); }
LRP_DEV void acc_zero(double& a) { a = 0.0; }

template <int S, typename SM, typename A, typename V>
LRP_DEV void add_grams(A (&acc)[SM::NV], const V (&p)[S], const V (&z)[S], const V (&r)[S]) {
#pragma unroll
  for (int t = 0; t < S; ++t) {
#pragma unroll
    for (int s = t; s < S; ++s) {
      acc_add(acc[SM::OG + up_idx<S>(t, s)], p[t], z[s]);
      acc_add(acc[SM::OZZ + up_idx<S>(t, s)], z[t], z[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      acc_add(acc[SM::OH + t * S + s], p[t], r[s]);
      acc_add(acc[SM::OZR + t * S + s], z[t], r[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s) acc_add(acc[SM::ORR + s], r[s], r[s]);
}

template <typename T, int S, int PITCH, int RB>
__global__ void __launch_bounds__(PITCH / 2, 1) k_bcg(Args ba) {
  using SM = Smem<T, S, PITCH>;
  using V = typename SM::T2;      // two columns (the same type as a coupling pair)
  using A = typename AccT<T>::t;
  constexpr int NV = SM::NV;
  const KryArgs& a = ba.k;
  if (a.in.stop && *a.in.stop) return;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const int mx = a.mx, my = a.my;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int c0 = 2 * tid;                       // this thread's columns c0, c0 + 1
  const bool has_w = c0 > 0, has_e = c0 + 2 < PITCH;
  const int r0 = crank * RB;
  const int rows = ba.rows;
  const size_t plane = (size_t)(rows + 2) * PITCH;
  const size_t rowel = (size_t)S * PITCH;
  const size_t bstride = (size_t)(rows + 2 * PADR) * rowel;
  const V* const cf0 = static_cast<const V*>(ba.cf) + PITCH;    // grid row 0, column 0
  const V* __restrict__ cfc = cf0 + c0;
  const T* __restrict__ sc = static_cast<const T*>(ba.scl) + PITCH + c0;

  extern __shared__ __align__(128) unsigned char bk_smem_raw[];
  SM& sh = *reinterpret_cast<SM*>(bk_smem_raw);

  const int slot = blockIdx.x / cs, nslots = gridDim.x / cs;
  T* const ws = static_cast<T*>(ba.ws) + (size_t)slot * ba.slot_elems;
  T* const Xg = ws;
  T* const R0g = ws + bstride;
  T* const R1g = ws + 2 * bstride;
  T* const P0g = ws + 3 * bstride;
  T* const P1g = ws + 4 * bstride;
  auto rowp = [&](T* b, int row) -> T* { return b + (size_t)(row + PADR) * rowel; };
  // the pair (c0, c0 + 1) of system s in row `row` of a block vector
  auto gv = [&](T* b, int row, int s) -> V& {
    return *reinterpret_cast<V*>(rowp(b, row) + (size_t)s * PITCH + c0);
  };
  auto sv = [&](T* p) -> V& { return *reinterpret_cast<V*>(p); };
  const T thr = (T)ba.thr;
  const T rtol2 = (T)(a.rtol * a.rtol);
  const int max_iter = a.max_iter;
  const V vzero{T(0), T(0)};
  int buf = 0;
  unsigned long long my_iters = 0;
  int my_status = 0;
  uint32_t ph = 0;   // parity of the next phase of every ring slot (bit i), the same in all threads

  if (tid == 0) {
    for (int i = 0; i < DR; ++i) mbar_init(saddr(&sh.mbar[i]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  cl.sync();   // every CTA runs before remote accesses to its shared memory

  auto wait_slot = [&](int i) {
    const uint32_t par = (ph >> i) & 1u;
    if (!mbar_wait(saddr(&sh.mbar[i]), par) && !mbar_wait(saddr(&sh.mbar[i]), par)) my_status |= 4;
    ph ^= 1u << i;
  };
  auto reduce = [&](const A (&acc)[NV]) {
    T v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = acc_val(acc[i]);
    cl_reduce<T, NV>(cl, v, sh, buf);
  };
  // 5-point product of the scaled matrix at one row: centre pair pc, its
  // west and east neighbours (columns c0 - 1 and c0 + 2) pwv, pev, the rows
  // above and below pn, ps; couplings e^ (ec), e^ of the column to the west
  // (ew), n^ of the row (nc) and of the row below (ns)
  auto stencil = [&](V pc, T pwv, T pev, V pn, V ps, V ec, V ew, V nc, V ns) -> V {
    const V pe{pc.y, pev};
    const V pw{pwv, pc.x};
    V z = vfma(ec, pe, pc);
    z = vfma(ew, pw, z);
    z = vfma(nc, pn, z);
    z = vfma(ns, ps, z);
    return z;
  };

  // ---- one iteration: X^ += P C1, R_new = R - (B^ P) C1, P_new = R_new - P C2,
  // B^ P_new and the Gram matrices of (P_new, B^ P_new, R_new), one reduction
  auto main_pass = [&](int cur) {
    T* const Pk = cur ? P1g : P0g;
    T* const Rk = cur ? R1g : R0g;
    T* const Rn = cur ? R0g : R1g;
    T* const Pn = cur ? P0g : P1g;
    const int q0 = r0 - 2, q1 = r0 + RB + 1;
    const uint32_t rbytes = (uint32_t)(rowel * sizeof(T)), cbytes = (uint32_t)(PITCH * sizeof(V));
    // row q into its ring slot: the old directions always, the old residual
    // for rows r0 - 1 .. r0 + RB, X^ for own rows, the couplings inside -1 .. rows
    auto issue = [&](int q) {
      const int i = (q - q0) % DR;
      const bool hasR = q >= r0 - 1 && q <= r0 + RB;
      const bool hasX = q >= r0 && q < r0 + RB;
      const bool hasC = q >= -1 && q <= rows;
      const uint32_t mb = saddr(&sh.mbar[i]);
      mbar_expect(mb, rbytes * (1u + (hasR ? 1u : 0u) + (hasX ? 1u : 0u)) + (hasC ? cbytes : 0u));
      bulk_g2s(&sh.ring[i][0][0][0], rowp(Pk, q), rbytes, mb);
      if (hasR) bulk_g2s(&sh.ring[i][1][0][0], rowp(Rk, q), rbytes, mb);
      if (hasX) bulk_g2s(&sh.ring[i][2][0][0], rowp(Xg, q), rbytes, mb);
      if (hasC) bulk_g2s(&sh.cfr[i][0], cf0 + (long)q * PITCH, cbytes, mb);
    };
    if (tid == 0) {
      fence_async_global();
      fence_async_shared();
      for (int q = q0; q <= q1 && q < q0 + DR; ++q) issue(q);
    }
    A acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc_zero(acc[v]);
    wait_slot(0);
    wait_slot(1);
    V ec_p = vzero, ew_p = vzero, nc_p = vzero, ns_p = vzero;   // couplings of the previous centre row
    V rprev[S];                                                 // its new residual
#pragma unroll
    for (int s = 0; s < S; ++s) rprev[s] = vzero;
    int is = 0, ic = 1, in = 2;   // ring slots of rows q - 2, q - 1, q
#pragma unroll 1
    for (int q = r0; q <= q1; ++q) {
      const int c = q - 1;   // centre row: r0 - 1 .. r0 + RB
      wait_slot(in);
      V ec, nc, ew;
      ld_cf_pair(&sh.cfr[ic][c0], ec, nc);
      ew = V{has_w ? sh.cfr[ic][c0 - 1].x : T(0), ec.x};
      V ns = vzero;
      if (c - 1 >= -1) {
        V e_s;
        ld_cf_pair(&sh.cfr[is][c0], e_s, ns);
      }
      V pc[S], z[S], rn[S], pn[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const T* pr = &sh.ring[ic][0][s][c0];
        pc[s] = sv(const_cast<T*>(pr));
        const T pwv = has_w ? pr[-1] : T(0);
        const T pev = has_e ? pr[2] : T(0);
        z[s] = stencil(pc[s], pwv, pev, sv(&sh.ring[in][0][s][c0]), sv(&sh.ring[is][0][s][c0]), ec,
                       ew, nc, ns);
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V v = sv(&sh.ring[ic][1][s][c0]);
#pragma unroll
        for (int t = 0; t < S; ++t) v = vfma(z[t], sh.nC1s[t][s], v);
        rn[s] = v;
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V v = rn[s];
#pragma unroll
        for (int t = 0; t < S; ++t) v = vfma(pc[t], sh.nC2s[t][s], v);
        pn[s] = v;
      }
      if (c >= r0 && c < r0 + RB) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          V xv = sv(&sh.ring[ic][2][s][c0]);
#pragma unroll
          for (int t = 0; t < S; ++t) xv = vfma(pc[t], sh.C1s[t][s], xv);
          gv(Xg, c, s) = xv;
          gv(Rn, c, s) = rn[s];
          gv(Pn, c, s) = pn[s];
        }
      }
#pragma unroll
      for (int s = 0; s < S; ++s) sv(&sh.pb[c & 3][s][c0]) = pn[s];
      __syncthreads();
      // the slot of row q - 3 is read by no thread any more: refill it
      if (tid == 0 && q - 3 >= q0 && q - 3 + DR <= q1) {
        fence_async_shared();
        issue(q - 3 + DR);
      }
      // B^ P_new of the own row m = c - 1 (its neighbours' new directions are in pb)
      const int m = c - 1;
      if (m >= r0) {
        V pm[S], zm[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const T* pr = &sh.pb[m & 3][s][c0];
          pm[s] = sv(const_cast<T*>(pr));
          const T pwv = has_w ? pr[-1] : T(0);
          const T pev = has_e ? pr[2] : T(0);
          zm[s] = stencil(pm[s], pwv, pev, sv(&sh.pb[c & 3][s][c0]), sv(&sh.pb[(m - 1) & 3][s][c0]),
                          ec_p, ew_p, nc_p, ns_p);
        }
        add_grams<S, SM>(acc, pm, zm, rprev);
      }
      ec_p = ec;
      ew_p = ew;
      nc_p = nc;
      ns_p = ns;
#pragma unroll
      for (int s = 0; s < S; ++s) rprev[s] = rn[s];
      is = ic;
      ic = in;
      in = in + 1 == DR ? 0 : in + 1;
    }
    fence_async_global();   // X^, R_new, P_new stores before the next pass's bulk copies
    reduce(acc);
  };

  const int nblk = (a.nsys + S - 1) / S;
  for (int blk = slot; blk < nblk; blk += nslots) {
    const int sys0 = blk * S;
    const int ncols = min(S, a.nsys - sys0);
    // ---- X^ = sqrt(c) x, own rows (systems beyond nsys: 0) --------------------
    for (int i = 0; i < RB; ++i) {
      const int row = r0 + i;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        T v2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = c0 + h;
          T v = T(0);
          if (col < mx && row < my && s < ncols) {
            const int sys = sys0 + s, k = row * mx + col;
            if (a.in.gen)
              v = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                           (uint32_t)(sys % a.in.ncol), (uint32_t)k);
            else if (a.in.x != nullptr) {
              const long ox = sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys);
              v = a.in.x_f64 ? (T) static_cast<const double*>(a.in.x)[ox + k]
                             : (T) static_cast<const float*>(a.in.x)[ox + k];
            }
            v *= sc[(long)row * PITCH + 2 * plane + h];
          }
          v2[h] = v;
        }
        gv(Xg, row, s) = V{v2[0], v2[1]};
      }
    }
    fence_async_global();
    cl.sync();   // X^ rows visible to the neighbouring CTAs
    int cur = 0;
    for (int j = 0; j < a.M; ++j) {
      // ---- d^ = X^ / c, R = d^ - B^ X^; d^.d^, r.r per system -----------------
      {
        A acc[2 * S];
#pragma unroll
        for (int v = 0; v < 2 * S; ++v) acc_zero(acc[v]);
        V xs[S], xc[S], xn[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          xs[s] = gv(Xg, r0 - 1, s);
          xc[s] = gv(Xg, r0, s);
        }
        V ns, e_s;
        ld_cf_pair(cfc + (long)(r0 - 1) * PITCH, e_s, ns);
        T* const Rk = cur ? R1g : R0g;
#pragma unroll 1
        for (int i = 0; i < RB; ++i) {
          const int row = r0 + i;
          V ec, nc;
          ld_cf_pair(cfc + (long)row * PITCH, ec, nc);
          const V ew{has_w ? cfc[(long)row * PITCH - 1].x : T(0), ec.x};
          const V ic{sc[(long)row * PITCH], sc[(long)row * PITCH + 1]};
#pragma unroll
          for (int s = 0; s < S; ++s) xn[s] = gv(Xg, row + 1, s);
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const T* xr = rowp(Xg, row) + (size_t)s * PITCH + c0;
            const T xw = has_w ? xr[-1] : T(0);
            const T xe = has_e ? xr[2] : T(0);
            const V bx = stencil(xc[s], xw, xe, xn[s], xs[s], ec, ew, nc, ns);
            const V d{ic.x * xc[s].x, ic.y * xc[s].y};
            const V rk{d.x - bx.x, d.y - bx.y};
            gv(Rk, row, s) = rk;
            acc_add(acc[s], d, d);
            acc_add(acc[S + s], rk, rk);
          }
          ns = nc;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            xs[s] = xc[s];
            xc[s] = xn[s];
          }
        }
        fence_async_global();
        T v[2 * S];
#pragma unroll
        for (int i = 0; i < 2 * S; ++i) v[i] = acc_val(acc[i]);
        cl_reduce<T, 2 * S>(cl, v, sh, buf);
        if (tid == 0) {
          bool go = false;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            sh.dd[s] = sh.tot[s];
            sh.rr[s] = sh.tot[S + s];
            go |= !(sh.rr[s] <= rtol2 * sh.dd[s]);   // NaN: not converged
          }
          sh.go = go && max_iter > 0;
          sh.brk = 0;
        }
        __syncthreads();
      }
      int it = 0;
      if (sh.go) {
        // ---- P = R; B^ P and the Gram matrices of (P, B^ P, R) --------------------
        A acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc_zero(acc[v]);
        T* const Rk = cur ? R1g : R0g;
        T* const Pk = cur ? P1g : P0g;
        V rs[S], rc[S], rnx[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          rs[s] = gv(Rk, r0 - 1, s);
          rc[s] = gv(Rk, r0, s);
        }
        V ns, e_s;
        ld_cf_pair(cfc + (long)(r0 - 1) * PITCH, e_s, ns);
#pragma unroll 1
        for (int i = 0; i < RB; ++i) {
          const int row = r0 + i;
          V ec, nc;
          ld_cf_pair(cfc + (long)row * PITCH, ec, nc);
          const V ew{has_w ? cfc[(long)row * PITCH - 1].x : T(0), ec.x};
          V z[S];
#pragma unroll
          for (int s = 0; s < S; ++s) rnx[s] = gv(Rk, row + 1, s);
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const T* rr_ = rowp(Rk, row) + (size_t)s * PITCH + c0;
            const T rw = has_w ? rr_[-1] : T(0);
            const T re = has_e ? rr_[2] : T(0);
            z[s] = stencil(rc[s], rw, re, rnx[s], rs[s], ec, ew, nc, ns);
            gv(Pk, row, s) = rc[s];
          }
          add_grams<S, SM>(acc, rc, z, rc);
          ns = nc;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            rs[s] = rc[s];
            rc[s] = rnx[s];
          }
        }
        fence_async_global();
        reduce(acc);
        if (wid == 0) block_coefficients<T, S>(thr, sh);
        __syncthreads();
      }
      while (sh.go && !sh.brk) {
        main_pass(cur);
        cur ^= 1;
        ++it;
        if (wid == 0) {
          if (lane == 0) {
            bool go = false;
#pragma unroll
            for (int s = 0; s < S; ++s) {
              sh.rr[s] = sh.tot[SM::ORR + s];
              go |= !(sh.rr[s] <= rtol2 * sh.dd[s]);
            }
            sh.go = go && it < max_iter;
          }
          __syncwarp();
          if (sh.go) block_coefficients<T, S>(thr, sh);
        }
        __syncthreads();
      }
      if (sh.brk) {
        my_status |= 2;
      } else {
        bool left = false;
#pragma unroll
        for (int s = 0; s < S; ++s) left |= !(sh.rr[s] <= rtol2 * sh.dd[s]);
        if (left) my_status |= 1;
      }
      my_iters += (unsigned long long)it * ncols;
      __syncthreads();
    }
    // ---- x = X^ / sqrt(c), own rows ---------------------------------------------------
    for (int i = 0; i < RB; ++i) {
      const int row = r0 + i;
      if (row >= my) continue;
      for (int s = 0; s < ncols; ++s) {
        const V xv = gv(Xg, row, s);
        const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys0 + s);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = c0 + h;
          if (col >= mx) continue;
          const T v = (h ? xv.y : xv.x) * sc[(long)row * PITCH + plane + h];
          const long k = (long)row * mx + col;
          if (a.out.y_f64)
            static_cast<double*>(a.out.y)[oy + k] = (double)v;
          else
            static_cast<float*>(a.out.y)[oy + k] = (float)v;
        }
      }
    }
    cl.sync();   // the neighbours' last reads of our rows are done before the next block
  }
  if (tid == 0 && crank == 0) {
    if (my_iters) atomicAdd(a.iters, my_iters);
  }
  if (tid == 0 && my_status) atomicOr(a.status, my_status);
}

struct Variant {
  const void* fn;
  size_t smem;
  int S, pitch, rb;
  int threads;   // pitch / 2: two grid columns per thread
};
Variant variant_f32(int pitch);
Variant variant_f64(int pitch);

template <typename T, int S, int PITCH, int RB>
Variant make_variant() {
  return Variant{(const void*)k_bcg<T, S, PITCH, RB>, sizeof(Smem<T, S, PITCH>), S, PITCH, RB,
                 PITCH / 2};
}

}  // namespace bk
}  // namespace lrp
