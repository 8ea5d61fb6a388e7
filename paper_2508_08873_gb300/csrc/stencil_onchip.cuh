// Conjugate gradients for the backward-Euler steps of a symmetric 5-point
// operator with every Krylov vector held on chip (the kernel template; the
// launch code is in stencil_onchip.cu, the instantiations in
// stencil_onchip_f32.cu and stencil_onchip_f64.cu).
//
// The iteration is Jacobi-preconditioned CG written as plain CG on the
// diagonally scaled system: with S = diag(sqrt(c)) (c the diagonal of
// B = I + dt A), B^ = S^-1 B S^-1 has a unit diagonal, x^ = S x and
// d^ = S^-1 d, and CG on B^ x^ = d^ produces the iterates of CG on B x = d
// preconditioned by diag(B) (the same Krylov spaces and scalars in exact
// arithmetic).  An iteration then needs only the scaled east and north
// couplings e^, n^ of every point (the west and south ones are the
// neighbours' e^ and n^, B^ being symmetric) and no diagonal; it stops when
// ||d^ - B^ x^|| <= rtol ||d^||, the residual of the scaled system.
//
// One system runs on one thread-block cluster of cs CTAs.  CTA c owns grid
// rows [c RPT, c RPT + RPT) (the row count padded to cs RPT with rows whose
// couplings and scales are 0, which stay 0), thread t owns grid column t
// (PITCH >= mx threads, the columns beyond mx inert likewise), and keeps its
// column's entries of p and r (and q = B^ p, in registers or, for QSM, in
// shared memory) for the whole propagation, x^ in shared memory.  Stencil
// neighbours: north and south are the thread's own rows; east and west come
// from the adjacent lanes by shuffles and, at warp edges, from a shared
// table of the warps' edge entries; the row above the CTA's first row and
// below its last (the halo) is a redundant copy of the neighbouring CTA's
// p and r, advanced with that CTA's q of the row (read through distributed
// shared memory after the reduction barrier that follows it) by the same
// fused multiply-adds, so that it stays bitwise equal to the owner's entries.
// The couplings are streamed from L2 (a pitched copy shared by every system
// of the launch) through a ring of KA rows in flight per thread
// (cp.async: each thread copies, and later reads, only its own column, so
// the ring needs no barrier beyond the thread's own wait_group).  An
// iteration reads no Krylov vector from global memory and synchronises the
// cluster twice, at its two reductions (p.q, then r.r).
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace lrp {
namespace oc {

namespace cg = cooperative_groups;

constexpr int MAXCS = 16;   // CTAs per cluster (non-portable cluster size)

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

// Explicitly rounded operations, so that a halo copy and the owner of a row
// compute the same values whatever the compiler contracts.
template <typename T> LRP_DEV T fma_rn(T a, T b, T c);
template <> LRP_DEV float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> LRP_DEV double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// The coefficient ring: copies (cp.async), waits and the reads of the ring
// are all volatile asm statements, which keep their order among themselves,
// and none of them clobbers memory, so that the compiler may interleave the
// rest of the arithmetic and shared-memory traffic of neighbouring rows
// around them (nothing else touches the ring).
template <int B> LRP_DEV void cpa(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(src), "n"(B));
}
LRP_DEV void cpa_commit() { asm volatile("cp.async.commit_group;"); }
template <int N> LRP_DEV void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }
LRP_DEV void cpa_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
LRP_DEV float2 ring_ld(const float2* p) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
               : "=f"(v.x), "=f"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}
LRP_DEV double2 ring_ld(const double2* p) {
  double2 v;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];"
               : "=d"(v.x), "=d"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}
// v is computed before this point: it consumes ring entries that the next
// copy into the same slot overwrites.
LRP_DEV void consumed(float v) { asm volatile("" ::"f"(v)); }
LRP_DEV void consumed(double v) { asm volatile("" ::"d"(v)); }

// Launch arguments.  cf: [rows + 2][PITCH] pairs (e^, n^) from grid row -1
// to row `rows` (rows = cs RPT; rows -1 and beyond my-1 are 0); scl: three
// planes [rows + 2][PITCH] of 1/c, 1/sqrt(c) and sqrt(c) (0 outside the grid).
struct Args {
  KryArgs k;
  const void* cf;
  const void* scl;
  int rows;
  // time-dependent operators (TD kernels): the layouts of the rows of the
  // time grid follow one another, cf_step pairs and scl_step scales apart
  long cf_step, scl_step;
};

template <typename T, int PITCH, int RPT, bool QSM, int KA>
struct Smem {
  static constexpr int NW = PITCH / 32;
  T xs[RPT][PITCH];                 // x^ of own rows
  T qs[QSM ? RPT : 1][PITCH];       // q (QSM)
  typename V2<T>::t ring[KA][PITCH];// (e^, n^) rows in flight
  T pedge[RPT][NW + 2][2];          // p of lanes 0 and 31 of warp w at [w + 1]; zero pads
  T wco[RPT][NW];                   // e^ of the column left of each warp's lane 0
  T junk[NW][32];                   // target of the edge-table stores of lanes 1..30
  T xedge[2][PITCH], redge[2][PITCH], qedge[2][PITCH];   // first and last row
  T red[4][NW];                     // per-warp partial sums
  T part[2][4][MAXCS];              // per-CTA partials of every CTA (pushed by each CTA)
  T scal[4];                        // scalars of the iteration, set by thread 0
  int flag[2];
};

// Cluster-wide sums of NV values in the working precision, in a fixed
// order (lanes, warps, CTAs, each by the same butterfly), so that every CTA
// gets bitwise the same totals; also a cluster barrier (shared-memory
// stores made before it by any CTA are visible after it).  Thread 0 then
// runs fin(tot) to set the iteration's scalars in shared memory, which
// every thread reads after the closing block barrier: no thread but one
// does scalar arithmetic (on GB300 a division in FP64 by every warp costs
// thousands of cycles of the sub-partitions' FP64 units).
template <typename T, int NV, typename SM, typename Fin>
LRP_DEV void cl_sum(cg::cluster_group& cl, const T (&v)[NV], SM& sh, int& buf, Fin fin) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cs = (int)cl.num_blocks(), crank = (int)cl.block_rank();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const T s = warp_sum<T>(v[i]);
    if (lane == 0) sh.red[i][w] = s;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const T s = warp_sum<T>(lane < SM::NW ? sh.red[i][lane] : T(0));
      if (lane < cs) *cl.map_shared_rank(&sh.part[buf][i][crank], lane) = s;
    }
  }
  cl.sync();
  if (w == 0) {
    T tot[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = warp_sum<T>(lane < cs ? sh.part[buf][i][lane] : T(0));
    if (lane == 0) fin(tot);
  }
  __syncthreads();
  buf ^= 1;
}

// TD: a time-dependent operator, every fine step its own couplings and scales
// (the system's steps J0 .. J0 + M - 1 of its interval, reversed for the
// adjoint; between steps x^ = S x is rescaled to the new diagonal).
template <typename T, int PITCH, int RPT, bool QSM, int KA, bool TD = false>
__global__ void __launch_bounds__(PITCH, 512 / PITCH) k_cg_onchip(Args oa) {
  using T2 = typename V2<T>::t;
  using SM = Smem<T, PITCH, RPT, QSM, KA>;
  constexpr int NW = SM::NW;
  const KryArgs& a = oa.k;
  if (a.in.stop && *a.in.stop) return;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const int mx = a.mx, my = a.my, n = a.n;
  const int col = threadIdx.x, lane = col & 31, wid = col >> 5;
  const int r0 = crank * RPT;
  const bool has_up = crank > 0, has_dn = crank < cs - 1;
  const size_t plane = (size_t)(oa.rows + 2) * PITCH;
  // this thread's column from our first row on: coupling pairs and scales
  const T2* __restrict__ cf0 = static_cast<const T2*>(oa.cf) + (size_t)(r0 + 1) * PITCH + col;
  const T* __restrict__ sc0 = static_cast<const T*>(oa.scl) + (size_t)(r0 + 1) * PITCH + col;
  const T2* __restrict__ cfc = cf0;
  const T* __restrict__ sc = sc0;

  extern __shared__ __align__(16) unsigned char oc_smem_raw[];
  SM& sh = *reinterpret_cast<SM*>(oc_smem_raw);
  // zero pads of the warp-edge table; e^ left of each warp's lane 0
  for (int t = col; t < RPT * 2; t += PITCH) {
    const int i = t >> 1, side = t & 1;
    sh.pedge[i][side ? NW + 1 : 0][0] = T(0);
    sh.pedge[i][side ? NW + 1 : 0][1] = T(0);
  }
  if (lane == 0)
    for (int i = 0; i < RPT; ++i) sh.wco[i][wid] = cfc[(long)i * PITCH - 1].x;
  T s_first = cfc[-PITCH].y;    // n^ of the row above ours: south coupling of row 0
  // TD: the couplings and scales of row `row` of the time grid (the warp-edge
  // couplings are read and used by each warp's lane 0 alone)
  auto set_row = [&](long row) {
    cfc = cf0 + row * oa.cf_step;
    sc = sc0 + row * oa.scl_step;
    if (lane == 0)
      for (int i = 0; i < RPT; ++i) sh.wco[i][wid] = cfc[(long)i * PITCH - 1].x;
    s_first = cfc[-PITCH].y;
  };
  cl.sync();   // every CTA runs before remote accesses to its shared memory

  // where this lane's p of row i goes in the warp-edge table: lanes 0 and 31
  // store into the table, the others into their scratch slot (one store per
  // lane, no divergent branch)
  auto edge_slot = [&](int i) -> T* {
    return lane == 0 ? &sh.pedge[i][wid + 1][0]
                     : lane == 31 ? &sh.pedge[i][wid + 1][1] : &sh.junk[wid][lane];
  };
  auto up_ = [&](T (*e)[PITCH]) -> T { return *cl.map_shared_rank(&e[1][col], crank - 1); };
  auto dn_ = [&](T (*e)[PITCH]) -> T { return *cl.map_shared_rank(&e[0][col], crank + 1); };
  auto issue = [&](const T2* cb, int i, int slot) {   // row i of the couplings into ring slot
    cpa<sizeof(T2)>(&sh.ring[slot][col], cb + (long)i * PITCH);
  };

  const T dt = (T)a.dt;
  const int slot = blockIdx.x / cs, nslots = gridDim.x / cs;
  int buf = 0;
  unsigned long long my_iters = 0;
  int my_status = 0;

  for (int sys = slot; sys < a.nsys; sys += nslots) {
    long J0 = 0;
    if constexpr (TD) {
      // the interval of the system (system map of the input, else of the
      // output, else of the source; else interval0 + sys / ncol): its steps
      const int* imap = a.in.map ? a.in.map : a.out.map ? a.out.map : a.src.map;
      const int interval = imap ? imap[2 * sys + 1] : a.in.interval0 + sys / a.in.ncol;
      J0 = (long)interval * a.M;
      if (J0 < 0 || J0 + a.M > a.nJ) continue;   // outside the time grid (checked on the host)
      set_row(a.adj ? J0 + a.M - 1 : J0);
    }
    // ---- x^ = S x ------------------------------------------------------------
    const long ox = a.in.gen || a.in.x == nullptr
        ? 0 : sys_offset(a.in.map, a.in.slot_stride, a.in.ldx, sys);
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      T v = T(0);
      if (col < mx && row < my) {
        const int k = row * mx + col;
        if (a.in.gen)
          v = gauss<T>(a.in.seed, a.in.stream, (uint32_t)(a.in.interval0 + sys / a.in.ncol),
                       (uint32_t)(sys % a.in.ncol), (uint32_t)k);
        else if (a.in.x != nullptr)
          v = a.in.x_f64 ? (T) static_cast<const double*>(a.in.x)[ox + k]
                         : (T) static_cast<const float*>(a.in.x)[ox + k];
        if (a.M > 0) v *= sc[(long)i * PITCH + 2 * plane];   // M = 0 returns x unchanged
      }
      sh.xs[i][col] = v;
    }
    sh.xedge[0][col] = sh.xs[0][col];
    sh.xedge[1][col] = sh.xs[RPT - 1][col];
    const double* csys = a.src.Q > 0
        ? a.src.c + sys_offset(a.src.map, a.src.c_slot_stride, a.src.cstride, sys) : nullptr;
    const double* gsys = (a.src.Q > 0 && a.src.map)
        ? a.src.g + (long)a.src.map[2 * sys] * a.src.g_slot_stride : a.src.g;
    cl.sync();   // x^ edges visible to the neighbours

    T p[RPT], r[RPT], qreg[QSM ? 1 : RPT];
    auto Q = [&](int i) -> T& {
      if constexpr (QSM) return sh.qs[i][col];
      else return qreg[i];
    };
    T p_up = T(0), r_up = T(0), p_dn = T(0), r_dn = T(0);
    for (int j = 0; j < a.M; ++j) {
      if constexpr (TD) {
        if (j > 0) {
          // the next step's matrix: x^ = S_J x rescaled from the previous S
          const T* sp = sc;
          set_row(a.adj ? J0 + a.M - 1 - j : J0 + j);
          cpa_wait_all();
          for (int i = 0; i < RPT; ++i)
            sh.xs[i][col] = sh.xs[i][col] * sp[(long)i * PITCH + plane] * sc[(long)i * PITCH + 2 * plane];
          sh.xedge[0][col] = sh.xs[0][col];
          sh.xedge[1][col] = sh.xs[RPT - 1][col];
          cl.sync();   // the neighbours' halo rows of x^ are read below
        }
      }
      // ---- d^ = x^ / c + dt S^-1 f,  r = p = d^ - B^ x^ ----------------------
      cpa_wait_all();
      T red2t[2] = {T(0), T(0)};     // d^.d^, r.r
      {
        const T xu = has_up ? up_(sh.xedge) : T(0);
        const T xd = has_dn ? dn_(sh.xedge) : T(0);
        auto row = [&](int i) -> T {
          const T2* cr = cfc + (long)i * PITCH;
          const T xc = sh.xs[i][col];
          const T xw = col > 0 ? sh.xs[i][col - 1] : T(0);
          const T xe = col + 1 < PITCH ? sh.xs[i][col + 1] : T(0);
          const T xso = i > 0 ? sh.xs[i - 1][col] : xu;
          const T xno = i < RPT - 1 ? sh.xs[i + 1][col] : xd;
          T f = T(0);
          if (csys && col < mx && r0 + i < my)
            for (int qq = 0; qq < a.src.Q; ++qq)
              f += (T)csys[(size_t)j * a.src.Q + qq] * (T)gsys[(size_t)qq * n + (r0 + i) * mx + col];
          const T* s = sc + (long)i * PITCH;
          const T d = s[0] * xc + dt * s[plane] * f;
          const T2 c2 = cr[0];
          T bx = xc;
          bx += c2.x * xe;
          bx += cr[-1].x * xw;
          bx += c2.y * xno;
          bx += cr[-PITCH].y * xso;
          const T rk = d - bx;
          red2t[0] += d * d;
          red2t[1] += rk * rk;
          if (i == 0) sh.redge[0][col] = rk;
          if (i == RPT - 1) sh.redge[1][col] = rk;
          *edge_slot(i) = rk;
          return rk;
        };
        if constexpr (QSM) {
#pragma unroll 1
          for (int i = 0; i < RPT; ++i) sh.qs[i][col] = row(i);
          T chk = T(0);
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            r[i] = sh.qs[i][col];
            p[i] = r[i];
            chk += r[i];
          }
          consumed(chk);
        } else {
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            r[i] = row(i);
            p[i] = r[i];
            asm volatile("" ::: "memory");   // one row's loads at a time
          }
        }
      }
      {
#pragma unroll
        for (int s = 0; s < KA; ++s) {
          issue(cfc, s, s);
          cpa_commit();
        }
      }
      // scal: [0] r.r, [1] rtol^2 d^.d^, [2] alpha, [3] beta; flag: [0] go on, [1] breakdown
      const T rtol2 = (T)(a.rtol * a.rtol);
      const int max_iter = a.max_iter;
      cl_sum<T, 2>(cl, red2t, sh, buf, [&](const T (&t)[2]) {
        sh.scal[0] = t[1];
        sh.scal[1] = rtol2 * t[0];
        sh.flag[0] = t[1] > rtol2 * t[0] && max_iter > 0;
        sh.flag[1] = 0;
      });
      if (has_up) { r_up = up_(sh.redge); p_up = r_up; }
      if (has_dn) { r_dn = dn_(sh.redge); p_dn = r_dn; }
      int it = 0;
      while (sh.flag[0]) {
        // ---- q = B^ p, p.q ------------------------------------------------------
        // Row i is in ring slot i % KA; row i refills the slot row i - 2 used
        // (with row i - 2 + KA), so that no row waits for its own result
        // before the next row's loads.  One commit per row: at row i at least
        // KA - 3 newer groups are in flight.
        T pq[1] = {T(0)};
        T cs_prev = s_first;
        T hist[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          cpa_wait<KA - 3>();
          const T2 c2 = ring_ld(&sh.ring[i % KA][col]);
          const T pc = p[i];
          // west: e^(k-1) p(k-1) is lane-1's product (lane 0: from the tables)
          const T vw_own = c2.x * pc;
          T vw = __shfl_up_sync(0xffffffffu, vw_own, 1);
          T pe = __shfl_down_sync(0xffffffffu, pc, 1);
          const T vw0 = sh.wco[i][wid] * sh.pedge[i][wid][1];
          const T pe31 = sh.pedge[i][wid + 2][0];
          vw = lane == 0 ? vw0 : vw;
          pe = lane == 31 ? pe31 : pe;
          const T ps = i > 0 ? p[i > 0 ? i - 1 : 0] : p_up;
          const T pn = i < RPT - 1 ? p[i + 1 < RPT ? i + 1 : i] : p_dn;
          T acc = pc + vw;
          acc = fma_rn(c2.x, pe, acc);
          acc = fma_rn(c2.y, pn, acc);
          acc = fma_rn(cs_prev, ps, acc);
          cs_prev = c2.y;
          Q(i) = acc;
          pq[0] = fma_rn(pc, acc, pq[0]);
          if (i == 0) sh.qedge[0][col] = acc;
          if (i == RPT - 1) sh.qedge[1][col] = acc;
          hist[i % 3] = acc;
          if (i >= 2) {
            consumed(hist[(i + 1) % 3]);           // row i - 2's result
            if (i - 2 + KA < RPT) issue(cfc, i - 2 + KA, (i - 2) % KA);
          }
          cpa_commit();
        }
        // every ring slot has been read: the next pass's first KA rows (the
        // couplings are constant) go in flight now, under the reductions
        consumed(hist[0] + hist[1] + hist[2]);
#pragma unroll
        for (int s = 0; s < KA; ++s) {
          issue(cfc, s, s);
          cpa_commit();
        }
        cl_sum<T, 1>(cl, pq, sh, buf, [&](const T (&t)[1]) {
          if (t[0] > T(0)) sh.scal[2] = sh.scal[0] / t[0];
          else sh.flag[1] = 1;
        });
        if (sh.flag[1]) { my_status |= 2; break; }
        const T alpha = sh.scal[2];
        // ---- x^ += alpha p, r -= alpha q, r.r -------------------------------------
        T rrt[1] = {T(0)};
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const T xn = fma_rn(alpha, p[i], sh.xs[i][col]);
          sh.xs[i][col] = xn;
          if (i == 0) sh.xedge[0][col] = xn;
          if (i == RPT - 1) sh.xedge[1][col] = xn;
          const T rk = fma_rn(-alpha, Q(i), r[i]);
          r[i] = rk;
          rrt[0] = fma_rn(rk, rk, rrt[0]);
        }
        if (has_up) r_up = fma_rn(-alpha, up_(sh.qedge), r_up);
        if (has_dn) r_dn = fma_rn(-alpha, dn_(sh.qedge), r_dn);
        ++it;
        cl_sum<T, 1>(cl, rrt, sh, buf, [&](const T (&t)[1]) {
          sh.scal[3] = t[0] / sh.scal[0];
          sh.scal[0] = t[0];
          sh.flag[0] = t[0] > sh.scal[1] && it < max_iter;
        });
        const T beta = sh.scal[3];
        // ---- p = r + beta p (own rows, halo copies, warp-edge table) -------------
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const T pk = fma_rn(beta, p[i], r[i]);
          p[i] = pk;
          *edge_slot(i) = pk;
        }
        if (has_up) p_up = fma_rn(beta, p_up, r_up);
        if (has_dn) p_dn = fma_rn(beta, p_dn, r_dn);
        __syncthreads();
      }
      if (!sh.flag[1] && sh.scal[0] > sh.scal[1]) my_status |= 1;
      my_iters += it;
      __syncthreads();   // x^ of the last update visible to the whole CTA
    }
    cpa_wait_all();
    // ---- x = S^-1 x^ ----------------------------------------------------------
    const long oy = sys_offset(a.out.map, a.out.slot_stride, a.out.ldy, sys);
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      if (col < mx && row < my) {
        const int k = row * mx + col;
        const T v = a.M > 0 ? sh.xs[i][col] * sc[(long)i * PITCH + plane] : sh.xs[i][col];
        if (a.out.y_f64)
          static_cast<double*>(a.out.y)[oy + k] = (double)v;
        else
          static_cast<float*>(a.out.y)[oy + k] = (float)v;
      }
    }
    cl.sync();   // neighbours have read our edge rows before the next system overwrites them
  }
  cpa_wait_all();
  if (threadIdx.x == 0 && crank == 0) {
    if (my_iters) atomicAdd(a.iters, my_iters);
    if (my_status) atomicOr(a.status, my_status);
  }
}

// Instantiation table: kernel pointer and shared-memory bytes per (PITCH, RPT).
struct Variant {
  const void* fn;
  size_t smem;
};
Variant variant_f32(int pitch, int rpt);
Variant variant_f64(int pitch, int rpt);

Variant variant_f32_td(int pitch, int rpt);

template <typename T, int PITCH, int RPT, bool QSM, int KA, bool TD = false>
Variant make_variant() {
  return Variant{(const void*)k_cg_onchip<T, PITCH, RPT, QSM, KA, TD>,
                 sizeof(Smem<T, PITCH, RPT, QSM, KA>)};
}

}  // namespace oc
}  // namespace lrp
