// Launch code of the on-chip CG propagator for symmetric 5-point operators
// (kernel in stencil_onchip.cuh): the coefficients of the diagonally scaled
// step matrix, the choice of the variant (grid pitch, rows per CTA, CTAs per
// cluster) and the launch.
#include <algorithm>
#include <cmath>

#include "stencil_onchip.cuh"

namespace lrp {

using oc::Variant;

// Scaled couplings and scales from the padded plan arrays (c, w, e, s, n,
// 1/c with mx zero entries on both sides, see stencil.cu): for grid row
// `row` in -1..rows and column `col` < pitch, cf = (e / sqrt(c c_east),
// n / sqrt(c c_north)) and scl = (1/c, 1/sqrt(c), sqrt(c)), all 0 outside
// the grid.  FP64 arithmetic, rounded to T.
template <typename T>
__global__ void k_oc_coef(int mx, int my, int pitch, int rows, const double* __restrict__ B,
                          typename oc::V2<T>::t* __restrict__ cf, T* __restrict__ scl) {
  const int n = mx * my;
  const size_t ld = (size_t)n + 2 * mx;
  const size_t plane = (size_t)(rows + 2) * pitch;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (rows + 2) * pitch) return;
  // time-dependent operators: grid row y of the launch is row y of the time
  // grid (its plan 6 ld values further, its layout 5 planes further)
  B += (size_t)blockIdx.y * 6 * ld;
  cf += (size_t)blockIdx.y * 5 * plane / 2;
  scl += (size_t)blockIdx.y * 5 * plane;
  const int row = t / pitch - 1, col = t % pitch;
  double e = 0.0, nn = 0.0, d = 0.0, si = 0.0, s = 0.0;
  if (row >= 0 && row < my && col < mx) {
    const size_t p = (size_t)mx + (size_t)row * mx + col;
    const double c = B[p];
    si = 1.0 / sqrt(c);
    s = sqrt(c);
    d = 1.0 / c;
    if (col + 1 < mx) e = B[2 * ld + p] / sqrt(c * B[p + 1]);
    if (row + 1 < my) nn = B[4 * ld + p] / sqrt(c * B[p + mx]);
  }
  cf[t].x = (T)e;
  cf[t].y = (T)nn;
  scl[t] = (T)d;
  scl[plane + t] = (T)si;
  scl[2 * plane + t] = (T)s;
}

// rows of the time grid a plan holds: one per fine step (two per step with
// an SDIRK stepper) for time-dependent operators, else one
static size_t oc_time_rows(const Operator* op) {
  return op->kind == 3 ? (size_t)op->nJ * (op->stepper ? 2 : 1) : 1;
}

lrp_status oc_coef_fill(Ctx* c, const Operator* op, const StencilPlan* plan, int prec, int pitch,
                        int rows, DevBuf& buf) {
  const size_t es = prec == 0 ? 8 : 4;
  const size_t tot = (size_t)(rows + 2) * pitch;
  const size_t nrows = oc_time_rows(op);
  const size_t need = tot * es * 5 * nrows;  // (e^, n^) pairs + three scale planes per row
  lrp_status s;
  // owned by the operator's context: plans outlive the contexts that use them
  if (buf.bytes < need && (s = dev_alloc(op->ctx, buf, need))) return s;
  const dim3 nb((unsigned)((tot + 255) / 256), (unsigned)nrows);
  if (prec == 0)
    k_oc_coef<double><<<nb, 256, 0, c->stream>>>(
        op->mx, op->my, pitch, rows, plan->b64.as<double>(),
        reinterpret_cast<double2*>(buf.ptr), static_cast<double*>(buf.ptr) + 2 * tot);
  else
    k_oc_coef<float><<<nb, 256, 0, c->stream>>>(
        op->mx, op->my, pitch, rows, plan->b64.as<double>(),
        reinterpret_cast<float2*>(buf.ptr), static_cast<float*>(buf.ptr) + 2 * tot);
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_err(c, e, "k_oc_coef");
  return LRP_OK;
}

lrp_status plan_layout(Ctx* c, Operator* op, StencilPlan* plan, int prec, int pitch, int rows,
                       void** ptr) {
  std::lock_guard<std::mutex> lk(op->plan_mu);
  for (auto& l : plan->layouts)
    if (l->prec == prec && l->pitch == pitch && l->rows == rows) {
      *ptr = l->buf.ptr;
      return LRP_OK;
    }
  auto nl = std::make_unique<StencilPlan::Layout>();
  nl->prec = prec;
  nl->pitch = pitch;
  nl->rows = rows;
  lrp_status s = oc_coef_fill(c, op, plan, prec, pitch, rows, nl->buf);
  if (s) return s;
  // published only once filled: other contexts (a server's) may use it at once
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_err(c, e, "k_oc_coef");
  *ptr = nl->buf.ptr;
  plan->layouts.push_back(std::move(nl));
  return LRP_OK;
}

static int oc_pitch(int mx) {
  for (int p : {64, 128, 256, 512})
    if (mx <= p) return p;
  return 0;
}

static Variant oc_variant(int prec, int pitch, int rpt, bool td = false) {
  if (td) return prec == 1 ? oc::variant_f32_td(pitch, rpt) : Variant{nullptr, 0};
  return prec == 0 ? oc::variant_f64(pitch, rpt) : oc::variant_f32(pitch, rpt);
}

// The variant for this grid and batch: the most CTAs in flight (then the
// larger row count); returns rows per CTA (0: none applies).
static int oc_choose(Ctx* c, int mx, int my, int nsys, int prec, int* cs_out, int* ncl_out,
                     bool td = false) {
  const int pitch = oc_pitch(mx);
  if (!pitch || my < 1) return 0;
  const int cands32[2] = {32, 16}, cands64[2] = {16, 8};
  const int* cands = prec == 0 ? cands64 : cands32;
  int best_rpt = 0, best_cs = 0, best_ncl = 0;
  long best = -1;
  for (int k = 0; k < 2; ++k) {
    const int rpt = cands[k];
    const int cs = (my + rpt - 1) / rpt;
    if (cs > oc::MAXCS) continue;
    if (c->p_krylov_cluster > 0 && cs != c->p_krylov_cluster) continue;
    const Variant v = oc_variant(prec, pitch, rpt, td);
    if (!v.fn || v.smem > 227 * 1024) continue;
    if (cudaFuncSetAttribute(v.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ||
        cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(pitch);
    cfg.gridDim = dim3(cs);
    cfg.dynamicSmemBytes = v.smem;
    int maxc = 0;
    if (cudaOccupancyMaxActiveClusters(&maxc, v.fn, &cfg) != cudaSuccess || maxc < 1) {
      cudaGetLastError();
      continue;
    }
    const int ncl = std::min(nsys, maxc);
    const long ctas = (long)ncl * cs;
    if (ctas > best) { best = ctas; best_rpt = rpt; best_cs = cs; best_ncl = ncl; }
  }
  *cs_out = best_cs;
  *ncl_out = best_ncl;
  return best_rpt;
}

bool stencil_onchip_fits(Ctx* c, const Operator* op, int prec, int nsys) {
  if (!op->symmetric || c->p_krylov_onchip == 2) return false;
  // time-dependent operators: FP32 solves
  const bool td = op->kind == 3;
  if (td && prec != 1) return false;
  int cs = 0, ncl = 0;
  return oc_choose(c, op->mx, op->my, std::max(nsys, 1), prec, &cs, &ncl, td) > 0;
}

bool stencil_onchip_applies(Ctx* c, const Operator* op, int prec, int nsys) {
  // the kernel runs backward-Euler steps
  if (op->stepper != 0) return false;
  return stencil_onchip_fits(c, op, prec, nsys);
}

lrp_status stencil_propagate_onchip(Ctx* c, Operator* op, StencilPlan* plan, int M, int nsys,
                                    int prec, const KryArgs& base) {
  int cs = 0, ncl = 0;
  const bool td = op->kind == 3;
  const int rpt = oc_choose(c, op->mx, op->my, nsys, prec, &cs, &ncl, td);
  if (!rpt) return set_err(c, LRP_EINVAL, "on-chip CG: no launch shape for this grid");
  const int pitch = oc_pitch(op->mx);
  const int rows = cs * rpt;
  const Variant v = oc_variant(prec, pitch, rpt, td);
  const size_t es = prec == 0 ? 8 : 4;
  const size_t tot = (size_t)(rows + 2) * pitch;
  void* cfp = nullptr;
  lrp_status s;
  if ((s = plan_layout(c, op, plan, prec, pitch, rows, &cfp))) return s;
  c->oc_last[0] = rpt;
  c->oc_last[1] = cs;
  c->oc_last[2] = ncl;
  oc::Args oa;
  oa.k = base;
  oa.cf = cfp;
  oa.scl = static_cast<char*>(cfp) + 2 * tot * es;
  oa.rows = rows;
  oa.cf_step = (long)(5 * tot / 2);           // pairs from one row of the time grid to the next
  oa.scl_step = (long)(5 * tot);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(pitch);
  cfg.gridDim = dim3(ncl * cs);
  cfg.dynamicSmemBytes = v.smem;
  cfg.stream = c->stream;
  const char* fam = prec == 0 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  void* args[1] = {&oa};
  cudaError_t e = cudaLaunchKernelExC(&cfg, v.fn, args);
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_cg_onchip launch");
  return LRP_OK;
}

}  // namespace lrp
