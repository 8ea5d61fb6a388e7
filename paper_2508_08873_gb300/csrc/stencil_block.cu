// Launch code of the block CG propagator for symmetric 5-point operators
// (kernel in stencil_block.cuh) and its FP32 instantiations: the systems of a
// propagation are taken S at a time (S = 4), every block on one thread-block
// cluster with its block vectors in a global-memory workspace (five block
// vectors per cluster in flight; the clusters in flight are chosen so that
// the workspaces stay within 96 MB, L2-resident, unless the context asks for
// a count).
#include <algorithm>

#include "stencil_block.cuh"

namespace lrp {

namespace bk {

constexpr int BS = 4;    // systems per block
constexpr int RBF = 32;  // rows per CTA

Variant variant_f32(int pitch) {
  switch (pitch) {
    case 64: return make_variant<float, BS, 64, RBF>();
    case 128: return make_variant<float, BS, 128, RBF>();
    case 256: return make_variant<float, BS, 256, RBF>();
    case 512: return make_variant<float, BS, 512, RBF>();
    default: return Variant{nullptr, 0, 0, 0, 0, 0};
  }
}

}  // namespace bk

static int bk_pitch(int mx, int prec) {
  for (int p : {64, 128, 256, 512})
    if (mx <= p) return (prec == 0 && p > 256) ? 0 : p;   // FP64: up to 256 columns
  return 0;
}

static bk::Variant bk_variant(int prec, int mx) {
  const int pitch = bk_pitch(mx, prec);
  if (!pitch) return bk::Variant{nullptr, 0, 0, 0, 0, 0};
  return prec == 0 ? bk::variant_f64(pitch) : bk::variant_f32(pitch);
}

bool stencil_block_applies(Ctx* c, const Operator* op, int prec, int nsys, int M, int Q) {
  if (c->p_krylov_block != bk::BS || !op->symmetric || M < 1 || Q > 0 || nsys < 2) return false;
  const bk::Variant v = bk_variant(prec, op->mx);
  if (!v.fn || op->my < 1) return false;
  return (op->my + v.rb - 1) / v.rb <= bk::MAXCS;
}

lrp_status stencil_propagate_block(Ctx* c, Operator* op, StencilPlan* plan, int M, int nsys,
                                   int prec, const KryArgs& base) {
  const bk::Variant v = bk_variant(prec, op->mx);
  if (!v.fn) return set_err(c, LRP_EINVAL, "block CG: no variant for this grid");
  const int cs = (op->my + v.rb - 1) / v.rb;
  if (cs > bk::MAXCS) return set_err(c, LRP_EINVAL, "block CG: grid has too many rows");
  const int rows = cs * v.rb;
  void* cfp = nullptr;
  lrp_status s;
  if ((s = plan_layout(c, op, plan, prec, v.pitch, rows, &cfp))) return s;
  const size_t es = prec == 0 ? 8 : 4;
  const size_t tot = (size_t)(rows + 2) * v.pitch;
  cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (!e) e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
  if (e) return cuda_err(c, e, "block CG attributes");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(v.threads);   // two grid columns per thread
  cfg.gridDim = dim3(cs);
  cfg.dynamicSmemBytes = v.smem;
  cfg.stream = c->stream;
  int maxc = 0;
  e = cudaOccupancyMaxActiveClusters(&maxc, v.fn, &cfg);
  if (e || maxc < 1) {
    cudaGetLastError();
    return set_err(c, LRP_EINVAL, "block CG: no cluster of this size fits");
  }
  // five block vectors (X^, R twice, P twice) of rows + 2 PADR rows per cluster;
  // clusters in flight: as many as keep the workspaces within 96 MB
  // (L2-resident), or the count the context asks for, at most all that fit
  const size_t slot_elems = 5 * (size_t)(rows + 2 * bk::PADR) * v.S * v.pitch;
  const size_t slot_bytes = slot_elems * es;
  const int nblk = (nsys + v.S - 1) / v.S;
  int ncl = c->p_krylov_block_clusters > 0
      ? c->p_krylov_block_clusters
      : (int)std::max<size_t>(1, ((size_t)96 << 20) / slot_bytes);
  ncl = std::max(1, std::min(std::min(ncl, maxc), nblk));
  const size_t need = (size_t)ncl * slot_bytes;
  if (c->bws.bytes < need)
    if ((s = dev_alloc(c, c->bws, need))) return s;
  // the pad rows of every block vector must read as 0
  e = cudaMemsetAsync(c->bws.ptr, 0, need, c->stream);
  if (e) return cuda_err(c, e, "block CG workspace");
  c->bk_last[0] = v.S;
  c->bk_last[1] = cs;
  c->bk_last[2] = ncl;
  bk::Args ba;
  ba.k = base;
  ba.cf = cfp;
  ba.scl = static_cast<char*>(cfp) + 2 * tot * es;
  ba.rows = rows;
  ba.ws = c->bws.ptr;
  ba.slot_elems = slot_elems;
  ba.thr = prec == 0 ? 1e-12 : 1e-6;
  cfg.gridDim = dim3(ncl * cs);
  const char* fam = prec == 0 ? "propagate_f64" : "propagate_f32";
  cudaEvent_t ev = nullptr;
  timer_begin(c, fam, &ev);
  void* args[1] = {&ba};
  e = cudaLaunchKernelExC(&cfg, v.fn, args);
  timer_end(c, fam, ev);
  if (e) return cuda_err(c, e, "k_bcg launch");
  return LRP_OK;
}

}  // namespace lrp
