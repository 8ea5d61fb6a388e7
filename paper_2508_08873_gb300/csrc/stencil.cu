// Batched backward-Euler propagator for 5-point stencil operators (2D).
#include "internal.h"

namespace lrp {

lrp_status stencil_propagate(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys,
                             int prec, const PropIn& in, const PropOut& out, const PropSrc& src) {
  return set_err(c, LRP_EINVAL, "5-point stencil operators are not supported yet");
}

}  // namespace lrp

using namespace lrp;
struct lrp_operator : public Operator {};

extern "C" lrp_status lrp_operator_stencil5(lrp_ctx* cc, int mx, int my, const double* C,
                                            const double* W, const double* E, const double* S,
                                            const double* N, lrp_operator** out) {
  Ctx* c = reinterpret_cast<Ctx*>(cc);
  if (!c || !out || !C || !W || !E || !S || !N || mx < 1 || my < 1) return LRP_EINVAL;
  cudaSetDevice(c->device);
  auto* op = new lrp_operator();
  op->ctx = c;
  ctx_retain(c);
  op->kind = 1;
  op->mx = mx;
  op->my = my;
  op->n = mx * my;
  const double* src[5] = {C, W, E, S, N};
  for (int k = 0; k < 5; ++k) {
    lrp_status s = dev_alloc(c, op->a64[k], sizeof(double) * op->n);
    if (!s) s = dev_alloc(c, op->a32[k], sizeof(float) * op->n);
    if (s) { delete op; return s; }
    cudaError_t e = cudaMemcpyAsync(op->a64[k].ptr, src[k], sizeof(double) * op->n,
                                    cudaMemcpyDefault, c->stream);
    if (e) { delete op; return cuda_err(c, e, "stencil upload"); }
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) { delete op; return cuda_err(c, e, "stencil upload"); }
  *out = op;
  return LRP_OK;
}
