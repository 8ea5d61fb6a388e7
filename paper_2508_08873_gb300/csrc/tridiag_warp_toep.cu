// Instantiation of the constant-coefficient one-warp cluster tridiagonal
// propagator (tri_warp.cuh), and the host side of its coefficients.
#define LRP_TRI_WARP_KERNEL
#include "tri_warp.cuh"

#include <cmath>

namespace lrp {

lrp_status tri_launch_warp_toep(Ctx* c, ClPlan* pl, ClKArgs& a) {
  if (!a.tz.on || a.src.Q > 0) return set_err(c, LRP_EINVAL, "constant-coefficient kernel: no data or a source");
  switch (pl->m) {
    case 16: return launch_cl_wt<16>(c, pl, a);
    case 15: return launch_cl_wt<15>(c, pl, a);
    case 14: return launch_cl_wt<14>(c, pl, a);
    case 13: return launch_cl_wt<13>(c, pl, a);
    case 12: return launch_cl_wt<12>(c, pl, a);
    case 11: return launch_cl_wt<11>(c, pl, a);
    case 10: return launch_cl_wt<10>(c, pl, a);
    case 9: return launch_cl_wt<9>(c, pl, a);
    case 8: return launch_cl_wt<8>(c, pl, a);
    default: return set_err(c, LRP_EINVAL, "warp cluster chunk length out of range");
  }
}

template <typename T>
lrp_status tri_launch_warp_block_toep(Ctx* c, ClPlan* pl, ClKArgs& a) {
  if (!a.tz.on || a.src.Q > 0) return set_err(c, LRP_EINVAL, "constant-coefficient kernel: no data or a source");
  switch (pl->m) {
    case 16: return launch_blk_wt<T, 16>(c, pl, a);
    case 15: return launch_blk_wt<T, 15>(c, pl, a);
    case 14: return launch_blk_wt<T, 14>(c, pl, a);
    case 13: return launch_blk_wt<T, 13>(c, pl, a);
    case 12: return launch_blk_wt<T, 12>(c, pl, a);
    case 11: return launch_blk_wt<T, 11>(c, pl, a);
    case 10: return launch_blk_wt<T, 10>(c, pl, a);
    case 9: return launch_blk_wt<T, 9>(c, pl, a);
    case 8: return launch_blk_wt<T, 8>(c, pl, a);
    default: return set_err(c, LRP_EINVAL, "warp chunk length out of range");
  }
}
template lrp_status tri_launch_warp_block_toep<double>(Ctx* c, ClPlan* pl, ClKArgs& a);
template lrp_status tri_launch_warp_block_toep<float>(Ctx* c, ClPlan* pl, ClKArgs& a);

void tri_toeplitz_coef(const Operator* op, double dt, int adjoint, int M, int m, ToepCoef* tz,
                       int prec) {
  *tz = ToepCoef{};
  if (!op->toeplitz || m < 3) return;
  const int n = op->n;
  if (n % m != 0 && (n + 1) % m != 0) return;
  const double a = dt * (adjoint ? op->tup : op->tlo);
  const double c = dt * (adjoint ? op->tlo : op->tup);
  const double d = 1.0 + dt * op->tdi;
  const double disc = d * d - 4.0 * a * c;
  if (!(d > 0.0) || !(disc > 0.0) || !std::isfinite(disc)) return;
  double dinf = 0.5 * (d + std::sqrt(disc));
  if (!(dinf > 0.0)) return;
  double l = a / dinf, u = c / dinf;
  if (prec != 0 && a * c > 0.0) {
    // FP32: l and u are rounded once for every row, so the sweeps apply
    // tridiag(dinf l, dinf (1 + l u), dinf u) with a bias of the order of the
    // FP32 rounding in every entry; the slowest-decaying modes, whose
    // eigenvalue d - 2 sqrt(a c) is the smallest, would accumulate it over
    // the steps.  The scale is set so that this smallest eigenvalue of the
    // swept matrix is the exact one.
    l = (double)(float)l;
    u = (double)(float)u;
    const double lu = l * u;
    const double lam = d - 2.0 * std::sqrt(a * c);
    const double lam_s = (1.0 - std::sqrt(lu)) * (1.0 - std::sqrt(lu));
    if (lam > 0.0 && lam_s > 0.0) dinf = lam / lam_s;
  }
  // the Sherman-Morrison denominator 1 + (d - dinf) phi_0 of a chunk
  double phi[32];
  const int mi = m - 1;
  for (int i = 0; i < mi; ++i) phi[i] = i == 0 ? 1.0 : 0.0;
  for (int i = 1; i < mi; ++i) phi[i] -= l * phi[i - 1];
  for (int i = mi - 2; i >= 0; --i) phi[i] -= u * phi[i + 1];
  const double den = 1.0 + (d - dinf) * phi[0] / dinf;
  if (!(std::fabs(den) > 1e-3)) return;
  // rescale period: dinf^P within 1e150 either way (1e15 in FP32)
  const double lg = std::fabs(std::log10(dinf));
  const double span = prec == 0 ? 150.0 : 15.0;
  const double Pd = lg > 0.0 ? std::floor(span / lg) : (double)(1 << 30);
  const int P = (int)std::max(1.0, std::min(Pd, (double)(1 << 30)));
  tz->on = 1;
  tz->P = P;
  tz->a = a;
  tz->d = d;
  tz->c = c;
  tz->dinf = dinf;
  tz->idinf = 1.0 / dinf;
  tz->l = l;
  tz->u = u;
  tz->rho = P < (1 << 30) ? std::pow(dinf, -(double)P) : 1.0;
  const long e = M >= 1 ? (long)M - (long)P * ((M - 1) / P) : 0;
  tz->fin = std::pow(dinf, -(double)e);
}

}  // namespace lrp
