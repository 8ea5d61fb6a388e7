// Entries of B = I + dt*A (or of its transpose) of a tridiagonal operator,
// with padding rows r >= n acting as identity rows.
#pragma once

namespace lrp {

__device__ __forceinline__ double b_lo(const double* lo, const double* up, int n, double dt,
                                       int adj, int r) {
  if (r <= 0 || r >= n) return 0.0;
  return dt * (adj ? up[r - 1] : lo[r]);
}
__device__ __forceinline__ double b_di(const double* di, int n, double dt, int r) {
  return r < n ? 1.0 + dt * di[r] : 1.0;
}
__device__ __forceinline__ double b_up(const double* lo, const double* up, int n, double dt,
                                       int adj, int r) {
  if (r >= n - 1) return 0.0;
  return dt * (adj ? lo[r + 1] : up[r]);
}

}  // namespace lrp
