/*
 * FP64 CPU oracle: numeric primitives of "A Parareal Algorithm with Low-Rank
 * Coarse Solvers" (Gander, Ohlberger, Rave; arXiv 2508.08873).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA
 * library is checked against.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header or constant table
 * with the CUDA path; the two are written independently from the paper and from
 * the published definitions cited below.
 *
 * Contents (every routine is FP64 and deliberately unblocked and unfused):
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11) and a Box-Muller
 *     (cosine branch) normal deviate.  The paper draws Gaussian sketch vectors
 *     (Sec. 2.1, rSVD step 1); the generator itself is unspecified there.
 *   - Tridiagonal Gaussian elimination without pivoting (Thomas algorithm),
 *     and the backward-Euler fine propagator F_n, its linear part F_n' and the
 *     adjoint F_n'^* built on it (Sec. 4: backward Euler with equidistant steps;
 *     Eq. (F_n_affine) for the affine split; Sec. 2.1 step 3 for the adjoint).
 *   - Banded LU without pivoting for 5-point stencils and the same propagators.
 *   - Modified Gram-Schmidt with one re-orthogonalisation pass and deflation
 *     (Sec. 2.1, rSVD steps 2 and 4).
 *   - One-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992) for the
 *     small matrix of rSVD step 5.
 *
 * Parity of every routine here is pinned by the CPU test suite against closed
 * forms, library routines and invariants (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3.2).                           */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof(c));
}

/* Standard normal for (seed, stream, interval, column, row).
 * Counter = (row, column, interval, stream); key = (low, high) words of seed.
 * Uniforms: U1 = (k1 + 1) 2^-53 in (0,1], U2 = k2 2^-53 in [0,1), where k1 is
 * the top 53 bits of (w0:w1) and k2 the top 53 bits of (w2:w3).
 * Box-Muller cosine branch: z = sqrt(-2 ln U1) cos(2 pi U2). */
double orc_gauss(uint64_t seed, uint32_t stream, uint32_t interval, uint32_t column,
                 uint32_t row) {
  uint32_t ctr[4] = {row, column, interval, stream};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  uint64_t k1 = (((uint64_t)w[0] << 32) | (uint64_t)w[1]) >> 11;
  uint64_t k2 = (((uint64_t)w[2] << 32) | (uint64_t)w[3]) >> 11;
  double u1 = ((double)k1 + 1.0) * 0x1.0p-53;
  double u2 = (double)k2 * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Column-major n x ncol block of normals for one interval (rSVD step 1). */
void orc_gauss_block(uint64_t seed, uint32_t stream, uint32_t interval, int n, int ncol,
                     double* out) {
  for (int j = 0; j < ncol; ++j)
    for (int i = 0; i < n; ++i)
      out[(size_t)j * n + i] = orc_gauss(seed, stream, interval, (uint32_t)j, (uint32_t)i);
}

/* Raw Philox words for tests (n counters with row = 0..n-1). */
void orc_philox_rows(uint64_t seed, uint32_t stream, uint32_t interval, uint32_t column, int n,
                     uint32_t* out /* n x 4 */) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (int i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, column, interval, stream};
    orc_philox4x32_10(ctr, key, out + 4 * (size_t)i);
  }
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal systems.                                                      */
/* Row i of the matrix: lo[i]*x[i-1] + di[i]*x[i] + up[i]*x[i+1] (lo[0] and  */
/* up[n-1] are ignored).                                                     */
/* ------------------------------------------------------------------------ */

/* Thomas algorithm: Gaussian elimination without pivoting.  Returns 0, or -1
 * if a pivot vanishes (the matrices used here are strictly diagonally
 * dominant, for which no pivoting is needed). work has length n. */
int orc_thomas(int n, const double* lo, const double* di, const double* up, const double* d,
               double* x, double* work) {
  double* cp = work;
  double piv = di[0];
  if (piv == 0.0) return -1;
  cp[0] = (n > 1 ? up[0] : 0.0) / piv;
  x[0] = d[0] / piv;
  for (int i = 1; i < n; ++i) {
    piv = di[i] - lo[i] * cp[i - 1];
    if (piv == 0.0) return -1;
    cp[i] = (i < n - 1 ? up[i] : 0.0) / piv;
    x[i] = (d[i] - lo[i] * x[i - 1]) / piv;
  }
  for (int i = n - 2; i >= 0; --i) x[i] -= cp[i] * x[i + 1];
  return 0;
}

/* Backward-Euler propagation over one coarse interval (Sec. 4; fine solver F_n).
 *   (I + dt*A) x_{j+1} = x_j + dt * sum_q cvals[j*Q+q] * g[q*n + .],  j = 0..M-1
 * A is the tridiagonal semi-discretisation with u_t = -A u + f.  The source is
 * separable, f(t_{j+1}, x) = sum_q c_q(t_{j+1}) g_q(x), sampled at the end of
 * each step (fully implicit).  Q = 0 gives the linear part F_n'.
 * adjoint != 0 applies the Euclidean adjoint of F_n', i.e. M solves with
 * (I + dt*A)^T; for a time-invariant A the order of the factors is immaterial.
 * x (length n) is overwritten.  Returns 0 or -1 on a zero pivot. */
int orc_tridiag_propagate(int n, const double* lo, const double* di, const double* up,
                          double dt, int M, int adjoint, int Q, const double* g,
                          const double* cvals, double* x) {
  double* bl = (double*)malloc(sizeof(double) * (size_t)n * 5);
  if (!bl) return -2;
  double* bd = bl + n;
  double* bu = bd + n;
  double* rhs = bu + n;
  double* work = rhs + n;
  for (int i = 0; i < n; ++i) {
    /* B = I + dt*A; the transpose swaps the roles of the off-diagonals. */
    double a_lo = adjoint ? (i > 0 ? up[i - 1] : 0.0) : lo[i];
    double a_up = adjoint ? (i < n - 1 ? lo[i + 1] : 0.0) : up[i];
    bl[i] = dt * a_lo;
    bd[i] = 1.0 + dt * di[i];
    bu[i] = dt * a_up;
  }
  int rc = 0;
  for (int j = 0; j < M && rc == 0; ++j) {
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int q = 0; q < Q; ++q) s += cvals[(size_t)j * Q + q] * g[(size_t)q * n + i];
      rhs[i] = x[i] + dt * s;
    }
    rc = orc_thomas(n, bl, bd, bu, rhs, x, work);
  }
  free(bl);
  return rc;
}

/* Many independent vectors (columns of X, n x nvec column-major), each with its
 * own source-coefficient block (cvals + v*cstride; cstride = 0 shares one). */
int orc_tridiag_propagate_many(int n, const double* lo, const double* di, const double* up,
                               double dt, int M, int adjoint, int Q, const double* g,
                               const double* cvals, long cstride, int nvec, double* X) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int v = 0; v < nvec; ++v) {
    int rc = orc_tridiag_propagate(n, lo, di, up, dt, M, adjoint, Q, g,
                                   cvals ? cvals + (size_t)v * cstride : NULL,
                                   X + (size_t)v * n);
    if (rc) bad = 1;
  }
  return bad ? -1 : 0;
}

/* Backward-Euler propagation with a time-dependent tridiagonal operator
 * (Experiment 2 of Sec. 4): fine step J (0-based over the whole time grid)
 * uses A_J, whose coefficients are rows J of LO, DI, UP (each of size nJ x n,
 * row J holding A(t_{J+1})).  The interval's first step is j0:
 *   (I + dt*A_{j0+j}) x_{j+1} = x_j + dt * sum_q cvals[j*Q+q] g[q*n + .],
 * j = 0..M-1, so F' = B_{j0+M-1}^{-1} ... B_{j0}^{-1} with B_J = I + dt A_J.
 * adjoint != 0 applies F'^* = B_{j0}^{-T} ... B_{j0+M-1}^{-T}: the
 * transposed solves in the reversed order of the steps (no source).
 * Returns 0, -1 on a zero pivot, -3 when the steps run past row nJ - 1. */
int orc_tridiag_td_propagate(int n, int nJ, const double* LO, const double* DI, const double* UP,
                             int j0, double dt, int M, int adjoint, int Q, const double* g,
                             const double* cvals, double* x) {
  if (j0 < 0 || j0 + M > nJ) return -3;
  double* bl = (double*)malloc(sizeof(double) * (size_t)n * 5);
  if (!bl) return -2;
  double* bd = bl + n;
  double* bu = bd + n;
  double* rhs = bu + n;
  double* work = rhs + n;
  int rc = 0;
  for (int t = 0; t < M && rc == 0; ++t) {
    const int J = adjoint ? j0 + M - 1 - t : j0 + t;
    const double* lo = LO + (size_t)J * n;
    const double* di = DI + (size_t)J * n;
    const double* up = UP + (size_t)J * n;
    for (int i = 0; i < n; ++i) {
      double a_lo = adjoint ? (i > 0 ? up[i - 1] : 0.0) : lo[i];
      double a_up = adjoint ? (i < n - 1 ? lo[i + 1] : 0.0) : up[i];
      bl[i] = dt * a_lo;
      bd[i] = 1.0 + dt * di[i];
      bu[i] = dt * a_up;
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int q = 0; q < Q; ++q) s += cvals[(size_t)t * Q + q] * g[(size_t)q * n + i];
      rhs[i] = x[i] + dt * s;
    }
    rc = orc_thomas(n, bl, bd, bu, rhs, x, work);
  }
  free(bl);
  return rc;
}

/* orc_tridiag_td_propagate for nvec vectors, vector v starting at step
 * j0s[v] (its interval times M); independent vectors run in parallel. */
int orc_tridiag_td_propagate_many(int n, int nJ, const double* LO, const double* DI,
                                  const double* UP, const int* j0s, double dt, int M, int adjoint,
                                  int Q, const double* g, const double* cvals, long cstride,
                                  int nvec, double* X) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int v = 0; v < nvec; ++v) {
    int rc = orc_tridiag_td_propagate(n, nJ, LO, DI, UP, j0s[v], dt, M, adjoint, Q, g,
                                      cvals ? cvals + (size_t)v * cstride : NULL,
                                      X + (size_t)v * n);
    if (rc == -3) bad |= 2;
    else if (rc) bad |= 1;
  }
  return (bad & 2) ? -3 : (bad ? -1 : 0);
}

/* ------------------------------------------------------------------------ */
/* 5-point stencils on an mx x my grid of interior nodes, node p = iy*mx+ix. */
/* A x at p = C[p] x_p + W[p] x_{p-1} + E[p] x_{p+1} + S[p] x_{p-mx}          */
/*            + N[p] x_{p+mx}; neighbours outside the grid are absent        */
/* (homogeneous Dirichlet).  B = I + dt*A is banded with half-bandwidth mx.  */
/* Band storage: lu[p*(2*mx+1) + (q - p + mx)] holds B[p][q].                */
/* ------------------------------------------------------------------------ */

static double* band_assemble(int mx, int my, const double* C, const double* W, const double* E,
                             const double* S, const double* N, double dt, int adjoint) {
  int n = mx * my, w = 2 * mx + 1;
  double* b = (double*)calloc((size_t)n * w, sizeof(double));
  if (!b) return NULL;
#define BAND(p, q) b[(size_t)(p) * w + ((q) - (p) + mx)]
  for (int p = 0; p < n; ++p) {
    int ix = p % mx, iy = p / mx;
    /* row p of A: (p,p)=C, (p,p-1)=W, (p,p+1)=E, (p,p-mx)=S, (p,p+mx)=N */
    BAND(p, p) += 1.0 + dt * C[p];
    if (!adjoint) {
      if (ix > 0) BAND(p, p - 1) += dt * W[p];
      if (ix < mx - 1) BAND(p, p + 1) += dt * E[p];
      if (iy > 0) BAND(p, p - mx) += dt * S[p];
      if (iy < my - 1) BAND(p, p + mx) += dt * N[p];
    } else {
      /* transpose: entry (q,p) of A goes to (p,q) */
      if (ix > 0) BAND(p - 1, p) += dt * W[p];
      if (ix < mx - 1) BAND(p + 1, p) += dt * E[p];
      if (iy > 0) BAND(p - mx, p) += dt * S[p];
      if (iy < my - 1) BAND(p + mx, p) += dt * N[p];
    }
  }
#undef BAND
  return b;
}

/* In-place banded LU without pivoting (Doolittle): L unit lower, U upper,
 * both stored in the band.  Returns 0, or -1 on a zero pivot. */
int orc_band_lu(int n, int bw, double* b) {
  int w = 2 * bw + 1;
#define BB(p, q) b[(size_t)(p) * w + ((q) - (p) + bw)]
  for (int k = 0; k < n; ++k) {
    double piv = BB(k, k);
    if (piv == 0.0) return -1;
    int iend = k + bw < n - 1 ? k + bw : n - 1;
    for (int i = k + 1; i <= iend; ++i) {
      double l = BB(i, k) / piv;
      BB(i, k) = l;
      if (l != 0.0)
        for (int j = k + 1; j <= iend; ++j) BB(i, j) -= l * BB(k, j);
    }
  }
#undef BB
  return 0;
}

/* Solve B x = d (trans = 0) or B^T x = d (trans = 1) with the factors of
 * orc_band_lu; x holds d on entry. */
void orc_band_solve(int n, int bw, const double* b, int trans, double* x) {
  int w = 2 * bw + 1;
#define BB(p, q) b[(size_t)(p) * w + ((q) - (p) + bw)]
  if (!trans) {
    for (int i = 0; i < n; ++i) {            /* L y = d */
      int j0 = i - bw > 0 ? i - bw : 0;
      double s = x[i];
      for (int j = j0; j < i; ++j) s -= BB(i, j) * x[j];
      x[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {       /* U x = y */
      int j1 = i + bw < n - 1 ? i + bw : n - 1;
      double s = x[i];
      for (int j = i + 1; j <= j1; ++j) s -= BB(i, j) * x[j];
      x[i] = s / BB(i, i);
    }
  } else {
    for (int i = 0; i < n; ++i) {            /* U^T y = d */
      int j0 = i - bw > 0 ? i - bw : 0;
      double s = x[i];
      for (int j = j0; j < i; ++j) s -= BB(j, i) * x[j];
      x[i] = s / BB(i, i);
    }
    for (int i = n - 1; i >= 0; --i) {       /* L^T x = y */
      int j1 = i + bw < n - 1 ? i + bw : n - 1;
      double s = x[i];
      for (int j = i + 1; j <= j1; ++j) s -= BB(j, i) * x[j];
      x[i] = s;
    }
  }
#undef BB
}

/* Backward-Euler propagation with a 5-point stencil operator: B = I + dt*A is
 * factored once (A is time-invariant), then M solves per vector; the source is
 * handled as in orc_tridiag_propagate.  adjoint solves with B^T. */
int orc_stencil_propagate_many(int mx, int my, const double* C, const double* W,
                               const double* E, const double* S, const double* N, double dt,
                               int M, int adjoint, int Q, const double* g, const double* cvals,
                               long cstride, int nvec, double* X) {
  int n = mx * my;
  double* b = band_assemble(mx, my, C, W, E, S, N, dt, 0);
  if (!b) return -2;
  if (orc_band_lu(n, mx, b)) { free(b); return -1; }
#pragma omp parallel for schedule(dynamic, 1)
  for (int v = 0; v < nvec; ++v) {
    double* x = X + (size_t)v * n;
    const double* cv = cvals ? cvals + (size_t)v * cstride : NULL;
    for (int j = 0; j < M; ++j) {
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int q = 0; q < Q; ++q) s += cv[(size_t)j * Q + q] * g[(size_t)q * n + i];
        x[i] += dt * s;
      }
      orc_band_solve(n, mx, b, adjoint, x);
    }
  }
  free(b);
  return 0;
}

/* Dense B = I + dt*A of a stencil operator, for tests on tiny grids. */
int orc_stencil_dense(int mx, int my, const double* C, const double* W, const double* E,
                      const double* S, const double* N, double dt, double* out /* n x n */) {
  int n = mx * my;
  double* b = band_assemble(mx, my, C, W, E, S, N, dt, 0);
  if (!b) return -2;
  int w = 2 * mx + 1;
  memset(out, 0, sizeof(double) * (size_t)n * n);
  for (int p = 0; p < n; ++p)
    for (int q = p - mx; q <= p + mx; ++q)
      if (q >= 0 && q < n) out[(size_t)p * n + q] = b[(size_t)p * w + (q - p + mx)];
  free(b);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Modified Gram-Schmidt, applied twice ("twice is enough"), with deflation. */
/* Column j of Y (n x k, column-major) is orthogonalised against the kept    */
/* columns; it is dropped when its norm after both passes is below           */
/* tau * (its norm before).  Kept columns go to Q in order; keep[j] = 1/0.   */
/* Returns the number r of kept columns.                                     */
/* ------------------------------------------------------------------------ */
int orc_mgs2(int n, int k, const double* Y, double tau, double* Q, int* keep) {
  int r = 0;
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  if (!v) return -2;
  for (int j = 0; j < k; ++j) {
    const double* y = Y + (size_t)j * n;
    double nrm0 = 0.0;
    for (int i = 0; i < n; ++i) { v[i] = y[i]; nrm0 += y[i] * y[i]; }
    nrm0 = sqrt(nrm0);
    for (int pass = 0; pass < 2; ++pass) {
      for (int c = 0; c < r; ++c) {          /* one basis vector at a time (MGS) */
        const double* q = Q + (size_t)c * n;
        double h = 0.0;
        for (int i = 0; i < n; ++i) h += q[i] * v[i];
        for (int i = 0; i < n; ++i) v[i] -= h * q[i];
      }
    }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm += v[i] * v[i];
    nrm = sqrt(nrm);
    if (nrm0 > 0.0 && nrm > tau * nrm0) {
      double* q = Q + (size_t)r * n;
      for (int i = 0; i < n; ++i) q[i] = v[i] / nrm;
      ++r;
      if (keep) keep[j] = 1;
    } else if (keep) {
      keep[j] = 0;
    }
  }
  free(v);
  return r;
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Hestenes): A (m x k, column-major, m >= k) =        */
/* U diag(s) V^T.  Columns of a working copy are rotated pairwise until all  */
/* pairs are numerically orthogonal (|a_p.a_q| <= eps sqrt(|a_p|^2 |a_q|^2)), */
/* then s = column norms, U = normalised columns, V = accumulated rotations. */
/* Output sorted by descending s.  Zero columns get s = 0 and an arbitrary   */
/* U column of zeros.  Returns the number of sweeps, or -1 if not converged. */
/* ------------------------------------------------------------------------ */
int orc_jacobi_svd(int m, int k, const double* A, double* U, double* s, double* V) {
  double* G = (double*)malloc(sizeof(double) * (size_t)m * k);
  double* Vw = (double*)malloc(sizeof(double) * (size_t)k * k);
  if (!G || !Vw) { free(G); free(Vw); return -2; }
  memcpy(G, A, sizeof(double) * (size_t)m * k);
  for (int i = 0; i < k * k; ++i) Vw[i] = 0.0;
  for (int i = 0; i < k; ++i) Vw[(size_t)i * k + i] = 1.0;
  const double eps = 2.220446049250313e-16;
  int sweep, converged = 0;
  for (sweep = 1; sweep <= 60 && !converged; ++sweep) {
    converged = 1;
    for (int p = 0; p < k - 1; ++p) {
      for (int q = p + 1; q < k; ++q) {
        double* ap = G + (size_t)p * m;
        double* aq = G + (size_t)q * m;
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < m; ++i) {
          alpha += ap[i] * ap[i];
          beta += aq[i] * aq[i];
          gamma += ap[i] * aq[i];
        }
        if (fabs(gamma) <= eps * sqrt(alpha * beta) || gamma == 0.0) continue;
        converged = 0;
        /* rotation that zeroes the (p,q) entry of the 2x2 Gram matrix */
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double sn = c * t;
        for (int i = 0; i < m; ++i) {
          double x = ap[i], y = aq[i];
          ap[i] = c * x - sn * y;
          aq[i] = sn * x + c * y;
        }
        double* vp = Vw + (size_t)p * k;
        double* vq = Vw + (size_t)q * k;
        for (int i = 0; i < k; ++i) {
          double x = vp[i], y = vq[i];
          vp[i] = c * x - sn * y;
          vq[i] = sn * x + c * y;
        }
      }
    }
  }
  /* singular values = column norms; sort descending (selection sort) */
  int* ord = (int*)malloc(sizeof(int) * (size_t)k);
  double* nr = (double*)malloc(sizeof(double) * (size_t)k);
  for (int j = 0; j < k; ++j) {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += G[(size_t)j * m + i] * G[(size_t)j * m + i];
    nr[j] = sqrt(t);
    ord[j] = j;
  }
  for (int a = 0; a < k; ++a)
    for (int b = a + 1; b < k; ++b)
      if (nr[ord[b]] > nr[ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
  for (int a = 0; a < k; ++a) {
    int j = ord[a];
    s[a] = nr[j];
    for (int i = 0; i < m; ++i)
      U[(size_t)a * m + i] = nr[j] > 0.0 ? G[(size_t)j * m + i] / nr[j] : 0.0;
    for (int i = 0; i < k; ++i) V[(size_t)a * k + i] = Vw[(size_t)j * k + i];
  }
  free(ord); free(nr); free(G); free(Vw);
  return converged ? sweep - 1 : -1;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops over independent vectors (timing on 1 core
 * or on all host cores); n <= 0 restores the default. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}
