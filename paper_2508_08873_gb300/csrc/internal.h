// Internal host-side structures and kernel launchers of the library.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <memory>
#include <string>
#include <vector>

#include "../../include/lrp.h"

namespace lrp {

struct Ctx;

// Device allocation owned by a context (counted against its HBM budget).
struct DevBuf {
  Ctx* ctx = nullptr;
  void* ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf();
  void release();
  template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

// Events recorded around the launches of one kernel family.
struct KernelTimer {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs;
  int launches = 0;
  double total_ms = 0.0;
};

struct Ctx {
  int device = 0;
  size_t budget = 0;
  std::atomic<size_t> in_use{0};
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string last_error;
  bool timing = false;
  std::map<std::string, KernelTimer> timers;
  int num_sms = 0;
  long launches = 0;       // kernels launched by this context (all families)
  // Tunable launch parameters (0 = automatic choice); see lrp_set_param.
  int p_sweep_rows = 0;      // rows per CTA slice of the coarse sweep (0: 1024)
  int p_tri_cluster = 0;     // CTAs per tridiagonal system for small batches (1..8)
  int p_tri_warp = 0;        // one-warp cluster kernel for FP64 small batches (0 auto, 1 off)
  int p_queue_cluster = 0;   // CTAs per cluster of the batched 2D work queue (1..16)
  int p_krylov_cluster = 0;  // CTAs per cluster of the 2D propagator (1..16)
  int p_krylov_onchip = 0;   // on-chip CG for symmetric 2D operators: 0 auto, 2 never
  int oc_last[3] = {0, 0, 0};  // last on-chip CG launch: rows per thread, CTAs per cluster, clusters
  int p_krylov_block = 0;    // block CG over this many systems for symmetric 2D operators (0 off, 4)
  int p_krylov_block_clusters = 0;  // clusters in flight of the block CG (0: workspaces within 96 MB)
  int p_krylov_refine = 0;   // FP64 2D steps by iterative refinement: 0 auto, 1 where it applies, 2 never
  int p_krylov_refine_digits = 0;   // relative tolerance 10^-digits of its FP32 solves (0: 1e-3)
  int p_krylov_stage = 0;    // FP32 global-memory Krylov kernel: 1 stages stencil inputs by bulk copies, 0 not
  int p_tri_refine = 0;      // FP64 1D steps from FP32 solves with pair residuals: 1 on, 0 off
  int p_tri_refine_rounds = 2;   // correction rounds per step of those steps (1..3)
  int p_tri_refine_cluster = 0;  // those steps: 0 one CTA per system, 1 a cluster of one-warp CTAs
  // Scratch of 2D propagations, per context (one host thread and one stream
  // each, so that a server's contexts and the caller's never share it): the
  // Krylov workspace and status, the block CG workspace, the refinement's
  // workspace and inner-solve status.  Released before the pool is drained.
  DevBuf kws, kstat, bws, irws, irstat, triws;
  int bk_last[3] = {0, 0, 0};  // last block CG launch: systems per block, CTAs per cluster, clusters
  int p_orth_cluster = 0;    // CTAs per cluster of the CGS2 kernel (0 auto, -1 one-CTA kernel)
  int p_tri_spt = 0;         // systems per thread of the cluster tridiagonal kernel (1, 2)
  int p_tri_chunk = 0;       // rows per chunk of the cluster tridiagonal kernel (8, 16)
  int p_orth_tc = 1;         // tensor-core CholeskyQR2 and lift for FP32 sketches (1 on, 0 off)
  int p_tri_wchunk = 0;      // rows per chunk of the one-warp cluster kernel (0 auto, 8..16)
  int p_tri_wsplit = 1;      // backward rows of the one-warp kernel after the barrier wait (0 none, 1 a third)
  int p_tri_wblock = 0;      // one-CTA-per-system warp kernel: 0 auto (FP32), 1 always, 2 never
  int p_tri_wtoep = 0;       // constant-coefficient one-warp kernel: 0 auto, 1 always (else EINVAL), 2 never
  int p_tri_group = 0;       // systems per CTA of the one-CTA-per-system kernel (1..16)
  // Caching allocator: released buffers are kept (up to pool_cap bytes) and
  // reused by later allocations of a similar size, so repeated builds and
  // solves do not pay cudaMalloc/cudaFree (cudaFree synchronises the device).
  std::mutex pool_mu;
  std::multimap<size_t, void*> pool;
  size_t pool_bytes = 0;
  size_t pool_cap = (size_t)16 << 30;
  // Handles (operators, coarse solvers) hold a reference; the context is
  // deleted when lrp_destroy has been called and the last handle is freed.
  int refs = 1;
};
void ctx_retain(Ctx* c);
void ctx_release(Ctx* c);
// A context whose own stream has the given CUDA stream priority (lower
// numbers run first); nullptr on failure.  Released with ctx_release.
Ctx* ctx_create(int device, size_t hbm_budget_bytes, int priority);

// Per-(dt, direction) factorisation of B = I + dt*A (or its transpose) for the
// partitioned tridiagonal solve: P chunks of m rows, interior Thomas factors,
// spikes, and the parallel-cyclic-reduction coefficients of the interface
// system.  Coefficients are stored chunk-minor: entry (row i of chunk t) at
// i*P + t.  Both FP64 and FP32 copies.
struct TriPlan {
  double dt = 0.0;
  int adjoint = 0;
  int n = 0, m = 0, P = 0, levels = 0;
  DevBuf coef64, coef32;   // [5][m][P]: l, inv, u, p, q
  DevBuf pcr64, pcr32;     // [2*levels + 1][P]: k1 per level, k2 per level, dinv
  DevBuf status;           // int: 0 ok, 1 zero pivot
};

// Two-level partition of B = I + dt*A for one system spread over a cluster of
// C CTAs (tridiag_cluster.cu): per-CTA chunk factors, local PCR factors,
// local spikes and the C x C super system.  b[k]: coef, lpcr, spk, sup.
struct ClPlan {
  double dt = 0.0;
  int adjoint = 0, C = 1, n = 0, m = 0, P = 0, Pc = 0, L = 0;
  int warp = 0;   // factors laid out for the one-warp-per-CTA kernel (Pc = 32)
  size_t sz[4] = {0, 0, 0, 0};
  DevBuf b64[4], b32[4];
  DevBuf status;
};

// B = I + dt*A (or its transpose) of a 5-point operator: [6][n + 2 mx] =
// centre, west, east, south, north couplings and 1/centre, each with a zero
// pad of mx entries on both sides; FP64 and FP32 copies.
struct StencilPlan {
  double dt = 0.0;
  int adjoint = 0;
  DevBuf b64, b32;
  DevBuf bs64, bs32;   // symmetric operators: the scaled matrix of CG (k_stencil_plan_scaled)
  // scaled couplings and scales laid out for the on-chip and block CG kernels
  // (stencil_onchip.cu), one per (precision, pitch, padded rows); each is
  // filled once and never changes (plans are shared by every context that
  // propagates with the operator, a server's included)
  struct Layout {
    int prec = 0, pitch = 0, rows = 0;
    DevBuf buf;
  };
  std::vector<std::unique_ptr<Layout>> layouts;
};

// Constant-coefficient (Toeplitz) data of a tridiagonal step matrix
// B = I + dt A for the one-warp kernel (see tri_warp.cuh): lower a, diagonal
// d, upper c; the steady pivot dinf of its LU factorisation (the larger root
// of p = d - a c / p) with l = a / dinf, u = c / dinf; the state is carried
// scaled by dinf per step and rescaled by rho = dinf^-P every P steps; fin
// undoes the scaling left after the last step.
struct ToepCoef {
  int on = 0;
  int P = 1;
  double a = 0.0, d = 1.0, c = 0.0, dinf = 1.0, idinf = 1.0, l = 0.0, u = 0.0;
  double rho = 1.0, fin = 1.0;
};

struct Operator {
  Ctx* ctx = nullptr;
  ~Operator();
  int kind = 0;            // 0 tridiagonal, 1 5-point stencil, 2 time-dependent tridiagonal,
                           // 3 time-dependent 5-point stencil
  int n = 0, mx = 0, my = 0;
  int nJ = 0;              // kinds 2, 3: fine steps of the time grid (a64[k] are nJ x n)
  // tridiagonal with constant coefficients (lo[1..n-1], di, up[0..n-2] each
  // one value): tlo, tdi, tup
  bool toeplitz = false;
  double tlo = 0.0, tdi = 0.0, tup = 0.0;
  DevBuf a64[5];           // tridiagonal: lo, di, up; stencil: C, W, E, S, N
  DevBuf a32[5];
  double rtol64 = 1e-12, rtol32 = 1e-6;
  int max_iter = 20000;
  bool symmetric = false;  // 5-point: CG when symmetric, else BiCGStab
  int stepper = 0;         // fine time stepper: lrp_stepper (tridiagonal operators)
  std::mutex plan_mu;      // plan lookup/creation (a server thread may propagate too)
  std::vector<std::unique_ptr<TriPlan>> plans;
  std::vector<std::unique_ptr<ClPlan>> cplans;
  std::vector<std::unique_ptr<StencilPlan>> splans;
  // Krylov iterations of 2D propagations (contexts of several threads, a
  // server's, may propagate with one operator)
  std::atomic<unsigned long long> krylov_iters{0};
};

struct Coarse {
  Ctx* ctx = nullptr;
  ~Coarse();
  const Operator* op = nullptr;
  double dt = 0.0;
  int M = 0, N = 0, R = 0, p = 0, ell = 0;
  uint64_t seed = 0;
  lrp_precision prec = LRP_PREC_F64;
  DevBuf U, S, V;          // FP64 factors: U, V [N][R][n], S [N][R] (zero padded)
  DevBuf U32, S32, V32;    // FP32 copies (coarse apply of the mixed mode)
  std::vector<int> Ri, rank_w, rank_v;
  std::vector<double> sigma;  // N x ell
  double delta = 0.0, eps = 0.0;
  int orth_tc_w = 0, orth_tc_v = 0;   // intervals orthonormalised on the tensor cores (steps 2, 4)
  // solve workspace (allocated on first use)
  DevBuf Kc;               // [N-1][R][R] chain matrices of the coarse sweep
  DevBuf ws_u, ws_F, ws_b, ws_norm, ws_d, ws_g, ws_c;
  DevBuf ws_cw, ws_cnt, ws_args;   // coarse-sweep workspace
  DevBuf ws_flag, ws_bh;           // stop flag + k_done; a posteriori bounds of every iteration
  DevBuf ws_argv;                  // sweep arguments of every iteration (N + 1)
  void* h_stat = nullptr;          // pinned host slots for the batched convergence checks
  size_t ws_gc_bytes = 0;
};

// ---- helpers ---------------------------------------------------------------
lrp_status set_err(Ctx* c, lrp_status s, const std::string& msg);
lrp_status cuda_err(Ctx* c, cudaError_t e, const char* where);
lrp_status dev_alloc(Ctx* c, DevBuf& b, size_t bytes);
bool is_device_ptr(const void* p);
void timer_begin(Ctx* c, const char* fam, cudaEvent_t* ev);
void timer_end(Ctx* c, const char* fam, cudaEvent_t ev);

// ---- time steppers ----------------------------------------------------------
// Two-stage SDIRK in stage-value form for u' = -A u (Butcher tableau
// (gamma, a21, b1, b2), a11 = a22 = gamma): with B = I + gamma dt A,
//   U1 = B^-1 u,  U2 = B^-1 (su u + s1 U1),  u_new = bu u + b1 U1 + b2 U2,
// su = 1 - a21/gamma, s1 = a21/gamma (from dt K1 = (U1 - u)/gamma), and the
// update u + dt (b1 K1 + b2 K2) written through U1, U2 likewise.
struct StepCoef {
  double gamma, su, s1, bu, b1, b2;
};
StepCoef step_coefficients(int stepper);
// Source samples per fine step of the operator: 2 for the SDIRK steppers
// (the stage times), else 1 (the step end).
int source_samples(const Operator* op);

// ---- tridiagonal propagator (tridiag.cu) -----------------------------------
// m_req = 0: the default chunk size for n; else the requested rows per chunk.
lrp_status tri_get_plan(Ctx* c, Operator* op, double dt, int adjoint, TriPlan** out, int m_req = 0);

// Input of a propagation: either vectors in memory or Gaussian sketch vectors
// generated in the kernel (system s -> interval s / ncol, column s % ncol).
// With a system map (2 ints per system: slot, interval), the vector of system
// s is at base + slot * slot_stride + interval * ld instead of base + s * ld.
__host__ __device__ inline long sys_offset(const int* map, long slot_stride, long ld, int s) {
  return map ? (long)map[2 * s] * slot_stride + (long)map[2 * s + 1] * ld : (long)s * ld;
}

struct PropIn {
  const void* x = nullptr;  // nsys x n (row stride ldx), type given by x_f64
  int x_f64 = 1;
  long ldx = 0;
  const int* map = nullptr; // optional system map (see sys_offset)
  long slot_stride = 0;
  int gen = 0;              // 1: generate N(0,1) entries instead of reading x
  uint64_t seed = 0;
  uint32_t stream = 0;      // Philox stream of the generated entries (0: Omega, 3: Psi)
  int ncol = 1;             // systems per interval (generated input; time-dependent operators)
  int interval0 = 0;        // interval of system 0 (generated input; time-dependent operators)
  const int* stop = nullptr; // optional device flag: nonzero at launch -> the kernel does nothing
};
struct PropOut {
  void* y = nullptr;        // nsys x n (row stride ldy)
  int y_f64 = 1;
  long ldy = 0;
  const int* map = nullptr;
  long slot_stride = 0;
};
struct PropSrc {
  int Q = 0;
  const double* g = nullptr;   // Q x n (device); with a map: + slot * g_slot_stride
  const double* c = nullptr;   // per system: c + s*cstride, M x Q (device)
  long cstride = 0;
  const int* map = nullptr;    // with a map: c + slot * c_slot_stride + interval * cstride
  long c_slot_stride = 0;
  long g_slot_stride = 0;
};

// Any operator: picks the tridiagonal (one CTA or a cluster per system) or the
// stencil propagator.  prec: 0 FP64, 1 FP32 arithmetic.
lrp_status propagate_any(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys, int prec,
                         const PropIn& in, const PropOut& out, const PropSrc& src);

// prec: 0 FP64, 1 FP32 arithmetic.
lrp_status tri_propagate(Ctx* c, Operator* op, TriPlan* plan, int M, int nsys, int prec,
                         const PropIn& in, const PropOut& out, const PropSrc& src);

// One system per cluster of C CTAs (small batches, n >= 2048).
// warp = 1: the one-warp-per-CTA FP64 kernel (8-row chunks, 32 chunks per CTA)
lrp_status tri_get_cluster_plan(Ctx* c, Operator* op, double dt, int adjoint, int C, int m,
                                ClPlan** out, int warp = 0);
// one system per CTA of C warps, with the factorisation of a warp plan
// (tri_get_cluster_plan with warp = 1); prec 0 = FP64, 1 = FP32
lrp_status tri_propagate_warp_block(Ctx* c, ClPlan* pl, int M, int nsys, int prec,
                                    const PropIn& in, const PropOut& out, const PropSrc& src,
                                    const ToepCoef* tz = nullptr);
lrp_status tri_propagate_cluster(Ctx* c, ClPlan* pl, int M, int nsys, int prec, int spt,
                                 const PropIn& in, const PropOut& out, const PropSrc& src,
                                 int stepper = 0, const ToepCoef* tz = nullptr);
// The constant-coefficient data of B = I + dt A (or its transpose) for M
// steps on chunks of m rows, if the operator is Toeplitz, its step matrix has
// a steady pivot, and n mod m is 0 or m - 1 (so that no chunk interior mixes
// rows of the system with padding rows); tz->on = 0 otherwise.
void tri_toeplitz_coef(const Operator* op, double dt, int adjoint, int M, int m, ToepCoef* tz,
                       int prec = 0);

// Time-dependent tridiagonal operators (tridiag_td.cu): one CTA per system,
// parallel cyclic reduction of every step's own matrix; system s runs the
// steps of interval (map ? map[2s+1] : in.interval0 + s / in.ncol).
// Backward-Euler steps of FP64 propagations of time-invariant tridiagonal
// operators (n <= 4096, forward, no source) to about 48 bits from FP32
// solves, each step refined by residuals in pairs of FP32 numbers
// (tridiag_ir.cu); applies when tri_refine = 1.
bool tri_ir_applies(Ctx* c, const Operator* op, int prec, int adjoint, int M, const PropIn& in,
                    const PropSrc& src);
lrp_status tri_propagate_ir(Ctx* c, Operator* op, double dt, int M, int nsys, const PropIn& in,
                            const PropOut& out);
lrp_status tri_td_propagate(Ctx* c, Operator* op, double dt, int M, int adjoint, int nsys,
                            int prec, const PropIn& in, const PropOut& out, const PropSrc& src);

// Allocation-free variant: factorisation into caller-provided scratch.
size_t tri_raw_scratch_bytes(int n);
lrp_status tri_raw_propagate(cudaStream_t stream, int num_sms, void* scratch, int n,
                             const double* lo, const double* di, const double* up, double dt,
                             int adjoint, int M, int nsys, int prec, const PropIn& in,
                             const PropOut& out, const PropSrc& src);

// ---- 5-point stencil propagation (stencil.cu) --------------------------------
// One Krylov propagation problem (5-point operator, a batch of systems).
struct KryArgs {
  int mx, my, n, M, nsys, bicg;
  double dt, rtol;
  int max_iter;
  // two-stage SDIRK steps (stepper != 0; dt is then gamma dt and B = I + gamma dt A):
  // the combination coefficients of step_coefficients; the workspace holds two
  // more vectors (the step's start state and first stage value)
  int stepper;
  double su, s1, bu, b1, b2;
  // time-dependent operators (kind 3): the plans of the steps follow one another
  // (B and Bs advance by b_step and bs_step elements per fine step); system s
  // runs steps J0 .. J0 + M - 1 with J0 = interval * M (the interval from the
  // call's system map, else interval0 + s / ncol of the input), the adjoint in
  // reversed order
  long b_step, bs_step;
  int nJ, adj;
  const void* B;            // [6][n + 2 mx] from element 0 of array 0 (after the pad):
                            // c, w, e, s, n, dinv (type T), zero pads of mx per side
  const void* Bs;           // CG (symmetric operators): [7][n + 2 mx], same layout: west,
                            // east, south, north couplings of S^-1 B S^-1, 1/c, 1/sqrt(c), sqrt(c)
  void* ws;                 // per cluster slot: nvec padded vectors of n + 2 mx values
  int nvec;
  PropIn in;
  PropOut out;
  PropSrc src;
  unsigned long long* iters;   // total Krylov iterations
  int* status;                 // bit 0: cap hit, bit 1: breakdown
  // in-kernel iterative refinement (k_krylov_queue_ir; B, Bs in FP64): the
  // FP32 plans of the same step matrix and the FP32 solves' tolerance
  const void* B32;
  const void* Bs32;
  double rtol_in;
  // FP32 k_krylov: stage the stencil inputs through dynamic shared memory
  // (bulk copies of the CTA's rows and halo rows); set by the launcher
  int stage;
};
lrp_status stencil_plan(Ctx* c, Operator* op, double dt, int adjoint, StencilPlan** out);
// On-chip CG (stencil_onchip.cu): symmetric operators with at most 512 grid
// columns and 16 x 32 (FP32) or 16 x 16 (FP64) rows; every Krylov vector in
// registers and shared memory.  base: the arguments of k_krylov (ws unused).
// Both CG kernels stop on the residual of the diagonally scaled system,
// ||D^1/2 (d - B x)|| <= rtol ||D^1/2 d||, D = diag(B)^-1.
bool stencil_onchip_applies(Ctx* c, const Operator* op, int prec, int nsys);
// Whether the on-chip kernel takes single solves with this operator's (stage)
// matrices at precision prec, whatever its stepper.
bool stencil_onchip_fits(Ctx* c, const Operator* op, int prec, int nsys);
// Scaled couplings (e^, n^) and scales (1/c, 1/sqrt(c), sqrt(c)) of the
// step matrix laid out [rows + 2][pitch] from grid row -1, into buf
// (allocated or grown as needed); T = double for prec 0, else float.
lrp_status oc_coef_fill(Ctx* c, const Operator* op, const StencilPlan* plan, int prec, int pitch,
                        int rows, DevBuf& buf);
// The layout of a plan for (prec, pitch, rows): found, or created and filled
// (the fill completed before it is published).  *ptr: its device address.
lrp_status plan_layout(Ctx* c, Operator* op, StencilPlan* plan, int prec, int pitch, int rows,
                       void** ptr);
// Block CG (stencil_block.cu): symmetric operators, propagations without a
// source, at least two systems; the systems are taken in blocks of
// p_krylov_block consecutive ones, each block on one cluster.
bool stencil_block_applies(Ctx* c, const Operator* op, int prec, int nsys, int M, int Q);
lrp_status stencil_propagate_block(Ctx* c, Operator* op, StencilPlan* plan, int M, int nsys,
                                   int prec, const KryArgs& base);
lrp_status stencil_propagate_onchip(Ctx* c, Operator* op, StencilPlan* plan, int M, int nsys,
                                    int prec, const KryArgs& base);
// FP64 steps (backward Euler, or each SDIRK stage solve) of 5-point operators
// by mixed-precision iterative refinement (stencil_refine.cu): FP64
// residuals, FP32 on-chip CG or BiCGStab corrections, the FP64 Krylov
// kernels' stopping test.  Applies (unless krylov_refine = 2, or the block CG
// was requested and applies) to nonsymmetric time-invariant operators, and to
// symmetric ones wherever the FP32 on-chip kernel takes the grid.
bool stencil_refine_applies(Ctx* c, const Operator* op, int prec, int nsys);
// One FP32 launch of the global-memory Krylov kernel (k_krylov<float>,
// backward-Euler steps) for the correction solves of the refinement of
// nonsymmetric operators; a: the kernel arguments without B, Bs, ws, nvec.
lrp_status krylov_f32_correction(Ctx* c, Operator* op, StencilPlan* plan, int nsys, KryArgs& a);
lrp_status stencil_propagate_refine(Ctx* c, Operator* op, StencilPlan* plan, int M, int nsys,
                                    const PropIn& in, const PropOut& out, const PropSrc& src,
                                    int adjoint);
size_t krylov_queue_nvec(int bicg);
// Device pointer of the stencil coefficients for KryArgs::B (past the pad).
const void* stencil_B(const StencilPlan* pl, const Operator* op, int prec);
// The same for KryArgs::Bs (symmetric operators; nullptr otherwise).
const void* stencil_Bs(const StencilPlan* pl, const Operator* op, int prec);
// prec: 0 FP64, 1 FP32, 2 FP64 steps by in-kernel iterative refinement
// (k_krylov_queue_ir, workspace krylov_queue_ir_bytes(n + 2 mx) per cluster)
int krylov_queue_clusters(Ctx* c, int prec, int cs);
size_t krylov_queue_ir_bytes(int maxld);
lrp_status krylov_queue_launch(Ctx* c, int prec, const KryArgs* d_probs, const int* d_items,
                               int nitems, unsigned int* d_counter, void* ws, size_t ws_stride,
                               int cs, int nclusters);

// ---- orthonormalisation, small SVD, lift (linalg.cu) -----------------------
// CGS2 with deflation of every interval's ell x n block (rows = vectors), in
// place.  Kept vectors are compacted to the front, dropped rows zeroed.
// Rcoef [N][ell][ell] (FP64): Rcoef[c][j] = coefficient of basis vector c in
// input vector j.  rank[N] (device int).
// Two-sided sketch core: B = Psi^T Q, C = B (B^T B)^-1, X^T = Z C into XT
// ([N][ell][n], sketch precision); status bit 1 set when B^T B is singular.
lrp_status two_sided_core(Ctx* c, int N, int ell, int ell2, int n, uint64_t seed, int f32,
                          const void* Q, const int* rank_w, const void* Z, void* XT, double* Bbuf,
                          double* Cbuf, int* status);
// skip: optional [N] flags; intervals with skip[i] != 0 are left untouched.
lrp_status orth_cgs2(Ctx* c, int N, int ell, int n, void* X, int x_f64, double tau,
                     double* Rcoef, int* rank, const int* skip = nullptr);
// CholeskyQR2 with the Gram products and triangular applies on the tensor
// cores (orth_tc.cu) for FP32 blocks with ell <= 64; same outputs as
// orth_cgs2.  Intervals whose scaled Gram is too ill-conditioned fall back to
// CGS2.  ws: orth_tc_workspace() bytes of device memory (allocated by the
// caller, so that the call can be captured in a graph); status: device int,
// bit 4 set when a tensor-core step failed (an mbarrier wait gave up or the
// second pass broke down); tc_count (device int, optional) is incremented
// once per interval orthonormalised on the tensor cores.
bool orth_tc_applies(Ctx* c, int ell, int x_f64);
size_t orth_tc_workspace(Ctx* c, int N, int ell, int n);
lrp_status orth_tc(Ctx* c, int N, int ell, int n, float* X, double tau, double* Rcoef, int* rank,
                   void* ws, size_t ws_bytes, int* status, int* tc_count = nullptr);
// Lift of step 6 on the tensor cores (FP32 bases, ell <= 64, R <= 64); same
// outputs as lift(); status bit 4 on a failed mbarrier wait.
bool lift_tc_applies(Ctx* c, int ell, int R, int b_f64);
lrp_status lift_tc(Ctx* c, int N, int ell, int R, int n, const float* W, const float* Vh,
                   const double* Psi, const double* Phi, const int* Ri, double* U, double* V,
                   float* U32, float* V32, int* status);
// R_i = min(R, rank_w, rank_v) and S (FP64, FP32; zero beyond R_i) of every
// interval from the ranks and singular values of the build (batch.cu).
__global__ void k_finish_ranks(int N, int R, int ell, const int* __restrict__ rw,
                               const int* __restrict__ rv, const double* __restrict__ sv,
                               int* __restrict__ Ri, double* __restrict__ S, float* __restrict__ S32);
// orth_tc when it applies and ws is large enough, else orth_cgs2.
lrp_status orth_auto(Ctx* c, int N, int ell, int n, void* X, int x_f64, double tau, double* Rcoef,
                     int* rank, void* ws, size_t ws_bytes, int* status, int* tc_count = nullptr);
// One-sided Jacobi SVD of M_i = Rz_i^T (ell x ell) for every interval.
// Outputs: s [N][ell] descending, Psi [N][ell][ell] (column r = left vector r,
// stored Psi[i*ell + r]), Phi [N][ell][ell] likewise; status (int) 0/1.
lrp_status small_svd(Ctx* c, int N, int ell, const double* Rz, const int* rank_v, double* s,
                     double* Psi, double* Phi, int* status);
// U_i[r] = sum_j Psi[j][r] W_i[j], V_i[r] = sum_j Phi[j][r] Vh_i[j], r < R.
lrp_status lift(Ctx* c, int N, int ell, int R, int n, const void* W, const void* Vh, int b_f64,
                const double* Psi, const double* Phi, const int* Ri, double* U, double* V,
                float* U32, float* V32);

lrp_status gaussian(Ctx* c, uint64_t seed, int interval, int ncol, int n, int f32, double* out);

// ---- coarse sweep (sweep.cu) ------------------------------------------------
struct SweepArgs {
  int N = 0, n = 0, R = 0;
  int first = 0;                  // interval where the sweep starts (delta = 0 there)
  double* u = nullptr;            // (N+1) x n, in place: u^{k-1} -> u^k
  const double* F = nullptr;      // N x n: F_i u^{k-1}_i (or b_i for the initial sweep)
  const void* U = nullptr;        // [N][R][n] (FP64, or FP32 when f32 = 1)
  const void* S = nullptr;        // [N][R]
  const void* V = nullptr;        // [N][R][n]
  const double* K = nullptr;      // [N-1][R][R]: K_i = V_{i+1}^T U_i diag(S_i)
  int f32 = 0;                    // coarse apply G'delta in FP32 (mixed mode)
  int initial = 0;                // 1: u^{-1} := 0 (initial coarse sweep)
  double delta = 0.0, eps = 0.0;
  double* du = nullptr;           // N+1: ||u^k_m - u^{k-1}_m||
  double* unorm = nullptr;        // N+1: ||u^k_m||
  double* bound = nullptr;        // N+1: a posteriori bound (Eq. apost_bound)
  double* summary = nullptr;      // [0] = max bound, [1] = max ||u^k_m||
  int rows = 0, nsl = 0;          // rows per slice, slices = ceil(n / rows)
  double* cw = nullptr;           // workspace, sweep_ws_doubles(N, nsl, R) doubles
  unsigned* cnt = nullptr;        // 2 completion counters, zero between launches
  // device-side stopping (single-problem solves): when stop != nullptr the
  // kernels do nothing while *stop != 0, and the apply's last CTA records
  // k_done[0] = iter and sets *stop when tol > 0 and max bound <= tol max ||u||
  int* stop = nullptr;
  int* k_done = nullptr;
  int iter = 0;
  double tol = 0.0;
};
// Coarse sweep of nprob problems of equal N and precision in two launches;
// h is uploaded to d_args (nprob entries) on the stream and must stay alive
// until the stream has passed the upload.
lrp_status coarse_sweep(Ctx* c, const SweepArgs* h, SweepArgs* d_args, int nprob);
// The same with upload = 0: d_args already holds h (uploaded earlier on the
// stream), so nothing is copied before the launches.
lrp_status coarse_sweep_ex(Ctx* c, const SweepArgs* h, SweepArgs* d_args, int nprob, int upload);
size_t sweep_ws_doubles(int N, int nsl, int R);
int sweep_rows(Ctx* c);
// K_i of a coarse handle (Coarse::Kc), formed from the factors its apply uses.
lrp_status coarse_chain(Ctx* c, Coarse* co);
// Per-handle sweep workspace (ws_cw, ws_cnt, ws_args) for slices of `rows`.
lrp_status coarse_sweep_workspace(Ctx* c, Coarse* co, int rows);

}  // namespace lrp
