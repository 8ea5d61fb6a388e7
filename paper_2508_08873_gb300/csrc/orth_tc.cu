// CholeskyQR2 of the FP32 sketch blocks with the Gram products and the
// triangular applies on the fifth-generation tensor cores (tcgen05, TF32
// operands in shared memory, FP32 accumulation in tensor memory), for steps 2
// and 4 of the randomized SVD (Sec. 2.1: orthonormal bases of the range of
// F_n' Omega and of F_n'^* W).
//
// For every interval, with Y the ell x n block (rows = vectors, ell <= 64):
//   G  = Y Y^T                        tcgen05 Gram, rows of n split over CTAs,
//                                     the split partials summed in FP64
//   D  = diag(G)^-1/2, D G D = L L^T  FP64 Cholesky, one CTA per interval
//   Q1 = D L^-1 ... applied as Q1^T = Y^T D L^-T    tcgen05 apply, in place
//   R1 = L^T D^-1
//   G2 = Q1 Q1^T = L2 L2^T, Q2^T = Q1^T L2^-T, R = L2^T R1   (second pass)
// so that y_j = sum_c R[c][j] q_c with R upper triangular: the same
// coefficient layout (Rcoef[c][j]) as the Gram-Schmidt kernels, so that the
// small matrix of step 5 is read off it unchanged.
//
// Every product is formed as hi*hi + hi*lo + lo*hi with x = hi + lo and
// hi = x rounded to TF32 (error-corrected TF32, Ootomo and Yokota 2022), which
// keeps the Gram at FP32 accuracy.  CholeskyQR2 is stable while kappa(Y)^2
// times the relative error of the Gram stays well below one (Yamamoto,
// Nakatsukasa, Yanagisawa and Fukaya 2015).  The condition number of the
// scaled Gram is bounded by ||D G D||_F ||L^-1||_F^2; an interval above
// TC_KAPPA_MAX (rank-deficient sketches of quickly decaying spectra) is left
// untouched here and orthonormalised by CGS2 with deflation instead.
//
// The lift of step 6 (U = W Psi, V = V^ Phi restricted to the leading R
// singular vectors) is the same contraction and runs on the same path.
//
// Shared-memory operands are K-major tiles of 32 FP32 values (128 bytes) per
// row with the 128-byte swizzle; every MMA is M = 128 (rows beyond the data
// are zero), N = the padded sketch width or rank, K = 8.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace lrp {
namespace {

constexpr int TC_THREADS = 128;            // four warps = the 128 lanes of tensor memory
constexpr int TC_MAXL = 64;                // widest block handled on the tensor cores
constexpr int TILE_ROWS = 128;             // M of every MMA
constexpr int TILE_BYTES = TILE_ROWS * 128;
constexpr uint32_t TMEM_COLS = 64;         // FP32 accumulator columns (>= N)
constexpr double TC_KAPPA_MAX = 1e5;       // bound on kappa(D G D) for the tensor-core path
constexpr long TC_SPIN = 1L << 22;         // polls of an mbarrier before giving up

LRP_DEV uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

LRP_DEV unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// Byte offset of element (r, k), k < 32, in a K-major tile with the 128-byte
// swizzle: the 16-byte chunk index of a row is XORed with the row index mod 8
// (the tile starts on a 1024-byte boundary).
LRP_DEV uint32_t sw128(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 2) ^ r) & 7) << 4) + ((k & 3) << 2));
}

// Shared-memory matrix descriptor: start address, leading-dimension offset
// (unused by swizzled K-major layouts), stride between 8-row groups = 1024
// bytes, descriptor version 1, 128-byte swizzle.
LRP_DEV uint64_t sdesc(uint32_t a) {
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::tf32: D in FP32, A and B in TF32, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

LRP_DEV float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

LRP_DEV void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

LRP_DEV void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

LRP_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
LRP_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
LRP_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

LRP_DEV void mbar_init(uint32_t a) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

LRP_DEV bool mbar_wait(uint32_t a, uint32_t parity) {
  for (long i = 0; i < TC_SPIN; ++i) {
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

LRP_DEV void tmem_alloc(uint32_t slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
               "r"(TMEM_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

LRP_DEV void tmem_free(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS)
               : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
LRP_DEV void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// Gram partials.  blockIdx.y = interval, blockIdx.x = split of the n columns
// (kchunk each, a multiple of 32).  Two shared-memory stages of (hi, lo)
// tiles: while the tensor core multiplies one, the CTA fills the other.
// part[iv][split][ell][ell] (FP32).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS) k_gram_tc(const float* __restrict__ X, int ell, int n,
                                                        int kchunk, int NB, float* __restrict__ part,
                                                        const int* __restrict__ active,
                                                        int* __restrict__ status) {
  extern __shared__ unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ int sfail;
  const int iv = blockIdx.y, sp = blockIdx.x, S = gridDim.x;
  if (active && !active[iv]) return;
  unsigned char* base = align1024(tc_smem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 4 * TILE_BYTES / 16; i += TC_THREADS)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(saddr(&mbar[0]));
    mbar_init(saddr(&mbar[1]));
    sfail = 0;
  }
  if (warp == 0) tmem_alloc(saddr(&tslot));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const int k0 = sp * kchunk, k1 = min(n, k0 + kchunk);
  const int nb = k1 > k0 ? (k1 - k0 + 31) / 32 : 0;
  const float* Xi = X + (size_t)iv * ell * n;
  const uint32_t idesc = idesc_tf32(TILE_ROWS, NB);
  // commit j (the MMAs of block j) arrives on mbar[j & 1], completing its
  // phase (j >> 1) & 1; thread 0 waits for the commits in issue order.
  // Thread t loads column k = t mod 32 of rows t/32, t/32 + 4, ...; the
  // values of the next two blocks are in flight in registers while a block
  // is staged and multiplied.
  const int kc = tid & 31, rg = tid >> 5;
  const int nrow = (ell - rg + 3) / 4;            // rows of this thread (<= 16)
  auto load = [&](float* v, int b) {
    const int col = k0 + b * 32 + kc;
    const bool in = b < nb && col < k1;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      v[j] = (in && j < nrow) ? Xi[(size_t)(rg + 4 * j) * n + col] : 0.f;
  };
  int issued = 0, waited = 0;
  auto stage = [&](const float* v, int b) -> bool {
    const int s = b & 1;
    if (b >= 2) {
      // the MMAs of block b-2 read this stage
      if (tid == 0 && !mbar_wait(saddr(&mbar[s]), (uint32_t)(((b - 2) >> 1) & 1))) sfail = 1;
      waited = b - 1;
      __syncthreads();
      if (sfail) return false;
    }
    unsigned char* hi = base + s * 2 * TILE_BYTES;
    unsigned char* lo = hi + TILE_BYTES;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j < nrow) {
        const float h = tf32_hi(v[j]);
        *reinterpret_cast<float*>(hi + sw128(rg + 4 * j, kc)) = h;
        *reinterpret_cast<float*>(lo + sw128(rg + 4 * j, kc)) = v[j] - h;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = saddr(hi), al = saddr(lo);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t dh = sdesc(ah + kk * 32), dl = sdesc(al + kk * 32);
        mma_tf32(tmem, dh, dh, idesc, (b | kk) != 0);
        mma_tf32(tmem, dh, dl, idesc, 1u);
        mma_tf32(tmem, dl, dh, idesc, 1u);
      }
      mma_commit(saddr(&mbar[s]));
    }
    issued = b + 1;
    return true;
  };
  float va[16], vb[16];
  load(va, 0);
  load(vb, 1);
  for (int b = 0; b < nb; b += 2) {
    if (!stage(va, b)) break;
    load(va, b + 2);
    if (b + 1 < nb) {
      if (!stage(vb, b + 1)) break;
      load(vb, b + 3);
    }
  }
  // every commit still outstanding (also after a failed wait: the tensor
  // memory is released only once the MMAs that write it are done)
  if (tid == 0)
    for (int j = waited; j < issued; ++j)
      if (!mbar_wait(saddr(&mbar[j & 1]), (uint32_t)((j >> 1) & 1))) sfail = 1;
  __syncthreads();
  tc_fence_after();
  float* out = part + ((size_t)iv * S + sp) * ell * ell;
  if (sfail) {
    if (tid == 0) atomicOr(status, 4);
  } else {
    const int r = warp * 32 + lane;
    for (int cb = 0; cb < NB / 16; ++cb) {
      float v[16];
      if (nb > 0) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (r < ell) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = cb * 16 + j;
          if (col < ell) out[(size_t)r * ell + col] = v[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem);
}

// ---------------------------------------------------------------------------
// Triangular apply in place: for the 128 columns i0..i0+127 of interval iv,
// Y^T[i][c] <- sum_k Y^T[i][k] T[k][c] with B[c][k] = T[k][c] given as
// FP32 (hi, lo) pairs Tb[iv][2][NB][KB*32].  blockIdx = (column block,
// interval); intervals with active[iv] = 0 are skipped.
// ---------------------------------------------------------------------------
template <int KB>
__global__ void __launch_bounds__(TC_THREADS) k_apply_tc(float* __restrict__ X, int ell, int n, int NB,
                                                         const float* __restrict__ Tb,
                                                         const int* __restrict__ active,
                                                         int* __restrict__ status) {
  extern __shared__ unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int sfail;
  const int iv = blockIdx.y, i0 = blockIdx.x * TILE_ROWS;
  if (!active[iv]) return;
  unsigned char* base = align1024(tc_smem);
  unsigned char* A = base;                                  // [KB][hi, lo] x TILE_BYTES
  unsigned char* B = base + KB * 2 * TILE_BYTES;            // [KB][hi, lo] x NB * 128
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(saddr(&mbar));
    sfail = 0;
  }
  if (warp == 0) tmem_alloc(saddr(&tslot));
  float* Xi = X + (size_t)iv * ell * n;
  const int gi = i0 + tid;                                  // this thread's row of A
#pragma unroll
  for (int k0 = 0; k0 < KB * 32; k0 += 16) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      v[j] = (k0 + j < ell && gi < n) ? Xi[(size_t)(k0 + j) * n + gi] : 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = k0 + j;
      const float h = tf32_hi(v[j]);
      unsigned char* t = A + (k >> 5) * 2 * TILE_BYTES;
      *reinterpret_cast<float*>(t + sw128(tid, k & 31)) = h;
      *reinterpret_cast<float*>(t + TILE_BYTES + sw128(tid, k & 31)) = v[j] - h;
    }
  }
  const int KP = KB * 32;
  const float* Ti = Tb + (size_t)iv * 2 * NB * KP;
  for (int idx = tid; idx < NB * KP; idx += TC_THREADS) {
    const int cc = idx / KP, k = idx % KP;
    unsigned char* t = B + (k >> 5) * 2 * (NB * 128);
    *reinterpret_cast<float*>(t + sw128(cc, k & 31)) = Ti[idx];
    *reinterpret_cast<float*>(t + NB * 128 + sw128(cc, k & 31)) = Ti[(size_t)NB * KP + idx];
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(TILE_ROWS, NB);
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      const uint32_t ah = saddr(A + kb * 2 * TILE_BYTES), al = ah + TILE_BYTES;
      const uint32_t bh = saddr(B + kb * 2 * NB * 128), bl = bh + NB * 128;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        mma_tf32(tmem, sdesc(ah + kk * 32), sdesc(bh + kk * 32), idesc, (kb | kk) != 0);
        mma_tf32(tmem, sdesc(ah + kk * 32), sdesc(bl + kk * 32), idesc, 1u);
        mma_tf32(tmem, sdesc(al + kk * 32), sdesc(bh + kk * 32), idesc, 1u);
      }
    }
    mma_commit(saddr(&mbar));
    if (!mbar_wait(saddr(&mbar), 0)) {
      sfail = 1;
      mbar_wait(saddr(&mbar), 0);
    }
  }
  __syncthreads();
  tc_fence_after();
  if (!sfail) {
    for (int cb = 0; cb < NB / 16; ++cb) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), v);
      if (gi < n) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = cb * 16 + j;
          if (cc < ell) Xi[(size_t)cc * n + gi] = v[j];
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(status, 4);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem);
}

// ---------------------------------------------------------------------------
// Lift of rSVD step 6 on the tensor cores: for the 128 columns i0.. of
// interval iv, out[c][i] = sum_k X[k][i] Bsrc[c][k] for c < R (Bsrc = Psi or
// Phi, FP64 rows of length ell, split into TF32 (hi, lo) pairs here), written
// in FP64 and FP32; rows c >= Ri[iv] are zero.  blockIdx.z = 0: U from W and
// Psi, 1: V from V^ and Phi.
// ---------------------------------------------------------------------------
template <int KB>
__global__ void __launch_bounds__(TC_THREADS) k_lift_tc(int ell, int R, int n, int NB,
                                                        const float* __restrict__ W,
                                                        const float* __restrict__ Vh,
                                                        const double* __restrict__ Psi,
                                                        const double* __restrict__ Phi,
                                                        const int* __restrict__ Ri,
                                                        double* __restrict__ U, double* __restrict__ V,
                                                        float* __restrict__ U32, float* __restrict__ V32,
                                                        int* __restrict__ status) {
  extern __shared__ unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int sfail;
  const int iv = blockIdx.y, i0 = blockIdx.x * TILE_ROWS, z = blockIdx.z;
  const float* X = (z ? Vh : W) + (size_t)iv * ell * n;
  const double* Bs = (z ? Phi : Psi) + (size_t)iv * ell * ell;
  double* out = (z ? V : U) + (size_t)iv * R * n;
  float* out32 = (z ? V32 : U32) + (size_t)iv * R * n;
  const int rk = min(R, Ri[iv]);
  unsigned char* base = align1024(tc_smem);
  unsigned char* A = base;                                  // [KB][hi, lo] x TILE_BYTES
  unsigned char* B = base + KB * 2 * TILE_BYTES;            // [KB][hi, lo] x NB * 128
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(saddr(&mbar));
    sfail = 0;
  }
  if (warp == 0) tmem_alloc(saddr(&tslot));
  const int gi = i0 + tid;
#pragma unroll
  for (int k0 = 0; k0 < KB * 32; k0 += 16) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      v[j] = (k0 + j < ell && gi < n) ? X[(size_t)(k0 + j) * n + gi] : 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = k0 + j;
      const float h = tf32_hi(v[j]);
      unsigned char* t = A + (k >> 5) * 2 * TILE_BYTES;
      *reinterpret_cast<float*>(t + sw128(tid, k & 31)) = h;
      *reinterpret_cast<float*>(t + TILE_BYTES + sw128(tid, k & 31)) = v[j] - h;
    }
  }
  const int KP = KB * 32;
  for (int idx = tid; idx < NB * KP; idx += TC_THREADS) {
    const int cc = idx / KP, k = idx % KP;
    const float b = (cc < rk && k < ell) ? (float)Bs[(size_t)cc * ell + k] : 0.f;
    const float h = tf32_hi(b);
    unsigned char* t = B + (k >> 5) * 2 * (NB * 128);
    *reinterpret_cast<float*>(t + sw128(cc, k & 31)) = h;
    *reinterpret_cast<float*>(t + NB * 128 + sw128(cc, k & 31)) = b - h;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(TILE_ROWS, NB);
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      const uint32_t ah = saddr(A + kb * 2 * TILE_BYTES), al = ah + TILE_BYTES;
      const uint32_t bh = saddr(B + kb * 2 * NB * 128), bl = bh + NB * 128;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        mma_tf32(tmem, sdesc(ah + kk * 32), sdesc(bh + kk * 32), idesc, (kb | kk) != 0);
        mma_tf32(tmem, sdesc(ah + kk * 32), sdesc(bl + kk * 32), idesc, 1u);
        mma_tf32(tmem, sdesc(al + kk * 32), sdesc(bh + kk * 32), idesc, 1u);
      }
    }
    mma_commit(saddr(&mbar));
    if (!mbar_wait(saddr(&mbar), 0)) {
      sfail = 1;
      mbar_wait(saddr(&mbar), 0);
    }
  }
  __syncthreads();
  tc_fence_after();
  if (!sfail) {
    for (int cb = 0; cb < NB / 16; ++cb) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), v);
      if (gi < n) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = cb * 16 + j;
          if (cc < R) {
            const float val = cc < rk ? v[j] : 0.f;
            out[(size_t)cc * n + gi] = (double)val;
            out32[(size_t)cc * n + gi] = val;
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(status, 4);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem);
}

// ---------------------------------------------------------------------------
// Per interval, FP64: sum of the Gram partials, diagonal scaling, Cholesky,
// L^-1, the condition test and the factors.  pass 1: active[iv] <- test,
// R1 = L^T D^-1, Tb = D L^-T; pass 2 (intervals with active = 1):
// Rcoef = L2^T D2^-1 R1, rank = ell, Tb = D2 L2^-T; a failed test in pass 2
// sets status bit 4.
// ---------------------------------------------------------------------------
constexpr int SM_THREADS = 256;

__global__ void __launch_bounds__(SM_THREADS) k_cholqr_small(int ell, int S, int NB, int KP,
                                                             const float* __restrict__ part, int pass,
                                                             int* __restrict__ active,
                                                             double* __restrict__ R1,
                                                             float* __restrict__ Tb,
                                                             double* __restrict__ Rcoef,
                                                             int* __restrict__ rank,
                                                             int* __restrict__ status,
                                                             int* __restrict__ tc_count) {
  extern __shared__ double small_smem[];
  const int ld = ell + 1;
  double* A = small_smem;                 // [ell][ell + 1]
  double* Li = A + (size_t)ell * ld;      // [ell][ell + 1]
  __shared__ double dsc[TC_MAXL];
  __shared__ double rinv[TC_MAXL];           // 1 / L_jj
  __shared__ double red[SM_THREADS / 32];
  __shared__ int sok;
  __shared__ double anorm;
  const int iv = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned FULL = 0xffffffffu;
  if (pass == 2 && !active[iv]) return;
  if (tid == 0) sok = 1;
  const float* P = part + (size_t)iv * S * ell * ell;
  for (int idx = tid; idx < ell * ell; idx += SM_THREADS) {
    double g = 0.0;
    for (int s = 0; s < S; ++s) g += (double)P[(size_t)s * ell * ell + idx];
    A[(size_t)(idx / ell) * ld + (idx % ell)] = g;
  }
  __syncthreads();
  for (int j = tid; j < ell; j += SM_THREADS) {
    const double d = A[(size_t)(j) * ld + (j)];
    const bool good = d > 0.0 && isfinite(d);
    dsc[j] = good ? sqrt(d) : 1.0;
    if (!good) sok = 0;
  }
  __syncthreads();
  // symmetrise and scale to a unit diagonal (lower triangle, via Li); ||A||_F
  double fa = 0.0;
  for (int idx = tid; idx < ell * ell; idx += SM_THREADS) {
    const int j = idx / ell, k = idx % ell;
    if (k <= j) {
      const double v = 0.5 * (A[(size_t)(j) * ld + (k)] + A[(size_t)(k) * ld + (j)]) / (dsc[j] * dsc[k]);
      Li[(size_t)(j) * ld + (k)] = v;
      fa += (k < j ? 2.0 : 1.0) * v * v;
    }
  }
  fa = warp_sum<double>(fa);
  if (lane == 0) red[warp] = fa;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < SM_THREADS / 32; ++w) t += red[w];
    anorm = sqrt(t);
  }
  __syncthreads();
  for (int idx = tid; idx < ell * ell; idx += SM_THREADS) {
    const int j = idx / ell, k = idx % ell;
    A[(size_t)(j) * ld + (k)] = k <= j ? Li[(size_t)(j) * ld + (k)] : 0.0;
  }
  __syncthreads();
  // Cholesky A = L L^T in place (lower)
  for (int j = 0; j < ell; ++j) {
    if (tid == 0) {
      double p = A[(size_t)(j) * ld + (j)];
      if (!(p > 0.0)) {
        sok = 0;
        p = 1.0;
      }
      const double l = sqrt(p);
      A[(size_t)(j) * ld + (j)] = l;
      rinv[j] = 1.0 / l;
    }
    __syncthreads();
    const double rl = rinv[j];
    for (int i = j + 1 + tid; i < ell; i += SM_THREADS) A[(size_t)(i) * ld + (j)] *= rl;
    __syncthreads();
    const int m = ell - j - 1;
    for (int idx = tid; idx < m * m; idx += SM_THREADS) {
      const int i = j + 1 + idx / m, k = j + 1 + idx % m;
      if (k <= i) A[(size_t)(i) * ld + (k)] -= A[(size_t)(i) * ld + (j)] * A[(size_t)(k) * ld + (j)];
    }
    __syncthreads();
  }
  // Li = L^-1 (lower): one warp per column, lanes hold rows lane and lane+32
  for (int c = warp; c < ell; c += SM_THREADS / 32) {
    double x0 = lane == c ? 1.0 : 0.0, x1 = lane + 32 == c ? 1.0 : 0.0;
    for (int k = c; k < ell; ++k) {
      double xk = k < 32 ? __shfl_sync(FULL, x0, k) : __shfl_sync(FULL, x1, k - 32);
      xk *= rinv[k];
      if (lane == (k & 31)) {
        if (k < 32) x0 = xk; else x1 = xk;
      }
      if (lane > k && lane < ell) x0 -= A[(size_t)(lane) * ld + (k)] * xk;
      if (lane + 32 > k && lane + 32 < ell) x1 -= A[(size_t)(lane + 32) * ld + (k)] * xk;
    }
    if (lane < ell) Li[(size_t)(lane) * ld + (c)] = lane >= c ? x0 : 0.0;
    if (lane + 32 < ell) Li[(size_t)(lane + 32) * ld + (c)] = lane + 32 >= c ? x1 : 0.0;
  }
  __syncthreads();
  // kappa(A) = ||A||_2 ||A^-1||_2 <= ||A||_F ||L^-1||_F^2
  double f = 0.0;
  for (int idx = tid; idx < ell * ell; idx += SM_THREADS) {
    const double v = Li[(size_t)(idx / ell) * ld + (idx % ell)];
    f += v * v;
  }
  f = warp_sum<double>(f);
  if (lane == 0) red[warp] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < SM_THREADS / 32; ++w) t += red[w];
    if (!(anorm * t <= TC_KAPPA_MAX)) sok = 0;
  }
  __syncthreads();
  const bool ok = sok != 0;
  if (pass == 1) {
    if (tid == 0) active[iv] = ok ? 1 : 0;
    if (!ok) return;
  } else if (!ok) {
    if (tid == 0) atomicOr(status, 4);
    return;
  }
  // B operand of the apply: B[c][k] = (D L^-T)[k][c] = Li[c][k] / dsc[k]
  float* T = Tb + (size_t)iv * 2 * NB * KP;
  for (int idx = tid; idx < NB * KP; idx += SM_THREADS) {
    const int c = idx / KP, k = idx % KP;
    const double b = (c < ell && k < ell && k <= c) ? Li[(size_t)(c) * ld + (k)] / dsc[k] : 0.0;
    const float bf = (float)b, h = tf32_hi(bf);
    T[idx] = h;
    T[(size_t)NB * KP + idx] = bf - h;
  }
  // R = L^T D^-1 (upper): R[c][j] = L[j][c] dsc[j]
  double* R1i = R1 + (size_t)iv * ell * ell;
  if (pass == 1) {
    for (int idx = tid; idx < ell * ell; idx += SM_THREADS) {
      const int c = idx / ell, j = idx % ell;
      R1i[idx] = c <= j ? A[(size_t)(j) * ld + (c)] * dsc[j] : 0.0;
    }
  } else {
    double* Rc = Rcoef + (size_t)iv * ell * ell;
    for (int idx = tid; idx < ell * ell; idx += SM_THREADS) {
      const int c = idx / ell, j = idx % ell;
      double s = 0.0;
      for (int k = c; k <= j; ++k) s += A[(size_t)(k) * ld + (c)] * dsc[k] * R1i[(size_t)k * ell + j];
      Rc[idx] = s;
    }
    if (tid == 0) {
      rank[iv] = ell;
      if (tc_count) atomicAdd(tc_count, 1);
    }
  }
}

struct TcLayout {
  int S = 0, kchunk = 0, NB = 0, KB = 0;
  size_t part = 0, tb = 0, r1 = 0, act = 0, total = 0;
};

TcLayout tc_layout(int num_sms, int N, int ell, int n) {
  TcLayout L;
  L.NB = (ell + 15) / 16 * 16;
  L.KB = (ell + 31) / 32;
  // splits of the rows: enough CTAs for every SM several times, at most 8192
  // rows per CTA
  int S = std::max((4 * num_sms + N - 1) / N, (n + 8191) / 8192);
  S = std::max(1, std::min(S, (n + 31) / 32));
  int kchunk = ((n + S - 1) / S + 31) / 32 * 32;
  S = (n + kchunk - 1) / kchunk;
  L.S = S;
  L.kchunk = kchunk;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  L.part = 0;
  L.tb = up(L.part + sizeof(float) * (size_t)N * S * ell * ell);
  L.r1 = up(L.tb + sizeof(float) * (size_t)N * 2 * L.NB * L.KB * 32);
  L.act = up(L.r1 + sizeof(double) * (size_t)N * ell * ell);
  L.total = up(L.act + sizeof(int) * (size_t)N);
  return L;
}

}  // namespace

bool orth_tc_applies(Ctx* c, int ell, int x_f64) {
  return !x_f64 && ell >= 1 && ell <= TC_MAXL && c->p_orth_tc != 0;
}

size_t orth_tc_workspace(Ctx* c, int N, int ell, int n) {
  if (ell < 1 || ell > TC_MAXL || N < 1 || n < 1) return 0;
  return tc_layout(c->num_sms, N, ell, n).total;
}

lrp_status orth_tc(Ctx* c, int N, int ell, int n, float* X, double tau, double* Rcoef, int* rank,
                   void* ws, size_t ws_bytes, int* status, int* tc_count) {
  if (N <= 0) return LRP_OK;
  const TcLayout L = tc_layout(c->num_sms, N, ell, n);
  if (ell < 1 || ell > TC_MAXL || !ws || ws_bytes < L.total)
    return set_err(c, LRP_EINVAL, "tensor-core orthonormalisation: workspace too small");
  unsigned char* w = static_cast<unsigned char*>(ws);
  float* part = reinterpret_cast<float*>(w + L.part);
  float* Tb = reinterpret_cast<float*>(w + L.tb);
  double* R1 = reinterpret_cast<double*>(w + L.r1);
  int* act = reinterpret_cast<int*>(w + L.act);
  const size_t smem_g = 4 * TILE_BYTES + 1024;
  const size_t smem_a = (size_t)L.KB * 2 * TILE_BYTES + (size_t)L.KB * 2 * L.NB * 128 + 1024;
  const size_t smem_s = sizeof(double) * 2 * (size_t)ell * (ell + 1);
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_g);
  if (!e) e = cudaFuncSetAttribute(k_cholqr_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
  if (!e)
    e = L.KB == 1 ? cudaFuncSetAttribute(k_apply_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a)
                  : cudaFuncSetAttribute(k_apply_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
  if (e) return cuda_err(c, e, "tensor-core orthonormalisation attributes");
  const dim3 gg(L.S, N), ga((n + TILE_ROWS - 1) / TILE_ROWS, N);
  cudaEvent_t ev = nullptr;
  timer_begin(c, "orth", &ev);
  for (int pass = 1; pass <= 2; ++pass) {
    k_gram_tc<<<gg, TC_THREADS, smem_g, c->stream>>>(X, ell, n, L.kchunk, L.NB, part,
                                                     pass == 2 ? act : nullptr, status);
    k_cholqr_small<<<N, SM_THREADS, smem_s, c->stream>>>(ell, L.S, L.NB, L.KB * 32, part, pass, act,
                                                          R1, Tb, Rcoef, rank, status, tc_count);
    if (L.KB == 1)
      k_apply_tc<1><<<ga, TC_THREADS, smem_a, c->stream>>>(X, ell, n, L.NB, Tb, act, status);
    else
      k_apply_tc<2><<<ga, TC_THREADS, smem_a, c->stream>>>(X, ell, n, L.NB, Tb, act, status);
  }
  e = cudaGetLastError();
  timer_end(c, "orth", ev);
  c->launches += 5;    // six launches above, one counted by timer_end
  if (e) return cuda_err(c, e, "tensor-core orthonormalisation");
  // intervals the test sent back: CGS2 with deflation on their untouched blocks
  return orth_cgs2(c, N, ell, n, X, 0, tau, Rcoef, rank, act);
}

bool lift_tc_applies(Ctx* c, int ell, int R, int b_f64) {
  return !b_f64 && ell >= 1 && ell <= TC_MAXL && R >= 1 && R <= TC_MAXL && c->p_orth_tc != 0;
}

lrp_status lift_tc(Ctx* c, int N, int ell, int R, int n, const float* W, const float* Vh,
                   const double* Psi, const double* Phi, const int* Ri, double* U, double* V,
                   float* U32, float* V32, int* status) {
  if (N <= 0 || R <= 0) return LRP_OK;
  if (ell > TC_MAXL || R > TC_MAXL) return set_err(c, LRP_EINVAL, "tensor-core lift: width above 64");
  const int NB = (R + 15) / 16 * 16, KB = (ell + 31) / 32;
  const size_t smem = (size_t)KB * 2 * TILE_BYTES + (size_t)KB * 2 * NB * 128 + 1024;
  cudaError_t e = KB == 1
      ? cudaFuncSetAttribute(k_lift_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
      : cudaFuncSetAttribute(k_lift_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return cuda_err(c, e, "tensor-core lift attributes");
  const dim3 grid((n + TILE_ROWS - 1) / TILE_ROWS, N, 2);
  cudaEvent_t ev = nullptr;
  timer_begin(c, "lift", &ev);
  if (KB == 1)
    k_lift_tc<1><<<grid, TC_THREADS, smem, c->stream>>>(ell, R, n, NB, W, Vh, Psi, Phi, Ri, U, V, U32,
                                                        V32, status);
  else
    k_lift_tc<2><<<grid, TC_THREADS, smem, c->stream>>>(ell, R, n, NB, W, Vh, Psi, Phi, Ri, U, V, U32,
                                                        V32, status);
  e = cudaGetLastError();
  timer_end(c, "lift", ev);
  return e ? cuda_err(c, e, "k_lift_tc") : LRP_OK;
}

lrp_status orth_auto(Ctx* c, int N, int ell, int n, void* X, int x_f64, double tau, double* Rcoef,
                     int* rank, void* ws, size_t ws_bytes, int* status, int* tc_count) {
  if (orth_tc_applies(c, ell, x_f64) && ws && ws_bytes >= orth_tc_workspace(c, N, ell, n))
    return orth_tc(c, N, ell, n, static_cast<float*>(X), tau, Rcoef, rank, ws, ws_bytes, status,
                   tc_count);
  return orth_cgs2(c, N, ell, n, X, x_f64, tau, Rcoef, rank);
}

}  // namespace lrp
