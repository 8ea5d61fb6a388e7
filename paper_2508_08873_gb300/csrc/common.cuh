// Shared device helpers of the sm_103a library: error plumbing, the
// Philox4x32-10 generator with Box-Muller deviates, and block reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define LRP_DEV __device__ __forceinline__

namespace lrp {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): 10 rounds of the 4x32 multiply-xor bijection with a
// Weyl-sequence key schedule.  Counter (row, column, interval, stream), key =
// the two 32-bit halves of the seed.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

LRP_DEV U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// Standard normal in FP64: U1 = (top 53 bits of x:y + 1) 2^-53 in (0, 1],
// U2 = (top 53 bits of z:w) 2^-53, z = sqrt(-2 ln U1) cos(2 pi U2).
LRP_DEV double gauss_f64(uint64_t seed, uint32_t stream, uint32_t interval, uint32_t column,
                         uint32_t row) {
  U4 w = philox10(U4{row, column, interval, stream}, (uint32_t)seed, (uint32_t)(seed >> 32));
  uint64_t a = (((uint64_t)w.x << 32) | w.y) >> 11;
  uint64_t b = (((uint64_t)w.z << 32) | w.w) >> 11;
  double u1 = ((double)a + 1.0) * 0x1.0p-53;
  double u2 = (double)b * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Same deviate computed in FP32 from the same Philox words (24-bit uniforms):
// the FP32 sketch path uses it; it agrees with gauss_f64 to FP32 accuracy
// except where U1 rounds differently near 0.
LRP_DEV float gauss_f32(uint64_t seed, uint32_t stream, uint32_t interval, uint32_t column,
                        uint32_t row) {
  U4 w = philox10(U4{row, column, interval, stream}, (uint32_t)seed, (uint32_t)(seed >> 32));
  float u1 = ((float)(w.x >> 8) + 1.0f) * 0x1.0p-24f;
  float u2 = (float)(w.z >> 8) * 0x1.0p-24f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

template <typename T> LRP_DEV T gauss(uint64_t s, uint32_t st, uint32_t i, uint32_t c, uint32_t r);
template <> LRP_DEV double gauss<double>(uint64_t s, uint32_t st, uint32_t i, uint32_t c, uint32_t r) {
  return gauss_f64(s, st, i, c, r);
}
template <> LRP_DEV float gauss<float>(uint64_t s, uint32_t st, uint32_t i, uint32_t c, uint32_t r) {
  return gauss_f32(s, st, i, c, r);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <typename T> LRP_DEV T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace lrp
