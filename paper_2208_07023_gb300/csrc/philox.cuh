// Philox4x32-10 counter-based generator for device code.
//
// Restated from Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers: As
// Easy as 1, 2, 3" (SC'11): each of the ten rounds multiplies words 0 and 2
// of the counter by two fixed odd constants, keeps the 64-bit products' high
// and low halves, and mixes the high halves with words 1 and 3 and the round
// key; the key advances by two Weyl constants between rounds.
#pragma once

#include <stdint.h>

namespace slm {

struct U4 {
  uint32_t v[4];
};

__host__ __device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1,
                                                     uint32_t c2, uint32_t c3,
                                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
#ifdef __CUDA_ARCH__
    const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
#else
    const uint32_t hi_a = (uint32_t)(((uint64_t)0xD2511F53u * c0) >> 32);
    const uint32_t hi_b = (uint32_t)(((uint64_t)0xCD9E8D57u * c2) >> 32);
#endif
    const uint32_t lo_a = 0xD2511F53u * c0;
    const uint32_t lo_b = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi_b ^ c1 ^ k0;
    const uint32_t n2 = hi_a ^ c3 ^ k1;
    c0 = n0;
    c1 = lo_b;
    c2 = n2;
    c3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  U4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

// Top 24 bits of a draw mapped to [0, 1): exact in float.
__host__ __device__ __forceinline__ float uniform24(uint32_t r) {
  return (float)(r >> 8) * 5.9604644775390625e-08f;  // 2^-24
}

}  // namespace slm
