// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Section 4.2), written
// from its published definition: ten rounds of two 32x32->64 multiplies with
// the key bumped by the Weyl constants between rounds.
#pragma once
#include <cstdint>

namespace rutv {

struct U4 { uint32_t x0, x1, x2, x3; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c.x0), lo0 = M0 * c.x0;
    uint32_t hi1 = __umulhi(M1, c.x2), lo1 = M1 * c.x2;
    c = U4{hi1 ^ c.x1 ^ k0, lo1, hi0 ^ c.x3 ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

}  // namespace rutv
