// philox.cuh -- Philox4x32-10 for the device, written from Salmon, Moraes, Dror,
// Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): ten rounds, each
// two 32x32->64 products (multipliers 0xD2511F53, 0xCD9E8D57) whose halves are
// xor-ed with the other words and the round key; the key is bumped by the Weyl
// constants (0x9E3779B9, 0xBB67AE85) between rounds.
#pragma once
#include <stdint.h>

namespace snn {

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// 24-bit uniform in [0, 1): (u >> 8) * 2^-24, exact in float.
__device__ __forceinline__ float unit24(uint32_t u) {
    return __fmul_rn(__uint2float_rn(u >> 8), 5.9604644775390625e-08f);
}

}  // namespace snn
