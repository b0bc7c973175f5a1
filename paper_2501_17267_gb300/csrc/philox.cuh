// philox.cuh -- Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), usable on host and device.
//
// A block of four 32-bit words is a bijective function of a 128-bit counter under a
// 64-bit key: ten rounds, each multiplying two counter words by fixed odd constants,
// mixing the high halves with the other two words and the round key, and bumping the
// key by the Weyl constants (golden ratio and sqrt(3) - 1 in 32-bit fixed point).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SG_HD __host__ __device__ __forceinline__
#else
#define SG_HD inline
#endif

namespace sg {

struct Philox4 {
    uint32_t v[4];
};

constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

SG_HD void philox_mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

// Counter (c0, c1, c2, c3), key (k0, k1).
SG_HD Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                            uint32_t k1)
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        uint32_t hA, lA, hB, lB;
        philox_mulhilo(kPhiloxMulA, c0, &hA, &lA);
        philox_mulhilo(kPhiloxMulB, c2, &hB, &lB);
        const uint32_t n0 = hB ^ c1 ^ k0;
        const uint32_t n2 = hA ^ c3 ^ k1;
        c0 = n0;
        c1 = lB;
        c2 = n2;
        c3 = lA;
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    Philox4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

// Counter domains (fourth counter word) and the reserved sweep value for the
// initial state.
constexpr uint32_t kDomainMetropolis = 0;
constexpr uint32_t kDomainExchange = 1;
constexpr uint32_t kDomainGenerate = 2;
constexpr uint32_t kDomainGauge = 3;
constexpr uint32_t kDomainTail = 4;  // low 24 bits of a Metropolis draw, counter (site, sweep, word, 4)
constexpr uint32_t kDomainFragment = 5;  // fragment anneals, counter (centre, sweep, 8q + read/4, 5)
constexpr uint32_t kSweepInit = 0xFFFFFFFFu;

}  // namespace sg
