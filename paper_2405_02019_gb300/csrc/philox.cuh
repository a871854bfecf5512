// Counter-based random numbers: Philox4x64-10 (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), usable on host and device.
//
// Each of the ten rounds multiplies words 0 and 2 of the counter block by two fixed
// odd 64-bit constants; the next block is (hi(c2*M1) ^ c1 ^ k0, lo(c2*M1),
// hi(c0*M0) ^ c3 ^ k1, lo(c0*M0)); the key advances by two Weyl increments after
// every round.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define SNN_HD __host__ __device__ __forceinline__
#else
#define SNN_HD inline
#endif

namespace snn {

struct Block4 {
    uint64_t w[4];
};

SNN_HD void mul_wide(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo)
{
#if defined(__CUDA_ARCH__)
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    const unsigned __int128 p = static_cast<unsigned __int128>(a) * b;
    hi = static_cast<uint64_t>(p >> 64);
    lo = static_cast<uint64_t>(p);
#endif
}

SNN_HD Block4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull;
    constexpr uint64_t kM1 = 0xCA5A826395121157ull;
    constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull;
    constexpr uint64_t kW1 = 0xBB67AE8584CAA73Bull;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int round = 0; round < 10; ++round) {
        uint64_t h0, l0, h1, l1;
        mul_wide(kM0, c0, h0, l0);
        mul_wide(kM1, c2, h1, l1);
        const uint64_t n0 = h1 ^ c1 ^ k0;
        const uint64_t n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
        k0 += kW0;
        k1 += kW1;
    }
    return Block4{{c0, c1, c2, c3}};
}

// Stream tags: the second key word of each random stream.
constexpr uint64_t kStreamConnect = 0xC0;   // synapse sampling
constexpr uint64_t kStreamInitial = 0x1A;   // initial membrane potentials
constexpr uint64_t kStreamThalamic = 0x7A;  // thalamic Poisson counts

}  // namespace snn
