// Counter-based start vectors: splitmix64 (Steele, Lea & Flood 2014) as a
// counter-based generator, Box-Muller for Gaussian entries.  The definition is the
// one stated for ftlm_lanczos in include/ftlm.h.
#pragma once

#include <cstdint>

#include "ftlm.h"

namespace ftlm {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t chain_key(uint64_t seed, int N, int K, uint32_t r)
{
    const uint64_t tag = ((uint64_t)N << 48) | ((uint64_t)K << 32) | (uint64_t)r;
    return sm64_mix(sm64_mix(seed + kGamma) + tag + kGamma);
}

__device__ __forceinline__ double start_value(uint64_t key, uint64_t t, int dist)
{
    if (dist == FTLM_VEC_RADEMACHER) {
        const uint64_t u = sm64_mix(key + (t + 1) * kGamma);
        return (u >> 63) ? -1.0 : 1.0;
    }
    const uint64_t u1 = sm64_mix(key + (2 * t + 1) * kGamma);
    const uint64_t u2 = sm64_mix(key + (2 * t + 2) * kGamma);
    const double U1 = ((double)(u1 >> 11) + 1.0) * 0x1p-53;
    const double U2 = (double)(u2 >> 11) * 0x1p-53;
    const double two_pi = 2.0 * 3.14159265358979323846;
    return sqrt(-2.0 * log(U1)) * cos(two_pi * U2);
}

}  // namespace ftlm
