// Loads and stores of B contiguous vector entries (one row of a block of B
// interleaved vectors), as 16-byte transactions where the width allows.
// stream = true marks data read once (evict-first).  ld_vec reads through the
// read-only (non-coherent) path unless streaming; ld_vec_coherent is for data the
// same kernel may have written (visible after a barrier; L2-coherent loads).
#pragma once

namespace ftlm {

template <int B> __device__ __forceinline__ void ld_vec(const float *p, float (&v)[B], bool stream)
{
    if constexpr (B % 4 == 0) {
#pragma unroll
        for (int i = 0; i < B / 4; ++i) {
            const float4 f = stream ? __ldcs(reinterpret_cast<const float4 *>(p) + i)
                                    : __ldg(reinterpret_cast<const float4 *>(p) + i);
            v[4 * i] = f.x, v[4 * i + 1] = f.y, v[4 * i + 2] = f.z, v[4 * i + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) v[i] = stream ? __ldcs(p + i) : __ldg(p + i);
    }
}
template <int B> __device__ __forceinline__ void ld_vec(const double *p, double (&v)[B], bool stream)
{
    if constexpr (B % 2 == 0) {
#pragma unroll
        for (int i = 0; i < B / 2; ++i) {
            const double2 d = stream ? __ldcs(reinterpret_cast<const double2 *>(p) + i)
                                     : __ldg(reinterpret_cast<const double2 *>(p) + i);
            v[2 * i] = d.x, v[2 * i + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) v[i] = stream ? __ldcs(p + i) : __ldg(p + i);
    }
}
template <int B> __device__ __forceinline__ void ld_vec_coherent(const float *p, float (&v)[B])
{
    if constexpr (B % 4 == 0) {
#pragma unroll
        for (int i = 0; i < B / 4; ++i) {
            const float4 f = __ldcg(reinterpret_cast<const float4 *>(p) + i);
            v[4 * i] = f.x, v[4 * i + 1] = f.y, v[4 * i + 2] = f.z, v[4 * i + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) v[i] = __ldcg(p + i);
    }
}
template <int B> __device__ __forceinline__ void ld_vec_coherent(const double *p, double (&v)[B])
{
    if constexpr (B % 2 == 0) {
#pragma unroll
        for (int i = 0; i < B / 2; ++i) {
            const double2 d = __ldcg(reinterpret_cast<const double2 *>(p) + i);
            v[2 * i] = d.x, v[2 * i + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) v[i] = __ldcg(p + i);
    }
}

template <int B> __device__ __forceinline__ void st_vec(float *p, const float (&v)[B])
{
    if constexpr (B % 4 == 0) {
#pragma unroll
        for (int i = 0; i < B / 4; ++i)
            __stcs(reinterpret_cast<float4 *>(p) + i, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) __stcs(p + i, v[i]);
    }
}
template <int B> __device__ __forceinline__ void st_vec(double *p, const double (&v)[B])
{
    if constexpr (B % 2 == 0) {
#pragma unroll
        for (int i = 0; i < B / 2; ++i) __stcs(reinterpret_cast<double2 *>(p) + i, make_double2(v[2 * i], v[2 * i + 1]));
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) __stcs(p + i, v[i]);
    }
}

}  // namespace ftlm
