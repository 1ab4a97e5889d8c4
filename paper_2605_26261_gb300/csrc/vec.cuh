// Loads and stores of B contiguous vector entries (one row of a block of B
// interleaved vectors), as 32-byte transactions (the 256-bit vector loads and
// stores of sm_100 and later) where the width allows, else 16-byte ones: a 32-byte
// row (8 floats or 4 doubles) is one DRAM sector and one load instruction.  Rows
// of 32 bytes or more must be 32-byte aligned.  stream = true marks data read once
// (evict-first).  ld_vec reads through the read-only (non-coherent) path unless
// streaming; ld_vec_coherent is for data the same kernel may have written
// (visible after a barrier; L2-coherent loads).
#pragma once

// Build option: 0 restricts every row transfer to 16-byte transactions.
#ifndef FTLM_VEC256
#define FTLM_VEC256 1
#endif

namespace ftlm {

namespace v256 {
__device__ __forceinline__ void ld_nc(const float *p, float *v)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}
__device__ __forceinline__ void ld_cs(const float *p, float *v)
{
    asm volatile("ld.global.cs.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void ld_cg(const float *p, float *v)
{
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void st_cs(float *p, const float *v)
{
    asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
__device__ __forceinline__ void ld_nc(const double *p, double *v)
{
    asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
}
__device__ __forceinline__ void ld_cs(const double *p, double *v)
{
    asm volatile("ld.global.cs.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void ld_cg(const double *p, double *v)
{
    asm volatile("ld.global.cg.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void st_cs(double *p, const double *v)
{
    asm volatile("st.global.cs.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
                 : "memory");
}
}  // namespace v256

template <int B> __device__ __forceinline__ void ld_vec(const float *p, float (&v)[B], bool stream)
{
    if constexpr (FTLM_VEC256 && B % 8 == 0) {
#pragma unroll
        for (int i = 0; i < B / 8; ++i) {
            if (stream) v256::ld_cs(p + 8 * i, v + 8 * i);
            else v256::ld_nc(p + 8 * i, v + 8 * i);
        }
    } else if constexpr (B % 4 == 0) {
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
    if constexpr (FTLM_VEC256 && B % 4 == 0) {
#pragma unroll
        for (int i = 0; i < B / 4; ++i) {
            if (stream) v256::ld_cs(p + 4 * i, v + 4 * i);
            else v256::ld_nc(p + 4 * i, v + 4 * i);
        }
    } else if constexpr (B % 2 == 0) {
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
    if constexpr (FTLM_VEC256 && B % 8 == 0) {
#pragma unroll
        for (int i = 0; i < B / 8; ++i) v256::ld_cg(p + 8 * i, v + 8 * i);
    } else if constexpr (B % 4 == 0) {
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
    if constexpr (FTLM_VEC256 && B % 4 == 0) {
#pragma unroll
        for (int i = 0; i < B / 4; ++i) v256::ld_cg(p + 4 * i, v + 4 * i);
    } else if constexpr (B % 2 == 0) {
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
    if constexpr (FTLM_VEC256 && B % 8 == 0) {
#pragma unroll
        for (int i = 0; i < B / 8; ++i) v256::st_cs(p + 8 * i, v + 8 * i);
    } else if constexpr (B % 4 == 0) {
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
    if constexpr (FTLM_VEC256 && B % 4 == 0) {
#pragma unroll
        for (int i = 0; i < B / 4; ++i) v256::st_cs(p + 4 * i, v + 4 * i);
    } else if constexpr (B % 2 == 0) {
#pragma unroll
        for (int i = 0; i < B / 2; ++i) __stcs(reinterpret_cast<double2 *>(p) + i, make_double2(v[2 * i], v[2 * i + 1]));
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) __stcs(p + i, v[i]);
    }
}

}  // namespace ftlm
