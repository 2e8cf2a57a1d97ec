// bsd_device.cuh -- device helpers shared by the kernel files: the message
// storage formats and the per-shot status bits.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace bsd {

#define FULLMASK 0xffffffffu

// ----------------------------------------------------------------------------
// message storage: float, binary16 or bfloat16; arithmetic is always float.
// A stored value is the round-to-nearest-even conversion of the float result,
// and a zero is stored as +0 (the sign rule treats -0 as positive anyway).
// ----------------------------------------------------------------------------
template <int P> struct Store;
template <> struct Store<0> {
    using T = float;
    static __device__ __forceinline__ float ld(const T* p, size_t i) { return p[i]; }
    static __device__ __forceinline__ void st(T* p, size_t i, float v) { p[i] = v; }
    static __device__ __forceinline__ float2 ld2(const T* p, size_t i) { return *reinterpret_cast<const float2*>(p + i); }
    static __device__ __forceinline__ void st2(T* p, size_t i, float a, float b)
    {
        *reinterpret_cast<float2*>(p + i) = make_float2(a, b);
    }
};
template <> struct Store<1> {
    using T = __half;
    static __device__ __forceinline__ float ld(const T* p, size_t i) { return __half2float(p[i]); }
    static __device__ __forceinline__ void st(T* p, size_t i, float v)
    {
        __half h = __float2half_rn(v);
        if ((__half_as_ushort(h) & 0x7fffu) == 0) h = __ushort_as_half(0);
        p[i] = h;
    }
    static __device__ __forceinline__ float2 ld2(const T* p, size_t i)
    {
        return __half22float2(*reinterpret_cast<const __half2*>(p + i));
    }
    static __device__ __forceinline__ void st2(T* p, size_t i, float a, float b)
    {
        __half ha = __float2half_rn(a), hb = __float2half_rn(b);
        if ((__half_as_ushort(ha) & 0x7fffu) == 0) ha = __ushort_as_half(0);
        if ((__half_as_ushort(hb) & 0x7fffu) == 0) hb = __ushort_as_half(0);
        *reinterpret_cast<__half2*>(p + i) = __halves2half2(ha, hb);
    }
};
template <> struct Store<2> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(const T* p, size_t i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ void st(T* p, size_t i, float v)
    {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        if ((__bfloat16_as_ushort(h) & 0x7fffu) == 0) h = __ushort_as_bfloat16(0);
        p[i] = h;
    }
    static __device__ __forceinline__ float2 ld2(const T* p, size_t i)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p + i));
    }
    static __device__ __forceinline__ void st2(T* p, size_t i, float a, float b)
    {
        __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
        if ((__bfloat16_as_ushort(ha) & 0x7fffu) == 0) ha = __ushort_as_bfloat16(0);
        if ((__bfloat16_as_ushort(hb) & 0x7fffu) == 0) hb = __ushort_as_bfloat16(0);
        *reinterpret_cast<__nv_bfloat162*>(p + i) = __halves2bfloat162(ha, hb);
    }
};

// the smallest of three floats (an exact operation; no operand is NaN here)
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

enum : uint32_t { ST_SEED = 1u, ST_BEAM = 2u, ST_FAILED = 4u, ST_NEAR = 8u, ST_RERUN = 16u };

}  // namespace bsd
