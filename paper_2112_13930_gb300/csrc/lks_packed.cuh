// lks_packed.cuh -- two 16-bit populations (nodes x0, x0 + 1) in one 32-bit word, for the
// two-nodes-per-thread kernels of 16-bit deviation storage.  lo() is the element at the lower
// address (node x0), hi() the one above it, pair() both as (lo, hi); pack() rounds each value to
// nearest even, exactly as the one-element store_s does.  FP16 words hold the deviations times
// kHalfScale (lks_device.cuh), removed on the way in and applied on the way out, as the
// one-element conversions do.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lks_device.cuh"

namespace lks {

template <typename S>
struct Packed;
template <>
struct Packed<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ float2 pair(uint32_t w) { return make_float2(lo(w), hi(w)); }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    }
};
template <>
struct Packed<__half> {
    static __device__ __forceinline__ float lo(uint32_t w) {
        return __fmul_rn(__half2float(__ushort_as_half((unsigned short)(w & 0xffffu))), kHalfUnscale);
    }
    static __device__ __forceinline__ float hi(uint32_t w) {
        return __fmul_rn(__half2float(__ushort_as_half((unsigned short)(w >> 16))), kHalfUnscale);
    }
    static __device__ __forceinline__ float2 pair(uint32_t w) {
        const __half2 h = *reinterpret_cast<const __half2*>(&w);
        return __fmul2_rn(__half22float2(h), make_float2(kHalfUnscale, kHalfUnscale));
    }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const float2 s = __fmul2_rn(make_float2(a, b), make_float2(kHalfScale, kHalfScale));
        __half2 v = __floats2half2_rn(s.x, s.y);
        return *reinterpret_cast<uint32_t*>(&v);
    }
};

}  // namespace lks
