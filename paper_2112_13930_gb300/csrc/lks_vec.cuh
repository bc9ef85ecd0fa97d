// lks_vec.cuh -- arithmetic on one node (double, float) or on two nodes at once (float2), for
// collision code written once for all three.  float2 uses the packed FP32 instructions of sm_100
// and later (add, mul, fma on .f32x2): each half is rounded exactly as the scalar float operation,
// so a node gets the same bits whether it is computed alone or in a pair.  Every operation is an
// explicit, individually rounded one: the compiler has nothing to contract.
#pragma once
#include <cuda_runtime.h>

#include "lks_device.cuh"

namespace lks {

__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double vneg(double a) { return -a; }
__device__ __forceinline__ double vrecip(double a) { return recip(a); }

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vrecip(float a) { return recip(a); }

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as b * (-1) + a: the product is exact, so the one rounding is that of a - b
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vrecip(float2 a) { return make_float2(recip(a.x), recip(a.y)); }

// A constant of the scalar type S in the vector type V.
template <typename V> struct VecOf;
template <> struct VecOf<double> {
    static __device__ __forceinline__ double set(double c) { return c; }
};
template <> struct VecOf<float> {
    static __device__ __forceinline__ float set(float c) { return c; }
};
template <> struct VecOf<float2> {
    static __device__ __forceinline__ float2 set(float c) { return make_float2(c, c); }
};

}  // namespace lks
