// lb_vec.cuh -- arithmetic on one cell (float) or on two neighbouring cells at once (float2).
//
// The per-cell physics in lb_cell.cuh is written once, as templates over T = float or float2.
// For float2 every operation maps to the paired FP32 instructions of sm_100-class GPUs
// (add/sub/mul/fma .f32x2: two IEEE FP32 operations per thread per instruction), so a thread
// that owns two cells issues one instruction where the scalar code issues two.  Each lane is
// rounded like the scalar operation, except that the compiler may fuse a paired product with
// the paired sum that consumes it (measured on GB300: it does so for a product followed by a
// difference), so the two forms agree to FP32 rounding rather than bitwise.
#pragma once
#include <cuda_runtime.h>

namespace vlb {
namespace vec {

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
          "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
}
__device__ __forceinline__ float2 operator*(float s, float2 b) { return __fmul2_rn(make_float2(s, s), b); }
__device__ __forceinline__ float2 operator*(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 operator+(float2 a, float s) { return __fadd2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 operator+(float s, float2 b) { return __fadd2_rn(make_float2(s, s), b); }
__device__ __forceinline__ float2 operator-(float2 a, float s) { return a - make_float2(s, s); }
__device__ __forceinline__ float2 operator-(float s, float2 b) { return make_float2(s, s) - b; }
__device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }

// fused multiply-add a * b + c, rounded once (per lane)
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float a, float2 b, float2 c) { return __ffma2_rn(make_float2(a, a), b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float b, float2 c) { return __ffma2_rn(a, make_float2(b, b), c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float c) { return __ffma2_rn(a, b, make_float2(c, c)); }
__device__ __forceinline__ float2 vfma(float a, float2 b, float c) { return __ffma2_rn(make_float2(a, a), b, make_float2(c, c)); }

// broadcast of a scalar
template <class T>
__device__ __forceinline__ T bc(float s);
template <>
__device__ __forceinline__ float bc<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 bc<float2>(float s) { return make_float2(s, s); }

// correctly rounded reciprocal (per lane)
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }

// lane access
__device__ __forceinline__ float lane(float a, int) { return a; }
__device__ __forceinline__ float lane(float2 a, int k) { return k ? a.y : a.x; }
template <class T>
struct Lanes;
template <>
struct Lanes<float> {
    static constexpr int N = 1;
};
template <>
struct Lanes<float2> {
    static constexpr int N = 2;
};

}  // namespace vec
}  // namespace vlb
