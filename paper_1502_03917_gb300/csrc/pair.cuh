// pair.cuh -- the two fields (y, lambda) of a node as one value.
//
// The smoothers treat y and lambda alike, so the kernels keep the scaled
// residual as interleaved pairs and do their arithmetic on pairs: on sm_100+
// an FP32 pair is one packed instruction (add / mul / fma of float2); FP64
// pairs are two scalar operations.
#pragma once
#include <cuda_runtime.h>

namespace aaomg {

template <typename T>
struct P2;
template <>
struct P2<float> {
    using t = float2;
};
template <>
struct P2<double> {
    using t = double2;
};

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psplat(float v) { return make_float2(v, v); }

__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 psplat(double v) { return make_double2(v, v); }

template <typename T>
__device__ __forceinline__ typename P2<T>::t pmake(T a, T b) {
    typename P2<T>::t v;
    v.x = a;
    v.y = b;
    return v;
}

}  // namespace aaomg
