// Packed FP32x2 arithmetic (sm_100+: add/sub/mul/fma.rn.f32x2) for kernels in
// which one thread carries two lattice sites: component .x belongs to the
// first site, .y to the second, and every operation acts on both at once
// with the rounding of the scalar FP32 operation.  Nothing is contracted
// implicitly: a multiply-add is written as fma().
#pragma once

#include <cuda_runtime.h>

namespace lbm {
namespace px {

struct P {
    float2 v;
    __device__ __forceinline__ P() {}
    __device__ __forceinline__ explicit P(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ P(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ P(float2 w) : v(w) {}
    __device__ __forceinline__ float a() const { return v.x; }
    __device__ __forceinline__ float b() const { return v.y; }
};

__device__ __forceinline__ P operator+(P x, P y) { return P(__fadd2_rn(x.v, y.v)); }
__device__ __forceinline__ P operator*(P x, P y) { return P(__fmul2_rn(x.v, y.v)); }
__device__ __forceinline__ P operator-(P x, P y) {
    unsigned long long r;
    const unsigned long long a = *reinterpret_cast<const unsigned long long*>(&x.v);
    const unsigned long long b = *reinterpret_cast<const unsigned long long*>(&y.v);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return P(*reinterpret_cast<const float2*>(&r));
}
__device__ __forceinline__ P& operator+=(P& x, P y) { return x = x + y; }
__device__ __forceinline__ P& operator-=(P& x, P y) { return x = x - y; }
// x * y + z, rounded once per component
__device__ __forceinline__ P fma(P x, P y, P z) { return P(__ffma2_rn(x.v, y.v, z.v)); }
// z - x * y, rounded once per component (x * y negated exactly)
__device__ __forceinline__ P fms(P x, P y, P z) { return P(__ffma2_rn(make_float2(-x.v.x, -x.v.y), y.v, z.v)); }
// 1/x per component, correctly rounded
__device__ __forceinline__ P recip(P x) { return P(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }

}  // namespace px
}  // namespace lbm
