// Packed FP32x2 arithmetic (sm_100 family: add/sub/mul/fma.rn.f32x2): two
// independent FP32 operations in one instruction, each lane rounded as its
// scalar counterpart. Written as inline PTX with explicit rounding, so the
// compiler never contracts a product and a sum into one fused operation
// (the error-free transformations of the double-float code rely on that).
#pragma once

#include <cuda_runtime.h>

namespace vl {
namespace x2 {

__device__ __forceinline__ unsigned long long pack(float2 a) {
    unsigned long long u;
    asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(a.x), "f"(a.y));
    return u;
}
__device__ __forceinline__ float2 unpack(unsigned long long u) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(u));
    return r;
}
__device__ __forceinline__ float2 add(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack(a)), "l"(pack(b)));
    return unpack(d);
}
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack(a)), "l"(pack(b)));
    return unpack(d);
}
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack(a)), "l"(pack(b)));
    return unpack(d);
}
// a * b + c with one rounding per lane
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pack(a)), "l"(pack(b)), "l"(pack(c)));
    return unpack(d);
}
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

}  // namespace x2
}  // namespace vl
