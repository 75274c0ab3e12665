// f32x2.cuh -- paired FP32 arithmetic (PTX add/sub/mul/fma .rn.f32x2, sm_100
// family).  Each half of a pair is one IEEE operation rounded to nearest, the
// same number as the scalar operation (no contraction), and one instruction
// issues both: for loops bound by instruction issue.
#pragma once

#include <cuda_runtime.h>

namespace dsps {

#ifdef __CUDACC__

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 x, y, z;\nmov.b64 x, {%2, %3};\nmov.b64 y, {%4, %5};\n"
        "add.rn.f32x2 z, x, y;\nmov.b64 {%0, %1}, z;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 x, y, z;\nmov.b64 x, {%2, %3};\nmov.b64 y, {%4, %5};\n"
        "sub.rn.f32x2 z, x, y;\nmov.b64 {%0, %1}, z;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 x, y, z;\nmov.b64 x, {%2, %3};\nmov.b64 y, {%4, %5};\n"
        "mul.rn.f32x2 z, x, y;\nmov.b64 {%0, %1}, z;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// a * b + c, each half fused (one rounding), like fmaf
__device__ __forceinline__ float2 fma2v(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n.reg .b64 x, y, z;\nmov.b64 x, {%2, %3};\nmov.b64 y, {%4, %5};\nmov.b64 z, {%6, %7};\n"
        "fma.rn.f32x2 z, x, y, z;\nmov.b64 {%0, %1}, z;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

#endif  // __CUDACC__

}  // namespace dsps
