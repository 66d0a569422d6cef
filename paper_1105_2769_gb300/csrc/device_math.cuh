// Device helpers: packed FP32 pair arithmetic (sm_100+ f32x2), pair distances
// from hi/lo split coordinates, and s^(-5/2).
#pragma once

#include <cuda_runtime.h>

// ----- packed FP32x2 arithmetic (one instruction, two lanes of a float2) -----
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 f2_splat(float v) { return make_float2(v, v); }

// ----- squared distance from hi/lo split coordinates -----
// A coordinate x (FP64) is carried as x_hi = fl32(x), x_lo = fl32(x - x_hi).
// The difference (p_hi - q_hi) + (p_lo - q_lo) keeps the input's FP64
// resolution for close pairs, which plain FP32 coordinates would lose
// (side-32 boxes have an FP32 ulp of 4e-6 against pair distances ~0.5).
__device__ __forceinline__ float pair_d2_hilo(float4 ph, float4 pl, float4 qh, float4 ql) {
    float dx = (ph.x - qh.x) + (pl.x - ql.x);
    float dy = (ph.y - qh.y) + (pl.y - ql.y);
    float dz = (ph.z - qh.z) + (pl.z - ql.z);
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// s^(-5/2) for s > 0: the hardware reciprocal square root, refined by one
// Newton-Raphson step for f(y) = 1/y^2 - s (y <- y (3 - s y^2) / 2), then
// raised to the fifth power.
__device__ __forceinline__ float inv_pow52f(float s) {
    float y = rsqrtf(s);
    float sy = s * y;
    float h = fmaf(-0.5f * sy, y, 1.5f);
    y = y * h;
    float y2 = y * y;
    return y2 * y2 * y;
}

__device__ __forceinline__ double inv_pow52d(double s) {
    double y = rsqrt(s);
    double y2 = y * y;
    return y2 * y2 * y;
}

// Tile-pair item index t -> (J, K), J <= K, ordered by J descending so the
// items with the most I tiles (I <= J) come first. Items with J' > J number
// M(M+1)/2 with M = NT-1-J.
__device__ __forceinline__ void decode_pair_item(long long t, int NT, int& J, int& K) {
    long long M = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (M > 0 && M * (M + 1) / 2 > t) --M;
    while ((M + 1) * (M + 2) / 2 <= t) ++M;
    J = NT - 1 - (int)M;
    K = J + (int)(t - M * (M + 1) / 2);
}
