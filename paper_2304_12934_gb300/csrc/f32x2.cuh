// Packed two-lane FP32 arithmetic (the .f32x2 forms of add, sub, mul and fma
// that sm_100-family parts issue as one instruction for both halves), and the
// error-free transformations built on them.
#pragma once
#include <cuda_runtime.h>
#include <string.h>

__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
// a * b + c, one rounding per lane
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// The same with one operand given as its packed 64-bit pattern (a kernel
// parameter holding two floats), which the compiler can read in place.
__device__ __forceinline__ float2 fma2k(float2 a, unsigned long long b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(b), "l"(f2_pack(c)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 fma2kk(float2 a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(b), "l"(c));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 add2k(float2 a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(b));
    return f2_unpack(r);
}
// host: the packed pattern of (v, v)
__host__ __device__ inline unsigned long long pack_splat(float v) {
    unsigned int u;
    memcpy(&u, &v, 4);
    return ((unsigned long long)u << 32) | u;
}

// Knuth's TwoSum per lane: s + err == a + b exactly (round to nearest, no
// overflow), whatever the magnitudes of a and b.
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2 &err) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    err = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
    return s;
}

// Compensated accumulator of exact terms p + e per lane (Neumaier/Kahan-Babuska
// with the term's own low part): after n additions the represented sum s + c
// is within about 2 u |sum| + n u^2 sum|terms| of the exact sum (u = 2^-24),
// as good as an FP64 sum of the same terms for the sizes used here.
struct Acc2 {
    float2 s, c;
    __device__ __forceinline__ void zero() { s = c = make_float2(0.f, 0.f); }
    // add the term p + e (e the rounding error of p, or zero)
    __device__ __forceinline__ void add(float2 p, float2 e) {
        float2 err;
        s = two_sum2(s, p, err);
        c = add2(c, add2(err, e));
    }
    __device__ __forceinline__ double total() const {
        return ((double)s.x + (double)c.x) + ((double)s.y + (double)c.y);
    }
};
