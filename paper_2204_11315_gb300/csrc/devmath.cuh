// devmath.cuh -- the few device intrinsics the codec and stencil arithmetic use.
//
// Every floating-point operation on the hot path goes through these explicitly
// rounded forms so that all kernel variants (in-core, streamed, fused) perform
// the same FP32 operations in the same order: the compiler may not contract a
// multiply and an add into an FMA behind our back.
#pragma once
#include <stdint.h>

#define OOCS_FN __device__ __forceinline__

OOCS_FN uint32_t f32_bits(float v) { return __float_as_uint(v); }
OOCS_FN float bits_f32(uint32_t b) { return __uint_as_float(b); }
OOCS_FN int f2i_rz(float v) { return __float2int_rz(v); }
OOCS_FN float i2f_rn(int v) { return __int2float_rn(v); }
OOCS_FN float fmul_rn(float a, float b) { return __fmul_rn(a, b); }
OOCS_FN float fadd_rn(float a, float b) { return __fadd_rn(a, b); }
OOCS_FN float fsub_rn(float a, float b) { return __fsub_rn(a, b); }
OOCS_FN float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// Packed pairs (sm_100 family f32x2 instructions): each lane of a pair is one
// IEEE round-to-nearest FP32 operation, exactly the scalar forms above.
OOCS_FN unsigned long long pk2(float2 v)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
OOCS_FN float2 upk2(unsigned long long r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
OOCS_FN float2 fadd2_rn(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
OOCS_FN float2 fsub2_rn(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
OOCS_FN float2 fmul2_rn(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
OOCS_FN float2 fma2_rn(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
    return upk2(d);
}
// index of the lowest set bit of a non-zero word
OOCS_FN int ctz64(uint64_t x) { return __ffsll((long long)x) - 1; }
OOCS_FN int ctz32(uint32_t x) { return __ffs((int)x) - 1; }
// number of leading zero bits (64 for 0)
OOCS_FN int clz64(uint64_t x) { return __clzll((long long)x); }
// byte permute: result byte i = byte (s >> 4i) & 7 of the 8-byte value (y:x)
OOCS_FN uint32_t prmt(uint32_t x, uint32_t y, uint32_t s) { return __byte_perm(x, y, s); }
