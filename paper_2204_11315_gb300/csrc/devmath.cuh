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
// index of the lowest set bit of a non-zero word
OOCS_FN int ctz64(uint64_t x) { return __ffsll((long long)x) - 1; }
OOCS_FN int ctz32(uint32_t x) { return __ffs((int)x) - 1; }
// byte permute: result byte i = byte (s >> 4i) & 7 of the 8-byte value (y:x)
OOCS_FN uint32_t prmt(uint32_t x, uint32_t y, uint32_t s) { return __byte_perm(x, y, s); }
