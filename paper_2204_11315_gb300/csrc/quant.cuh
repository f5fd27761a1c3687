// quant.cuh -- the block quantiser, device side.
//
// The simpler fixed-rate codec that a comparison of compression libraries
// (Sec. 7, future work (1)) sets against the transform codec of codec.cuh:
// the same 4x4x4 block (index i + 4j + 16k) and the same 64*rate bits, so
// stores, slots and the scheduler do not change.  Bits are numbered from bit
// 0 of word 0 upwards:
//
//   bits 0..7   header: 0 = all-zero block, else emax + 127 with
//               emax = max(frexp exponent of max|v|, -126), so max|v| < 2^emax
//   then        64 values of q = rate - 1 bits, in block index order, each the
//               two's complement of n = clamp(rint(v 2^(q-1-emax)), +-(2^(q-1)-1))
//   last 56     zero
//
// Decoding returns RN(RN(n) 2^(emax-q+1)).  No transform, no bit planes: a
// value costs a few integer operations, so the kernels move bytes rather than
// issue instructions.  Rate in [2, 32]; a block with an infinity or a NaN
// is written as an all-zero block and reported (bq_encode_block returns false).
//
// Exact scaling in FP32: 2^s with |s| up to 156 is not a float, so it is
// applied as two factors 2^(s/2) and 2^(s - s/2), each a normal float.
// Encoding, the product only grows (s >= 0) or shrinks (s < 0) monotonically;
// an intermediate that falls below the normal range ends in a value of
// magnitude < 2^-126, which rounds to the integer 0 either way.  Decoding,
// |RN(n)| is in [1, 2^30] and the first factor is >= 2^-78, so the first
// product is exact and the second is the only rounding.
#pragma once
#include <stdint.h>

#include "devmath.cuh"

namespace oocs {

// 2^e as a float for e in [-126, 127] (built from its exponent bits)
OOCS_FN float pow2f(int e) { return bits_f32((uint32_t)(e + 127) << 23); }

// v 2^s exactly (or to 0 when the result is below the normal range)
OOCS_FN float scale2(float v, int s)
{
    const int s1 = s / 2;  // truncation: |s1|, |s - s1| <= 78
    return fmul_rn(fmul_rn(v, pow2f(s1)), pow2f(s - s1));
}

// Emit(i, word) receives the 2*rate words in order i = 0 .. 2*rate-1.
// Returns false for a block holding an infinity or a NaN, which is written as
// an all-zero block (the same rule as the transform codec).
template <class Emit>
OOCS_FN bool bq_encode_block(const float (&v)[64], int rate, Emit &&emit)
{
    uint32_t mbits = 0;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        const uint32_t a = f32_bits(v[j]) & 0x7fffffffu;
        mbits = a > mbits ? a : mbits;
    }
    const int nw = 2 * rate;
    if (mbits == 0 || mbits >= 0x7f800000u) {
#pragma unroll 1
        for (int i = 0; i < nw; ++i)
            emit(i, 0u);
        return mbits == 0;
    }
    // biased exponent E of max|v|: frexp exponent E - 126 (normal), clamped to -126
    const int be = (int)(mbits >> 23);
    const int emax = (be > 0 ? be : 0) - 126;
    const int q = rate - 1;
    const int s = q - 1 - emax;
    const int lim = (int)((1u << (q - 1)) - 1u);
    const uint32_t mask = (1u << q) - 1u;
    uint64_t acc = (uint64_t)(emax + 127);
    int nbits = 8, wi = 0;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        int n = __float2int_rn(scale2(v[j], s));
        n = n > lim ? lim : (n < -lim ? -lim : n);
        acc |= (uint64_t)((uint32_t)n & mask) << nbits;
        nbits += q;
        if (nbits >= 32) {
            emit(wi++, (uint32_t)acc);
            acc >>= 32;
            nbits -= 32;
        }
    }
    // 8 + 64 q = 64 rate - 56 bits: at most one partial word, then zeros
    if (nbits > 0)
        emit(wi++, (uint32_t)acc);
#pragma unroll 1
    for (; wi < nw; ++wi)
        emit(wi, 0u);
    return true;
}

// Read(i) returns word i (i < 2*rate).
template <class Read>
OOCS_FN void bq_decode_block(int rate, Read &&read, float (&v)[64])
{
    const uint32_t w0 = read(0);
    const int hdr = (int)(w0 & 0xffu);
    if (hdr == 0) {
#pragma unroll
        for (int j = 0; j < 64; ++j)
            v[j] = 0.0f;
        return;
    }
    const int q = rate - 1;
    const int e = hdr - 127 - q + 1;
    const uint32_t mask = (1u << q) - 1u;
    uint64_t acc = (uint64_t)(w0 >> 8);
    int have = 24, ri = 1;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        if (have < q) {
            acc |= (uint64_t)read(ri++) << have;
            have += 32;
        }
        const uint32_t u = (uint32_t)acc & mask;
        acc >>= q;
        have -= q;
        const int n = (int)(u << (32 - q)) >> (32 - q);  // sign-extend the q-bit field
        v[j] = scale2(i2f_rn(n), e);
    }
}

}  // namespace oocs
