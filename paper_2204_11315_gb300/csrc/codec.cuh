// codec.cuh -- fixed-rate block codec, device side.
//
// The paper streams chunks through a fixed-rate transform codec (cuZFP, Sec. 4.2,
// "customized compression rate"; Sec. 5: 32 bits per double, ratio 1/2).  This
// is this project's own implementation of that kind of codec, following the
// published ZFP method (Lindstrom, IEEE TVCG 2014) with a bitstream of its own.
// One 4x4x4 block of FP32 values (index i + 4j + 16k for (x,y,z) = (i,j,k)) is
// coded into exactly 64*rate bits = 2*rate little-endian 32-bit words:
//
//   bits 0..7   header h: 0 = all-zero block, else emax + 127, where emax is
//               the largest frexp exponent in the block clamped to >= -95
//   bits 8..    embedded bit planes 31..0 of the 64 transform coefficients
//               (negabinary, sequency order) with group testing, cut at the
//               rate budget and zero padded.
//
// The stages are: quantise q = trunc(v * 2^(29-emax)); 4-point lifting along
// x, y, z; order by (i+j+k, i^2+j^2+k^2, index); negabinary; plane coding.
// Decoding inverts them and returns RN(q) * 2^(emax-29).
//
// GPU design: one thread codes one block.  Bit planes are formed by two 32x32
// bit-matrix transposes (no per-bit loop); the plane loop stays rolled (its 64
// words live in the thread's local memory: unrolling it 32 times overflowed
// the instruction cache, and per-thread columns of shared memory cost the
// decoder its L1), and each plane is emitted in closed form: the verbatim
// part is one masked word, and all of the plane's group-test tokens are built
// as one string of at most 127 bits and written with one or two puts.  The
// string is the plane's new bits with every one doubled, which a 256-entry
// table in shared memory gives a byte at a time (a lookup per byte instead
// of a loop step per new one: 11-17 % less encode time on heat-smoothed
// fields, whose planes gain many coefficients at once).
// A block holding an infinity or a NaN is coded as an all-zero block and
// reported to the caller (encode_block returns false).
#pragma once
#include <stdint.h>

#include <type_traits>

#include "devmath.cuh"

namespace oocs {

constexpr uint32_t kNegaMask = 0xAAAAAAAAu;

// compile-time loop: f(integral_constant<int, I>) for I = B .. E-1
template <int B, int E, class F>
OOCS_FN void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// Sequency order, built at compile time by enumerating the keys in increasing
// order (i+j+k from 0 to 9, then i^2+j^2+k^2 from 0 to 27, then the index).
struct SeqTable {
    int v[64];
};

constexpr SeqTable make_seq_table()
{
    SeqTable t{};
    int n = 0;
    for (int s = 0; s <= 9; ++s)
        for (int q = 0; q <= 27; ++q)
            for (int idx = 0; idx < 64; ++idx) {
                int i = idx & 3, j = (idx >> 2) & 3, k = idx >> 4;
                if (i + j + k == s && i * i + j * j + k * k == q)
                    t.v[n++] = idx;
            }
    return t;
}

template <int I>
constexpr int kSeq = make_seq_table().v[I];

// ---------------------------------------------------------------- transform --

// 32-bit two's complement arithmetic with defined wrap-around (valid data never
// wraps: three guard bits keep every lifting value below 2^30 in magnitude).
OOCS_FN int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
OOCS_FN int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }
OOCS_FN int32_t wdbl(int32_t a) { return (int32_t)((uint32_t)a << 1); }

// The method's forward 4-point decorrelating lift (exact rational form
// (1/16)[4 4 4 4; 5 1 -1 -5; -4 4 4 -4; -2 6 -6 2]); >> is floor halving.
OOCS_FN void lift_fwd(int32_t &a, int32_t &b, int32_t &c, int32_t &d)
{
    a = wadd(a, d) >> 1;
    d = wsub(d, a);
    c = wadd(c, b) >> 1;
    b = wsub(b, c);
    a = wadd(a, c) >> 1;
    c = wsub(c, a);
    d = wadd(d, b) >> 1;
    b = wsub(b, d);
    d = wadd(d, b >> 1);
    b = wsub(b, d >> 1);
}

OOCS_FN void lift_inv(int32_t &a, int32_t &b, int32_t &c, int32_t &d)
{
    b = wadd(b, d >> 1);
    d = wsub(d, b >> 1);
    b = wadd(b, d);
    d = wsub(wdbl(d), b);
    c = wadd(c, a);
    a = wsub(wdbl(a), c);
    b = wadd(b, c);
    c = wsub(wdbl(c), b);
    d = wadd(d, a);
    a = wsub(wdbl(a), d);
}

OOCS_FN void xform_fwd(int32_t (&q)[64])
{
#pragma unroll
    for (int l = 0; l < 16; ++l)  // x lines: (j, k) = (l & 3, l >> 2)
        lift_fwd(q[4 * l + 0], q[4 * l + 1], q[4 * l + 2], q[4 * l + 3]);
#pragma unroll
    for (int l = 0; l < 16; ++l) {  // y lines: (i, k) = (l & 3, l >> 2)
        const int o = (l & 3) + 16 * (l >> 2);
        lift_fwd(q[o + 0], q[o + 4], q[o + 8], q[o + 12]);
    }
#pragma unroll
    for (int l = 0; l < 16; ++l)  // z lines: (i, j) = (l & 3, l >> 2)
        lift_fwd(q[l + 0], q[l + 16], q[l + 32], q[l + 48]);
}

OOCS_FN void xform_inv(int32_t (&q)[64])
{
#pragma unroll
    for (int l = 0; l < 16; ++l)
        lift_inv(q[l + 0], q[l + 16], q[l + 32], q[l + 48]);
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        const int o = (l & 3) + 16 * (l >> 2);
        lift_inv(q[o + 0], q[o + 4], q[o + 8], q[o + 12]);
    }
#pragma unroll
    for (int l = 0; l < 16; ++l)
        lift_inv(q[4 * l + 0], q[4 * l + 1], q[4 * l + 2], q[4 * l + 3]);
}

// In-place 32x32 bit-matrix transpose: afterwards bit i of a[p] is what bit p
// of a[i] was.  Five block-swap levels; the 16- and 8-bit levels move whole
// bytes (one byte permute per word), the 4-, 2- and 1-bit levels use masked
// xor swaps.
OOCS_FN void transpose32(uint32_t (&a)[32])
{
#pragma unroll
    for (int k = 0; k < 16; ++k) {  // swap 16-bit halves of rows k and k+16
        const uint32_t lo = prmt(a[k], a[k + 16], 0x5410);
        const uint32_t hi = prmt(a[k], a[k + 16], 0x7632);
        a[k] = lo;
        a[k + 16] = hi;
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {  // swap bytes of rows k and k+8
        if ((k & 8) == 0 && k < 24) {
            const uint32_t lo = prmt(a[k], a[k + 8], 0x6240);
            const uint32_t hi = prmt(a[k], a[k + 8], 0x7351);
            a[k] = lo;
            a[k + 8] = hi;
        }
    }
    uint32_t m = 0x0F0F0F0Fu;
#pragma unroll
    for (int j = 4; j != 0; j >>= 1, m ^= (m << j)) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if ((k & j) == 0) {
                uint32_t t = ((a[k] >> j) ^ a[k + j]) & m;
                a[k] ^= t << j;
                a[k + j] ^= t;
            }
        }
    }
}

OOCS_FN uint64_t low_mask64(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// ----------------------------------------------------------------- bit I/O --

template <class Sink>
struct BitWriter {
    Sink &sink;
    int nwords;
    uint64_t acc = 0;
    int nacc = 0;
    int widx = 0;

    OOCS_FN BitWriter(Sink &s, int nw) : sink(s), nwords(nw) {}

    // append the low n bits of `bits`, n in [0, 32]
    OOCS_FN void put(uint32_t bits, int n)
    {
        if (n < 32)
            bits &= (1u << n) - 1u;
        acc |= (uint64_t)bits << nacc;
        nacc += n;
        if (nacc >= 32) {
            sink(widx++, (uint32_t)acc);
            acc >>= 32;
            nacc -= 32;
        }
    }
    OOCS_FN void put64(uint64_t bits, int n)  // n in [0, 64]
    {
        if (n > 32) {
            put((uint32_t)bits, 32);
            put((uint32_t)(bits >> 32), n - 32);
        } else {
            put((uint32_t)bits, n);
        }
    }
    OOCS_FN void finish()
    {
        if (nacc > 0)
            sink(widx++, (uint32_t)acc);
        while (widx < nwords)
            sink(widx++, 0u);
    }
};

template <class Src>
struct BitReader {
    Src &src;
    uint64_t win = 0;   // unread bits, least significant first
    int nwin = 0;       // valid bits in win
    int ridx = 0;       // index of n0
    uint32_t n0, n1, n2, n3;  // the next four words, loaded ahead so that a
                              // refill seldom waits for a load

    OOCS_FN explicit BitReader(Src &s) : src(s)
    {
        n0 = src(0);
        n1 = src(1);
        n2 = src(2);
        n3 = src(3);
    }
    OOCS_FN void fill()
    {
        if (nwin < 32) {
            win |= (uint64_t)n0 << nwin;
            nwin += 32;
            n0 = n1;
            n1 = n2;
            n2 = n3;
            n3 = src(++ridx + 3);
        }
    }
    OOCS_FN uint32_t peek(int n)  // n in [1, 32]
    {
        fill();
        uint32_t v = (uint32_t)win;
        return n < 32 ? (v & ((1u << n) - 1u)) : v;
    }
    OOCS_FN void skip(int n)  // n in [0, 32]
    {
        fill();
        win >>= n;
        nwin -= n;
    }
    OOCS_FN uint32_t get(int n)  // n in [0, 32]; one refill check
    {
        fill();
        const uint32_t v = (uint32_t)(win & ((1ull << n) - 1ull));
        win >>= n;
        nwin -= n;
        return v;
    }
    OOCS_FN uint64_t get64(int n)  // n in [0, 64]
    {
        if (n > 32) {
            uint64_t lo = get(32);
            return lo | ((uint64_t)get(n - 32) << 32);
        }
        return get(n);
    }
};

// ------------------------------------------------------------------- codec --

// The doubling table of encode_block: entry c holds byte c with each one
// doubled ("1" -> "11", least significant bit first) in bits 0..15 and that
// string's length, 8 + popcount(c), in bits 16..31.  Filled by the threads of
// a CTA (index tid of nthreads) into shared memory before encoding.
OOCS_FN void fill_doubling_table(uint32_t *t, int tid, int nthreads)
{
    for (int c = tid; c < 256; c += nthreads) {
        uint32_t d = 0;
        int o = 0;
        for (int j = 0; j < 8; ++j) {
            if ((c >> j) & 1) {
                d |= 3u << o;
                o += 2;
            } else {
                o += 1;
            }
        }
        t[c] = d | ((uint32_t)o << 16);
    }
}

// Encode one block.  sink(word_index, word) receives words 0 .. 2*rate-1 in
// order; dbl is the doubling table (fill_doubling_table).  Returns false for
// a block holding an infinity or a NaN, which is written as an all-zero block
// (the codec is defined for finite values).
template <class Sink>
OOCS_FN bool encode_block(const float (&v)[64], int rate, const uint32_t *dbl, Sink &&sink)
{
    const int nwords = 2 * rate;
    uint32_t mag = 0;
#pragma unroll
    for (int i = 0; i < 64; ++i)
        mag = max(mag, f32_bits(v[i]) & 0x7FFFFFFFu);
    BitWriter<Sink> bw(sink, nwords);
    if (mag == 0 || mag >= 0x7F800000u) {
        bw.finish();
        return mag == 0;
    }
    // emax = max(biased - 126, -95); header = emax + 127
    const int hdr = max((int)(mag >> 23), 31) + 1;
    const int emax = hdr - 127;
    const float scale = bits_f32((uint32_t)(156 - emax) << 23);  // 2^(29 - emax)

    int32_t q[64];
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        q[i] = f2i_rz(fmul_rn(v[i], scale));
        any |= (uint32_t)q[i];
    }
    if (any == 0) {
        // only a block clamped at emax = -95 (all |v| < 2^-124) quantises to
        // zero: every plane is one group-test 0, which the zero padding writes
        bw.put((uint32_t)hdr, 8);
        bw.finish();
        return true;
    }
    xform_fwd(q);

    uint32_t lo[32], hi[32];  // negabinary coefficients in sequency order
    static_for<0, 64>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const uint32_t u = ((uint32_t)q[kSeq<i>] + kNegaMask) ^ kNegaMask;
        if constexpr (i < 32)
            lo[i] = u;
        else
            hi[i - 32] = u;
    });
    transpose32(lo);  // lo[p] / hi[p]: plane p of coefficients 0..31 / 32..63
    transpose32(hi);

    bw.put((uint32_t)hdr, 8);
    int left = 64 * rate - 8;
    int n = 0;  // leading coefficients already significant
    for (int p = 31; p >= 0 && left > 0; --p) {
        const uint64_t X = ((uint64_t)hi[p] << 32) | lo[p];
        const int t = min(n, left);
        bw.put64(X, t);  // verbatim bits of the significant coefficients
        left -= t;
        if (t < n || left == 0)  // the budget ended inside (or right after) them
            break;
        if (n == 64)  // every coefficient significant: the plane is all verbatim
            continue;
        const uint64_t Y = X >> n;  // the bits of coefficients n .. 63
        if (Y == 0) {  // group test 0: nothing new in this plane
            bw.put(0u, 1);
            --left;
            continue;
        }
        // The plane's group-test tokens as one string.  With f_1 < .. < f_k
        // the window positions of Y's ones, the tokens are a leading 1 (the
        // first group test), then for each one its zeros and itself, followed
        // by a 1 (the next group test) except after the last, which a 0 (the
        // final group test) follows.  After the leading 1 the string is
        // therefore Y's bits from 0 to f_k with every one doubled (U), cut
        // after the last one (whose group-test 1 is dropped), then the final
        // 0.  When the last one is coefficient 63 it is implied: neither it
        // nor the final 0 is sent.  U has at most 127 bits, built a byte of Y
        // at a time from the doubling table.
        const int fk = 63 - clz64(Y);  // window position of the last new one
        const int k = __popcll(Y);     // new ones
        uint64_t ulo = 0, uhi = 0;
        {
            int off = 0;
            const int nb = (fk >> 3) + 1;
            for (int i = 0; i < nb; ++i) {
                const uint32_t e = dbl[(uint32_t)(Y >> (8 * i)) & 0xFFu];
                const uint64_t d = e & 0xFFFFu;
                if (off < 64) {
                    ulo |= d << off;
                    if (off > 48)
                        uhi |= d >> (64 - off);
                } else {
                    uhi |= d << (off - 64);
                }
                off += (int)(e >> 16);
            }
        }
        const bool implied = n + fk == 63;
        const int keep = fk + k + (implied ? 0 : 1);  // bits of the string before its tail
        const int len = implied ? keep : keep + 1;    // + the final group-test 0
        uint64_t tlo = 1ull | (ulo << 1);
        uint64_t thi = (uhi << 1) | (ulo >> 63);
        if (keep < 64) {
            tlo &= (1ull << keep) - 1ull;
            thi = 0;
        } else if (keep < 128) {
            thi &= (1ull << (keep - 64)) - 1ull;
        }
        const int w = min(len, left);  // the budget may cut the string
        if (w > 64) {
            bw.put64(tlo, 64);
            bw.put64(thi, w - 64);
        } else {
            bw.put64(tlo, w);
        }
        left -= w;
        n += fk + 1;
    }
    bw.finish();
    return true;
}

// Decode one block.  src(word_index) returns word i of the block (0 past the end).
template <class Src>
OOCS_FN void decode_block(int rate, Src &&src, float (&v)[64])
{
    const uint32_t w0 = src(0);
    const int hdr = (int)(w0 & 0xFFu);
    if (hdr == 0) {
#pragma unroll
        for (int i = 0; i < 64; ++i)
            v[i] = 0.0f;
        return;
    }
    const int emax = max(hdr, 32) - 127;  // headers 1..31 are never written: clamp as the encoder does
    if ((w0 >> 8) == 0u && (src(1) & 0xFFu) == 0u) {
        // bits 8..39 zero: each of the 32 planes is a group-test 0 with no
        // significant coefficient (the budget holds >= 56 bits), so every
        // coefficient is 0 and every value +0
#pragma unroll
        for (int i = 0; i < 64; ++i)
            v[i] = 0.0f;
        return;
    }
    BitReader<Src> br(src);
    br.skip(8);

    uint32_t lo[32], hi[32];
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        lo[p] = 0u;
        hi[p] = 0u;
    }
    int left = 64 * rate - 8;
    int n = 0;
    for (int p = 31; p >= 0 && left > 0; --p) {
        const int t = min(n, left);
        uint64_t X = br.get64(t);
        left -= t;
        if (t == n) {
            while (n < 64 && left > 0) {
                br.fill();  // >= 32 valid bits
                const uint32_t w = (uint32_t)br.win;
                if (!(w & 1u)) {  // group test 0: plane done
                    br.win >>= 1;
                    br.nwin -= 1;
                    --left;
                    break;
                }
                {
                    // fast path: the whole token lies in the 31 bits after the
                    // group-test bit and inside the budget
                    const int lim0 = 63 - n;
                    const uint32_t after = w >> 1;
                    const int z0 = after ? ctz32(after) : 32;
                    if (z0 < lim0 && z0 < 31 && z0 + 2 <= left) {
                        br.win >>= z0 + 2;
                        br.nwin -= z0 + 2;
                        left -= z0 + 2;
                        X |= 1ull << (n + z0);
                        n += z0 + 1;
                        continue;
                    }
                    if (z0 >= lim0 && lim0 < 31 && lim0 + 1 <= left) {  // the implied last one
                        br.win >>= lim0 + 1;
                        br.nwin -= lim0 + 1;
                        left -= lim0 + 1;
                        X |= 1ull << 63;
                        n = 64;
                        continue;
                    }
                }
                br.skip(1);  // general path: consume the group-test 1
                --left;
                const int lim = 63 - n;  // zeros possible before the implied last one
                const int avail = min(lim, left);
                int z = 0;
                bool found = false;
                while (z < avail) {
                    const int c = min(32, avail - z);
                    const uint32_t w = br.peek(c);
                    if (w) {
                        const int o = ctz32(w);
                        br.skip(o + 1);
                        z += o;
                        found = true;
                        break;
                    }
                    br.skip(c);
                    z += c;
                }
                if (found) {
                    left -= z + 1;
                    X |= 1ull << (n + z);
                    n += z + 1;
                } else {
                    left -= z;
                    if (z == lim) {
                        X |= 1ull << 63;
                        n = 64;
                    }
                }
            }
        }
        lo[p] = (uint32_t)X;
        hi[p] = (uint32_t)(X >> 32);
    }
    transpose32(lo);  // back to coefficient words
    transpose32(hi);

    int32_t q[64];
    static_for<0, 64>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const uint32_t u = (i < 32) ? lo[i & 31] : hi[i & 31];
        q[kSeq<i>] = (int32_t)((u ^ kNegaMask) - kNegaMask);
    });
    xform_inv(q);
    const float scale = bits_f32((uint32_t)(98 + emax) << 23);  // 2^(emax - 29)
#pragma unroll
    for (int i = 0; i < 64; ++i)
        v[i] = fmul_rn(i2f_rn(q[i]), scale);
}

}  // namespace oocs
