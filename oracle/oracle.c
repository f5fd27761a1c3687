/*
 * oracle.c -- CPU oracle for the compressed out-of-core stencil method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path in
 * paper_2204_11315_gb300/, and the CUDA path never calls it.
 *
 * What it computes, plainly and slowly:
 *
 *   1. In-core star stencils in FP64 (Sec. 3.1 "Out-of-core stencil
 *      computation", Sec. 6 the 25-point acoustic wave code): one time step of
 *        heat (first order in time):   u' = c0 u + sum_d c_d s_d(u)
 *        wave (leapfrog, second order): u' = 2u - up + m (c0 u + sum_d c_d s_d(u) + w delta_src)
 *      where s_d(u)(p) = (u[p-d ex] + u[p+d ex]) + (u[p-d ey] + u[p+d ey])
 *                        + (u[p-d ez] + u[p+d ez]),  d = 1..r.
 *      Points within r of any face (the Dirichlet shell) keep their value.
 *
 *   2. The fixed-rate block codec the method integrates (Sec. 4.2: a
 *      transform-based fixed-rate floating-point compressor with a
 *      user-chosen rate; Sec. 5: rate 32 bits per double, i.e. ratio 1/2).
 *      The paper uses cuZFP and describes none of its internals, so this
 *      follows the published ZFP method (Lindstrom, "Fixed-Rate Compressed
 *      Floating-Point Arrays", IEEE TVCG 2014) step by step, with a bitstream
 *      of this project's own:
 *        (1) block floating point: common exponent emax of a 4x4x4 block,
 *            clamped below at CODEC_EMIN;
 *        (2) quantise: q = trunc(v * 2^(29 - emax)) as int32 (three guard bits,
 *            so no lifting step can leave int32);
 *        (3) decorrelating transform: the method's 4-point lifting transform
 *            along x, then y, then z;
 *        (4) reorder the 64 coefficients by total sequency i+j+k;
 *        (5) two's complement -> negabinary;
 *        (6) embedded bit-plane coding, most significant plane first, with
 *            group testing of not-yet-significant coefficients, stopped at
 *            exactly 64*rate bits (8 header bits included).
 *      Decoding is the inverse, with v = float(q) * 2^(emax - 29).
 *
 *   3. A plain block quantiser, the simpler fixed-rate codec the comparison of
 *      compression libraries (Sec. 7, future work (1)) sets against the
 *      transform codec.  Same 4x4x4 block, same 64*rate bits per block:
 *        header: 8 bits, 0 for an all-zero block, else emax + 127, where
 *                emax = max(frexp exponent of max|v|, -126), so max|v| < 2^emax;
 *        values: q = rate - 1 bits each, in block index order, two's
 *                complement n = clamp(rint(v 2^(q-1-emax)), -(2^(q-1)-1),
 *                2^(q-1)-1), rint rounding half to even; the last 56 bits of
 *                the block are zero.
 *      Decoding gives v = fl32(fl32(n) 2^(emax-q+1)) (round to nearest).
 *
 * Readings where the paper is silent are listed with the project design notes;
 * they are: the header is the 8-bit biased exponent emax+127 (0 = all-zero
 * block); emax is clamped to >= -95, so |v| < 2^-124 quantises to 0; the
 * sequency tie-break is (i^2+j^2+k^2, then linear index); 32 planes are coded.
 *
 * Floating point: built with -ffp-contract=off and without fast-math; all
 * stencil arithmetic is FP64.  OpenMP is used only to make the loops run on
 * all host cores; every point is computed exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(x, y, z) (((int64_t)(z) * ny + (y)) * nx + (x))

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1. star stencils, FP64                                                   */
/* ------------------------------------------------------------------------ */

/* One time step on the whole grid.
 * scheme 0 = heat: out = L(u).  scheme 1 = wave: out = 2u - up + m (L(u) + w at src).
 * coef[0..r] = [centre, c1..cr].  src = linear index of the source voxel or -1.
 * Shell points (distance < r to a face) are copied from u.               */
void oracle_star_step(int64_t nx, int64_t ny, int64_t nz, int r, const double *coef,
                      int scheme, const double *m, const double *u, const double *up,
                      double *out, int64_t src, double w)
{
    const int64_t sx = 1, sy = nx, sz = nx * ny;
    int64_t z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; z++) {
        for (int64_t y = 0; y < ny; y++) {
            for (int64_t x = 0; x < nx; x++) {
                int64_t p = IDX(x, y, z);
                int shell = x < r || y < r || z < r || x >= nx - r || y >= ny - r || z >= nz - r;
                if (shell) {
                    out[p] = u[p];
                    continue;
                }
                double L = coef[0] * u[p];
                for (int d = 1; d <= r; d++) {
                    double s = (u[p - d * sx] + u[p + d * sx]) + (u[p - d * sy] + u[p + d * sy])
                             + (u[p - d * sz] + u[p + d * sz]);
                    L += coef[d] * s;
                }
                if (scheme == 0) {
                    out[p] = L;
                } else {
                    if (p == src)
                        L += w;
                    out[p] = 2.0 * u[p] - up[p] + m[p] * L;
                }
            }
        }
    }
}

/* nsteps heat steps in place (u holds the result), scratch has the grid size. */
void oracle_heat_run(int64_t nx, int64_t ny, int64_t nz, int r, const double *coef,
                     int nsteps, double *u, double *scratch)
{
    for (int n = 0; n < nsteps; n++) {
        oracle_star_step(nx, ny, nz, r, coef, 0, NULL, u, NULL, scratch, -1, 0.0);
        memcpy(u, scratch, (size_t)(nx * ny * nz) * sizeof(double));
    }
}

/* nsteps leapfrog steps.  On entry (u, up) = (u^t, u^(t-1)); on return
 * (u, up) = (u^(t+nsteps), u^(t+nsteps-1)).  Step n (0-based) adds w[n] at src. */
void oracle_wave_run(int64_t nx, int64_t ny, int64_t nz, const double *coef, const double *m,
                     int nsteps, double *u, double *up, double *scratch, int64_t src,
                     const double *w)
{
    size_t bytes = (size_t)(nx * ny * nz) * sizeof(double);
    for (int n = 0; n < nsteps; n++) {
        oracle_star_step(nx, ny, nz, 4, coef, 1, m, u, up, scratch, src, w ? w[n] : 0.0);
        memcpy(up, u, bytes);
        memcpy(u, scratch, bytes);
    }
}

/* ------------------------------------------------------------------------ */
/* 2. fixed-rate block codec                                                */
/* ------------------------------------------------------------------------ */

#define CODEC_EMIN (-95)
#define CODEC_PLANES 32
#define NBMASK 0xAAAAAAAAu

/* (1) Block floating point.  Returns the 8-bit header: 0 for a block of
 * zeros, else emax + 127 where emax = max over the block of the frexp
 * exponent e (|v| in [2^(e-1), 2^e)), clamped to >= CODEC_EMIN.          */
int oracle_block_header(const float *v)
{
    int have = 0, emax = 0;
    for (int i = 0; i < 64; i++) {
        if (v[i] != 0.0f) {
            int e;
            frexp(fabs((double)v[i]), &e);
            if (!have || e > emax)
                emax = e;
            have = 1;
        }
    }
    if (!have)
        return 0;
    if (emax < CODEC_EMIN)
        emax = CODEC_EMIN;
    return emax + 127;
}

/* (2) q_i = trunc(v_i * 2^(29-emax)); exact in FP64, truncated toward zero. */
void oracle_quantize(const float *v, int emax, int32_t *q)
{
    double s = ldexp(1.0, 29 - emax);
    for (int i = 0; i < 64; i++)
        q[i] = (int32_t)((double)v[i] * s);
}

/* inverse of (2): v = float(q * 2^(emax-29)), one rounding to FP32 */
void oracle_dequantize(const int32_t *q, int emax, float *v)
{
    double s = ldexp(1.0, emax - 29);
    for (int i = 0; i < 64; i++)
        v[i] = (float)((double)q[i] * s);
}

/* floor(a / 2) for any sign */
static int64_t fl2(int64_t a) { return (a >= 0) ? a / 2 : -((-a + 1) / 2); }

/* The transform is defined in 32-bit two's complement arithmetic: every
 * intermediate result is reduced modulo 2^32 into [-2^31, 2^31).  Valid data
 * never wraps (three guard bits keep every value below 2^30 in magnitude);
 * the flag below records any wrap so the range tests can assert that, and the
 * rule makes the decoding of arbitrary words well defined.               */
int oracle_xform_overflow = 0;

static int64_t w32(int64_t a)
{
    int64_t r = ((a % 4294967296LL) + 4294967296LL) % 4294967296LL; /* [0, 2^32) */
    if (r >= 2147483648LL)
        r -= 4294967296LL;
    if (r != a)
        oracle_xform_overflow = 1;
    return r;
}

/* (3) The method's forward 4-point lifting transform on (a, b, c, d).
 * Exact rational form (before floor rounding):
 *   a' = ( 4a + 4b + 4c + 4d)/16     b' = ( 5a +  b -  c - 5d)/16
 *   c' = (-4a + 4b + 4c - 4d)/16     d' = (-2a + 6b - 6c + 2d)/16
 * realised as averaging/differencing lifting steps with floor halving.    */
static void fwd_lift(int32_t *p, int stride)
{
    int64_t a = p[0], b = p[stride], c = p[2 * stride], d = p[3 * stride];
    a = fl2(w32(a + d)); d = w32(d - a);        /* pair (a, d): mean and half difference */
    c = fl2(w32(c + b)); b = w32(b - c);        /* pair (b, c) */
    a = fl2(w32(a + c)); c = w32(c - a);        /* means of the means */
    d = fl2(w32(d + b)); b = w32(b - d);        /* half differences combined */
    d = w32(d + fl2(b)); b = w32(b - fl2(d));   /* final rotation of the odd pair */
    p[0] = (int32_t)a; p[stride] = (int32_t)b; p[2 * stride] = (int32_t)c; p[3 * stride] = (int32_t)d;
}

/* inverse of fwd_lift: the same steps undone in reverse order */
static void inv_lift(int32_t *p, int stride)
{
    int64_t a = p[0], b = p[stride], c = p[2 * stride], d = p[3 * stride];
    b = w32(b + fl2(d)); d = w32(d - fl2(b));
    b = w32(b + d);      d = w32(2 * d - b);
    c = w32(c + a);      a = w32(2 * a - c);
    b = w32(b + c);      c = w32(2 * c - b);
    d = w32(d + a);      a = w32(2 * a - d);
    p[0] = (int32_t)a; p[stride] = (int32_t)b; p[2 * stride] = (int32_t)c; p[3 * stride] = (int32_t)d;
}

void oracle_fwd_lift4(int32_t *v4) { fwd_lift(v4, 1); }
void oracle_inv_lift4(int32_t *v4) { inv_lift(v4, 1); }

/* Block value index i + 4j + 16k for (x, y, z) = (i, j, k).  Forward: x lines,
 * then y lines, then z lines.  Inverse: z, then y, then x.                */
void oracle_fwd_xform(int32_t *q)
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            fwd_lift(q + 4 * j + 16 * k, 1);
    for (int k = 0; k < 4; k++)
        for (int i = 0; i < 4; i++)
            fwd_lift(q + i + 16 * k, 4);
    for (int j = 0; j < 4; j++)
        for (int i = 0; i < 4; i++)
            fwd_lift(q + i + 4 * j, 16);
}

void oracle_inv_xform(int32_t *q)
{
    for (int j = 0; j < 4; j++)
        for (int i = 0; i < 4; i++)
            inv_lift(q + i + 4 * j, 16);
    for (int k = 0; k < 4; k++)
        for (int i = 0; i < 4; i++)
            inv_lift(q + i + 16 * k, 4);
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            inv_lift(q + 4 * j + 16 * k, 1);
}

/* (4) Sequency order: perm[n] = block index of the n-th coefficient, sorted by
 * (i+j+k, i^2+j^2+k^2, i+4j+16k) ascending.  Plain selection sort.         */
void oracle_sequency_order(int *perm)
{
    int64_t key[64];
    for (int idx = 0; idx < 64; idx++) {
        int i = idx & 3, j = (idx >> 2) & 3, k = idx >> 4;
        key[idx] = (int64_t)(i + j + k) * 100000 + (i * i + j * j + k * k) * 100 + idx;
        perm[idx] = idx;
    }
    for (int a = 0; a < 64; a++)
        for (int b = a + 1; b < 64; b++)
            if (key[perm[b]] < key[perm[a]]) {
                int t = perm[a];
                perm[a] = perm[b];
                perm[b] = t;
            }
}

/* (5) two's complement <-> negabinary (base -2 digits in a uint32) */
uint32_t oracle_to_negabinary(int32_t x) { return ((uint32_t)x + NBMASK) ^ NBMASK; }
int32_t oracle_from_negabinary(uint32_t u) { return (int32_t)((u ^ NBMASK) - NBMASK); }

/* bit writer / reader over little-endian 32-bit words, bit b = word b/32, bit b%32 */
typedef struct {
    uint32_t *w;
    int pos;
    int left; /* remaining budget in bits */
} bitw;

static int put_bit(bitw *s, int bit)
{
    if (s->left <= 0)
        return 0;
    if (bit)
        s->w[s->pos >> 5] |= 1u << (s->pos & 31);
    s->pos++;
    s->left--;
    return 1;
}

typedef struct {
    const uint32_t *w;
    int pos;
    int left;
} bitr;

/* returns 0/1, or -1 when the budget is exhausted */
static int get_bit(bitr *s)
{
    if (s->left <= 0)
        return -1;
    int b = (s->w[s->pos >> 5] >> (s->pos & 31)) & 1u;
    s->pos++;
    s->left--;
    return b;
}

/* (6) Embedded coding of 64 negabinary coefficients (already in sequency
 * order) into at most `budget` bits appended to s.  For each plane p from 31
 * down to 0, with X = bit p of every coefficient and n = number of leading
 * coefficients already significant:
 *   - the first n bits of X are sent as they are;
 *   - then, while n < 64: one group-test bit says whether any of bits n..63 is
 *     set; if not, the plane ends.  If so, bits n, n+1, ... are sent until a 1
 *     has been sent, and n moves past it.  When the scan reaches the last
 *     coefficient (n = 63) its bit must be 1 and is not sent.
 * Coding stops as soon as the budget is spent.                             */
void oracle_encode_planes(const uint32_t *u, int budget, uint32_t *words, int bitpos)
{
    bitw s = {words, bitpos, budget};
    int n = 0;
    for (int p = CODEC_PLANES - 1; p >= 0; p--) {
        int bit[64];
        for (int i = 0; i < 64; i++)
            bit[i] = (u[i] >> p) & 1u;
        for (int i = 0; i < n; i++)
            if (!put_bit(&s, bit[i]))
                return;
        while (n < 64) {
            int any = 0;
            for (int i = n; i < 64; i++)
                any |= bit[i];
            if (!put_bit(&s, any))
                return;
            if (!any)
                break;
            for (;;) {
                if (n == 63) { /* implied one */
                    n = 64;
                    break;
                }
                int b = bit[n];
                if (!put_bit(&s, b))
                    return;
                n++;
                if (b)
                    break;
            }
        }
    }
}

/* Inverse of oracle_encode_planes.  Writes the 64 coefficients (sequency
 * order) and returns the lowest plane index that was decoded completely
 * (32 when not even plane 31 was complete).                               */
int oracle_decode_planes(const uint32_t *words, int bitpos, int budget, uint32_t *u)
{
    bitr s = {words, bitpos, budget};
    int n = 0;
    int lowest_complete = CODEC_PLANES;
    memset(u, 0, 64 * sizeof(uint32_t));
    for (int p = CODEC_PLANES - 1; p >= 0; p--) {
        for (int i = 0; i < n; i++) {
            int b = get_bit(&s);
            if (b < 0)
                return lowest_complete;
            if (b)
                u[i] |= 1u << p;
        }
        while (n < 64) {
            int any = get_bit(&s);
            if (any < 0)
                return lowest_complete;
            if (!any)
                break;
            for (;;) {
                if (n == 63) {
                    u[63] |= 1u << p;
                    n = 64;
                    break;
                }
                int b = get_bit(&s);
                if (b < 0)
                    return lowest_complete;
                if (b)
                    u[n] |= 1u << p;
                n++;
                if (b)
                    break;
            }
        }
        lowest_complete = p;
    }
    return lowest_complete;
}

/* 1 if any of the 64 values is an infinity or a NaN.  The codec is defined
 * for finite values only; such a block is written as an all-zero block and
 * the encoder reports it (a reading of this project: the paper's codec input
 * is a simulation field, which is finite unless the run has blown up).    */
static int block_nonfinite(const float *v)
{
    for (int i = 0; i < 64; i++)
        if (!isfinite(v[i]))
            return 1;
    return 0;
}

/* Encode one block of 64 floats (index i + 4j + 16k) at `rate` bits/value
 * into words[0 .. 2*rate): exactly 64*rate bits, zero padded.  Returns 0, or
 * 1 for a block holding a non-finite value (then coded as all zeros).     */
int oracle_encode_block(const float *v, int rate, uint32_t *words)
{
    int nwords = 2 * rate, maxbits = 64 * rate;
    memset(words, 0, (size_t)nwords * sizeof(uint32_t));
    if (block_nonfinite(v))
        return 1;
    int hdr = oracle_block_header(v);
    for (int b = 0; b < 8; b++)
        if ((hdr >> b) & 1)
            words[0] |= 1u << b;
    if (hdr == 0)
        return 0;
    int emax = hdr - 127;
    int32_t q[64];
    oracle_quantize(v, emax, q);
    oracle_fwd_xform(q);
    int perm[64];
    oracle_sequency_order(perm);
    uint32_t u[64];
    for (int n = 0; n < 64; n++)
        u[n] = oracle_to_negabinary(q[perm[n]]);
    oracle_encode_planes(u, maxbits - 8, words, 8);
    return 0;
}

/* Decode one block; returns the lowest completely decoded plane (32 for a
 * zero block, which decodes to +0.0 everywhere).                          */
int oracle_decode_block(const uint32_t *words, int rate, float *v)
{
    int hdr = (int)(words[0] & 0xFFu);
    if (hdr == 0) {
        for (int i = 0; i < 64; i++)
            v[i] = 0.0f;
        return CODEC_PLANES;
    }
    /* the encoder never writes headers 1..31 (emax is clamped to >= -95); a
     * decoder given one applies the same clamp                               */
    int emax = hdr - 127;
    if (emax < CODEC_EMIN)
        emax = CODEC_EMIN;
    uint32_t u[64];
    int low = oracle_decode_planes(words, 8, 64 * rate - 8, u);
    int perm[64];
    oracle_sequency_order(perm);
    int32_t q[64];
    for (int n = 0; n < 64; n++)
        q[perm[n]] = oracle_from_negabinary(u[n]);
    oracle_inv_xform(q);
    oracle_dequantize(q, emax, v);
    return low;
}

/* Field layout: block (bx, by, bz) of an [nz][ny][nx] field (all multiples of
 * 4) is stored at byte offset ((bz * (ny/4) + by) * (nx/4) + bx) * 8*rate,
 * i.e. 4-plane block layers one after another, blocks x-fastest in a layer. */
static void gather(const float *f, int64_t nx, int64_t ny, int64_t bx, int64_t by, int64_t bz,
                   float *v)
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            for (int i = 0; i < 4; i++)
                v[i + 4 * j + 16 * k] = f[IDX(4 * bx + i, 4 * by + j, 4 * bz + k)];
}

static void scatter(float *f, int64_t nx, int64_t ny, int64_t bx, int64_t by, int64_t bz,
                    const float *v)
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            for (int i = 0; i < 4; i++)
                f[IDX(4 * bx + i, 4 * by + j, 4 * bz + k)] = v[i + 4 * j + 16 * k];
}

/* Returns the number of blocks that held a non-finite value. */
int64_t oracle_encode_field(const float *f, int64_t nx, int64_t ny, int64_t nz, int rate,
                            uint32_t *out)
{
    int64_t bnx = nx / 4, bny = ny / 4, bnz = nz / 4, b, bad = 0;
    int64_t nb = bnx * bny * bnz;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (b = 0; b < nb; b++) {
        int64_t bx = b % bnx, by = (b / bnx) % bny, bz = b / (bnx * bny);
        float v[64];
        gather(f, nx, ny, bx, by, bz, v);
        bad += oracle_encode_block(v, rate, out + b * 2 * rate);
    }
    return bad;
}

void oracle_decode_field(const uint32_t *in, int64_t nx, int64_t ny, int64_t nz, int rate,
                         float *f, int8_t *lowest_plane /* may be NULL, one per block */)
{
    int64_t bnx = nx / 4, bny = ny / 4, bnz = nz / 4, b;
    int64_t nb = bnx * bny * bnz;
#pragma omp parallel for schedule(static)
    for (b = 0; b < nb; b++) {
        int64_t bx = b % bnx, by = (b / bnx) % bny, bz = b / (bnx * bny);
        float v[64];
        int low = oracle_decode_block(in + b * 2 * rate, rate, v);
        if (lowest_plane)
            lowest_plane[b] = (int8_t)low;
        scatter(f, nx, ny, bx, by, bz, v);
    }
}

/* ------------------------------------------------------------------------ */
/* 3. adjoint of the leapfrog wave steps, FP64                              */
/* ------------------------------------------------------------------------ */
/*
 * Forward (interior points; the Dirichlet shell stays 0 when it starts at 0):
 *   u^(n+1) = 2 u^n - u^(n-1) + m (L u^n + w_n e_src),   u^0 = u^(-1) = 0,
 *   J = 1/2 sum_{n=1..N} sum_{x,y} (u^n(x, y, z_r) - d^n(x, y))^2.
 * Its discrete adjoint (Lagrange multipliers of the step equations):
 *   lam^n = 2 lam^(n+1) - lam^(n+2) + L (m lam^(n+1)) + r^n e_(z_r),
 *   lam^(N+1) = lam^(N+2) = 0,  r^n = u^n(z_r) - d^n,
 *   dJ/dm = sum_{n=0..N-1} lam^(n+1) (L u^n + w_n e_src).
 * L is the symmetric star operator on the interior with zero shell values, so
 * its transpose applied to (m lam) is L applied to the product.            */

/* L u at interior points (0 on the shell) */
static void star_apply(int64_t nx, int64_t ny, int64_t nz, int r, const double *coef,
                       const double *u, double *out)
{
    const int64_t sx = 1, sy = nx, sz = nx * ny;
    int64_t z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                int64_t p = IDX(x, y, z);
                if (x < r || y < r || z < r || x >= nx - r || y >= ny - r || z >= nz - r) {
                    out[p] = 0.0;
                    continue;
                }
                double L = coef[0] * u[p];
                for (int d = 1; d <= r; d++)
                    L += coef[d] * ((u[p - d * sx] + u[p + d * sx]) + (u[p - d * sy] + u[p + d * sy]) +
                                    (u[p - d * sz] + u[p + d * sz]));
                out[p] = L;
            }
}

void oracle_star_apply(int64_t nx, int64_t ny, int64_t nz, int r, const double *coef, const double *u,
                       double *out)
{
    star_apply(nx, ny, nz, r, coef, u, out);
}

/* One adjoint step: lam_new = 2 lam - lam_prev + L(m lam) + (res at plane z_r).
 * res (nx*ny, may be NULL) is added at plane zr of the interior.  Shell
 * points of lam_new are 0.                                                 */
void oracle_wave_adjoint_step(int64_t nx, int64_t ny, int64_t nz, const double *coef,
                              const double *m, const double *lam, const double *lam_prev,
                              double *lam_new, const double *res, int64_t zr, double *scratch)
{
    int64_t n = nx * ny * nz, i;
    for (i = 0; i < n; i++)
        scratch[n + i] = m[i] * lam[i];  /* second half of scratch: m lam */
    star_apply(nx, ny, nz, 4, coef, scratch + n, scratch);
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                int64_t p = IDX(x, y, z);
                if (x < 4 || y < 4 || z < 4 || x >= nx - 4 || y >= ny - 4 || z >= nz - 4) {
                    lam_new[p] = 0.0;
                    continue;
                }
                double v = 2.0 * lam[p] - lam_prev[p] + scratch[p];
                if (res && z == zr)
                    v += res[y * nx + x];
                lam_new[p] = v;
            }
}

/* Misfit and gradient of the wave workload by forward run + adjoint run.
 * Inputs: m (n), wavelet w[0..N), source index src (or -1), receiver plane zr,
 * observed data d[N][ny][nx] (d[n-1] is compared with u^n).  Outputs: J and
 * grad_m (n).  Keeps all N+1 states (small grids only).                    */
double oracle_wave_misfit_gradient(int64_t nx, int64_t ny, int64_t nz, const double *coef,
                                   const double *m, int nsteps, int64_t src, const double *w,
                                   int64_t zr, const double *d, double *grad_m)
{
    int64_t n = nx * ny * nz, plane = nx * ny;
    double *U = (double *)calloc((size_t)(nsteps + 2) * n, sizeof(double)); /* U[k] = u^(k-1) */
    double *lam = (double *)calloc((size_t)3 * n, sizeof(double));
    double *scratch = (double *)calloc((size_t)2 * n, sizeof(double));
    double *res = (double *)calloc((size_t)plane, sizeof(double));
    double J = 0.0;
    /* forward: U[0] = u^-1 = 0, U[1] = u^0 = 0 */
    for (int k = 0; k < nsteps; k++) {
        oracle_star_step(nx, ny, nz, 4, coef, 1, m, U + (int64_t)(k + 1) * n, U + (int64_t)k * n,
                         U + (int64_t)(k + 2) * n, src, w ? w[k] : 0.0);
    }
    for (int k = 1; k <= nsteps; k++)
        for (int64_t q = 0; q < plane; q++) {
            double r = U[(int64_t)(k + 1) * n + zr * plane + q] - d[(int64_t)(k - 1) * plane + q];
            J += 0.5 * r * r;
        }
    /* adjoint: lam[0] = lam^(n+2), lam[1] = lam^(n+1); gradient uses u^n = U[n+1] */
    for (int64_t q = 0; q < n; q++)
        grad_m[q] = 0.0;
    double *lpp = lam, *lp = lam + n, *lc = lam + 2 * n;
    double *Lu = scratch; /* reused below after the adjoint step */
    for (int k = nsteps; k >= 1; k--) {
        /* lam^k from lam^(k+1) = lp, lam^(k+2) = lpp, residual of u^k */
        for (int64_t q = 0; q < plane; q++)
            res[q] = U[(int64_t)(k + 1) * n + zr * plane + q] - d[(int64_t)(k - 1) * plane + q];
        oracle_wave_adjoint_step(nx, ny, nz, coef, m, lp, lpp, lc, res, zr, scratch);
        /* gradient term n = k-1: lam^k (L u^(k-1) + w_(k-1) e_src) */
        star_apply(nx, ny, nz, 4, coef, U + (int64_t)k * n, Lu);
        for (int64_t q = 0; q < n; q++) {
            double t = Lu[q];
            if (q == src && w)
                t += w[k - 1];
            grad_m[q] += lc[q] * t;
        }
        double *t = lpp;
        lpp = lp;
        lp = lc;
        lc = t;
    }
    free(U);
    free(lam);
    free(scratch);
    free(res);
    return J;
}

/* ---------------------------------------------------------------------------
 * Block quantiser (item 3 of the header): the bits of a block are numbered
 * from bit 0 of word 0 upwards (bit p is bit p % 32 of word p / 32), and are
 * written and read one at a time.
 * ------------------------------------------------------------------------- */
static void bq_put_bit(uint32_t *words, int p, unsigned bit)
{
    if (bit)
        words[p / 32] |= 1u << (p % 32);
}

static unsigned bq_get_bit(const uint32_t *words, int p) { return (words[p / 32] >> (p % 32)) & 1u; }

/* 0 for an all-zero block, else emax + 127 (in 1 .. 255) */
int oracle_bq_header(const float *v)
{
    float mx = 0.0f;
    for (int i = 0; i < 64; i++)
        if (fabsf(v[i]) > mx)
            mx = fabsf(v[i]);
    if (mx == 0.0f)
        return 0;
    int e;
    frexpf(mx, &e); /* mx = f 2^e, f in [0.5, 1) */
    if (e < -126)
        e = -126;
    return e + 127;
}

/* Returns 0, or 1 for a block holding a non-finite value, which is written
 * as an all-zero block (the same rule as the transform codec).            */
int oracle_bq_encode_block(const float *v, int rate, uint32_t *words)
{
    const int q = rate - 1;
    const int64_t lim = ((int64_t)1 << (q - 1)) - 1;
    memset(words, 0, (size_t)(2 * rate) * sizeof(uint32_t));
    if (block_nonfinite(v))
        return 1;
    const int hdr = oracle_bq_header(v);
    for (int b = 0; b < 8; b++)
        bq_put_bit(words, b, (hdr >> b) & 1);
    if (hdr == 0)
        return 0;
    const int emax = hdr - 127;
    for (int j = 0; j < 64; j++) {
        /* v 2^(q-1-emax) is exact in double for every finite float */
        double x = rint(ldexp((double)v[j], q - 1 - emax));
        int64_t n = (int64_t)x;
        if (n > lim)
            n = lim;
        if (n < -lim)
            n = -lim;
        const uint64_t u = (uint64_t)n; /* two's complement, low q bits kept */
        for (int b = 0; b < q; b++)
            bq_put_bit(words, 8 + j * q + b, (unsigned)((u >> b) & 1u));
    }
    return 0;
}

void oracle_bq_decode_block(const uint32_t *words, int rate, float *v)
{
    const int q = rate - 1;
    int hdr = 0;
    for (int b = 0; b < 8; b++)
        hdr |= (int)bq_get_bit(words, b) << b;
    if (hdr == 0) {
        for (int j = 0; j < 64; j++)
            v[j] = 0.0f;
        return;
    }
    const int emax = hdr - 127;
    for (int j = 0; j < 64; j++) {
        int64_t n = 0;
        for (int b = 0; b < q; b++)
            n |= (int64_t)bq_get_bit(words, 8 + j * q + b) << b;
        if (n >> (q - 1)) /* sign bit of the q-bit field */
            n -= (int64_t)1 << q;
        const float fn = (float)n; /* round to nearest */
        v[j] = (float)((double)fn * ldexp(1.0, emax - q + 1)); /* exact product, one rounding */
    }
}

int64_t oracle_bq_encode_field(const float *f, int64_t nx, int64_t ny, int64_t nz, int rate, uint32_t *out)
{
    int64_t bnx = nx / 4, bny = ny / 4, bnz = nz / 4, b, bad = 0;
    int64_t nb = bnx * bny * bnz;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (b = 0; b < nb; b++) {
        int64_t bx = b % bnx, by = (b / bnx) % bny, bz = b / (bnx * bny);
        float v[64];
        gather(f, nx, ny, bx, by, bz, v);
        bad += oracle_bq_encode_block(v, rate, out + b * 2 * rate);
    }
    return bad;
}

void oracle_bq_decode_field(const uint32_t *in, int64_t nx, int64_t ny, int64_t nz, int rate, float *f)
{
    int64_t bnx = nx / 4, bny = ny / 4, bnz = nz / 4, b;
    int64_t nb = bnx * bny * bnz;
#pragma omp parallel for schedule(static)
    for (b = 0; b < nb; b++) {
        int64_t bx = b % bnx, by = (b / bnx) % bny, bz = b / (bnx * bny);
        float v[64];
        oracle_bq_decode_block(in + b * 2 * rate, rate, v);
        scatter(f, nx, ny, bx, by, bz, v);
    }
}
