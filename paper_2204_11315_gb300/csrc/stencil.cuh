// stencil.cuh -- the per-point star-stencil update, shared by every kernel.
//
// All kernels (in-core, streamed, fused with the codec) call these functions,
// so a point gets the same FP32 operations in the same order wherever it is
// computed; that is what makes a slab-streamed run bit-exact against an in-core
// run (temporal blocking recomputes halo points redundantly, Sec. 3.1).
//
//   s_d   = ((u[x-d] + u[x+d]) + (u[y-d] + u[y+d])) + (u[z-d] + u[z+d])
//   L     = fma(c_r, s_r, ... fma(c_1, s_1, c_0 * u))
//   heat: u' = L
//   wave: u' = fma(m, L (+ w at the source), (u + u) - up)
//   adjoint of the wave step (stencil applied to mu = m lam):
//         lam' = ((lam + lam) - lam_pp) + L (+ r at the receiver plane)
//   gradient of the wave misfit (stencil applied to u):
//         g' = fma(lam, L (+ w at the source), g)
#pragma once
#include "devmath.cuh"

namespace oocs {

enum { kHeat = 0, kWave = 1, kAdjoint = 2, kGradient = 3 };

struct StarCoef {
    float c[5];
};

OOCS_FN float nbr_sum(float xm, float xp, float ym, float yp, float zm, float zp)
{
    return fadd_rn(fadd_rn(fadd_rn(xm, xp), fadd_rn(ym, yp)), fadd_rn(zm, zp));
}

// L = c0 u + sum_d c_d s_d, accumulated from d = 1 upwards
template <int R>
OOCS_FN float star_L(const StarCoef &c, float u, const float (&s)[R + 1])
{
    float L = fmul_rn(c.c[0], u);
#pragma unroll
    for (int d = 1; d <= R; ++d)
        L = fma_rn(c.c[d], s[d], L);
    return L;
}

OOCS_FN float wave_update(float L, float u, float up, float m, bool at_src, float w)
{
    if (at_src)
        L = fadd_rn(L, w);
    return fma_rn(m, L, fsub_rn(fadd_rn(u, u), up));
}

OOCS_FN float adjoint_update(float L, float lam, float lam_pp, bool at_rcv, float r)
{
    const float v = fadd_rn(fsub_rn(fadd_rn(lam, lam), lam_pp), L);
    return at_rcv ? fadd_rn(v, r) : v;
}

OOCS_FN float gradient_update(float L, float lam, float g, bool at_src, float w)
{
    return fma_rn(lam, at_src ? fadd_rn(L, w) : L, g);
}

// The same operations on a pair of x-adjacent points (f32x2), for points
// without a source or receiver term: lane by lane the scalar forms above.
OOCS_FN float2 nbr_sum2(float2 xm, float2 xp, float2 ym, float2 yp, float2 zm, float2 zp)
{
    return fadd2_rn(fadd2_rn(fadd2_rn(xm, xp), fadd2_rn(ym, yp)), fadd2_rn(zm, zp));
}

template <int R>
OOCS_FN float2 star_L2(const StarCoef &c, float2 u, const float2 (&s)[R + 1])
{
    float2 L = fmul2_rn(make_float2(c.c[0], c.c[0]), u);
#pragma unroll
    for (int d = 1; d <= R; ++d)
        L = fma2_rn(make_float2(c.c[d], c.c[d]), s[d], L);
    return L;
}

OOCS_FN float2 wave_update2(float2 L, float2 u, float2 up, float2 m)
{
    return fma2_rn(m, L, fsub2_rn(fadd2_rn(u, u), up));
}

OOCS_FN float2 adjoint_update2(float2 L, float2 lam, float2 lam_pp)
{
    return fadd2_rn(fsub2_rn(fadd2_rn(lam, lam), lam_pp), L);
}

}  // namespace oocs
