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
#pragma once
#include "devmath.cuh"

namespace oocs {

enum { kHeat = 0, kWave = 1 };

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

}  // namespace oocs
