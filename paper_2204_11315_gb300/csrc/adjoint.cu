// adjoint.cu -- gradient of the receiver misfit of the leapfrog wave scheme:
// the discrete adjoint step, gradient accumulation, the receiver residual and
// the velocity <-> model maps, as device-level C ABI entry points.
//
// Forward (interior points, zero Dirichlet shell; Sec. 6 wave code):
//   u^(n+1) = 2 u^n - u^(n-1) + m (L u^n + w_n e_src),  J = 1/2 sum_n |u^n(z_r) - d^n|^2.
// Adjoint, backwards in time, with mu = m lam carried along:
//   lam^n = 2 lam^(n+1) - lam^(n+2) + L(mu^(n+1)) + r^n e_(z_r),  mu^n = m lam^n,
//   dJ/dm += lam^(n+1) (L u^n + w_n e_src).
// L is symmetric on the interior, so the transposed step applies the stencil to
// m lam (not m L lam).  Kernels: one thread per (x, y) column marching z with a
// register queue of the stencil field; x-y neighbours come through the L1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "../../include/oocs.h"
#include "capi_internal.h"
#include "stencil.cuh"

namespace oocs {
namespace {

constexpr int kAX = 32, kAY = 8;

struct AdjArgs {
    const float *field;  // stencil input: mu (adjoint step) or u (gradient)
    const float *lam;    // lam^(n+1)
    float *acc;          // adjoint: lam^(n+2) in, lam^n out; gradient: dJ/dm in/out
    float *mu_out;       // adjoint: m lam^n
    const float *m;
    const float *res;    // adjoint: residual plane at zr (or null)
    int zr;
    int nx, ny, nz;
    StarCoef c;
    int src_x, src_y, src_z;
    float w;
};

template <bool GRADIENT>
__global__ void __launch_bounds__(kAX *kAY) k_adjoint(const AdjArgs a)
{
    constexpr int R = 4;
    const int x = blockIdx.x * kAX + threadIdx.x;
    const int y = blockIdx.y * kAY + threadIdx.y;
    if (x >= a.nx || y >= a.ny)
        return;
    const int64_t plane = (int64_t)a.nx * a.ny;
    const int64_t col = (int64_t)y * a.nx + x;
    const bool xy_in = x >= R && x < a.nx - R && y >= R && y < a.ny - R;
    auto F = [&](int z) -> float { return (z >= 0 && z < a.nz) ? __ldg(a.field + z * plane + col) : 0.0f; };
    float q[2 * R + 1];
    q[0] = 0.0f;
#pragma unroll
    for (int i = 1; i <= 2 * R; ++i)
        q[i] = F(i - 1 - R);
    for (int z = 0; z < a.nz; ++z) {
#pragma unroll
        for (int i = 0; i < 2 * R; ++i)
            q[i] = q[i + 1];
        q[2 * R] = F(z + R);
        const int64_t p = z * plane + col;
        const bool in = xy_in && z >= R && z < a.nz - R;
        float L = 0.0f;
        if (in) {
            const float *row = a.field + p;
            float s[R + 1];
            s[0] = 0.0f;
#pragma unroll
            for (int d = 1; d <= R; ++d)
                s[d] = nbr_sum(__ldg(row - d), __ldg(row + d), __ldg(row - d * a.nx), __ldg(row + d * a.nx),
                               q[R - d], q[R + d]);
            L = star_L<R>(a.c, q[R], s);
        }
        if constexpr (GRADIENT) {
            if (in) {
                const float t = (x == a.src_x && y == a.src_y && z == a.src_z) ? fadd_rn(L, a.w) : L;
                a.acc[p] = fma_rn(__ldg(a.lam + p), t, a.acc[p]);
            }
        } else {
            float out = 0.0f;
            if (in) {
                const float lam = __ldg(a.lam + p);
                out = fadd_rn(fsub_rn(fadd_rn(lam, lam), a.acc[p]), L);
                if (a.res && z == a.zr)
                    out = fadd_rn(out, __ldg(a.res + col));
            }
            a.acc[p] = out;
            a.mu_out[p] = in ? fmul_rn(__ldg(a.m + p), out) : 0.0f;
        }
    }
}

__global__ void k_residual(const float *__restrict__ u, const float *__restrict__ d, float *__restrict__ r,
                           int64_t n, double *misfit)
{
    __shared__ double part[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = fsub_rn(u[i], d[i]);
        r[i] = v;
        acc += (double)v * (double)v;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && misfit)
        atomicAdd(misfit, 0.5 * part[0]);
}

// m = (v s)^2  and  dJ/dv = dJ/dm * 2 s^2 v,  s = dt / dx
__global__ void k_model(const float *__restrict__ v, float *__restrict__ m, int64_t n, float s)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float t = fmul_rn(v[i], s);
        m[i] = fmul_rn(t, t);
    }
}

__global__ void k_velocity_grad(const float *__restrict__ gm, const float *__restrict__ v, float *__restrict__ gv,
                                int64_t n, float s)
{
    const float k = fmul_rn(fmul_rn(2.0f, s), s);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gv[i] = fmul_rn(fmul_rn(k, v[i]), gm[i]);
}

oocs_status bad(const std::string &msg)
{
    set_last_error(msg);
    return OOCS_ERR_INVALID_ARG;
}

oocs_status launched(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
        return OOCS_ERR_CUDA;
    }
    return OOCS_OK;
}

oocs_status wave_desc_ok(const oocs_desc *d)
{
    if (!d)
        return bad("desc is NULL");
    if (d->scheme != OOCS_WAVE || d->radius != 4)
        return bad("the adjoint needs the wave scheme (25-point star, radius 4)");
    if (d->nx < 9 || d->ny < 9 || d->nz < 9 || d->nx % 4 || d->ny % 4 || d->nz % 4)
        return bad("nx, ny, nz must be multiples of 4 larger than the shell");
    return OOCS_OK;
}

AdjArgs base_args(const oocs_desc *d)
{
    AdjArgs a = {};
    a.nx = (int)d->nx;
    a.ny = (int)d->ny;
    a.nz = (int)d->nz;
    for (int i = 0; i < 5; ++i)
        a.c.c[i] = d->coef[i];
    a.src_z = -1;
    a.zr = -1;
    return a;
}

unsigned grid1d(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace
}  // namespace oocs

using namespace oocs;

extern "C" {

oocs_status oocs_adjoint_step(const oocs_desc *desc, const float *lam, float *lam_prev, const float *mu,
                              float *mu_out, const float *m, const float *res, int64_t zr, void *stream)
{
    oocs_status s = wave_desc_ok(desc);
    if (s != OOCS_OK)
        return s;
    if (!lam || !lam_prev || !mu || !mu_out || !m || mu == mu_out)
        return bad("lam, lam_prev, mu, mu_out, m must be distinct device arrays (mu_out != mu)");
    if (res && (zr < 4 || zr >= desc->nz - 4))
        return bad("receiver plane must be an interior plane");
    AdjArgs a = base_args(desc);
    a.field = mu;
    a.lam = lam;
    a.acc = lam_prev;
    a.mu_out = mu_out;
    a.m = m;
    a.res = res;
    a.zr = (int)zr;
    dim3 grid((unsigned)((desc->nx + kAX - 1) / kAX), (unsigned)((desc->ny + kAY - 1) / kAY));
    k_adjoint<false><<<grid, dim3(kAX, kAY), 0, static_cast<cudaStream_t>(stream)>>>(a);
    return launched("adjoint step");
}

oocs_status oocs_gradient_accumulate(const oocs_desc *desc, float *grad_m, const float *lam, const float *u,
                                     float w, const int64_t *src_xyz, void *stream)
{
    oocs_status s = wave_desc_ok(desc);
    if (s != OOCS_OK)
        return s;
    if (!grad_m || !lam || !u)
        return bad("grad_m, lam and u are required");
    AdjArgs a = base_args(desc);
    a.field = u;
    a.lam = lam;
    a.acc = grad_m;
    if (src_xyz) {
        a.src_x = (int)src_xyz[0];
        a.src_y = (int)src_xyz[1];
        a.src_z = (int)src_xyz[2];
        a.w = w;
    }
    dim3 grid((unsigned)((desc->nx + kAX - 1) / kAX), (unsigned)((desc->ny + kAY - 1) / kAY));
    k_adjoint<true><<<grid, dim3(kAX, kAY), 0, static_cast<cudaStream_t>(stream)>>>(a);
    return launched("gradient accumulation");
}

oocs_status oocs_receiver_residual(const float *u_plane, const float *d_plane, int64_t n, float *res,
                                   double *misfit, void *stream)
{
    if (!u_plane || !d_plane || !res || n <= 0)
        return bad("u_plane, d_plane, res and n > 0 are required");
    k_residual<<<grid1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(u_plane, d_plane, res, n, misfit);
    return launched("receiver residual");
}

oocs_status oocs_model_from_velocity(const float *v, float *m, int64_t n, float dt_over_dx, void *stream)
{
    if (!v || !m || n <= 0)
        return bad("v, m and n > 0 are required");
    k_model<<<grid1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(v, m, n, dt_over_dx);
    return launched("model from velocity");
}

oocs_status oocs_velocity_gradient(const float *grad_m, const float *v, float *grad_v, int64_t n,
                                   float dt_over_dx, void *stream)
{
    if (!grad_m || !v || !grad_v || n <= 0)
        return bad("grad_m, v, grad_v and n > 0 are required");
    k_velocity_grad<<<grid1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(grad_m, v, grad_v, n, dt_over_dx);
    return launched("velocity gradient");
}

}  // extern "C"
