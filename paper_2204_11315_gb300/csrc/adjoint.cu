// adjoint.cu -- gradient of the receiver misfit of the leapfrog wave scheme:
// the discrete adjoint step, gradient accumulation, the receiver residual, the
// velocity <-> model maps, and a forward / backward driver with checkpoints,
// as device-level C ABI entry points.
//
// Forward (interior points, zero Dirichlet shell; Sec. 6 wave code):
//   u^(n+1) = 2 u^n - u^(n-1) + m (L u^n + w_n e_src),  J = 1/2 sum_n |u^n(z_r) - d^n|^2.
// Adjoint, backwards in time, with mu = m lam carried along:
//   lam^n = 2 lam^(n+1) - lam^(n+2) + L(mu^(n+1)) + r^n e_(z_r),  mu^n = m lam^n,
//   dJ/dm += lam^(n+1) (L u^n + w_n e_src).
// L is symmetric on the interior, so the transposed step applies the stencil to
// m lam (not m L lam).  The adjoint and gradient steps run in the TMA-fed
// z-march kernel of the forward step (kernels.cu, schemes kAdjoint and
// kGradient), so all three steps share its pipeline and its arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "../../include/oocs.h"
#include "capi_internal.h"
#include "kernels.h"
#include "stencil.cuh"

namespace oocs {
namespace {

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
    if (d->nx < 12 || d->ny < 12 || d->nz < 12 || d->nx % 4 || d->ny % 4 || d->nz % 4)
        return bad("nx, ny, nz must be multiples of 4, at least 12");
    return OOCS_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// whole-grid launch of one scheme of the z-march kernel
StepLaunch grid_launch(const oocs_desc *d, int scheme)
{
    StepLaunch L;
    memset(&L, 0, sizeof(L));
    L.scheme = scheme;
    L.radius = 4;
    L.tile = d->step_tile;
    L.nx = d->nx;
    L.ny = d->ny;
    L.nz = d->nz;
    L.gz0 = 0;
    L.wp = d->nz;
    L.z_lo = 0;
    L.z_hi = d->nz;
    for (int i = 0; i < 5; ++i)
        L.coef[i] = d->coef[i];
    L.src_z = -1;
    L.zr = -1;
    return L;
}

oocs_status step_launched(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
        return OOCS_ERR_CUDA;
    }
    return launched(what);
}

// Workspace of the misfit driver: the checkpoints (u^s, u^(s-1)) of every
// segment s = 0, K, 2K, ..., then K + 5 FP32 fields: P = u^(s-1), the
// segment's states u^s .. u^(s+K-1), lam, lam_prev, mu, mu_out.  The forward
// pass uses the first two fields as its (u, u_prev) pair.
struct GradLayout {
    int64_t n = 0, field = 0, ckpt = 0, nseg = 0, ckpt_total = 0, total = 0;
};

int64_t round256(int64_t b) { return (b + 255) / 256 * 256; }

GradLayout grad_layout(const oocs_desc *d, int32_t nsteps, int32_t K, int32_t rate)
{
    GradLayout g;
    g.n = d->nx * d->ny * d->nz;
    g.field = round256(g.n * 4);
    g.ckpt = round256(rate ? g.n / 8 * rate : g.n * 4);
    g.nseg = (nsteps + K - 1) / K;
    g.ckpt_total = 2 * g.nseg * g.ckpt;
    g.total = g.ckpt_total + (int64_t)(K + 5) * g.field;
    return g;
}

oocs_status driver_args(const oocs_desc *d, const int64_t *src, int64_t zr, int32_t nsteps, int32_t K,
                        int32_t rate, const void *ws, int64_t ws_bytes)
{
    oocs_status s = wave_desc_ok(d);
    if (s != OOCS_OK)
        return s;
    if (nsteps < 1 || K < 1)
        return bad("nsteps and checkpoint_every must be positive");
    if (rate < 0 || rate > 32)
        return bad("rate_bits must be 0 (raw checkpoints) or in [1, 32]");
    if (!src || src[0] < 0 || src[1] < 0 || src[2] < 0 || src[0] >= d->nx || src[1] >= d->ny || src[2] >= d->nz)
        return bad("source voxel outside the grid");
    if (zr < 4 || zr >= d->nz - 4)
        return bad("receiver plane must be an interior plane");
    if (!ws || !aligned16(ws))
        return bad("workspace must be a 16-byte aligned device array");
    if (ws_bytes < grad_layout(d, nsteps, K, rate).total)
        return bad("workspace too small (oocs_misfit_workspace_bytes)");
    return OOCS_OK;
}

// one forward leapfrog step: out <- u^(n+1) from (cur, prev) = (u^n, u^(n-1))
cudaError_t wave_step(const oocs_desc *d, const float *cur, const float *prev, const float *m, float *out,
                      const int64_t *src, const float *w, int32_t nw, int64_t n, cudaStream_t st)
{
    StepLaunch L = grid_launch(d, kWave);
    L.cur = cur;
    L.prev = prev;
    L.m = m;
    L.out = out;
    if (n >= 0 && n < nw) {
        L.src_x = src[0];
        L.src_y = src[1];
        L.src_z = src[2];
        L.w = w[n];
    }
    return launch_star_step(L, st);
}

cudaError_t save_field(const float *f, const oocs_desc *d, int32_t rate, void *dst, cudaStream_t st)
{
    if (!rate)
        return cudaMemcpyAsync(dst, f, d->nx * d->ny * d->nz * 4, cudaMemcpyDeviceToDevice, st);
    return launch_encode_layers(f, d->nx, d->ny, d->nz / 4, rate, kCodecTransform, dst, st);
}

cudaError_t load_field(const void *src, const oocs_desc *d, int32_t rate, float *f, cudaStream_t st)
{
    if (!rate)
        return cudaMemcpyAsync(f, src, d->nx * d->ny * d->nz * 4, cudaMemcpyDeviceToDevice, st);
    return launch_decode_layers(src, d->nx, d->ny, d->nz / 4, rate, kCodecTransform, f, st);
}

unsigned grid1d(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace
}  // namespace oocs

using namespace oocs;

extern "C" {

oocs_status oocs_adjoint_step(const oocs_desc *desc, const float *lam, float *lam_prev, const float *mu,
                              float *mu_out, const float *m, const float *res, int64_t zr, void *stream)
try {
    oocs_status s = wave_desc_ok(desc);
    if (s != OOCS_OK)
        return s;
    if (!lam || !lam_prev || !mu || !mu_out || !m || mu == mu_out)
        return bad("lam, lam_prev, mu, mu_out, m must be distinct device arrays (mu_out != mu)");
    if (!aligned16(lam) || !aligned16(lam_prev) || !aligned16(mu) || !aligned16(mu_out) || !aligned16(m) ||
        (res && !aligned16(res)))
        return bad("device arrays must be 16-byte aligned");
    if (res && (zr < 4 || zr >= desc->nz - 4))
        return bad("receiver plane must be an interior plane");
    StepLaunch L = grid_launch(desc, kAdjoint);
    L.cur = mu;
    L.prev = lam_prev;
    L.m = m;
    L.c2 = lam;
    L.out = lam_prev;
    L.out2 = mu_out;
    L.res = res;
    L.zr = res ? zr : -1;
    return step_launched(launch_star_step(L, static_cast<cudaStream_t>(stream)), "adjoint step");
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_gradient_accumulate(const oocs_desc *desc, float *grad_m, const float *lam, const float *u,
                                     float w, const int64_t *src_xyz, void *stream)
try {
    oocs_status s = wave_desc_ok(desc);
    if (s != OOCS_OK)
        return s;
    if (!grad_m || !lam || !u)
        return bad("grad_m, lam and u are required");
    if (!aligned16(grad_m) || !aligned16(lam) || !aligned16(u))
        return bad("device arrays must be 16-byte aligned");
    StepLaunch L = grid_launch(desc, kGradient);
    L.cur = u;
    L.prev = grad_m;
    L.m = lam;
    L.out = grad_m;
    if (src_xyz) {
        L.src_x = src_xyz[0];
        L.src_y = src_xyz[1];
        L.src_z = src_xyz[2];
        L.w = w;
    }
    return step_launched(launch_star_step(L, static_cast<cudaStream_t>(stream)), "gradient accumulation");
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_receiver_residual(const float *u_plane, const float *d_plane, int64_t n, float *res,
                                   double *misfit, void *stream)
try {
    if (!u_plane || !d_plane || !res || n <= 0)
        return bad("u_plane, d_plane, res and n > 0 are required");
    k_residual<<<grid1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(u_plane, d_plane, res, n, misfit);
    return launched("receiver residual");
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_model_from_velocity(const float *v, float *m, int64_t n, float dt_over_dx, void *stream)
try {
    if (!v || !m || n <= 0)
        return bad("v, m and n > 0 are required");
    k_model<<<grid1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(v, m, n, dt_over_dx);
    return launched("model from velocity");
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_velocity_gradient(const float *grad_m, const float *v, float *grad_v, int64_t n,
                                   float dt_over_dx, void *stream)
try {
    if (!grad_m || !v || !grad_v || n <= 0)
        return bad("grad_m, v, grad_v and n > 0 are required");
    k_velocity_grad<<<grid1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(grad_m, v, grad_v, n, dt_over_dx);
    return launched("velocity gradient");
} catch (...) {
    return exception_status(nullptr);
}

int64_t oocs_misfit_workspace_bytes(const oocs_desc *desc, int32_t nsteps, int32_t checkpoint_every,
                                    int32_t rate_bits)
{
    if (!desc || nsteps < 1 || checkpoint_every < 1 || rate_bits < 0 || rate_bits > 32)
        return -1;
    return grad_layout(desc, nsteps, checkpoint_every, rate_bits).total;
}

oocs_status oocs_misfit_forward(const oocs_desc *desc, const float *m, const int64_t *src_xyz, const float *w,
                                int32_t nw, int64_t zr, const float *d_obs, int32_t nsteps,
                                int32_t checkpoint_every, int32_t rate_bits, void *workspace,
                                int64_t workspace_bytes, float *res, double *misfit, void *stream)
try {
    oocs_status s = driver_args(desc, src_xyz, zr, nsteps, checkpoint_every, rate_bits, workspace,
                                workspace_bytes);
    if (s != OOCS_OK)
        return s;
    if (!m || !d_obs || !res || !misfit || (nw > 0 && !w) || !aligned16(m))
        return bad("m, d_obs, res, misfit are required (and w when nw > 0)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GradLayout g = grad_layout(desc, nsteps, checkpoint_every, rate_bits);
    unsigned char *base = static_cast<unsigned char *>(workspace);
    float *u = reinterpret_cast<float *>(base + g.ckpt_total);
    float *up = reinterpret_cast<float *>(base + g.ckpt_total + g.field);
    const int64_t plane = desc->nx * desc->ny;
    cudaError_t e = cudaMemsetAsync(misfit, 0, sizeof(double), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(u, 0, g.n * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(up, 0, g.n * 4, st);
    for (int32_t n = 0; e == cudaSuccess && n < nsteps; ++n) {
        if (n % checkpoint_every == 0) {
            unsigned char *ck = base + 2 * (n / checkpoint_every) * g.ckpt;
            e = save_field(u, desc, rate_bits, ck, st);
            if (e == cudaSuccess)
                e = save_field(up, desc, rate_bits, ck + g.ckpt, st);
            if (e != cudaSuccess)
                break;
        }
        e = wave_step(desc, u, up, m, up, src_xyz, w, nw, n, st);  // up <- u^(n+1)
        if (e != cudaSuccess)
            break;
        std::swap(u, up);
        k_residual<<<grid1d(plane), 256, 0, st>>>(u + zr * plane, d_obs + n * plane, res + n * plane, plane,
                                                  misfit);
        e = cudaGetLastError();
    }
    return step_launched(e, "misfit forward");
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_misfit_backward(const oocs_desc *desc, const float *m, const int64_t *src_xyz, const float *w,
                                 int32_t nw, int64_t zr, const float *res, int32_t nsteps,
                                 int32_t checkpoint_every, int32_t rate_bits, void *workspace,
                                 int64_t workspace_bytes, float *grad_m, void *stream)
try {
    oocs_status s = driver_args(desc, src_xyz, zr, nsteps, checkpoint_every, rate_bits, workspace,
                                workspace_bytes);
    if (s != OOCS_OK)
        return s;
    if (!m || !res || !grad_m || (nw > 0 && !w) || !aligned16(m) || !aligned16(res) || !aligned16(grad_m))
        return bad("m, res, grad_m are required and 16-byte aligned (and w when nw > 0)");
    if ((desc->nx * desc->ny * 4) % 16)
        return bad("residual planes must stay 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t K = checkpoint_every;
    const GradLayout g = grad_layout(desc, nsteps, K, rate_bits);
    unsigned char *base = static_cast<unsigned char *>(workspace);
    auto field = [&](int64_t i) { return reinterpret_cast<float *>(base + g.ckpt_total + i * g.field); };
    float *P = field(0);
    auto S = [&](int64_t i) { return field(1 + i); };  // S(i) = u^(s+i)
    float *lam = field(K + 1), *lam_prev = field(K + 2), *mu = field(K + 3), *mu_out = field(K + 4);
    const int64_t plane = desc->nx * desc->ny;
    cudaError_t e = cudaSuccess;
    for (float *f : {lam, lam_prev, mu, grad_m})
        if (e == cudaSuccess)
            e = cudaMemsetAsync(f, 0, g.n * 4, st);
    for (int64_t seg = g.nseg - 1; e == cudaSuccess && seg >= 0; --seg) {
        const int64_t s0 = seg * K, e0 = std::min<int64_t>(s0 + K, nsteps);
        const unsigned char *ck = base + 2 * seg * g.ckpt;
        e = load_field(ck, desc, rate_bits, S(0), st);
        if (e == cudaSuccess)
            e = load_field(ck + g.ckpt, desc, rate_bits, P, st);
        // the states the gradient terms n = s0 .. e0-1 need: u^s0 .. u^(e0-1)
        for (int64_t i = 1; e == cudaSuccess && i < e0 - s0; ++i)
            e = wave_step(desc, S(i - 1), i == 1 ? P : S(i - 2), m, S(i), src_xyz, w, nw, s0 + i - 1, st);
        for (int64_t k = e0; e == cudaSuccess && k > s0; --k) {
            StepLaunch L = grid_launch(desc, kAdjoint);  // lam_prev <- lam^k
            L.cur = mu;
            L.prev = lam_prev;
            L.m = m;
            L.c2 = lam;
            L.out = lam_prev;
            L.out2 = mu_out;
            L.res = res + (k - 1) * plane;
            L.zr = zr;
            e = launch_star_step(L, st);
            if (e != cudaSuccess)
                break;
            std::swap(lam, lam_prev);
            std::swap(mu, mu_out);
            StepLaunch G = grid_launch(desc, kGradient);  // term n = k-1
            G.cur = S(k - 1 - s0);
            G.prev = grad_m;
            G.m = lam;
            G.out = grad_m;
            if (k - 1 < nw) {
                G.src_x = src_xyz[0];
                G.src_y = src_xyz[1];
                G.src_z = src_xyz[2];
                G.w = w[k - 1];
            }
            e = launch_star_step(G, st);
        }
    }
    return step_launched(e, "misfit backward");
} catch (...) {
    return exception_status(nullptr);
}

}  // extern "C"
