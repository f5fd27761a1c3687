// kernels.cu -- sm_103a kernels: star-stencil time step and the block codec.
//
// Stencil step (Sec. 3.1, Sec. 6 25-point acoustic code): a 2.5D z-march.  A
// CTA owns a 32 x 16 tile of the x-y plane and walks its share of the z range.
// Each thread keeps the 2R+1 values u(z-R .. z+R) of its two columns in a
// register queue (one coalesced load per plane), and the x-y neighbours of
// plane z come from a (16+2R) x (32+2R) shared-memory tile.  Nothing here is a
// dense contraction, so the kernel is HBM-bound and uses no tensor cores.
//
// Codec (Sec. 4.2): one thread per 4x4x4 block; 16 float4 loads per block
// (consecutive threads read consecutive blocks of a row: coalesced).
#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "kernels.h"
#include "stencil.cuh"

namespace oocs {

constexpr int kTX = 32;
constexpr int kTY = 16;
constexpr int kRows = 2;  // rows per thread: ty and ty + kTY/kRows
constexpr int kStepThreads = kTX * (kTY / kRows);

struct StepArgs {
    const float *cur;
    const float *prev;
    const float *m;
    float *out;
    int nx, ny, nz;
    int64_t plane;
    int gz0, wp;
    int z_lo, z_hi, zchunk;
    StarCoef c;
    int src_x, src_y, src_zw;
    float w;
};

template <int R, int SCHEME>
__global__ void __launch_bounds__(kStepThreads) k_star_step(const StepArgs a)
{
    constexpr int W = kTX + 2 * R;
    constexpr int H = kTY + 2 * R;
    constexpr int kHalo = 2 * R * W + 2 * R * kTY;
    constexpr int kDy = kTY / kRows;
    __shared__ float tile[H][W];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int x0 = blockIdx.x * kTX;
    const int y0 = blockIdx.y * kTY;
    const int x = x0 + tx;
    const int zs = a.z_lo + blockIdx.z * a.zchunk;
    const int ze = min(zs + a.zchunk, a.z_hi);

    auto load_cur = [&](int z, int xx, int yy) -> float {
        return (z >= 0 && z < a.wp && xx >= 0 && xx < a.nx && yy >= 0 && yy < a.ny)
                   ? __ldg(a.cur + (int64_t)z * a.plane + (int64_t)yy * a.nx + xx)
                   : 0.0f;
    };

    float q[kRows][2 * R + 1];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        q[r][0] = 0.0f;
#pragma unroll
        for (int i = 1; i <= 2 * R; ++i)
            q[r][i] = load_cur(zs - R - 1 + i, x, y0 + ty + r * kDy);
    }

    for (int z = zs; z < ze; ++z) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
#pragma unroll
            for (int i = 0; i < 2 * R; ++i)
                q[r][i] = q[r][i + 1];
            q[r][2 * R] = load_cur(z + R, x, y0 + ty + r * kDy);
            tile[ty + r * kDy + R][tx + R] = q[r][R];
        }
        for (int i = tid; i < kHalo; i += kStepThreads) {
            int hy, hx;
            if (i < R * W) {
                hy = i / W;
                hx = i % W;
            } else if (i < 2 * R * W) {
                const int j = i - R * W;
                hy = kTY + R + j / W;
                hx = j % W;
            } else {
                const int j = i - 2 * R * W;
                const int col = j % (2 * R);
                hy = R + j / (2 * R);
                hx = col < R ? col : kTX + col;
            }
            tile[hy][hx] = load_cur(z, x0 + hx - R, y0 + hy - R);
        }
        __syncthreads();

        const int gz = a.gz0 + z;
        const bool zshell = gz < R || gz >= a.nz - R;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int ly = ty + r * kDy;
            const int y = y0 + ly;
            if (x < a.nx && y < a.ny) {
                const int64_t p = (int64_t)z * a.plane + (int64_t)y * a.nx + x;
                const float u = q[r][R];
                float res = u;  // Dirichlet shell keeps its value
                if (!(zshell || x < R || x >= a.nx - R || y < R || y >= a.ny - R)) {
                    float s[R + 1];
                    s[0] = 0.0f;
#pragma unroll
                    for (int d = 1; d <= R; ++d)
                        s[d] = nbr_sum(tile[ly + R][tx + R - d], tile[ly + R][tx + R + d],
                                       tile[ly + R - d][tx + R], tile[ly + R + d][tx + R],
                                       q[r][R - d], q[r][R + d]);
                    const float L = star_L<R>(a.c, u, s);
                    if constexpr (SCHEME == kHeat) {
                        res = L;
                    } else {
                        const bool at_src = (x == a.src_x && y == a.src_y && z == a.src_zw);
                        res = wave_update(L, u, a.prev[p], a.m[p], at_src, a.w);
                    }
                }
                a.out[p] = res;
            }
        }
        __syncthreads();
    }
}

template <int R, int SCHEME>
static cudaError_t launch_step_t(const StepArgs &a, int tiles_x, int tiles_y, int nchunks,
                                 cudaStream_t s)
{
    dim3 grid(tiles_x, tiles_y, nchunks);
    dim3 block(kTX, kTY / kRows, 1);
    k_star_step<R, SCHEME><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_star_step(const StepLaunch &L, cudaStream_t s)
{
    if (L.z_hi <= L.z_lo)
        return cudaSuccess;
    StepArgs a;
    a.cur = L.cur;
    a.prev = L.prev;
    a.m = L.m;
    a.out = L.out;
    a.nx = (int)L.nx;
    a.ny = (int)L.ny;
    a.nz = (int)L.nz;
    a.plane = L.nx * L.ny;
    a.gz0 = (int)L.gz0;
    a.wp = (int)L.wp;
    a.z_lo = (int)L.z_lo;
    a.z_hi = (int)L.z_hi;
    for (int i = 0; i < 5; ++i)
        a.c.c[i] = L.coef[i];
    a.src_x = (int)L.src_x;
    a.src_y = (int)L.src_y;
    a.src_zw = L.src_z >= 0 ? (int)(L.src_z - L.gz0) : -1;
    a.w = L.w;

    const int tiles_x = (int)((L.nx + kTX - 1) / kTX);
    const int tiles_y = (int)((L.ny + kTY - 1) / kTY);
    const int nplanes = a.z_hi - a.z_lo;
    // enough CTAs for ~2 waves at 8 CTAs/SM on 152 SMs, but at least 8R
    // planes per CTA so the 2R-plane queue prologue stays a small overhead
    const int target = 2 * 152 * 8;
    const int min_planes = 8 * L.radius;
    int nchunks = (target + tiles_x * tiles_y - 1) / (tiles_x * tiles_y);
    const int max_chunks = (nplanes + min_planes - 1) / min_planes;
    if (nchunks > max_chunks)
        nchunks = max_chunks;
    if (nchunks < 1)
        nchunks = 1;
    a.zchunk = (nplanes + nchunks - 1) / nchunks;
    nchunks = (nplanes + a.zchunk - 1) / a.zchunk;

    if (L.radius == 1 && L.scheme == kHeat)
        return launch_step_t<1, kHeat>(a, tiles_x, tiles_y, nchunks, s);
    if (L.radius == 4 && L.scheme == kHeat)
        return launch_step_t<4, kHeat>(a, tiles_x, tiles_y, nchunks, s);
    if (L.radius == 1 && L.scheme == kWave)
        return launch_step_t<1, kWave>(a, tiles_x, tiles_y, nchunks, s);
    if (L.radius == 4 && L.scheme == kWave)
        return launch_step_t<4, kWave>(a, tiles_x, tiles_y, nchunks, s);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ codec --

constexpr int kCodecThreads = 128;

__global__ void __launch_bounds__(kCodecThreads)
    k_encode_layers(const float *__restrict__ planes, int nx, int ny, int64_t nblocks, int rate,
                    uint32_t *__restrict__ out)
{
    const int64_t b = (int64_t)blockIdx.x * kCodecThreads + threadIdx.x;
    if (b >= nblocks)
        return;
    const int bnx = nx >> 2, bny = ny >> 2;
    const int bx = (int)(b % bnx);
    const int64_t t = b / bnx;
    const int by = (int)(t % bny);
    const int64_t bl = t / bny;
    const int64_t plane = (int64_t)nx * ny;
    const float *base = planes + 4 * bl * plane + (int64_t)(4 * by) * nx + 4 * bx;
    float v[64];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(base + k * plane + (int64_t)j * nx));
            v[16 * k + 4 * j + 0] = f.x;
            v[16 * k + 4 * j + 1] = f.y;
            v[16 * k + 4 * j + 2] = f.z;
            v[16 * k + 4 * j + 3] = f.w;
        }
    uint32_t *o = out + b * (int64_t)(2 * rate);
    encode_block(v, rate, [&](int i, uint32_t w) { o[i] = w; });
}

__global__ void __launch_bounds__(kCodecThreads)
    k_decode_layers(const uint32_t *__restrict__ in, int nx, int ny, int64_t nblocks, int rate,
                    float *__restrict__ planes)
{
    const int64_t b = (int64_t)blockIdx.x * kCodecThreads + threadIdx.x;
    if (b >= nblocks)
        return;
    const int bnx = nx >> 2, bny = ny >> 2;
    const int bx = (int)(b % bnx);
    const int64_t t = b / bnx;
    const int by = (int)(t % bny);
    const int64_t bl = t / bny;
    const int64_t plane = (int64_t)nx * ny;
    const uint32_t *src = in + b * (int64_t)(2 * rate);
    const int nw = 2 * rate;
    float v[64];
    decode_block(rate, [&](int i) -> uint32_t { return i < nw ? __ldg(src + i) : 0u; }, v);
    float *base = planes + 4 * bl * plane + (int64_t)(4 * by) * nx + 4 * bx;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4 *>(base + k * plane + (int64_t)j * nx) =
                make_float4(v[16 * k + 4 * j + 0], v[16 * k + 4 * j + 1], v[16 * k + 4 * j + 2],
                            v[16 * k + 4 * j + 3]);
}

cudaError_t launch_encode_layers(const float *planes, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, void *blocks, cudaStream_t s)
{
    const int64_t nb = (nx / 4) * (ny / 4) * nlayers;
    if (nb == 0)
        return cudaSuccess;
    const int64_t grid = (nb + kCodecThreads - 1) / kCodecThreads;
    k_encode_layers<<<(unsigned)grid, kCodecThreads, 0, s>>>(planes, (int)nx, (int)ny, nb, rate,
                                                             static_cast<uint32_t *>(blocks));
    return cudaGetLastError();
}

cudaError_t launch_decode_layers(const void *blocks, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, float *planes, cudaStream_t s)
{
    const int64_t nb = (nx / 4) * (ny / 4) * nlayers;
    if (nb == 0)
        return cudaSuccess;
    const int64_t grid = (nb + kCodecThreads - 1) / kCodecThreads;
    k_decode_layers<<<(unsigned)grid, kCodecThreads, 0, s>>>(
        static_cast<const uint32_t *>(blocks), (int)nx, (int)ny, nb, rate, planes);
    return cudaGetLastError();
}

}  // namespace oocs
