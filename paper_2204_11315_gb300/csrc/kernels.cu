// kernels.cu -- sm_103a kernels: star-stencil time step and the block codec.
//
// Stencil step (Sec. 3.1, Sec. 6 25-point acoustic code): a 2.5D z-march.  A
// CTA owns 64 x 16 tiles of the x-y plane and walks its share of their z
// range.  The u planes (with their x-y halo) arrive by TMA into a
// shared-memory ring several planes ahead of use; each consumer thread keeps
// u(z-R .. z+R) of its 2 x 4 points in a register queue.  Nothing here is a dense contraction, so the
// kernel is HBM-bound and uses no tensor cores.
//
// Codec (Sec. 4.2): one thread per 4x4x4 block; 16 float4 loads per block
// (consecutive threads read consecutive blocks of a row: coalesced); the
// transform encoder's CTA first fills its doubling table in shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <utility>

#include "codec.cuh"
#include "kernels.h"
#include "quant.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace oocs {

// Launch with programmatic stream serialization: the kernel may begin while its
// predecessor in the stream drains (every kernel here waits in
// pdl_wait_prior_grid before touching global memory).
template <class... KArgs, class... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

constexpr int kVX = 2;                  // x-adjacent points per thread (float2)
constexpr int kTX = 32 * kVX;           // tile width (x) = 64
constexpr int kRPT = 4;                 // consecutive rows per thread
constexpr int kConsumerWarps = 4;              // default tile: 4 consumer warps, 64 x 16
constexpr int kTY = kConsumerWarps * kRPT;         // default tile height (y) = 16
constexpr int kStepThreads = 32 * (kConsumerWarps + 1);  // + one producer warp
// The step kernel also comes with CW = 2 consumer warps (64 x 8 tiles), a
// choice of oocs_desc.step_tile that the autotuner searches.
template <int CW>
constexpr int tile_h() { return CW * kRPT; }
constexpr int kBoxW = kTX + 8;          // u tile loaded from x0-4 (16-byte aligned) to x0+kTX+4

// centre fields streamed beside the stencil field: wave (prev, m), adjoint
// (lam^(n+2), m, lam^(n+1)), gradient (dJ/dm, lam^(n+1))
template <int SCHEME>
constexpr int centre_fields() { return SCHEME == kHeat ? 0 : SCHEME == kAdjoint ? 3 : 2; }

template <int R, int NCF, int CW = kConsumerWarps>
struct StepCfg {
    static constexpr int TY = tile_h<CW>();                     // tile rows
    static constexpr int H = TY + 2 * R;                        // u tile rows
    static constexpr uint32_t kUBytes = H * kBoxW * 4;          // one TMA box of u
    static constexpr int kUStage = ((kUBytes + 127) / 128 * 128) / 4;  // floats per ring stage
    static constexpr int NSU = (2 * R + 2) > 6 ? (2 * R + 2) : 6;  // u ring stages (>= R+1 ahead)
    static constexpr int NSC = NCF == 3 ? 3 : 4;                // centre-field ring stages
    static constexpr int kCStage = kTX * TY;                    // floats per centre field and stage
    static constexpr uint32_t kCBytes = kCStage * 4;
    static constexpr int Q = 2 * R + 1;                         // register queue length
    static constexpr size_t smem_bytes()
    {
        return 128 + (size_t)NSU * kUStage * 4 + (size_t)NCF * NSC * kCStage * 4 + 2 * (NSU + NSC) * 8;
    }
    // fused encode: a 4-plane layer of the tile's results and the compressed
    // words of its (kTX / 4) x (TY / 4) blocks (rate up to 32)
    static constexpr int kEncBlocks = (kTX / 4) * (TY / 4);
    static constexpr int kEncStride = 2 * 32 + 1;
    static constexpr size_t enc_bytes() { return (size_t)4 * TY * kTX * 4 + (size_t)kEncBlocks * kEncStride * 4; }
};

struct StepArgs {
    float *out;
    float *out2;       // kAdjoint: m * out
    const float *res;  // kAdjoint: residual plane or null
    int zr;            // kAdjoint: global plane of res
    int nx, ny, nz;
    int64_t plane;
    int gz0;
    int z_lo, z_hi;
    int zchunk;         // > 0: chunked launch; 0: balanced launch
    int tiles_y, ntiles;
    StarCoef c;
    int src_x, src_y, src_zw;
    float w;
    const float *w_dev;  // device-side amplitude (see StepLaunch)
    const int64_t *t_dev;
    int64_t t_rel, nw;
    uint32_t *enc_out;   // fused encode (see StepLaunch): the out slot's blocks
    int enc_rate;
    int enc_layer0;      // global layer of enc_out's first layer
};

// Whether the step adds a source amplitude, and which (resolved once per
// thread before the z march).
OOCS_FN bool source_amplitude(const StepArgs &a, float &w)
{
    if (!a.w_dev) {
        w = a.w;
        return true;
    }
    const int64_t t = *a.t_dev + a.t_rel;
    if (t < 0 || t >= a.nw)
        return false;
    w = a.w_dev[t];
    return true;
}

// A piece of a CTA's work: tile (x0, y0), window planes [zs, ze).
struct StepSeg {
    int x0, y0, zs, ze;
};

// The CTA's segments, in order.  Chunked launch: grid (tiles_x, tiles_y,
// chunks), one segment per CTA.  Balanced launch: 1-D grid of G CTAs; the
// ntiles * P tile-planes (P = z_hi - z_lo), in tile-major order with tiles
// numbered y fastest, are split into G equal contiguous ranges, so every CTA
// does the same work and a range may end one tile's z range and start the
// next one's.  With y fastest, the tiles above and below (whose 2R-row halo
// is most of the extra u reads) are walked about P - ntiles P / G planes
// apart, so the shared halo rows are still in L2.
struct SegCursor {
    int64_t pos = 0, end = 0;
    bool chunk_done = false;

    OOCS_FN void init(const StepArgs &a)
    {
        if (a.zchunk == 0) {
            const int64_t total = (int64_t)a.ntiles * (a.z_hi - a.z_lo);
            pos = total * blockIdx.x / gridDim.x;
            end = total * (blockIdx.x + 1) / gridDim.x;
        }
    }
    template <int TY = kTY>
    OOCS_FN bool next(const StepArgs &a, StepSeg &s)
    {
        if (a.zchunk > 0) {
            if (chunk_done)
                return false;
            chunk_done = true;
            s.x0 = blockIdx.x * kTX;
            s.y0 = blockIdx.y * TY;
            s.zs = a.z_lo + blockIdx.z * a.zchunk;
            s.ze = min(s.zs + a.zchunk, a.z_hi);
            return s.zs < s.ze;
        }
        if (pos >= end)
            return false;
        const int P = a.z_hi - a.z_lo;
        const int64_t t = pos / P;
        const int64_t e = min(end, (t + 1) * P);
        s.x0 = (int)(t / a.tiles_y) * kTX;
        s.y0 = (int)(t % a.tiles_y) * TY;
        s.zs = a.z_lo + (int)(pos - t * P);
        s.ze = a.z_lo + (int)(e - t * P);
        pos = e;
        return true;
    }
};

// One time step over window planes [z_lo, z_hi).  A CTA walks the z range of
// one or more 64 x 16 tiles (segments, above), warp-specialised: warp 4 is
// the producer, which streams u tiles (with a 4-column / R-row halo) into an
// NSU-deep shared-memory ring and the centre fields (wave: prev, m) into an
// NSC-deep ring by TMA, each stage guarded by a "full" mbarrier (TMA bytes
// landed) and an "empty" mbarrier (all four consumer warps done with it);
// ring positions come from running counts of planes, so the rings carry on
// from one segment to the next.  Consumer warps run decoupled, with no
// CTA-wide barrier per plane.  Consumer thread (tx, w) owns the 2 x 4 points
// x = x0 + 2 tx + {0, 1}, y = y0 + 4 w + {0..3}; it keeps u(z-R .. z+R) of
// them in a register queue, takes x neighbours from 64-bit shared loads and y
// neighbours inside its four rows from the queue.  Planes outside the window
// or grid arrive zero-filled from TMA.  For R = 4, a warp whose 64 x 4 points
// are all interior, on a plane without the source or receivers, takes a path
// without per-point tests.
//
// kAdjoint and kGradient (the wave misfit's adjoint, see kernels.h) use the
// same pipeline with three and two centre fields.
template <int R, int SCHEME, int CW, bool ENC = false>
__global__ void __launch_bounds__(32 * (CW + 1), CW == kConsumerWarps ? 2 : 3)
    k_star_step(const __grid_constant__ CUtensorMap tm_cur, const __grid_constant__ CUtensorMap tm_prev,
                const __grid_constant__ CUtensorMap tm_m, const __grid_constant__ CUtensorMap tm_c2,
                const StepArgs a)
{
    static_assert(!ENC || (R == 1 && SCHEME == kHeat), "the fused encode is built for the heat step");
    constexpr int NCF = centre_fields<SCHEME>();
    using C = StepCfg<R, NCF, CW>;
    constexpr int Q = C::Q;
    constexpr bool kFastPath = R == 4;
    extern __shared__ unsigned char smem_raw[];
    float *us = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *cs = us + C::NSU * C::kUStage;  // centre field f, stage st at cs + (f NSC + st) kCStage
    uint64_t *ufull = reinterpret_cast<uint64_t *>(cs + NCF * C::NSC * C::kCStage);
    uint64_t *uempty = ufull + C::NSU;
    uint64_t *cfull = uempty + C::NSU;
    uint64_t *cempty = cfull + C::NSC;
    // fused encode: the layer of results and the blocks' compressed words
    [[maybe_unused]] float *lay = reinterpret_cast<float *>(cempty + C::NSC);
    [[maybe_unused]] uint32_t *rows = reinterpret_cast<uint32_t *>(lay + 4 * C::TY * kTX);
    __shared__ uint32_t dbl[ENC ? 256 : 1];

    const int tx = threadIdx.x, wid = threadIdx.y;
    if constexpr (ENC)
        fill_doubling_table(dbl, 32 * wid + tx, 32 * (CW + 1));

    if (wid == 0 && tx == 0) {
        for (int i = 0; i < C::NSU; ++i) {
            mbar_init(&ufull[i], 1);
            mbar_init(&uempty[i], CW);
        }
        for (int i = 0; i < C::NSC; ++i) {
            mbar_init(&cfull[i], 1);
            mbar_init(&cempty[i], CW);
        }
        fence_barrier_init();
    }
    __syncthreads();  // the only CTA-wide barrier
    // everything above overlaps the previous kernel's tail; global memory is
    // touched only after it has completed
    pdl_launch_dependents();
    pdl_wait_prior_grid();

    SegCursor cur;
    cur.init(a);
    StepSeg sg;

    if (wid == CW) {
        // ------------------------------------------------ producer warp --
        if (tx != 0)
            return;
        bool good = true;
        uint32_t un = 0, cn = 0;  // u planes / centre-field planes issued so far
        while (good && cur.template next<C::TY>(a, sg)) {
            // u planes in order (queue prologue first), the centre fields of
            // plane z alongside the u plane R ahead of it
            for (int p = sg.zs - R; p < sg.ze + R; ++p) {
                const uint32_t st = un % C::NSU, n = un / C::NSU;
                if (n > 0 && !mbar_wait(&uempty[st], (n - 1) & 1)) {
                    good = false;
                    break;
                }
                mbar_arrive_expect_tx(&ufull[st], C::kUBytes);
                tma_load_3d(us + st * C::kUStage, &tm_cur, sg.x0 - 4, sg.y0 - R, p, &ufull[st]);
                ++un;
                const int z = p - R;
                if (NCF > 0 && z >= sg.zs && z < sg.ze) {
                    const uint32_t cst = cn % C::NSC, cnn = cn / C::NSC;
                    if (cnn > 0 && !mbar_wait(&cempty[cst], (cnn - 1) & 1)) {
                        good = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&cfull[cst], NCF * C::kCBytes);
                    tma_load_3d(cs + cst * C::kCStage, &tm_prev, sg.x0, sg.y0, z, &cfull[cst]);
                    tma_load_3d(cs + (C::NSC + cst) * C::kCStage, &tm_m, sg.x0, sg.y0, z, &cfull[cst]);
                    if constexpr (NCF == 3)
                        tma_load_3d(cs + (2 * C::NSC + cst) * C::kCStage, &tm_c2, sg.x0, sg.y0, z, &cfull[cst]);
                    ++cn;
                }
            }
        }
        // drain: everything requested lands before the CTA may retire
        for (uint32_t i = un > (uint32_t)C::NSU ? un - C::NSU : 0; i < un; ++i)
            mbar_wait(&ufull[i % C::NSU], (i / C::NSU) & 1);
        for (uint32_t i = cn > (uint32_t)C::NSC ? cn - C::NSC : 0; i < cn; ++i)
            mbar_wait(&cfull[i % C::NSC], (i / C::NSC) & 1);
        return;
    }

    // --------------------------------------------------- consumer warps --
    // the source term of this step: its voxel's x (-1 when the step adds
    // nothing) and amplitude
    [[maybe_unused]] float w_src = 0.0f;
    [[maybe_unused]] int src_x = a.src_x;
    if constexpr (SCHEME == kWave || SCHEME == kGradient)
        if (src_x >= 0 && !source_amplitude(a, w_src))
            src_x = -1;
    const int ucol = 4 + kVX * tx;
    auto urow = [&](int rel_row) { return (R + kRPT * wid + rel_row) * kBoxW + ucol; };
    uint32_t ucn = 0, ccn = 0;  // u planes / centre-field planes consumed before this segment
    bool good = true;
    while (good && cur.template next<C::TY>(a, sg)) {
        const int x0 = sg.x0, y0 = sg.y0, zs = sg.zs, ze = sg.ze;
        const int pu0 = zs - R;  // first u plane of the queue
        auto u_cnt = [&](int p) { return ucn + (uint32_t)(p - pu0); };
        auto u_stage = [&](int p) { return u_cnt(p) % C::NSU; };
        auto u_phase = [&](int p) { return (u_cnt(p) / C::NSU) & 1; };
        auto release_u = [&](int p) {
            __syncwarp();
            if (tx == 0)
                mbar_arrive(&uempty[u_stage(p)]);
        };

        // register queue: in iteration z, q[r][i] = u(z - R + i) at row 4 wid + r
        float2 q[kRPT][Q];
#pragma unroll
        for (int r = 0; r < kRPT; ++r)
            q[r][2 * R] = make_float2(0.0f, 0.0f);
        for (int i = 0; i < 2 * R && good; ++i) {
            const int p = pu0 + i;
            good = mbar_wait(&ufull[u_stage(p)], u_phase(p));
            if (!good)
                break;
            const float *P = us + u_stage(p) * C::kUStage;
#pragma unroll
            for (int r = 0; r < kRPT; ++r) {
#pragma unroll
                for (int j = 0; j < 2 * R; ++j)  // shift towards 0, newest at 2R:
                    q[r][j] = q[r][j + 1];       // ends with q[1 .. 2R] = u(zs-R .. zs+R-1)
                q[r][2 * R] = *reinterpret_cast<const float2 *>(P + urow(r));
            }
            if (p < zs)  // planes before the segment are only queue inputs
                release_u(p);
        }

        const int x = x0 + kVX * tx;  // first of the thread's two columns
        const bool x_ok = x < a.nx;   // nx is a multiple of 4: both columns or neither
        bool in_x[kVX];
#pragma unroll
        for (int c = 0; c < kVX; ++c)
            in_x[c] = (x + c) >= R && (x + c) < a.nx - R;
        const int wy0 = y0 + kRPT * wid;  // the warp's first row
        bool row_ok[kRPT], in_y[kRPT];
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            row_ok[r] = x_ok && wy0 + r < a.ny;
            in_y[r] = wy0 + r >= R && wy0 + r < a.ny - R;
        }
        // every point of the warp's 64 x 4 block is interior in x and y
        const bool warp_in = x0 >= R && x0 + kTX <= a.nx - R && wy0 >= R && wy0 + kRPT <= a.ny - R;
        const bool src_in_warp =
            a.src_x >= x0 && a.src_x < x0 + kTX && a.src_y >= wy0 && a.src_y < wy0 + kRPT;

        // Fused encode, after the fourth plane of each layer (segments are
        // whole layers): the consumer warps meet, the threads of the tile's
        // blocks each encode one 4x4x4 block from the layer in shared memory,
        // the warps meet again and copy the words out, a block row of the tile
        // being one contiguous run of the out slot.  Every consumer warp
        // passes both barriers of every layer, also after a wait has run out.
        [[maybe_unused]] auto enc_layer_end = [&](int z) {
            if (((z - zs) & 3) != 3)
                return;
            constexpr int NBX = kTX / 4, NBY = C::TY / 4;
            const int t = 32 * wid + tx;
            const int nw = 2 * a.enc_rate;
            named_bar_sync(1, 32 * CW);
            if (good && t < NBX * NBY) {
                const int bx = t % NBX, by = t / NBX;
                if (x0 + 4 * bx < a.nx && y0 + 4 * by < a.ny) {
                    float v[64];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 f =
                                *reinterpret_cast<const float4 *>(lay + (k * C::TY + 4 * by + j) * kTX + 4 * bx);
                            v[16 * k + 4 * j + 0] = f.x;
                            v[16 * k + 4 * j + 1] = f.y;
                            v[16 * k + 4 * j + 2] = f.z;
                            v[16 * k + 4 * j + 3] = f.w;
                        }
                    uint32_t *row = rows + t * C::kEncStride;
                    if (!encode_block(v, a.enc_rate, dbl, [&](int i, uint32_t w) { row[i] = w; }))
                        atomicOr(&g_device_error, kErrNonFinite);
                }
            }
            named_bar_sync(1, 32 * CW);
            if (good) {
                const int64_t BX = a.nx / 4, BY = a.ny / 4;
                const int64_t layer = (a.gz0 + z - 3) / 4 - a.enc_layer0;
                const int nbv = min(NBX, (a.nx - x0) / 4);
                for (int by = 0; by < NBY && y0 + 4 * by < a.ny; ++by) {
                    uint32_t *dst = a.enc_out + ((layer * BY + (y0 / 4 + by)) * BX + x0 / 4) * nw;
                    const uint32_t *src = rows + by * NBX * C::kEncStride;
                    for (int w = t; w < nbv * nw; w += 32 * CW)
                        dst[w] = src[(w / nw) * C::kEncStride + w % nw];
                }
            }
        };

        for (int z = zs; (ENC || good) && z < ze; ++z) {
            const int pn = z + R;
            if (good)
                good = mbar_wait(&ufull[u_stage(pn)], u_phase(pn));
            const uint32_t cc = ccn + (uint32_t)(z - zs);
            const int cst = (int)(cc % C::NSC);
            if (NCF > 0 && good)
                good = mbar_wait(&cfull[cst], (cc / C::NSC) & 1);
            if (!good) {
                if constexpr (ENC) {
                    enc_layer_end(z);
                    continue;
                }
                break;
            }
            const float *Pn = us + u_stage(pn) * C::kUStage;
            const float *P = us + u_stage(z) * C::kUStage;
            const int gz = a.gz0 + z;
            const bool z_interior = gz >= R && gz < a.nz - R;
#pragma unroll
            for (int r = 0; r < kRPT; ++r) {
#pragma unroll
                for (int j = 0; j < 2 * R; ++j)
                    q[r][j] = q[r][j + 1];
                q[r][2 * R] = *reinterpret_cast<const float2 *>(Pn + urow(r));
            }
            // y neighbours outside the thread's rows: R rows above, R below
            float2 above[R], below[R];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                above[d - 1] = *reinterpret_cast<const float2 *>(P + urow(-d));
                below[d - 1] = *reinterpret_cast<const float2 *>(P + urow(kRPT - 1 + d));
            }
            [[maybe_unused]] const bool rcv_plane = SCHEME == kAdjoint && a.res != nullptr && gz == a.zr;
            auto rows = [&](auto FAST) {
                constexpr bool kFast = decltype(FAST)::value;
#pragma unroll
                for (int r = 0; r < kRPT; ++r) {
                    if (!kFast && !row_ok[r])
                        continue;
                    float xv[10];  // columns x-4 .. x+5 of row r (five 64-bit loads)
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        const float2 v = *reinterpret_cast<const float2 *>(P + urow(r) - 4 + 2 * i);
                        xv[2 * i] = v.x;
                        xv[2 * i + 1] = v.y;
                    }
                    const float2 uc = q[r][R];
                    const int y = wy0 + r;
                    float2 cv[NCF > 0 ? NCF : 1];
                    if constexpr (NCF > 0) {
                        const int ci = cst * C::kCStage + (kRPT * wid + r) * kTX + kVX * tx;
#pragma unroll
                        for (int f = 0; f < NCF; ++f)
                            cv[f] = *reinterpret_cast<const float2 *>(cs + f * C::NSC * C::kCStage + ci);
                    }
                    [[maybe_unused]] float2 rv = make_float2(0.0f, 0.0f);
                    if constexpr (SCHEME == kAdjoint && !kFast) {
                        if (rcv_plane)
                            rv = __ldg(reinterpret_cast<const float2 *>(a.res + (int64_t)y * a.nx + x));
                    }
                    if constexpr (kFast) {
                        // every point interior, no source or receiver: the pair of
                        // x-adjacent points in packed f32x2 operations
                        float2 s2[R + 1];
                        s2[0] = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int d = 1; d <= R; ++d) {
                            const float2 ym = (r - d >= 0) ? q[(r - d) >= 0 ? r - d : 0][R]
                                                           : above[(d - r - 1) >= 0 ? d - r - 1 : 0];
                            const float2 yp = (r + d < kRPT) ? q[(r + d) < kRPT ? r + d : 0][R]
                                                             : below[(r + d - kRPT) >= 0 ? r + d - kRPT : 0];
                            s2[d] = nbr_sum2(make_float2(xv[4 - d], xv[5 - d]), make_float2(xv[4 + d], xv[5 + d]),
                                             ym, yp, q[r][R - d], q[r][R + d]);
                        }
                        const float2 L2 = star_L2<R>(a.c, uc, s2);
                        float2 o2;
                        if constexpr (SCHEME == kHeat) {
                            o2 = L2;
                        } else if constexpr (SCHEME == kWave) {
                            o2 = wave_update2(L2, uc, cv[0], cv[1]);
                        } else if constexpr (SCHEME == kAdjoint) {
                            o2 = adjoint_update2(L2, cv[2], cv[0]);
                        } else {
                            o2 = fma2_rn(cv[1], L2, cv[0]);
                        }
                        const int64_t o = (int64_t)z * a.plane + (int64_t)y * a.nx + x;
                        *reinterpret_cast<float2 *>(a.out + o) = o2;
                        if constexpr (SCHEME == kAdjoint)
                            if (a.out2)
                                *reinterpret_cast<float2 *>(a.out2 + o) = fmul2_rn(cv[1], o2);
                        continue;
                    }
                    float res[kVX];
                    [[maybe_unused]] float res2[kVX];
#pragma unroll
                    for (int c = 0; c < kVX; ++c) {
                        const float u = c ? uc.y : uc.x;
                        // shell: heat / wave keep u (Dirichlet), the adjoint is
                        // zero there, the gradient keeps its value
                        if constexpr (SCHEME == kAdjoint) {
                            res[c] = 0.0f;
                            res2[c] = 0.0f;
                        } else if constexpr (SCHEME == kGradient) {
                            res[c] = c ? cv[0].y : cv[0].x;
                        } else {
                            res[c] = u;
                        }
                        if (kFast || (z_interior && in_y[r] && in_x[c])) {
                            float s[R + 1];
                            s[0] = 0.0f;
#pragma unroll
                            for (int d = 1; d <= R; ++d) {
                                const float2 ym = (r - d >= 0) ? q[(r - d) >= 0 ? r - d : 0][R]
                                                               : above[(d - r - 1) >= 0 ? d - r - 1 : 0];
                                const float2 yp = (r + d < kRPT) ? q[(r + d) < kRPT ? r + d : 0][R]
                                                                 : below[(r + d - kRPT) >= 0 ? r + d - kRPT : 0];
                                const float2 zm = q[r][R - d];
                                const float2 zp = q[r][R + d];
                                s[d] = nbr_sum(xv[4 + c - d], xv[4 + c + d], c ? ym.y : ym.x, c ? yp.y : yp.x,
                                               c ? zm.y : zm.x, c ? zp.y : zp.x);
                            }
                            const float L = star_L<R>(a.c, u, s);
                            [[maybe_unused]] const bool at_src =
                                !kFast && (x + c == src_x && y == a.src_y && z == a.src_zw);
                            if constexpr (SCHEME == kHeat) {
                                res[c] = L;
                            } else if constexpr (SCHEME == kWave) {
                                res[c] = wave_update(L, u, c ? cv[0].y : cv[0].x, c ? cv[1].y : cv[1].x, at_src,
                                                     w_src);
                            } else if constexpr (SCHEME == kAdjoint) {
                                res[c] = adjoint_update(L, c ? cv[2].y : cv[2].x, c ? cv[0].y : cv[0].x,
                                                        !kFast && rcv_plane, c ? rv.y : rv.x);
                                res2[c] = fmul_rn(c ? cv[1].y : cv[1].x, res[c]);
                            } else {
                                res[c] = gradient_update(L, c ? cv[1].y : cv[1].x, c ? cv[0].y : cv[0].x, at_src,
                                                         w_src);
                            }
                        }
                    }
                    if constexpr (ENC) {
                        *reinterpret_cast<float2 *>(lay + (((z - zs) & 3) * C::TY + kRPT * wid + r) * kTX +
                                                    kVX * tx) = make_float2(res[0], res[1]);
                        continue;
                    }
                    const int64_t o = (int64_t)z * a.plane + (int64_t)y * a.nx + x;
                    *reinterpret_cast<float2 *>(a.out + o) = make_float2(res[0], res[1]);
                    if constexpr (SCHEME == kAdjoint)
                        if (a.out2)
                            *reinterpret_cast<float2 *>(a.out2 + o) = make_float2(res2[0], res2[1]);
                }
            };
            if (kFastPath && warp_in && z_interior && !(src_in_warp && z == a.src_zw) && !rcv_plane)
                rows(std::true_type{});
            else
                rows(std::false_type{});
            // plane z (xy neighbours) and its centre-field stage are done
            __syncwarp();
            if (tx == 0) {
                mbar_arrive(&uempty[u_stage(z)]);
                if (NCF > 0)
                    mbar_arrive(&cempty[cst]);
            }
            if constexpr (ENC)
                enc_layer_end(z);
        }
        if (!good)
            break;
        // the last R planes only fed the queue
        for (int p = ze; p < ze + R; ++p)
            release_u(p);
        ucn += (uint32_t)(ze - zs + 2 * R);
        ccn += NCF > 0 ? (uint32_t)(ze - zs) : 0u;
    }
}

// Two heat steps in one z-march (kernel-level temporal blocking of the
// 7-point stencil, Sec. 3.1 / Fig. 1b applied on chip): steps j and j+1 of a
// visit read the step j-1 planes once and write the step j+1 planes once; the
// step j planes live only in shared memory.  A CTA's output is a 64 x 16 tile
// (as in k_star_step); it computes step j on the tile plus a one-point x-y
// halo (66 x 18, the halo points recomputed by the neighbouring tiles too)
// from step j-1 values on a two-point halo (72 x 20 TMA boxes).
//
// Consumer thread (tx, w) owns the 2 x 4 points x0 + 2 tx + {0, 1},
// y0 + 4 w + {0..3} of both steps, keeps their step j-1 and step j values of
// three consecutive planes in register queues (the z neighbours), and takes
// x-y neighbours from shared memory; the 164 halo points of a step j plane
// are split over the four warps.  Per output plane z: step j plane z+1 is
// computed into a three-plane ring, the consumer warps meet at a named
// barrier, and output plane z is computed.  Every point goes through the same
// operations as in k_star_step<1, kHeat> (shell and out-of-grid points copy
// their input), and a step j value outside step j's trapezoid is never read
// by an interior output point, so the result is bit-identical to two single
// steps.
constexpr int kH2InW = kBoxW;            // 72: input row, x0 - 4 .. x0 + 67
constexpr int kH2InH = kTY + 4;          // 20: input rows, y0 - 2 .. y0 + 17
constexpr int kH2MidH = kTY + 2;         // 18: step j rows, y0 - 1 .. y0 + 16
constexpr int kH2NS = 6;                 // input ring stages
constexpr int kH2NM = 3;                 // step j ring planes
constexpr uint32_t kH2InBytes = kH2InW * kH2InH * 4;
constexpr int kH2InStage = ((kH2InBytes + 127) / 128 * 128) / 4;   // floats
constexpr int kH2MidPlane = kH2InW * kH2MidH;                     // floats
constexpr size_t kH2Smem = 128 + (size_t)kH2NS * kH2InStage * 4 + (size_t)kH2NM * kH2MidPlane * 4 + 2 * kH2NS * 8;

// one heat point: the step-kernel arithmetic (nbr_sum, star_L<1>)
OOCS_FN float heat_point(const StarCoef &c, float u, float xm, float xp, float ym, float yp, float zm, float zp)
{
    float sd[2];
    sd[0] = 0.0f;
    sd[1] = nbr_sum(xm, xp, ym, yp, zm, zp);
    return star_L<1>(c, u, sd);
}

__global__ void __launch_bounds__(kStepThreads, 3)
    k_heat_step2(const __grid_constant__ CUtensorMap tm_in, const StepArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    float *ins = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *mids = ins + kH2NS * kH2InStage;
    uint64_t *full = reinterpret_cast<uint64_t *>(mids + kH2NM * kH2MidPlane);
    uint64_t *empty = full + kH2NS;
    const int tx = threadIdx.x, wid = threadIdx.y;
    if (wid == 0 && tx == 0) {
        for (int i = 0; i < kH2NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kConsumerWarps);
        }
        fence_barrier_init();
    }
    __syncthreads();
    pdl_launch_dependents();
    pdl_wait_prior_grid();

    SegCursor cur;
    cur.init(a);
    StepSeg sg;
    if (wid == kConsumerWarps) {
        // ------------------------------------------------ producer warp --
        if (tx != 0)
            return;
        bool good = true;
        uint32_t n = 0;  // input planes issued so far
        while (good && cur.next(a, sg)) {
            for (int p = sg.zs - 2; p < sg.ze + 2; ++p) {
                const uint32_t st = n % kH2NS, k = n / kH2NS;
                if (k > 0 && !mbar_wait(&empty[st], (k - 1) & 1)) {
                    good = false;
                    break;
                }
                mbar_arrive_expect_tx(&full[st], kH2InBytes);
                tma_load_3d(ins + st * kH2InStage, &tm_in, sg.x0 - 4, sg.y0 - 2, p, &full[st]);
                ++n;
            }
        }
        for (uint32_t i = n > (uint32_t)kH2NS ? n - kH2NS : 0; i < n; ++i)
            mbar_wait(&full[i % kH2NS], (i / kH2NS) & 1);
        return;
    }

    // --------------------------------------------------- consumer warps --
    // A wait that runs out (kErrWaitTimeout) only stops the computing: every
    // consumer warp still passes the same sequence of named barriers, so no
    // warp is left waiting at one for a warp that gave up.
    const StarCoef c = a.c;
    uint32_t icn = 0;  // input planes consumed before this segment
    uint32_t mcn = 0;  // step j planes computed before this segment
    bool good = true;
    const int col0 = 4 + kVX * tx;  // the thread's first column (72-wide rows)
    while (cur.next(a, sg)) {
        const int x0 = sg.x0, y0 = sg.y0, zs = sg.zs, ze = sg.ze;
        const int pi0 = zs - 2;  // first input plane of the segment
        auto in_slot = [&](int p) { return (icn + (uint32_t)(p - pi0)) % kH2NS; };
        auto in_phase = [&](int p) { return ((icn + (uint32_t)(p - pi0)) / kH2NS) & 1; };
        auto in_plane = [&](int p) { return ins + in_slot(p) * kH2InStage; };
        auto mid_plane = [&](int q) { return mids + ((mcn + (uint32_t)(q - (zs - 1))) % kH2NM) * kH2MidPlane; };
        auto wait_in = [&](int p) {
            if (good)
                good = __all_sync(0xffffffffu, mbar_wait(&full[in_slot(p)], in_phase(p)));
        };
        auto release = [&](int p) {
            __syncwarp();
            if (tx == 0)
                mbar_arrive(&empty[in_slot(p)]);
        };
        auto interior = [&](int x, int y, int gz) {
            return x >= 1 && x < a.nx - 1 && y >= 1 && y < a.ny - 1 && gz >= 1 && gz < a.nz - 1;
        };
        const int x = x0 + kVX * tx;
        const int wy0 = y0 + kRPT * wid;
        // queues of the thread's own points: step j-1 (in) and step j (mid)
        // values of planes p-1, p, p+1 around the plane being computed
        float2 inq[kRPT][3], midq[kRPT][3];
        auto load_in_own = [&](int p, float2 (&dst)[kRPT]) {
            const float *P = in_plane(p);
#pragma unroll
            for (int r = 0; r < kRPT; ++r)
                dst[r] = *reinterpret_cast<const float2 *>(P + (2 + kRPT * wid + r) * kH2InW + col0);
        };
        // step j plane q: own points from the queue inq (planes q-1, q, q+1
        // at slots 0..2), halo points from the ring; written to the mid ring
        auto mid_step = [&](int q) {
            const float *P0 = in_plane(q);
            float *M = mid_plane(q);
            const int gz = a.gz0 + q;
#pragma unroll
            for (int r = 0; r < kRPT; ++r) {
                const int y = wy0 + r;
                const int ir = 2 + kRPT * wid + r;  // input row
                const float2 u = inq[r][1];
                const float2 ym = (r > 0) ? inq[r > 0 ? r - 1 : 0][1]
                                          : *reinterpret_cast<const float2 *>(P0 + (ir - 1) * kH2InW + col0);
                const float2 yp = (r < kRPT - 1) ? inq[r < kRPT - 1 ? r + 1 : 0][1]
                                                 : *reinterpret_cast<const float2 *>(P0 + (ir + 1) * kH2InW + col0);
                // x neighbours: the next lane's columns (loads only at the warp's edges)
                float xl = __shfl_up_sync(0xffffffffu, u.y, 1), xr = __shfl_down_sync(0xffffffffu, u.x, 1);
                if (tx == 0)
                    xl = P0[ir * kH2InW + col0 - 1];
                if (tx == 31)
                    xr = P0[ir * kH2InW + col0 + 2];
                float2 m;
                m.x = interior(x, y, gz) ? heat_point(c, u.x, xl, u.y, ym.x, yp.x, inq[r][0].x, inq[r][2].x) : u.x;
                m.y = interior(x + 1, y, gz) ? heat_point(c, u.y, u.x, xr, ym.y, yp.y, inq[r][0].y, inq[r][2].y)
                                             : u.y;
                midq[r][2] = m;
                *reinterpret_cast<float2 *>(M + (1 + kRPT * wid + r) * kH2InW + col0) = m;
            }
            // halo: warp 0 row y0-1, warp 3 row y0+16 (columns x0-1 .. x0+64),
            // warp 1 column x0-1, warp 2 column x0+64 (rows y0 .. y0+15)
            const float *Pm = in_plane(q - 1), *Pp = in_plane(q + 1);
            auto halo = [&](int mrow, int col) {
                const int ir = mrow + 1;
                const int o = ir * kH2InW + col;
                const float u = P0[o];
                const int hx = x0 - 4 + col, hy = y0 - 1 + mrow;
                M[mrow * kH2InW + col] =
                    interior(hx, hy, gz) ? heat_point(c, u, P0[o - 1], P0[o + 1], P0[o - kH2InW], P0[o + kH2InW],
                                                      Pm[o], Pp[o])
                                         : u;
            };
            if (wid == 0 || wid == kConsumerWarps - 1) {
                // a halo row: the pair of columns of each lane as in mid_step's
                // own points, then the two end columns
                const int mrow = wid == 0 ? 0 : kH2MidH - 1;
                const int ir = mrow + 1;
                const int o = ir * kH2InW + col0;
                const float2 u = *reinterpret_cast<const float2 *>(P0 + o);
                const float2 ym = *reinterpret_cast<const float2 *>(P0 + o - kH2InW);
                const float2 yp = *reinterpret_cast<const float2 *>(P0 + o + kH2InW);
                const float2 zm = *reinterpret_cast<const float2 *>(Pm + o);
                const float2 zp = *reinterpret_cast<const float2 *>(Pp + o);
                float xl = __shfl_up_sync(0xffffffffu, u.y, 1), xr = __shfl_down_sync(0xffffffffu, u.x, 1);
                if (tx == 0)
                    xl = P0[o - 1];
                if (tx == 31)
                    xr = P0[o + 2];
                const int hy = y0 - 1 + mrow;
                float2 m;
                m.x = interior(x, hy, gz) ? heat_point(c, u.x, xl, u.y, ym.x, yp.x, zm.x, zp.x) : u.x;
                m.y = interior(x + 1, hy, gz) ? heat_point(c, u.y, u.x, xr, ym.y, yp.y, zm.y, zp.y) : u.y;
                *reinterpret_cast<float2 *>(M + mrow * kH2InW + col0) = m;
                if (tx < 2)
                    halo(mrow, tx == 0 ? 3 : 4 + kTX);
            } else if (tx < kTY) {
                halo(1 + tx, wid == 1 ? 3 : 4 + kTX);
            }
        };
        // the previous segment's output planes are done before its step j
        // planes are overwritten
        named_bar_sync(1, 32 * kConsumerWarps);
        // prologue: input planes zs-2 .. zs+1 and step j planes zs-1, zs
        for (int p = zs - 2; p <= zs + 1; ++p)
            wait_in(p);
        if (good) {
            float2 t[kRPT];
            load_in_own(zs - 2, t);
#pragma unroll
            for (int r = 0; r < kRPT; ++r)
                inq[r][0] = t[r];
            load_in_own(zs - 1, t);
#pragma unroll
            for (int r = 0; r < kRPT; ++r)
                inq[r][1] = t[r];
            load_in_own(zs, t);
#pragma unroll
            for (int r = 0; r < kRPT; ++r)
                inq[r][2] = t[r];
            mid_step(zs - 1);
#pragma unroll
            for (int r = 0; r < kRPT; ++r) {
                midq[r][1] = midq[r][2];
                inq[r][0] = inq[r][1];
                inq[r][1] = inq[r][2];
            }
            load_in_own(zs + 1, t);
#pragma unroll
            for (int r = 0; r < kRPT; ++r)
                inq[r][2] = t[r];
            mid_step(zs);
        }
        release(zs - 2);
        release(zs - 1);
        for (int z = zs; z < ze; ++z) {
            // queues: midq[.][1] = mid(z-1), midq[.][2] = mid(z); inq = in(z-1 .. z+1)
            wait_in(z + 2);
            if (good) {
                float2 t[kRPT];
                load_in_own(z + 2, t);
#pragma unroll
                for (int r = 0; r < kRPT; ++r) {
                    midq[r][0] = midq[r][1];
                    midq[r][1] = midq[r][2];
                    inq[r][0] = inq[r][1];
                    inq[r][1] = inq[r][2];
                    inq[r][2] = t[r];
                }
                mid_step(z + 1);  // midq[.][2] = mid(z+1)
            }
            release(z);
            named_bar_sync(1, 32 * kConsumerWarps);  // step j planes z-1 .. z+1 are complete
            if (!good)
                continue;
            const float *M0 = mid_plane(z);
            const int gz = a.gz0 + z;
#pragma unroll
            for (int r = 0; r < kRPT; ++r) {
                const int y = wy0 + r;
                const int mr = 1 + kRPT * wid + r;  // mid row
                const float2 u = midq[r][1];
                const float2 ym = (r > 0) ? midq[r > 0 ? r - 1 : 0][1]
                                          : *reinterpret_cast<const float2 *>(M0 + (mr - 1) * kH2InW + col0);
                const float2 yp = (r < kRPT - 1) ? midq[r < kRPT - 1 ? r + 1 : 0][1]
                                                 : *reinterpret_cast<const float2 *>(M0 + (mr + 1) * kH2InW + col0);
                float xl = __shfl_up_sync(0xffffffffu, u.y, 1), xr = __shfl_down_sync(0xffffffffu, u.x, 1);
                if (tx == 0)
                    xl = M0[mr * kH2InW + col0 - 1];
                if (tx == 31)
                    xr = M0[mr * kH2InW + col0 + 2];
                float2 o;
                o.x = interior(x, y, gz) ? heat_point(c, u.x, xl, u.y, ym.x, yp.x, midq[r][0].x, midq[r][2].x) : u.x;
                o.y = interior(x + 1, y, gz) ? heat_point(c, u.y, u.x, xr, ym.y, yp.y, midq[r][0].y, midq[r][2].y)
                                             : u.y;
                if (x < a.nx && y < a.ny)
                    *reinterpret_cast<float2 *>(a.out + (int64_t)z * a.plane + (int64_t)y * a.nx + x) = o;
            }
        }
        // input planes ze and ze+1 only fed the last step j plane
        release(ze);
        release(ze + 1);
        icn += (uint32_t)(ze - zs + 4);
        mcn += (uint32_t)(ze - zs + 2);
    }
}

// ---- host side: tensor maps and launch geometry

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// [planes][ny][nx] FP32 buffer, box (bw, bh, 1), zero fill out of bounds
static cudaError_t make_plane_map(CUtensorMap *m, const float *base, int64_t nx, int64_t ny,
                                  int64_t planes, uint32_t bw, uint32_t bh)
{
    auto enc = tensor_map_encoder();
    if (!enc)
        return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (nx * 4) % 16)
        return cudaErrorMisalignedAddress;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(nx * 4), (cuuint64_t)(nx * ny * 4)};
    cuuint32_t box[3] = {bw, bh, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Per-device launch facts, looked up once per device ordinal (a process may
// drive several GPUs, from several host threads): the SM count, and for each
// step-kernel instance whether its dynamic shared-memory opt-in was applied on
// that device (cudaFuncSetAttribute acts on the current device only) and how
// many of its CTAs fit on an SM.
constexpr int kMaxDevices = 64;
constexpr int kStepInstances = 17;  // (radius, scheme, tile) instances of k_star_step + the fused encode

struct DevInfo {
    int sms = 0;
    int resident[kStepInstances] = {};  // 0: not yet opted in on this device
};

static std::mutex g_dev_mu;
static DevInfo g_dev[kMaxDevices];

static cudaError_t current_device(int &dev)
{
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices))
        e = cudaErrorInvalidDevice;
    return e;
}

// SM count of the current device (0 if it cannot be read).
static int device_sms()
{
    int dev = 0;
    if (current_device(dev) != cudaSuccess)
        return 0;
    std::lock_guard<std::mutex> lock(g_dev_mu);
    DevInfo &info = g_dev[dev];
    if (info.sms == 0 && cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        info.sms = 0;
    return info.sms;
}

template <int R, int SCHEME, int CW, bool ENC = false>
constexpr int step_instance() { return ENC ? 16 : (R == 4 ? 4 : 0) + SCHEME + (CW == kConsumerWarps ? 0 : 8); }

// Applies the step kernel's shared-memory opt-in on the current device (once
// per device) and returns its CTAs per SM and the device's SM count.
template <int R, int SCHEME, int CW, bool ENC = false>
static cudaError_t step_residency(int &resident, int &sms)
{
    using C = StepCfg<R, centre_fields<SCHEME>(), CW>;
    static_assert(step_instance<R, SCHEME, CW, ENC>() < kStepInstances, "instance table too small");
    int dev = 0;
    cudaError_t e = current_device(dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(g_dev_mu);
    DevInfo &info = g_dev[dev];
    if (info.sms == 0) {
        e = cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
    }
    int &res = info.resident[step_instance<R, SCHEME, CW, ENC>()];
    if (res == 0) {
        const size_t smem = C::smem_bytes() + (ENC ? C::enc_bytes() : 0);
        auto kern = k_star_step<R, SCHEME, CW, ENC>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * (CW + 1), smem);
        if (e != cudaSuccess)
            return e;
        if (n < 1)
            return cudaErrorInvalidConfiguration;
        res = n;
    }
    resident = res;
    sms = info.sms;
    return cudaSuccess;
}

// Launch geometry of a z-march over window planes [a.z_lo, a.z_hi) of an
// nx x ny grid of 64 x ty tiles, with `slots` CTAs resident at once.
// Chunked launch when some z chunking (>= min_planes per CTA) fills the last
// wave of CTAs to 90 %; otherwise (short windows on a plane whose tiles do not
// fill the SMs evenly, e.g. 256 tiles on 304 slots) one wave of equal
// tile-plane ranges.  Sets a.zchunk, a.tiles_y and a.ntiles.
static dim3 step_grid(int64_t nx, int64_t ny, int slots, StepArgs &a, int min_planes = 12, int ty = kTY)
{
    const int tiles_x = (int)((nx + kTX - 1) / kTX);
    const int tiles_y = (int)((ny + ty - 1) / ty);
    const int tiles = tiles_x * tiles_y;
    const int nplanes = a.z_hi - a.z_lo;
    a.tiles_y = tiles_y;
    a.ntiles = tiles;
    int best = 1;
    double best_eff = 0.0;
    const int max_chunks = std::max(1, nplanes / min_planes);
    for (int nc = 1; nc <= max_chunks && nc <= 64; ++nc) {
        const int zc = (nplanes + nc - 1) / nc;
        const int real = (nplanes + zc - 1) / zc;
        const long total = (long)tiles * real;
        const long waves = (total + slots - 1) / slots;
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = nc;
        }
    }
    if (best_eff >= 0.9) {
        a.zchunk = (nplanes + best - 1) / best;
        return dim3(tiles_x, tiles_y, (nplanes + a.zchunk - 1) / a.zchunk);
    }
    a.zchunk = 0;
    const int64_t total = (int64_t)tiles * nplanes;
    return dim3((unsigned)std::min<int64_t>(slots, (total + 15) / 16), 1, 1);
}

// Launch geometry of the fused-encode step: always chunked, every chunk a
// whole number of 4-plane layers (at least three), the chunk count chosen for
// the fullest last wave of CTAs.
static dim3 enc_grid(int64_t nx, int64_t ny, int slots, StepArgs &a, int ty)
{
    const int tiles_x = (int)((nx + kTX - 1) / kTX);
    const int tiles_y = (int)((ny + ty - 1) / ty);
    const int tiles = tiles_x * tiles_y;
    const int layers = (a.z_hi - a.z_lo) / 4;
    a.tiles_y = tiles_y;
    a.ntiles = tiles;
    int best = 1;
    double best_eff = 0.0;
    for (int nc = 1; nc <= std::max(1, layers / 3) && nc <= 64; ++nc) {
        const int lc = (layers + nc - 1) / nc;
        const int real = (layers + lc - 1) / lc;
        const long total = (long)tiles * real;
        const long waves = (total + slots - 1) / slots;
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = nc;
        }
    }
    const int lc = (layers + best - 1) / best;
    a.zchunk = 4 * lc;
    return dim3(tiles_x, tiles_y, (layers + lc - 1) / lc);
}

template <int R, int SCHEME, int CW = kConsumerWarps, bool ENC = false>
static cudaError_t launch_step_t(const StepLaunch &L, StepArgs a, cudaStream_t s)
{
    using C = StepCfg<R, centre_fields<SCHEME>(), CW>;
    const size_t smem = C::smem_bytes() + (ENC ? C::enc_bytes() : 0);
    auto kern = k_star_step<R, SCHEME, CW, ENC>;
    int resident = 0, sms = 0;
    {
        cudaError_t e = step_residency<R, SCHEME, CW, ENC>(resident, sms);
        if (e != cudaSuccess)
            return e;
    }
    constexpr int NCF = centre_fields<SCHEME>();
    CUtensorMap mc, mp, mm, m2;
    cudaError_t e = make_plane_map(&mc, L.cur, L.nx, L.ny, L.wp, kBoxW, C::H);
    if (e == cudaSuccess)
        e = make_plane_map(&mp, NCF >= 1 ? L.prev : L.cur, L.nx, L.ny, L.wp, kTX, C::TY);
    if (e == cudaSuccess)
        e = make_plane_map(&mm, NCF >= 2 ? L.m : L.cur, L.nx, L.ny, L.wp, kTX, C::TY);
    if (e == cudaSuccess)
        e = make_plane_map(&m2, NCF >= 3 ? L.c2 : L.cur, L.nx, L.ny, L.wp, kTX, C::TY);
    if (e != cudaSuccess)
        return e;

    const dim3 grid = ENC ? enc_grid(L.nx, L.ny, sms * resident, a, C::TY)
                          : step_grid(L.nx, L.ny, sms * resident, a, 12, C::TY);
    dim3 block(32, CW + 1, 1);
    return launch_pdl(kern, grid, block, smem, s, mc, mp, mm, m2, a);
}

cudaError_t launch_heat_step2(const StepLaunch &L, cudaStream_t s)
{
    if (L.z_hi <= L.z_lo)
        return cudaSuccess;
    if (L.scheme != kHeat || L.radius != 1)
        return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = current_device(dev);
    if (e != cudaSuccess)
        return e;
    int resident = 0, sms = 0;
    {
        static int res_dev[kMaxDevices] = {};
        std::lock_guard<std::mutex> lock(g_dev_mu);
        DevInfo &info = g_dev[dev];
        if (info.sms == 0 && (e = cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        if (res_dev[dev] == 0) {
            e = cudaFuncSetAttribute(k_heat_step2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kH2Smem);
            if (e != cudaSuccess)
                return e;
            int n = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_heat_step2, kStepThreads, kH2Smem);
            if (e != cudaSuccess)
                return e;
            if (n < 1)
                return cudaErrorInvalidConfiguration;
            res_dev[dev] = n;
        }
        resident = res_dev[dev];
        sms = info.sms;
    }
    CUtensorMap m;
    e = make_plane_map(&m, L.cur, L.nx, L.ny, L.wp, kH2InW, kH2InH);
    if (e != cudaSuccess)
        return e;
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.out = L.out;
    a.nx = (int)L.nx;
    a.ny = (int)L.ny;
    a.nz = (int)L.nz;
    a.plane = L.nx * L.ny;
    a.gz0 = (int)L.gz0;
    a.z_lo = (int)L.z_lo;
    a.z_hi = (int)L.z_hi;
    for (int i = 0; i < 5; ++i)
        a.c.c[i] = L.coef[i];
    a.src_x = a.src_y = a.src_zw = -1;
    // a segment re-reads a 4-plane z halo and recomputes two step j planes:
    // keep z chunks long
    const dim3 grid = step_grid(L.nx, L.ny, sms * resident, a, 24);
    return launch_pdl(k_heat_step2, grid, dim3(32, kConsumerWarps + 1, 1), kH2Smem, s, m, a);
}

// Decode fused into the first heat step of a visit (radius 1, transform
// codec; the opt-in oocs_desc.codec_fusion): the window's codec blocks are
// decoded into shared memory, a 4-plane layer at a time, and step 1 reads
// them there, so the decoded window is never written to HBM.  A CTA of four
// warps owns a 64 x 16 tile and a z chunk of step 1's planes; it keeps two
// decoded layers of the tile plus a one-block halo (72 x 24 points: 18 x 6
// blocks, the halo blocks decoded again by the neighbouring tiles) and
// decodes the next layer when the plane after the current one needs it.
// Thread (tx, w) updates the 2 x 4 points x0 + 2 tx + {0, 1}, y0 + 4 w +
// {0..3} with the operations of k_star_step<1, kHeat> in the same order
// (shell and out-of-grid points keep their input), so the result equals the
// separate decode and step bit for bit.
constexpr int kDSW = kTX + 8;      // 72: decoded columns, x0 - 4 .. x0 + 67
constexpr int kDSH = kTY + 8;      // 24: decoded rows, y0 - 4 .. y0 + 19
constexpr int kDSBX = kDSW / 4;    // 18 blocks across
constexpr int kDSBY = kDSH / 4;    // 6 blocks down
constexpr int kDSLayer = 4 * kDSH * kDSW;  // floats per decoded layer
constexpr size_t kDSSmem = (size_t)2 * kDSLayer * 4;

struct DecStepArgs {
    float *out;                 // step 1 result, window buffer
    const uint32_t *blk[2];     // codec blocks of window layers [0, nl0) and [nl0, nl0 + nl1)
    int nl0, nl1;
    int nx, ny, nz;
    int gz0, wp;                // global plane of window plane 0; window planes
    int z_lo, z_hi, zchunk;
    int rate;
    StarCoef c;
};

__global__ void __launch_bounds__(32 * kConsumerWarps, 3) k_decode_heat_step(const DecStepArgs a)
{
    extern __shared__ float dsm[];
    pdl_launch_dependents();
    pdl_wait_prior_grid();
    const int tx = threadIdx.x, wid = threadIdx.y, t = 32 * wid + tx;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int zs = a.z_lo + blockIdx.z * a.zchunk, ze = min(zs + a.zchunk, a.z_hi);
    const int BX = a.nx / 4, BY = a.ny / 4, nw = 2 * a.rate;
    int held[2] = {-1, -1};  // window layer in each slot (the same in every thread)

    // window layer L into slot (L & 1): block (bxi, byi) of the tile's 18 x 6
    // by thread bxi + 18 byi; blocks outside the grid or window are zero
    auto load_layer = [&](int L) {
        float *dst = dsm + (L & 1) * kDSLayer;
        __syncthreads();  // the slot's previous layer is no longer read
        if (t < kDSBX * kDSBY) {
            const int bxi = t % kDSBX, byi = t / kDSBX;
            const int gbx = x0 / 4 - 1 + bxi, gby = y0 / 4 - 1 + byi;
            float v[64];
            if (L >= 0 && L < a.nl0 + a.nl1 && gbx >= 0 && gbx < BX && gby >= 0 && gby < BY) {
                const int seg = L < a.nl0 ? 0 : 1;
                const int ls = seg ? L - a.nl0 : L;
                const uint32_t *src = a.blk[seg] + (((int64_t)ls * BY + gby) * BX + gbx) * nw;
                decode_block(a.rate, [&](int i) -> uint32_t { return i < nw ? __ldg(src + i) : 0u; }, v);
            } else {
#pragma unroll
                for (int i = 0; i < 64; ++i)
                    v[i] = 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    *reinterpret_cast<float4 *>(dst + (k * kDSH + 4 * byi + j) * kDSW + 4 * bxi) =
                        make_float4(v[16 * k + 4 * j], v[16 * k + 4 * j + 1], v[16 * k + 4 * j + 2],
                                    v[16 * k + 4 * j + 3]);
        }
        held[L & 1] = L;
        __syncthreads();
    };
    // value of window plane z at tile-relative row ry, column cx (both offset by 4)
    auto at = [&](int z, int ry, int cx) -> float {
        if (z < 0 || z >= a.wp)
            return 0.0f;
        const int L = z >> 2;
        return dsm[(L & 1) * kDSLayer + ((z & 3) * kDSH + ry) * kDSW + cx];
    };

    const int x = x0 + kVX * tx;
    const bool x_ok = x < a.nx;
    for (int z = zs; z < ze; ++z) {
        // planes z - 1 .. z + 1 resident (at most two layers)
        const int la = (z - 1) >> 2, lb = (z + 1) >> 2;
        if (z - 1 >= 0 && held[la & 1] != la)
            load_layer(la);
        if (z + 1 < a.wp && held[lb & 1] != lb)
            load_layer(lb);
        if (held[(z >> 2) & 1] != (z >> 2))
            load_layer(z >> 2);
        const int gz = a.gz0 + z;
        const bool z_interior = gz >= 1 && gz < a.nz - 1;
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const int y = y0 + kRPT * wid + r;
            if (!x_ok || y >= a.ny)
                continue;
            const int ry = 4 + kRPT * wid + r;
            float res[kVX];
#pragma unroll
            for (int c = 0; c < kVX; ++c) {
                const int cx = 4 + kVX * tx + c;
                const float u = at(z, ry, cx);
                res[c] = u;
                const bool in_x = (x + c) >= 1 && (x + c) < a.nx - 1;
                const bool in_y = y >= 1 && y < a.ny - 1;
                if (z_interior && in_y && in_x) {
                    float s[2];
                    s[0] = 0.0f;
                    s[1] = nbr_sum(at(z, ry, cx - 1), at(z, ry, cx + 1), at(z, ry - 1, cx), at(z, ry + 1, cx),
                                   at(z - 1, ry, cx), at(z + 1, ry, cx));
                    res[c] = star_L<1>(a.c, u, s);
                }
            }
            const int64_t o = (int64_t)z * a.nx * a.ny + (int64_t)y * a.nx + x;
            *reinterpret_cast<float2 *>(a.out + o) = make_float2(res[0], res[1]);
        }
    }
}

cudaError_t launch_decode_heat_step(const StepLaunch &L, const void *blk0, int64_t nl0, const void *blk1,
                                    int64_t nl1, int rate, cudaStream_t s)
{
    if (L.z_hi <= L.z_lo)
        return cudaSuccess;
    if (L.scheme != kHeat || L.radius != 1 || rate < 1 || rate > 32 || L.nx % 4 != 0 || L.ny % 4 != 0 ||
        L.gz0 % 4 != 0 || L.wp != 4 * (nl0 + nl1) || (nl0 > 0 && !blk0) || (nl1 > 0 && !blk1))
        return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = current_device(dev);
    if (e != cudaSuccess)
        return e;
    int resident = 0, sms = 0;
    {
        static int res_dev[kMaxDevices] = {};
        std::lock_guard<std::mutex> lock(g_dev_mu);
        DevInfo &info = g_dev[dev];
        if (info.sms == 0 && (e = cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        if (res_dev[dev] == 0) {
            e = cudaFuncSetAttribute(k_decode_heat_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDSSmem);
            if (e != cudaSuccess)
                return e;
            int n = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_decode_heat_step, 32 * kConsumerWarps, kDSSmem);
            if (e != cudaSuccess)
                return e;
            if (n < 1)
                return cudaErrorInvalidConfiguration;
            res_dev[dev] = n;
        }
        resident = res_dev[dev];
        sms = info.sms;
    }
    DecStepArgs a;
    memset(&a, 0, sizeof(a));
    a.out = L.out;
    a.blk[0] = static_cast<const uint32_t *>(blk0);
    a.blk[1] = static_cast<const uint32_t *>(blk1);
    a.nl0 = (int)nl0;
    a.nl1 = (int)nl1;
    a.nx = (int)L.nx;
    a.ny = (int)L.ny;
    a.nz = (int)L.nz;
    a.gz0 = (int)L.gz0;
    a.wp = (int)L.wp;
    a.z_lo = (int)L.z_lo;
    a.z_hi = (int)L.z_hi;
    a.rate = rate;
    for (int i = 0; i < 5; ++i)
        a.c.c[i] = L.coef[i];
    // z chunks for the fullest last wave, at least 16 planes each (a chunk
    // decodes its planes' layers plus up to two more)
    StepArgs g;
    memset(&g, 0, sizeof(g));
    g.z_lo = a.z_lo;
    g.z_hi = a.z_hi;
    const dim3 grid0 = step_grid(L.nx, L.ny, sms * resident, g, 16);
    const int nplanes = a.z_hi - a.z_lo;
    a.zchunk = g.zchunk > 0 ? g.zchunk : nplanes;
    const dim3 grid((unsigned)g.ntiles / (unsigned)g.tiles_y, (unsigned)g.tiles_y,
                    (unsigned)((nplanes + a.zchunk - 1) / a.zchunk));
    (void)grid0;
    return launch_pdl(k_decode_heat_step, grid, dim3(32, kConsumerWarps, 1), kDSSmem, s, a);
}

cudaError_t launch_star_step(const StepLaunch &L, cudaStream_t s)
{
    if (L.z_hi <= L.z_lo)
        return cudaSuccess;
    StepArgs a;
    a.out = L.out;
    a.out2 = L.out2;
    a.res = L.res;
    a.zr = (int)L.zr;
    a.nx = (int)L.nx;
    a.ny = (int)L.ny;
    a.nz = (int)L.nz;
    a.plane = L.nx * L.ny;
    a.gz0 = (int)L.gz0;
    a.z_lo = (int)L.z_lo;
    a.z_hi = (int)L.z_hi;
    a.zchunk = 0;
    for (int i = 0; i < 5; ++i)
        a.c.c[i] = L.coef[i];
    a.src_x = (int)L.src_x;
    a.src_y = (int)L.src_y;
    a.src_zw = L.src_z >= 0 ? (int)(L.src_z - L.gz0) : -1;
    a.w = L.w;
    a.w_dev = L.w_dev;
    a.t_dev = L.t_dev;
    a.t_rel = L.t_rel;
    a.nw = L.nw;
    a.enc_out = static_cast<uint32_t *>(L.enc_out);
    a.enc_rate = L.enc_rate;
    a.enc_layer0 = (int)L.enc_layer0;
    if (L.tile != 0 && L.tile != 1)
        return cudaErrorInvalidValue;
    if (L.enc_out) {  // the fused encode: heat, radius 1, whole layers, transform codec
        if (L.scheme != kHeat || L.radius != 1 || L.tile != 0 || L.enc_rate < 1 || L.enc_rate > 32 ||
            (L.gz0 + L.z_lo) % 4 != 0 || (L.z_hi - L.z_lo) % 4 != 0 || L.nx % 4 != 0 || L.ny % 4 != 0)
            return cudaErrorInvalidValue;
        return launch_step_t<1, kHeat, kConsumerWarps, true>(L, a, s);
    }
    const bool t8 = L.tile == 1;  // 64 x 8 tiles
    if (L.radius == 1 && L.scheme == kHeat)
        return t8 ? launch_step_t<1, kHeat, 2>(L, a, s) : launch_step_t<1, kHeat>(L, a, s);
    if (L.radius == 4 && L.scheme == kHeat)
        return t8 ? launch_step_t<4, kHeat, 2>(L, a, s) : launch_step_t<4, kHeat>(L, a, s);
    if (L.radius == 1 && L.scheme == kWave)
        return t8 ? launch_step_t<1, kWave, 2>(L, a, s) : launch_step_t<1, kWave>(L, a, s);
    if (L.radius == 4 && L.scheme == kWave)
        return t8 ? launch_step_t<4, kWave, 2>(L, a, s) : launch_step_t<4, kWave>(L, a, s);
    if (L.radius == 4 && L.scheme == kAdjoint && L.c2)
        return t8 ? launch_step_t<4, kAdjoint, 2>(L, a, s) : launch_step_t<4, kAdjoint>(L, a, s);
    if (L.radius == 4 && L.scheme == kGradient)
        return t8 ? launch_step_t<4, kGradient, 2>(L, a, s) : launch_step_t<4, kGradient>(L, a, s);
    return cudaErrorInvalidValue;
}

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

// out[i] = a[i] * b[i] (one rounding), n a multiple of 4, 16-byte aligned arrays
__global__ void __launch_bounds__(256) k_product(float *__restrict__ out, const float *__restrict__ a,
                                                 const float *__restrict__ b, int64_t n4)
{
    pdl_launch_dependents();
    pdl_wait_prior_grid();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 x = reinterpret_cast<const float4 *>(a)[i];
        const float4 y = reinterpret_cast<const float4 *>(b)[i];
        reinterpret_cast<float4 *>(out)[i] =
            make_float4(fmul_rn(x.x, y.x), fmul_rn(x.y, y.y), fmul_rn(x.z, y.z), fmul_rn(x.w, y.w));
    }
}

cudaError_t launch_product(float *out, const float *a, const float *b, int64_t n, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    const int64_t n4 = n / 4;
    const unsigned grid = (unsigned)std::min<int64_t>((n4 + 255) / 256, (int64_t)std::max(device_sms(), 1) * 8);
    return launch_pdl(k_product, dim3(grid), dim3(256), 0, s, out, a, b, n4);
}

// One thread waits on an mbarrier that no thread arrives on, through the
// bounded wait every kernel here uses: after kWaitLimitNs it records
// kErrWaitTimeout in the device error word and returns.  Failure detection
// exercised without a GPU fault.
__global__ void k_stuck_wait()
{
    __shared__ uint64_t bar;
    mbar_init(&bar, 1);
    fence_barrier_init();
    mbar_wait(&bar, 0);  // phase 0 never completes
}

cudaError_t launch_stuck_wait(cudaStream_t s)
{
    k_stuck_wait<<<1, 1, 0, s>>>();
    return cudaGetLastError();
}

cudaError_t launch_set_i64(int64_t *p, int64_t v, cudaStream_t s)
{
    k_set_i64<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

cudaError_t read_device_error(unsigned int *code, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(code, g_device_error, sizeof(unsigned int));
    if (e == cudaSuccess && clear && *code) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(unsigned int));
    }
    return e;
}

// ------------------------------------------------------------------ codec --

constexpr int kCodecThreads = 128;

// Locate global block b in a segment list; returns the segment and the block's
// (bx, by, layer) inside it.  A launch codes fewer than 2^31 blocks (checked
// by the launchers), so the index arithmetic is 32-bit.
OOCS_FN int find_segment(const CodecSegments &sg, int64_t b, int bnx, int bny, int &bx, int &by,
                         int64_t &bl)
{
    int g = 0;
#pragma unroll 1
    while (g + 1 < sg.nseg && b >= sg.first[g + 1])
        ++g;
    const uint32_t lb = (uint32_t)(b - sg.first[g]);
    const uint32_t t = lb / (uint32_t)bnx;
    bx = (int)(lb - t * (uint32_t)bnx);
    const uint32_t l = t / (uint32_t)bny;
    by = (int)(t - l * (uint32_t)bny);
    bl = l;
    return g;
}

// The encoder's compressed words pass through shared memory, one row of
// 2 rate + 1 words per thread, so that global memory sees contiguous, coalesced
// runs of words instead of 32 lanes each writing a word of a different
// 8 rate-byte block.
OOCS_FN uint32_t *segment_word(const CodecSegments &sg, int64_t blk, int rate, int wi)
{
    int g = 0;
#pragma unroll 1
    while (g + 1 < sg.nseg && blk >= sg.first[g + 1])
        ++g;
    return static_cast<uint32_t *>(sg.blocks[g]) + (blk - sg.first[g]) * (int64_t)(2 * rate) + wi;
}

template <int KIND>
__global__ void __launch_bounds__(kCodecThreads, 6)
    k_encode_layers(const CodecSegments sg, int nx, int ny, int rate)
{
    extern __shared__ uint32_t sw[];
    __shared__ uint32_t dbl[KIND == kCodecTransform ? 256 : 1];  // the transform encoder's doubling table
    if constexpr (KIND == kCodecTransform) {
        fill_doubling_table(dbl, threadIdx.x, kCodecThreads);
        __syncthreads();
    }
    pdl_launch_dependents();
    pdl_wait_prior_grid();
    const int nw = 2 * rate, stride = 2 * rate + 1;
    const int64_t total = sg.first[sg.nseg];
    const int64_t b0 = (int64_t)blockIdx.x * kCodecThreads;
    const int64_t b = b0 + threadIdx.x;
    if (b < total) {
        int bx, by;
        int64_t bl;
        const int g = find_segment(sg, b, nx >> 2, ny >> 2, bx, by, bl);
        const int64_t plane = (int64_t)nx * ny;
        const float *base = sg.planes[g] + 4 * bl * plane + (int64_t)(4 * by) * nx + 4 * bx;
        float v[64];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 f =
                    __ldg(reinterpret_cast<const float4 *>(base + k * plane + (int64_t)j * nx));
                v[16 * k + 4 * j + 0] = f.x;
                v[16 * k + 4 * j + 1] = f.y;
                v[16 * k + 4 * j + 2] = f.z;
                v[16 * k + 4 * j + 3] = f.w;
            }
        uint32_t *row = sw + threadIdx.x * stride;
        bool finite;
        if constexpr (KIND == kCodecQuant)
            finite = bq_encode_block(v, rate, [&](int i, uint32_t w) { row[i] = w; });
        else
            finite = encode_block(v, rate, dbl, [&](int i, uint32_t w) { row[i] = w; });
        if (!finite)
            atomicOr(&g_device_error, kErrNonFinite);
    }
    __syncthreads();
    // each warp copies whole blocks out, its lanes over the block's words
    const int nblk = (int)(total - b0 < kCodecThreads ? total - b0 : kCodecThreads);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int g0 = 0;
#pragma unroll 1
    while (g0 + 1 < sg.nseg && b0 >= sg.first[g0 + 1])
        ++g0;
    if (b0 + nblk <= sg.first[g0 + 1]) {
        // all of the CTA's blocks in one segment: their words are contiguous
        uint32_t *dst = static_cast<uint32_t *>(sg.blocks[g0]) + (b0 - sg.first[g0]) * (int64_t)nw;
        for (int blk = warp; blk < nblk; blk += kCodecThreads / 32)
            for (int wi = lane; wi < nw; wi += 32)
                dst[blk * nw + wi] = sw[blk * stride + wi];
    } else {
        for (int blk = warp; blk < nblk; blk += kCodecThreads / 32) {
            uint32_t *dst = segment_word(sg, b0 + blk, rate, 0);
            for (int wi = lane; wi < nw; wi += 32)
                dst[wi] = sw[blk * stride + wi];
        }
    }
}

// Writes a decoded block's 64 values to its 4 x 4 x 4 place in the planes.
OOCS_FN void store_block(const CodecSegments &sg, int g, int nx, int ny, int bx, int by, int64_t bl,
                         const float (&v)[64])
{
    const int64_t plane = (int64_t)nx * ny;
    float *base = sg.planes[g] + 4 * bl * plane + (int64_t)(4 * by) * nx + 4 * bx;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4 *>(base + k * plane + (int64_t)j * nx) =
                make_float4(v[16 * k + 4 * j + 0], v[16 * k + 4 * j + 1], v[16 * k + 4 * j + 2],
                            v[16 * k + 4 * j + 3]);
}

template <int KIND>
__global__ void __launch_bounds__(kCodecThreads, 6)
    k_decode_layers(const CodecSegments sg, int nx, int ny, int rate)
{
    extern __shared__ uint32_t sw[];
    pdl_launch_dependents();
    pdl_wait_prior_grid();
    const int64_t b = (int64_t)blockIdx.x * kCodecThreads + threadIdx.x;
    const int nw = 2 * rate;
    if constexpr (KIND == kCodecTransform) {
        if (b >= sg.first[sg.nseg])
            return;
        int bx, by;
        int64_t bl;
        const int g = find_segment(sg, b, nx >> 2, ny >> 2, bx, by, bl);
        // a thread's words share its block's cache lines: the first load of
        // each line brings the rest into L1
        const uint32_t *src = static_cast<const uint32_t *>(sg.blocks[g]) + (b - sg.first[g]) * (int64_t)nw;
        float v[64];
        decode_block(rate, [&](int i) -> uint32_t { return i < nw ? __ldg(src + i) : 0u; }, v);
        store_block(sg, g, nx, ny, bx, by, bl, v);
    } else {
        // quantiser: a warp with a coded block copies its 32 blocks' words to
        // shared memory (coalesced, eight blocks' loads in flight), so that
        // the bit streams are not read by chains of dependent global loads;
        // an all-zero warp needs nothing more than the headers
        const bool live = b < sg.first[sg.nseg];
        const int stride = 2 * rate + 1, lane = threadIdx.x & 31;
        int bx = 0, by = 0, g = 0;
        int64_t bl = 0;
        const uint32_t *src = nullptr;
        uint32_t w0 = 0u;
        if (live) {
            g = find_segment(sg, b, nx >> 2, ny >> 2, bx, by, bl);
            src = static_cast<const uint32_t *>(sg.blocks[g]) + (b - sg.first[g]) * (int64_t)nw;
            w0 = __ldg(src);
        }
        const unsigned coded = __ballot_sync(0xffffffffu, live && (w0 & 0xFFu) != 0u);
        uint32_t *row = sw + threadIdx.x * stride;
        if (coded) {
            uint32_t *wrows = sw + (threadIdx.x & ~31) * stride;
            // lane 0's block starts the warp's run of blocks
            const uint32_t *wsrc = reinterpret_cast<const uint32_t *>(
                __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(src), 0));
            const unsigned alive = __ballot_sync(0xffffffffu, live);  // a prefix of the lanes
            const int nlive = __popc(alive);
            // the live blocks are consecutive when the last one is in lane 0's
            // segment (the common case); else each lane copies its own words
            const int g_last = __shfl_sync(0xffffffffu, g, nlive - 1);
            const int g_first = __shfl_sync(0xffffffffu, g, 0);
            if (g_first == g_last) {
                constexpr int kDepth = 8;
                for (int base = 0; base < nlive; base += kDepth) {
                    uint32_t r0[kDepth], r1[kDepth];
#pragma unroll
                    for (int u = 0; u < kDepth; ++u) {
                        const int blk = base + u;
                        r0[u] = (blk < nlive && lane < nw) ? __ldg(wsrc + blk * nw + lane) : 0u;
                        r1[u] = (blk < nlive && lane + 32 < nw) ? __ldg(wsrc + blk * nw + lane + 32) : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < kDepth; ++u) {
                        const int blk = base + u;
                        if (blk < nlive) {
                            if (lane < nw)
                                wrows[blk * stride + lane] = r0[u];
                            if (lane + 32 < nw)
                                wrows[blk * stride + lane + 32] = r1[u];
                        }
                    }
                }
            } else if (live) {
                for (int i = 0; i < nw; ++i)
                    row[i] = __ldg(src + i);
            }
            __syncwarp();
        }
        if (!live)
            return;
        float v[64];
        if (coded) {
            bq_decode_block(rate, [&](int i) -> uint32_t { return row[i]; }, v);
        } else {
#pragma unroll
            for (int i = 0; i < 64; ++i)
                v[i] = 0.0f;
        }
        store_block(sg, g, nx, ny, bx, by, bl, v);
    }
}

static cudaError_t seal_segments(CodecSegments &sg, int64_t nx, int64_t ny, const int64_t *nlayers)
{
    if (sg.nseg < 0 || sg.nseg > kMaxCodecSegments)
        return cudaErrorInvalidValue;
    sg.first[0] = 0;
    for (int g = 0; g < sg.nseg; ++g)
        sg.first[g + 1] = sg.first[g] + (nx / 4) * (ny / 4) * nlayers[g];
    return cudaSuccess;
}

static bool codec_ok(int rate, int kind)
{
    return (kind == kCodecTransform && rate >= 1 && rate <= 32) || (kind == kCodecQuant && rate >= 2 && rate <= 32);
}

cudaError_t launch_encode_segments(CodecSegments sg, const int64_t *nlayers, int64_t nx, int64_t ny,
                                   int rate, int kind, cudaStream_t s)
{
    if (!codec_ok(rate, kind))
        return cudaErrorInvalidValue;
    cudaError_t e = seal_segments(sg, nx, ny, nlayers);
    if (e != cudaSuccess)
        return e;
    const int64_t nb = sg.first[sg.nseg];
    if (nb == 0)
        return cudaSuccess;
    if (nb >= (int64_t)1 << 31)  // the kernels' block indices are 32-bit within a segment
        return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((nb + kCodecThreads - 1) / kCodecThreads));
    const size_t smem = (size_t)kCodecThreads * (2 * rate + 1) * 4;
    if (kind == kCodecQuant)
        return launch_pdl(k_encode_layers<kCodecQuant>, grid, dim3(kCodecThreads), smem, s, sg, (int)nx, (int)ny,
                          rate);
    return launch_pdl(k_encode_layers<kCodecTransform>, grid, dim3(kCodecThreads), smem, s, sg, (int)nx, (int)ny,
                      rate);
}

cudaError_t launch_decode_segments(CodecSegments sg, const int64_t *nlayers, int64_t nx, int64_t ny,
                                   int rate, int kind, cudaStream_t s)
{
    if (!codec_ok(rate, kind))
        return cudaErrorInvalidValue;
    cudaError_t e = seal_segments(sg, nx, ny, nlayers);
    if (e != cudaSuccess)
        return e;
    const int64_t nb = sg.first[sg.nseg];
    if (nb == 0)
        return cudaSuccess;
    if (nb >= (int64_t)1 << 31)  // the kernels' block indices are 32-bit within a segment
        return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((nb + kCodecThreads - 1) / kCodecThreads));
    if (kind == kCodecQuant)  // staging rows for the warps with coded blocks
        return launch_pdl(k_decode_layers<kCodecQuant>, grid, dim3(kCodecThreads),
                          (size_t)kCodecThreads * (2 * rate + 1) * 4, s, sg, (int)nx, (int)ny, rate);
    return launch_pdl(k_decode_layers<kCodecTransform>, grid, dim3(kCodecThreads), 0, s, sg, (int)nx, (int)ny,
                      rate);
}

cudaError_t launch_encode_layers(const float *planes, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, int kind, void *blocks, cudaStream_t s)
{
    CodecSegments sg;
    sg.nseg = 1;
    sg.planes[0] = const_cast<float *>(planes);
    sg.blocks[0] = blocks;
    return launch_encode_segments(sg, &nlayers, nx, ny, rate, kind, s);
}

cudaError_t launch_decode_layers(const void *blocks, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, int kind, float *planes, cudaStream_t s)
{
    CodecSegments sg;
    sg.nseg = 1;
    sg.planes[0] = planes;
    sg.blocks[0] = const_cast<void *>(blocks);
    return launch_decode_segments(sg, &nlayers, nx, ny, rate, kind, s);
}

}  // namespace oocs
