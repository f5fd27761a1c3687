// kernels.h -- host-side launchers of the sm_103a kernels (internal interface
// between the scheduler in capi.cu and the kernels in kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace oocs {

// One time step of the star stencil over window-relative planes [z_lo, z_hi)
// of a window buffer whose plane 0 is global plane gz0 (Sec. 3.1 temporal
// blocking computes a shrinking trapezoid of planes per step).
//
// The same kernel runs the two steps of the wave misfit's discrete adjoint
// (kAdjoint, kGradient); the fields then play these roles:
//   scheme     cur (stencil)   prev          m       c2     out           out2
//   kHeat      u^n             -             -       -      u^(n+1)       -
//   kWave      u^n             u^(n-1)       m       -      u^(n+1)       -
//   kAdjoint   m lam^(n+1)     lam^(n+2)     m       lam^(n+1)  lam^n     m lam^n (or null)
//   kGradient  u^n             dJ/dm         lam^(n+1)  -   dJ/dm         -
// (out may alias prev; kAdjoint adds res at global plane zr, kGradient adds w
// at the source voxel.)
struct StepLaunch {
    int scheme;          // kHeat / kWave / kAdjoint / kGradient
    int radius;          // 1 or 4 (4 for kAdjoint / kGradient)
    const float *cur;    // stencil input, window buffer
    const float *prev;   // first centre field (see the table)
    const float *m;      // second centre field
    const float *c2;     // kAdjoint: third centre field
    float *out;          // result, window buffer
    float *out2;         // kAdjoint: m * result
    const float *res;    // kAdjoint: residual plane (nx * ny) or null
    int64_t zr;          // kAdjoint: global plane of res
    int64_t nx, ny, nz;  // grid (nz = global planes)
    int64_t gz0;         // global z of window plane 0
    int64_t wp;          // planes in the window buffers
    int64_t z_lo, z_hi;  // window-relative planes to compute
    float coef[5];
    int64_t src_x, src_y, src_z;  // global source voxel, src_z < 0: none
    float w;                      // source amplitude for this step
    // device-side amplitude (for launches recorded in a CUDA graph): if w_dev
    // is set, the step at time t = *t_dev + t_rel adds w_dev[t] when
    // 0 <= t < nw and nothing otherwise, instead of `w`
    const float *w_dev;
    const int64_t *t_dev;
    int64_t t_rel;
    int64_t nw;
    int tile;  // 0: 64 x 16 tiles (4 consumer warps); 1: 64 x 8 tiles (2)
    // heat with radius 1 only: when enc_out is set, the step encodes its
    // planes [z_lo, z_hi) (whole 4-plane layers) with the transform codec at
    // enc_rate straight into the blocks at enc_out, whose first layer is
    // global layer enc_layer0, instead of writing them to `out`
    void *enc_out;
    int enc_rate;
    int64_t enc_layer0;
};

cudaError_t launch_star_step(const StepLaunch &L, cudaStream_t s);

// Two heat steps (radius 1) in one launch: L describes the second of the two
// (its planes [z_lo, z_hi), written to L.out from the step-before-last values
// in L.cur; the middle step stays on chip).  Bit-identical to two
// launch_star_step calls.
cudaError_t launch_heat_step2(const StepLaunch &L, cudaStream_t s);

// Decode fused into the first heat step of a visit (radius 1, transform codec
// at `rate`): L describes step 1 (its planes [z_lo, z_hi) written to L.out);
// window layers [0, nl0) are decoded from the codec blocks at blk0 and
// [nl0, nl0 + nl1) from those at blk1 (wp = 4 (nl0 + nl1)), into shared
// memory only.  Bit-identical to a decode into the window and one
// launch_star_step.
cudaError_t launch_decode_heat_step(const StepLaunch &L, const void *blk0, int64_t nl0, const void *blk1,
                                    int64_t nl1, int rate, cudaStream_t s);

// out = a * b elementwise (FP32, one rounding each); n a multiple of 4.
cudaError_t launch_product(float *out, const float *a, const float *b, int64_t n, cudaStream_t s);

// A kernel whose only wait never completes: it ends after the bounded-wait
// limit with kErrWaitTimeout in the device error word (failure-detection test).
cudaError_t launch_stuck_wait(cudaStream_t s);

// *p = v in stream order (one thread).
cudaError_t launch_set_i64(int64_t *p, int64_t v, cudaStream_t s);

// Read (and optionally clear) the device error word set by kernels whose
// bounded waits ran out (0 = no error).
cudaError_t read_device_error(unsigned int *code, bool clear);

// Up to kMaxCodecSegments runs of whole 4-plane layers coded by one launch:
// segment g maps nlayers[g] layers of FP32 planes at planes[g] to / from the
// codec blocks at blocks[g] (first[] is filled by the launcher).
constexpr int kMaxCodecSegments = 8;
struct CodecSegments {
    float *planes[kMaxCodecSegments];
    void *blocks[kMaxCodecSegments];
    int64_t first[kMaxCodecSegments + 1];
    int nseg = 0;
};

// Codec of a block (8 rate bytes per 4x4x4 block either way): the transform
// codec (codec.cuh, rate 1..32) or the block quantiser (quant.cuh, rate 2..32).
// The launchers return cudaErrorInvalidValue for another kind or rate.
enum CodecKind { kCodecTransform = 0, kCodecQuant = 1 };

cudaError_t launch_encode_segments(CodecSegments sg, const int64_t *nlayers, int64_t nx, int64_t ny,
                                   int rate, int kind, cudaStream_t s);
cudaError_t launch_decode_segments(CodecSegments sg, const int64_t *nlayers, int64_t nx, int64_t ny,
                                   int rate, int kind, cudaStream_t s);

// Fixed-rate codec over whole 4-plane layers.  planes: first FP32 plane of the
// first layer; blocks: first block of the first layer.
cudaError_t launch_encode_layers(const float *planes, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, int kind, void *blocks, cudaStream_t s);
cudaError_t launch_decode_layers(const void *blocks, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, int kind, float *planes, cudaStream_t s);

}  // namespace oocs
