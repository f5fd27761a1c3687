// kernels.h -- host-side launchers of the sm_103a kernels (internal interface
// between the scheduler in capi.cu and the kernels in kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace oocs {

// One time step of the star stencil over window-relative planes [z_lo, z_hi)
// of a window buffer whose plane 0 is global plane gz0 (Sec. 3.1 temporal
// blocking computes a shrinking trapezoid of planes per step).
struct StepLaunch {
    int scheme;          // kHeat / kWave
    int radius;          // 1 or 4
    const float *cur;    // u at the previous time level, window buffer
    const float *prev;   // wave: u two levels back (may alias out)
    const float *m;      // wave: model field
    float *out;          // result, window buffer
    int64_t nx, ny, nz;  // grid (nz = global planes)
    int64_t gz0;         // global z of window plane 0
    int64_t wp;          // planes in the window buffers
    int64_t z_lo, z_hi;  // window-relative planes to compute
    float coef[5];
    int64_t src_x, src_y, src_z;  // global source voxel, src_z < 0: none
    float w;                      // source amplitude for this step
};

cudaError_t launch_star_step(const StepLaunch &L, cudaStream_t s);

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

cudaError_t launch_encode_segments(CodecSegments sg, const int64_t *nlayers, int64_t nx, int64_t ny,
                                   int rate, cudaStream_t s);
cudaError_t launch_decode_segments(CodecSegments sg, const int64_t *nlayers, int64_t nx, int64_t ny,
                                   int rate, cudaStream_t s);

// Fixed-rate codec over whole 4-plane layers.  planes: first FP32 plane of the
// first layer; blocks: first block of the first layer.
cudaError_t launch_encode_layers(const float *planes, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, void *blocks, cudaStream_t s);
cudaError_t launch_decode_layers(const void *blocks, int64_t nx, int64_t ny, int64_t nlayers,
                                 int rate, float *planes, cudaStream_t s);

}  // namespace oocs
