/*
 * oocs.h -- compressed out-of-core 3D stencil sweeps on one GPU (C ABI).
 *
 * Method: Shen et al., "Compression-Based Optimizations for Out-of-Core GPU
 * Stencil Computation".  A grid larger than the device budget lives in host
 * memory as a stack of z-slabs ("chunks", Sec. 3.1).  Each slab is copied to
 * the GPU with a halo of h >= k*r planes (temporal blocking, Sec. 3.1), its
 * overlap with the previous slab is reused on the device (region sharing,
 * Sec. 3.1 and Sec. 4.1), it is decompressed, advanced k time steps,
 * recompressed with a fixed-rate block codec (Sec. 4.2) and copied back.  All
 * slabs share ONE device working buffer (single working buffer, Sec. 5), and
 * three streams are ordered by events as in Algorithm 1 ("Conflict-free
 * scheduling") so that no two slabs touch the working buffer at once.
 *
 * Conventions for every entry point:
 *  - Fields are FP32, layout [z][y][x] with x fastest; nx, ny, nz are
 *    multiples of 4.  Points within `radius` of a face are the Dirichlet
 *    shell and never change.
 *  - The caller owns all memory: the device workspace, the host stores and
 *    any raw host arrays.  The library allocates only CUDA events and small
 *    host metadata, and frees only what it allocated.
 *  - Every call returns an oocs_status and never aborts, throws or traps (a
 *    host allocation that fails inside the library returns
 *    OOCS_ERR_HOST_ALLOC).
 *    OOCS_ERR_CUDA, OOCS_ERR_TIMEOUT and OOCS_ERR_NONFINITE are sticky on a
 *    context until oocs_destroy; the text of the last error is in
 *    oocs_last_error().
 *  - Calls that enqueue GPU work are asynchronous with respect to the host;
 *    completion and device-side errors surface in oocs_synchronize().
 *  - A context is used by one host thread at a time.
 *  - Stream arguments are cudaStream_t values passed as void*.
 */
#ifndef OOCS_H
#define OOCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OOCS_OK = 0,
    OOCS_ERR_INVALID_ARG = 1,  /* bad pointer, size, shape, rate or state of an argument */
    OOCS_ERR_BUDGET = 2,       /* the plan does not fit the device budget / workspace    */
    OOCS_ERR_HOST_ALLOC = 3,   /* host metadata allocation failed                         */
    OOCS_ERR_CUDA = 4,         /* a CUDA call failed (sticky)                             */
    OOCS_ERR_TIMEOUT = 5,      /* oocs_synchronize ran out of time (sticky)               */
    OOCS_ERR_STATE = 6,        /* call not valid in the context's current state           */
    OOCS_ERR_UNSUPPORTED = 7,  /* valid request the library does not implement            */
    OOCS_ERR_NONFINITE = 8     /* the codec was handed an Inf or NaN (sticky); see below  */
} oocs_status;

/* Time schemes (Sec. 6 uses a 25-point acoustic wave code).
 *  OOCS_HEAT: u' = c0 u + sum_{d=1..r} c_d s_d(u)                 (first order in time)
 *  OOCS_WAVE: u' = 2u - up + m (c0 u + sum_d c_d s_d(u) + w[t] at the source)  (leapfrog)
 * with s_d(u)(p) = (u[p-d ex] + u[p+d ex]) + (u[p-d ey] + u[p+d ey]) + (u[p-d ez] + u[p+d ez]). */
enum { OOCS_HEAT = 0, OOCS_WAVE = 1, OOCS_WAVE_ADJOINT = 2 };

/* Fields of a context.  HEAT streams U.  WAVE streams U (u^t), U_PREV (u^(t-1))
 * and the read-only model M = (v dt/dx)^2 (the paper's read-only dataset,
 * Sec. 6.2); the write-only dataset is device-only.                        */
enum { OOCS_FIELD_U = 0, OOCS_FIELD_U_PREV = 1, OOCS_FIELD_M = 2 };

/* OOCS_WAVE_ADJOINT: oocs_step(ctx, n) takes n time steps of the WAVE
 * scheme's discrete adjoint, each a sweep over the slabs in reverse z order,
 * with the gradient of a receiver misfit accumulated on the device.  At time
 * index k (oocs_set_time, then counting down) a step reads lam^k (field LAM),
 * lam^(k+1) (LAM_PREV, interior only) and the forward state u^(k-1), adds
 * lam^k (L u^(k-1) + w[k-1] at the source) to dJ/dm (field GRAD, on the
 * device, zero at create), writes lam^(k-1) = 2 lam^k - lam^(k+1) +
 * L(m lam^k) + r^(k-2) at the receiver plane into LAM_PREV's store, then the
 * LAM and LAM_PREV stores trade roles and the time index becomes k-1.
 * u^(k-1) is read from the state record (oocs_set_state_record: entry
 * k-1-t0) when one is set, else from the FWD store (then n must be 1).  The
 * steps of one call are pipelined: a slab visit waits only for the previous
 * step's copies of the slabs its window touches.  r^n = planes[n] of
 * oocs_set_receiver.  m (field M) is kept on the device (readonly_resident
 * must be 1); temporal_depth is 1; the halo is one 4-plane layer; no region
 * sharing (whole windows are copied).  GRAD is read with
 * oocs_decompress_device.                                                   */
enum { OOCS_FIELD_LAM = 0, OOCS_FIELD_LAM_PREV = 1, OOCS_FIELD_FWD = 3, OOCS_FIELD_GRAD = 4 };

/* Fixed-rate codecs of the host store.  Both code each 4x4x4 block of FP32
 * values (index i + 4j + 16k) into exactly 8*rate bytes, so they share the
 * store layout, the plan and the schedule.
 *  TRANSFORM: the ZFP method (block-floating-point quantisation, decorrelating
 *   lifting transform, embedded bit-plane coding; cuZFP in the paper, Sec. 4.2),
 *   with this library's own bitstream.
 *  QUANT: an 8-bit header (0 = all-zero block, else emax + 127 with
 *   emax = max(frexp exponent of max|v|, -126)), then 64 two's complement
 *   fields of q = rate - 1 bits, n = clamp(rint(v 2^(q-1-emax)), +-(2^(q-1)-1)),
 *   bits numbered from bit 0 of word 0; decodes to RN(RN(n) 2^(emax-q+1)).  */
enum { OOCS_CODEC_TRANSFORM = 0, OOCS_CODEC_QUANT = 1 };

/* Working-buffer schemes (Sec. 5): 1 = single working buffer shared by the
 * three streams (the paper's method); 3 = classic, one per stream (Fig. 6a). */
enum { OOCS_SWB = 1, OOCS_CLASSIC = 3 };

#define OOCS_MAX_RADIUS 4

typedef struct {
    int64_t nx, ny, nz;          /* full grid incl. the Dirichlet shell; multiples of 4      */
    int32_t scheme;              /* OOCS_HEAT or OOCS_WAVE                                    */
    int32_t radius;              /* r: 1 or 4 (star stencils; WAVE requires 4)                */
    float coef[OOCS_MAX_RADIUS + 1]; /* [centre, c1 .. cr]; copied at create               */
    uint64_t device_budget;      /* bytes of device workspace the context may use            */
    int32_t rate_bits;           /* 0 = uncompressed store; 1..32 = fixed rate, bits/value   */
    int32_t temporal_depth;      /* k >= 1 steps per slab visit; 0 = 4                        */
    int32_t slab_planes;         /* T, multiple of 4; 0 = largest T that fits device_budget  */
    int32_t working_buffers;     /* OOCS_SWB (1) or OOCS_CLASSIC (3)                          */
    int32_t readonly_resident;   /* WAVE: 0 = stream the read-only model M with every slab
                                  * visit, as the paper does (Sec. 6.2); 1 = keep M on the
                                  * device as FP32 (decoded once from its store) for the
                                  * context's life, counted in the workspace, so only U and
                                  * U_PREV cross the host link.  Ignored for HEAT.           */
    int32_t codec;               /* rate_bits > 0: OOCS_CODEC_TRANSFORM (0, the paper's kind of
                                  * codec, Sec. 4.2; rate 1..32) or OOCS_CODEC_QUANT (1, a plain
                                  * block quantiser, the comparison of Sec. 7 (1); rate 2..32) */
    int32_t step_fusion;         /* HEAT with radius 1: 0 = one kernel per step (default);
                                  * 1 = the k steps of a slab visit run as pairs of steps
                                  * fused in one kernel (temporal blocking on chip: the middle
                                  * step stays in shared memory), the odd one out alone.
                                  * Bit-identical either way; the fused pairs halve the step
                                  * kernels' HBM traffic but measured slower on GB300.
                                  * Ignored for WAVE.                                          */
    int32_t step_tile;           /* x-y tile of the step kernel's z-march (Sec. 3.1 kernels):
                                  * 0 = 64 x 16 points per CTA (four consumer warps, the
                                  * default); 1 = 64 x 8 (two consumer warps: twice the
                                  * tiles, for planes too small to fill the GPU).  Results
                                  * are bit-identical; the autotuner searches it.            */
    int32_t codec_fusion;        /* HEAT with radius 1 and the transform codec at rate > 0:
                                  * 0 = separate decode and encode kernels around the steps
                                  * of a slab visit (the default); 1 = the codec in the steps
                                  * (Sec. 4.2: decompression on the way into the kernel,
                                  * compression on the way out): step 1 decodes the window's
                                  * blocks into shared memory and the last step encodes each
                                  * 4-plane layer of its results in its epilogue straight
                                  * into the output slot (a visit of one step keeps its
                                  * encode kernel), so the window never goes through HBM as
                                  * FP32.  Byte-identical stores either way; measured slower
                                  * on GB300.  Requires step_fusion = 0.  Ignored otherwise. */
} oocs_desc;

/* Resolved plan (Sec. 3.1 chunking and temporal blocking; Sec. 6.2 memory model). */
typedef struct {
    int32_t slab_planes;         /* T                                                        */
    int32_t temporal_depth;      /* k                                                        */
    int32_t halo_planes;         /* h = 4 * ceil(k r / 4)                                    */
    int32_t num_slabs;           /* S = ceil(nz / T)                                         */
    int32_t window_planes;       /* min(T + 2h, nz)                                          */
    int32_t fields_in;           /* streamed host->device fields (HEAT 1, WAVE 3)            */
    int32_t fields_out;          /* streamed device->host fields (HEAT 1, WAVE 2)            */
    int32_t readonly_resident;   /* 1 if M is kept on the device (fields_in is then 2)       */
    uint64_t layer_bytes;        /* bytes of one 4-plane layer of one field in the store     */
    uint64_t host_store_bytes;   /* bytes of one field's host store = nz/4 * layer_bytes     */
    uint64_t workspace_bytes;    /* device workspace for this desc                           */
    uint64_t workspace_swb_bytes;     /* same plan with one working buffer                  */
    uint64_t workspace_classic_bytes; /* same plan with three working buffers               */
} oocs_plan;

/* Per kernel class counters.  `units` are grid values processed: for LOAD the
 * values decoded (or copied) into the working buffer, for STEP the points
 * updated (including the redundant halo recomputation of temporal blocking),
 * for STORE the values encoded (or copied) out of it.  `device_ms` is the sum
 * of CUDA-event durations of those launches on their own streams, collected
 * only while profiling is on (oocs_set_profiling) and read at
 * oocs_synchronize; the k STEP launches of one slab visit are timed as one
 * interval (gaps between them included).                                   */
typedef struct {
    uint64_t launches;
    uint64_t units;
    double device_ms;
} oocs_kernel_stats;

typedef struct {
    uint64_t h2d_bytes;          /* bytes copied host->device by oocs_step so far            */
    uint64_t d2h_bytes;          /* bytes copied device->host by oocs_step so far            */
    uint64_t kernel_launches;    /* kernels launched by oocs_step so far                     */
    uint64_t steps_done;         /* time steps enqueued so far (the global time index t)     */
    uint64_t passes_done;        /* slab sweeps enqueued so far                              */
    uint64_t slabs_done;         /* slab visits enqueued so far                              */
    uint64_t workspace_bytes;    /* device bytes the context uses                            */
    double last_step_ms;         /* device time of the last completed oocs_step (events)    */
    oocs_kernel_stats load;      /* decode / copy of staged layers into the working buffer  */
    oocs_kernel_stats step;      /* stencil time steps                                       */
    oocs_kernel_stats store;     /* encode / copy of the slab interior out of it            */
    oocs_kernel_stats h2d;       /* host->device copies of a visit (units: bytes)            */
    oocs_kernel_stats d2h;       /* device->host copies of a visit (units: bytes)            */
} oocs_stats;

typedef struct oocs_ctx oocs_ctx;

/* Plan `desc` without touching the GPU.  Fills *plan.  OOCS_ERR_INVALID_ARG
 * for a malformed desc; OOCS_ERR_BUDGET when no slab thickness T >= max(4, 2h)
 * fits device_budget.  Thread-safe; no context needed.                      */
oocs_status oocs_query(const oocs_desc *desc, oocs_plan *plan);

/* Create a context on the current CUDA device.  `workspace` is a device
 * allocation of `workspace_bytes` >= plan.workspace_bytes, 256-byte aligned,
 * owned by the caller and kept alive until oocs_destroy.  streams[0..2] are
 * the three cudaStream_t the method pipelines over (Algorithm 1); they must be
 * distinct, non-null and stay valid for the context's life.                */
oocs_status oocs_create(const oocs_desc *desc, void *workspace, uint64_t workspace_bytes,
                        void *const streams[3], oocs_ctx **out);

/* Bind the host store of `field` (OOCS_FIELD_*): `bytes` >= plan.host_store_bytes
 * of host memory, page-locked (cudaHostAlloc / pinned torch tensor) for the
 * copies to overlap.  Layout: nz/4 layers of plan.layer_bytes; with
 * rate_bits > 0 a layer holds (nx/4)(ny/4) codec blocks of 8*rate_bits bytes,
 * block (bx, by) at ((by * nx/4) + bx) * 8*rate_bits; with rate_bits = 0 it is
 * the raw FP32 planes.  Updated in place by oocs_step.  With
 * desc.readonly_resident the device copy of M is (re)made from its store at
 * the first oocs_step after oocs_bind_field(M); oocs_compress(M) and
 * oocs_compress_device(M) update it as they code (the values the store
 * decodes to; oocs_compress at rate 0 leaves it to the next oocs_step);
 * later writes to the M store by other means are not seen until one of them. */
oocs_status oocs_bind_field(oocs_ctx *ctx, int32_t field, void *host_store, uint64_t bytes);

/* Set the point source of the WAVE scheme: voxel (x, y, z) receives w[t] at
 * the step that advances from time t (0-based, counted over the context's
 * life).  w (host, nw values) is copied.  Steps t >= nw add nothing.        */
oocs_status oocs_set_source(oocs_ctx *ctx, int64_t x, int64_t y, int64_t z, const float *w,
                            int32_t nw);

/* WAVE: after every step t < nplanes (t counted over the context's life, as
 * for the source), copy plane zr of the new state u^(t+1) to planes[t]
 * (device array of nplanes * nx * ny FP32, written on the visit's stream in
 * step order).  nplanes = 0 stops recording.  WAVE_ADJOINT: planes[n] is the
 * residual r^n added at plane zr (read).  The receiver record a misfit and its
 * adjoint need (no counterpart in the paper's forward-only runs).          */
oocs_status oocs_set_receiver(oocs_ctx *ctx, int64_t zr, float *planes, int64_t nplanes);

/* HEAT and WAVE: record the compressed states the sweep writes (for
 * WAVE_ADJOINT the record is read instead: entry k-1-t0 is the forward state
 * u^(k-1) of the adjoint step at time index k, see OOCS_WAVE_ADJOINT).  A slab visit
 * that advances the field from time t to t+k copies the encoded interior of
 * its new u^(t+k) (and, for WAVE, of u^(t+k-1)) into stores[t+k - t0]
 * (stores[t+k-1 - t0]) as well as into the field's own store, when that index
 * lies in [0, n) and the entry is non-null; after the call's work is done a
 * recorded store holds exactly the bytes U's store held after that state was
 * written.  So with temporal_depth 1 (HEAT) or <= 2 (WAVE) every state a call
 * passes through is recorded; with deeper blocking, those at the ends of the
 * visits.  stores: n pointers to caller-owned pinned host memory of at least
 * host_store_bytes each (the list is copied; the memory must stay valid until
 * the work is synchronized).  Copies run on the visit's stream after its own
 * device->host copy and count in d2h_bytes.  n = 0 stops recording.  A batch
 * member with a record (or receiver planes) cannot be captured as a graph
 * (OOCS_ERR_UNSUPPORTED).  The checkpoints and recomputed forward states of the
 * out-of-core misfit gradient (no counterpart in the paper).                */
oocs_status oocs_set_state_record(oocs_ctx *ctx, void *const *stores, int64_t t0, int64_t n);

/* Fill the bound store of `field` from a raw FP32 host array of nx*ny*nz
 * values (initial compression of the chunks, Algorithm 1 input (1)): copies
 * go through the workspace and the codec kernels, using streams[0..1].
 * Asynchronous: `src` must stay valid until oocs_synchronize.
 * In place: the store may be the first host_store_bytes of `src` itself (the
 * compressed layers of planes [z0, z1) never lie above the raw planes
 * [z0, z1), and the chunks are ordered so that nothing is overwritten before
 * it is read), so a field that fills most of host memory needs no second
 * array.  Any other overlap of the store and `src` is OOCS_ERR_INVALID_ARG. */
oocs_status oocs_compress(oocs_ctx *ctx, int32_t field, const float *src);

/* Inverse of oocs_compress: decode the bound store of `field` into the raw
 * FP32 host array `dst` of nx*ny*nz values.  Asynchronous.  In place as for
 * oocs_compress: the store may start at `dst` (the array then holds the
 * decoded field, the store is consumed).                                   */
oocs_status oocs_decompress(oocs_ctx *ctx, int32_t field, float *dst);

/* Planes [z0, z0 + nplanes) (whole 4-plane layers) of `field` between a
 * device FP32 array holding exactly those planes and the bound host store:
 * oocs_compress_device encodes them into their store layers (a copy at rate
 * 0), oocs_decompress_device decodes them back.  For filling or reading a
 * store larger than any host staging array.  Runs on streams[0], so the
 * device array must be complete in that stream's order (data written on
 * another stream: synchronize it first); asynchronous (the array must stay
 * valid until oocs_synchronize).                                           */
oocs_status oocs_compress_device(oocs_ctx *ctx, int32_t field, const float *src, int64_t z0, int64_t nplanes);
oocs_status oocs_decompress_device(oocs_ctx *ctx, int32_t field, float *dst, int64_t z0, int64_t nplanes);

/* Page-locked host memory of exactly `bytes` for host stores, zero-filled:
 * anonymous pages with transparent-huge-page advice, registered with
 * cudaHostRegister (portable).  Free with oocs_host_free, which rejects any
 * other pointer (OOCS_ERR_INVALID_ARG).  OOCS_ERR_HOST_ALLOC if it fails.   */
oocs_status oocs_host_alloc(uint64_t bytes, void **ptr);
oocs_status oocs_host_free(void *ptr);

/* Set the context's global time index t (the index of the source sample the
 * next step adds; 0 after oocs_create).  For restarting from a stored state.
 * Takes effect for work enqueued after the call.                           */
oocs_status oocs_set_time(oocs_ctx *ctx, int64_t t);

/* Advance the bound fields `nsteps` time steps: ceil(nsteps/k) sweeps over
 * the S slabs (the last with the remainder), each slab streamed through the
 * three-stream pipeline of Algorithm 1 with the single working buffer.
 * Asynchronous; the host stores hold the new state after oocs_synchronize.
 * The call's work opens and closes with a join of the three streams: it
 * starts after whatever the caller ordered before it on streams[0], and an
 * event the caller records on streams[0] after the call completes with it. */
oocs_status oocs_step(oocs_ctx *ctx, int32_t nsteps);

/* Failure detection without a GPU fault: enqueue on streams[0] a one-thread
 * kernel that waits on an mbarrier no thread ever arrives on, through the
 * bounded wait every kernel of the library uses.  After about one second the
 * wait gives up and records its timeout in the device error word; the next
 * oocs_synchronize returns OOCS_ERR_CUDA ("a kernel's bounded wait ran out"),
 * sticky on this context, and clears the word, so other contexts (and the
 * GPU) stay usable.  For tests of the error path.                          */
oocs_status oocs_selftest_stuck_wait(oocs_ctx *ctx);

/* Host-side fault injection, for tests of the error path (no GPU fault is
 * involved): after this call, the nth_call-th CUDA runtime call the context
 * checks (counting from 1; enqueues of copies, kernels and events, event and
 * stream queries) is reported as failed once it has been issued, exactly as
 * if CUDA had returned an error: the entry point that made it returns
 * OOCS_ERR_CUDA, sticky on the context ("injected failure" in
 * oocs_last_error).  Work already enqueued still runs; destroy the context
 * and create a new one to go on.  nth_call = 0 disarms.  Not in the paper:
 * failure detection of the runtime around its Algorithm 1.                */
oocs_status oocs_set_fault_injection(oocs_ctx *ctx, int64_t nth_call);

/* Wait for all work of the context, at most timeout_ns nanoseconds
 * (0 = no limit).  OOCS_ERR_TIMEOUT if it is still running (sticky; the work
 * goes on, and a later cudaStreamSynchronize of the streams waits for it);
 * OOCS_ERR_CUDA on a device error or a bounded wait that ran out;
 * OOCS_ERR_NONFINITE when the codec met an infinity or a NaN in a field it
 * encoded (a run past the stability limit, or bad input).  The fixed-rate
 * codec (Sec. 4.2) is defined for finite values: a 4x4x4 block holding a
 * non-finite value is stored as an all-zero block, and the stores no longer
 * describe the run.  Device-side errors are read from, and cleared in, the
 * device's error word (see oocs_device_errors).                           */
oocs_status oocs_synchronize(oocs_ctx *ctx, uint64_t timeout_ns);

/* The device error word of the current device, for callers of the
 * device-level entry points (oocs_encode_device, oocs_incore_run, ...), which
 * have no context to report through: the OR of OOCS_DEVERR_* flags raised by
 * kernels since it was last cleared.  Synchronises the device; clears the
 * word if `clear` is non-zero.  The word is shared by every context and call
 * on the device (oocs_synchronize also reads and clears it).              */
enum { OOCS_DEVERR_WAIT_TIMEOUT = 1, OOCS_DEVERR_NONFINITE = 2 };
oocs_status oocs_device_errors(uint32_t *flags, int32_t clear);

oocs_status oocs_get_stats(const oocs_ctx *ctx, oocs_stats *out);

/* Per-launch event timing of the work enqueued by oocs_step.  `classes` is a
 * bit mask of OOCS_PROF_LOAD | OOCS_PROF_STEP | OOCS_PROF_STORE (kernels) and
 * OOCS_PROF_H2D | OOCS_PROF_D2H (a visit's copies); 0 = off.  Adds two event
 * records per timed item on its own stream.                                */
enum { OOCS_PROF_LOAD = 1, OOCS_PROF_STEP = 2, OOCS_PROF_STORE = 4, OOCS_PROF_H2D = 8, OOCS_PROF_D2H = 16 };
oocs_status oocs_set_profiling(oocs_ctx *ctx, int32_t classes);

/* The timeline of the profiled items collected at the last oocs_synchronize:
 * per item its class (0 load, 1 step, 2 store, 3 h2d, 4 d2h), the stream
 * (0..2) and slab visit (counted over the context's life) it ran on, and its
 * start and end in milliseconds after the start of the last oocs_step call
 * enqueued before that synchronize (items of earlier calls come out
 * negative).  Copies min(count, capacity) entries; *count = entries kept.
 * The Nsight-style view of a sweep (which copy or kernel waits on which), for
 * the scheduling of Algorithm 1 (Fig. 8).                                  */
typedef struct {
    int32_t cls;
    int32_t stream;
    int64_t visit;
    double start_ms, end_ms;
} oocs_timeline_entry;
oocs_status oocs_get_timeline(const oocs_ctx *ctx, oocs_timeline_entry *entries, int64_t capacity,
                              int64_t *count);

/* Text of the last error of ctx, or of the last failed context-free call in
 * this thread when ctx is NULL.  Never NULL; valid until the next call.    */
const char *oocs_last_error(const oocs_ctx *ctx);

/* Release events and metadata (waits for outstanding work first).  The
 * caller's workspace, stores and streams are not touched.                  */
oocs_status oocs_destroy(oocs_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Device-level entry points (no context).  All pointers are device pointers
 * unless stated; all calls are asynchronous on `stream`.
 * ------------------------------------------------------------------------- */

/* In-core reference run of `nsteps` steps of desc's scheme on device-resident
 * fields (Sec. 3.1 stencil without chunking), with the same FP32 arithmetic
 * as oocs_step.  HEAT: u (in/out), scratch = nx*ny*nz floats.  WAVE: u = u^t,
 * u_prev = u^(t-1) (both in/out), m read-only, scratch = nx*ny*nz floats;
 * t0 = time index of u on entry (for the source), src_xyz and w as in
 * oocs_set_source (w is a HOST array; src_xyz may be NULL for no source).  */
oocs_status oocs_incore_run(const oocs_desc *desc, float *u, float *u_prev, const float *m,
                            float *scratch, int32_t nsteps, int64_t t0,
                            const int64_t *src_xyz, const float *w, int32_t nw, void *stream);

/* oocs_incore_run for callers that cannot allocate device memory.  The paper
 * has no counterpart: this exists for callers such as a plugin inside a host
 * application whose allocator owns the whole device memory pool, or a
 * latency-critical loop where cudaMalloc / cudaFree would synchronise the
 * device.  Same arguments and results as oocs_incore_run without `scratch`:
 * the grid-sized scratch field comes from a library-owned static device array
 * of OOCS_NOALLOC_MAX_VALUES floats (32 MiB), which every GPU that loads the
 * library holds until the process exits.  Grids with nx*ny*nz above that
 * maximum are rejected with OOCS_ERR_INVALID_ARG.  Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call.
 *  - The first call made with a device current looks up the array's device
 *    address (cudaGetSymbolAddress) and caches it per device and context; a
 *    context created anew (after cudaDeviceReset) is looked up again.  Make
 *    the first call on a device before any stream capture.
 *  - Every call shares the one array and it keeps the last call's contents;
 *    nothing in it needs to start at zero (each step overwrites all of it
 *    before reading it).  Calls that overlap on the GPU (other streams, other
 *    host threads) race on the array: serialise them.                      */
#define OOCS_NOALLOC_MAX_VALUES (8u << 20)
oocs_status oocs_incore_run_noalloc(const oocs_desc *desc, float *u, float *u_prev, const float *m,
                                    int32_t nsteps, int64_t t0, const int64_t *src_xyz,
                                    const float *w, int32_t nw, void *stream);

/* ---------------------------------------------------------------------------
 * Gradient of the receiver misfit of the WAVE scheme (device arrays, in-core).
 * Forward: u^(n+1) = 2u^n - u^(n-1) + m (L u^n + w_n e_src), u^0 = u^(-1) = 0,
 * J = 1/2 sum_{n=1..N} sum_xy (u^n(x, y, z_r) - d^n(x, y))^2.  Discrete adjoint,
 * backwards in time: lam^n = 2 lam^(n+1) - lam^(n+2) + L(m lam^(n+1)) + r^n at z_r,
 * lam^(N+1) = lam^(N+2) = 0, r^n = u^n(z_r) - d^n, and
 * dJ/dm = sum_{n=0..N-1} lam^(n+1) (L u^n + w_n e_src).  desc must describe the
 * WAVE scheme; only nx, ny, nz and coef are used.  Fields are nx*ny*nz FP32,
 * zero on the shell.  Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */

/* One adjoint step.  In: lam = lam^(n+1), lam_prev = lam^(n+2), mu = m lam^(n+1).
 * Out: lam_prev <- lam^n (in place), mu_out <- m lam^n (mu_out != mu).
 * res: the residual plane r^n (nx*ny, device) added at plane zr, or NULL.   */
oocs_status oocs_adjoint_step(const oocs_desc *desc, const float *lam, float *lam_prev, const float *mu,
                              float *mu_out, const float *m, const float *res, int64_t zr, void *stream);

/* grad_m += lam (L u + w at src_xyz) on the interior (src_xyz may be NULL). */
oocs_status oocs_gradient_accumulate(const oocs_desc *desc, float *grad_m, const float *lam, const float *u,
                                     float w, const int64_t *src_xyz, void *stream);

/* res = u_plane - d_plane (n values) and *misfit += 1/2 sum res^2 (misfit is a
 * device double, may be NULL).                                              */
oocs_status oocs_receiver_residual(const float *u_plane, const float *d_plane, int64_t n, float *res,
                                   double *misfit, void *stream);

/* m = (v dt/dx)^2 and its chain rule grad_v = grad_m 2 v (dt/dx)^2 (n values). */
oocs_status oocs_model_from_velocity(const float *v, float *m, int64_t n, float dt_over_dx, void *stream);
oocs_status oocs_velocity_gradient(const float *grad_m, const float *v, float *grad_v, int64_t n,
                                   float dt_over_dx, void *stream);

/* Forward / backward driver of the misfit gradient with checkpoints.  The
 * forward run from rest keeps, every `checkpoint_every` steps (K), the pair
 * (u^s, u^(s-1)) in `workspace`, compressed by the fixed-rate block codec at
 * `rate_bits` (Sec. 4.2; 0 = raw FP32 copies); the backward run walks the
 * segments in reverse, decodes each checkpoint, recomputes the segment's states
 * and applies the adjoint and gradient steps above, so the device holds the
 * checkpoints plus K + 5 fields instead of all nsteps states.
 *   workspace: device, 16-byte aligned, at least oocs_misfit_workspace_bytes()
 *     bytes, owned by the caller; the backward call reads the checkpoints the
 *     forward call with the same arguments left there.
 *   src_xyz, w (nw values; w_n = 0 for n >= nw): host arrays.
 *   d_obs, res: device [nsteps][ny][nx]; res[n] = u^(n+1)(z_r) - d_obs[n].
 *   misfit: device double, set to J.  grad_m: device field, set to dJ/dm.
 * Errors: OOCS_ERR_INVALID_ARG for a non-WAVE desc, bad sizes, pointers or a
 * short workspace (nothing is launched); OOCS_ERR_CUDA for launch failures. */
int64_t oocs_misfit_workspace_bytes(const oocs_desc *desc, int32_t nsteps, int32_t checkpoint_every,
                                    int32_t rate_bits);
oocs_status oocs_misfit_forward(const oocs_desc *desc, const float *m, const int64_t *src_xyz, const float *w,
                                int32_t nw, int64_t zr, const float *d_obs, int32_t nsteps,
                                int32_t checkpoint_every, int32_t rate_bits, void *workspace,
                                int64_t workspace_bytes, float *res, double *misfit, void *stream);
oocs_status oocs_misfit_backward(const oocs_desc *desc, const float *m, const int64_t *src_xyz, const float *w,
                                 int32_t nw, int64_t zr, const float *res, int32_t nsteps,
                                 int32_t checkpoint_every, int32_t rate_bits, void *workspace,
                                 int64_t workspace_bytes, float *grad_m, void *stream);

/* Fixed-rate block codec (Sec. 4.2) on device arrays.  encode: field
 * [nz][ny][nx] FP32 -> (nx/4)(ny/4)(nz/4) blocks of 8*rate bytes in layer
 * order (block (bx,by,bz) at ((bz*(ny/4)+by)*(nx/4)+bx)).  decode: inverse.
 * codec OOCS_CODEC_TRANSFORM with rate in [1, 32] or OOCS_CODEC_QUANT with
 * rate in [2, 32]; dims multiples of 4; pointers 16-byte aligned.  A block
 * holding an Inf or NaN is encoded as all zeros and raises
 * OOCS_DEVERR_NONFINITE in the device error word (oocs_device_errors).     */
oocs_status oocs_encode_device(const float *field, int64_t nx, int64_t ny, int64_t nz,
                               int32_t rate, int32_t codec, void *blocks, void *stream);
oocs_status oocs_decode_device(const void *blocks, int64_t nx, int64_t ny, int64_t nz,
                               int32_t rate, int32_t codec, float *field, void *stream);

/* ---------------------------------------------------------------------------
 * Schedule trace (no GPU needed): the operations oocs_step would enqueue, in
 * enqueue order, for a fresh context, so their ordering can be checked on the
 * host.  This is the DAG of Fig. 8(a) as built by Algorithm 1's scheduling.
 * ------------------------------------------------------------------------- */
enum { OOCS_OP_WAIT = 1, OOCS_OP_RECORD = 2, OOCS_OP_H2D = 3, OOCS_OP_D2H = 4, OOCS_OP_LOAD = 5,
       OOCS_OP_STEP = 6, OOCS_OP_STORE = 7 };
/* resources: the working buffer set, staging slots in / out, a host store */
enum { OOCS_RES_WORK = 1, OOCS_RES_IN_SLOT = 2, OOCS_RES_OUT_SLOT = 3, OOCS_RES_HOST = 4 };

typedef struct {
    int32_t kind;     /* OOCS_RES_*                                                 */
    int32_t index;    /* working-buffer set, slot number, or host field id          */
    int64_t lo, hi;   /* 4-plane layers [lo, hi) in global z                        */
    int32_t write;    /* 1 = written, 0 = read                                      */
    int32_t reserved;
} oocs_trace_access;

typedef struct {
    int32_t op;       /* OOCS_OP_*                                                  */
    int32_t stream;   /* 0..2                                                       */
    int32_t event;    /* WAIT / RECORD: event id (same id = same CUDA event); else -1 */
    int32_t naccess;
    int64_t visit;    /* slab visit number g of the op (-1 for events)              */
    oocs_trace_access access[4];
} oocs_trace_op;

/* Trace ncalls successive oocs_step(nsteps[i]) calls for `desc`.  Writes up to
 * `capacity` ops and the total needed to *count; OOCS_ERR_INVALID_ARG (with
 * *count set) when capacity is too small.  Allocates and frees host memory
 * only; touches no GPU.                                                    */
oocs_status oocs_trace_schedule(const oocs_desc *desc, const int32_t *nsteps, int32_t ncalls,
                                oocs_trace_op *ops, int64_t capacity, int64_t *count);

/* ---------------------------------------------------------------------------
 * Batches: many independent problems (any mix of HEAT and WAVE descs, each
 * with its own grid, T, k and rate, all OOCS_SWB) advanced through ONE
 * Algorithm-1 pipeline: one device workspace whose working buffer and staging
 * slots are sized for the largest problem (plus one resident model per WAVE
 * problem with readonly_resident), the same three streams, events and slab
 * visit sequence.  A batch step runs rounds in which every unfinished problem
 * sweeps its slabs once (k of its own steps), so copies of one problem's
 * visits overlap the kernels of another's.  Results are those of running each
 * problem alone with the same desc.  The paper has no batching; this is the
 * serving pattern built on its pipeline.
 * ------------------------------------------------------------------------- */
typedef struct oocs_batch oocs_batch;

/* Device workspace bytes a batch of the n descs needs. */
oocs_status oocs_batch_query(const oocs_desc *descs, int32_t n, uint64_t *workspace_bytes);

/* Create a batch on the current device: descs[0..n-1] (copied), a 256-byte
 * aligned device workspace of >= oocs_batch_query bytes and three distinct
 * streams, all owned by the caller and kept alive until oocs_batch_destroy.
 * Each problem is a context (oocs_batch_context) used with oocs_bind_field,
 * oocs_set_source, oocs_compress, oocs_decompress, oocs_set_time,
 * oocs_get_stats, oocs_set_profiling and oocs_step (that problem alone, through
 * the batch's pipeline); oocs_destroy refuses it.                          */
oocs_status oocs_batch_create(const oocs_desc *descs, int32_t n, void *workspace, uint64_t workspace_bytes,
                              void *const streams[3], oocs_batch **out);
oocs_status oocs_batch_context(oocs_batch *batch, int32_t i, oocs_ctx **ctx);

/* Advance every problem by nsteps (asynchronous; oocs_batch_synchronize). */
oocs_status oocs_batch_step(oocs_batch *batch, int32_t nsteps);

/* Capture one oocs_batch_step(nsteps) as a CUDA graph (nothing runs; the
 * problems' time indices and stats are unchanged), and replay it with
 * oocs_batch_launch, which advances every problem by nsteps per call with one
 * graph launch instead of thousands of launches and copies.  A replay always
 * follows all previously enqueued work, and may be mixed with direct steps.
 * Source amplitudes are read at replay time from a device copy of the
 * wavelet (made by oocs_set_source) at each problem's current time index, so
 * replays give the same results as direct steps.  OOCS_ERR_UNSUPPORTED if a
 * wavelet has more than 65536 samples; OOCS_ERR_STATE while profiling is on.
 * A new capture replaces the old one.                                      */
oocs_status oocs_batch_capture(oocs_batch *batch, int32_t nsteps);
oocs_status oocs_batch_launch(oocs_batch *batch);

/* Wait for everything enqueued on the batch (timeout_ns = 0: no limit). */
oocs_status oocs_batch_synchronize(oocs_batch *batch, uint64_t timeout_ns);
oocs_status oocs_batch_destroy(oocs_batch *batch);

/* oocs_trace_schedule for a batch: ncalls successive oocs_batch_step calls.
 * Host field ids are 3 i + field for problem i; d2h event ids are unique per
 * problem and slab.  No GPU is touched.                                    */
oocs_status oocs_batch_trace_schedule(const oocs_desc *descs, int32_t n, const int32_t *nsteps, int32_t ncalls,
                                      oocs_trace_op *ops, int64_t capacity, int64_t *count);

/* Library version string. */
const char *oocs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OOCS_H */
