// capi.cu -- the C ABI of include/oocs.h: planner, context, and the slab
// scheduler of the single-working-buffer pipeline.
//
// Scheduling (Sec. 5, Algorithm 1 "Conflict-free scheduling", Fig. 8).  Slab
// visits are numbered g = 0, 1, 2, ... over all sweeps; visit g runs on
// stream g % 3 and owns staging slot g % 3.  Its operations, in stream order:
//
//   wait  decoded[g-2]            staging slot g%3 is free (visit g-2 has read
//                                 the overlap it borrowed from slot (g-3)%3)
//   wait  d2h[s], d2h[s+1]        host layers it reads were written back by the
//                                 previous sweep (cross-sweep read-after-write)
//   H2D   new layers -> slot      region sharing: only layers not already on
//                                 the device (Sec. 3.1, Fig. 2)
//   record h2d[g]
//   wait  wrel[g-1], h2d[g-1]     the working buffer is free (SWB, Sec. 5) and
//                                 the borrowed overlap has landed
//   load  slot g-1 (overlap) + slot g -> working buffer (decode, Sec. 4.2)
//   record decoded[g]
//   k steps on the shrinking trapezoid (temporal blocking, Sec. 3.1)
//   store working buffer interior -> out slot (encode)
//   record wrel[g]
//   D2H   out slot -> host layers [z0, z1), in place
//   record d2h[s]
//
// This is the DAG of Fig. 8(a) with each stream waiting on its cyclic
// predecessor before touching the working buffer; it adds the two hazards the
// paper's listing leaves implicit (the borrowed overlap and the in-place host
// store across sweeps) and the missing epilogue (every visit enqueues its own
// compress and copy-back).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/oocs.h"
#include "capi_internal.h"
#include "kernels.h"
#include "stencil.cuh"

using namespace oocs;

namespace {

thread_local std::string g_last_error = "no error";

const char *kVersion = "oocs 0.1 (sm_103a)";

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

struct Layout {
    // byte offsets inside the workspace
    uint64_t w_off[3][4];     // [working buffer][buffer]
    uint64_t in_off[3][3];    // [slot][field_in]
    uint64_t out_off[3][2];   // [slot][field_out]
    uint64_t ro_off;          // resident FP32 copy of M (readonly_resident), else 0
    uint64_t ro_bytes;
    uint64_t src_off;         // wave: device time index + wavelet (graph replays), else 0
    uint64_t g_off;           // adjoint: dJ/dm on the device, else 0
    uint64_t total;
    int nwb;                  // working buffers (1 SWB, 3 classic)
    int nbuf;                 // buffers per working set (heat 2, wave 3, adjoint 4)
    uint64_t buf_bytes;       // one window buffer
    uint64_t in_slot_bytes;   // one staging slot of one field
    uint64_t out_slot_bytes;
};

// wavelet samples a context keeps on the device for replayed graphs
constexpr int64_t kMaxDeviceWavelet = 1 << 16;
constexpr uint64_t kSrcRegionBytes = 256 + (uint64_t)kMaxDeviceWavelet * 4;

struct Derived {
    int r, k, h, T, S, wp, fin, fout;
    int fin_stream;  // fields crossing the link per visit (fin minus a resident M)
    bool ro_res;     // M kept on the device
    uint64_t layer_bytes;
    int64_t slot_layers_in, slot_layers_out;
};

// fields bound to host stores: heat U; wave U, U_PREV, M; adjoint LAM, LAM_PREV, M, FWD
int bound_fields(const oocs_desc &d) { return d.scheme == OOCS_HEAT ? 1 : d.scheme == OOCS_WAVE ? 3 : 4; }

Derived derive(const oocs_desc &d, int T)
{
    Derived v;
    v.r = d.radius;
    v.k = d.scheme == OOCS_WAVE_ADJOINT ? 1 : d.temporal_depth > 0 ? d.temporal_depth : 4;
    v.h = (int)(4 * ceil_div((int64_t)v.k * v.r, 4));
    v.T = T;
    v.S = (int)ceil_div(d.nz, T);
    v.wp = (int)std::min<int64_t>(T + 2 * (int64_t)v.h, d.nz);
    v.fin = d.scheme == OOCS_WAVE ? 3 : 1;
    v.fout = d.scheme == OOCS_WAVE ? 2 : 1;
    v.ro_res = d.scheme == OOCS_WAVE && d.readonly_resident != 0;
    v.fin_stream = v.fin - (v.ro_res ? 1 : 0);
    if (d.scheme == OOCS_WAVE_ADJOINT) {  // in: LAM, LAM_PREV, FWD; out: LAM_PREV; M resident
        v.fin = v.fin_stream = 3;
        v.fout = 1;
        v.ro_res = true;
    }
    v.layer_bytes = d.rate_bits > 0 ? (uint64_t)(d.nx / 4) * (d.ny / 4) * 8ull * d.rate_bits
                                    : (uint64_t)4 * d.nx * d.ny * 4;
    // region sharing leaves T + h new planes per visit; the adjoint copies whole windows
    v.slot_layers_in = std::min<int64_t>(ceil_div(d.scheme == OOCS_WAVE_ADJOINT ? v.wp : T + v.h, 4), d.nz / 4);
    v.slot_layers_out = std::min<int64_t>(T / 4, d.nz / 4);
    return v;
}

Layout layout_for(const oocs_desc &d, const Derived &v, int nwb)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    L.nwb = nwb;
    // window buffers: heat u, u'; wave u, u_prev and m (m lives in the
    // resident copy when readonly_resident)
    L.nbuf = d.scheme == OOCS_WAVE && !v.ro_res ? 3 : 2;
    if (d.scheme == OOCS_WAVE_ADJOINT)
        L.nbuf = 4;  // lam^k, lam^(k+1) -> lam^(k-1), u^(k-1), m lam^k
    L.buf_bytes = align_up((uint64_t)v.wp * d.nx * d.ny * 4, 256);
    L.in_slot_bytes = align_up((uint64_t)v.slot_layers_in * v.layer_bytes, 256);
    L.out_slot_bytes = align_up((uint64_t)v.slot_layers_out * v.layer_bytes, 256);
    uint64_t off = 0;
    for (int w = 0; w < nwb; ++w)
        for (int b = 0; b < L.nbuf; ++b) {
            L.w_off[w][b] = off;
            off += L.buf_bytes;
        }
    for (int q = 0; q < 3; ++q)
        for (int f = 0; f < v.fin_stream; ++f) {
            L.in_off[q][f] = off;
            off += L.in_slot_bytes;
        }
    for (int q = 0; q < 3; ++q)
        for (int f = 0; f < v.fout; ++f) {
            L.out_off[q][f] = off;
            off += L.out_slot_bytes;
        }
    if (v.ro_res) {
        L.ro_off = off;
        L.ro_bytes = align_up((uint64_t)d.nz * d.nx * d.ny * 4, 256);
        off += L.ro_bytes;
    }
    if (d.scheme == OOCS_WAVE) {
        L.src_off = off;
        off += kSrcRegionBytes;
    }
    if (d.scheme == OOCS_WAVE_ADJOINT) {  // dJ/dm, accumulated on the device
        L.g_off = off;
        off += align_up((uint64_t)d.nz * d.nx * d.ny * 4, 256);
    }
    L.total = off;
    return L;
}

oocs_status validate_desc(const oocs_desc *d, std::string &err)
{
    if (!d) {
        err = "desc is NULL";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->nx < 4 || d->ny < 4 || d->nz < 4 || d->nx % 4 || d->ny % 4 || d->nz % 4) {
        err = "nx, ny, nz must be positive multiples of 4";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->nx > (1 << 30) || d->ny > (1 << 30) || d->nz > (1 << 30)) {
        err = "grid dimension too large";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->scheme != OOCS_HEAT && d->scheme != OOCS_WAVE && d->scheme != OOCS_WAVE_ADJOINT) {
        err = "scheme must be OOCS_HEAT, OOCS_WAVE or OOCS_WAVE_ADJOINT";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->scheme == OOCS_WAVE_ADJOINT &&
        (d->radius != 4 || d->temporal_depth > 1 || d->readonly_resident != 1 || d->working_buffers != OOCS_SWB)) {
        err = "the wave adjoint needs radius 4, temporal_depth 1, readonly_resident 1 and one working buffer";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->radius != 1 && d->radius != 4) {
        err = "radius must be 1 or 4";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->scheme == OOCS_WAVE && d->radius != 4) {
        err = "the wave scheme uses the 25-point star (radius 4)";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->nx <= 2 * d->radius || d->ny <= 2 * d->radius || d->nz <= 2 * d->radius) {
        err = "grid must be larger than the Dirichlet shell";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->rate_bits < 0 || d->rate_bits > 32) {
        err = "rate_bits must be 0 (uncompressed) or 1..32";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->codec != OOCS_CODEC_TRANSFORM && d->codec != OOCS_CODEC_QUANT) {
        err = "codec must be OOCS_CODEC_TRANSFORM (0) or OOCS_CODEC_QUANT (1)";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->codec_fusion != 0 && d->codec_fusion != 1) {
        err = "codec_fusion must be 0 or 1";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->codec_fusion == 1 && d->step_fusion == 1) {
        err = "codec_fusion and step_fusion cannot both be 1";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->step_tile != 0 && d->step_tile != 1) {
        err = "step_tile must be 0 or 1";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->step_fusion != 0 && d->step_fusion != 1) {
        err = "step_fusion must be 0 or 1";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->codec == OOCS_CODEC_QUANT && d->rate_bits == 1) {
        err = "the block quantiser needs rate_bits >= 2";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->temporal_depth < 0 || d->temporal_depth > 64) {
        err = "temporal_depth must be 0 (auto) or 1..64";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->slab_planes < 0 || d->slab_planes % 4) {
        err = "slab_planes must be 0 (auto) or a positive multiple of 4";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->working_buffers != OOCS_SWB && d->working_buffers != OOCS_CLASSIC) {
        err = "working_buffers must be 1 (SWB) or 3 (classic)";
        return OOCS_ERR_INVALID_ARG;
    }
    if (d->readonly_resident != 0 && d->readonly_resident != 1) {
        err = "readonly_resident must be 0 or 1";
        return OOCS_ERR_INVALID_ARG;
    }
    return OOCS_OK;
}

bool slab_ok(const oocs_desc &d, int T, int h)
{
    if (T < 4 || T % 4)
        return false;
    if (T >= d.nz)
        return true;    // one slab
    return T >= 2 * h;  // the overlap of slab s lies in slab s-1's staging slot
}

oocs_status plan_impl(const oocs_desc *d, oocs_plan *p, std::string &err)
{
    oocs_status st = validate_desc(d, err);
    if (st != OOCS_OK)
        return st;
    if (!p) {
        err = "plan is NULL";
        return OOCS_ERR_INVALID_ARG;
    }
    const int nwb = d->working_buffers;
    int T = d->slab_planes;
    Derived v0 = derive(*d, 4);
    if (T > 0) {
        if (T > d->nz)
            T = (int)d->nz;
        if (!slab_ok(*d, T, v0.h)) {
            err = "slab_planes must be >= 2 * halo (" + std::to_string(2 * v0.h) + ") when nz > T";
            return OOCS_ERR_INVALID_ARG;
        }
        Derived v = derive(*d, T);
        if (layout_for(*d, v, nwb).total > d->device_budget) {
            err = "slab of " + std::to_string(T) + " planes needs " +
                  std::to_string(layout_for(*d, v, nwb).total) + " bytes > device_budget";
            return OOCS_ERR_BUDGET;
        }
    } else {
        int best = 0;
        for (int64_t t = 4; t <= d->nz; t += 4) {
            if (!slab_ok(*d, (int)t, v0.h))
                continue;
            Derived v = derive(*d, (int)t);
            if (layout_for(*d, v, nwb).total <= d->device_budget)
                best = (int)t;
            else if (best)
                break;
        }
        if (!best) {
            err = "no slab thickness fits device_budget";
            return OOCS_ERR_BUDGET;
        }
        T = best;
    }
    Derived v = derive(*d, T);
    memset(p, 0, sizeof(*p));
    p->slab_planes = T;
    p->temporal_depth = v.k;
    p->halo_planes = v.h;
    p->num_slabs = v.S;
    p->window_planes = v.wp;
    p->fields_in = v.fin_stream;
    p->fields_out = v.fout;
    p->readonly_resident = v.ro_res ? 1 : 0;
    p->layer_bytes = v.layer_bytes;
    p->host_store_bytes = (uint64_t)(d->nz / 4) * v.layer_bytes;
    p->workspace_bytes = layout_for(*d, v, nwb).total;
    p->workspace_swb_bytes = layout_for(*d, v, 1).total;
    p->workspace_classic_bytes = layout_for(*d, v, 3).total;
    return OOCS_OK;
}

}  // namespace

void oocs::set_last_error(const std::string &msg) { g_last_error = msg; }

struct oocs_batch;

struct oocs_ctx {
    oocs_desc d;
    oocs_plan p;
    Derived v;
    Layout L;
    char *ws = nullptr;
    cudaStream_t st[3] = {};
    char *store[4] = {};  // by field id (bound_fields of the scheme)
    int store_id[4] = {0, 1, 2, 3};  // trace: the physical store behind each field (the
                                     // adjoint's LAM and LAM_PREV stores trade roles every step)
    uint64_t store_bytes[4] = {};

    bool has_src = false;
    int64_t src[3] = {0, 0, -1};
    std::vector<float> w;

    // receiver plane: WAVE records plane zr of u^(t+1) into planes[t] after
    // every step t < nplanes (device array [nplanes][ny][nx])
    float *rec = nullptr;
    int64_t rec_z = -1, rec_n = 0;

    // state record (oocs_set_state_record): host stores receiving the encoded
    // states u^t a visit writes, srec[t - srec_t0] (null entries skipped)
    std::vector<char *> srec;
    int64_t srec_t0 = 0;

    cudaEvent_t ev_decoded[3] = {}, ev_h2d[3] = {}, ev_wrel[3] = {}, ev_join[3] = {};
    cudaEvent_t ev_out[3] = {};    // out slot q copied back (streams by role)
    cudaEvent_t ev_codec[2] = {};  // oocs_compress / oocs_decompress: a chunk's raw copy has run
    std::vector<cudaEvent_t> ev_d2h;
    std::vector<char> d2h_recorded;
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
    bool timing_pending = false;

    uint64_t g = 0;  // slab visits enqueued
    oocs_stats stats;
    bool ro_dirty = true;  // resident M must be (re)made from its store

    // trace mode (oocs_trace_schedule): scheduling operations are recorded
    // here instead of being issued to CUDA
    std::vector<oocs_trace_op> *trace = nullptr;

    // per-launch event timing (oocs_set_profiling): bit mask of kernel classes
    int prof = 0;
    std::vector<cudaEvent_t> ev_pool;  // created on demand, reused after collection
    size_t ev_used = 0;
    struct Pending {
        int cls, stream;
        int64_t visit;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<oocs_timeline_entry> timeline;  // of the last collection
    oocs_status sticky = OOCS_OK;
    std::string err = "no error";

    // host-side fault injection (oocs_set_fault_injection): the inject_at-th
    // CUDA call checked after arming is reported as failed
    int64_t inject_at = 0, inject_seen = 0;

    // member of a batch (oocs_batch_create): the workspace, the three streams,
    // the Algorithm-1 events and the visit counter belong to the batch
    oocs_batch *batch = nullptr;
    int host_base = 0;  // trace: host field ids of this problem start here
    int d2h_base = 0;   // trace: d2h event ids of this problem start here

    float *wbuf(int wb, int b) const { return reinterpret_cast<float *>(ws + L.w_off[wb][b]); }
    char *in_slot(int q, int f) const { return ws + L.in_off[q][f]; }
    char *out_slot(int q, int f) const { return ws + L.out_off[q][f]; }
    float *ro_m() const { return reinterpret_cast<float *>(ws + L.ro_off); }
    float *grad() const { return reinterpret_cast<float *>(ws + L.g_off); }
    int64_t *t_dev() const { return reinterpret_cast<int64_t *>(ws + L.src_off); }
    float *w_dev() const { return reinterpret_cast<float *>(ws + L.src_off + 256); }
    int64_t t_capture = 0;  // time index when the batch's graph was captured
};

// A batch of independent problems advanced through one Algorithm-1 pipeline:
// one workspace (every region sized for the largest problem, so visits of
// different problems use the same staging slots and working buffer), three
// streams, one set of events and one visit counter.
struct oocs_batch {
    std::vector<oocs_ctx *> ctx;
    char *ws = nullptr;
    cudaStream_t st[3] = {};
    cudaEvent_t ev_decoded[3] = {}, ev_h2d[3] = {}, ev_wrel[3] = {}, ev_join[3] = {}, ev_out[3] = {};
    uint64_t g = 0;
    std::vector<oocs_trace_op> *trace = nullptr;
    // CUDA graph of one oocs_batch_step (oocs_batch_capture / oocs_batch_launch)
    bool capturing = false;
    std::vector<cudaEvent_t> cap_recorded;  // events recorded since the capture began
    cudaGraphExec_t exec = nullptr;
    int32_t graph_steps = 0;
    std::vector<oocs_stats> graph_delta;  // per problem: what one replay enqueues
    bool recorded_in_capture(cudaEvent_t e) const
    {
        return std::find(cap_recorded.begin(), cap_recorded.end(), e) != cap_recorded.end();
    }
};

namespace {

oocs_status fail(oocs_ctx *c, oocs_status s, const std::string &msg)
{
    if (c) {
        c->err = msg;
        if (s == OOCS_ERR_CUDA || s == OOCS_ERR_TIMEOUT || s == OOCS_ERR_NONFINITE)
            c->sticky = s;
    } else {
        g_last_error = msg;
    }
    return s;
}

// true when fault injection is armed on c and this checked call is the one
// chosen to fail
bool inject_now(oocs_ctx *c)
{
    return c && c->inject_at > 0 && ++c->inject_seen == c->inject_at;
}

#define CU(ctx, call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), OOCS_ERR_CUDA,                                                \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
        if (inject_now(ctx))                                                                 \
            return fail((ctx), OOCS_ERR_CUDA, std::string(#call) + ": injected failure");    \
    } while (0)

// in-field index -> context field id
int in_field_id(const oocs_ctx *c, int f)
{
    (void)c;
    return f;  // heat: U; wave: U, U_PREV, M
}

// make every stream wait for the work enqueued so far on all three
oocs_status sched_record(oocs_ctx *c, int si, int ev);
oocs_status sched_wait(oocs_ctx *c, int si, int ev);

oocs_status join_streams(oocs_ctx *c)
{
    for (int i = 0; i < 3; ++i) {
        oocs_status r = sched_record(c, i, 400 + i);
        if (r != OOCS_OK)
            return r;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (i != j) {
                oocs_status r = sched_wait(c, i, 400 + j);
                if (r != OOCS_OK)
                    return r;
            }
    return OOCS_OK;
}

oocs_status check_ready(oocs_ctx *c)
{
    if (!c)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "ctx is NULL");
    if (c->sticky != OOCS_OK)
        return c->sticky;
    return OOCS_OK;
}

// ---- scheduling primitives: issued to CUDA, or recorded in trace mode

enum : int { kEvDecoded = 100, kEvH2D = 200, kEvWrel = 300, kEvJoin = 400, kEvT0 = 500, kEvT1 = 501,
             kEvOut = 600, kEvD2H = 1000 };

cudaEvent_t event_of(oocs_ctx *c, int id)
{
    if (id >= kEvD2H)
        return c->ev_d2h[id - kEvD2H - c->d2h_base];
    if (id == kEvT0)
        return c->ev_t0;
    if (id == kEvT1)
        return c->ev_t1;
    switch (id / 100) {
    case 1: return c->ev_decoded[id % 100];
    case 2: return c->ev_h2d[id % 100];
    case 3: return c->ev_wrel[id % 100];
    case 6: return c->ev_out[id % 100];
    default: return c->ev_join[id % 100];
    }
}

void trace_push(oocs_ctx *c, int op, int si, int ev, int64_t visit,
                std::initializer_list<oocs_trace_access> acc)
{
    oocs_trace_op t;
    memset(&t, 0, sizeof(t));
    t.op = op;
    t.stream = si;
    t.event = ev;
    t.visit = visit;
    for (const auto &a : acc)
        if (t.naccess < 4)
            t.access[t.naccess++] = a;
    c->trace->push_back(t);
}

oocs_trace_access acc(int kind, int index, int64_t lo, int64_t hi, bool write)
{
    oocs_trace_access a;
    memset(&a, 0, sizeof(a));
    a.kind = kind;
    a.index = index;
    a.lo = lo;
    a.hi = hi;
    a.write = write ? 1 : 0;
    return a;
}

oocs_status sched_wait(oocs_ctx *c, int si, int ev)
{
    if (c->trace) {
        trace_push(c, OOCS_OP_WAIT, si, ev, -1, {});
        return OOCS_OK;
    }
    cudaEvent_t e = event_of(c, ev);
    // inside a graph capture, an event last recorded before the capture began
    // belongs to work that a replay always follows (oocs_batch_launch joins
    // the streams first): its wait is dropped
    if (c->batch && c->batch->capturing && !c->batch->recorded_in_capture(e))
        return OOCS_OK;
    CU(c, cudaStreamWaitEvent(c->st[si], e, 0));
    return OOCS_OK;
}

oocs_status sched_record(oocs_ctx *c, int si, int ev)
{
    if (c->trace) {
        trace_push(c, OOCS_OP_RECORD, si, ev, -1, {});
        return OOCS_OK;
    }
    cudaEvent_t e = event_of(c, ev);
    if (c->batch && c->batch->capturing)
        c->batch->cap_recorded.push_back(e);
    CU(c, cudaEventRecord(e, c->st[si]));
    return OOCS_OK;
}

#define SCHED(call)                  \
    do {                             \
        oocs_status r_ = (call);     \
        if (r_ != OOCS_OK)           \
            return r_;               \
    } while (0)

enum { kClsLoad = 0, kClsStep = 1, kClsStore = 2, kClsH2D = 3, kClsD2H = 4 };

oocs_kernel_stats &cls_stats(oocs_ctx *c, int cls)
{
    switch (cls) {
    case kClsLoad: return c->stats.load;
    case kClsStep: return c->stats.step;
    case kClsStore: return c->stats.store;
    case kClsH2D: return c->stats.h2d;
    default: return c->stats.d2h;
    }
}

oocs_status take_event(oocs_ctx *c, cudaEvent_t *e)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t n = nullptr;
        CU(c, cudaEventCreate(&n));
        c->ev_pool.push_back(n);
    }
    *e = c->ev_pool[c->ev_used++];
    return OOCS_OK;
}

// Bracket one kernel (or device copy) of class `cls` on stream s: counts it
// and, while profiling, records events around it.
struct KernelScope {
    oocs_ctx *c;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    oocs_status begin(oocs_ctx *cc, cudaStream_t ss, int cls)
    {
        c = cc;
        s = ss;
        if (!(c->prof & (1 << cls)))
            return OOCS_OK;
        oocs_status r = take_event(c, &a);
        if (r != OOCS_OK)
            return r;
        CU(c, cudaEventRecord(a, s));
        return OOCS_OK;
    }
    oocs_status end(int cls, uint64_t units, uint64_t launches = 1)
    {
        oocs_kernel_stats &k = cls_stats(c, cls);
        k.launches += launches;
        k.units += units;
        if (!a)
            return OOCS_OK;
        cudaEvent_t b;
        oocs_status r = take_event(c, &b);
        if (r != OOCS_OK)
            return r;
        CU(c, cudaEventRecord(b, s));
        int si = 0;
        while (si < 2 && c->st[si] != s)
            ++si;
        c->pending.push_back({cls, si, (int64_t)c->g, a, b});
        return OOCS_OK;
    }
};

// fold the durations of completed profiled launches into the stats
void collect_profile(oocs_ctx *c)
{
    if (!c->pending.empty())
        c->timeline.clear();
    for (const auto &p : c->pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            cls_stats(c, p.cls).device_ms += ms;
        float t0 = 0.0f, t1 = 0.0f;
        if (cudaEventElapsedTime(&t0, c->ev_t0, p.a) == cudaSuccess &&
            cudaEventElapsedTime(&t1, c->ev_t0, p.b) == cudaSuccess)
            c->timeline.push_back({p.cls, p.stream, p.visit, (double)t0, (double)t1});
        cudaGetLastError();
    }
    c->pending.clear();
    c->ev_used = 0;
}

// Copy (rate 0) or decode (rate > 0) layers [l0, l1) held in staging memory
// `src` (whose first layer is src_l0) into window buffer `dst` (first plane w0).
oocs_status load_layers(oocs_ctx *c, const char *src, int64_t src_l0, int64_t l0, int64_t l1,
                        float *dst, int64_t w0, cudaStream_t s)
{
    if (l1 <= l0)
        return OOCS_OK;
    const char *from = src + (l0 - src_l0) * c->v.layer_bytes;
    float *to = dst + (4 * l0 - w0) * c->d.nx * c->d.ny;
    KernelScope ks;
    oocs_status r = ks.begin(c, s, kClsLoad);
    if (r != OOCS_OK)
        return r;
    if (c->d.rate_bits == 0) {
        CU(c, cudaMemcpyAsync(to, from, (l1 - l0) * c->v.layer_bytes, cudaMemcpyDeviceToDevice, s));
    } else {
        CU(c, launch_decode_layers(from, c->d.nx, c->d.ny, l1 - l0, c->d.rate_bits, c->d.codec, to, s));
        c->stats.kernel_launches++;
    }
    return ks.end(kClsLoad, (uint64_t)(l1 - l0) * 4 * c->d.nx * c->d.ny);
}

// Copy (rate 0) or encode (rate > 0) window planes of layers [l0, l1) into `dst`.
oocs_status store_layers(oocs_ctx *c, const float *src, int64_t w0, int64_t l0, int64_t l1,
                         char *dst, cudaStream_t s)
{
    if (l1 <= l0)
        return OOCS_OK;
    const float *from = src + (4 * l0 - w0) * c->d.nx * c->d.ny;
    KernelScope ks;
    oocs_status r = ks.begin(c, s, kClsStore);
    if (r != OOCS_OK)
        return r;
    if (c->d.rate_bits == 0) {
        CU(c, cudaMemcpyAsync(dst, from, (l1 - l0) * c->v.layer_bytes, cudaMemcpyDeviceToDevice, s));
    } else {
        CU(c, launch_encode_layers(from, c->d.nx, c->d.ny, l1 - l0, c->d.rate_bits, c->d.codec, dst, s));
        c->stats.kernel_launches++;
    }
    return ks.end(kClsStore, (uint64_t)(l1 - l0) * 4 * c->d.nx * c->d.ny);
}

// Make the resident FP32 copy of M (readonly_resident) from its host store,
// on stream 0: raw planes are copied; compressed layers go in chunks of T
// planes through staging slot 0 and are decoded into place, so the resident
// values are exactly those a per-visit decode would produce.
oocs_status upload_resident(oocs_ctx *c)
{
    const oocs_desc &d = c->d;
    const Derived &v = c->v;
    cudaStream_t st = c->st[0];
    const int64_t plane_f = d.nx * d.ny;
    const char *store = c->store[OOCS_FIELD_M];
    if (d.rate_bits == 0) {
        const uint64_t bytes = (uint64_t)d.nz * plane_f * 4;
        CU(c, cudaMemcpyAsync(c->ro_m(), store, bytes, cudaMemcpyHostToDevice, st));
        c->stats.h2d_bytes += bytes;
    } else {
        char *blk = c->in_slot(0, 0);  // holds slot_layers_in >= T/4 layers
        for (int64_t z0 = 0; z0 < d.nz; z0 += v.T) {
            const int64_t z1 = std::min<int64_t>(z0 + v.T, d.nz);
            const uint64_t bytes = (uint64_t)(z1 - z0) / 4 * v.layer_bytes;
            CU(c, cudaMemcpyAsync(blk, store + (uint64_t)(z0 / 4) * v.layer_bytes, bytes, cudaMemcpyHostToDevice,
                                  st));
            CU(c, launch_decode_layers(blk, d.nx, d.ny, (z1 - z0) / 4, d.rate_bits, d.codec, c->ro_m() + z0 * plane_f, st));
            c->stats.h2d_bytes += bytes;
            c->stats.kernel_launches++;
        }
    }
    c->ro_dirty = false;
    return OOCS_OK;
}

// Enqueue one slab visit (slab s, k_eff steps starting at global time t).
oocs_status enqueue_slab(oocs_ctx *c, int s, int k_eff, int64_t t)
{
    const Derived &v = c->v;
    const oocs_desc &d = c->d;
    const uint64_t g = c->g;
    const int q = (int)(g % 3);
    const int qp = (int)((g + 2) % 3);  // slot of visit g-1
    const int wb = (d.working_buffers == OOCS_SWB) ? 0 : q;
    // Streams by role with one working buffer: host->device copies on stream
    // 0, kernels on stream 1, device->host copies on stream 2, ordered by the
    // same events as Algorithm 1 (Fig. 8a).  With the round robin of the
    // listing (visit g's copies and kernels all on stream g % 3) a visit's
    // next copy waits in its stream behind the copy-back of the visit three
    // before, and on GB300 kernels of one visit were then measured waiting
    // for the copies of the next (every other visit idle ~7 ms of ~12).
    // Classic mode (three working buffers) keeps the round robin, whose
    // kernels of consecutive visits may overlap.
    const bool roles = d.working_buffers == OOCS_SWB;
    const int sh = roles ? 0 : q, sk = roles ? 1 : q, sd = roles ? 2 : q;
    cudaStream_t st_h = c->st[sh], st_k = c->st[sk], st_d = c->st[sd];

    const int64_t z0 = (int64_t)s * v.T;
    const int64_t z1 = std::min<int64_t>(z0 + v.T, d.nz);
    const int64_t w0 = std::max<int64_t>(z0 - v.h, 0);
    const int64_t w1 = std::min<int64_t>(z1 + v.h, d.nz);
    // layers new to the device: all of the window for the first slab of a
    // sweep, else only what lies above the overlap kept from slab s-1
    const int64_t n0 = (s == 0) ? w0 : std::min<int64_t>(z0 + v.h, w1);
    const int64_t n1 = w1;

    // 1. staging slot q is free once visit g-2 has read its borrowed overlap
    if (g >= 2)
        SCHED(sched_wait(c, sh, kEvDecoded + (int)((g - 2) % 3)));
    // 2. host layers [n0, n1) were last written by slabs s and s+1 of the previous sweep
    for (int ss = s; ss <= s + 1 && ss < v.S; ++ss)
        if (c->d2h_recorded[ss])
            SCHED(sched_wait(c, sh, kEvD2H + c->d2h_base + ss));
    // 3. H2D of the new layers of every streamed field
    if (c->trace) {
        if (n1 > n0) {
            oocs_trace_access a[4] = {acc(OOCS_RES_IN_SLOT, q, n0 / 4, n1 / 4, true)};
            for (int f = 0; f < v.fin_stream; ++f)
                a[1 + f] = acc(OOCS_RES_HOST, c->host_base + in_field_id(c, f), n0 / 4, n1 / 4, false);
            trace_push(c, OOCS_OP_H2D, sh, -1, (int64_t)g, {a[0], a[1]});
            for (int f = 1; f < v.fin_stream; ++f)
                c->trace->back().access[c->trace->back().naccess++] = a[1 + f];
        }
    } else {
        KernelScope ks;
        oocs_status r = ks.begin(c, st_h, kClsH2D);
        if (r != OOCS_OK)
            return r;
        for (int f = 0; f < v.fin_stream; ++f) {
            const int id = in_field_id(c, f);
            const uint64_t bytes = (uint64_t)(n1 - n0) / 4 * v.layer_bytes;
            if (bytes) {
                CU(c, cudaMemcpyAsync(c->in_slot(q, f), c->store[id] + (uint64_t)(n0 / 4) * v.layer_bytes,
                                      bytes, cudaMemcpyHostToDevice, st_h));
            }
        }
        r = ks.end(kClsH2D, (uint64_t)v.fin_stream * (uint64_t)(n1 - n0) / 4 * v.layer_bytes);
        if (r != OOCS_OK)
            return r;
    }
    c->stats.h2d_bytes += (uint64_t)v.fin_stream * (uint64_t)(n1 - n0) / 4 * v.layer_bytes;
    SCHED(sched_record(c, sh, kEvH2D + q));
    // 4. the visit's own layers have landed (when copies have a stream of
    //    their own); the working buffer is released by visit g-1 (single
    //    working buffer); the overlap borrowed from visit g-1's slot has landed
    if (roles)
        SCHED(sched_wait(c, sk, kEvH2D + q));
    if (g >= 1 && d.working_buffers == OOCS_SWB)
        SCHED(sched_wait(c, sk, kEvWrel + (int)((g - 1) % 3)));
    if (s > 0)
        SCHED(sched_wait(c, sk, kEvH2D + qp));
    // 5. load / decode the window at time t
    // slot of slab s-1 holds layers starting at its own n0
    const int64_t pz0 = (int64_t)(s - 1) * v.T;
    const int64_t pn0 = (s <= 1) ? 0 : pz0 + v.h;
    const int64_t plane_f = d.nx * d.ny;
    // heat with codec_fusion: step 1 decodes the window itself (shared memory
    // only), so there is no decode launch and the staging slots are released
    // after step 1
    const bool dec_fused = d.codec_fusion == 1 && d.scheme == OOCS_HEAT && d.radius == 1 && d.rate_bits > 0 &&
                           d.codec == OOCS_CODEC_TRANSFORM && d.step_fusion == 0;
    if (dec_fused) {
        // decoded by step 1 (below): counted as loaded, with no launch of its own
        c->stats.load.units += (uint64_t)v.fin_stream * (w1 - w0) * plane_f;
    } else if (c->trace) {
        if (s > 0)
            trace_push(c, OOCS_OP_LOAD, sk, -1, (int64_t)g,
                       {acc(OOCS_RES_IN_SLOT, qp, w0 / 4, n0 / 4, false),
                        acc(OOCS_RES_IN_SLOT, q, n0 / 4, n1 / 4, false),
                        acc(OOCS_RES_WORK, wb, w0 / 4, w1 / 4, true)});
        else
            trace_push(c, OOCS_OP_LOAD, sk, -1, (int64_t)g,
                       {acc(OOCS_RES_IN_SLOT, q, n0 / 4, n1 / 4, false),
                        acc(OOCS_RES_WORK, wb, w0 / 4, w1 / 4, true)});
    } else if (d.rate_bits > 0) {
        // one decode launch for every field and both source slots
        CodecSegments sg;
        int64_t nl[kMaxCodecSegments];
        for (int f = 0; f < v.fin_stream; ++f) {
            float *dst = c->wbuf(wb, f);  // heat: U -> buf 0; wave: U, U_PREV, M -> 0, 1, 2
            if (s > 0 && n0 > w0) {
                sg.blocks[sg.nseg] = c->in_slot(qp, f) + (w0 / 4 - pn0 / 4) * v.layer_bytes;
                sg.planes[sg.nseg] = dst;
                nl[sg.nseg++] = (n0 - w0) / 4;
            }
            if (n1 > n0) {
                sg.blocks[sg.nseg] = c->in_slot(q, f);
                sg.planes[sg.nseg] = dst + (n0 - w0) * plane_f;
                nl[sg.nseg++] = (n1 - n0) / 4;
            }
        }
        KernelScope ks;
        oocs_status r = ks.begin(c, st_k, kClsLoad);
        if (r != OOCS_OK)
            return r;
        CU(c, launch_decode_segments(sg, nl, d.nx, d.ny, d.rate_bits, d.codec, st_k));
        c->stats.kernel_launches++;
        r = ks.end(kClsLoad, (uint64_t)v.fin_stream * (w1 - w0) * plane_f);
        if (r != OOCS_OK)
            return r;
    } else {
        for (int f = 0; f < v.fin_stream; ++f) {
            float *dst = c->wbuf(wb, f);
            if (s > 0) {
                oocs_status r = load_layers(c, c->in_slot(qp, f), pn0 / 4, w0 / 4, n0 / 4, dst, w0, st_k);
                if (r != OOCS_OK)
                    return r;
            }
            oocs_status r = load_layers(c, c->in_slot(q, f), n0 / 4, n0 / 4, n1 / 4, dst, w0, st_k);
            if (r != OOCS_OK)
                return r;
        }
    }
    if (!dec_fused)
        SCHED(sched_record(c, sk, kEvDecoded + q));

    // 6. k_eff steps over the shrinking trapezoid
    int cur = 0, oth = 1;
    StepLaunch Ls;
    memset(&Ls, 0, sizeof(Ls));
    Ls.scheme = d.scheme == OOCS_WAVE ? kWave : kHeat;
    Ls.radius = d.radius;
    Ls.tile = d.step_tile;
    Ls.nx = d.nx;
    Ls.ny = d.ny;
    Ls.nz = d.nz;
    Ls.gz0 = w0;
    Ls.wp = w1 - w0;
    for (int i = 0; i <= d.radius; ++i)
        Ls.coef[i] = d.coef[i];
    // the k step launches of a visit are timed as one group (two events per
    // visit), so profiling does not sit between consecutive step kernels
    KernelScope ks_steps;
    {
        oocs_status r = ks_steps.begin(c, st_k, kClsStep);
        if (r != OOCS_OK)
            return r;
    }
    uint64_t step_units = 0;
    // heat: pairs of steps in one fused launch (the middle step on chip)
    const bool fuse = d.scheme == OOCS_HEAT && d.radius == 1 && d.step_fusion == 1;
    // heat: the last step encodes the interior into the out slot itself,
    // which must then be free before the steps (copied back by visit g-3)
    // (a single step that also decodes leaves the encode to its own kernel)
    const bool enc_fused = d.codec_fusion == 1 && d.scheme == OOCS_HEAT && d.radius == 1 && d.rate_bits > 0 &&
                           d.codec == OOCS_CODEC_TRANSFORM && !fuse && !(dec_fused && k_eff == 1);
    if (enc_fused && roles && g >= 3)
        SCHED(sched_wait(c, sk, kEvOut + q));
    uint64_t launches = 0;
    for (int j = 1; j <= k_eff; ++j) {
        if (fuse && j + 1 <= k_eff) {
            const int64_t lo1 = std::max<int64_t>(z0 - (int64_t)(k_eff - j) * v.r, 0);
            const int64_t hi1 = std::min<int64_t>(z1 + (int64_t)(k_eff - j) * v.r, d.nz);
            const int64_t lo = std::max<int64_t>(z0 - (int64_t)(k_eff - j - 1) * v.r, 0);
            const int64_t hi = std::min<int64_t>(z1 + (int64_t)(k_eff - j - 1) * v.r, d.nz);
            Ls.z_lo = lo - w0;
            Ls.z_hi = hi - w0;
            Ls.cur = c->wbuf(wb, cur);
            Ls.out = c->wbuf(wb, oth);
            if (c->trace)
                trace_push(c, OOCS_OP_STEP, sk, -1, (int64_t)g, {acc(OOCS_RES_WORK, wb, w0 / 4, w1 / 4, true)});
            else
                CU(c, launch_heat_step2(Ls, st_k));
            c->stats.kernel_launches++;
            ++launches;
            step_units += (uint64_t)(hi1 - lo1 + hi - lo) * d.nx * d.ny;
            std::swap(cur, oth);
            ++j;
            continue;
        }
        const int64_t lo = std::max<int64_t>(z0 - (int64_t)(k_eff - j) * v.r, 0);
        const int64_t hi = std::min<int64_t>(z1 + (int64_t)(k_eff - j) * v.r, d.nz);
        Ls.z_lo = lo - w0;
        Ls.z_hi = hi - w0;
        Ls.cur = c->wbuf(wb, cur);
        Ls.prev = c->wbuf(wb, oth);
        Ls.m = d.scheme != OOCS_WAVE ? nullptr : v.ro_res ? c->ro_m() + w0 * plane_f : c->wbuf(wb, 2);
        Ls.out = c->wbuf(wb, oth);
        const int64_t tstep = t + j - 1;
        Ls.src_z = -1;
        Ls.w = 0.0f;
        Ls.w_dev = nullptr;
        Ls.t_dev = nullptr;
        if (c->has_src && c->batch && c->batch->capturing) {
            // recorded in a graph: the amplitude is read at replay time from
            // the device wavelet at the replay's own time index
            Ls.src_x = c->src[0];
            Ls.src_y = c->src[1];
            Ls.src_z = c->src[2];
            Ls.w_dev = c->w_dev();
            Ls.t_dev = c->t_dev();
            Ls.t_rel = tstep - c->t_capture;
            Ls.nw = (int64_t)c->w.size();
        } else if (c->has_src && tstep < (int64_t)c->w.size()) {
            Ls.src_x = c->src[0];
            Ls.src_y = c->src[1];
            Ls.src_z = c->src[2];
            Ls.w = c->w[tstep];
        }
        Ls.enc_out = nullptr;
        Ls.tile = d.step_tile;
        if (enc_fused && j == k_eff) {  // (the fused encode is built for the 64 x 16 tile)
            Ls.enc_out = c->out_slot(q, 0);
            Ls.enc_rate = d.rate_bits;
            Ls.enc_layer0 = z0 / 4;
            Ls.tile = 0;
        }
        const bool dec_here = dec_fused && j == 1;
        if (c->trace && dec_here) {  // the step that reads the staging slots
            if (s > 0)
                trace_push(c, OOCS_OP_STEP, sk, -1, (int64_t)g,
                           {acc(OOCS_RES_IN_SLOT, qp, w0 / 4, n0 / 4, false),
                            acc(OOCS_RES_IN_SLOT, q, n0 / 4, n1 / 4, false),
                            acc(OOCS_RES_WORK, wb, w0 / 4, w1 / 4, true)});
            else
                trace_push(c, OOCS_OP_STEP, sk, -1, (int64_t)g,
                           {acc(OOCS_RES_IN_SLOT, q, n0 / 4, n1 / 4, false),
                            acc(OOCS_RES_WORK, wb, w0 / 4, w1 / 4, true)});
        } else if (c->trace && Ls.enc_out) {  // the step that writes the out slot
            trace_push(c, OOCS_OP_STEP, sk, -1, (int64_t)g,
                       {acc(OOCS_RES_WORK, wb, w0 / 4, w1 / 4, true), acc(OOCS_RES_OUT_SLOT, q, z0 / 4, z1 / 4, true)});
        } else if (c->trace) {
            trace_push(c, OOCS_OP_STEP, sk, -1, (int64_t)g, {acc(OOCS_RES_WORK, wb, w0 / 4, w1 / 4, true)});
        } else if (dec_here) {
            const bool borrow = s > 0 && n0 > w0;
            const char *blk0 = borrow ? c->in_slot(qp, 0) + (w0 / 4 - pn0 / 4) * v.layer_bytes : nullptr;
            CU(c, launch_decode_heat_step(Ls, blk0, borrow ? (n0 - w0) / 4 : 0, c->in_slot(q, 0), (n1 - n0) / 4,
                                          d.rate_bits, st_k));
        } else {
            CU(c, launch_star_step(Ls, st_k));
        }
        if (dec_here)
            SCHED(sched_record(c, sk, kEvDecoded + q));
        c->stats.kernel_launches++;
        ++launches;
        step_units += (uint64_t)(hi - lo) * d.nx * d.ny;
        // the receiver plane lies in this slab's interior, which every step of
        // the visit computes: record u^(tstep+1) there
        if (c->rec && c->rec_z >= z0 && c->rec_z < z1 && tstep < c->rec_n && !c->trace)
            CU(c, cudaMemcpyAsync(c->rec + tstep * plane_f, Ls.out + (c->rec_z - w0) * plane_f,
                                  (size_t)plane_f * 4, cudaMemcpyDeviceToDevice, st_k));
        std::swap(cur, oth);
    }
    {
        oocs_status r = ks_steps.end(kClsStep, step_units, launches);
        if (r != OOCS_OK)
            return r;
    }
    // 7. interior [z0, z1) -> out slot(s): u^(t+k) and, for the wave, u^(t+k-1);
    //    the slot was copied back by visit g-3 (by role: on another stream)
    if (roles && g >= 3 && !enc_fused)
        SCHED(sched_wait(c, sk, kEvOut + q));
    if (c->trace) {
        if (!enc_fused)
            trace_push(c, OOCS_OP_STORE, sk, -1, (int64_t)g,
                       {acc(OOCS_RES_WORK, wb, z0 / 4, z1 / 4, false),
                        acc(OOCS_RES_OUT_SLOT, q, z0 / 4, z1 / 4, true)});
    } else if (enc_fused) {
        // encoded by the last step: counted as stored, with no launch of its own
        c->stats.store.units += (uint64_t)(z1 - z0) * plane_f;
    } else if (d.rate_bits > 0) {
        // one encode launch for both output fields
        CodecSegments sg;
        int64_t nl[kMaxCodecSegments];
        const int src_buf[2] = {cur, oth};
        for (int f = 0; f < v.fout; ++f) {
            sg.blocks[sg.nseg] = c->out_slot(q, f);
            sg.planes[sg.nseg] = c->wbuf(wb, src_buf[f]) + (z0 - w0) * plane_f;
            nl[sg.nseg++] = (z1 - z0) / 4;
        }
        KernelScope ks;
        oocs_status r = ks.begin(c, st_k, kClsStore);
        if (r != OOCS_OK)
            return r;
        CU(c, launch_encode_segments(sg, nl, d.nx, d.ny, d.rate_bits, d.codec, st_k));
        c->stats.kernel_launches++;
        r = ks.end(kClsStore, (uint64_t)v.fout * (z1 - z0) * plane_f);
        if (r != OOCS_OK)
            return r;
    } else {
        oocs_status r = store_layers(c, c->wbuf(wb, cur), w0, z0 / 4, z1 / 4, c->out_slot(q, 0), st_k);
        if (r != OOCS_OK)
            return r;
        if (v.fout == 2) {
            r = store_layers(c, c->wbuf(wb, oth), w0, z0 / 4, z1 / 4, c->out_slot(q, 1), st_k);
            if (r != OOCS_OK)
                return r;
        }
    }
    SCHED(sched_record(c, sk, kEvWrel + q));
    // 8. D2H into the host store, in place (after the encode, by role on
    //    the copy-back stream)
    if (roles)
        SCHED(sched_wait(c, sd, kEvWrel + q));
    if (c->trace) {
        trace_push(c, OOCS_OP_D2H, sd, -1, (int64_t)g,
                   {acc(OOCS_RES_OUT_SLOT, q, z0 / 4, z1 / 4, false),
                    acc(OOCS_RES_HOST, c->host_base, z0 / 4, z1 / 4, true)});
        if (v.fout == 2)
            c->trace->back().access[c->trace->back().naccess++] =
                acc(OOCS_RES_HOST, c->host_base + 1, z0 / 4, z1 / 4, true);
    }
    {
        KernelScope ks;
        if (!c->trace) {
            oocs_status r = ks.begin(c, st_d, kClsD2H);
            if (r != OOCS_OK)
                return r;
        }
        for (int f = 0; f < v.fout; ++f) {
            const uint64_t bytes = (uint64_t)(z1 - z0) / 4 * v.layer_bytes;
            if (!c->trace)
                CU(c, cudaMemcpyAsync(c->store[f] + (uint64_t)(z0 / 4) * v.layer_bytes, c->out_slot(q, f),
                                      bytes, cudaMemcpyDeviceToHost, st_d));
            c->stats.d2h_bytes += bytes;
        }
        if (!c->trace) {
            oocs_status r = ks.end(kClsD2H, (uint64_t)v.fout * (uint64_t)(z1 - z0) / 4 * v.layer_bytes);
            if (r != OOCS_OK)
                return r;
        }
    }
    // 8b. the same layers into the state record: out slot f holds u^(t+k-f);
    //     nothing in the pipeline reads the record, and the out slot is
    //     rewritten only by visit g+3 on this stream
    for (int f = 0; f < v.fout && !c->srec.empty(); ++f) {
        const int64_t i = t + k_eff - f - c->srec_t0;
        if (i < 0 || i >= (int64_t)c->srec.size() || !c->srec[i])
            continue;
        const uint64_t bytes = (uint64_t)(z1 - z0) / 4 * v.layer_bytes;
        if (!c->trace)
            CU(c, cudaMemcpyAsync(c->srec[i] + (uint64_t)(z0 / 4) * v.layer_bytes, c->out_slot(q, f), bytes,
                                  cudaMemcpyDeviceToHost, st_d));
        c->stats.d2h_bytes += bytes;
    }
    SCHED(sched_record(c, sd, kEvD2H + c->d2h_base + s));
    if (roles)
        SCHED(sched_record(c, sd, kEvOut + q));
    c->d2h_recorded[s] = 1;
    c->g++;
    c->stats.slabs_done++;
    return OOCS_OK;
}

// One slab visit of the wave adjoint at time index k (temporal depth 1, the
// time walk of Sec. 3.1 run backwards): copy the windows of lam^k and u^(k-1)
// and the interior of lam^(k+1) to the device, decode them into the working
// buffer, form m lam^k, add the gradient term lam^k (L u^(k-1) + w[k-1] e_src)
// to the device-resident dJ/dm, take the adjoint step on the interior, encode
// lam^(k-1) and copy it back over lam^(k+1)'s host layers.
oocs_status enqueue_adjoint_slab(oocs_ctx *c, int s, int64_t k, const char *fwd, bool chained)
{
    const Derived &v = c->v;
    const oocs_desc &d = c->d;
    const uint64_t g = c->g;
    const int q = (int)(g % 3);
    // streams by role, as in enqueue_slab: host->device copies on stream 0,
    // kernels on stream 1, device->host copies on stream 2
    const int sh = 0, sk = 1, sd = 2;
    cudaStream_t st_h = c->st[sh], st_k = c->st[sk], st_d = c->st[sd];
    const int64_t z0 = (int64_t)s * v.T;
    const int64_t z1 = std::min<int64_t>(z0 + v.T, d.nz);
    const int64_t w0 = std::max<int64_t>(z0 - v.h, 0);
    const int64_t w1 = std::min<int64_t>(z1 + v.h, d.nz);
    const int64_t plane_f = d.nx * d.ny;
    // slot q, field f: 0 = lam^k (window), 1 = lam^(k+1) (interior), 2 = u^(k-1) (window)
    const int store_of[3] = {OOCS_FIELD_LAM, OOCS_FIELD_LAM_PREV, OOCS_FIELD_FWD};
    const int64_t l0[3] = {w0 / 4, z0 / 4, w0 / 4}, l1[3] = {w1 / 4, z1 / 4, w1 / 4};
    float *W0 = c->wbuf(0, 0), *W1 = c->wbuf(0, 1), *W2 = c->wbuf(0, 2), *W3 = c->wbuf(0, 3);

    const int par = (int)(k & 1);  // this step's set of per-slab D2H events
    // 1. staging slot q is free once visit g-2 has decoded it
    if (g >= 2)
        SCHED(sched_wait(c, sh, kEvDecoded + (int)((g - 2) % 3)));
    // 2. the window of lam^k was written by the previous step (k+1) of this
    //    call over slabs s-1 .. s+1; waiting for those copies also orders this
    //    visit's later write of lam^(k-1) after the previous step's reads of
    //    the store it overwrites (each of those visits read before it wrote)
    if (chained)
        for (int ss = std::max(s - 1, 0); ss <= std::min(s + 1, v.S - 1); ++ss)
            if (c->d2h_recorded[(1 - par) * v.S + ss])
                SCHED(sched_wait(c, sh, kEvD2H + c->d2h_base + (1 - par) * v.S + ss));
    // 3. H2D of the windows of lam^k and u^(k-1) and the interior of lam^(k+1)
    if (c->trace) {
        trace_push(c, OOCS_OP_H2D, sh, -1, (int64_t)g,
                   {acc(OOCS_RES_IN_SLOT, q, w0 / 4, w1 / 4, true),
                    acc(OOCS_RES_HOST, c->host_base + c->store_id[OOCS_FIELD_LAM], l0[0], l1[0], false),
                    acc(OOCS_RES_HOST, c->host_base + c->store_id[OOCS_FIELD_LAM_PREV], l0[1], l1[1], false),
                    acc(OOCS_RES_HOST, c->host_base + 3, l0[2], l1[2], false)});
    } else {
        KernelScope ks;
        oocs_status r = ks.begin(c, st_h, kClsH2D);
        if (r != OOCS_OK)
            return r;
        const char *src[3] = {c->store[store_of[0]], c->store[store_of[1]], fwd};
        uint64_t bytes = 0;
        for (int f = 0; f < 3; ++f) {
            CU(c, cudaMemcpyAsync(c->in_slot(q, f), src[f] + (uint64_t)l0[f] * v.layer_bytes,
                                  (uint64_t)(l1[f] - l0[f]) * v.layer_bytes, cudaMemcpyHostToDevice, st_h));
            bytes += (uint64_t)(l1[f] - l0[f]) * v.layer_bytes;
        }
        r = ks.end(kClsH2D, bytes);
        if (r != OOCS_OK)
            return r;
    }
    for (int f = 0; f < 3; ++f)
        c->stats.h2d_bytes += (uint64_t)(l1[f] - l0[f]) * v.layer_bytes;
    SCHED(sched_record(c, sh, kEvH2D + q));
    // 4. the visit's layers have landed; the working buffer is free once
    //    visit g-1 has encoded from it (implied on the kernel stream)
    SCHED(sched_wait(c, sk, kEvH2D + q));
    if (g >= 1)
        SCHED(sched_wait(c, sk, kEvWrel + (int)((g - 1) % 3)));
    // 5. decode lam^k, lam^(k+1) (interior planes, at their window positions), u^(k-1)
    float *dst[3] = {W0, W1 + (z0 - w0) * plane_f, W2};
    if (c->trace) {
        trace_push(c, OOCS_OP_LOAD, sk, -1, (int64_t)g,
                   {acc(OOCS_RES_IN_SLOT, q, w0 / 4, w1 / 4, false), acc(OOCS_RES_WORK, 0, w0 / 4, w1 / 4, true)});
    } else {
        KernelScope ks;
        oocs_status r = ks.begin(c, st_k, kClsLoad);
        if (r != OOCS_OK)
            return r;
        if (d.rate_bits > 0) {
            CodecSegments sg;
            int64_t nl[kMaxCodecSegments];
            for (int f = 0; f < 3; ++f) {
                sg.blocks[sg.nseg] = c->in_slot(q, f);
                sg.planes[sg.nseg] = dst[f];
                nl[sg.nseg++] = l1[f] - l0[f];
            }
            CU(c, launch_decode_segments(sg, nl, d.nx, d.ny, d.rate_bits, d.codec, st_k));
            c->stats.kernel_launches++;
        } else {
            for (int f = 0; f < 3; ++f)
                CU(c, cudaMemcpyAsync(dst[f], c->in_slot(q, f), (uint64_t)(l1[f] - l0[f]) * v.layer_bytes,
                                      cudaMemcpyDeviceToDevice, st_k));
        }
        r = ks.end(kClsLoad, (uint64_t)(2 * (w1 - w0) + (z1 - z0)) * plane_f);
        if (r != OOCS_OK)
            return r;
    }
    SCHED(sched_record(c, sk, kEvDecoded + q));
    // 6. m lam^k over the window, the gradient term, the adjoint step
    StepLaunch G;
    memset(&G, 0, sizeof(G));
    G.radius = 4;
    G.tile = d.step_tile;
    G.nx = d.nx;
    G.ny = d.ny;
    G.nz = d.nz;
    G.gz0 = w0;
    G.wp = w1 - w0;
    G.z_lo = z0 - w0;
    G.z_hi = z1 - w0;
    for (int i = 0; i <= 4; ++i)
        G.coef[i] = d.coef[i];
    G.src_z = -1;
    StepLaunch A = G;
    G.scheme = kGradient;
    G.cur = W2;
    G.prev = c->grad() + w0 * plane_f;
    G.m = W0;
    G.out = c->grad() + w0 * plane_f;
    if (c->has_src && k - 1 >= 0 && k - 1 < (int64_t)c->w.size()) {
        G.src_x = c->src[0];
        G.src_y = c->src[1];
        G.src_z = c->src[2];
        G.w = c->w[k - 1];
    }
    A.scheme = kAdjoint;
    A.cur = W3;
    A.prev = W1;
    A.m = c->ro_m() + w0 * plane_f;
    A.c2 = W0;
    A.out = W1;
    A.out2 = nullptr;
    A.zr = -1;
    if (c->rec && k - 2 >= 0 && k - 2 < c->rec_n) {
        A.res = c->rec + (k - 2) * plane_f;
        A.zr = c->rec_z;
    }
    if (c->trace) {
        for (int i = 0; i < 3; ++i)
            trace_push(c, OOCS_OP_STEP, sk, -1, (int64_t)g, {acc(OOCS_RES_WORK, 0, w0 / 4, w1 / 4, true)});
    } else {
        KernelScope ks;
        oocs_status r = ks.begin(c, st_k, kClsStep);
        if (r != OOCS_OK)
            return r;
        CU(c, launch_product(W3, c->ro_m() + w0 * plane_f, W0, (w1 - w0) * plane_f, st_k));
        CU(c, launch_star_step(G, st_k));
        CU(c, launch_star_step(A, st_k));
        c->stats.kernel_launches += 3;
        r = ks.end(kClsStep, (uint64_t)(z1 - z0) * plane_f, 2);
        if (r != OOCS_OK)
            return r;
    }
    // 7. encode lam^(k-1) on the interior into the out slot (copied back by
    //    visit g-3 on the copy-back stream)
    if (g >= 3)
        SCHED(sched_wait(c, sk, kEvOut + q));
    if (c->trace) {
        trace_push(c, OOCS_OP_STORE, sk, -1, (int64_t)g,
                   {acc(OOCS_RES_WORK, 0, z0 / 4, z1 / 4, false), acc(OOCS_RES_OUT_SLOT, q, z0 / 4, z1 / 4, true)});
    } else {
        oocs_status r = store_layers(c, W1, w0, z0 / 4, z1 / 4, c->out_slot(q, 0), st_k);
        if (r != OOCS_OK)
            return r;
    }
    SCHED(sched_record(c, sk, kEvWrel + q));
    // 8. D2H over lam^(k+1)'s layers of the host store, after the encode
    SCHED(sched_wait(c, sd, kEvWrel + q));
    const uint64_t bytes = (uint64_t)(z1 - z0) / 4 * v.layer_bytes;
    if (c->trace)
        trace_push(c, OOCS_OP_D2H, sd, -1, (int64_t)g,
                   {acc(OOCS_RES_OUT_SLOT, q, z0 / 4, z1 / 4, false),
                    acc(OOCS_RES_HOST, c->host_base + c->store_id[OOCS_FIELD_LAM_PREV], z0 / 4, z1 / 4, true)});
    else {
        KernelScope ks;
        oocs_status r = ks.begin(c, st_d, kClsD2H);
        if (r != OOCS_OK)
            return r;
        CU(c, cudaMemcpyAsync(c->store[OOCS_FIELD_LAM_PREV] + (uint64_t)(z0 / 4) * v.layer_bytes, c->out_slot(q, 0),
                              bytes, cudaMemcpyDeviceToHost, st_d));
        r = ks.end(kClsD2H, bytes);
        if (r != OOCS_OK)
            return r;
    }
    c->stats.d2h_bytes += bytes;
    SCHED(sched_record(c, sd, kEvD2H + c->d2h_base + par * v.S + s));
    SCHED(sched_record(c, sd, kEvOut + q));
    c->d2h_recorded[par * v.S + s] = 1;
    c->g++;
    c->stats.slabs_done++;
    return OOCS_OK;
}

}  // namespace

// ============================================================== C ABI ======

oocs_status oocs::exception_status(oocs_ctx *ctx)
{
    try {
        fail(ctx, OOCS_ERR_HOST_ALLOC, "a host allocation inside the library failed");
    } catch (...) {
    }
    return OOCS_ERR_HOST_ALLOC;
}

// oocs_host_alloc's mappings and their sizes (for munmap)
static std::mutex g_host_mu;
static std::map<void *, uint64_t> g_host_maps;

// The transparent huge page size (the kernel's PMD size: 2 MiB with 4 KiB
// base pages, 512 MiB with 64 KiB), 2 MiB if it cannot be read.
static uint64_t huge_page_bytes()
{
    uint64_t hp = 2ull << 20;
    if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long v = 0;
        if (fscanf(f, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0 && v <= (1ull << 30))
            hp = v;
        fclose(f);
    }
    return hp;
}

extern "C" {

const char *oocs_version(void) { return kVersion; }

oocs_status oocs_query(const oocs_desc *desc, oocs_plan *plan)
try {
    std::string err;
    oocs_status s = plan_impl(desc, plan, err);
    if (s != OOCS_OK)
        g_last_error = err;
    return s;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_create(const oocs_desc *desc, void *workspace, uint64_t workspace_bytes,
                        void *const streams[3], oocs_ctx **out)
try {
    if (!out)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    oocs_plan p;
    std::string err;
    oocs_status s = plan_impl(desc, &p, err);
    if (s != OOCS_OK)
        return fail(nullptr, s, err);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
    if (workspace_bytes < p.workspace_bytes)
        return fail(nullptr, OOCS_ERR_BUDGET,
                    "workspace of " + std::to_string(workspace_bytes) + " bytes < plan's " +
                        std::to_string(p.workspace_bytes));
    if (!streams || !streams[0] || !streams[1] || !streams[2] || streams[0] == streams[1] ||
        streams[1] == streams[2] || streams[0] == streams[2])
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "three distinct non-null streams are required");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "workspace is not device memory");
    }
    oocs_ctx *c = new (std::nothrow) oocs_ctx();
    if (!c)
        return fail(nullptr, OOCS_ERR_HOST_ALLOC, "cannot allocate the context");
    c->d = *desc;
    if (c->d.temporal_depth == 0)
        c->d.temporal_depth = p.temporal_depth;
    c->p = p;
    c->v = derive(c->d, p.slab_planes);
    c->L = layout_for(c->d, c->v, c->d.working_buffers);
    c->ws = static_cast<char *>(workspace);
    for (int i = 0; i < 3; ++i)
        c->st[i] = static_cast<cudaStream_t>(streams[i]);
    memset(&c->stats, 0, sizeof(c->stats));
    c->stats.workspace_bytes = p.workspace_bytes;
    // the adjoint keeps the last D2H of each slab for two steps (step parity)
    const int nd2h = c->d.scheme == OOCS_WAVE_ADJOINT ? 2 * c->v.S : c->v.S;
    c->ev_d2h.assign(nd2h, nullptr);
    c->d2h_recorded.assign(nd2h, 0);
    auto mk = [&](cudaEvent_t *e) {
        return cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    };
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
        e = mk(&c->ev_decoded[i]);
        if (e == cudaSuccess) e = mk(&c->ev_h2d[i]);
        if (e == cudaSuccess) e = mk(&c->ev_wrel[i]);
        if (e == cudaSuccess) e = mk(&c->ev_join[i]);
        if (e == cudaSuccess) e = mk(&c->ev_out[i]);
    }
    for (int i = 0; i < nd2h && e == cudaSuccess; ++i)
        e = mk(&c->ev_d2h[i]);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = mk(&c->ev_codec[i]);
    if (e == cudaSuccess)
        e = cudaEventCreate(&c->ev_t0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&c->ev_t1);
    if (e == cudaSuccess && c->d.scheme == OOCS_WAVE_ADJOINT)  // dJ/dm starts at zero
        e = cudaMemsetAsync(c->grad(), 0, (size_t)c->d.nz * c->d.nx * c->d.ny * 4, c->st[0]);
    if (e != cudaSuccess) {
        std::string msg = std::string("cudaEventCreate: ") + cudaGetErrorString(e);
        oocs_destroy(c);
        return fail(nullptr, OOCS_ERR_CUDA, msg);
    }
    *out = c;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_bind_field(oocs_ctx *ctx, int32_t field, void *host_store, uint64_t bytes)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    const int nf = bound_fields(ctx->d);
    if (field < 0 || field >= nf)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "field id not used by this scheme");
    if (!host_store || bytes < ctx->p.host_store_bytes)
        return fail(ctx, OOCS_ERR_INVALID_ARG,
                    "host store needs " + std::to_string(ctx->p.host_store_bytes) + " bytes");
    ctx->store[field] = static_cast<char *>(host_store);
    ctx->store_bytes[field] = bytes;
    if (field == OOCS_FIELD_M)
        ctx->ro_dirty = true;
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_set_source(oocs_ctx *ctx, int64_t x, int64_t y, int64_t z, const float *w, int32_t nw)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    if (ctx->d.scheme == OOCS_HEAT)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "a point source needs the wave scheme");
    if (x < 0 || y < 0 || z < 0 || x >= ctx->d.nx || y >= ctx->d.ny || z >= ctx->d.nz || nw < 0 ||
        (nw > 0 && !w))
        return fail(ctx, OOCS_ERR_INVALID_ARG, "source voxel outside the grid or bad wavelet");
    ctx->has_src = nw > 0;
    ctx->src[0] = x;
    ctx->src[1] = y;
    ctx->src[2] = z;
    ctx->w.assign(w, w + nw);
    // the device copy read by replayed graphs (at most kMaxDeviceWavelet samples)
    const int64_t nd = std::min<int64_t>(nw, kMaxDeviceWavelet);
    if (nd > 0 && !ctx->trace && ctx->L.src_off)
        CU(ctx, cudaMemcpyAsync(ctx->w_dev(), ctx->w.data(), (size_t)nd * 4, cudaMemcpyHostToDevice, ctx->st[0]));
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_set_receiver(oocs_ctx *ctx, int64_t zr, float *planes, int64_t nplanes)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    if (ctx->d.scheme == OOCS_HEAT)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "receiver planes belong to the wave scheme and its adjoint");
    if (nplanes < 0 || (nplanes > 0 && (!planes || zr < 0 || zr >= ctx->d.nz)))
        return fail(ctx, OOCS_ERR_INVALID_ARG, "receiver plane outside the grid or no device array");
    ctx->rec = nplanes > 0 ? planes : nullptr;
    ctx->rec_z = zr;
    ctx->rec_n = nplanes;
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_selftest_stuck_wait(oocs_ctx *ctx)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    s = join_streams(ctx);
    if (s != OOCS_OK)
        return s;
    CU(ctx, launch_stuck_wait(ctx->st[0]));
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_set_state_record(oocs_ctx *ctx, void *const *stores, int64_t t0, int64_t n)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    if (n < 0 || (n > 0 && !stores))
        return fail(ctx, OOCS_ERR_INVALID_ARG, "n must be >= 0 and stores non-null when n > 0");
    // the copies already enqueued read the old list's pointers by value
    ctx->srec.assign(n > 0 ? reinterpret_cast<char *const *>(stores) : nullptr,
                     n > 0 ? reinterpret_cast<char *const *>(stores) + n : nullptr);
    ctx->srec_t0 = t0;
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

static oocs_status codec_field(oocs_ctx *ctx, int32_t field, const float *src, float *dst, bool enc)
{
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    const int nf = bound_fields(ctx->d);
    if (field < 0 || field >= nf || !ctx->store[field])
        return fail(ctx, OOCS_ERR_STATE, "field is not bound");
    if (enc ? !src : !dst)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "raw host array is NULL");
    const oocs_desc &d = ctx->d;
    const uint64_t plane_bytes = (uint64_t)d.nx * d.ny * 4;
    // the store may share memory with the raw array only in place: starting at
    // its first byte (the compressed layers of planes [z0, z1) then lie at or
    // below the raw planes [z0, z1), see the chunk order below)
    {
        const uintptr_t r0 = reinterpret_cast<uintptr_t>(enc ? (const void *)src : (const void *)dst);
        const uintptr_t r1 = r0 + (uintptr_t)d.nz * plane_bytes;
        const uintptr_t s0 = reinterpret_cast<uintptr_t>(ctx->store[field]);
        const uintptr_t s1 = s0 + (uintptr_t)ctx->p.host_store_bytes;
        if (s0 < r1 && r0 < s1 && s0 != r0)
            return fail(ctx, OOCS_ERR_INVALID_ARG,
                        "the store overlaps the raw array without starting at its address (only in place is allowed)");
    }
    if (enc && field == OOCS_FIELD_M)
        ctx->ro_dirty = true;
    // a resident M is decoded from each chunk's blocks while they are on the
    // device (the values the store decodes to), so no step has to upload it
    const bool ro_keep = enc && field == OOCS_FIELD_M && ctx->v.ro_res && d.rate_bits > 0;
    s = join_streams(ctx);
    if (s != OOCS_OK)
        return s;
    if (d.rate_bits == 0) {
        const uint64_t bytes = (uint64_t)d.nz * plane_bytes;
        if (enc)
            CU(ctx, cudaMemcpyAsync(ctx->store[field], src, bytes, cudaMemcpyHostToHost, ctx->st[0]));
        else
            CU(ctx, cudaMemcpyAsync(dst, ctx->store[field], bytes, cudaMemcpyHostToHost, ctx->st[0]));
        return join_streams(ctx);
    }
    // chunks of T planes through working buffer 0's first two buffers and
    // out slots 0 / 1 of field 0, alternating between streams 0 and 1.
    // Compression walks the chunks upwards in z, decompression downwards, and
    // a chunk's device->host copy waits until the previous chunk (on the other
    // stream) has read its host bytes: then a store that lives in place in the
    // raw array (compressed layers of planes [z0, z1) at or below the raw
    // planes [z0, z1)) is never overwritten before it is read, and never
    // overwrites raw planes still to be read.
    const int64_t T = ctx->v.T;
    const int64_t nchunks = ceil_div(d.nz, T);
    for (int64_t chunk = 0; chunk < nchunks; ++chunk) {
        const int64_t z0 = (enc ? chunk : nchunks - 1 - chunk) * T;
        const int64_t z1 = std::min<int64_t>(z0 + T, d.nz);
        const int i = (int)(chunk & 1);
        cudaStream_t st = ctx->st[i];
        float *raw = ctx->wbuf(0, i);
        char *blk = ctx->out_slot(i, 0);
        const uint64_t cbytes = (uint64_t)(z1 - z0) / 4 * ctx->v.layer_bytes;
        char *host_blk = ctx->store[field] + (uint64_t)(z0 / 4) * ctx->v.layer_bytes;
        if (enc) {
            CU(ctx, cudaMemcpyAsync(raw, src + z0 * d.nx * d.ny, (z1 - z0) * plane_bytes,
                                    cudaMemcpyHostToDevice, st));
            CU(ctx, cudaEventRecord(ctx->ev_codec[i], st));
            CU(ctx, launch_encode_layers(raw, d.nx, d.ny, (z1 - z0) / 4, d.rate_bits, d.codec, blk, st));
            if (chunk > 0)
                CU(ctx, cudaStreamWaitEvent(st, ctx->ev_codec[i ^ 1], 0));
            CU(ctx, cudaMemcpyAsync(host_blk, blk, cbytes, cudaMemcpyDeviceToHost, st));
            if (ro_keep)
                CU(ctx, launch_decode_layers(blk, d.nx, d.ny, (z1 - z0) / 4, d.rate_bits, d.codec,
                                             ctx->ro_m() + z0 * d.nx * d.ny, st));
        } else {
            CU(ctx, cudaMemcpyAsync(blk, host_blk, cbytes, cudaMemcpyHostToDevice, st));
            CU(ctx, cudaEventRecord(ctx->ev_codec[i], st));
            CU(ctx, launch_decode_layers(blk, d.nx, d.ny, (z1 - z0) / 4, d.rate_bits, d.codec, raw, st));
            if (chunk > 0)
                CU(ctx, cudaStreamWaitEvent(st, ctx->ev_codec[i ^ 1], 0));
            CU(ctx, cudaMemcpyAsync(dst + z0 * d.nx * d.ny, raw, (z1 - z0) * plane_bytes,
                                    cudaMemcpyDeviceToHost, st));
        }
    }
    s = join_streams(ctx);
    if (s == OOCS_OK && ro_keep)
        ctx->ro_dirty = false;
    return s;
}

oocs_status oocs_compress(oocs_ctx *ctx, int32_t field, const float *src)
try {
    return codec_field(ctx, field, src, nullptr, true);
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_decompress(oocs_ctx *ctx, int32_t field, float *dst)
try {
    return codec_field(ctx, field, nullptr, dst, false);
} catch (...) {
    return exception_status(ctx);
}

// Planes [z0, z0 + nplanes) of `field` between a device array holding them
// and the host store, in chunks of T planes through working buffer 0 and the
// first out (encode) or in (decode) slot of field 0, on stream 0.
static oocs_status codec_range_device(oocs_ctx *ctx, int32_t field, const float *src, float *dst, int64_t z0,
                                      int64_t nplanes, bool enc)
{
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    const oocs_desc &d = ctx->d;
    if ((enc ? !src : !dst) || (reinterpret_cast<uintptr_t>(enc ? (const void *)src : (const void *)dst) & 15))
        return fail(ctx, OOCS_ERR_INVALID_ARG, "device array must be non-null and 16-byte aligned");
    if (z0 < 0 || nplanes < 0 || z0 % 4 || nplanes % 4 || z0 + nplanes > d.nz)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "planes must be whole 4-plane layers inside the grid");
    if (d.scheme == OOCS_WAVE_ADJOINT && field == OOCS_FIELD_GRAD) {  // lives on the device
        s = join_streams(ctx);
        if (s != OOCS_OK)
            return s;
        float *g = ctx->grad() + z0 * d.nx * d.ny;
        CU(ctx, cudaMemcpyAsync(enc ? g : dst, enc ? src : g, (size_t)nplanes * d.nx * d.ny * 4,
                                cudaMemcpyDeviceToDevice, ctx->st[0]));
        return join_streams(ctx);
    }
    const int nf = bound_fields(ctx->d);
    if (field < 0 || field >= nf || !ctx->store[field])
        return fail(ctx, OOCS_ERR_STATE, "field is not bound");
    // a resident M takes the written planes' decoded values as they are
    // coded (a copy at rate 0); if it was not made yet, the next step makes it
    const bool ro_keep = enc && field == OOCS_FIELD_M && ctx->v.ro_res;
    if (enc && field == OOCS_FIELD_M && !ro_keep)
        ctx->ro_dirty = true;
    s = join_streams(ctx);
    if (s != OOCS_OK)
        return s;
    cudaStream_t st = ctx->st[0];
    const int64_t plane = d.nx * d.ny;
    const int64_t T = ctx->v.T;  // the slots hold at least T/4 layers
    for (int64_t c0 = 0; c0 < nplanes; c0 += T) {
        const int64_t n = std::min<int64_t>(T, nplanes - c0);
        char *host = ctx->store[field] + (uint64_t)((z0 + c0) / 4) * ctx->v.layer_bytes;
        const uint64_t cbytes = (uint64_t)n / 4 * ctx->v.layer_bytes;
        if (d.rate_bits == 0) {
            if (enc)
                CU(ctx, cudaMemcpyAsync(host, src + c0 * plane, cbytes, cudaMemcpyDeviceToHost, st));
            else
                CU(ctx, cudaMemcpyAsync(dst + c0 * plane, host, cbytes, cudaMemcpyHostToDevice, st));
            if (ro_keep)
                CU(ctx, cudaMemcpyAsync(ctx->ro_m() + (z0 + c0) * plane, src + c0 * plane, cbytes,
                                        cudaMemcpyDeviceToDevice, st));
        } else if (enc) {
            char *blk = ctx->out_slot(0, 0);
            CU(ctx, launch_encode_layers(src + c0 * plane, d.nx, d.ny, n / 4, d.rate_bits, d.codec, blk, st));
            CU(ctx, cudaMemcpyAsync(host, blk, cbytes, cudaMemcpyDeviceToHost, st));
            if (ro_keep)
                CU(ctx, launch_decode_layers(blk, d.nx, d.ny, n / 4, d.rate_bits, d.codec,
                                             ctx->ro_m() + (z0 + c0) * plane, st));
        } else {
            char *blk = ctx->in_slot(0, 0);
            CU(ctx, cudaMemcpyAsync(blk, host, cbytes, cudaMemcpyHostToDevice, st));
            CU(ctx, launch_decode_layers(blk, d.nx, d.ny, n / 4, d.rate_bits, d.codec, dst + c0 * plane, st));
        }
    }
    s = join_streams(ctx);
    if (s == OOCS_OK && ro_keep && z0 == 0 && nplanes == d.nz)  // the whole device copy was written
        ctx->ro_dirty = false;
    return s;
}

oocs_status oocs_compress_device(oocs_ctx *ctx, int32_t field, const float *src, int64_t z0, int64_t nplanes)
try {
    return codec_range_device(ctx, field, src, nullptr, z0, nplanes, true);
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_decompress_device(oocs_ctx *ctx, int32_t field, float *dst, int64_t z0, int64_t nplanes)
try {
    return codec_range_device(ctx, field, nullptr, dst, z0, nplanes, false);
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_host_alloc(uint64_t bytes, void **ptr)
try {
    if (!ptr || bytes == 0)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "bytes > 0 and an output pointer are required");
    *ptr = nullptr;
    // Anonymous pages with transparent-huge-page advice, touched by several
    // threads (parallel page faults: the kernel zeroes the pages) and then
    // page-locked by cudaHostRegister.  The mapping starts on a huge-page
    // boundary and covers whole huge pages, so every page of the buffer can
    // be a huge page.  Measured on GB300 hosts: memory from cudaHostAlloc, or
    // anonymous memory in base pages, lost host->device copy speed in its
    // first gigabytes after a minute of traffic (1.6 GB copies from 7.6 ms to
    // 60-360 ms; 20-step calls of the 2560^2 x 5120 heat run from 2.3 to
    // 8.9 s), while huge-page memory kept its speed (eight calls of 2.249 s).
    const uint64_t hp = huge_page_bytes();
    const uint64_t maplen = (bytes + hp - 1) / hp * hp;
    void *raw = mmap(nullptr, maplen + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw == MAP_FAILED)
        return fail(nullptr, OOCS_ERR_HOST_ALLOC, "mmap of " + std::to_string(bytes) + " bytes failed");
    const uintptr_t r0 = reinterpret_cast<uintptr_t>(raw);
    const uintptr_t a0 = (r0 + hp - 1) / hp * hp;
    if (a0 > r0)
        munmap(raw, a0 - r0);
    if (r0 + maplen + hp > a0 + maplen)
        munmap(reinterpret_cast<void *>(a0 + maplen), r0 + maplen + hp - (a0 + maplen));
    void *p = reinterpret_cast<void *>(a0);
    madvise(p, maplen, MADV_HUGEPAGE);  // advice only: ignored where unsupported
    {
        const long pg = std::max<long>(sysconf(_SC_PAGESIZE), 4096);
        const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        const uint64_t per = (bytes + nt - 1) / nt;
        auto touch = [p, pg](uint64_t a, uint64_t b) {
            volatile char *c = static_cast<volatile char *>(p);
            for (uint64_t o = a; o < b; o += (uint64_t)pg)
                c[o] = 0;
        };
        std::vector<std::thread> th;
        uint64_t done = 0;  // [0, done) is handed to threads; the rest is touched here
        try {
            for (unsigned i = 0; i < nt; ++i) {
                const uint64_t a = std::min<uint64_t>(bytes, (uint64_t)i * per);
                const uint64_t b = std::min<uint64_t>(bytes, a + per);
                th.emplace_back(touch, a, b);
                done = b;
            }
        } catch (...) {  // no thread could be started: touch the rest on this one
        }
        touch(done, bytes);
        for (auto &t : th)
            t.join();
    }
    cudaError_t e = cudaHostRegister(p, bytes, cudaHostRegisterPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        munmap(p, maplen);
        return fail(nullptr, OOCS_ERR_HOST_ALLOC,
                    "cudaHostRegister of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        g_host_maps[p] = maplen;
    }
    *ptr = p;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_host_free(void *ptr)
try {
    if (!ptr)
        return OOCS_OK;
    uint64_t bytes = 0;
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        auto it = g_host_maps.find(ptr);
        if (it == g_host_maps.end())
            return fail(nullptr, OOCS_ERR_INVALID_ARG, "not a pointer from oocs_host_alloc");
        bytes = it->second;
        g_host_maps.erase(it);
    }
    if (cudaHostUnregister(ptr) != cudaSuccess)
        cudaGetLastError();
    munmap(ptr, bytes);
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_set_time(oocs_ctx *ctx, int64_t t)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    if (t < 0)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "time index must be >= 0");
    ctx->stats.steps_done = (uint64_t)t;
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_step(oocs_ctx *ctx, int32_t nsteps)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    if (nsteps < 0)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "nsteps must be >= 0");
    const int nf = bound_fields(ctx->d);
    for (int f = 0; f < nf; ++f)
        if (!ctx->store[f])
            return fail(ctx, OOCS_ERR_STATE, "all fields of the scheme must be bound before oocs_step");
    if (nsteps == 0)
        return OOCS_OK;
    if (ctx->batch) {  // one problem of a batch through the batch's pipeline
        if (ctx->batch->capturing)
            return fail(ctx, OOCS_ERR_STATE, "the batch is capturing a graph");
        ctx->g = ctx->batch->g;
    }
    s = join_streams(ctx);
    if (s != OOCS_OK)
        return s;
    s = sched_record(ctx, 0, kEvT0);
    if (s != OOCS_OK)
        return s;
    if (ctx->v.ro_res && ctx->ro_dirty && !ctx->trace) {
        s = upload_resident(ctx);
        if (s != OOCS_OK)
            return s;
    }
    s = join_streams(ctx);
    if (s != OOCS_OK)
        return s;
    int64_t t = (int64_t)ctx->stats.steps_done;
    if (ctx->d.scheme == OOCS_WAVE_ADJOINT) {
        // nsteps adjoint steps from time index t down, each a sweep over the
        // slabs in reverse z order; after each, the stores of lam^k and the
        // new lam^(k-1) trade roles.  Steps of one call are chained by the
        // per-slab D2H events of the previous step (parity sets), not joined.
        if (t < nsteps)
            return fail(ctx, OOCS_ERR_STATE, "the adjoint's time index must be >= nsteps (oocs_set_time)");
        std::vector<const char *> fwd(nsteps, ctx->store[OOCS_FIELD_FWD]);
        if (!ctx->srec.empty()) {
            for (int j = 0; j < nsteps; ++j) {
                const int64_t i = t - j - 1 - ctx->srec_t0;
                if (i < 0 || i >= (int64_t)ctx->srec.size() || !ctx->srec[i])
                    return fail(ctx, OOCS_ERR_STATE,
                                "the state record holds no forward state u^" + std::to_string(t - j - 1));
                fwd[j] = ctx->srec[i];
            }
        } else if (nsteps > 1 && !ctx->trace) {
            return fail(ctx, OOCS_ERR_INVALID_ARG,
                        "more than one adjoint step per call reads the forward states from a state record");
        }
        std::fill(ctx->d2h_recorded.begin(), ctx->d2h_recorded.end(), 0);  // the opening join orders the rest
        for (int j = 0; j < nsteps; ++j) {
            const int64_t k = t - j;
            for (int sl = ctx->v.S - 1; sl >= 0; --sl) {
                s = enqueue_adjoint_slab(ctx, sl, k, fwd[j], j > 0);
                if (s != OOCS_OK)
                    return s;
            }
            std::swap(ctx->store[OOCS_FIELD_LAM], ctx->store[OOCS_FIELD_LAM_PREV]);
            std::swap(ctx->store_bytes[OOCS_FIELD_LAM], ctx->store_bytes[OOCS_FIELD_LAM_PREV]);
            std::swap(ctx->store_id[OOCS_FIELD_LAM], ctx->store_id[OOCS_FIELD_LAM_PREV]);
            ctx->stats.passes_done++;
        }
        ctx->stats.steps_done = (uint64_t)(t - nsteps);
        s = join_streams(ctx);
        if (s != OOCS_OK)
            return s;
        s = sched_record(ctx, 0, kEvT1);
        if (s != OOCS_OK)
            return s;
        ctx->timing_pending = !ctx->trace;
        return OOCS_OK;
    }
    int left = nsteps;
    while (left > 0) {
        const int k_eff = std::min(left, ctx->v.k);
        for (int sl = 0; sl < ctx->v.S; ++sl) {
            s = enqueue_slab(ctx, sl, k_eff, t);
            if (s != OOCS_OK)
                return s;
        }
        t += k_eff;
        left -= k_eff;
        ctx->stats.passes_done++;
    }
    ctx->stats.steps_done = (uint64_t)t;
    s = join_streams(ctx);
    if (s != OOCS_OK)
        return s;
    s = sched_record(ctx, 0, kEvT1);
    if (s != OOCS_OK)
        return s;
    if (ctx->batch)
        ctx->batch->g = ctx->g;
    ctx->timing_pending = !ctx->trace;
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_synchronize(oocs_ctx *ctx, uint64_t timeout_ns)
try {
    if (!ctx)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "ctx is NULL");
    if (ctx->sticky != OOCS_OK)
        return ctx->sticky;
    // mark the end of everything enqueued so far on each stream, then poll
    for (int i = 0; i < 3; ++i)
        CU(ctx, cudaEventRecord(ctx->ev_join[i], ctx->st[i]));
    const auto t_start = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < 3 && e == cudaSuccess; ++i)
            e = cudaEventQuery(ctx->ev_join[i]);
        if (e == cudaSuccess)
            break;
        if (e != cudaErrorNotReady)
            return fail(ctx, OOCS_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
        if (timeout_ns) {
            const auto el = std::chrono::duration_cast<std::chrono::nanoseconds>(
                                std::chrono::steady_clock::now() - t_start)
                                .count();
            if ((uint64_t)el > timeout_ns)
                return fail(ctx, OOCS_ERR_TIMEOUT, "oocs_synchronize: timed out");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (int i = 0; i < 3; ++i) {
        cudaError_t e = cudaStreamQuery(ctx->st[i]);
        if (e != cudaSuccess && e != cudaErrorNotReady)
            return fail(ctx, OOCS_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(e));
    }
    unsigned int code = 0;
    CU(ctx, read_device_error(&code, true));
    if (code & OOCS_DEVERR_WAIT_TIMEOUT)
        return fail(ctx, OOCS_ERR_CUDA, "a kernel's bounded wait ran out (device error " +
                                            std::to_string(code) + ")");
    if (code & OOCS_DEVERR_NONFINITE)
        return fail(ctx, OOCS_ERR_NONFINITE,
                    "the codec met an infinity or a NaN: the blocks holding one were stored as zeros");
    if (code)
        return fail(ctx, OOCS_ERR_CUDA, "device error " + std::to_string(code));
    if (ctx->timing_pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->ev_t0, ctx->ev_t1) == cudaSuccess)
            ctx->stats.last_step_ms = ms;
        ctx->timing_pending = false;
    }
    collect_profile(ctx);
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_get_timeline(const oocs_ctx *ctx, oocs_timeline_entry *entries, int64_t capacity,
                              int64_t *count)
try {
    if (!ctx || !count || capacity < 0 || (capacity > 0 && !entries))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "ctx and count are required, entries when capacity > 0");
    const int64_t n = (int64_t)ctx->timeline.size();
    for (int64_t i = 0; i < std::min(n, capacity); ++i)
        entries[i] = ctx->timeline[i];
    *count = n;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_set_fault_injection(oocs_ctx *ctx, int64_t nth_call)
try {
    if (!ctx || nth_call < 0)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "ctx is NULL or nth_call < 0");
    ctx->inject_at = nth_call;
    ctx->inject_seen = 0;
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_device_errors(uint32_t *flags, int32_t clear)
try {
    if (!flags)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "flags is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    unsigned int code = 0;
    if (e == cudaSuccess)
        e = read_device_error(&code, clear != 0);
    if (e != cudaSuccess)
        return fail(nullptr, OOCS_ERR_CUDA, std::string("oocs_device_errors: ") + cudaGetErrorString(e));
    *flags = code;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_get_stats(const oocs_ctx *ctx, oocs_stats *out)
try {
    if (!ctx || !out)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "ctx or out is NULL");
    *out = ctx->stats;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_set_profiling(oocs_ctx *ctx, int32_t classes)
try {
    oocs_status s = check_ready(ctx);
    if (s != OOCS_OK)
        return s;
    if (classes < 0 || classes > 31)
        return fail(ctx, OOCS_ERR_INVALID_ARG, "profiling mask must be in [0, 31]");
    ctx->prof = classes;
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

oocs_status oocs_trace_schedule(const oocs_desc *desc, const int32_t *nsteps, int32_t ncalls,
                                oocs_trace_op *ops, int64_t capacity, int64_t *count)
try {
    if (!count || (ncalls > 0 && !nsteps) || ncalls < 0 || capacity < 0 || (capacity > 0 && !ops))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "bad trace arguments");
    *count = 0;
    oocs_plan p;
    std::string err;
    oocs_status s = plan_impl(desc, &p, err);
    if (s != OOCS_OK)
        return fail(nullptr, s, err);
    oocs_ctx *c = new (std::nothrow) oocs_ctx();
    if (!c)
        return fail(nullptr, OOCS_ERR_HOST_ALLOC, "cannot allocate the context");
    std::vector<oocs_trace_op> trace;
    c->trace = &trace;
    c->d = *desc;
    if (c->d.temporal_depth == 0)
        c->d.temporal_depth = p.temporal_depth;
    c->p = p;
    c->v = derive(c->d, p.slab_planes);
    c->L = layout_for(c->d, c->v, c->d.working_buffers);
    memset(&c->stats, 0, sizeof(c->stats));
    c->ev_d2h.assign(c->d.scheme == OOCS_WAVE_ADJOINT ? 2 * c->v.S : c->v.S, nullptr);
    c->d2h_recorded.assign(c->ev_d2h.size(), 0);
    static char dummy;
    for (int f = 0; f < 4; ++f)
        c->store[f] = &dummy;  // never dereferenced in trace mode
    if (c->d.scheme == OOCS_WAVE_ADJOINT) {  // adjoint steps count down from here
        int64_t total = 0;
        for (int i = 0; i < ncalls; ++i)
            total += nsteps[i];
        c->stats.steps_done = (uint64_t)total;
    }
    for (int i = 0; i < ncalls && s == OOCS_OK; ++i)
        s = oocs_step(c, nsteps[i]);
    if (s != OOCS_OK) {
        std::string msg = c->err;
        delete c;
        return fail(nullptr, s, msg);
    }
    *count = (int64_t)trace.size();
    delete c;
    if ((int64_t)trace.size() > capacity)
        return fail(nullptr, OOCS_ERR_INVALID_ARG,
                    "trace needs " + std::to_string(trace.size()) + " entries");
    for (size_t i = 0; i < trace.size(); ++i)
        ops[i] = trace[i];
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

const char *oocs_last_error(const oocs_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

static void destroy_ctx(oocs_ctx *ctx)
{
    for (int i = 0; i < 3; ++i)
        if (ctx->st[i] && !ctx->trace)
            cudaStreamSynchronize(ctx->st[i]);
    auto kill = [](cudaEvent_t &e) {
        if (e)
            cudaEventDestroy(e);
        e = nullptr;
    };
    if (!ctx->batch)  // a batch owns the shared pipeline events
        for (int i = 0; i < 3; ++i) {
            kill(ctx->ev_decoded[i]);
            kill(ctx->ev_h2d[i]);
            kill(ctx->ev_wrel[i]);
            kill(ctx->ev_join[i]);
            kill(ctx->ev_out[i]);
        }
    for (auto &e : ctx->ev_d2h)
        kill(e);
    kill(ctx->ev_codec[0]);
    kill(ctx->ev_codec[1]);
    for (auto &e : ctx->ev_pool)
        kill(e);
    kill(ctx->ev_t0);
    kill(ctx->ev_t1);
    delete ctx;
}

oocs_status oocs_destroy(oocs_ctx *ctx)
try {
    if (!ctx)
        return OOCS_OK;
    if (ctx->batch)
        return fail(ctx, OOCS_ERR_STATE, "this context belongs to a batch (oocs_batch_destroy)");
    destroy_ctx(ctx);
    return OOCS_OK;
} catch (...) {
    return exception_status(ctx);
}

// ------------------------------------------------------- device-level API --

oocs_status oocs_incore_run(const oocs_desc *desc, float *u, float *u_prev, const float *m,
                            float *scratch, int32_t nsteps, int64_t t0, const int64_t *src_xyz,
                            const float *w, int32_t nw, void *stream)
try {
    std::string err;
    oocs_status s = validate_desc(desc, err);
    if (s != OOCS_OK)
        return fail(nullptr, s, err);
    const bool wave = desc->scheme == OOCS_WAVE;
    if (!u || !scratch || (wave && (!u_prev || !m)) || nsteps < 0 || (nw > 0 && !w))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "missing device array or bad nsteps/wavelet");
    if (src_xyz && (src_xyz[0] < 0 || src_xyz[1] < 0 || src_xyz[2] < 0 || src_xyz[0] >= desc->nx ||
                    src_xyz[1] >= desc->ny || src_xyz[2] >= desc->nz))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "source voxel outside the grid");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t bytes = (uint64_t)desc->nx * desc->ny * desc->nz * 4;
    StepLaunch Ls;
    memset(&Ls, 0, sizeof(Ls));
    Ls.scheme = wave ? kWave : kHeat;
    Ls.radius = desc->radius;
    Ls.tile = desc->step_tile;
    Ls.nx = desc->nx;
    Ls.ny = desc->ny;
    Ls.nz = desc->nz;
    Ls.gz0 = 0;
    Ls.wp = desc->nz;
    Ls.z_lo = 0;
    Ls.z_hi = desc->nz;
    for (int i = 0; i <= desc->radius; ++i)
        Ls.coef[i] = desc->coef[i];
    float *bufs[3] = {u, wave ? u_prev : scratch, scratch};
    int cur = 0, oth = 1;
    for (int j = 0; j < nsteps; ++j) {
        Ls.cur = bufs[cur];
        Ls.prev = bufs[oth];
        Ls.out = bufs[oth];
        Ls.m = m;
        Ls.src_z = -1;
        Ls.w = 0.0f;
        const int64_t tstep = t0 + j;
        if (wave && src_xyz && tstep >= 0 && tstep < nw) {
            Ls.src_x = src_xyz[0];
            Ls.src_y = src_xyz[1];
            Ls.src_z = src_xyz[2];
            Ls.w = w[tstep];
        }
        cudaError_t e = launch_star_step(Ls, st);
        if (e != cudaSuccess)
            return fail(nullptr, OOCS_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
        std::swap(cur, oth);
    }
    // bring the result back into the caller's (u, u_prev)
    cudaError_t e = cudaSuccess;
    if (cur == 1) {
        if (!wave) {
            e = cudaMemcpyAsync(u, scratch, bytes, cudaMemcpyDeviceToDevice, st);
        } else {
            // cur = u_prev buffer, prev = u buffer: swap via scratch
            e = cudaMemcpyAsync(scratch, u_prev, bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(u_prev, u, bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(u, scratch, bytes, cudaMemcpyDeviceToDevice, st);
        }
    }
    if (e != cudaSuccess)
        return fail(nullptr, OOCS_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

static oocs_status codec_args(int64_t nx, int64_t ny, int64_t nz, int32_t rate, int32_t codec, const void *a,
                              const void *b)
{
    if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "dims must be positive multiples of 4");
    if (codec != OOCS_CODEC_TRANSFORM && codec != OOCS_CODEC_QUANT)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "codec must be OOCS_CODEC_TRANSFORM or OOCS_CODEC_QUANT");
    if (rate < (codec == OOCS_CODEC_QUANT ? 2 : 1) || rate > 32)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "rate must be in [1, 32] (transform) or [2, 32] (quantiser)");
    if (!a || !b || (reinterpret_cast<uintptr_t>(a) & 15) || (reinterpret_cast<uintptr_t>(b) & 15))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "pointers must be non-null and 16-byte aligned");
    return OOCS_OK;
}

oocs_status oocs_encode_device(const float *field, int64_t nx, int64_t ny, int64_t nz, int32_t rate,
                               int32_t codec, void *blocks, void *stream)
try {
    oocs_status s = codec_args(nx, ny, nz, rate, codec, field, blocks);
    if (s != OOCS_OK)
        return s;
    cudaError_t e = launch_encode_layers(field, nx, ny, nz / 4, rate, codec, blocks,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return fail(nullptr, OOCS_ERR_CUDA, std::string("encode: ") + cudaGetErrorString(e));
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_decode_device(const void *blocks, int64_t nx, int64_t ny, int64_t nz, int32_t rate,
                               int32_t codec, float *field, void *stream)
try {
    oocs_status s = codec_args(nx, ny, nz, rate, codec, blocks, field);
    if (s != OOCS_OK)
        return s;
    cudaError_t e = launch_decode_layers(blocks, nx, ny, nz / 4, rate, codec, field,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return fail(nullptr, OOCS_ERR_CUDA, std::string("decode: ") + cudaGetErrorString(e));
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

}  // extern "C"

// ============================================================ batches ======

namespace {

// Shared layout of a batch: every region sized for the largest problem (so
// all problems' visits use the same working buffer and staging slots), then
// one resident FP32 model per problem that keeps it on the device.
Layout batch_layout(const std::vector<oocs_desc> &d, const std::vector<Derived> &v, std::vector<uint64_t> &ro_off,
                    std::vector<uint64_t> &ro_bytes, std::vector<uint64_t> &src_off)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    L.nwb = 1;
    int fin = 0, fout = 0;
    for (size_t i = 0; i < d.size(); ++i) {
        const Layout Li = layout_for(d[i], v[i], 1);
        L.nbuf = std::max(L.nbuf, Li.nbuf);
        L.buf_bytes = std::max(L.buf_bytes, Li.buf_bytes);
        L.in_slot_bytes = std::max(L.in_slot_bytes, Li.in_slot_bytes);
        L.out_slot_bytes = std::max(L.out_slot_bytes, Li.out_slot_bytes);
        fin = std::max(fin, v[i].fin_stream);
        fout = std::max(fout, v[i].fout);
    }
    uint64_t off = 0;
    for (int b = 0; b < L.nbuf; ++b) {
        L.w_off[0][b] = off;
        off += L.buf_bytes;
    }
    for (int q = 0; q < 3; ++q)
        for (int f = 0; f < fin; ++f) {
            L.in_off[q][f] = off;
            off += L.in_slot_bytes;
        }
    for (int q = 0; q < 3; ++q)
        for (int f = 0; f < fout; ++f) {
            L.out_off[q][f] = off;
            off += L.out_slot_bytes;
        }
    ro_off.assign(d.size(), 0);
    ro_bytes.assign(d.size(), 0);
    for (size_t i = 0; i < d.size(); ++i)
        if (v[i].ro_res) {
            ro_off[i] = off;
            ro_bytes[i] = align_up((uint64_t)d[i].nz * d[i].nx * d[i].ny * 4, 256);
            off += ro_bytes[i];
        }
    src_off.assign(d.size(), 0);
    for (size_t i = 0; i < d.size(); ++i)
        if (d[i].scheme == OOCS_WAVE) {
            src_off[i] = off;
            off += kSrcRegionBytes;
        }
    L.total = off;
    return L;
}

oocs_status batch_plans(const oocs_desc *descs, int32_t n, std::vector<oocs_desc> &d, std::vector<oocs_plan> &p,
                        std::vector<Derived> &v, std::string &err)
{
    if (!descs || n < 1 || n > 4096) {
        err = "need 1..4096 problem descriptions";
        return OOCS_ERR_INVALID_ARG;
    }
    d.assign(descs, descs + n);
    p.resize(n);
    v.resize(n);
    for (int32_t i = 0; i < n; ++i) {
        oocs_status s = plan_impl(&d[i], &p[i], err);
        if (s != OOCS_OK) {
            err = "problem " + std::to_string(i) + ": " + err;
            return s;
        }
        if (d[i].working_buffers != OOCS_SWB) {
            err = "problem " + std::to_string(i) + ": a batch runs one working buffer (OOCS_SWB)";
            return OOCS_ERR_INVALID_ARG;
        }
        if (d[i].scheme == OOCS_WAVE_ADJOINT) {
            err = "problem " + std::to_string(i) + ": the wave adjoint runs in a context of its own";
            return OOCS_ERR_INVALID_ARG;
        }
        if (d[i].temporal_depth == 0)
            d[i].temporal_depth = p[i].temporal_depth;
        v[i] = derive(d[i], p[i].slab_planes);
    }
    return OOCS_OK;
}

// Members are plain contexts whose workspace regions, streams and pipeline
// events are the batch's.  With `trace`, nothing touches CUDA.
oocs_status batch_build(oocs_batch *b, const std::vector<oocs_desc> &d, const std::vector<oocs_plan> &p,
                        const std::vector<Derived> &v, char *ws)
{
    std::vector<uint64_t> ro_off, ro_bytes, src_off;
    const Layout L = batch_layout(d, v, ro_off, ro_bytes, src_off);
    b->ws = ws;
    int d2h_base = 0;
    for (size_t i = 0; i < d.size(); ++i) {
        oocs_ctx *c = new (std::nothrow) oocs_ctx();
        if (!c)
            return fail(nullptr, OOCS_ERR_HOST_ALLOC, "cannot allocate a context");
        b->ctx.push_back(c);
        c->batch = b;
        c->trace = b->trace;
        c->d = d[i];
        c->p = p[i];
        c->v = v[i];
        c->L = L;
        c->L.ro_off = ro_off[i];
        c->L.ro_bytes = ro_bytes[i];
        c->L.src_off = src_off[i];
        c->ws = ws;
        for (int k = 0; k < 3; ++k) {
            c->st[k] = b->st[k];
            c->ev_decoded[k] = b->ev_decoded[k];
            c->ev_h2d[k] = b->ev_h2d[k];
            c->ev_wrel[k] = b->ev_wrel[k];
            c->ev_join[k] = b->ev_join[k];
            c->ev_out[k] = b->ev_out[k];
        }
        memset(&c->stats, 0, sizeof(c->stats));
        c->stats.workspace_bytes = L.total;
        c->host_base = 3 * (int)i;
        c->d2h_base = d2h_base;
        d2h_base += c->v.S;
        c->ev_d2h.assign(c->v.S, nullptr);
        c->d2h_recorded.assign(c->v.S, 0);
        if (b->trace)
            continue;
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < c->v.S && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&c->ev_d2h[k], cudaEventDisableTiming);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&c->ev_codec[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreate(&c->ev_t0);
        if (e == cudaSuccess)
            e = cudaEventCreate(&c->ev_t1);
        if (e != cudaSuccess)
            return fail(nullptr, OOCS_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
    return OOCS_OK;
}

void batch_free(oocs_batch *b)
{
    if (!b)
        return;
    if (!b->trace)
        for (int i = 0; i < 3; ++i)
            if (b->st[i])
                cudaStreamSynchronize(b->st[i]);
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    for (oocs_ctx *c : b->ctx)
        destroy_ctx(c);
    auto kill = [](cudaEvent_t &e) {
        if (e)
            cudaEventDestroy(e);
        e = nullptr;
    };
    for (int i = 0; i < 3; ++i) {
        kill(b->ev_decoded[i]);
        kill(b->ev_h2d[i]);
        kill(b->ev_wrel[i]);
        kill(b->ev_join[i]);
        kill(b->ev_out[i]);
    }
    delete b;
}

oocs_status batch_ready(oocs_batch *b)
{
    if (!b)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "batch is NULL");
    for (oocs_ctx *c : b->ctx) {
        oocs_status s = check_ready(c);
        if (s != OOCS_OK)
            return fail(nullptr, s, c->err);
        const int nf = bound_fields(c->d);
        for (int f = 0; f < nf; ++f)
            if (!c->store[f])
                return fail(nullptr, OOCS_ERR_STATE, "every field of every problem must be bound");
    }
    return OOCS_OK;
}

// Enqueue nsteps of every problem: rounds in which each unfinished problem
// sweeps its slabs once (k of its own steps), all through the batch's
// pipeline.  In a capture the streams fork from and join back into stream 0.
oocs_status batch_enqueue(oocs_batch *b, int32_t nsteps, bool capture)
{
    oocs_ctx *c0 = b->ctx[0];
    if (capture) {
        SCHED(sched_record(c0, 0, kEvJoin + 0));
        SCHED(sched_wait(c0, 1, kEvJoin + 0));
        SCHED(sched_wait(c0, 2, kEvJoin + 0));
    } else {
        SCHED(join_streams(c0));
    }
    std::vector<int32_t> left(b->ctx.size(), nsteps);
    for (bool more = true; more;) {
        more = false;
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            oocs_ctx *c = b->ctx[i];
            if (left[i] <= 0)
                continue;
            const int k_eff = std::min(left[i], c->v.k);
            const int64_t t = (int64_t)c->stats.steps_done;
            c->g = b->g;
            for (int sl = 0; sl < c->v.S; ++sl) {
                oocs_status s = enqueue_slab(c, sl, k_eff, t);
                if (s != OOCS_OK) {
                    b->g = c->g;
                    return fail(nullptr, s, c->err);
                }
            }
            b->g = c->g;
            c->stats.steps_done = (uint64_t)(t + k_eff);
            c->stats.passes_done++;
            left[i] -= k_eff;
            more = more || left[i] > 0;
        }
    }
    if (capture) {
        SCHED(sched_record(c0, 1, kEvJoin + 1));
        SCHED(sched_record(c0, 2, kEvJoin + 2));
        SCHED(sched_wait(c0, 0, kEvJoin + 1));
        SCHED(sched_wait(c0, 0, kEvJoin + 2));
        return OOCS_OK;
    }
    return join_streams(c0);
}

oocs_status batch_uploads(oocs_batch *b)
{
    for (oocs_ctx *c : b->ctx)
        if (c->v.ro_res && c->ro_dirty && !c->trace) {
            oocs_status s = upload_resident(c);
            if (s != OOCS_OK)
                return fail(nullptr, s, c->err);
        }
    return OOCS_OK;
}

void add_stats(oocs_stats &a, const oocs_stats &d, int sign)
{
    auto f = [&](uint64_t &x, uint64_t y) { x = sign > 0 ? x + y : x - y; };
    f(a.h2d_bytes, d.h2d_bytes);
    f(a.d2h_bytes, d.d2h_bytes);
    f(a.kernel_launches, d.kernel_launches);
    f(a.steps_done, d.steps_done);
    f(a.passes_done, d.passes_done);
    f(a.slabs_done, d.slabs_done);
    for (int k = 0; k < 5; ++k) {
        oocs_kernel_stats &x = k == 0 ? a.load : k == 1 ? a.step : k == 2 ? a.store : k == 3 ? a.h2d : a.d2h;
        const oocs_kernel_stats &y = k == 0 ? d.load : k == 1 ? d.step : k == 2 ? d.store : k == 3 ? d.h2d : d.d2h;
        f(x.launches, y.launches);
        f(x.units, y.units);
    }
}

oocs_stats stats_diff(const oocs_stats &after, const oocs_stats &before)
{
    oocs_stats d = after;
    add_stats(d, before, -1);
    d.workspace_bytes = 0;
    d.last_step_ms = 0.0;
    d.load.device_ms = d.step.device_ms = d.store.device_ms = 0.0;
    return d;
}

}  // namespace

extern "C" {

oocs_status oocs_batch_query(const oocs_desc *descs, int32_t n, uint64_t *workspace_bytes)
try {
    if (!workspace_bytes)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "workspace_bytes is NULL");
    std::vector<oocs_desc> d;
    std::vector<oocs_plan> p;
    std::vector<Derived> v;
    std::string err;
    oocs_status s = batch_plans(descs, n, d, p, v, err);
    if (s != OOCS_OK)
        return fail(nullptr, s, err);
    std::vector<uint64_t> ro_off, ro_bytes, src_off;
    *workspace_bytes = batch_layout(d, v, ro_off, ro_bytes, src_off).total;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_create(const oocs_desc *descs, int32_t n, void *workspace, uint64_t workspace_bytes,
                              void *const streams[3], oocs_batch **out)
try {
    if (!out)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::vector<oocs_desc> d;
    std::vector<oocs_plan> p;
    std::vector<Derived> v;
    std::string err;
    oocs_status s = batch_plans(descs, n, d, p, v, err);
    if (s != OOCS_OK)
        return fail(nullptr, s, err);
    std::vector<uint64_t> ro_off, ro_bytes, src_off;
    const uint64_t need = batch_layout(d, v, ro_off, ro_bytes, src_off).total;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
    if (workspace_bytes < need)
        return fail(nullptr, OOCS_ERR_BUDGET,
                    "workspace of " + std::to_string(workspace_bytes) + " bytes < batch's " + std::to_string(need));
    if (!streams || !streams[0] || !streams[1] || !streams[2] || streams[0] == streams[1] ||
        streams[1] == streams[2] || streams[0] == streams[2])
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "three distinct non-null streams are required");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "workspace is not device memory");
    }
    oocs_batch *b = new (std::nothrow) oocs_batch();
    if (!b)
        return fail(nullptr, OOCS_ERR_HOST_ALLOC, "cannot allocate the batch");
    for (int i = 0; i < 3; ++i)
        b->st[i] = static_cast<cudaStream_t>(streams[i]);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&b->ev_decoded[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_h2d[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_wrel[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return fail(nullptr, OOCS_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
    s = batch_build(b, d, p, v, static_cast<char *>(workspace));
    if (s != OOCS_OK) {
        std::string msg = g_last_error;
        batch_free(b);
        return fail(nullptr, s, msg);
    }
    *out = b;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_context(oocs_batch *b, int32_t i, oocs_ctx **ctx)
try {
    if (!b || !ctx || i < 0 || i >= (int32_t)b->ctx.size())
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "bad batch, index or output pointer");
    *ctx = b->ctx[i];
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_step(oocs_batch *b, int32_t nsteps)
try {
    oocs_status s = batch_ready(b);
    if (s != OOCS_OK)
        return s;
    if (nsteps < 0)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (b->capturing)
        return fail(nullptr, OOCS_ERR_STATE, "the batch is capturing a graph");
    if (nsteps == 0)
        return OOCS_OK;
    SCHED(join_streams(b->ctx[0]));
    SCHED(batch_uploads(b));
    return batch_enqueue(b, nsteps, false);
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_capture(oocs_batch *b, int32_t nsteps)
try {
    oocs_status s = batch_ready(b);
    if (s != OOCS_OK)
        return s;
    if (nsteps < 1)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "nsteps must be >= 1");
    for (oocs_ctx *c : b->ctx) {
        if (c->has_src && (int64_t)c->w.size() > kMaxDeviceWavelet)
            return fail(nullptr, OOCS_ERR_UNSUPPORTED,
                        "a source wavelet longer than " + std::to_string(kMaxDeviceWavelet) +
                            " samples cannot be read by a replayed graph; use oocs_batch_step");
        if (c->prof)
            return fail(nullptr, OOCS_ERR_STATE, "turn profiling off before capturing");
        if (c->rec || !c->srec.empty())
            return fail(nullptr, OOCS_ERR_UNSUPPORTED,
                        "receiver planes and state records are indexed by the time step, which a replayed "
                        "graph does not advance; use oocs_batch_step");
        c->t_capture = (int64_t)c->stats.steps_done;
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    // everything before, and the uploads of resident models, run now
    SCHED(join_streams(b->ctx[0]));
    SCHED(batch_uploads(b));
    SCHED(join_streams(b->ctx[0]));
    std::vector<oocs_stats> before;
    std::vector<std::vector<char>> d2h_before;
    for (oocs_ctx *c : b->ctx) {
        before.push_back(c->stats);
        d2h_before.push_back(c->d2h_recorded);
        std::fill(c->d2h_recorded.begin(), c->d2h_recorded.end(), 0);
    }
    const uint64_t g0 = b->g;
    b->cap_recorded.clear();
    cudaError_t e = cudaStreamBeginCapture(b->st[0], cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return fail(nullptr, OOCS_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    b->capturing = true;
    s = batch_enqueue(b, nsteps, true);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->st[0], &graph);
    b->capturing = false;
    // an event last recorded inside a capture cannot be waited on outside it:
    // record each again, for real, on stream 0 (the capture ran nothing, and
    // later calls are ordered by their opening join anyway)
    for (cudaEvent_t ev : b->cap_recorded)
        if (cudaEventRecord(ev, b->st[0]) != cudaSuccess && e == cudaSuccess)
            e = cudaGetLastError();
    if (s == OOCS_OK && e == cudaSuccess)
        e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph)
        cudaGraphDestroy(graph);
    // nothing ran: the host-side state goes back to before the capture
    b->graph_delta.clear();
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        oocs_ctx *c = b->ctx[i];
        b->graph_delta.push_back(stats_diff(c->stats, before[i]));
        c->stats = before[i];
        if (s != OOCS_OK || e != cudaSuccess)
            c->d2h_recorded = d2h_before[i];
    }
    if (s != OOCS_OK || e != cudaSuccess) {
        b->g = g0;
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGetLastError();
        if (s != OOCS_OK)
            return s;
        return fail(nullptr, OOCS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    b->graph_steps = nsteps;
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_launch(oocs_batch *b)
try {
    oocs_status s = batch_ready(b);
    if (s != OOCS_OK)
        return s;
    if (!b->exec)
        return fail(nullptr, OOCS_ERR_STATE, "no captured graph (oocs_batch_capture)");
    oocs_ctx *c0 = b->ctx[0];
    SCHED(join_streams(c0));
    SCHED(batch_uploads(b));
    // the time index each problem's replayed source steps count from
    for (oocs_ctx *c : b->ctx)
        if (c->has_src)
            CU(c0, launch_set_i64(c->t_dev(), (int64_t)c->stats.steps_done, b->st[0]));
    SCHED(join_streams(c0));
    CU(c0, cudaGraphLaunch(b->exec, b->st[0]));
    // later work on streams 1 and 2 follows the graph
    SCHED(sched_record(c0, 0, kEvJoin + 0));
    SCHED(sched_wait(c0, 1, kEvJoin + 0));
    SCHED(sched_wait(c0, 2, kEvJoin + 0));
    for (size_t i = 0; i < b->ctx.size(); ++i)
        add_stats(b->ctx[i]->stats, b->graph_delta[i], +1);
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_synchronize(oocs_batch *b, uint64_t timeout_ns)
try {
    if (!b)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "batch is NULL");
    for (oocs_ctx *c : b->ctx) {
        oocs_status s = oocs_synchronize(c, timeout_ns);
        if (s != OOCS_OK)
            return fail(nullptr, s, c->err);
    }
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_destroy(oocs_batch *b)
try {
    batch_free(b);
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

oocs_status oocs_batch_trace_schedule(const oocs_desc *descs, int32_t n, const int32_t *nsteps, int32_t ncalls,
                                      oocs_trace_op *ops, int64_t capacity, int64_t *count)
try {
    if (!count || (ncalls > 0 && !nsteps) || ncalls < 0 || capacity < 0 || (capacity > 0 && !ops))
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "bad trace arguments");
    *count = 0;
    std::vector<oocs_desc> d;
    std::vector<oocs_plan> p;
    std::vector<Derived> v;
    std::string err;
    oocs_status s = batch_plans(descs, n, d, p, v, err);
    if (s != OOCS_OK)
        return fail(nullptr, s, err);
    std::vector<oocs_trace_op> trace;
    oocs_batch *b = new (std::nothrow) oocs_batch();
    if (!b)
        return fail(nullptr, OOCS_ERR_HOST_ALLOC, "cannot allocate the batch");
    b->trace = &trace;
    s = batch_build(b, d, p, v, nullptr);
    static char dummy;
    for (oocs_ctx *c : b->ctx)
        for (int f = 0; f < 4; ++f)
            c->store[f] = &dummy;  // never dereferenced in trace mode
    for (int32_t i = 0; i < ncalls && s == OOCS_OK; ++i)
        if (nsteps[i] > 0)
            s = batch_enqueue(b, nsteps[i], false);
    std::string msg = g_last_error;
    batch_free(b);
    if (s != OOCS_OK)
        return fail(nullptr, s, msg);
    *count = (int64_t)trace.size();
    if ((int64_t)trace.size() > capacity)
        return fail(nullptr, OOCS_ERR_INVALID_ARG, "trace needs " + std::to_string(trace.size()) + " entries");
    for (size_t i = 0; i < trace.size(); ++i)
        ops[i] = trace[i];
    return OOCS_OK;
} catch (...) {
    return exception_status(nullptr);
}

}  // extern "C"
