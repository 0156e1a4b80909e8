// stream.cu -- grouped transforms on HOST-resident channels, streamed through
// the GPU in chunks so that the host->device copy of one chunk, the transform
// of the previous one and the device->host copy of the one before run at the
// same time (two copy streams plus the caller's stream).
//
// The channels (l-major, as in dsbt_forward_grouped) are cut into nchunks
// contiguous channel ranges; a range may start or end inside an l group, and
// each chunk is one grouped call with the counts of the groups it covers.  Two
// device slots for input and two for output alternate between chunks.  Every
// output element is computed by the same arithmetic as the device entry points
// (the transform of a channel does not depend on the other channels of a call).
#include <math.h>

#include <algorithm>
#include <vector>

#include "plan.cuh"

namespace dsbt {

namespace {

constexpr int kSlots = 2;

size_t elem_bytes(int dtype) {
    switch (dtype) {
        case DSBT_F64: return 8;
        case DSBT_C128: return 16;
        case DSBT_F32: return 4;
        default: return 8;   // DSBT_C64
    }
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Chunks {
    long long total = 0;
    int n = 0;
    long long max_chan = 0;
    long long begin(int k) const { return total * k / n; }
};

int plan_chunks(const dsbt_plan* p, const int* counts, int nchunks, Chunks* c) {
    DSBT_CHECK_ARG(p != nullptr && counts != nullptr, "NULL argument");
    DSBT_CHECK_ARG(nchunks >= 0 && nchunks <= 4096, "nchunks=%d out of range", nchunks);
    long long total = 0;
    for (int l = 0; l <= p->l_max; ++l) {
        DSBT_CHECK_ARG(counts[l] >= 0, "counts[%d] negative", l);
        total += counts[l];
    }
    DSBT_CHECK_ARG(total < (1LL << 30), "too many channels");
    c->total = total;
    c->n = (int)std::max(1LL, std::min<long long>(nchunks == 0 ? 8 : nchunks, std::max(1LL, total)));
    c->max_chan = 0;
    for (int k = 0; k < c->n; ++k) c->max_chan = std::max(c->max_chan, c->begin(k + 1) - c->begin(k));
    return DSBT_OK;
}

size_t slot_bytes(const dsbt_plan* p, const Chunks& c, int dtype) {
    return a256((size_t)c.max_chan * p->N * elem_bytes(dtype));
}

size_t stream_ws_bytes(const dsbt_plan* p, const Chunks& c, int dtype) {
    return 2 * kSlots * slot_bytes(p, c, dtype) + dsbt_workspace_size(p, (int)c.max_chan, dtype) + 256;
}

int run_streamed(int which, const dsbt_plan* p, const int* counts, int dtype, double tau, const void* host_in,
                 void* host_out, int nchunks, void* ws, size_t ws_b, cudaStream_t st) {
    Chunks c;
    int rc = plan_chunks(p, counts, nchunks, &c);
    if (rc) return rc;
    DSBT_CHECK_ARG(valid_dtype(dtype), "dtype=%d invalid", dtype);
    DSBT_CHECK_ARG(which != 2 || dtype == DSBT_C64 || dtype == DSBT_C128, "kinetic step needs a complex dtype");
    DSBT_CHECK_ARG(which != 2 || isfinite(tau), "tau must be finite");
    if (c.total == 0) return DSBT_OK;
    DSBT_CHECK_ARG(host_in != nullptr && host_out != nullptr && host_in != host_out, "bad host buffers");
    DSBT_CHECK_ARG(ws != nullptr && ws_b >= stream_ws_bytes(p, c, dtype), "workspace too small (need %zu bytes)",
                   stream_ws_bytes(p, c, dtype));
    const size_t eb = elem_bytes(dtype), row = (size_t)p->N * eb, sb = slot_bytes(p, c, dtype);
    unsigned char* base = (unsigned char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    unsigned char* in_slot[kSlots];
    unsigned char* out_slot[kSlots];
    for (int s = 0; s < kSlots; ++s) {
        in_slot[s] = base + s * sb;
        out_slot[s] = base + (kSlots + s) * sb;
    }
    void* gws = base + 2 * kSlots * sb;
    const size_t gws_b = dsbt_workspace_size(p, (int)c.max_chan, dtype);

    // first channel of each l group
    const int L = p->l_max + 1;
    std::vector<long long> chan0(L + 1, 0);
    for (int l = 0; l < L; ++l) chan0[l + 1] = chan0[l] + counts[l];

    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev;   // start, then per chunk: in, comp, out
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (s_in) cudaStreamDestroy(s_in);
        if (s_out) cudaStreamDestroy(s_out);
    };
    if (cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking) != cudaSuccess) {
        cleanup();
        set_error("stream creation failed");
        return DSBT_ERR_CUDA;
    }
    ev.resize(1 + 3 * (size_t)c.n, nullptr);
    for (auto& e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            e = nullptr;
            cleanup();
            set_error("event creation failed");
            return DSBT_ERR_CUDA;
        }
    auto EV = [&](int k, int kind) { return ev[1 + 3 * (size_t)k + kind]; };   // kind 0 in, 1 comp, 2 out
    cudaError_t ce = cudaSuccess;
    // earlier work on the caller's stream (e.g. producers of host_in) comes first
    ce = cudaEventRecord(ev[0], st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s_in, ev[0], 0);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s_out, ev[0], 0);
    std::vector<int> sub(L);
    for (int k = 0; k < c.n && ce == cudaSuccess && !rc; ++k) {
        const int slot = k % kSlots;
        const long long a = c.begin(k), b = c.begin(k + 1);
        if (a == b) continue;
        for (int l = 0; l < L; ++l)
            sub[l] = (int)std::max(0LL, std::min(b, chan0[l + 1]) - std::max(a, chan0[l]));
        // host -> device, once the transform of chunk k - kSlots has read this slot
        if (k >= kSlots) ce = cudaStreamWaitEvent(s_in, EV(k - kSlots, 1), 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(in_slot[slot], (const unsigned char*)host_in + a * row, (size_t)(b - a) * row,
                                 cudaMemcpyHostToDevice, s_in);
        if (ce == cudaSuccess) ce = cudaEventRecord(EV(k, 0), s_in);
        // transform on the caller's stream, once the input landed and the
        // device->host copy of chunk k - kSlots has read the output slot
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, EV(k, 0), 0);
        if (ce == cudaSuccess && k >= kSlots) ce = cudaStreamWaitEvent(st, EV(k - kSlots, 2), 0);
        if (ce != cudaSuccess) break;
        rc = grouped_device_call(which, p, sub.data(), dtype, tau, in_slot[slot], out_slot[slot], gws, gws_b, st);
        if (rc) break;
        ce = cudaEventRecord(EV(k, 1), st);
        // device -> host
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s_out, EV(k, 1), 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync((unsigned char*)host_out + a * row, out_slot[slot], (size_t)(b - a) * row,
                                 cudaMemcpyDeviceToHost, s_out);
        if (ce == cudaSuccess) ce = cudaEventRecord(EV(k, 2), s_out);
    }
    // the caller's stream completes after the last copy back
    if (ce == cudaSuccess && !rc) {
        ce = cudaEventRecord(ev[0], s_out);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, ev[0], 0);
    }
    cleanup();
    if (ce != cudaSuccess) {
        set_error("streamed transform: %s", cudaGetErrorString(ce));
        return DSBT_ERR_CUDA;
    }
    return rc;
}

}  // namespace
}  // namespace dsbt

using namespace dsbt;

extern "C" size_t dsbt_host_workspace_size(const dsbt_plan* plan, const int* counts, int dtype, int nchunks) {
    Chunks c;
    if (!valid_dtype(dtype) || plan_chunks(plan, counts, nchunks, &c) != DSBT_OK) return 0;
    return stream_ws_bytes(plan, c, dtype);
}

extern "C" int dsbt_forward_grouped_host(const dsbt_plan* plan, const int* counts, int dtype, const void* host_in,
                                         void* host_out, int nchunks, void* workspace, size_t workspace_bytes,
                                         void* stream) {
    return run_streamed(0, plan, counts, dtype, 0.0, host_in, host_out, nchunks, workspace, workspace_bytes,
                        (cudaStream_t)stream);
}

extern "C" int dsbt_inverse_grouped_host(const dsbt_plan* plan, const int* counts, int dtype, const void* host_in,
                                         void* host_out, int nchunks, void* workspace, size_t workspace_bytes,
                                         void* stream) {
    return run_streamed(1, plan, counts, dtype, 0.0, host_in, host_out, nchunks, workspace, workspace_bytes,
                        (cudaStream_t)stream);
}

extern "C" int dsbt_kinetic_grouped_host(const dsbt_plan* plan, const int* counts, int dtype, double tau,
                                         const void* host_in, void* host_out, int nchunks, void* workspace,
                                         size_t workspace_bytes, void* stream) {
    return run_streamed(2, plan, counts, dtype, tau, host_in, host_out, nchunks, workspace, workspace_bytes,
                        (cudaStream_t)stream);
}
