// capi.cu -- C ABI entry points: argument checks, group tables, workspace
// layout, and the kernel sequence of each call.
//
//   forward  (Eqs. (18), (24)):  in -> F_l (sine/cosine kernel) -> T_l contraction -> out
//   inverse  (Eq. (25)):         in -> T_l^T contraction -> F_l^T kernel -> out
//   kinetic  (Eq. (81), A = 0):  in -> F_l -> T_l with exp(-i k~^2 tau/2) in the
//                                epilogue -> T_l^T -> F_l^T -> out
#include <math.h>

#include "plan.cuh"

namespace dsbt {

namespace {

// TF32 split of caller data into planar lines (complex channel c -> lines 2c, 2c+1).
__global__ void k_split_lines(const float* __restrict__ in, float* __restrict__ hi, float* __restrict__ lo,
                              long long total) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const float v = in[i];
    const float h = round_tf32(v);
    hi[i] = h;
    lo[i] = round_tf32(v - h);
}

__global__ void k_split_lines_c(const float2* __restrict__ in, float* __restrict__ hi,
                                float* __restrict__ lo, int N, long long total) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long long c = i / N, n = i % N;
    const float2 v = in[i];
    const float hr = round_tf32(v.x), hi_ = round_tf32(v.y);
    const size_t o = (size_t)(2 * c) * N + n;
    hi[o] = hr;
    lo[o] = round_tf32(v.x - hr);
    hi[o + N] = hi_;
    lo[o + N] = round_tf32(v.y - hi_);
}

// FP16 pair of caller data for the interval-scheme contraction: one CTA per
// channel (N values, or N complex values = two lines) computes ||psi||, picks
// 2^e with ||2^e psi|| in [2^12, 2^13) and writes hi = fp16(2^e x),
// lo = fp16(2^e x - hi) to the channel's planar lines and 2^-e to scale[line].
__global__ void k_split_f16(const float* __restrict__ in, int cplx, int N, __half* __restrict__ hi,
                            __half* __restrict__ lo, float* __restrict__ scale) {
    const long long c = blockIdx.x;
    const int per = cplx ? 2 : 1;
    const float* x = in + c * (long long)N * per;
    float part = 0.f;
    for (int i = threadIdx.x; i < N * per; i += blockDim.x) part += x[i] * x[i];
    __shared__ float red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const float nrm = sqrtf(red[0]);
    const int e = (nrm > 0.f && isfinite(nrm)) ? 12 - ilogbf(nrm) : 0;
    const float fs = ldexpf(1.f, e);
    const long long line = c * per;
    if (threadIdx.x < per) scale[line + threadIdx.x] = ldexpf(1.f, -e);
    for (int i = threadIdx.x; i < N * per; i += blockDim.x) {
        const int part_ = cplx ? (i & 1) : 0, n = cplx ? (i >> 1) : i;
        const float v = x[i] * fs;
        const __half h = __float2half_rn(v);
        const size_t o = (size_t)(line + part_) * N + n;
        hi[o] = h;
        lo[o] = __float2half_rn(v - __half2float(h));
    }
}

// Interleaved complex128 channels <-> planar real lines (channel c -> lines
// 2c, 2c+1), for the O(N l log N) FP64 contraction, which works on planar lines.
__global__ void k_deinterleave64(const double2* __restrict__ in, double* __restrict__ lines, int N, long long total) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long long c = i / N, n = i % N;
    const double2 v = in[i];
    lines[(2 * c) * N + n] = v.x;
    lines[(2 * c + 1) * N + n] = v.y;
}

__global__ void k_interleave64(const double* __restrict__ lines, double2* __restrict__ out, int N, long long total) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long long c = i / N, n = i % N;
    out[i] = make_double2(lines[(2 * c) * N + n], lines[(2 * c + 1) * N + n]);
}

// exp(-i k~_n^2 tau / 2) on the unified momentum grid (Eq. (65)): storage index
// k of parity class par (0: even l, n = k + 1; 1: odd l, n = k) maps to
// k~ = n dk, except the odd-l coefficient n = 0, which takes k~_N = N dk.
// Kinetic phase table exp(-i k^2 tau / 2): rows = 2 by parity of l with
// k = k~_n = n dk (n = 0 -> N dk) when knl is NULL, else rows = l_max + 1 with
// the plan's corrected momenta knl[l][s].
__global__ void k_phase(double2* ph64, float2* ph32, int N, double dk, double tau, const double* __restrict__ knl,
                        int rows) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * N) return;
    double kt;
    if (knl) {
        kt = knl[i];
    } else {
        const int par = i / N, k = i % N;
        int n = (par == 0) ? k + 1 : k;
        if (n == 0) n = N;
        kt = n * dk;
    }
    double s, c;
    sincos(-0.5 * kt * kt * tau, &s, &c);
    if (ph64) ph64[i] = make_double2(c, s);
    if (ph32) ph32[i] = make_float2((float)c, (float)s);
}

// Rows of the phase table (see k_phase).
inline int phase_rows(const dsbt_plan* p) { return p->knl ? p->l_max + 1 : 2; }

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Workspace {
    // FP64 path
    double* f64a;
    double* f64b;
    double2* ph64;
    double* fast;    // scratch of the DSBT_PLAN_FAST64 contraction (or nullptr)
    // TF32 path
    float* hi_a;
    float* lo_a;
    float* hi_b;
    float* lo_b;
    float* planar;   // aliases hi_a
    float2* ph32;
    int* sched;      // tile-scheduler counter of the tensor-core contraction
    // interval-scheme path (plans with DSBT_PLAN_FAST_SPLIT): FP16 pairs of the
    // lines before (a) and between (b) the contractions, per-line unscale
    // factors, the augmented lines; planar aliases the a pair
    __half* h_hi_a;
    __half* h_lo_a;
    __half* h_hi_b;
    __half* h_lo_b;
    float* scale;
    void* ftc;
};

size_t lines_of(int total_channels, int dtype) {
    return (size_t)total_channels * (is_complex(dtype) ? 2 : 1);
}

size_t ws_bytes(const dsbt_plan* p, int total_channels, int dtype) {
    const size_t R = lines_of(total_channels, dtype);
    const int N = p->N;
    const size_t PR = (size_t)phase_rows(p) * N;
    if (is_fp64(dtype))
        return align256(R * N * sizeof(double)) * 2 + align256(PR * sizeof(double2)) +
               align256(fast_scratch_bytes(p, (int)R)) + 256;
    if (p->ftc)   // FP16 pairs a, b (4 B per value each), scale, phase, counter, augmented lines
        return align256(R * N * 4) * 2 + align256(R * sizeof(float)) + align256(PR * sizeof(float2)) + 256 +
               align256(ftc_scratch_bytes(p, R)) + 256;
    return align256(R * N * sizeof(float)) * 4 + align256(PR * sizeof(float2)) + 256 + 256;
}

Workspace carve(const dsbt_plan* pl, void* base, int total_channels, int dtype) {
    const int N = pl->N;
    const size_t PR = (size_t)phase_rows(pl) * N;
    Workspace w{};
    const size_t R = lines_of(total_channels, dtype);
    unsigned char* p = (unsigned char*)(((uintptr_t)base + 255) & ~(uintptr_t)255);
    if (is_fp64(dtype)) {
        const size_t b = align256(R * N * sizeof(double));
        w.f64a = (double*)p;
        w.f64b = (double*)(p + b);
        w.ph64 = (double2*)(p + 2 * b);
        w.fast = pl->fast ? (double*)(p + 2 * b + align256(PR * sizeof(double2))) : nullptr;
    } else if (pl->ftc) {
        const size_t b = align256(R * N * 4);   // one FP16 pair of every line
        w.h_hi_a = (__half*)p;
        w.h_lo_a = w.h_hi_a + R * N;
        w.planar = (float*)p;                   // FP32 lines after the last contraction
        w.h_hi_b = (__half*)(p + b);
        w.h_lo_b = w.h_hi_b + R * N;
        w.scale = (float*)(p + 2 * b);
        unsigned char* q = p + 2 * b + align256(R * sizeof(float));
        w.ph32 = (float2*)q;
        w.sched = (int*)(q + align256(PR * sizeof(float2)));
        w.ftc = q + align256(PR * sizeof(float2)) + 256;
    } else {
        const size_t b = align256(R * N * sizeof(float));
        w.hi_a = (float*)p;
        w.lo_a = (float*)(p + b);
        w.hi_b = (float*)(p + 2 * b);
        w.lo_b = (float*)(p + 3 * b);
        w.planar = w.hi_a;
        w.ph32 = (float2*)(p + 4 * b);
        w.sched = (int*)(p + 4 * b + align256(PR * sizeof(float2)));
    }
    return w;
}

int build_groups(const dsbt_plan* p, const int* counts, int ngroups_in, const int* ls, int dtype,
                 GroupTable& g) {
    g.ngroups = 0;
    int chan = 0, line = 0;
    const int per = is_complex(dtype) ? 2 : 1;
    for (int i = 0; i < ngroups_in; ++i) {
        const int c = counts[i];
        DSBT_CHECK_ARG(c >= 0, "negative channel count for l=%d", ls[i]);
        DSBT_CHECK_ARG(ls[i] >= 0 && ls[i] <= p->l_max, "l=%d outside the plan's 0..%d", ls[i], p->l_max);
        if (c == 0) continue;
        DSBT_CHECK_ARG(g.ngroups < kMaxGroups, "too many groups");
        DSBT_CHECK_ARG((long long)chan + c < (1LL << 30), "too many channels");
        g.l[g.ngroups] = ls[i];
        g.chan0[g.ngroups] = chan;
        g.line0[g.ngroups] = line;
        ++g.ngroups;
        chan += c;
        line += c * per;
    }
    g.chan0[g.ngroups] = chan;
    g.line0[g.ngroups] = line;
    g.total_lines = line;
    return DSBT_OK;
}

int check_common(const dsbt_plan* p, int dtype, const void* in, void* out, void* ws, size_t ws_b,
                 int total_channels) {
    DSBT_CHECK_ARG(p != nullptr, "plan is NULL");
    DSBT_CHECK_ARG(valid_dtype(dtype), "dtype=%d invalid", dtype);
    if (total_channels == 0) return DSBT_OK;
    DSBT_CHECK_ARG(in != nullptr && out != nullptr, "in/out is NULL");
    DSBT_CHECK_ARG(in != out, "in and out must not alias");
    DSBT_CHECK_ARG(ws != nullptr, "workspace is NULL");
    const size_t need = ws_bytes(p, total_channels, dtype);
    DSBT_CHECK_ARG(ws_b >= need, "workspace too small: %zu < %zu bytes", ws_b, need);
    if (is_fp64(dtype) && !p->T64) {
        set_error("FP64 dtype needs a plan built with DSBT_PLAN_FP64");
        return DSBT_ERR_UNSUPPORTED;
    }
    if (!is_fp64(dtype) && !p->has_tmaps && !p->ftc) {
        set_error("FP32 dtype needs a plan built with DSBT_PLAN_TF32X3 or DSBT_PLAN_FAST_SPLIT");
        return DSBT_ERR_UNSUPPORTED;
    }
    return DSBT_OK;
}

int run_forward(const dsbt_plan* p, const GroupTable& g, int dtype, const void* in, void* out,
                void* ws, cudaStream_t st) {
    if (g.total_lines == 0) return DSBT_OK;
    const bool cplx = is_complex(dtype);
    Workspace w = carve(p, ws, g.chan0[g.ngroups], dtype);
    int rc;
    if (is_fp64(dtype)) {
        rc = dct_forward_f64(p, g, cplx, (const double*)in, w.f64a, st);
        if (rc) return rc;
        if (p->fast && cplx) {   // O(N l log N) contraction on planar lines, then interleave
            rc = contract_f64(p, g, +1, w.f64a, 0, w.f64b, 0, nullptr, st, w.fast);
            if (rc) return rc;
            const long long total = (long long)g.chan0[g.ngroups] * p->N;
            ProfScope ps(kKSplit, st);
            k_interleave64<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(w.f64b, (double2*)out, p->N, total);
            DSBT_CUDA_TRY(cudaGetLastError());
            return DSBT_OK;
        }
        return contract_f64(p, g, +1, w.f64a, 0, (double*)out, cplx ? 1 : 0, nullptr, st, w.fast);
    }
    if (p->ftc) {   // interval scheme on FP16 pairs
        rc = dct_forward_f16(p, g, cplx, (const float*)in, w.h_hi_a, w.h_lo_a, w.scale, st);
        if (rc) return rc;
        return contract_split_fast(p, g, +1, w.h_hi_a, w.h_lo_a, w.scale, cplx ? kOutUserC64 : kOutUserF32, out,
                                   nullptr, nullptr, w.ftc, st);
    }
    rc = dct_forward_f32(p, g, cplx, (const float*)in, w.hi_a, w.lo_a, st);
    if (rc) return rc;
    return contract_tf32x3(p, g, +1, w.hi_a, w.lo_a, cplx ? kOutUserC64 : kOutUserF32, (float*)out,
                           nullptr, nullptr, w.sched, st);
}

int run_inverse(const dsbt_plan* p, const GroupTable& g, int dtype, const void* in, void* out,
                void* ws, cudaStream_t st) {
    if (g.total_lines == 0) return DSBT_OK;
    const bool cplx = is_complex(dtype);
    Workspace w = carve(p, ws, g.chan0[g.ngroups], dtype);
    int rc;
    if (is_fp64(dtype)) {
        const double* src = (const double*)in;
        if (p->fast && cplx) {   // planar lines for the O(N l log N) contraction
            const long long total = (long long)g.chan0[g.ngroups] * p->N;
            {
                ProfScope ps(kKSplit, st);
                k_deinterleave64<<<(unsigned)((total + 255) / 256), 256, 0, st>>>((const double2*)in, w.f64b, p->N,
                                                                                   total);
            }
            DSBT_CUDA_TRY(cudaGetLastError());
            src = w.f64b;
        }
        rc = contract_f64(p, g, -1, src, (cplx && src == in) ? 1 : 0, w.f64a, 0, nullptr, st, w.fast);
        if (rc) return rc;
        return dct_inverse_f64(p, g, cplx, w.f64a, (double*)out, st);
    }
    if (p->ftc) {   // interval scheme on FP16 pairs
        {
            ProfScope ps(kKSplit, st);
            k_split_f16<<<(unsigned)g.chan0[g.ngroups], 256, 0, st>>>((const float*)in, cplx ? 1 : 0, p->N,
                                                                       w.h_hi_b, w.h_lo_b, w.scale);
        }
        DSBT_CUDA_TRY(cudaGetLastError());
        rc = contract_split_fast(p, g, -1, w.h_hi_b, w.h_lo_b, w.scale, kOutPlanarF32, w.planar, nullptr, nullptr,
                                 w.ftc, st);
        if (rc) return rc;
        return dct_inverse_f32(p, g, cplx, w.planar, (float*)out, st);
    }
    const long long total = (long long)g.chan0[g.ngroups] * p->N;
    const int bs = 256;
    {
    ProfScope ps(kKSplit, st);
    if (cplx)
        k_split_lines_c<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>((const float2*)in, w.hi_b, w.lo_b,
                                                                          p->N, total);
    else
        k_split_lines<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>((const float*)in, w.hi_b, w.lo_b,
                                                                        total);
    }
    DSBT_CUDA_TRY(cudaGetLastError());
    rc = contract_tf32x3(p, g, -1, w.hi_b, w.lo_b, kOutPlanarF32, w.planar, nullptr, nullptr, w.sched, st);
    if (rc) return rc;
    return dct_inverse_f32(p, g, cplx, w.planar, (float*)out, st);
}

int run_kinetic(const dsbt_plan* p, const GroupTable& g, int dtype, double tau, const void* in, void* out,
                void* ws, cudaStream_t st) {
    if (g.total_lines == 0) return DSBT_OK;
    Workspace w = carve(p, ws, g.chan0[g.ngroups], dtype);
    const int N = p->N;
    int rc;
    if (is_fp64(dtype)) {
        {
            ProfScope ps(kKPhase, st);
            const int rows = phase_rows(p);
            k_phase<<<(rows * N + 255) / 256, 256, 0, st>>>(w.ph64, nullptr, N, p->dk, tau, p->knl, rows);
        }
        DSBT_CUDA_TRY(cudaGetLastError());
        rc = dct_forward_f64(p, g, true, (const double*)in, w.f64a, st);
        if (!rc) rc = contract_f64(p, g, +1, w.f64a, 0, w.f64b, 0, w.ph64, st, w.fast);
        if (!rc) rc = contract_f64(p, g, -1, w.f64b, 0, w.f64a, 0, nullptr, st, w.fast);
        if (!rc) rc = dct_inverse_f64(p, g, true, w.f64a, (double*)out, st);
        return rc;
    }
    {
        ProfScope ps(kKPhase, st);
        const int rows = phase_rows(p);
        k_phase<<<(rows * N + 255) / 256, 256, 0, st>>>(nullptr, w.ph32, N, p->dk, tau, p->knl, rows);
    }
    DSBT_CUDA_TRY(cudaGetLastError());
    if (p->ftc) {   // interval scheme on FP16 pairs; the lines stay scaled until the last contraction
        rc = dct_forward_f16(p, g, true, (const float*)in, w.h_hi_a, w.h_lo_a, w.scale, st);
        if (!rc)
            rc = contract_split_fast(p, g, +1, w.h_hi_a, w.h_lo_a, w.scale, kOutPlanarSplit, w.h_hi_b, w.h_lo_b,
                                     w.ph32, w.ftc, st);
        if (!rc)
            rc = contract_split_fast(p, g, -1, w.h_hi_b, w.h_lo_b, w.scale, kOutPlanarF32, w.planar, nullptr,
                                     nullptr, w.ftc, st);
        if (!rc) rc = dct_inverse_f32(p, g, true, w.planar, (float*)out, st);
        return rc;
    }
    rc = dct_forward_f32(p, g, true, (const float*)in, w.hi_a, w.lo_a, st);
    if (!rc) rc = contract_tf32x3(p, g, +1, w.hi_a, w.lo_a, kOutPlanarSplit, w.hi_b, w.lo_b, w.ph32, w.sched, st);
    if (!rc) rc = contract_tf32x3(p, g, -1, w.hi_b, w.lo_b, kOutPlanarF32, w.planar, nullptr, nullptr, w.sched, st);
    if (!rc) rc = dct_inverse_f32(p, g, true, w.planar, (float*)out, st);
    return rc;
}

int grouped_call(int which, const dsbt_plan* p, const int* counts, int dtype, double tau, const void* in,
                 void* out, void* ws, size_t ws_b, void* stream, const long long* uoff = nullptr) {
    DSBT_CHECK_ARG(p != nullptr, "plan is NULL");
    DSBT_CHECK_ARG(counts != nullptr, "counts is NULL");
    int ls[kMaxGroups];
    long long total = 0;
    for (int l = 0; l <= p->l_max; ++l) {
        ls[l] = l;
        DSBT_CHECK_ARG(counts[l] >= 0, "counts[%d] negative", l);
        total += counts[l];
    }
    DSBT_CHECK_ARG(total < (1LL << 30), "too many channels");
    int rc = check_common(p, dtype, in, out, ws, ws_b, (int)total);
    if (rc || total == 0) return rc;
    GroupTable g;
    rc = build_groups(p, counts, p->l_max + 1, ls, dtype, g);
    if (rc) return rc;
    if (uoff) {   // channels gathered from the caller's arrays by offset: interval-scheme C64 paths only
        DSBT_CHECK_ARG(p->ftc != nullptr && dtype == DSBT_C64 && which != 1,
                       "channel offsets need a DSBT_PLAN_FAST_SPLIT plan, complex64, forward or kinetic");
        g.uoff = uoff;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (which == 0) return run_forward(p, g, dtype, in, out, ws, st);
    if (which == 1) return run_inverse(p, g, dtype, in, out, ws, st);
    DSBT_CHECK_ARG(is_complex(dtype), "kinetic step needs a complex dtype");
    DSBT_CHECK_ARG(isfinite(tau), "tau must be finite");
    return run_kinetic(p, g, dtype, tau, in, out, ws, st);
}

int single_call(int which, const dsbt_plan* p, int l, int nchan, int dtype, const void* in, void* out,
                void* ws, size_t ws_b, void* stream) {
    DSBT_CHECK_ARG(p != nullptr, "plan is NULL");
    DSBT_CHECK_ARG(l >= 0 && l <= p->l_max, "l=%d outside the plan's 0..%d", l, p->l_max);
    DSBT_CHECK_ARG(nchan >= 0 && nchan < (1 << 30), "nchan=%d invalid", nchan);
    int rc = check_common(p, dtype, in, out, ws, ws_b, nchan);
    if (rc || nchan == 0) return rc;
    GroupTable g;
    rc = build_groups(p, &nchan, 1, &l, dtype, g);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    return which == 0 ? run_forward(p, g, dtype, in, out, ws, st) : run_inverse(p, g, dtype, in, out, ws, st);
}

}  // namespace

// Grouped forward with a scratch buffer supplied by the caller of this
// function (used by entry points that bring their own scratch memory).
int forward_grouped_with_scratch(const dsbt_plan* p, const int* counts, int dtype, const void* in,
                                 void* out, void* scratch, size_t scratch_bytes, cudaStream_t st) {
    return grouped_call(0, p, counts, dtype, 0.0, in, out, scratch, scratch_bytes, st);
}

// Grouped forward (which = 0), inverse (1) or kinetic step (2) on device
// buffers with a caller-supplied workspace (the host-streamed entry points).
int grouped_device_call(int which, const dsbt_plan* p, const int* counts, int dtype, double tau,
                        const void* in, void* out, void* ws, size_t ws_b, cudaStream_t st, const long long* uoff) {
    return grouped_call(which, p, counts, dtype, tau, in, out, ws, ws_b, st, uoff);
}

// Grouped kinetic step with a scratch buffer supplied by the caller of this
// function (the TDSE propagator's inner call).
int kinetic_grouped_with_scratch(const dsbt_plan* p, const int* counts, int dtype, double tau,
                                 const void* in, void* out, void* scratch, size_t scratch_bytes,
                                 cudaStream_t st) {
    return grouped_call(2, p, counts, dtype, tau, in, out, scratch, scratch_bytes, st);
}

}  // namespace dsbt

using namespace dsbt;

extern "C" size_t dsbt_workspace_size(const dsbt_plan* plan, int total_channels, int dtype) {
    if (!plan || total_channels < 0 || !valid_dtype(dtype)) return 0;
    return ws_bytes(plan, total_channels, dtype);
}

extern "C" int dsbt_forward(const dsbt_plan* plan, int l, int nchan, int dtype, const void* in, void* out,
                            void* workspace, size_t workspace_bytes, void* stream) {
    return single_call(0, plan, l, nchan, dtype, in, out, workspace, workspace_bytes, stream);
}

extern "C" int dsbt_inverse(const dsbt_plan* plan, int l, int nchan, int dtype, const void* in, void* out,
                            void* workspace, size_t workspace_bytes, void* stream) {
    return single_call(1, plan, l, nchan, dtype, in, out, workspace, workspace_bytes, stream);
}

extern "C" int dsbt_forward_grouped(const dsbt_plan* plan, const int* counts, int dtype, const void* in,
                                    void* out, void* workspace, size_t workspace_bytes, void* stream) {
    return grouped_call(0, plan, counts, dtype, 0.0, in, out, workspace, workspace_bytes, stream);
}

extern "C" int dsbt_inverse_grouped(const dsbt_plan* plan, const int* counts, int dtype, const void* in,
                                    void* out, void* workspace, size_t workspace_bytes, void* stream) {
    return grouped_call(1, plan, counts, dtype, 0.0, in, out, workspace, workspace_bytes, stream);
}

extern "C" int dsbt_kinetic_grouped(const dsbt_plan* plan, const int* counts, int dtype, double tau,
                                    const void* in, void* out, void* workspace, size_t workspace_bytes,
                                    void* stream) {
    return grouped_call(2, plan, counts, dtype, tau, in, out, workspace, workspace_bytes, stream);
}

extern "C" int dsbt_device_status(const dsbt_plan* plan, int reset, int* status_out) {
    DSBT_CHECK_ARG(plan != nullptr && status_out != nullptr, "NULL argument");
    unsigned s = 0;
    DSBT_CUDA_TRY(cudaMemcpy(&s, plan->status, sizeof(s), cudaMemcpyDeviceToHost));
    *status_out = (int)s;
    if (reset) DSBT_CUDA_TRY(cudaMemset(plan->status, 0, sizeof(unsigned)));
    return DSBT_OK;
}
