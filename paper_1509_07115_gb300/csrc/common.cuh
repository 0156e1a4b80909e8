// common.cuh -- shared host/device helpers of the DSBT library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/dsbt.h"

namespace dsbt {

// ----------------------------------------------------------------- error state

void set_error(const char* fmt, ...);

#define DSBT_CUDA_TRY(expr)                                                            \
    do {                                                                               \
        cudaError_t e__ = (expr);                                                      \
        if (e__ != cudaSuccess) {                                                      \
            ::dsbt::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,              \
                              cudaGetErrorString(e__));                                \
            return DSBT_ERR_CUDA;                                                      \
        }                                                                              \
    } while (0)

#define DSBT_CHECK_ARG(cond, ...)                                                      \
    do {                                                                               \
        if (!(cond)) {                                                                 \
            ::dsbt::set_error(__VA_ARGS__);                                            \
            return DSBT_ERR_INVALID;                                                   \
        }                                                                              \
    } while (0)

// ----------------------------------------------------------------- launch attributes

// Raises the dynamic shared-memory limit of kernel `fn` on the current device
// to `bytes` the first time it is needed there (profile.cu).  The limit is a
// per-device attribute of each kernel; setting it before every launch would be
// correct but can wait for the device, which stalls a host that queues work
// ahead on several streams.  Thread-safe.
int ensure_smem(const void* fn, size_t bytes);

// ----------------------------------------------------------------- index helpers

__host__ __device__ inline int parity_p(int l) { return (l & 1) ? 0 : 1; }   // p_l
__host__ __device__ inline int n0_of(int l) { return (l + 2) / 2; }           // ceil((l+1)/2)
// Number of completion rows n in [p_l, n0_l - 1] (Sec. 2.5).
__host__ __device__ inline int n_extra(int l) { return n0_of(l) - parity_p(l); }
// Momentum of storage row s (row n = s + p_l) of T_l in units of dk for the
// kinetic energy (Eq. (65) and the remark after it): n on the regular rows;
// the completion rows n < n0_l (n = 0 of odd l among them) project onto
// non-regular high-frequency functions and take the largest grid momentum N.
__host__ __device__ inline int k_index(int l, int s, int N) {
    const int n = s + parity_p(l);
    return n < n0_of(l) ? N : n;
}
// Entry of the parity phase table (rows s = 0..N-1 with momentum n = s + p,
// n = 0 -> N) that holds the phase of storage row s of T_l.
__host__ __device__ inline int phase_entry(int l, int s, int N) {
    return (s + parity_p(l) < n0_of(l)) ? ((l & 1) ? 0 : N - 1) : s;
}

inline bool is_complex(int dtype) { return dtype == DSBT_C128 || dtype == DSBT_C64; }
inline bool is_fp64(int dtype) { return dtype == DSBT_F64 || dtype == DSBT_C128; }
inline bool valid_dtype(int dtype) { return dtype >= DSBT_F64 && dtype <= DSBT_C64; }

// Channel groups of one call (one group per angular momentum present).
constexpr int kMaxGroups = 72;

struct GroupTable {
    int ngroups;
    int total_lines;            // real lines over all groups
    int l[kMaxGroups];          // angular momentum of the group
    int chan0[kMaxGroups + 1];  // first channel of the group (prefix, +1 sentinel)
    int line0[kMaxGroups + 1];  // first real line (complex channel = 2 lines)
    // Element offset of each channel in the caller's arrays (device array, one
    // per channel), or nullptr: channel c at c * N.  Set only for the
    // interval-scheme path of the uneven batch, which gathers the channels of
    // several transforms on one grid into one call.
    const long long* uoff = nullptr;
};

// Device-side status word written by kernels whose waits gave up.
enum : unsigned { kStatusOk = 0, kStatusTimeout = 1 };

// ----------------------------------------------------------------- TF32 split

// Round an FP32 value to TF32 (10 explicit mantissa bits), nearest-even.
// Finite inputs only.
__host__ __device__ inline float round_tf32(float x) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, 4);
#endif
    u += 0x0FFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float y;
    memcpy(&y, &u, 4);
    return y;
#endif
}

}  // namespace dsbt
