// noalloc.cu -- grouped forward DSBT that allocates no memory.
//
// Some callers cannot allocate device memory at call time: a host program
// whose device memory is owned by a framework allocator that forbids direct
// cudaMalloc, a latency-critical loop that cannot afford cudaMalloc's implicit
// device synchronisation, or a deployment with a device-memory budget fixed at
// start-up.  For them this file provides dsbt_forward_grouped_noalloc, which
// runs the same kernels as dsbt_forward_grouped but takes its scratch (the
// intermediate sine/cosine coefficients between the two kernels) from a
// file-scope device array of fixed size instead of a caller workspace.
//
// The array is reserved on every GPU that loads this library, for the life of
// the process.  Host code cannot use its name as a device address, so every
// call looks the address up with cudaGetSymbolAddress, with the plan's device
// current.  The lookup allocates nothing and is cheap; doing it per call (no
// cache) keeps the address right after a cudaDeviceReset, which reloads the
// module at a new address.
#include "plan.cuh"

namespace dsbt {

int forward_grouped_with_scratch(const dsbt_plan* p, const int* counts, int dtype, const void* in,
                                 void* out, void* scratch, size_t scratch_bytes, cudaStream_t st);

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB per device

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the array on the current device.
int static_scratch(void** out) {
    void* ptr = nullptr;
    DSBT_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_static_scratch));
    *out = ptr;
    return DSBT_OK;
}

}  // namespace
}  // namespace dsbt

using namespace dsbt;

extern "C" int dsbt_forward_grouped_noalloc(const dsbt_plan* plan, const int* counts, int dtype,
                                            const void* in, void* out, void* stream) {
    DSBT_CHECK_ARG(plan != nullptr && counts != nullptr, "dsbt_forward_grouped_noalloc: NULL argument");
    DSBT_CHECK_ARG(valid_dtype(dtype), "dsbt_forward_grouped_noalloc: dtype=%d invalid", dtype);
    long long total = 0;
    for (int l = 0; l <= plan->l_max; ++l) {
        DSBT_CHECK_ARG(counts[l] >= 0, "counts[%d] negative", l);
        total += counts[l];
    }
    DSBT_CHECK_ARG(total < (1LL << 30), "too many channels");
    const size_t need = dsbt_workspace_size(plan, (int)total, dtype);
    DSBT_CHECK_ARG(need <= kStaticScratchBytes,
                   "dsbt_forward_grouped_noalloc: needs %zu bytes of scratch, the static array holds %zu "
                   "(use dsbt_forward_grouped with a workspace)",
                   need, kStaticScratchBytes);
    int dev = 0;
    DSBT_CUDA_TRY(cudaGetDevice(&dev));
    DSBT_CHECK_ARG(dev == plan->device, "current device %d is not the plan's device %d", dev, plan->device);
    void* scratch = nullptr;
    int rc = static_scratch(&scratch);
    if (rc) return rc;
    return forward_grouped_with_scratch(plan, counts, dtype, in, out, scratch, kStaticScratchBytes,
                                        (cudaStream_t)stream);
}
