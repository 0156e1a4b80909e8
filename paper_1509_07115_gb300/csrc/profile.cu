// profile.cu -- launch counting and optional per-kernel CUDA-event timing.
//
// Every kernel launch of the library goes through a ProfScope, which bumps a
// process-wide launch counter and, while profiling is enabled, records a pair
// of CUDA events on the launch stream around the launch.  dsbt_profile_read
// synchronises on the recorded events and sums their elapsed times per kernel.
#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "plan.cuh"

namespace dsbt {

namespace {

const char* kNames[kNumKernels] = {"plan_build", "dct_forward", "dct_inverse", "contract_f64",
                                   "contract_tf32x3", "kinetic_phase", "split_lines", "tdse_potential",
                                   "tdse_angular", "tdse_reduce"};

std::atomic<long long> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;

struct Rec {
    int kid;
    cudaEvent_t a, b;
};
std::vector<Rec> g_recs;

}  // namespace

int ensure_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;   // (kernel, device) -> bytes set
    int dev = 0;
    DSBT_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = done[{fn, dev}];
    if (have >= bytes) return DSBT_OK;
    DSBT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
    return DSBT_OK;
}

ProfScope::ProfScope(int kid, cudaStream_t st) : kid_(kid), st_(st), a_(nullptr), b_(nullptr) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_enabled.load(std::memory_order_relaxed)) {
        if (cudaEventCreate(&a_) == cudaSuccess && cudaEventCreate(&b_) == cudaSuccess) {
            cudaEventRecord(a_, st_);
        } else {
            a_ = b_ = nullptr;
        }
    }
}

ProfScope::~ProfScope() {
    if (a_ && b_) {
        cudaEventRecord(b_, st_);
        std::lock_guard<std::mutex> lk(g_mu);
        g_recs.push_back(Rec{kid_, a_, b_});
    }
}

int profile_set_enabled(int on) { return g_enabled.exchange(on ? 1 : 0); }

}  // namespace dsbt

using namespace dsbt;

extern "C" long long dsbt_launch_count(void) { return g_launches.load(); }

extern "C" int dsbt_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
    g_enabled.store(on ? 1 : 0);
    return DSBT_OK;
}

extern "C" const char* dsbt_kernel_name(int kernel_id) {
    if (kernel_id < 0 || kernel_id >= kNumKernels) return nullptr;
    return kNames[kernel_id];
}

extern "C" int dsbt_profile_read(int kernel_id, int* launches, double* total_ms) {
    DSBT_CHECK_ARG(kernel_id >= 0 && kernel_id < kNumKernels, "kernel id %d out of range", kernel_id);
    std::lock_guard<std::mutex> lk(g_mu);
    int n = 0;
    double ms = 0.0;
    for (auto& r : g_recs) {
        if (r.kid != kernel_id) continue;
        DSBT_CUDA_TRY(cudaEventSynchronize(r.b));
        float t = 0.f;
        DSBT_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        ++n;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    return DSBT_OK;
}
