// dct_f32.cu -- the FP32 sine / cosine kernels of the split-FP16 path (the
// forward transform with FP16-pair output, the inverse from planar FP32
// lines), with one instantiation per plan grid N = 256 q, q = 1..32: N fixed
// at compile time turns every padded shared-memory index into one base per
// thread plus constant offsets.  Kept apart from dct.cu so that the two
// translation units compile in parallel.
#include "dct_kernels.cuh"

namespace dsbt {

namespace {

// (q, odd part of q) for N = 256 q
#define DSBT_DCT_GRIDS(X) X(1, 1) X(2, 1) X(3, 3) X(4, 1) X(5, 5) X(6, 3) X(7, 7) X(8, 1) X(9, 9) X(10, 5) \
    X(11, 11) X(12, 3) X(13, 13) X(14, 7) X(15, 15) X(16, 1) X(17, 17) X(18, 9) X(19, 19) X(20, 5) X(21, 21)   \
    X(22, 11) X(23, 23) X(24, 3) X(25, 25) X(26, 13) X(27, 27) X(28, 7) X(29, 29) X(30, 15) X(31, 31) X(32, 1)

FwdKernel<float> fwd_kernel_f16(int N) {
    if (N % 256) return nullptr;
    switch (N / 256) {
#define DSBT_CASE(q, Q) \
    case q: return k_dct_fwd<float, kSplitF16, Q, 256 * q>;
        DSBT_DCT_GRIDS(DSBT_CASE)
#undef DSBT_CASE
    }
    return nullptr;
}

InvKernel<float> inv_kernel_f32(int N) {
    if (N % 256) return nullptr;
    switch (N / 256) {
#define DSBT_CASE(q, Q) \
    case q: return k_dct_inv<float, Q, 256 * q>;
        DSBT_DCT_GRIDS(DSBT_CASE)
#undef DSBT_CASE
    }
    return nullptr;
}

}  // namespace

int dct_forward_f16(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in, __half* out_hi,
                    __half* out_lo, float* scale, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    FwdKernel<float> k = fwd_kernel_f16(p->N);
    DSBT_CHECK_ARG(k != nullptr, "dct: N=%d not of the form 256 q, q <= 32", p->N);
    int rc = launch_cfg(k, p->N, sizeof(float2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctFwd, st);
    k<<<nblocks(g, p->N), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out_hi, out_lo, scale, p->tw32, p->post32);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int dct_inverse_f32(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in,
                    float* out, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    InvKernel<float> k = inv_kernel_f32(p->N);
    DSBT_CHECK_ARG(k != nullptr, "dct: N=%d not of the form 256 q, q <= 32", p->N);
    int rc = launch_cfg(k, p->N, sizeof(float2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctInv, st);
    k<<<nblocks(g, p->N), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out, p->tw32, p->post32);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

}  // namespace dsbt
