// dct.cu -- host entry points of the batched orthonormal sine / cosine
// transforms F_l and F_l^T (Sec. 2.2, Eq. (16)) for the FP64 path and the
// dense split-TF32 path; the kernels are in dct_kernels.cuh, the FP32 kernels
// of the split-FP16 path in dct_f32.cu.
#include "dct_kernels.cuh"

namespace dsbt {

// Grids with their own compile-time instantiation (the power-of-two sizes of
// the common workloads); the rest take N at run time.
template <typename R, int MODE>
static FwdKernel<R> fwd_kernel(int N) {
    if (N == 2048) return k_dct_fwd<R, MODE, 1, 2048>;
    if (N == 4096) return k_dct_fwd<R, MODE, 1, 4096>;
    if (N == 8192) return k_dct_fwd<R, MODE, 1, 8192>;
    switch (odd_part(N)) {
#define DSBT_CASE(q) \
    case q: return k_dct_fwd<R, MODE, q, 0>;
        DSBT_DCT_Q_CASES(DSBT_CASE)
#undef DSBT_CASE
    }
    return nullptr;
}

template <typename R>
static InvKernel<R> inv_kernel(int N) {
    if (N == 2048) return k_dct_inv<R, 1, 2048>;
    if (N == 4096) return k_dct_inv<R, 1, 4096>;
    if (N == 8192) return k_dct_inv<R, 1, 8192>;
    switch (odd_part(N)) {
#define DSBT_CASE(q) \
    case q: return k_dct_inv<R, q, 0>;
        DSBT_DCT_Q_CASES(DSBT_CASE)
#undef DSBT_CASE
    }
    return nullptr;
}

int dct_forward_f64(const dsbt_plan* p, const GroupTable& g, bool cplx, const double* in,
                    double* out, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    FwdKernel<double> k = fwd_kernel<double, kPlain>(p->N);
    DSBT_CHECK_ARG(k != nullptr, "dct: N=%d not of the form 256 q, q <= 32", p->N);
    int rc = launch_cfg(k, p->N, sizeof(double2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctFwd, st);
    k<<<nblocks(g, p->N), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out, nullptr, nullptr, p->tw64, p->post64);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int dct_forward_f32(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in,
                    float* out_hi, float* out_lo, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    FwdKernel<float> k = fwd_kernel<float, kSplitTF32>(p->N);
    DSBT_CHECK_ARG(k != nullptr, "dct: N=%d not of the form 256 q, q <= 32", p->N);
    int rc = launch_cfg(k, p->N, sizeof(float2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctFwd, st);
    k<<<nblocks(g, p->N), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out_hi, out_lo, nullptr, p->tw32, p->post32);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int dct_inverse_f64(const dsbt_plan* p, const GroupTable& g, bool cplx, const double* in,
                    double* out, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    InvKernel<double> k = inv_kernel<double>(p->N);
    DSBT_CHECK_ARG(k != nullptr, "dct: N=%d not of the form 256 q, q <= 32", p->N);
    int rc = launch_cfg(k, p->N, sizeof(double2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctInv, st);
    k<<<nblocks(g, p->N), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out, p->tw64, p->post64);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}


}  // namespace dsbt
