// plan.cuh -- internal plan layout and kernel launchers of the DSBT library.
#pragma once

#include <vector>

#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace dsbt { struct FastData; struct FtcData; }

struct dsbt_plan {
    int N;
    int l_max;
    int flags;
    int device;
    double r_max;
    double dk;                 // pi / r_max
    size_t nn;                 // N * N
    // FP64 factors, [(l_max+1)][N][N], entry (n - p_l, m - p_l) of T_l
    double* T64;
    // FP64 transposes T_l^T (same layout), kept with DSBT_PLAN_FP64 so that the
    // inverse contraction of narrow groups also reads contiguous rows
    double* Tt64;
    // split-TF32 factors (FP32 containers holding TF32 values), same layout:
    // T = Thi + Tlo (A operand of the forward contraction) and the transposes
    // Tt = T^T (A operand of the inverse contraction).
    float* Thi;
    float* Tlo;
    float* Tthi;
    float* Ttlo;
    // FFT twiddles w^t = exp(-2 pi i t / N), t < N, and the cosine-transform
    // post-twiddles exp(-i pi k / (2N)), k < N.
    double2* tw64;
    double2* post64;
    float2* tw32;
    float2* post32;
    // corrected momenta [(l_max+1)][N] of DSBT_PLAN_KCORR (else nullptr: the
    // kinetic phase uses k~_n = n dk by parity)
    double* knl;
    // hierarchical FP64 data of DSBT_PLAN_FAST64 (fast64.cu), else nullptr
    dsbt::FastData* fast;
    // interval bases and projections of DSBT_PLAN_FAST_SPLIT (fast_split.cu), else nullptr
    dsbt::FtcData* ftc;
    unsigned* status;          // device status word (kStatusOk / kStatusTimeout)
    unsigned spin_limit;       // polls of a bounded mbarrier wait in the tensor-core kernels
    double check_err;
    bool has_tmaps;
    CUtensorMap tm_T_hi, tm_T_lo, tm_Tt_hi, tm_Tt_lo;
};

namespace dsbt {

// ---- launch accounting (profile.cu)
enum KernelId {
    kKPlan = 0, kKDctFwd, kKDctInv, kKContract64, kKContractTF32, kKPhase, kKSplit,
    kKTdsePot, kKTdseAng, kKTdseReduce, kNumKernels
};
// Wraps one kernel launch: counts it and, while profiling is enabled, records
// CUDA events on `st` before the launch and at scope exit.
class ProfScope {
  public:
    ProfScope(int kid, cudaStream_t st);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    int kid_;
    cudaStream_t st_;
    cudaEvent_t a_, b_;
};

// Turns event recording on/off without clearing records; returns the old state.
int profile_set_enabled(int on);

// ---- grouped calls on device buffers with a caller workspace (capi.cu):
// which = 0 forward, 1 inverse, 2 kinetic step (dsbt_*_grouped semantics).
// uoff (device, one per channel in call order, optional): the channel's element
// offset in `in` / `out` instead of c * N (interval-scheme plans, complex64,
// forward and kinetic only).
int grouped_device_call(int which, const dsbt_plan* p, const int* counts, int dtype, double tau,
                        const void* in, void* out, void* ws, size_t ws_b, cudaStream_t st,
                        const long long* uoff = nullptr);

// ---- plan build (plan.cu)
int plan_build_factors(dsbt_plan* p, cudaStream_t st);
int plan_probe(dsbt_plan* p, cudaStream_t st);
// Default polls of a bounded mbarrier wait (tc_ptx.cuh kSpinLimit).
unsigned tc_default_spin_limit();
int build_first_rows(double* dst, int N, int lmax, int R, cudaStream_t st);
int plan_twiddles_only(int N, double r_max, cudaStream_t st, dsbt_plan** out);
void plan_release(dsbt_plan* p);

// ---- TMA descriptors (tma.cu)
// Encode a 2-D FP32 tensor map over a row-major [rows][cols] array with a box of
// box_cols x box_rows and 128-byte swizzling.
void kcorr_table(int N, double r_max, int l_max, std::vector<double>& out);

int encode_tmap_f32_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                          uint32_t box_rows, uint32_t box_cols);
// The same over FP16 elements (box_cols = 64).
int encode_tmap_f16_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                          uint32_t box_rows, uint32_t box_cols);

// ---- sine/cosine transforms (dct.cu)
// Forward F_l for every channel of the group table; writes planar lines.
//   FP64: in = double (real or interleaved complex), out64 = [lines][N] double
//   FP32: in = float, out_hi/out_lo = TF32 split of the result, [lines][N]
int dct_forward_f64(const dsbt_plan* p, const GroupTable& g, bool cplx, const double* in,
                    double* out, cudaStream_t st);
int dct_forward_f32(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in,
                    float* out_hi, float* out_lo, cudaStream_t st);
//   FP16 split: out_hi/out_lo = FP16 pair of 2^e f per channel (||2^e psi|| in
//   [2^12, 2^13)), scale[line] = 2^-e
int dct_forward_f16(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in, __half* out_hi,
                    __half* out_lo, float* scale, cudaStream_t st);
// Inverse F_l^T from planar lines to the caller's layout.
int dct_inverse_f64(const dsbt_plan* p, const GroupTable& g, bool cplx, const double* in,
                    double* out, cudaStream_t st);
int dct_inverse_f32(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in,
                    float* out, cudaStream_t st);

// ---- FP64 contraction (gemm_f64.cu)
// in_cplx / out_cplx = 1: the caller's interleaved complex layout (line 2j+s of a
// group is part s of its channel j); 0: planar lines [line][N].
// dir = +1: out = T_l in (forward), dir = -1: out = T_l^T in (inverse).
// phase: optional complex phase per coefficient applied to the result (kinetic
// step), indexed [parity][N] as double2; nullptr for none.
int contract_f64(const dsbt_plan* p, const GroupTable& g, int dir, const double* in, int in_cplx,
                 double* out, int out_cplx, const double2* phase, cudaStream_t st,
                 double* fast_scratch = nullptr);
// DSBT_PLAN_FAST64 (fast64.cu)
bool fast_supported(int N);
int fast_build(dsbt_plan* p, cudaStream_t st);
void fast_free(dsbt_plan* p);
size_t fast_scratch_bytes(const dsbt_plan* p, int lines);
int contract_f64_fast(const dsbt_plan* p, const GroupTable& g, int dir, const double* in, double* out,
                      const double2* phase, double* scratch, cudaStream_t st);
// Orthonormal basis [len][64] of the polynomials of degree < min(64, len) on
// the points x_t = (2t+1)/len - 1 (Arnoldi with two Gram-Schmidt passes).
void poly_basis(int len, std::vector<double>& Q);
// DSBT_PLAN_FAST_SPLIT (fast_split.cu)
bool ftc_supported(int N);
int ftc_build(dsbt_plan* p, cudaStream_t st);
void ftc_free(dsbt_plan* p);
size_t ftc_scratch_bytes(const dsbt_plan* p, size_t lines);
// Units between a unit's two kinds of tiles in the interval-scheme launch.
void ftc_set_lag(dsbt_plan* p, int lag);
// The interval-scheme contraction on FP16 pairs of planar lines scaled per
// line by 1 / scale[line] (see dct_forward_f16), one launch per direction.
// Output modes: kOutPlanarSplit writes the scaled FP16 pair (out0 hi, out1
// lo); kOutUserC64 / kOutUserF32 / kOutPlanarF32 write unscaled FP32.
// `scratch` holds ftc_scratch_bytes of the call's lines (the augmented lines
// and the launch's counters, zeroed here).
int contract_split_fast(const dsbt_plan* p, const GroupTable& g, int dir, const __half* in_hi, const __half* in_lo,
                        const float* scale, int out_mode, void* out0, void* out1, const float2* phase, void* scratch,
                        cudaStream_t st);

// ---- angular rule of the TDSE (tdse.cu), shared with tdse3d.cu
// L-point Gauss-Legendre nodes x (cos theta) and weights w.
void tdse_gauss_legendre(int L, std::vector<double>& x, std::vector<double>& w);
// P[i][j], i < L: rows l = m + i of the normalised associated Legendre functions
// times sqrt(w_j), orthonormalised on the rule (an orthogonal L x L matrix).
void tdse_angular_rows(int L, int m, const std::vector<double>& x, const std::vector<double>& w,
                       std::vector<double>& P);

// ---- split-TF32 tensor-core contraction (gemm_tf32x3.cu)
// B operand: TF32 split lines [lines][N] (hi, lo).  `sched` is a device int
// (zeroed here before the launch) for the dynamic tile scheduler.  Output modes:
enum OutMode { kOutUserC64 = 0, kOutUserF32 = 1, kOutPlanarF32 = 2, kOutPlanarSplit = 3 };
int contract_tf32x3(const dsbt_plan* p, const GroupTable& g, int dir, const float* in_hi,
                    const float* in_lo, int out_mode, float* out0, float* out1,
                    const float2* phase, int* sched, cudaStream_t st);

}  // namespace dsbt
