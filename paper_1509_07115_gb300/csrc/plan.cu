// plan.cu -- DSBT plan: GPU generation of the Fourier-to-Bessel factors T_l.
//
// The factors follow Sec. 2.3-2.5 of the paper:
//   regular rows n >= n0_l (Eqs. (38) Tdef, (39) Ldef, (42) alpha_n):
//     T_{n.} = u / ||u||,  u_m = [P_l(n-m, 2n-1) - P_l(n-m-1, 2n-1)] sqrt(w_m) (m < n),
//     u_n = 1, zero above the diagonal.  (The diagonal of I - L is
//     2/(1 + P_l(-1, 2n-1)) and every entry of the row carries that positive
//     factor, which the normalisation removes.)
//   completion rows p_l <= n < n0_l (Eq. (43) Tadd):
//     T_{nm} proportional to P_{2n-p}(N_l - m, 2N_l) sqrt(w_m), unit norm.
//
// DLOP values are generated in FP64 along x (not along the degree) with the
// second-order difference equation of the Hahn polynomials Q_l(x; 0, 0, M),
//     l(l+1) Q(x) = B(x) Q(x+1) - [B(x) + D(x)] Q(x) + D(x) Q(x-1),
//     B(x) = (x+1)(x-M),  D(x) = x(x-M-1),  Q(0) = 1,
// written for the backward difference d(x) = Q(x+1) - Q(x) that the rows need:
//     d(x) = [l(l+1) Q(x) + D(x) d(x-1)] / B(x),   Q(x+1) = Q(x) + d(x),
// marching from the grid end x = 0 towards the middle.  On that side of the
// grid the wanted polynomial is the dominant solution, so the march keeps
// FP64 accuracy for every l <= 64, and carrying d(x) instead of Q(x) avoids
// the cancellation of O(M^2) terms of the plain form (the three-term
// recurrence in the degree, by contrast, loses all digits in the first rows
// when l approaches 2n).
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>

#include <mutex>
#include <new>

#include "plan.cuh"

namespace dsbt {

static thread_local char g_err[512];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// ------------------------------------------------------------------ kernels

// s + c += v with Neumaier's compensation (the row norms must not lose the
// small entries against large partial sums).
__device__ __forceinline__ void neumaier_add(double& s, double& c, double v) {
    const double t = s + v;
    c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}

// One thread per (l, storage row r < R): writes row r of T_l into
// T64[l][r][0..N) (which the caller zeroed; R = N builds the whole matrix).
// Two passes over x: the first accumulates ||u||^2, the second writes u / ||u||,
// so nothing is re-read from memory.
__global__ void k_build_rows(double* __restrict__ T64, int N, int lmax, int R) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)(lmax + 1) * R) return;
    const int l = (int)(gid / R);
    const int r = (int)(gid % R);
    const int p = parity_p(l);
    const int n = r + p;
    const int n0 = n0_of(l);
    const int Nl = N + p - 1;
    double* row = T64 + ((size_t)l * R + r) * (size_t)N;
    const double ll1 = (double)l * (double)(l + 1);
    const double sqrt_half = 0.70710678118654752440;

    if (n >= n0) {
        const double M = 2.0 * n - 1.0;
        const int X = n - p;   // differences at i = 1..X, i = n - m
        double ss = 0.0, sc = 0.0;   // Neumaier-compensated sum of u_m^2, m < n
        for (int pass = 0; pass < 2; ++pass) {
            const double inv = (pass == 0) ? 0.0 : 1.0 / sqrt(1.0 + (ss + sc));   // + u_n^2 = 1
            double q = 1.0, d = 0.0;
            for (int x = 0; x < X; ++x) {
                const double xd = (double)x;
                const double B = (xd + 1.0) * (xd - M);
                const double D = xd * (xd - M - 1.0);
                d = (ll1 * q + D * d) / B;
                q += d;
                const int m = n - (x + 1);
                const double u = d * (m == 0 ? sqrt_half : 1.0);
                if (pass == 0) neumaier_add(ss, sc, __dmul_rn(u, u));
                else row[m - p] = u * inv;
            }
            if (pass == 1) row[n - p] = inv;
        }
    } else {
        // completion row: degree e = 2n - p on the grid 0..2 N_l, x = N_l - m
        const int e = 2 * n - p;
        const double M = 2.0 * Nl;
        const double ee1 = (double)e * (double)(e + 1);
        const int X = Nl - p;  // x = 0..X
        double ss = 0.0, sc = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            const double inv = (pass == 0) ? 0.0 : 1.0 / sqrt(ss + sc);
            double q = 1.0, d = 0.0;
            for (int x = 0; x <= X; ++x) {
                const int m = Nl - x;
                const double v = q * (m == 0 ? sqrt_half : 1.0);
                if (pass == 0) neumaier_add(ss, sc, __dmul_rn(v, v));
                else row[m - p] = v * inv;
                const double xd = (double)x;
                const double B = (xd + 1.0) * (xd - M);
                const double D = xd * (xd - M - 1.0);
                d = (ee1 * q + D * d) / B;
                q += d;
            }
        }
    }
}

// FP64 transpose of T_l (32x32 shared-memory tiles).
__global__ void k_transpose64(const double* __restrict__ T64, double* __restrict__ Tt64, int N) {
    __shared__ double t[32][33];
    const size_t off = (size_t)blockIdx.z * N * N;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        t[k][threadIdx.x] = T64[off + (size_t)(r0 + k) * N + c0 + threadIdx.x];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        Tt64[off + (size_t)(c0 + k) * N + r0 + threadIdx.x] = t[threadIdx.x][k];
}

// TF32 split of T_l and of its transpose (32x32 shared-memory tiles).
__global__ void k_split_T(const double* __restrict__ T64, float* __restrict__ Thi,
                          float* __restrict__ Tlo, float* __restrict__ Tthi,
                          float* __restrict__ Ttlo, int N) {
    __shared__ float hi_s[32][33];
    __shared__ float lo_s[32][33];
    const size_t off = (size_t)blockIdx.z * N * N;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        const double v = T64[off + (size_t)r * N + c];
        const float h = round_tf32((float)v);
        const float lo = round_tf32((float)(v - (double)h));
        Thi[off + (size_t)r * N + c] = h;
        Tlo[off + (size_t)r * N + c] = lo;
        hi_s[k][threadIdx.x] = h;
        lo_s[k][threadIdx.x] = lo;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = c0 + k, c = r0 + threadIdx.x;   // transposed position
        Tthi[off + (size_t)r * N + c] = hi_s[threadIdx.x][k];
        Ttlo[off + (size_t)r * N + c] = lo_s[threadIdx.x][k];
    }
}

__device__ inline double probe_value(int l, int m, int probe) {
    // deterministic pseudo-random value in [-1, 1) (splitmix64 of the indices)
    unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(1 + m + 131071 * l + 7919 * probe);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// y = T_l x for every l: one warp per row (coalesced row reads).
__global__ void k_probe_fwd(const double* __restrict__ T64, double* __restrict__ y, int N, int probe) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.y;
    if (warp >= N) return;
    const double* row = T64 + ((size_t)l * N + warp) * N;
    double s = 0.0;
    for (int m = lane; m < N; m += 32) s += row[m] * probe_value(l, m, probe);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[(size_t)l * N + warp] = s;
}

// z = T_l^T y, error max |z - x| accumulated as the bit pattern of a
// non-negative double (monotone under unsigned comparison).
__global__ void k_probe_bwd(const double* __restrict__ T64, const double* __restrict__ y, int N,
                            int probe, unsigned long long* __restrict__ err_bits) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (m >= N) return;
    const double* Tl = T64 + (size_t)l * N * N;
    const double* yl = y + (size_t)l * N;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s += Tl[(size_t)n * N + m] * yl[n];
    const double e = fabs(s - probe_value(l, m, probe));
    atomicMax(err_bits, (unsigned long long)__double_as_longlong(e));
}

__global__ void k_twiddles(double2* tw64, double2* post64, float2* tw32, float2* post32, int N) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    double s, c;
    sincospi(-2.0 * (double)t / (double)N, &s, &c);
    tw64[t] = make_double2(c, s);
    tw32[t] = make_float2((float)c, (float)s);
    sincospi(-(double)t / (2.0 * (double)N), &s, &c);
    post64[t] = make_double2(c, s);
    post32[t] = make_float2((float)c, (float)s);
}

// ------------------------------------------------------------------ host side

// Rows r < R of T_l (l = 0..lmax) for a grid of N points, FP64, into
// dst[l][r][N] (device, zeroed here).
int build_first_rows(double* dst, int N, int lmax, int R, cudaStream_t st) {
    DSBT_CUDA_TRY(cudaMemsetAsync(dst, 0, (size_t)(lmax + 1) * R * N * sizeof(double), st));
    const long long threads = (long long)(lmax + 1) * R;
    ProfScope ps(kKPlan, st);
    k_build_rows<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(dst, N, lmax, R);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

// Orthogonality probe of the FP64 factors (Eq. (25), T^{-1} = T^T): two
// pseudo-random vectors x per l, max |T^T (T x) - x| into p->check_err;
// DSBT_ERR_PLAN_CHECK above 1e-12.
int plan_probe(dsbt_plan* p, cudaStream_t st) {
    const int N = p->N, L = p->l_max + 1;
    double* y = nullptr;
    unsigned long long* err = nullptr;
    DSBT_CUDA_TRY(cudaMallocAsync((void**)&y, (size_t)L * N * sizeof(double), st));
    DSBT_CUDA_TRY(cudaMallocAsync((void**)&err, sizeof(unsigned long long), st));
    DSBT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned long long), st));
    for (int probe = 0; probe < 2; ++probe) {
        ProfScope ps(kKPlan, st);
        dim3 gf((N * 32 + 255) / 256, L);
        k_probe_fwd<<<gf, 256, 0, st>>>(p->T64, y, N, probe);
        dim3 gb((N + 255) / 256, L);
        k_probe_bwd<<<gb, 256, 0, st>>>(p->T64, y, N, probe, err);
    }
    DSBT_CUDA_TRY(cudaGetLastError());
    unsigned long long err_h = 0;
    DSBT_CUDA_TRY(cudaMemcpyAsync(&err_h, err, sizeof(err_h), cudaMemcpyDeviceToHost, st));
    DSBT_CUDA_TRY(cudaFreeAsync(y, st));
    DSBT_CUDA_TRY(cudaFreeAsync(err, st));
    DSBT_CUDA_TRY(cudaStreamSynchronize(st));
    double e;
    memcpy(&e, &err_h, sizeof(e));
    p->check_err = e;   // |x| <= 1 with max close to 1, so this is the relative error
    if (!(e <= 1e-12)) {
        set_error("plan check failed: max |T^T T x - x| = %.3e", e);
        return DSBT_ERR_PLAN_CHECK;
    }
    return DSBT_OK;
}

int plan_build_factors(dsbt_plan* p, cudaStream_t st) {
    const int N = p->N, L = p->l_max + 1;
    const size_t bytes64 = (size_t)L * p->nn * sizeof(double);
    DSBT_CUDA_TRY(cudaMemsetAsync(p->T64, 0, bytes64, st));
    {
        const long long threads = (long long)L * N;
        const int bs = 128;
        ProfScope ps(kKPlan, st);
        k_build_rows<<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(p->T64, N, p->l_max, N);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    {
        const int nthreads = 256;
        ProfScope ps(kKPlan, st);
        k_twiddles<<<(N + nthreads - 1) / nthreads, nthreads, 0, st>>>(p->tw64, p->post64, p->tw32,
                                                                       p->post32, N);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    int rc = plan_probe(p, st);
    if (rc) return rc;
    if (p->flags & DSBT_PLAN_FP64) {
        dim3 grid(N / 32, N / 32, L), block(32, 8);
        ProfScope ps(kKPlan, st);
        k_transpose64<<<grid, block, 0, st>>>(p->T64, p->Tt64, N);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    if (p->flags & DSBT_PLAN_TF32X3) {
        dim3 grid(N / 32, N / 32, L), block(32, 8);
        ProfScope ps(kKPlan, st);
        k_split_T<<<grid, block, 0, st>>>(p->T64, p->Thi, p->Tlo, p->Tthi, p->Ttlo, N);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    return DSBT_OK;
}

// A plan that holds only the FFT twiddles of an N-point grid (no factors):
// used by the batch of uneven transforms for its sine/cosine kernels.
int plan_twiddles_only(int N, double r_max, cudaStream_t st, dsbt_plan** out) {
    dsbt_plan* p = new (std::nothrow) dsbt_plan();
    if (!p) return DSBT_ERR_NOMEM;
    p->N = N;
    p->l_max = -1;
    p->r_max = r_max;
    p->dk = M_PI / r_max;
    p->nn = (size_t)N * N;
    p->spin_limit = tc_default_spin_limit();
    cudaGetDevice(&p->device);
    bool ok = cudaMalloc((void**)&p->tw64, N * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void**)&p->post64, N * sizeof(double2)) == cudaSuccess &&
              cudaMalloc((void**)&p->tw32, N * sizeof(float2)) == cudaSuccess &&
              cudaMalloc((void**)&p->post32, N * sizeof(float2)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(p->tw64); cudaFree(p->post64); cudaFree(p->tw32); cudaFree(p->post32);
        delete p;
        set_error("plan_twiddles_only: device allocation failed");
        return DSBT_ERR_NOMEM;
    }
    k_twiddles<<<(N + 255) / 256, 256, 0, st>>>(p->tw64, p->post64, p->tw32, p->post32, N);
    DSBT_CUDA_TRY(cudaGetLastError());
    *out = p;
    return DSBT_OK;
}

static void plan_free(dsbt_plan* p) {
    if (!p) return;
    fast_free(p);
    ftc_free(p);
    cudaFree(p->T64);
    cudaFree(p->Tt64);
    cudaFree(p->knl);
    cudaFree(p->Thi);
    cudaFree(p->Tlo);
    cudaFree(p->Tthi);
    cudaFree(p->Ttlo);
    cudaFree(p->tw64);
    cudaFree(p->post64);
    cudaFree(p->tw32);
    cudaFree(p->post32);
    cudaFree(p->status);
    delete p;
}

void plan_release(dsbt_plan* p) { plan_free(p); }

}  // namespace dsbt

using namespace dsbt;

extern "C" const char* dsbt_last_error(void) { return g_err; }

extern "C" int dsbt_plan_create(int N, double r_max, int l_max, int flags, void* stream,
                                dsbt_plan** out) {
    g_err[0] = 0;
    DSBT_CHECK_ARG(out != nullptr, "dsbt_plan_create: out is NULL");
    *out = nullptr;
    DSBT_CHECK_ARG(N >= 256 && N <= 8192 && N % 256 == 0,
                   "dsbt_plan_create: N=%d must be a multiple of 256 in [256, 8192]", N);
    DSBT_CHECK_ARG(l_max >= 0 && l_max <= 64, "dsbt_plan_create: l_max=%d not in [0, 64]", l_max);
    DSBT_CHECK_ARG(n0_of(l_max) <= N, "dsbt_plan_create: l_max too large for N");
    DSBT_CHECK_ARG(r_max > 0.0 && isfinite(r_max), "dsbt_plan_create: r_max must be positive");
    DSBT_CHECK_ARG((flags & (DSBT_PLAN_FP64 | DSBT_PLAN_TF32X3 | DSBT_PLAN_FAST_SPLIT)) != 0 &&
                       (flags & ~(DSBT_PLAN_FP64 | DSBT_PLAN_TF32X3 | DSBT_PLAN_KCORR | DSBT_PLAN_FAST64 |
                                  DSBT_PLAN_FAST_SPLIT)) == 0,
                   "dsbt_plan_create: flags=%d invalid", flags);
    DSBT_CHECK_ARG(!(flags & DSBT_PLAN_FAST64) || ((flags & DSBT_PLAN_FP64) && fast_supported(N)),
                   "dsbt_plan_create: DSBT_PLAN_FAST64 needs DSBT_PLAN_FP64 and N / 64 a power of two");
    DSBT_CHECK_ARG(!(flags & DSBT_PLAN_FAST_SPLIT) || ftc_supported(N),
                   "dsbt_plan_create: DSBT_PLAN_FAST_SPLIT needs N a multiple of 128 with 2 to 64 leaves");
    cudaStream_t st = (cudaStream_t)stream;
    dsbt_plan* p = new (std::nothrow) dsbt_plan();
    if (!p) {
        set_error("dsbt_plan_create: host allocation failed");
        return DSBT_ERR_NOMEM;
    }
    p->N = N;
    p->l_max = l_max;
    p->flags = flags;
    p->r_max = r_max;
    p->dk = M_PI / r_max;
    p->nn = (size_t)N * N;
    p->spin_limit = tc_default_spin_limit();
    cudaGetDevice(&p->device);
    const size_t L = (size_t)l_max + 1;
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        return cudaMalloc(ptr, bytes) == cudaSuccess;
    };
    bool ok = alloc((void**)&p->T64, L * p->nn * sizeof(double));
    if (ok && (flags & DSBT_PLAN_FP64)) ok = alloc((void**)&p->Tt64, L * p->nn * sizeof(double));
    if (ok && (flags & DSBT_PLAN_TF32X3)) {
        ok = alloc((void**)&p->Thi, L * p->nn * sizeof(float)) &&
             alloc((void**)&p->Tlo, L * p->nn * sizeof(float)) &&
             alloc((void**)&p->Tthi, L * p->nn * sizeof(float)) &&
             alloc((void**)&p->Ttlo, L * p->nn * sizeof(float));
    }
    ok = ok && alloc((void**)&p->tw64, N * sizeof(double2)) &&
         alloc((void**)&p->post64, N * sizeof(double2)) &&
         alloc((void**)&p->tw32, N * sizeof(float2)) &&
         alloc((void**)&p->post32, N * sizeof(float2)) &&
         alloc((void**)&p->status, sizeof(unsigned));
    if (ok && (flags & DSBT_PLAN_KCORR)) ok = alloc((void**)&p->knl, L * N * sizeof(double));
    if (!ok) {
        cudaGetLastError();
        plan_free(p);
        set_error("dsbt_plan_create: device allocation failed (N=%d, l_max=%d)", N, l_max);
        return DSBT_ERR_NOMEM;
    }
    if (cudaMemsetAsync(p->status, 0, sizeof(unsigned), st) != cudaSuccess) {
        plan_free(p);
        set_error("dsbt_plan_create: memset failed");
        return DSBT_ERR_CUDA;
    }
    if (flags & DSBT_PLAN_KCORR) {   // corrected momenta, computed on the host
        std::vector<double> k;
        kcorr_table(N, r_max, l_max, k);
        if (cudaMemcpy(p->knl, k.data(), k.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            plan_free(p);
            set_error("dsbt_plan_create: momentum table upload failed");
            return DSBT_ERR_CUDA;
        }
    }
    int rc = plan_build_factors(p, st);
    if (rc == DSBT_OK && (flags & DSBT_PLAN_FAST64)) rc = fast_build(p, st);
    if (rc == DSBT_OK && (flags & DSBT_PLAN_FAST_SPLIT)) rc = ftc_build(p, st);
    if (rc == DSBT_OK && (flags & DSBT_PLAN_TF32X3)) {
        const uint64_t rows = (uint64_t)L * N;
        rc = encode_tmap_f32_sw128(&p->tm_T_hi, p->Thi, rows, N, 128, 32);
        if (rc == DSBT_OK) rc = encode_tmap_f32_sw128(&p->tm_T_lo, p->Tlo, rows, N, 128, 32);
        if (rc == DSBT_OK) rc = encode_tmap_f32_sw128(&p->tm_Tt_hi, p->Tthi, rows, N, 128, 32);
        if (rc == DSBT_OK) rc = encode_tmap_f32_sw128(&p->tm_Tt_lo, p->Ttlo, rows, N, 128, 32);
        p->has_tmaps = (rc == DSBT_OK);
    }
    if (rc == DSBT_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("dsbt_plan_create: %s", cudaGetErrorString(cudaGetLastError()));
        rc = DSBT_ERR_CUDA;
    }
    if (rc != DSBT_OK) {
        plan_free(p);
        return rc;
    }
    if (!(flags & DSBT_PLAN_FP64)) {
        // the FP64 copy was only needed to build and check; keep memory lean
        cudaFree(p->T64);
        p->T64 = nullptr;
    }
    *out = p;
    return DSBT_OK;
}

extern "C" int dsbt_plan_destroy(dsbt_plan* plan) {
    if (!plan) return DSBT_OK;
    cudaDeviceSynchronize();
    plan_free(plan);
    return DSBT_OK;
}

extern "C" int dsbt_plan_info(const dsbt_plan* plan, int* N, int* l_max, int* flags,
                              double* check_err) {
    DSBT_CHECK_ARG(plan != nullptr, "dsbt_plan_info: plan is NULL");
    if (N) *N = plan->N;
    if (l_max) *l_max = plan->l_max;
    if (flags) *flags = plan->flags;
    if (check_err) *check_err = plan->check_err;
    return DSBT_OK;
}

extern "C" int dsbt_plan_get_T(const dsbt_plan* plan, int l, double* dst, void* stream) {
    DSBT_CHECK_ARG(plan != nullptr && dst != nullptr, "dsbt_plan_get_T: NULL argument");
    DSBT_CHECK_ARG(l >= 0 && l <= plan->l_max, "dsbt_plan_get_T: l=%d out of range", l);
    if (!plan->T64) {
        set_error("dsbt_plan_get_T: plan was built without DSBT_PLAN_FP64");
        return DSBT_ERR_UNSUPPORTED;
    }
    DSBT_CUDA_TRY(cudaMemcpyAsync(dst, plan->T64 + (size_t)l * plan->nn, plan->nn * sizeof(double),
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DSBT_OK;
}

extern "C" int dsbt_plan_check(dsbt_plan* plan, double* err_out, void* stream) {
    DSBT_CHECK_ARG(plan != nullptr, "dsbt_plan_check: plan is NULL");
    if (!plan->T64) {
        set_error("dsbt_plan_check: plan was built without DSBT_PLAN_FP64");
        return DSBT_ERR_UNSUPPORTED;
    }
    const int rc = plan_probe(plan, (cudaStream_t)stream);
    if (err_out) *err_out = plan->check_err;
    return rc;
}

extern "C" int dsbt_plan_set_spin_limit(dsbt_plan* plan, unsigned polls) {
    DSBT_CHECK_ARG(plan != nullptr, "dsbt_plan_set_spin_limit: plan is NULL");
    plan->spin_limit = polls ? polls : tc_default_spin_limit();
    return DSBT_OK;
}

extern "C" int dsbt_plan_set_fast_lag(dsbt_plan* plan, int lag) {
    DSBT_CHECK_ARG(plan != nullptr, "dsbt_plan_set_fast_lag: plan is NULL");
    DSBT_CHECK_ARG(lag >= 1, "dsbt_plan_set_fast_lag: lag must be >= 1 (got %d)", lag);
    if (!plan->ftc) {
        set_error("dsbt_plan_set_fast_lag: plan was built without DSBT_PLAN_FAST_SPLIT");
        return DSBT_ERR_UNSUPPORTED;
    }
    ftc_set_lag(plan, lag);
    return DSBT_OK;
}

extern "C" int dsbt_plan_perturb_T(dsbt_plan* plan, int l, int row, int col, double delta, void* stream) {
    DSBT_CHECK_ARG(plan != nullptr, "dsbt_plan_perturb_T: plan is NULL");
    DSBT_CHECK_ARG(l >= 0 && l <= plan->l_max && row >= 0 && row < plan->N && col >= 0 && col < plan->N,
                   "dsbt_plan_perturb_T: index out of range");
    if (!plan->T64) {
        set_error("dsbt_plan_perturb_T: plan was built without DSBT_PLAN_FP64");
        return DSBT_ERR_UNSUPPORTED;
    }
    double* e = plan->T64 + (size_t)l * plan->nn + (size_t)row * plan->N + col;
    double v = 0.0;
    DSBT_CUDA_TRY(cudaMemcpyAsync(&v, e, sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DSBT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    v += delta;
    DSBT_CUDA_TRY(cudaMemcpyAsync(e, &v, sizeof(v), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    DSBT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return DSBT_OK;
}
