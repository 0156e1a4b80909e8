// gemm_f64.cu -- FP64 contraction with the Fourier-to-Bessel factor T_l.
//
// Forward (Eq. (24)):  b[c][n] = sum_m T_l[n][m] f[c][m]
// Inverse (Eq. (25)):  f[c][m] = sum_n T_l[n][m] b[c][n]   (T^{-1} = T^T)
// T_l is lower triangular apart from its first n_extra rows (the completion
// rows of Sec. 2.5, Eq. (43)), which are dense.  Forward row tiles below the
// completion rows stop at the diagonal; inverse tiles read the completion rows
// plus the rows at and below the diagonal.
//
// Wide groups (>= 16 real lines) use a 64 x 64 shared-memory tile, 4 x 4 outputs
// per thread.  Narrow groups (the TDSE case: one complex channel per l) use one
// warp per output row (forward, coalesced row reads and a shuffle reduction) or
// one thread per output column (inverse, coalesced column reads).
#include "plan.cuh"

namespace dsbt {

namespace {

constexpr int BM = 64, BC = 64, BK = 16;
constexpr int kNarrow = 8;   // groups with at most this many lines use the narrow kernel

struct Lines {
    const double* base;
    int cplx;   // interleaved user complex layout
    __device__ __forceinline__ const double* ptr(const GroupTable& g, int gi, int j, int k, int N) const {
        if (cplx) return base + ((size_t)(g.chan0[gi] + (j >> 1)) * N + k) * 2 + (j & 1);
        return base + (size_t)(g.line0[gi] + j) * N + k;
    }
};

struct OutLines {
    double* base;
    int cplx;
    __device__ __forceinline__ double* ptr(const GroupTable& g, int gi, int j, int k, int N) const {
        if (cplx) return base + ((size_t)(g.chan0[gi] + (j >> 1)) * N + k) * 2 + (j & 1);
        return base + (size_t)(g.line0[gi] + j) * N + k;
    }
};

__device__ __forceinline__ int group_lines(const GroupTable& g, int gi) {
    return g.line0[gi + 1] - g.line0[gi];
}

// K-block ranges of a tile of output rows [r0, r0 + rows): returns up to two
// half-open ranges in units of BK.
__device__ __forceinline__ void k_ranges(int dir, int r0, int rows, int nx, int N, int& a0, int& a1,
                                         int& b0, int& b1) {
    const int KB = N / BK;
    if (dir > 0) {
        a0 = 0;
        a1 = (r0 < nx) ? KB : min(KB, (r0 + rows + BK - 1) / BK);
        b0 = b1 = 0;
    } else {
        a0 = 0;
        a1 = (nx + BK - 1) / BK;
        b0 = max(a1, r0 / BK);
        b1 = KB;
        if (r0 < nx || a1 >= b0) { a1 = KB; b0 = b1 = 0; }
    }
}

__global__ void __launch_bounds__(256) k_contract64_tile(GroupTable g, const double* __restrict__ T64,
                                                         int N, int dir, Lines in, OutLines out,
                                                         const double2* __restrict__ phase) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BC + 1];
    const int gi = blockIdx.y;
    const int nl = group_lines(g, gi);
    if (nl <= kNarrow) return;
    const int CT = (nl + BC - 1) / BC;
    const int RT = N / BM;
    if ((int)blockIdx.x >= RT * CT) return;
    // heavy row tiles first: forward cost grows with the row index, inverse shrinks
    int rt = blockIdx.x / CT;
    const int ct = blockIdx.x % CT;
    if (dir > 0) rt = RT - 1 - rt;
    const int l = g.l[gi];
    const int nx = n_extra(l);
    const double* T = T64 + (size_t)l * N * N;
    const int r0 = rt * BM, c0 = ct * BC;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    int a0, a1, b0, b1;
    k_ranges(dir, r0, BM, nx, N, a0, a1, b0, b1);
    for (int seg = 0; seg < 2; ++seg) {
        const int kb0 = seg ? b0 : a0, kb1 = seg ? b1 : a1;
        for (int kb = kb0; kb < kb1; ++kb) {
            const int k0 = kb * BK;
            // A tile: As[kk][i] = A[r0+i][k0+kk], A = T (forward) or T^T (inverse)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = tid + t * 256;
                if (dir > 0) {
                    const int kk = e & 15, i = e >> 4;
                    As[kk][i] = T[(size_t)(r0 + i) * N + k0 + kk];
                } else {
                    const int i = e & 63, kk = e >> 6;
                    As[kk][i] = T[(size_t)(k0 + kk) * N + r0 + i];
                }
            }
            // B tile: Bs[kk][j] = line (c0 + j) at k0 + kk
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = tid + t * 256;
                const int kk = e & 15, j = e >> 4;
                const int c = c0 + j;
                Bs[kk][j] = (c < nl) ? *in.ptr(g, gi, c, k0 + kk, N) : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
    const int par = l & 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            const int c = c0 + tx * 4 + j;
            double re = acc[i][j], im = acc[i][j + 1];
            if (phase) {   // lines (c, c+1) are the real and imaginary parts of one channel
                const double2 ph = phase[(size_t)par * N + r];
                const double t = re * ph.x - im * ph.y;
                im = re * ph.y + im * ph.x;
                re = t;
            }
            if (c < nl) *out.ptr(g, gi, c, r, N) = re;
            if (c + 1 < nl) *out.ptr(g, gi, c + 1, r, N) = im;
        }
    }
}

// Narrow forward: one warp per output row n, up to kNarrow lines.
__global__ void __launch_bounds__(256) k_contract64_rows(GroupTable g, const double* __restrict__ T64,
                                                         int N, Lines in, OutLines out,
                                                         const double2* __restrict__ phase) {
    const int gi = blockIdx.y;
    const int nl = group_lines(g, gi);
    if (nl > kNarrow) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= N || nl == 0) return;
    const int r = N - 1 - warp;   // longest rows first
    const int l = g.l[gi];
    const int nx = n_extra(l);
    const double* row = T64 + ((size_t)l * N + r) * N;
    const int kend = (r < nx) ? N : r + 1;
    double acc[kNarrow];
#pragma unroll
    for (int j = 0; j < kNarrow; ++j) acc[j] = 0.0;
    for (int k = lane; k < kend; k += 32) {
        const double t = row[k];
#pragma unroll
        for (int j = 0; j < kNarrow; ++j)
            if (j < nl) acc[j] = fma(t, *in.ptr(g, gi, j, k, N), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < kNarrow; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if (lane == 0) {
        const double2 ph = phase ? phase[(size_t)(l & 1) * N + r] : make_double2(1.0, 0.0);
        for (int j = 0; j < nl; j += 2) {
            double re = acc[j], im = (j + 1 < nl) ? acc[j + 1] : 0.0;
            if (phase) {
                const double t = re * ph.x - im * ph.y;
                im = re * ph.y + im * ph.x;
                re = t;
            }
            *out.ptr(g, gi, j, r, N) = re;
            if (j + 1 < nl) *out.ptr(g, gi, j + 1, r, N) = im;
        }
    }
}

// Narrow inverse: one thread per output column m.
__global__ void __launch_bounds__(256) k_contract64_cols(GroupTable g, const double* __restrict__ T64,
                                                         int N, Lines in, OutLines out) {
    const int gi = blockIdx.y;
    const int nl = group_lines(g, gi);
    if (nl > kNarrow) return;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N || nl == 0) return;
    const int l = g.l[gi];
    const int nx = n_extra(l);
    const double* T = T64 + (size_t)l * N * N;
    double acc[kNarrow];
#pragma unroll
    for (int j = 0; j < kNarrow; ++j) acc[j] = 0.0;
    for (int seg = 0; seg < 2; ++seg) {
        const int n_beg = seg ? max(m, nx) : 0, n_end = seg ? N : min(nx, N);
        for (int n = n_beg; n < n_end; ++n) {
            const double t = T[(size_t)n * N + m];
#pragma unroll
            for (int j = 0; j < kNarrow; ++j)
                if (j < nl) acc[j] = fma(t, *in.ptr(g, gi, j, n, N), acc[j]);
        }
    }
    for (int j = 0; j < nl; ++j) *out.ptr(g, gi, j, m, N) = acc[j];
}

}  // namespace

int contract_f64(const dsbt_plan* p, const GroupTable& g, int dir, const double* in, int in_cplx,
                 double* out, int out_cplx, const double2* phase, cudaStream_t st) {
    if (!p->T64) {
        set_error("FP64 path needs a plan built with DSBT_PLAN_FP64");
        return DSBT_ERR_UNSUPPORTED;
    }
    if (dir < 0 && phase) {
        set_error("contract_f64: phase only on the forward contraction");
        return DSBT_ERR_INVALID;
    }
    const int N = p->N;
    int max_ct = 0, any_wide = 0, any_narrow = 0;
    for (int i = 0; i < g.ngroups; ++i) {
        const int nl = g.line0[i + 1] - g.line0[i];
        if (nl > kNarrow) {
            any_wide = 1;
            max_ct = max(max_ct, (nl + BC - 1) / BC);
        } else if (nl > 0) {
            any_narrow = 1;
        }
    }
    if (g.ngroups == 0) return DSBT_OK;
    Lines li{in, in_cplx};
    OutLines lo{out, out_cplx};
    if (any_wide) {
        dim3 grid((N / BM) * max_ct, g.ngroups);
        ProfScope ps(kKContract64, st);
        k_contract64_tile<<<grid, 256, 0, st>>>(g, p->T64, N, dir, li, lo, phase);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    if (any_narrow) {
        if (dir > 0) {
            dim3 grid((N * 32 + 255) / 256, g.ngroups);
            ProfScope ps(kKContract64, st);
            k_contract64_rows<<<grid, 256, 0, st>>>(g, p->T64, N, li, lo, phase);
        } else {
            dim3 grid((N + 255) / 256, g.ngroups);
            ProfScope ps(kKContract64, st);
            k_contract64_cols<<<grid, 256, 0, st>>>(g, p->T64, N, li, lo);
        }
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    return DSBT_OK;
}

}  // namespace dsbt
