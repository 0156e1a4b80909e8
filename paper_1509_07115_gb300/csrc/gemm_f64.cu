// gemm_f64.cu -- FP64 contraction with the Fourier-to-Bessel factor T_l.
//
// Forward (Eq. (24)):  b[c][n] = sum_m T_l[n][m] f[c][m]
// Inverse (Eq. (25)):  f[c][m] = sum_n T_l[n][m] b[c][n]   (T^{-1} = T^T)
// T_l is lower triangular apart from its first n_extra rows (the completion
// rows of Sec. 2.5, Eq. (43)), which are dense.  Forward row tiles below the
// completion rows stop at the diagonal; inverse tiles read the completion rows
// plus the rows at and below the diagonal.
//
// Wide groups (> 8 real lines) use a 64 x 64 shared-memory tile, 4 x 4 outputs
// per thread.  Narrow groups (the TDSE case: one complex channel per l) use one
// warp per output row with coalesced row reads and a shuffle reduction, on T_l
// for the forward and on the plan's FP64 copy of T_l^T for the inverse.
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
                                                         const double2* __restrict__ phase, int per_l) {
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
    const int par = per_l ? l : (l & 1);   // phase table row: per l, or by parity
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            const int c = c0 + tx * 4 + j;
            double re = acc[i][j], im = acc[i][j + 1];
            if (phase) {   // lines (c, c+1) are the real and imaginary parts of one channel
                const double2 ph = phase[(size_t)par * N + (per_l ? r : phase_entry(l, r, N))];
                const double t = re * ph.x - im * ph.y;
                im = re * ph.y + im * ph.x;
                re = t;
            }
            if (c < nl) *out.ptr(g, gi, c, r, N) = re;
            if (c + 1 < nl) *out.ptr(g, gi, c + 1, r, N) = im;
        }
    }
}

// Narrow groups (<= kNarrow lines): one warp per output row of A = T_l
// (forward) or A = T_l^T (inverse), lanes along K with four independent loads in
// flight, shuffle reduction.  Forward rows stop at the diagonal; inverse rows read
// the completion rows (K < n_extra) and K >= the row index.  Templated on the
// largest line count NLMAX and on the caller layouts, with the line base
// pointers computed once per warp, so the inner loop is loads and FMAs only.
template <int NLMAX, bool ICPLX, bool OCPLX>
__global__ void __launch_bounds__(256) k_contract64_rows(GroupTable g, const double* __restrict__ A64,
                                                         int N, int dir, const double* __restrict__ inb,
                                                         double* __restrict__ outb,
                                                         const double2* __restrict__ phase, int per_l) {
    const int gi = blockIdx.y;
    const int nl = group_lines(g, gi);
    if (nl > kNarrow || nl == 0) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int r = (dir > 0) ? N - 1 - warp : warp;   // longest rows first
    const int l = g.l[gi];
    const int nx = n_extra(l);
    const double* row = A64 + ((size_t)l * N + r) * N;
    constexpr int XS = ICPLX ? 2 : 1;   // element stride of a line in the caller layout
    const double* xp[NLMAX];
#pragma unroll
    for (int j = 0; j < NLMAX; ++j)
        xp[j] = ICPLX ? inb + (size_t)(g.chan0[gi] + (j >> 1)) * N * 2 + (j & 1)
                      : inb + (size_t)(g.line0[gi] + j) * N;
    int s0b, s0e, s1b, s1e;   // K ranges [s0b, s0e) and [s1b, s1e)
    if (dir > 0) {
        s0b = 0; s0e = (r < nx) ? N : r + 1; s1b = s1e = 0;
    } else if (r < nx) {
        s0b = 0; s0e = N; s1b = s1e = 0;
    } else {
        s0b = 0; s0e = nx; s1b = r; s1e = N;
    }
    double acc[NLMAX];
#pragma unroll
    for (int j = 0; j < NLMAX; ++j) acc[j] = 0.0;
    for (int seg = 0; seg < 2; ++seg) {
        const int kb = seg ? s1b : s0b, ke = seg ? s1e : s0e;
        int k = kb + lane;
        for (; k + 96 < ke; k += 128) {
            double t[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) t[q] = row[k + 32 * q];
#pragma unroll
            for (int j = 0; j < NLMAX; ++j) {
                if (j < nl) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[j] = fma(t[q], xp[j][(size_t)(k + 32 * q) * XS], acc[j]);
                }
            }
        }
        for (; k < ke; k += 32) {
            const double t = row[k];
#pragma unroll
            for (int j = 0; j < NLMAX; ++j)
                if (j < nl) acc[j] = fma(t, xp[j][(size_t)k * XS], acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NLMAX; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if (lane == 0) {
        const double2 ph = phase ? (per_l ? phase[(size_t)l * N + r] : phase[(size_t)(l & 1) * N + phase_entry(l, r, N)]) : make_double2(1.0, 0.0);
#pragma unroll
        for (int j = 0; j < NLMAX; j += 2) {   // compile-time indices keep acc[] in registers
            if (j < nl) {
                double re = acc[j], im = (j + 1 < nl && j + 1 < NLMAX) ? acc[(j + 1) % NLMAX] : 0.0;
                if (phase) {
                    const double t = re * ph.x - im * ph.y;
                    im = re * ph.y + im * ph.x;
                    re = t;
                }
                double* o0 = OCPLX ? outb + ((size_t)(g.chan0[gi] + (j >> 1)) * N + r) * 2
                                   : outb + (size_t)(g.line0[gi] + j) * N + r;
                *o0 = re;
                if (j + 1 < nl) {
                    if (OCPLX) o0[1] = im;
                    else o0[N] = im;
                }
            }
        }
    }
}

template <int NLMAX>
static void launch_rows(dim3 grid, cudaStream_t st, const GroupTable& g, const double* A, int N, int dir,
                        const double* in, int in_cplx, double* out, int out_cplx, const double2* phase, int per_l) {
    if (in_cplx && out_cplx)
        k_contract64_rows<NLMAX, true, true><<<grid, 256, 0, st>>>(g, A, N, dir, in, out, phase, per_l);
    else if (in_cplx)
        k_contract64_rows<NLMAX, true, false><<<grid, 256, 0, st>>>(g, A, N, dir, in, out, phase, per_l);
    else if (out_cplx)
        k_contract64_rows<NLMAX, false, true><<<grid, 256, 0, st>>>(g, A, N, dir, in, out, phase, per_l);
    else
        k_contract64_rows<NLMAX, false, false><<<grid, 256, 0, st>>>(g, A, N, dir, in, out, phase, per_l);
}

}  // namespace

int contract_f64(const dsbt_plan* p, const GroupTable& g, int dir, const double* in, int in_cplx,
                 double* out, int out_cplx, const double2* phase, cudaStream_t st, double* fast_scratch) {
    if (!p->T64) {
        set_error("FP64 path needs a plan built with DSBT_PLAN_FP64");
        return DSBT_ERR_UNSUPPORTED;
    }
    if (dir < 0 && phase) {
        set_error("contract_f64: phase only on the forward contraction");
        return DSBT_ERR_INVALID;
    }
    if (p->fast && fast_scratch && !in_cplx && !out_cplx && g.ngroups > 0)   // planar lines: O(N l log N) path
        return contract_f64_fast(p, g, dir, in, out, phase, fast_scratch, st);
    const int N = p->N;
    const int per_l = p->knl != nullptr;   // phase table rows per l (corrected momenta) or by parity
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
        k_contract64_tile<<<grid, 256, 0, st>>>(g, p->T64, N, dir, li, lo, phase, per_l);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    if (any_narrow) {
        int nlmax = 0;
        for (int i = 0; i < g.ngroups; ++i) {
            const int nl = g.line0[i + 1] - g.line0[i];
            if (nl <= kNarrow) nlmax = max(nlmax, nl);
        }
        dim3 grid((N * 32 + 255) / 256, g.ngroups);
        const double* A = dir > 0 ? p->T64 : p->Tt64;
        ProfScope ps(kKContract64, st);
        if (nlmax <= 1) launch_rows<1>(grid, st, g, A, N, dir, in, in_cplx, out, out_cplx, phase, per_l);
        else if (nlmax <= 2) launch_rows<2>(grid, st, g, A, N, dir, in, in_cplx, out, out_cplx, phase, per_l);
        else if (nlmax <= 4) launch_rows<4>(grid, st, g, A, N, dir, in, in_cplx, out, out_cplx, phase, per_l);
        else launch_rows<8>(grid, st, g, A, N, dir, in, in_cplx, out, out_cplx, phase, per_l);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    return DSBT_OK;
}

}  // namespace dsbt
