// fast64.cu -- FP64 multiplication by T_l and T_l^T in O(N l log N) work,
// for plans built with DSBT_PLAN_FAST64 (the stable counterpart of the fast
// scheme of Sec. 2.6).
//
// On a regular row n of T_l the entries left of the diagonal are
// T_nm = alpha_n P'_l(n - m, 2n) sqrt(w_m): a polynomial of degree l - 1 in m
// times sqrt(w_m) (w_0 = 1/2 for odd l).  Columns are cut into leaves of B = 64
// points and a binary tree of intervals above them.  Row r (leaf J = r / B)
// takes its own leaf's columns up to the diagonal directly (near field) and
// every other column through the intervals of the dyadic decomposition of
// leaves 0..J-1 (one interval per set bit j of J, index (J >> j) - 1): on such
// an interval I of length L_j = B 2^j the row is exactly
//     T_{r,I} = sqrt(w_I) (Q_j beta_{r,j}),
// with Q_j an orthonormal basis [L_j][K] of the polynomials of degree < K on
// the interval's points (K = the plan's l_max; the first l columns suffice for
// T_l), beta_{r,j} = Q_j^T (T_{r,I} / sqrt(w_I)) computed from the FP64 T_l at
// plan creation.  Forward: moments M_I = Q_j^T (sqrt(w) f)_I per line, leaves
// first, then parents from children through the K x K transfer matrices
// A_{j,h} = Q_{j-1}^T Q_j[half h] (the parent basis restricted to a child is a
// polynomial of degree < K there); b_r = near + sum_j beta_{r,j} . M.
// Inverse: W_I = sum_{r using I} beta_{r,j} b_r, pushed down the tree through
// the same A, f_c = sqrt(w_c) (Q_0 W_leaf)_c + near + completion rows.  The
// completion rows (n < n0_l) are dense and applied directly.  The bases are
// built on the host by Arnoldi on the point grid with two Gram-Schmidt passes,
// so every coefficient is a bounded projection (no monomial cancellation).
#include <math.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "plan.cuh"

namespace dsbt {

namespace {

constexpr int FB = 64;    // leaf size
constexpr int KM = 64;    // basis width stored (>= l_max)

__host__ __device__ inline double sqrt_w(int l, int c) { return ((l & 1) && c == 0) ? 0.70710678118654752440 : 1.0; }

// Orthonormal polynomial basis Q[t][k], t < len, k < KM, on x_t = (2t+1)/len - 1.
void basis(int len, std::vector<double>& Q) {
    const int K = std::min(KM, len);
    Q.assign((size_t)len * KM, 0.0);
    std::vector<double> v(len), x(len);
    for (int t = 0; t < len; ++t) x[t] = (2.0 * t + 1.0) / len - 1.0;
    for (int t = 0; t < len; ++t) Q[(size_t)t * KM] = 1.0 / sqrt((double)len);
    for (int k = 1; k < K; ++k) {
        for (int t = 0; t < len; ++t) v[t] = x[t] * Q[(size_t)t * KM + k - 1];
        for (int pass = 0; pass < 2; ++pass)
            for (int q = 0; q < k; ++q) {
                double d = 0.0;
                for (int t = 0; t < len; ++t) d += v[t] * Q[(size_t)t * KM + q];
                for (int t = 0; t < len; ++t) v[t] -= d * Q[(size_t)t * KM + q];
            }
        double nrm = 0.0;
        for (int t = 0; t < len; ++t) nrm += v[t] * v[t];
        nrm = 1.0 / sqrt(nrm);
        for (int t = 0; t < len; ++t) Q[(size_t)t * KM + k] = v[t] * nrm;
    }
}

// beta[l][j][r][k]: projection of row r of T_l on level j's interval of its
// decomposition (zero where unused).  Block: KM threads (k); grid (r, j, l).
__global__ void k_fast_beta(const double* __restrict__ T64, const double* __restrict__ Q,
                            const size_t* __restrict__ qoff, double* __restrict__ beta, int N, int levels) {
    const int r = blockIdx.x, j = blockIdx.y, l = blockIdx.z, k = threadIdx.x;
    const int J = r / FB;
    double s = 0.0;
    if (r >= n_extra(l) && ((J >> j) & 1) && k < l) {
        const int len = FB << j;
        const int lo = ((J >> j) - 1) * len;
        const double* row = T64 + ((size_t)l * N + r) * N + lo;
        const double* Qj = Q + qoff[j];
        for (int t = 0; t < len; ++t) s = fma(row[t] / sqrt_w(l, lo + t), Qj[(size_t)t * KM + k], s);
    }
    beta[(((size_t)l * levels + j) * N + r) * KM + k] = s;
}

struct FastArgs {
    const double* Q;       // all levels, [len_j][KM] at qoff[j]
    const size_t* qoff;
    const double* A;       // [levels][2][KM][KM] (level 0 unused)
    const double* beta;    // [L][levels][N][KM]
    const double* T64;
    int N, nleaf, levels, R;
};

__device__ __forceinline__ size_t mpos(const FastArgs& a, int j, int i, int line, int k) {
    // scratch layout: level j block at sum_{j' < j} (nleaf >> j') R KM
    size_t off = 0;
    for (int q = 0; q < j; ++q) off += (size_t)(a.nleaf >> q) * a.R * KM;
    return off + ((size_t)i * a.R + line) * KM + k;
}

// Leaf moments M_0[leaf][line][k] = sum_t Q_0[t][k] sqrt(w) f[line][leaf B + t].
__global__ void k_fast_leaf_moments(FastArgs a, GroupTable g, const double* __restrict__ in, double* M) {
    const int leaf = blockIdx.x, gi = blockIdx.y;
    const int l = g.l[gi], K = l, line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const double* Q0 = a.Q + a.qoff[0];
    for (int p = threadIdx.x; p < nl * K; p += blockDim.x) {
        const int line = p / K, k = p % K;
        const double* x = in + (size_t)(line0 + line) * a.N + leaf * FB;
        double s = 0.0;
        for (int t = 0; t < FB; ++t) s = fma(Q0[(size_t)t * KM + k], sqrt_w(l, leaf * FB + t) * x[t], s);
        M[mpos(a, 0, leaf, line0 + line, k)] = s;
    }
}

// Parent moments from children: M_j[i][k] = sum_k' (M_{j-1}[2i][k'] A0[k'][k] + M_{j-1}[2i+1][k'] A1[k'][k]).
__global__ void k_fast_merge(FastArgs a, GroupTable g, int j, double* M) {
    const int i = blockIdx.x, gi = blockIdx.y;
    const int K = g.l[gi], line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const double* A0 = a.A + ((size_t)j * 2 + 0) * KM * KM;
    const double* A1 = a.A + ((size_t)j * 2 + 1) * KM * KM;
    for (int p = threadIdx.x; p < nl * K; p += blockDim.x) {
        const int line = line0 + p / K, k = p % K;
        const double* c0 = M + mpos(a, j - 1, 2 * i, line, 0);
        const double* c1 = M + mpos(a, j - 1, 2 * i + 1, line, 0);
        double s = 0.0;
        for (int q = 0; q < K; ++q) s = fma(c0[q], A0[(size_t)q * KM + k], fma(c1[q], A1[(size_t)q * KM + k], s));
        M[mpos(a, j, i, line, k)] = s;
    }
}

// b[line][r] = completion rows densely; regular rows: near field + far field;
// optional kinetic phase on the (re, im) line pairs.  One thread per row.
__global__ void __launch_bounds__(128) k_fast_eval(FastArgs a, GroupTable g, const double* __restrict__ in,
                                                   const double* __restrict__ M, double* __restrict__ out,
                                                   const double2* __restrict__ phase, int per_l) {
    const int gi = blockIdx.y;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = g.l[gi], K = l, line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const int N = a.N;
    if (r >= N) return;
    const double* Trow = a.T64 + ((size_t)l * N + r) * N;
    const int J = r / FB, ne = n_extra(l);
    double2 ph = make_double2(1.0, 0.0);
    if (phase) ph = per_l ? phase[(size_t)l * N + r] : phase[(size_t)(l & 1) * N + phase_entry(l, r, N)];
    for (int line = 0; line < nl; line += (phase ? 2 : 1)) {
        double acc[2] = {0.0, 0.0};
        const int np = phase ? 2 : 1;
        for (int h = 0; h < np; ++h) {
            const double* x = in + (size_t)(line0 + line + h) * N;
            double s = 0.0;
            if (r < ne) {
                for (int c = 0; c < N; ++c) s = fma(Trow[c], x[c], s);
            } else {
                for (int c = J * FB; c <= r; ++c) s = fma(Trow[c], x[c], s);
                for (int j = 0; j < a.levels; ++j) {
                    if (!((J >> j) & 1)) continue;
                    const int i = (J >> j) - 1;
                    const double* be = a.beta + (((size_t)l * a.levels + j) * N + r) * KM;
                    const double* m = M + mpos(a, j, i, line0 + line + h, 0);
                    for (int k = 0; k < K; ++k) s = fma(be[k], m[k], s);
                }
            }
            acc[h] = s;
        }
        if (phase) {
            const double re = acc[0] * ph.x - acc[1] * ph.y, im = acc[0] * ph.y + acc[1] * ph.x;
            out[(size_t)(line0 + line) * N + r] = re;
            out[(size_t)(line0 + line + 1) * N + r] = im;
        } else {
            out[(size_t)(line0 + line) * N + r] = acc[0];
        }
    }
}

// W_j[i][line][k] = sum over the rows of interval i's right sibling (regular
// rows only) of beta_{r,j}[k] b[line][r]; intervals whose sibling is missing
// or that no row uses stay zero.  Grid (interval slot, group), all levels.
__global__ void k_fast_w(FastArgs a, GroupTable g, const double* __restrict__ in, double* W) {
    int slot = blockIdx.x, j = 0;
    while (j < a.levels && slot >= (a.nleaf >> j)) { slot -= a.nleaf >> j; ++j; }
    const int i = slot, gi = blockIdx.y;
    const int l = g.l[gi], K = l, line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const int N = a.N, len = FB << j;
    const bool used = (i & 1) == 0 && (i + 1) < (a.nleaf >> j);
    const int r0 = max((i + 1) * len, n_extra(l)), r1 = min((i + 2) * len, N);
    for (int p = threadIdx.x; p < nl * K; p += blockDim.x) {
        const int line = line0 + p / K, k = p % K;
        double s = 0.0;
        if (used) {
            const double* x = in + (size_t)line * N;
            const double* be = a.beta + (((size_t)l * a.levels + j) * N) * KM + k;
            for (int r = r0; r < r1; ++r) s = fma(be[(size_t)r * KM], x[r], s);
        }
        W[mpos(a, j, i, line, k)] = s;
    }
}

// Push W from level j to level j-1: W_{j-1}[2i+h][k'] += sum_k A_h[k'][k] W_j[i][k].
__global__ void k_fast_push(FastArgs a, GroupTable g, int j, double* W) {
    const int i = blockIdx.x, gi = blockIdx.y;
    const int K = g.l[gi], line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    for (int p = threadIdx.x; p < 2 * nl * K; p += blockDim.x) {
        const int h = p / (nl * K), rest = p % (nl * K);
        const int line = line0 + rest / K, kq = rest % K;
        const double* Ah = a.A + ((size_t)j * 2 + h) * KM * KM + (size_t)kq * KM;
        const double* w = W + mpos(a, j, i, line, 0);
        double s = 0.0;
        for (int k = 0; k < K; ++k) s = fma(Ah[k], w[k], s);
        W[mpos(a, j - 1, 2 * i + h, line, kq)] += s;
    }
}

// f[line][c] = sqrt(w_c) (Q_0 W_leaf)_c + near field (rows of c's leaf at or
// below the diagonal) + completion rows.  One thread per column.
__global__ void __launch_bounds__(128) k_fast_leaf_out(FastArgs a, GroupTable g, const double* __restrict__ in,
                                                       const double* __restrict__ W, double* __restrict__ out) {
    const int gi = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = g.l[gi], K = l, line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const int N = a.N;
    if (c >= N) return;
    const double* T = a.T64 + (size_t)l * N * N;
    const int leaf = c / FB, ne = n_extra(l);
    const double* Q0 = a.Q + a.qoff[0] + (size_t)(c - leaf * FB) * KM;
    const double sw = sqrt_w(l, c);
    const int r_lo = max(c, ne), r_hi = min((leaf + 1) * FB, N);
    for (int line = 0; line < nl; ++line) {
        const double* x = in + (size_t)(line0 + line) * N;
        double s = 0.0;
        for (int r = 0; r < ne; ++r) s = fma(T[(size_t)r * N + c], x[r], s);
        for (int r = r_lo; r < r_hi; ++r) s = fma(T[(size_t)r * N + c], x[r], s);
        const double* w = W + mpos(a, 0, leaf, line0 + line, 0);
        double f = 0.0;
        for (int k = 0; k < K; ++k) f = fma(Q0[k], w[k], f);
        out[(size_t)(line0 + line) * N + c] = s + sw * f;
    }
}

}  // namespace

struct FastData {
    int nleaf = 0, levels = 0;
    double* Q = nullptr;
    size_t* qoff = nullptr;
    double* A = nullptr;
    double* beta = nullptr;
};

bool fast_supported(int N) {
    const int nleaf = N / FB;
    return N % FB == 0 && nleaf >= 2 && (nleaf & (nleaf - 1)) == 0;
}

int fast_build(dsbt_plan* p, cudaStream_t st) {
    const int N = p->N;
    DSBT_CHECK_ARG(fast_supported(N), "DSBT_PLAN_FAST64 needs N / 64 a power of two (N = %d)", N);
    DSBT_CHECK_ARG(p->l_max <= KM, "DSBT_PLAN_FAST64: l_max %d above %d", p->l_max, KM);
    FastData* f = new (std::nothrow) FastData();
    if (!f) return DSBT_ERR_NOMEM;
    p->fast = f;
    f->nleaf = N / FB;
    f->levels = 0;
    while ((1 << f->levels) < f->nleaf) ++f->levels;   // levels j = 0 .. levels-1, intervals up to N / 2
    const int levels = f->levels;
    // bases (host, threads over levels) and transfer matrices
    std::vector<std::vector<double>> Qh(levels);
    std::vector<std::thread> pool;
    for (int j = 0; j < levels; ++j) pool.emplace_back([&, j]() { basis(FB << j, Qh[j]); });
    for (auto& t : pool) t.join();
    std::vector<size_t> qoff(levels);
    size_t qtot = 0;
    for (int j = 0; j < levels; ++j) {
        qoff[j] = qtot;
        qtot += Qh[j].size();
    }
    std::vector<double> Qall(qtot), Ah((size_t)levels * 2 * KM * KM, 0.0);
    for (int j = 0; j < levels; ++j) std::copy(Qh[j].begin(), Qh[j].end(), Qall.begin() + qoff[j]);
    for (int j = 1; j < levels; ++j) {
        const int half = FB << (j - 1);
        for (int h = 0; h < 2; ++h)
            for (int q = 0; q < KM; ++q)
                for (int k = 0; k < KM; ++k) {
                    double s = 0.0;
                    for (int t = 0; t < half; ++t) s += Qh[j - 1][(size_t)t * KM + q] * Qh[j][(size_t)(h * half + t) * KM + k];
                    Ah[(((size_t)j * 2 + h) * KM + q) * KM + k] = s;
                }
    }
    const size_t L = (size_t)p->l_max + 1;
    bool ok = cudaMalloc((void**)&f->Q, qtot * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&f->qoff, levels * sizeof(size_t)) == cudaSuccess &&
              cudaMalloc((void**)&f->A, Ah.size() * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&f->beta, L * levels * N * KM * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMemcpy(f->Q, Qall.data(), qtot * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(f->qoff, qoff.data(), levels * sizeof(size_t), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(f->A, Ah.data(), Ah.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        set_error("DSBT_PLAN_FAST64: device allocation or copy failed");
        return DSBT_ERR_NOMEM;
    }
    dim3 grid(N, levels, (unsigned)L);
    k_fast_beta<<<grid, KM, 0, st>>>(p->T64, f->Q, f->qoff, f->beta, N, levels);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

void fast_free(dsbt_plan* p) {
    if (!p || !p->fast) return;
    cudaFree(p->fast->Q);
    cudaFree(p->fast->qoff);
    cudaFree(p->fast->A);
    cudaFree(p->fast->beta);
    delete p->fast;
    p->fast = nullptr;
}

size_t fast_scratch_bytes(const dsbt_plan* p, int lines) {
    if (!p->fast) return 0;
    size_t n = 0;
    for (int j = 0; j < p->fast->levels; ++j) n += (size_t)(p->fast->nleaf >> j) * lines * KM;
    return n * sizeof(double);
}

int contract_f64_fast(const dsbt_plan* p, const GroupTable& g, int dir, const double* in, double* out,
                      const double2* phase, double* scratch, cudaStream_t st) {
    const FastData* f = p->fast;
    FastArgs a{f->Q, f->qoff, f->A, f->beta, p->T64, p->N, f->nleaf, f->levels, g.total_lines};
    const int per_l = p->knl != nullptr;
    const unsigned gy = (unsigned)g.ngroups;
    ProfScope ps(kKContract64, st);
    if (dir > 0) {
        k_fast_leaf_moments<<<dim3(f->nleaf, gy), 256, 0, st>>>(a, g, in, scratch);
        for (int j = 1; j < f->levels; ++j) k_fast_merge<<<dim3(f->nleaf >> j, gy), 256, 0, st>>>(a, g, j, scratch);
        k_fast_eval<<<dim3((p->N + 127) / 128, gy), 128, 0, st>>>(a, g, in, scratch, out, phase, per_l);
    } else {
        int slots = 0;
        for (int j = 0; j < f->levels; ++j) slots += f->nleaf >> j;
        k_fast_w<<<dim3(slots, gy), 256, 0, st>>>(a, g, in, scratch);
        for (int j = f->levels - 1; j >= 1; --j) k_fast_push<<<dim3(f->nleaf >> j, gy), 256, 0, st>>>(a, g, j, scratch);
        k_fast_leaf_out<<<dim3((p->N + 127) / 128, gy), 128, 0, st>>>(a, g, in, scratch, out);
    }
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

}  // namespace dsbt
