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
// plan creation.  Forward: moments M_I = Q_j^T (sqrt(w) f)_I of every used
// interval (one with a right sibling), projected directly from f, then
// b_r = near + sum_j beta_{r,j} . M.  Inverse: W_I = sum_{r using I}
// beta_{r,j} b_r, then f_c = sqrt(w_c) sum_j (Q_j W_{I_j(c)})_c + near, over
// the used intervals I_j(c) holding c.  Direct projection costs about as many
// multiply-adds as the leaf-to-root merge through K x K transfer matrices
// would for K near 64, and has no chain of dependent levels.  The completion
// rows (n < n0_l) are dense and applied directly.  The bases are built on the
// host by Arnoldi on the point grid with two Gram-Schmidt passes, so every
// coefficient is a bounded projection (no monomial cancellation).
//
// On this part FP64 multiply-adds are the bound (a few per clock per SM), so
// the kernels keep every lane on useful multiply-adds: lanes run over rows or
// columns with the basis index k in the loop, and the few reductions across
// lanes are shuffles over row chunks.
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
    const double* QT;      // all levels, [KM][len_j] at qoff[j]
    const size_t* qoff;
    const double* beta;    // [L][levels][N][KM]
    const double* betaT;   // [L][levels][KM][N]
    const double* nearT;   // [L][nleaf][FB][FB]: nearT[l][J][c][t] = T_l[J B + t][J B + c]
    const double* T64;
    int N, nleaf, levels, R;
};

__device__ __forceinline__ size_t mpos(const FastArgs& a, int j, int i, int line, int k) {
    // scratch layout: level j block at sum_{j' < j} (nleaf >> j') R KM
    size_t off = 0;
    for (int q = 0; q < j; ++q) off += (size_t)(a.nleaf >> q) * a.R * KM;
    return off + ((size_t)i * a.R + line) * KM + k;
}

// Groups are ordered by l, and the work of a block grows with l.  Projection
// blocks take their group through this interleaving (0, n-1, 1, n-2, ...) so
// that every run of consecutive blocks mixes light and heavy groups.
__device__ __forceinline__ int interleave(int t, int n) { return (t & 1) ? n - 1 - (t >> 1) : (t >> 1); }

constexpr int PROJ_THREADS = 256;

// Interval i of level j is used when its right sibling exists (i even): the
// rows of the sibling take it as a far interval.  Level j has nleaf >> (j+1)
// used intervals, its rows are cut into nch_j <= 32 chunks, and a block takes
// PROJ_THREADS / nch_j (line, k) pairs.  Blocks run over (level, tile, interval,
// group), largest intervals first.
__device__ __forceinline__ int proj_chunks(int j) { return min(32, 1 << j); }

__device__ __forceinline__ bool proj_block(const FastArgs& a, int ngroups, int pmax, int b, int& j, int& gi,
                                           int& i, int& tile) {
    for (j = a.levels - 1; j >= 0; --j) {
        const int used = a.nleaf >> (j + 1);
        const int per = PROJ_THREADS / proj_chunks(j);
        const int count = used * ngroups * ((pmax + per - 1) / per);
        if (b < count) {
            gi = interleave(b % ngroups, ngroups);
            b /= ngroups;
            i = 2 * (b % used);
            tile = b / used;
            return true;
        }
        b -= count;
    }
    return false;
}

// Projections onto the bases of the used intervals:
//   forward (dir > 0): M_j[i][line][k] = sum_{t in I} Q_j[t][k] sqrt(w_t) f[line][t]
//   inverse (dir < 0): W_j[i][line][k] = sum_{r in sibling} beta_{r,j}[k] b[line][r]
// over the (line, k) pairs p = line K + k of a group (beta is zero on
// completion rows, so those rows drop out).  Both operands are [row][KM].
// Lane = (pair, chunk): a lane sums one chunk of len / nch rows, then the nch
// lanes of a pair add their sums by shuffles.
__global__ void __launch_bounds__(PROJ_THREADS) k_fast_project(FastArgs a, GroupTable g, int dir, int pmax,
                                                               const double* __restrict__ in,
                                                               double* __restrict__ out) {
    int j, gi, i, tile;
    if (!proj_block(a, g.ngroups, pmax, blockIdx.x, j, gi, i, tile)) return;
    const int l = g.l[gi], K = l, line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const int P = nl * K;
    const int nch = proj_chunks(j), ppw = 32 / nch;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pw = (tile * (PROJ_THREADS / 32) + warp) * ppw;   // first pair of the warp
    if (pw >= P) return;                                          // whole warp idle
    const int q = lane & (nch - 1), pq = pw + lane / nch;
    const int N = a.N, len = FB << j, clen = len / nch;
    const int t0 = dir > 0 ? i * len : (i + 1) * len;
    double acc = 0.0;
    if (pq < P) {
        const int line = pq / K, k = pq % K;
        const double* x = in + (size_t)(line0 + line) * N + t0 + q * clen;
        const double* o = (dir > 0 ? a.Q + a.qoff[j] : a.beta + (((size_t)l * a.levels + j) * N + t0) * KM) +
                          (size_t)q * clen * KM + k;
        const double x0 = (dir > 0 && t0 + q * clen == 0) ? sqrt_w(l, 0) * x[0] : x[0];
        acc = o[0] * x0;
#pragma unroll 8
        for (int t = 1; t < clen; ++t) acc = fma(o[(size_t)t * KM], x[t], acc);
    }
    for (int s = nch >> 1; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    if (q == 0 && pq < P) out[mpos(a, j, i, line0 + pq / K, pq % K)] = acc;
}

__device__ __forceinline__ void store_pair(double* out, size_t o0, int N, double s0, double s1, bool two,
                                           const double2* phase, double2 ph) {
    if (phase) {
        out[o0] = s0 * ph.x - s1 * ph.y;
        out[o0 + N] = s0 * ph.y + s1 * ph.x;
    } else {
        out[o0] = s0;
        if (two) out[o0 + N] = s1;
    }
}

// Forward output, lines in pairs (with a kinetic phase the pairs are the
// (re, im) lines of a channel).  blockIdx.x < nleaf: leaf J, one thread per
// regular row r = J B + t: near field sum_{c <= r in J} T_rc f_c from the
// transposed leaf block, far field sum_j beta_{r,j} . M_j over the set bits j
// of J.  blockIdx.x >= nleaf: completion rows, one warp per row (dense dot).
__global__ void __launch_bounds__(FB) k_fast_eval(FastArgs a, GroupTable g, const double* __restrict__ in,
                                                  const double* __restrict__ M, double* __restrict__ out,
                                                  const double2* __restrict__ phase, int per_l) {
    const int gi = gridDim.y - 1 - blockIdx.y, xb = blockIdx.x;   // largest l first
    const int l = g.l[gi], K = l, line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const int N = a.N, ne = n_extra(l);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (xb >= a.nleaf) {
        const int r = (xb - a.nleaf) * (FB / 32) + w;
        if (r >= ne) return;
        const double* Trow = a.T64 + ((size_t)l * N + r) * N;
        double2 ph = make_double2(1.0, 0.0);
        if (phase) ph = per_l ? phase[(size_t)l * N + r] : phase[(size_t)(l & 1) * N + phase_entry(l, r, N)];
        for (int line = 0; line < nl; line += 2) {
            const bool two = line + 1 < nl;
            const double* x0 = in + (size_t)(line0 + line) * N;
            const double* x1 = two ? x0 + N : x0;
            double s0 = 0.0, s1 = 0.0;
            for (int c = lane; c < N; c += 32) {
                const double t = Trow[c];
                s0 = fma(t, x0[c], s0);
                s1 = fma(t, x1[c], s1);
            }
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (lane == 0) store_pair(out, (size_t)(line0 + line) * N + r, N, s0, s1, two, phase, ph);
        }
        return;
    }
    const int J = xb, r = J * FB + threadIdx.x;
    if (J * FB + w * 32 + 31 < ne) return;   // the whole warp holds completion rows
    const double* nt = a.nearT + (((size_t)l * a.nleaf + J) * FB) * FB + threadIdx.x;
    const int cmax = (w + 1) * 32;           // T_rc = 0 for c > r
    double2 ph = make_double2(1.0, 0.0);
    if (phase) ph = per_l ? phase[(size_t)l * N + r] : phase[(size_t)(l & 1) * N + phase_entry(l, r, N)];
    for (int line = 0; line < nl; line += 2) {
        const bool two = line + 1 < nl;
        const double* x0 = in + (size_t)(line0 + line) * N + J * FB;
        const double* x1 = two ? x0 + N : x0;
        double s0 = 0.0, s1 = 0.0;
        for (int c = 0; c < cmax; ++c) {
            const double t = nt[(size_t)c * FB];
            s0 = fma(t, x0[c], s0);
            s1 = fma(t, x1[c], s1);
        }
        for (int j = 0; j < a.levels; ++j) {
            if (!((J >> j) & 1)) continue;
            const int i = (J >> j) - 1;
            const double* be = a.betaT + (((size_t)l * a.levels + j) * KM) * N + r;
            const double* m0 = M + mpos(a, j, i, line0 + line, 0);
            const double* m1 = two ? m0 + KM : m0;
            for (int k = 0; k < K; ++k) {
                const double b = be[(size_t)k * N];
                s0 = fma(b, m0[k], s0);
                s1 = fma(b, m1[k], s1);
            }
        }
        if (r >= ne) store_pair(out, (size_t)(line0 + line) * N + r, N, s0, s1, two, phase, ph);
    }
}

// Inverse output f = T^T b, one thread per column c of leaf J = blockIdx.x:
// completion rows (dense), near field sum_{r >= c in J} T_rc b_r (T_rc = 0 for
// r < c, so a warp starts at its first column), far field
// sqrt(w_c) sum_j (Q_j W_j[i])_c over the levels j whose interval i holding c
// is used.
__global__ void __launch_bounds__(FB) k_fast_leaf_out(FastArgs a, GroupTable g, const double* __restrict__ in,
                                                      const double* __restrict__ W, double* __restrict__ out) {
    const int gi = gridDim.y - 1 - blockIdx.y, J = blockIdx.x;   // largest l first
    const int l = g.l[gi], K = l, line0 = g.line0[gi], nl = g.line0[gi + 1] - line0;
    const int N = a.N, ne = n_extra(l);
    const int c = J * FB + threadIdx.x, w = threadIdx.x >> 5;
    const double* T = a.T64 + (size_t)l * N * N + c;
    const double sw = sqrt_w(l, c);
    const int r_lo = max(ne, J * FB + w * 32), r_hi = (J + 1) * FB;
    for (int line = 0; line < nl; line += 2) {
        const bool two = line + 1 < nl;
        const double* x0 = in + (size_t)(line0 + line) * N;
        const double* x1 = two ? x0 + N : x0;
        double s0 = 0.0, s1 = 0.0;
        for (int r = 0; r < ne; ++r) {
            const double t = T[(size_t)r * N];
            s0 = fma(t, x0[r], s0);
            s1 = fma(t, x1[r], s1);
        }
        for (int r = r_lo; r < r_hi; ++r) {
            const double t = T[(size_t)r * N];
            s0 = fma(t, x0[r], s0);
            s1 = fma(t, x1[r], s1);
        }
        double f0 = 0.0, f1 = 0.0;
        for (int j = 0; j < a.levels; ++j) {
            const int i = J >> j;
            if ((i & 1) || i + 1 >= (a.nleaf >> j)) continue;
            const int len = FB << j;
            const double* qt = a.QT + a.qoff[j] + (c - i * len);
            const double* w0 = W + mpos(a, j, i, line0 + line, 0);
            const double* w1 = two ? w0 + KM : w0;
            for (int k = 0; k < K; ++k) {
                const double q = qt[(size_t)k * len];
                f0 = fma(q, w0[k], f0);
                f1 = fma(q, w1[k], f1);
            }
        }
        out[(size_t)(line0 + line) * N + c] = fma(sw, f0, s0);
        if (two) out[(size_t)(line0 + line + 1) * N + c] = fma(sw, f1, s1);
    }
}

// Build-time layouts: betaT[l][j][k][r] = beta[l][j][r][k] and the transposed
// diagonal leaf blocks nearT[l][J][c][t] = T_l[J B + t][J B + c].
__global__ void k_fast_transpose_beta(const double* __restrict__ beta, double* __restrict__ betaT, int N) {
    const size_t lj = blockIdx.y;
    const int r = blockIdx.x, k = threadIdx.x;
    betaT[(lj * KM + k) * N + r] = beta[(lj * N + r) * KM + k];
}

__global__ void k_fast_near(const double* __restrict__ T64, double* __restrict__ nearT, int N, int nleaf) {
    const int J = blockIdx.x, l = blockIdx.y, c = threadIdx.x;
    for (int t = 0; t < FB; ++t)
        nearT[(((size_t)l * nleaf + J) * FB + c) * FB + t] = T64[((size_t)l * N + J * FB + t) * N + J * FB + c];
}

}  // namespace

struct FastData {
    int nleaf = 0, levels = 0;
    double* Q = nullptr;
    double* QT = nullptr;
    size_t* qoff = nullptr;
    double* beta = nullptr;
    double* betaT = nullptr;
    double* nearT = nullptr;
};

void poly_basis(int len, std::vector<double>& Q) { basis(len, Q); }

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
    // orthonormal bases of the levels (host, one thread per level), both layouts
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
    std::vector<double> Qall(qtot), QTall(qtot);
    for (int j = 0; j < levels; ++j) {
        const int len = FB << j;
        for (int t = 0; t < len; ++t)
            for (int k = 0; k < KM; ++k) {
                Qall[qoff[j] + (size_t)t * KM + k] = Qh[j][(size_t)t * KM + k];
                QTall[qoff[j] + (size_t)k * len + t] = Qh[j][(size_t)t * KM + k];
            }
    }
    const size_t L = (size_t)p->l_max + 1;
    const size_t nbeta = L * levels * N * KM;
    bool ok = cudaMalloc((void**)&f->Q, qtot * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&f->QT, qtot * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&f->qoff, levels * sizeof(size_t)) == cudaSuccess &&
              cudaMalloc((void**)&f->beta, nbeta * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&f->betaT, nbeta * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&f->nearT, L * N * FB * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMemcpy(f->Q, Qall.data(), qtot * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(f->QT, QTall.data(), qtot * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(f->qoff, qoff.data(), levels * sizeof(size_t), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        set_error("DSBT_PLAN_FAST64: device allocation or copy failed");
        return DSBT_ERR_NOMEM;
    }
    k_fast_beta<<<dim3(N, levels, (unsigned)L), KM, 0, st>>>(p->T64, f->Q, f->qoff, f->beta, N, levels);
    k_fast_transpose_beta<<<dim3(N, (unsigned)(L * levels)), KM, 0, st>>>(f->beta, f->betaT, N);
    k_fast_near<<<dim3(f->nleaf, (unsigned)L), FB, 0, st>>>(p->T64, f->nearT, N, f->nleaf);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

void fast_free(dsbt_plan* p) {
    if (!p || !p->fast) return;
    cudaFree(p->fast->Q);
    cudaFree(p->fast->QT);
    cudaFree(p->fast->qoff);
    cudaFree(p->fast->beta);
    cudaFree(p->fast->betaT);
    cudaFree(p->fast->nearT);
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
    FastArgs a{f->Q, f->QT, f->qoff, f->beta, f->betaT, f->nearT, p->T64, p->N, f->nleaf, f->levels, g.total_lines};
    const int per_l = p->knl != nullptr;
    int pmax = 0, lmax = 0;
    for (int gi = 0; gi < g.ngroups; ++gi) {
        pmax = std::max(pmax, (g.line0[gi + 1] - g.line0[gi]) * g.l[gi]);
        lmax = std::max(lmax, g.l[gi]);
    }
    ProfScope ps(kKContract64, st);
    if (pmax > 0) {
        long long blocks = 0;
        for (int j = 0; j < f->levels; ++j) {
            const int per = PROJ_THREADS / std::min(32, 1 << j);
            blocks += (long long)(f->nleaf >> (j + 1)) * g.ngroups * ((pmax + per - 1) / per);
        }
        k_fast_project<<<(unsigned)blocks, PROJ_THREADS, 0, st>>>(a, g, dir, pmax, in, scratch);
    }
    if (dir > 0) {
        const int ncomp = (n_extra(lmax) + FB / 32 - 1) / (FB / 32);
        k_fast_eval<<<dim3(f->nleaf + ncomp, g.ngroups), FB, 0, st>>>(a, g, in, scratch, out, phase, per_l);
    } else {
        k_fast_leaf_out<<<dim3(f->nleaf, g.ngroups), FB, 0, st>>>(a, g, in, scratch, out);
    }
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

}  // namespace dsbt
