// batch.cu -- a batch of uneven transforms (different grids N_t and l_max_t)
// in one persistent tensor-core launch per direction, with shared factors.
//
// Shared factors.  The regular rows of T_l (Sec. 2.4, Eqs. (38)-(42)) depend on
// n, m and l only, not on the grid size: row n is built from P_l(., 2n-1).
// Only the completion rows n < n0_l (Sec. 2.5, Eq. (43)) depend on N through
// P_{2n-p}(N_l - m, 2N_l).  So one split-TF32 factor set built at
// (N_max, l_max) serves every N <= N_max: for N_t the forward uses rows 0..31
// (completion rows and the first regular rows) from a small per-N table and all
// other rows from the shared set; the inverse reads K block 0 (rows n < 32 of
// T) from the per-N table, transposed, and all other K blocks from the shared
// T^T.  Memory: 4 x 4 B x (l_max+1) N_max^2 for the shared set plus
// 4 x 4 B x (l_max+1) x 32 x N per distinct N.
//
// The batched contraction is the split-TF32 kernel of gemm_tf32x3.cu with a
// device-side list of (transform, l) groups: tiles of all transforms come from
// one dynamic queue, and the TMA producer chooses the factor source per tile.
// The batch owns its workspace and tensor maps, so a whole step can be captured
// into one CUDA graph (dsbt_batch_capture_kinetic).  An autotuner times the
// tile order (transform-major; l-major; l-major with row tiles interleaved
// across transforms so that tiles reading the same slab of the shared factors
// run together) and the column-tile width (128, 192, 256 lines) on the batch's
// own shapes at creation and keeps the fastest.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "plan.cuh"
#include "tc_ptx.cuh"

namespace dsbt {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BK = 32;
constexpr int BN_MAX = 256;
constexpr int BBOX = 64;
constexpr int STAGES = 2;
constexpr int KC = 4;
constexpr int EPI_WARPS = 8;
constexpr int QS = 4;
constexpr int A_BYTES = BM * BK * 4;
constexpr int B_BYTES = BN_MAX * BK * 4;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
constexpr int CROWS = 32;   // rows of the per-N tables (>= every completion-row count)

struct BGroup {
    int t, l, N, nl;   // transform, angular momentum, grid, real lines
    int bline0;        // first line of the group in the transform's planar buffers
    int ct, t0;        // column tiles, first tile
    int cidx;          // distinct-N index of the per-N tables
    long long uoff;    // complex-element offset of the group's first channel (caller layout)
};

struct BTrans {
    float* a_hi;       // forward B operand / inverse output (planar FP32 aliases a_hi)
    float* a_lo;
    float* b_hi;       // forward output / inverse B operand
    float* b_lo;
    float2* phase;     // [2][N]
    int N;
    int nlines;
};

struct __align__(64) BMaps {
    CUtensorMap m[4];
};

enum : int { kModeUserC64 = 0, kModeSplit = 1, kModePlanar = 2 };

struct KR {
    int a0, a1, b0, b1, up;
    __device__ __forceinline__ int count() const { return (a1 - a0) + (b1 - b0); }
    __device__ __forceinline__ int at(int i) const {
        if (up) return (i < a1 - a0) ? (a0 + i) : (b0 + i - (a1 - a0));
        const int nb = b1 - b0;
        return (i < nb) ? (b1 - 1 - i) : (a1 - 1 - (i - nb));
    }
};

__device__ __forceinline__ KR kranges(int dir, int rt, int nx, int KB, int walk_up) {
    KR k;
    const int r0 = rt * BM;
    k.up = (dir > 0) || walk_up;
    k.a0 = 0;
    k.b0 = k.b1 = 0;
    if (r0 < nx) { k.a1 = KB; return k; }
    if (dir > 0) { k.a1 = min(KB, (r0 + BM) / BK); return k; }
    k.a1 = (nx + BK - 1) / BK;
    k.b0 = max(k.a1, r0 / BK);
    k.b1 = KB;
    return k;
}

struct BTile {
    int g, rt, ct, nmma;
};

__device__ __forceinline__ BTile bdecode(const BGroup* __restrict__ gs, int ng, int dir, int bn_cap, int t,
                                        const int2* __restrict__ tl_list) {
    if (tl_list) {   // explicit tile list: (group, rt << 8 | column tile)
        const int2 e = tl_list[t];
        BTile tl;
        tl.g = e.x;
        tl.rt = e.y >> 8;
        tl.ct = e.y & 255;
        int left = gs[e.x].nl - tl.ct * bn_cap;
        if (left > bn_cap) left = bn_cap;
        tl.nmma = (left + 15) & ~15;
        return tl;
    }
    int lo = 0, hi = ng - 1;
    while (lo < hi) {   // last group with t0 <= t
        const int mid = (lo + hi + 1) >> 1;
        if (gs[mid].t0 <= t) lo = mid; else hi = mid - 1;
    }
    const BGroup& G = gs[lo];
    BTile tl;
    const int local = t - G.t0;
    const int q = local / G.ct;
    tl.g = lo;
    tl.ct = local - q * G.ct;
    const int RT = G.N / BM;
    tl.rt = (dir > 0) ? (q == 0 ? 0 : RT - q) : q;
    int left = G.nl - tl.ct * bn_cap;
    if (left > bn_cap) left = bn_cap;
    tl.nmma = (left + 15) & ~15;
    return tl;
}

__global__ void __launch_bounds__(NTHREADS, 1)
k_contract_batch(const __grid_constant__ CUtensorMap tF_hi, const __grid_constant__ CUtensorMap tF_lo,
                 const __grid_constant__ CUtensorMap tF96_hi, const __grid_constant__ CUtensorMap tF96_lo,
                 const __grid_constant__ CUtensorMap tI_hi, const __grid_constant__ CUtensorMap tI_lo,
                 const BGroup* __restrict__ groups, int ngroups, int total, const BTrans* __restrict__ trans,
                 const BMaps* __restrict__ tmaps, const BMaps* __restrict__ cmaps, int Nmax, int dir, int mode,
                 int bn_cap, float2* __restrict__ out_user, unsigned* status, int* sched,
                 const int2* __restrict__ tl_list, int walk_up) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* stage_base = smem;
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* main_full = empty + STAGES;
    uint64_t* main_empty = main_full + 1;
    uint64_t* tq_full = main_empty + 1;
    uint64_t* tq_empty = tq_full + QS;
    int* tile_q = (int*)(tq_empty + QS);
    uint32_t* tmem_slot = (uint32_t*)(tile_q + QS);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(main_full, 1);
        mbar_init(main_empty, EPI_WARPS);
        for (int q = 0; q < QS; ++q) {
            mbar_init(&tq_full[q], 1);
            mbar_init(&tq_empty[q], 1 + EPI_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer + tile scheduler
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int qslot = 0;
            uint32_t qphase = 0;
            while (ok) {
                if (!mbar_wait(&tq_empty[qslot], qphase ^ 1, abort_flag, status)) { ok = false; break; }
                int t = atomicAdd(sched, 1);
                if (t >= total) t = -1;
                tile_q[qslot] = t;
                mbar_arrive(&tq_full[qslot]);
                if (++qslot == QS) { qslot = 0; qphase ^= 1; }
                if (t < 0) break;
                const BTile tl = bdecode(groups, ngroups, dir, bn_cap, t, tl_list);
                const BGroup G = groups[tl.g];
                const KR kr = kranges(dir, tl.rt, n_extra(G.l), G.N / BK, walk_up);
                const int nbox = (tl.nmma + BBOX - 1) / BBOX;
                const uint32_t bytes = 2 * A_BYTES + 2 * nbox * BBOX * BK * 4;
                const int brow = G.bline0 + tl.ct * bn_cap;
                const CUtensorMap* mb_hi = &tmaps[G.t].m[dir > 0 ? 0 : 2];
                const CUtensorMap* mb_lo = &tmaps[G.t].m[dir > 0 ? 1 : 3];
                const int nkb = kr.count();
                for (int i = 0; i < nkb; ++i) {
                    const int kb = kr.at(i);
                    if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, status)) { ok = false; break; }
                    unsigned char* sb = stage_base + stage * STAGE_BYTES;
                    mbar_expect_tx(&full[stage], bytes);
                    if (dir > 0) {
                        if (tl.rt == 0) {   // rows 0..31 from the per-N table, 32..127 shared
                            tma_load_2d(sb, &cmaps[G.cidx].m[0], &full[stage], kb * BK, G.l * CROWS);
                            tma_load_2d(sb + A_BYTES, &cmaps[G.cidx].m[1], &full[stage], kb * BK, G.l * CROWS);
                            tma_load_2d(sb + CROWS * 128, &tF96_hi, &full[stage], kb * BK, G.l * Nmax + CROWS);
                            tma_load_2d(sb + A_BYTES + CROWS * 128, &tF96_lo, &full[stage], kb * BK,
                                        G.l * Nmax + CROWS);
                        } else {
                            tma_load_2d(sb, &tF_hi, &full[stage], kb * BK, G.l * Nmax + tl.rt * BM);
                            tma_load_2d(sb + A_BYTES, &tF_lo, &full[stage], kb * BK, G.l * Nmax + tl.rt * BM);
                        }
                    } else {
                        if (kb == 0) {      // K block 0 (rows n < 32 of T) from the per-N table
                            tma_load_2d(sb, &cmaps[G.cidx].m[2], &full[stage], 0, G.l * G.N + tl.rt * BM);
                            tma_load_2d(sb + A_BYTES, &cmaps[G.cidx].m[3], &full[stage], 0,
                                        G.l * G.N + tl.rt * BM);
                        } else {
                            tma_load_2d(sb, &tI_hi, &full[stage], kb * BK, G.l * Nmax + tl.rt * BM);
                            tma_load_2d(sb + A_BYTES, &tI_lo, &full[stage], kb * BK, G.l * Nmax + tl.rt * BM);
                        }
                    }
                    for (int b = 0; b < nbox; ++b) {
                        tma_load_2d(sb + 2 * A_BYTES + b * BBOX * 128, mb_hi, &full[stage], kb * BK, brow + b * BBOX);
                        tma_load_2d(sb + 2 * A_BYTES + B_BYTES + b * BBOX * 128, mb_lo, &full[stage], kb * BK,
                                    brow + b * BBOX);
                    }
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t mphase = 0;
            bool ok = true;
            const uint32_t d_main = tmem_base, d_corr = tmem_base + 256;
            int qslot = 0;
            uint32_t qphase = 0;
            while (ok) {
                if (!mbar_wait(&tq_full[qslot], qphase, abort_flag, status)) break;
                const int t = ((volatile int*)tile_q)[qslot];
                mbar_arrive(&tq_empty[qslot]);
                if (++qslot == QS) { qslot = 0; qphase ^= 1; }
                if (t < 0) break;
                const BTile tl = bdecode(groups, ngroups, dir, bn_cap, t, tl_list);
                const BGroup G = groups[tl.g];
                const KR kr = kranges(dir, tl.rt, n_extra(G.l), G.N / BK, walk_up);
                const uint32_t idesc = idesc_tf32(BM, tl.nmma);
                const int nkb = kr.count();
                uint32_t acc_corr = 0;
                for (int c0 = 0; c0 < nkb && ok; c0 += KC) {
                    if (!mbar_wait(main_empty, mphase ^ 1, abort_flag, status)) { ok = false; break; }
                    mphase ^= 1;
                    tc_fence_after();
                    uint32_t acc_main = 0;
                    const int c1 = min(nkb, c0 + KC);
                    for (int i = c0; i < c1; ++i) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, status)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(stage_base + stage * STAGE_BYTES);
                        const uint32_t sa_lo = sa + A_BYTES;
                        const uint32_t sb_hi = sa + 2 * A_BYTES;
                        const uint32_t sb_lo = sb_hi + B_BYTES;
#pragma unroll
                        for (int ks = 0; ks < BK / 8; ++ks) {
                            const uint32_t off = ks * 32;
                            const uint64_t dah = sdesc_sw128(sa + off), dal = sdesc_sw128(sa_lo + off);
                            const uint64_t dbh = sdesc_sw128(sb_hi + off), dbl = sdesc_sw128(sb_lo + off);
                            mma_tf32(d_main, dah, dbh, idesc, acc_main);
                            mma_tf32(d_corr, dah, dbl, idesc, acc_corr);
                            mma_tf32(d_corr, dal, dbh, idesc, 1);
                            acc_main = 1;
                            acc_corr = 1;
                        }
                        mma_commit(&empty[stage]);
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(main_full);
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int half = ew >> 2;
        uint32_t mphase = 0;
        int qslot = 0;
        uint32_t qphase = 0;
        while (true) {
            if (!mbar_wait(&tq_full[qslot], qphase, abort_flag, status)) break;
            const int t = ((volatile int*)tile_q)[qslot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&tq_empty[qslot]);
            if (++qslot == QS) { qslot = 0; qphase ^= 1; }
            if (t < 0) break;
            const BTile tl = bdecode(groups, ngroups, dir, bn_cap, t, tl_list);
            const BGroup G = groups[tl.g];
            const KR kr = kranges(dir, tl.rt, n_extra(G.l), G.N / BK, walk_up);
            const int nkb = kr.count();
            const int N = G.N;
            const int row = tl.rt * BM + quarter * 32 + lane;
            const int cbase = tl.ct * bn_cap + half * 128;
            const int ncols = min(min(128, tl.nmma - half * 128), G.nl - cbase);
            const int nch = (tl.nmma > half * 128) ? ((min(tl.nmma - half * 128, 128) + 31) >> 5) : 0;
            const uint32_t tl_addr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 128);
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0.f;
            bool ok = true;
            for (int c0 = 0; c0 < nkb; c0 += KC) {
                if (!mbar_wait(main_full, mphase, abort_flag, status)) { ok = false; break; }
                mphase ^= 1;
                tc_fence_after();
                const bool last = c0 + KC >= nkb;
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    if (ch < nch) {
                        float v[32];
                        tmem_ld32(tl_addr + ch * 32, v);
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[ch * 32 + j] += v[j];
                        if (last) {
                            tmem_ld32(tl_addr + 256 + ch * 32, v);
#pragma unroll
                            for (int j = 0; j < 32; ++j) acc[ch * 32 + j] += v[j];
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(main_empty);
            }
            if (!ok) break;
            if (ncols <= 0) continue;
            const BTrans T = trans[G.t];
            if (mode == kModeUserC64) {
                float2* o = out_user + G.uoff + (size_t)(cbase >> 1) * N;
#pragma unroll
                for (int j = 0; j < 128; j += 2)
                    if (j < ncols) o[(size_t)(j >> 1) * N + row] = make_float2(acc[j], acc[j + 1]);
            } else if (mode == kModePlanar) {
                float* o = T.a_hi + (size_t)(G.bline0 + cbase) * N;
#pragma unroll
                for (int j = 0; j < 128; ++j)
                    if (j < ncols) o[(size_t)j * N + row] = acc[j];
            } else {
                const float2 ph = T.phase[(size_t)(G.l & 1) * N + row];
                float* oh = T.b_hi + (size_t)(G.bline0 + cbase) * N;
                float* ol = T.b_lo + (size_t)(G.bline0 + cbase) * N;
#pragma unroll
                for (int j = 0; j < 128; j += 2) {
                    if (j < ncols) {
                        const float re = acc[j] * ph.x - acc[j + 1] * ph.y;
                        const float im = acc[j] * ph.y + acc[j + 1] * ph.x;
                        const float hr = round_tf32(re), hi = round_tf32(im);
                        const size_t o = (size_t)j * N + row;
                        oh[o] = hr;
                        ol[o] = round_tf32(re - hr);
                        oh[o + N] = hi;
                        ol[o + N] = round_tf32(im - hi);
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

// exp(-i k~^2 tau / 2) per transform (k~ of Eq. (65) with dk = pi / (N_t dr)).
__global__ void k_phase_batch(const BTrans* __restrict__ trans, double dr, double tau) {
    const BTrans T = trans[blockIdx.x];
    const double dk = M_PI / (T.N * dr);
    for (int i = threadIdx.x; i < 2 * T.N; i += blockDim.x) {
        const int par = i / T.N, k = i % T.N;
        int n = (par == 0) ? k + 1 : k;
        if (n == 0) n = T.N;
        const double kt = n * dk;
        double s, c;
        sincos(-0.5 * kt * kt * tau, &s, &c);
        T.phase[i] = make_float2((float)c, (float)s);
    }
}

// Per-N tables from FP64 rows r < 32: forward [l][32][N] and inverse [l][N][32].
__global__ void k_split_comp(const double* __restrict__ rows, float* __restrict__ fh, float* __restrict__ fl,
                             float* __restrict__ ih, float* __restrict__ il, int N, int L) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)L * CROWS * N) return;
    const int m = (int)(i % N);
    const int r = (int)((i / N) % CROWS);
    const int l = (int)(i / ((long long)N * CROWS));
    const double v = rows[i];
    const float h = round_tf32((float)v);
    const float lo = round_tf32((float)(v - (double)h));
    fh[i] = h;
    fl[i] = lo;
    const size_t o = ((size_t)l * N + m) * CROWS + r;
    ih[o] = h;
    il[o] = lo;
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace dsbt

struct dsbt_batch {
    int T = 0, L = 0, Nmax = 0;
    double dr = 0;
    dsbt_plan* shared = nullptr;
    CUtensorMap tF96_hi, tF96_lo;
    std::vector<int> N, lmax, counts_off, counts, nchan, nlines, cidx;
    std::vector<long long> uoff;          // complex-element offset of each transform
    long long total_elems = 0;            // complex elements of one batch input
    std::vector<int> dN;                  // distinct N
    std::vector<dsbt_plan*> tw;           // twiddle-only plans per distinct N
    float* comp = nullptr;                // per-N tables
    double* comp64 = nullptr;
    unsigned char* ws = nullptr;          // owned workspace
    size_t ws_bytes = 0;
    std::vector<dsbt::BTrans> trans_h;
    dsbt::BTrans* trans_d = nullptr;
    dsbt::BMaps* tmaps_d = nullptr;
    dsbt::BMaps* cmaps_d = nullptr;
    dsbt::BGroup* groups_d[3] = {nullptr, nullptr, nullptr};   // per tile order
    int2* tiles_d[2] = {nullptr, nullptr};                       // order 2: forward / inverse tile lists
    int ngroups = 0, total_tiles[3] = {0, 0, 0};   // tiles per order at the current width
    int* sched = nullptr;
    int order = 0, bn_cap = 256;          // autotuned
    float tune_ms[3][3] = {{0}};
    std::vector<dsbt::GroupTable> gtab;   // per transform, for the sine/cosine kernels
};

namespace dsbt {
namespace {

void batch_free(dsbt_batch* b) {
    if (!b) return;
    if (b->shared) plan_release(b->shared);
    for (auto* p : b->tw) plan_release(p);
    cudaFree(b->comp);
    cudaFree(b->comp64);
    cudaFree(b->ws);
    cudaFree(b->trans_d);
    cudaFree(b->tmaps_d);
    cudaFree(b->cmaps_d);
    cudaFree(b->groups_d[0]);
    cudaFree(b->groups_d[1]);
    cudaFree(b->groups_d[2]);
    cudaFree(b->tiles_d[0]);
    cudaFree(b->tiles_d[1]);
    cudaFree(b->sched);
    delete b;
}

const int kBnCaps[3] = {128, 192, 256};

// Group list in one of two orders; returns the tile count for bn_cap.
std::vector<BGroup> make_groups(const dsbt_batch* b, int order, int bn_cap, int* total) {
    struct Item { int t, l; double work; };
    std::vector<Item> items;
    for (int t = 0; t < b->T; ++t)
        for (int l = 0; l <= b->lmax[t]; ++l)
            if (b->counts[b->counts_off[t] + l] > 0)
                items.push_back({t, l, (double)b->counts[b->counts_off[t] + l] * b->N[t] * b->N[t]});
    if (order == 0) {   // transform-major: largest transform first, l descending inside
        std::vector<double> tw(b->T, 0.0);
        for (auto& it : items) tw[it.t] += it.work;
        std::stable_sort(items.begin(), items.end(), [&](const Item& x, const Item& y) {
            if (x.t != y.t) return tw[x.t] > tw[y.t] || (tw[x.t] == tw[y.t] && x.t < y.t);
            return x.l > y.l;
        });
    } else {            // l-major (orders 1, 2): all transforms' groups of the same l together
        std::stable_sort(items.begin(), items.end(), [&](const Item& x, const Item& y) {
            if (x.l != y.l) return x.l > y.l;
            return b->N[x.t] > b->N[y.t];
        });
    }
    std::vector<BGroup> gs;
    int t0 = 0;
    for (auto& it : items) {
        BGroup G;
        G.t = it.t;
        G.l = it.l;
        G.N = b->N[it.t];
        const int off = b->counts_off[it.t];
        int chan_before = 0;
        for (int l = 0; l < it.l; ++l) chan_before += b->counts[off + l];
        G.nl = 2 * b->counts[off + it.l];
        G.bline0 = 2 * chan_before;
        G.ct = (G.nl + bn_cap - 1) / bn_cap;
        G.t0 = t0;
        G.cidx = b->cidx[it.t];
        G.uoff = b->uoff[it.t] + (long long)chan_before * G.N;
        t0 += (G.N / BM) * G.ct;
        gs.push_back(G);
    }
    *total = t0;
    return gs;
}

// Order 2: within each l (descending), tiles by row tile across all transforms
// that have it (forward: longest K first, rt = RT-1 .. 1 then rt = 0;
// inverse: rt = 0 .. RT-1), so tiles reading the same slab of the shared T_l
// (or T_l^T) run at the same time.  Entries: (group, rt << 8 | column tile).
std::vector<int2> make_tile_list(const std::vector<BGroup>& gs, int dir) {
    std::vector<int2> out;
    size_t i = 0;
    while (i < gs.size()) {
        size_t j = i;
        int rtmax = 0;
        while (j < gs.size() && gs[j].l == gs[i].l) { rtmax = std::max(rtmax, gs[j].N / BM); ++j; }
        std::vector<int> rts;
        if (dir > 0) { for (int rt = rtmax - 1; rt >= 1; --rt) rts.push_back(rt); rts.push_back(0); }
        else for (int rt = 0; rt < rtmax; ++rt) rts.push_back(rt);
        for (int rt : rts)
            for (size_t g = i; g < j; ++g)
                if (rt < gs[g].N / BM)
                    for (int c = 0; c < gs[g].ct; ++c) out.push_back(make_int2((int)g, (rt << 8) | c));
        i = j;
    }
    return out;
}

int upload_groups(dsbt_batch* b, int order, int bn_cap, cudaStream_t st) {
    int total = 0;
    std::vector<BGroup> gs = make_groups(b, order, bn_cap, &total);
    b->ngroups = (int)gs.size();
    b->total_tiles[order] = total;
    if (!b->groups_d[order])
        DSBT_CUDA_TRY(cudaMalloc((void**)&b->groups_d[order], gs.size() * sizeof(BGroup)));
    DSBT_CUDA_TRY(cudaMemcpyAsync(b->groups_d[order], gs.data(), gs.size() * sizeof(BGroup),
                                  cudaMemcpyHostToDevice, st));
    if (order == 2) {
        for (const BGroup& g : gs)
            if (g.ct > 255) {   // the tile list packs the column tile into 8 bits
                set_error("group of %d lines too wide for the row-interleaved order", g.nl);
                return DSBT_ERR_UNSUPPORTED;
            }
        for (int d = 0; d < 2; ++d) {
            std::vector<int2> tl = make_tile_list(gs, d == 0 ? +1 : -1);
            if ((int)tl.size() != total) {
                set_error("tile list size mismatch");
                return DSBT_ERR_INVALID;
            }
            cudaFree(b->tiles_d[d]);
            b->tiles_d[d] = nullptr;
            DSBT_CUDA_TRY(cudaMalloc((void**)&b->tiles_d[d], tl.size() * sizeof(int2)));
            DSBT_CUDA_TRY(cudaMemcpyAsync(b->tiles_d[d], tl.data(), tl.size() * sizeof(int2),
                                          cudaMemcpyHostToDevice, st));
        }
    }
    DSBT_CUDA_TRY(cudaStreamSynchronize(st));
    return DSBT_OK;
}

int launch_contract(const dsbt_batch* b, int order, int bn_cap, int total, int dir, int mode, float2* out_user,
                    cudaStream_t st) {
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
    static bool attr = false;
    if (!attr) {
        DSBT_CUDA_TRY(cudaFuncSetAttribute(k_contract_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        attr = true;
    }
    int dev = 0, nsm = 0;
    DSBT_CUDA_TRY(cudaGetDevice(&dev));
    DSBT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = total < nsm ? total : nsm;
    if (grid == 0) return DSBT_OK;
    DSBT_CUDA_TRY(cudaMemsetAsync(b->sched, 0, sizeof(int), st));
    const dsbt_plan* s = b->shared;
    ProfScope ps(kKContractTF32, st);
    k_contract_batch<<<grid, NTHREADS, smem, st>>>(s->tm_T_hi, s->tm_T_lo, b->tF96_hi, b->tF96_lo, s->tm_Tt_hi,
                                                   s->tm_Tt_lo, b->groups_d[order], b->ngroups, total,
                                                   b->trans_d, b->tmaps_d, b->cmaps_d, b->Nmax, dir, mode, bn_cap,
                                                   out_user, s->status, b->sched,
                                                   order == 2 ? b->tiles_d[dir > 0 ? 0 : 1] : nullptr,
                                                   order == 2 ? 1 : 0);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int run_batch(const dsbt_batch* b, int kinetic, double tau, const float* in, float* out, cudaStream_t st) {
    int rc;
    if (kinetic) {
        ProfScope ps(kKPhase, st);
        k_phase_batch<<<b->T, 256, 0, st>>>(b->trans_d, b->dr, tau);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    for (int t = 0; t < b->T; ++t) {
        const dsbt_plan* tp = b->tw[b->cidx[t]];
        rc = dct_forward_f32(tp, b->gtab[t], true, in + 2 * b->uoff[t], b->trans_h[t].a_hi, b->trans_h[t].a_lo, st);
        if (rc) return rc;
    }
    const int total = b->total_tiles[b->order];
    if (!kinetic)
        return launch_contract(b, b->order, b->bn_cap, total, +1, kModeUserC64, (float2*)out, st);
    rc = launch_contract(b, b->order, b->bn_cap, total, +1, kModeSplit, nullptr, st);
    if (!rc) rc = launch_contract(b, b->order, b->bn_cap, total, -1, kModePlanar, nullptr, st);
    if (rc) return rc;
    for (int t = 0; t < b->T; ++t) {
        const dsbt_plan* tp = b->tw[b->cidx[t]];
        rc = dct_inverse_f32(tp, b->gtab[t], true, b->trans_h[t].a_hi, out + 2 * b->uoff[t], st);
        if (rc) return rc;
    }
    return DSBT_OK;
}

// Times the forward contraction for each (order, column-tile width) on the
// batch's own shapes (workspace contents do not affect the timing) and keeps
// the fastest.
int autotune(dsbt_batch* b, cudaStream_t st) {
    cudaEvent_t e0, e1;
    DSBT_CUDA_TRY(cudaEventCreate(&e0));
    DSBT_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int order = 0; order < 3; ++order) {
        for (int ci = 0; ci < 3; ++ci) {
            const int cap = kBnCaps[ci];
            int rc = upload_groups(b, order, cap, st);
            if (rc == DSBT_ERR_UNSUPPORTED && order == 2) {   // not offered for this batch
                b->tune_ms[order][ci] = -1.f;
                continue;
            }
            if (rc) return rc;
            const int total = b->total_tiles[order];
            rc = launch_contract(b, order, cap, total, +1, kModeSplit, nullptr, st);   // warm-up
            if (rc) return rc;
            DSBT_CUDA_TRY(cudaEventRecord(e0, st));
            rc = launch_contract(b, order, cap, total, +1, kModeSplit, nullptr, st);
            if (rc) return rc;
            DSBT_CUDA_TRY(cudaEventRecord(e1, st));
            DSBT_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            DSBT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            b->tune_ms[order][ci] = ms;
            if (ms < best) {
                best = ms;
                b->order = order;
                b->bn_cap = cap;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // final group tables for the chosen width (all orders kept consistent)
    for (int order = 0; order < 3; ++order) {
        int rc = upload_groups(b, order, b->bn_cap, st);
        if (rc && !(rc == DSBT_ERR_UNSUPPORTED && order == 2)) return rc;
    }
    return DSBT_OK;
}

}  // namespace
}  // namespace dsbt

using namespace dsbt;

extern "C" int dsbt_batch_create(int ntrans, const int* N, const int* l_max, const int* counts, double dr,
                                 int autotune_tiles, void* stream, dsbt_batch** out) {
    DSBT_CHECK_ARG(out != nullptr && N != nullptr && l_max != nullptr && counts != nullptr,
                   "dsbt_batch_create: NULL argument");
    *out = nullptr;
    DSBT_CHECK_ARG(ntrans >= 1 && ntrans <= 4096, "dsbt_batch_create: ntrans=%d out of range", ntrans);
    DSBT_CHECK_ARG(dr > 0.0 && isfinite(dr), "dsbt_batch_create: dr must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    dsbt_batch* b = new (std::nothrow) dsbt_batch();
    if (!b) return DSBT_ERR_NOMEM;
    b->T = ntrans;
    b->dr = dr;
    int off = 0;
    long long uoff = 0;
    for (int t = 0; t < ntrans; ++t) {
        if (!(N[t] >= 256 && N[t] <= 8192 && N[t] % 256 == 0) || !(l_max[t] >= 0 && l_max[t] <= 64)) {
            delete b;
            set_error("dsbt_batch_create: transform %d: N=%d, l_max=%d not supported", t, N[t], l_max[t]);
            return DSBT_ERR_INVALID;
        }
        b->N.push_back(N[t]);
        b->lmax.push_back(l_max[t]);
        b->counts_off.push_back(off);
        int nc = 0;
        for (int l = 0; l <= l_max[t]; ++l) {
            if (counts[off + l] < 0) {
                delete b;
                set_error("dsbt_batch_create: negative count");
                return DSBT_ERR_INVALID;
            }
            b->counts.push_back(counts[off + l]);
            nc += counts[off + l];
        }
        off += l_max[t] + 1;
        b->nchan.push_back(nc);
        b->nlines.push_back(2 * nc);
        b->uoff.push_back(uoff);
        uoff += (long long)nc * N[t];
        b->Nmax = std::max(b->Nmax, N[t]);
        b->L = std::max(b->L, l_max[t] + 1);
    }
    b->total_elems = uoff;
    // shared factors at (N_max, l_max)
    int rc = dsbt_plan_create(b->Nmax, b->Nmax * dr, b->L - 1, DSBT_PLAN_TF32X3, stream, &b->shared);
    if (rc) { batch_free(b); return rc; }
    rc = encode_tmap_f32_sw128(&b->tF96_hi, b->shared->Thi, (uint64_t)b->L * b->Nmax, b->Nmax, 96, 32);
    if (!rc) rc = encode_tmap_f32_sw128(&b->tF96_lo, b->shared->Tlo, (uint64_t)b->L * b->Nmax, b->Nmax, 96, 32);
    if (rc) { batch_free(b); return rc; }
    // distinct grids: twiddles and per-N tables
    for (int t = 0; t < ntrans; ++t) {
        auto it = std::find(b->dN.begin(), b->dN.end(), N[t]);
        if (it == b->dN.end()) {
            b->cidx.push_back((int)b->dN.size());
            b->dN.push_back(N[t]);
        } else {
            b->cidx.push_back((int)(it - b->dN.begin()));
        }
    }
    const int ND = (int)b->dN.size();
    size_t comp_elems = 0, comp64_max = 0;
    for (int d = 0; d < ND; ++d) {
        comp_elems += 4 * (size_t)b->L * CROWS * b->dN[d];
        comp64_max = std::max(comp64_max, (size_t)b->L * CROWS * b->dN[d]);
    }
    if (cudaMalloc((void**)&b->comp, comp_elems * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&b->comp64, comp64_max * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        set_error("dsbt_batch_create: device allocation failed (per-N tables)");
        return DSBT_ERR_NOMEM;
    }
    std::vector<BMaps> cm(ND);
    size_t coff = 0;
    for (int d = 0; d < ND; ++d) {
        const int Nd = b->dN[d];
        dsbt_plan* tp = nullptr;
        rc = plan_twiddles_only(Nd, Nd * dr, st, &tp);
        if (rc) { batch_free(b); return rc; }
        b->tw.push_back(tp);
        rc = build_first_rows(b->comp64, Nd, b->L - 1, CROWS, st);
        if (rc) { batch_free(b); return rc; }
        const size_t n1 = (size_t)b->L * CROWS * Nd;
        float *fh = b->comp + coff, *fl = fh + n1, *ih = fl + n1, *il = ih + n1;
        coff += 4 * n1;
        k_split_comp<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(b->comp64, fh, fl, ih, il, Nd, b->L);
        if (cudaGetLastError() != cudaSuccess) { batch_free(b); set_error("k_split_comp launch failed"); return DSBT_ERR_CUDA; }
        rc = encode_tmap_f32_sw128(&cm[d].m[0], fh, (uint64_t)b->L * CROWS, Nd, CROWS, 32);
        if (!rc) rc = encode_tmap_f32_sw128(&cm[d].m[1], fl, (uint64_t)b->L * CROWS, Nd, CROWS, 32);
        if (!rc) rc = encode_tmap_f32_sw128(&cm[d].m[2], ih, (uint64_t)b->L * Nd, CROWS, BM, 32);
        if (!rc) rc = encode_tmap_f32_sw128(&cm[d].m[3], il, (uint64_t)b->L * Nd, CROWS, BM, 32);
        if (rc) { batch_free(b); return rc; }
        if (cudaStreamSynchronize(st) != cudaSuccess) { batch_free(b); set_error("per-N table build failed"); return DSBT_ERR_CUDA; }
    }
    cudaFree(b->comp64);
    b->comp64 = nullptr;
    // owned workspace: per transform a_hi, a_lo, b_hi, b_lo [lines][N] + phase [2][N]
    size_t wbytes = 0;
    std::vector<size_t> woff(ntrans);
    for (int t = 0; t < ntrans; ++t) {
        woff[t] = wbytes;
        wbytes += 4 * a256((size_t)b->nlines[t] * N[t] * sizeof(float)) + a256(2 * (size_t)N[t] * sizeof(float2));
    }
    if (cudaMalloc((void**)&b->ws, wbytes + 256) != cudaSuccess || cudaMalloc((void**)&b->sched, 256) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        set_error("dsbt_batch_create: workspace allocation of %zu bytes failed", wbytes);
        return DSBT_ERR_NOMEM;
    }
    b->ws_bytes = wbytes;
    cudaMemsetAsync(b->ws, 0, wbytes, st);
    std::vector<BMaps> tm(ntrans);
    for (int t = 0; t < ntrans; ++t) {
        BTrans T;
        const size_t lb = a256((size_t)b->nlines[t] * N[t] * sizeof(float));
        unsigned char* p = b->ws + woff[t];
        T.a_hi = (float*)p;
        T.a_lo = (float*)(p + lb);
        T.b_hi = (float*)(p + 2 * lb);
        T.b_lo = (float*)(p + 3 * lb);
        T.phase = (float2*)(p + 4 * lb);
        T.N = N[t];
        T.nlines = b->nlines[t];
        b->trans_h.push_back(T);
        const uint64_t rows = (uint64_t)std::max(1, b->nlines[t]);
        rc = encode_tmap_f32_sw128(&tm[t].m[0], T.a_hi, rows, N[t], BBOX, 32);
        if (!rc) rc = encode_tmap_f32_sw128(&tm[t].m[1], T.a_lo, rows, N[t], BBOX, 32);
        if (!rc) rc = encode_tmap_f32_sw128(&tm[t].m[2], T.b_hi, rows, N[t], BBOX, 32);
        if (!rc) rc = encode_tmap_f32_sw128(&tm[t].m[3], T.b_lo, rows, N[t], BBOX, 32);
        if (rc) { batch_free(b); return rc; }
        // sine/cosine group table of this transform (channels l-major)
        GroupTable g;
        g.ngroups = 0;
        int chan = 0;
        for (int l = 0; l <= l_max[t]; ++l) {
            const int c = b->counts[b->counts_off[t] + l];
            if (!c) continue;
            g.l[g.ngroups] = l;
            g.chan0[g.ngroups] = chan;
            g.line0[g.ngroups] = 2 * chan;
            ++g.ngroups;
            chan += c;
        }
        g.chan0[g.ngroups] = chan;
        g.line0[g.ngroups] = 2 * chan;
        g.total_lines = 2 * chan;
        b->gtab.push_back(g);
    }
    bool ok = cudaMalloc((void**)&b->trans_d, ntrans * sizeof(BTrans)) == cudaSuccess &&
              cudaMalloc((void**)&b->tmaps_d, ntrans * sizeof(BMaps)) == cudaSuccess &&
              cudaMalloc((void**)&b->cmaps_d, ND * sizeof(BMaps)) == cudaSuccess;
    ok = ok && cudaMemcpy(b->trans_d, b->trans_h.data(), ntrans * sizeof(BTrans), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->tmaps_d, tm.data(), ntrans * sizeof(BMaps), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->cmaps_d, cm.data(), ND * sizeof(BMaps), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        set_error("dsbt_batch_create: table upload failed");
        return DSBT_ERR_CUDA;
    }
    for (int order = 0; order < 3; ++order) {
        rc = upload_groups(b, order, 256, st);
        if (rc == DSBT_ERR_UNSUPPORTED && order == 2) { rc = DSBT_OK; continue; }
        if (rc) { batch_free(b); return rc; }
    }
    if (autotune_tiles) {
        rc = autotune(b, st);
        if (rc) { batch_free(b); return rc; }
    }
    *out = b;
    return DSBT_OK;
}

extern "C" int dsbt_batch_destroy(dsbt_batch* b) {
    if (!b) return DSBT_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return DSBT_OK;
}

extern "C" int dsbt_batch_info(const dsbt_batch* b, long long* total_elems, int* order, int* bn_cap,
                               float* tune_ms) {
    DSBT_CHECK_ARG(b != nullptr, "dsbt_batch_info: NULL batch");
    if (total_elems) *total_elems = b->total_elems;
    if (order) *order = b->order;
    if (bn_cap) *bn_cap = b->bn_cap;
    if (tune_ms)
        for (int o = 0; o < 3; ++o)
            for (int c = 0; c < 3; ++c) tune_ms[o * 3 + c] = b->tune_ms[o][c];
    return DSBT_OK;
}

extern "C" int dsbt_batch_set_tiles(dsbt_batch* b, int order, int bn_cap, void* stream) {
    DSBT_CHECK_ARG(b != nullptr, "dsbt_batch_set_tiles: NULL batch");
    DSBT_CHECK_ARG(order >= 0 && order <= 2, "dsbt_batch_set_tiles: order %d not in 0..2", order);
    DSBT_CHECK_ARG(bn_cap == 128 || bn_cap == 192 || bn_cap == 256, "dsbt_batch_set_tiles: width %d", bn_cap);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = upload_groups(b, order, bn_cap, st);
    if (rc) return rc;
    for (int o = 0; o < 3; ++o) {   // keep every order's table at the new width
        if (o == order) continue;
        rc = upload_groups(b, o, bn_cap, st);
        if (rc && !(rc == DSBT_ERR_UNSUPPORTED && o == 2)) return rc;
    }
    b->order = order;
    b->bn_cap = bn_cap;
    return DSBT_OK;
}

extern "C" int dsbt_batch_forward(const dsbt_batch* b, const void* in, void* out, void* stream) {
    DSBT_CHECK_ARG(b != nullptr && in != nullptr && out != nullptr && in != out, "dsbt_batch_forward: bad argument");
    return run_batch(b, 0, 0.0, (const float*)in, (float*)out, (cudaStream_t)stream);
}

extern "C" int dsbt_batch_kinetic(const dsbt_batch* b, double tau, const void* in, void* out, void* stream) {
    DSBT_CHECK_ARG(b != nullptr && in != nullptr && out != nullptr && in != out, "dsbt_batch_kinetic: bad argument");
    DSBT_CHECK_ARG(isfinite(tau), "dsbt_batch_kinetic: tau must be finite");
    return run_batch(b, 1, tau, (const float*)in, (float*)out, (cudaStream_t)stream);
}

extern "C" int dsbt_batch_capture_kinetic(const dsbt_batch* b, double tau, const void* in, void* out,
                                          void** graph_exec) {
    DSBT_CHECK_ARG(b != nullptr && in != nullptr && out != nullptr && graph_exec != nullptr && in != out,
                   "dsbt_batch_capture_kinetic: bad argument");
    *graph_exec = nullptr;
    cudaStream_t cs;
    DSBT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    // one uncaptured run sets every kernel attribute before capture
    int rc = run_batch(b, 1, tau, (const float*)in, (float*)out, cs);
    if (!rc && cudaStreamSynchronize(cs) != cudaSuccess) rc = DSBT_ERR_CUDA;
    const int was = profile_set_enabled(0);
    cudaGraph_t g = nullptr;
    if (!rc && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = DSBT_ERR_CUDA;
    if (!rc) {
        rc = run_batch(b, 1, tau, (const float*)in, (float*)out, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (!rc && e != cudaSuccess) {
            set_error("graph capture failed: %s", cudaGetErrorString(e));
            rc = DSBT_ERR_CUDA;
        }
    }
    profile_set_enabled(was);
    cudaGraphExec_t ge = nullptr;
    if (!rc && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
        set_error("graph instantiation failed");
        rc = DSBT_ERR_CUDA;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    *graph_exec = (void*)ge;
    return DSBT_OK;
}

extern "C" int dsbt_graph_launch(void* graph_exec, void* stream) {
    DSBT_CHECK_ARG(graph_exec != nullptr, "dsbt_graph_launch: NULL graph");
    DSBT_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)graph_exec, (cudaStream_t)stream));
    return DSBT_OK;
}

extern "C" int dsbt_graph_destroy(void* graph_exec) {
    if (graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)graph_exec);
    return DSBT_OK;
}
